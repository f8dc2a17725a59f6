// C-ABI of the length ladder (variable-length reads; see rope_ladder.cu).
//
// A ladder is one index per window length N_j over one packed copy of the
// reference. rope_ladder_map buckets and sorts the reads on the device, reads
// the bucket sizes back (the one host synchronisation of the call), then runs
// each non-empty bucket (encode its read heads, scan, merge) on one of a few
// internal streams so that the tail of one bucket's scan overlaps the next
// bucket's work; the caller's stream waits for all of them.
//
// The per-bucket work of a call is captured once into a CUDA graph and
// replayed by later calls with the same bucket sizes, buffers and options:
// the first call of such a key runs eagerly (and tunes the scans' shape
// classes), the second captures and launches the graph, later ones launch it.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <set>
#include <vector>

#include "rope_host.h"

using namespace rope;

namespace {
constexpr int kLadderStreams = 4;
}

struct rope_ladder {
  int device = 0;
  rope_params p{};
  std::vector<int32_t> lens;
  std::vector<rope_index*> idx;  // idx[0] owns the packed reference
  int32_t* lens_dev = nullptr;
  int64_t* sizes_host = nullptr;  // pinned: base[nbk] then count[nbk]
  cudaStream_t streams[kLadderStreams] = {};
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[kLadderStreams] = {};
  cudaEvent_t done = nullptr;  // end of the last call, on its caller's stream
  bool done_recorded = false;
  // per-call scratch (bucketing, permutation, encodings), kept so that a
  // captured graph can refer to it; grown on demand
  uint8_t* scratch = nullptr;
  size_t scratch_bytes = 0;
  // candidate lists of the buckets run on each internal stream (graph path)
  Candidate* arena[kLadderStreams] = {};
  size_t arena_bytes[kLadderStreams] = {};
  std::map<std::vector<int64_t>, cudaGraphExec_t> graphs;
  std::set<std::vector<int64_t>> seen, no_graph;
};

namespace {

void drop_graphs(rope_ladder* lad) {
  for (auto& kv : lad->graphs) cudaGraphExecDestroy(kv.second);
  lad->graphs.clear();
  lad->seen.clear();
}

}  // namespace

extern "C" int32_t rope_ladder_lengths(int32_t n_min, int32_t n_max, int32_t steps_per_octave, int32_t* out_host,
                                       int32_t cap) {
  if (n_min < 1 || n_max < n_min || steps_per_octave < 1 || steps_per_octave > 64) return -1;
  int32_t n = 0, last = 0;
  for (int j = 0;; ++j) {
    const double v = std::floor((double)n_min * std::pow(2.0, (double)j / steps_per_octave));
    if (v > (double)n_max) break;
    const int32_t len = (int32_t)v;
    if (len == last) continue;
    if (out_host && n < cap) out_host[n] = len;
    ++n;
    last = len;
  }
  return n;
}

extern "C" void rope_ladder_free(rope_ladder* lad) {
  if (!lad) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(lad->device);
  cudaDeviceSynchronize();
  // buckets 1.. borrow bucket 0's packed reference: free them first
  for (size_t j = lad->idx.size(); j-- > 0;) rope_index_free(lad->idx[j]);
  if (lad->lens_dev) cudaFree(lad->lens_dev);
  if (lad->sizes_host) cudaFreeHost(lad->sizes_host);
  for (int i = 0; i < kLadderStreams; ++i) {
    if (lad->streams[i]) cudaStreamDestroy(lad->streams[i]);
    if (lad->join[i]) cudaEventDestroy(lad->join[i]);
  }
  if (lad->fork) cudaEventDestroy(lad->fork);
  if (lad->done) cudaEventDestroy(lad->done);
  drop_graphs(lad);
  if (lad->scratch) cudaFree(lad->scratch);
  for (int i = 0; i < kLadderStreams; ++i)
    if (lad->arena[i]) cudaFree(lad->arena[i]);
  cudaSetDevice(prev);
  delete lad;
}

extern "C" rope_status rope_ladder_create(const rope_params* p, const uint8_t* ref, int64_t len, int32_t n_min,
                                          int32_t n_max, int32_t steps_per_octave, rope_ladder** out,
                                          cudaStream_t stream) {
  if (!out) return host_fail(ROPE_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!p || !ref) return host_fail(ROPE_ERR_INVALID_ARG, "NULL pointer");
  if (n_min < p->s) return host_fail(ROPE_ERR_INVALID_ARG, "n_min=%d shorter than the s-mer (s=%d)", n_min, p->s);
  if (len < n_min) return host_fail(ROPE_ERR_INVALID_ARG, "reference shorter than n_min");
  const int64_t top = n_max < len ? n_max : len;
  const int32_t nbk = rope_ladder_lengths(n_min, (int32_t)top, steps_per_octave, nullptr, 0);
  if (nbk < 1) return host_fail(ROPE_ERR_INVALID_ARG, "bad ladder (n_min=%d n_max=%d steps=%d)", n_min, n_max,
                                steps_per_octave);
  if (nbk > kLadderMaxBuckets)
    return host_fail(ROPE_ERR_UNSUPPORTED, "ladder of %d lengths; at most %d", nbk, kLadderMaxBuckets);
  DeviceCtx* c;
  rope_status st = host_ctx(&c);
  if (st != ROPE_OK) return st;

  rope_ladder* lad = new rope_ladder();
  auto cleanup = [&](rope_status s) {
    rope_ladder_free(lad);
    return s;
  };
  cudaGetDevice(&lad->device);
  lad->p = *p;
  lad->lens.resize(nbk);
  rope_ladder_lengths(n_min, (int32_t)top, steps_per_octave, lad->lens.data(), nbk);
  for (int j = 0; j < nbk; ++j) {
    rope_params pj = *p;
    pj.window_len = lad->lens[j];
    rope_index* ij = nullptr;
    st = encode_reference_impl(&pj, ref, len, j == 0 ? nullptr : lad->idx[0]->ix.packed, &ij, stream);
    if (st != ROPE_OK) return cleanup(st);
    lad->idx.push_back(ij);
  }
  lad->p.bin_of_mer_host = nullptr;
  lad->p.window_len = lad->lens[0];
  cudaError_t e = cudaMalloc(&lad->lens_dev, sizeof(int32_t) * nbk);
  if (e == cudaSuccess)
    e = cudaMemcpy(lad->lens_dev, lad->lens.data(), sizeof(int32_t) * nbk, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMallocHost(&lad->sizes_host, sizeof(int64_t) * 2 * nbk);
  for (int i = 0; i < kLadderStreams && e == cudaSuccess; ++i) {
    e = cudaStreamCreateWithFlags(&lad->streams[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&lad->join[i], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&lad->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&lad->done, cudaEventDisableTiming);
  if (e != cudaSuccess) return cleanup(host_fail(ROPE_ERR_CUDA, "ladder set-up: %s", cudaGetErrorString(e)));
  *out = lad;
  return ROPE_OK;
}

extern "C" int32_t rope_ladder_graph_count(const rope_ladder* lad) {
  return lad ? (int32_t)lad->graphs.size() : 0;
}

extern "C" int32_t rope_ladder_size(const rope_ladder* lad) { return lad ? (int32_t)lad->lens.size() : 0; }

extern "C" const rope_index* rope_ladder_bucket(const rope_ladder* lad, int32_t j) {
  if (!lad || j < 0 || j >= (int32_t)lad->idx.size()) return nullptr;
  return lad->idx[j];
}

extern "C" rope_status rope_ladder_map(const rope_ladder* lad, const uint8_t* seqs, const int64_t* offsets,
                                       int64_t n_reads, const rope_score_opts* opts, int64_t* out_win,
                                       float* out_score, int32_t* out_len, cudaStream_t stream) {
  if (!lad || !opts) return host_fail(ROPE_ERR_INVALID_ARG, "NULL ladder or opts");
  if (n_reads < 0) return host_fail(ROPE_ERR_INVALID_ARG, "n_reads < 0");
  if (opts->k < 1 || opts->k > 32) return host_fail(ROPE_ERR_INVALID_ARG, "k=%d outside [1,32]", opts->k);
  if (opts->j_begin != 0 || opts->j_end != 0)
    return host_fail(ROPE_ERR_INVALID_ARG, "window ranges are per bucket; the ladder scans every window");
  if (n_reads == 0) return ROPE_OK;
  if (!seqs || !offsets || !out_win || !out_score) return host_fail(ROPE_ERR_INVALID_ARG, "NULL pointer");
  DeviceCtx* c;
  rope_status st = host_ctx(&c);
  if (st != ROPE_OK) return st;
  const int nbk = (int)lad->lens.size();
  const int D = lad->idx[0]->ix.D, m = lad->p.m;
  const bool bf16 = prec_tc(opts->precision);  // the tensor-core scans take the BF16 encoding
  const int slot = host_prof_begin(stream);

  rope_ladder* L = const_cast<rope_ladder*>(lad);  // buffers and graphs are cached in the ladder

  // scratch, one block kept in the ladder: bucket | hist | base,count | perm | emb_f32 | norms | emb_bf16
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  const size_t b_bucket = al(sizeof(int32_t) * n_reads);
  const size_t b_hist = al(sizeof(int64_t) * ladder_hist_entries(n_reads, nbk));
  const size_t b_sizes = al(sizeof(int64_t) * 2 * nbk);
  const size_t b_perm = al(sizeof(int64_t) * n_reads);
  const size_t b_f32 = al(sizeof(float) * 2 * D * n_reads);
  const size_t b_norm = al(sizeof(float) * (1 + m) * n_reads);
  const size_t b_bf16 = bf16 ? al(sizeof(uint16_t) * 2 * D * n_reads) : 0;
  const size_t need = b_bucket + b_hist + b_sizes + b_perm + b_f32 + b_norm + b_bf16;
  // the previous call (maybe on another stream) is done with the scratch
  if (L->done_recorded) cudaStreamWaitEvent(stream, L->done, 0);
  auto fail_prof = [&](rope_status s) {
    if (slot >= 0)
      for (int w = 1; w <= 3; ++w) host_prof_mark(slot, w, stream);
    return s;
  };
  cudaError_t e = cudaSuccess;
  if (need > L->scratch_bytes) {
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess)
      return fail_prof(host_fail(ROPE_ERR_CUDA, "ladder: %s", cudaGetErrorString(e)));
    drop_graphs(L);  // they refer to the old block
    if (L->scratch) cudaFree(L->scratch);
    L->scratch = nullptr;
    L->scratch_bytes = 0;
    if ((e = cudaMalloc(&L->scratch, need + need / 4)) != cudaSuccess) {
      cudaGetLastError();
      return fail_prof(host_fail(ROPE_ERR_OOM, "ladder scratch of %zu bytes: %s", need, cudaGetErrorString(e)));
    }
    L->scratch_bytes = need + need / 4;
  }
  uint8_t* scratch = L->scratch;
  int32_t* bucket = reinterpret_cast<int32_t*>(scratch);
  int64_t* hist = reinterpret_cast<int64_t*>(scratch + b_bucket);
  int64_t* sizes = reinterpret_cast<int64_t*>(scratch + b_bucket + b_hist);
  int64_t* perm = reinterpret_cast<int64_t*>(scratch + b_bucket + b_hist + b_sizes);
  float* emb_f32 = reinterpret_cast<float*>(scratch + b_bucket + b_hist + b_sizes + b_perm);
  float* norms = reinterpret_cast<float*>(scratch + b_bucket + b_hist + b_sizes + b_perm + b_f32);
  uint16_t* emb_bf16 =
      bf16 ? reinterpret_cast<uint16_t*>(scratch + b_bucket + b_hist + b_sizes + b_perm + b_f32 + b_norm) : nullptr;

  e = launch_fill_empty(out_win, out_score, n_reads * opts->k, stream);
  if (e == cudaSuccess)
    e = launch_ladder_sort(offsets, n_reads, lad->lens_dev, nbk, bucket, out_len, hist, sizes, sizes + nbk, perm,
                           stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(lad->sizes_host, sizes, sizeof(int64_t) * 2 * nbk, cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return fail_prof(host_fail(ROPE_ERR_CUDA, "ladder bucketing: %s", cudaGetErrorString(e)));
  host_prof_mark(slot, 1, stream);

  // the buckets' work: each non-empty bucket on an internal stream, round robin
  struct Work {
    int j;
    int64_t base, cnt;
    int si;
  };
  std::vector<Work> work;
  int next = 0;
  for (int j = 0; j < nbk; ++j) {
    const int64_t cnt = lad->sizes_host[nbk + j];
    if (cnt > 0) work.push_back(Work{j, lad->sizes_host[j], cnt, next++ % kLadderStreams});
  }
  // ROPE_GRAPH_LOG=1: report where a capture gets invalidated
  const bool log_graph = getenv("ROPE_GRAPH_LOG") != nullptr;
  auto capture_broken = [&](cudaStream_t s, const char* step, int j) {
    cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cst) != cudaSuccess || cst == cudaStreamCaptureStatusInvalidated) {
      fprintf(stderr, "rotormap ladder: capture invalidated after the %s of bucket %d\n", step, j);
      return true;
    }
    return false;
  };
  // Enqueues every bucket; with arenas, each scan's candidate lists go to its
  // stream's arena (no allocation, no tuning), as a captured graph needs.
  auto enqueue = [&](bool arenas, cudaStream_t origin) -> rope_status {
    cudaError_t ee;
    if ((ee = cudaEventRecord(lad->fork, origin)) != cudaSuccess)
      return host_fail(ROPE_ERR_CUDA, "ladder fork: %s", cudaGetErrorString(ee));
    bool used[kLadderStreams] = {};
    rope_status rs = ROPE_OK;
    for (const Work& w : work) {
      cudaStream_t s = lad->streams[w.si];
      if (!used[w.si]) {
        used[w.si] = true;
        if (s != origin && (ee = cudaStreamWaitEvent(s, lad->fork, 0)) != cudaSuccess) {
          rs = host_fail(ROPE_ERR_CUDA, "ladder fork: %s", cudaGetErrorString(ee));
          break;
        }
      }
      const rope_index* ij = lad->idx[w.j];
      float* f32 = emb_f32 + w.base * 2 * D;
      uint16_t* b16 = bf16 ? emb_bf16 + w.base * 2 * D : nullptr;
      float* nr = norms + w.base * (1 + m);
      ee = launch_encode_reads(ij->enc, seqs, offsets, w.cnt, f32, b16, nr, c->status, s, perm + w.base);
      if (ee != cudaSuccess) {
        rs = host_fail(ROPE_ERR_CUDA, "ladder encode: %s", cudaGetErrorString(ee));
        break;
      }
      ExtCandidates ext{L->arena[w.si], L->arena_bytes[w.si]};
      if (arenas && log_graph && capture_broken(s, "encode", w.j)) break;
      rs = score_topk_impl(ij, f32, b16, nr, w.cnt, opts, out_win, out_score, s, -1, perm + w.base,
                           arenas ? &ext : nullptr);
      if (rs != ROPE_OK) break;
      if (arenas && log_graph && capture_broken(s, "scan/merge", w.j)) break;
    }
    // join every stream that took work, even after an error
    for (int i = 0; i < kLadderStreams; ++i) {
      if (!used[i] || lad->streams[i] == origin) continue;
      cudaEventRecord(lad->join[i], lad->streams[i]);
      cudaStreamWaitEvent(origin, lad->join[i], 0);
    }
    return rs;
  };

  std::vector<int64_t> key = {n_reads, (int64_t)(uintptr_t)seqs, (int64_t)(uintptr_t)offsets,
                              (int64_t)(uintptr_t)out_win, (int64_t)(uintptr_t)out_score, opts->k, opts->sep,
                              opts->precision, opts->rescore, opts->cand_depth, opts->rescore_depth, opts->n_ranges};
  for (const Work& w : work) key.push_back(w.cnt);
  st = ROPE_OK;
  auto it = L->graphs.find(key);
  if (it != L->graphs.end()) {
    if ((e = cudaGraphLaunch(it->second, stream)) != cudaSuccess)
      st = host_fail(ROPE_ERR_CUDA, "ladder graph launch: %s", cudaGetErrorString(e));
  } else if (L->seen.count(key) && !L->no_graph.count(key)) {
    // second call with this key: size the arenas, capture, launch
    size_t want[kLadderStreams] = {};
    for (const Work& w : work) {
      size_t b = 0;
      if ((st = topk_cand_bytes(lad->idx[w.j], w.cnt, opts, &b)) != ROPE_OK) return fail_prof(st);
      want[w.si] = std::max(want[w.si], b);
    }
    for (int i = 0; i < kLadderStreams && st == ROPE_OK; ++i) {
      if (want[i] <= L->arena_bytes[i]) continue;
      cudaStreamSynchronize(stream);
      drop_graphs(L);
      L->seen.insert(key);
      if (L->arena[i]) cudaFree(L->arena[i]);
      L->arena[i] = nullptr;
      L->arena_bytes[i] = 0;
      if ((e = cudaMalloc(&L->arena[i], want[i])) != cudaSuccess) {
        cudaGetLastError();
        st = host_fail(ROPE_ERR_OOM, "ladder candidate arena of %zu bytes: %s", want[i], cudaGetErrorString(e));
        break;
      }
      L->arena_bytes[i] = want[i];
    }
    if (st != ROPE_OK) return fail_prof(st);
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    // captured from the ladder's first stream (the caller's stream may be the
    // legacy default stream, which cannot be captured); launched on the caller's
    cudaStream_t origin = lad->streams[0];
    e = cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal);
    rope_status cs = ROPE_OK;
    if (e == cudaSuccess) {
      cs = enqueue(true, origin);
      const cudaError_t ee = cudaStreamEndCapture(origin, &graph);
      if (e == cudaSuccess) e = ee;
    }
    if (e == cudaSuccess && cs == ROPE_OK) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e == cudaSuccess && cs == ROPE_OK && exec) {
      L->graphs[key] = exec;
      if ((e = cudaGraphLaunch(exec, stream)) != cudaSuccess)
        st = host_fail(ROPE_ERR_CUDA, "ladder graph launch: %s", cudaGetErrorString(e));
    } else {
      // capture refused: remember it and run the buckets eagerly
      if (getenv("ROPE_GRAPH_LOG"))
        fprintf(stderr, "rotormap ladder: no graph (capture: %s; enqueue: %s)\n", cudaGetErrorString(e),
                cs == ROPE_OK ? "ok" : rope_last_error());
      cudaGetLastError();
      if (exec) cudaGraphExecDestroy(exec);
      L->no_graph.insert(key);
      st = enqueue(false, stream);
    }
  } else {
    L->seen.insert(key);
    st = enqueue(false, stream);
  }
  if (st != ROPE_OK) return fail_prof(st);
  host_prof_mark(slot, 2, stream);
  cudaEventRecord(L->done, stream);
  L->done_recorded = true;
  host_prof_mark(slot, 3, stream);
  return ROPE_OK;
}
