// Threshold regime (§3.4 per-fragment cutting thresholds, §3.5 multi-locus
// output), first half: the threshold of each reference window for a target
// mutation rate, the mean fidelity between the window and n_s mutated copies
// of it.
//
// A copy is the first N letters of a walk from the window's start in which
// each reference letter is mutated with probability err: deleted, preceded
// by a random inserted letter, or substituted by one of the three other
// letters, each with probability 1/3 (past the reference end the walk reads
// A). The draws come from SplitMix64 (Steele, Lea and Flood, 2014): the
// stream of copy t of window j is keyed by output j*n_s + t of the
// generator started at `seed`, and reference letter d of the walk uses
// outputs 3d, 3d+1, 3d+2 of that stream (mutation?, kind, letter), compared
// in double precision, so the copies are fixed by (seed, j, t) alone.
//
// One thread per (window, copy): it walks and encodes its copy (FP32 direct
// sum in location order, its accumulator in shared memory); the first thread
// of each window's group also encodes the window; the group's fidelities are
// summed in copy order by a fixed shuffle tree.
#include <cuda_runtime.h>

#include "rope_internal.h"

namespace rope {

struct ThrArgs {
  EncTables tb;            // map [4^s], read-frame phases [m * n_loc]
  const uint32_t* packed;  // 2-bit packed reference
  int64_t L;
  int32_t stride, score_mode;
  int64_t j0, count;       // windows [j0, j0 + count)
  double err;
  uint64_t seed;
  int32_t n_samples;       // a power of two <= 32
  float* out;              // [count]
};

__device__ __forceinline__ uint32_t thr_letter(const uint32_t* __restrict__ packed, int64_t L, int64_t pos) {
  return pos < L ? (__ldg(packed + (pos >> 4)) >> ((pos & 15) * 2)) & 3u : 0u;
}

// adds letter c as the next letter of a string being encoded: the s-mer
// ending at it (first letter most significant) gets the phase of its location
__device__ __forceinline__ void thr_push(const EncTables& tb, uint32_t c, uint32_t& code, int& n, float2* acc) {
  const uint32_t mask = (1u << (2 * tb.s)) - 1u;
  code = ((code << 2) | c) & mask;
  ++n;
  if (n >= tb.s) {
    const int loc = n - tb.s;
    const int b = tb.map[code];
    const int n_loc = tb.N - tb.s + 1;
    for (int k = 0; k < tb.m; ++k) {
      const float2 ph = tb.phase[(size_t)k * n_loc + loc];
      acc[k * tb.nb + b].x += ph.x;
      acc[k * tb.nb + b].y += ph.y;
    }
  }
}

__device__ __forceinline__ double thr_fidelity(const float2* x, const float2* c, int off, int D) {
  double ipr = 0, ipi = 0, nx = 0, nc = 0;
  for (int i = off; i < off + D; ++i) {
    ipr += (double)x[i].x * c[i].x + (double)x[i].y * c[i].y;
    ipi += (double)x[i].x * c[i].y - (double)x[i].y * c[i].x;
    nx += (double)x[i].x * x[i].x + (double)x[i].y * x[i].y;
    nc += (double)c[i].x * c[i].x + (double)c[i].y * c[i].y;
  }
  if (nx <= (double)kZeroNorm2 || nc <= (double)kZeroNorm2) return 0.0;
  return (ipr * ipr + ipi * ipi) / (nx * nc);
}

__global__ void thresholds_kernel(ThrArgs a) {
  extern __shared__ __align__(16) float2 thr_smem[];
  const int D = a.tb.D, N = a.tb.N, ns = a.n_samples;
  const int t = threadIdx.x % ns;                 // copy number within the window's group
  const int g = threadIdx.x / ns;                 // group in the block
  const int groups = blockDim.x / ns;
  float2* acc = thr_smem + (size_t)threadIdx.x * D;              // this copy's encoding
  float2* win = thr_smem + (size_t)blockDim.x * D + (size_t)g * D;  // the window's encoding
  for (int64_t j_rel = (int64_t)blockIdx.x * groups + g; j_rel - g < a.count;
       j_rel += (int64_t)gridDim.x * groups) {
    const bool live = j_rel < a.count;
    const int64_t j = a.j0 + j_rel;
    const int64_t w = j * a.stride;
    for (int i = 0; i < D; ++i) acc[i] = make_float2(0.f, 0.f);
    if (t == 0)
      for (int i = 0; i < D; ++i) win[i] = make_float2(0.f, 0.f);
    if (live) {
      if (t == 0) {
        uint32_t code = 0;
        int n = 0;
        for (int i = 0; i < N; ++i) thr_push(a.tb, thr_letter(a.packed, a.L, w + i), code, n, win);
      }
      const uint64_t key = sm64_out(a.seed, (uint64_t)j * ns + t);
      uint32_t code = 0;
      int n = 0;
      for (int64_t d = 0; n < N; ++d) {
        uint32_t c = thr_letter(a.packed, a.L, w + d);
        if (sm64_unit(sm64_out(key, 3 * (uint64_t)d)) < a.err) {
          const int kind = (int)(sm64_unit(sm64_out(key, 3 * (uint64_t)d + 1)) * 3.0);
          const uint64_t z2 = sm64_out(key, 3 * (uint64_t)d + 2);
          if (kind == 0) continue;  // deletion
          if (kind == 1) {          // insertion before the letter
            thr_push(a.tb, (uint32_t)(z2 >> 62), code, n, acc);
            if (n < N) thr_push(a.tb, c, code, n, acc);
            continue;
          }
          c = (c + 1u + (uint32_t)(int)(sm64_unit(z2) * 3.0)) & 3u;  // substitution
        }
        thr_push(a.tb, c, code, n, acc);
      }
    }
    __syncthreads();
    double f = 0.0;
    if (live) {
      if (a.score_mode == 1) {
        for (int k = 0; k < a.tb.m; ++k) f += thr_fidelity(acc, win, k * a.tb.nb, a.tb.nb);
        f /= a.tb.m;
      } else {
        f = thr_fidelity(acc, win, 0, D);
      }
    }
    // sum over the group's copies in copy order (fixed tree)
    for (int o = 1; o < ns; o <<= 1) {
      const double other = __shfl_down_sync(0xffffffffu, f, o);
      if ((t & (2 * o - 1)) == 0) f += other;
    }
    if (live && t == 0) a.out[j_rel] = (float)(f / ns);
    __syncthreads();
  }
}

cudaError_t launch_thresholds(const ThrArgs& a, cudaStream_t st) {
  if (a.count <= 0) return cudaSuccess;
  const int threads = 128;
  const int groups = threads / a.n_samples;
  const size_t smem = ((size_t)threads + groups) * a.tb.D * sizeof(float2);
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  if (smem > (size_t)optin) return cudaErrorInvalidValue;
  e = cudaFuncSetAttribute(thresholds_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int64_t blocks = (a.count + groups - 1) / groups;
  if (blocks > 152 * 64) blocks = 152 * 64;
  thresholds_kernel<<<(unsigned)blocks, threads, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace rope

// ---------------------------------------------------------------- C ABI

#include "rope_host.h"

extern "C" rope_status rope_fragment_thresholds(const rope_index* idx, double err, int32_t n_samples, uint64_t seed,
                                                int64_t j_begin, int64_t count, float* out, cudaStream_t stream) {
  using namespace rope;
  if (!idx) return host_fail(ROPE_ERR_INVALID_ARG, "index is NULL");
  if (!(err >= 0.0 && err <= 1.0)) return host_fail(ROPE_ERR_INVALID_ARG, "err outside [0,1]");
  if (n_samples < 1 || n_samples > 32 || (n_samples & (n_samples - 1)))
    return host_fail(ROPE_ERR_INVALID_ARG, "n_samples=%d: a power of two in [1,32]", n_samples);
  if (j_begin < 0 || count < 0 || j_begin + count > idx->ix.W) return host_fail(ROPE_ERR_INVALID_ARG, "bad window range");
  if (count == 0) return ROPE_OK;
  if (!out) return host_fail(ROPE_ERR_INVALID_ARG, "NULL pointer");
  if (idx->dense) {
    // materialised index: the copies are walked, then encoded by the read
    // encoder, and compared with the windows' stored FP32 rows, a chunk of
    // windows at a time (scratch of about 2 GB at most)
    DeviceCtx* c;
    rope_status st = host_ctx(&c);
    if (st != ROPE_OK) return st;
    const DevIndex& ix = idx->ix;
    const int N = ix.N, D = ix.D, m = ix.m;
    const size_t per_copy = (size_t)N + 8 + (size_t)2 * D * sizeof(float) + (size_t)(1 + m) * sizeof(float);
    int64_t chunk = (int64_t)(((size_t)2 << 30) / (per_copy * n_samples));
    if (chunk < 1) chunk = 1;
    if (chunk > count) chunk = count;
    const int64_t n_copy = chunk * n_samples;
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t b_copy = al((size_t)n_copy * N), b_off = al((size_t)(n_copy + 1) * sizeof(int64_t));
    const size_t b_emb = al((size_t)n_copy * 2 * D * sizeof(float));
    const size_t b_norm = al((size_t)n_copy * (1 + m) * sizeof(float));
    uint8_t* scratch = nullptr;
    if ((st = host_pool_alloc(c, (void**)&scratch, b_copy + b_off + b_emb + b_norm, stream)) != ROPE_OK) return st;
    uint8_t* copies = scratch;
    int64_t* coff = reinterpret_cast<int64_t*>(scratch + b_copy);
    float* emb = reinterpret_cast<float*>(scratch + b_copy + b_off);
    float* norms = reinterpret_cast<float*>(scratch + b_copy + b_off + b_emb);
    cudaError_t e = launch_iota_offsets(coff, n_copy, N, stream);
    for (int64_t w0 = 0; w0 < count && e == cudaSuccess; w0 += chunk) {
      const int64_t cw = count - w0 < chunk ? count - w0 : chunk;
      MutArgs ma{};
      ma.packed = ix.packed;
      ma.L = ix.L;
      ma.j0 = j_begin + w0;
      ma.stride = ix.stride;
      ma.n_samples = n_samples;
      ma.err = err;
      ma.n = cw * n_samples;
      ma.N = N;
      ma.seed = seed;
      ma.out = copies;
      ma.status = c->status;
      e = launch_mutate(ma, stream);
      if (e == cudaSuccess)
        e = launch_encode_reads(idx->enc, copies, coff, cw * n_samples, emb, nullptr, norms, c->status, stream);
      if (e == cudaSuccess) e = launch_window_thresholds(ix, emb, norms, j_begin + w0, cw, n_samples, out + w0, stream);
    }
    cudaFreeAsync(scratch, stream);
    if (e != cudaSuccess) return host_fail(ROPE_ERR_CUDA, "thresholds launch: %s", cudaGetErrorString(e));
    return ROPE_OK;
  }
  if (idx->ix.D > 64) return host_fail(ROPE_ERR_UNSUPPORTED, "thresholds take complex dimension <= 64");
  ThrArgs a{};
  a.tb = idx->enc;
  a.packed = idx->ix.packed;
  a.L = idx->ix.L;
  a.stride = idx->ix.stride;
  a.score_mode = idx->ix.score_mode;
  a.j0 = j_begin;
  a.count = count;
  a.err = err;
  a.seed = seed;
  a.n_samples = n_samples;
  a.out = out;
  const cudaError_t e = launch_thresholds(a, stream);
  if (e != cudaSuccess) return host_fail(ROPE_ERR_CUDA, "thresholds launch: %s", cudaGetErrorString(e));
  return ROPE_OK;
}
