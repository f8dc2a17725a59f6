// C ABI of the learned reranker (see include/rotormap.h): Levenshtein labels,
// candidate features, the network's weights / training step / prediction /
// checkpoint, and mapping with pruning.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "rope_host.h"

using namespace rope;

struct rope_reranker {
  int device = 0;
  int32_t F = 0, H = 0;
  int64_t step = 0;
  MlpWeights w{};
  float* master = nullptr;  // [P] FP32 parameters: W1 [H,F], b1 [H], w2 [H], b2
  float* m1 = nullptr;      // [P] AdamW first moments
  float* m2 = nullptr;      // [P] AdamW second moments
  float* grad = nullptr;    // [P]
  float* loss = nullptr;    // [1]
  float* pre = nullptr;     // [cap, H] training scratch
  float* dy = nullptr;      // [cap]
  float* sq = nullptr;      // [cap]
  int64_t cap = 0;
  std::vector<void*> owned;
  int64_t P() const { return (int64_t)H * F + 2 * H + 1; }
};

namespace {

template <class T>
rope_status dalloc(rope_reranker* r, T** p, size_t n) {
  void* d = nullptr;
  cudaError_t e = cudaMalloc(&d, n * sizeof(T) + 16);
  if (e != cudaSuccess) return host_fail(ROPE_ERR_OOM, "cudaMalloc: %s", cudaGetErrorString(e));
  r->owned.push_back(d);
  *p = static_cast<T*>(d);
  return ROPE_OK;
}

rope_status reserve(rope_reranker* r, int64_t B) {
  if (B <= r->cap) return ROPE_OK;
  // free the old scratch (the stream order is kept by a device sync)
  cudaDeviceSynchronize();
  for (void** q : {(void**)&r->pre, (void**)&r->dy, (void**)&r->sq}) {
    if (*q) {
      for (auto it = r->owned.begin(); it != r->owned.end(); ++it)
        if (*it == *q) {
          r->owned.erase(it);
          break;
        }
      cudaFree(*q);
      *q = nullptr;
    }
  }
  int64_t cap = B < 4096 ? 4096 : B;
  rope_status st;
  if ((st = dalloc(r, &r->pre, (size_t)cap * r->H)) != ROPE_OK) return st;
  if ((st = dalloc(r, &r->dy, (size_t)cap)) != ROPE_OK) return st;
  if ((st = dalloc(r, &r->sq, (size_t)cap)) != ROPE_OK) return st;
  r->cap = cap;
  return ROPE_OK;
}

// host parameters -> FP32 master + BF16/FP32 working copies
rope_status upload_params(rope_reranker* r, const float* p) {
  const int64_t HF = (int64_t)r->H * r->F;
  std::vector<__nv_bfloat16> W1(HF), w2(r->H);
  for (int64_t i = 0; i < HF; ++i) W1[i] = __float2bfloat16_rn(p[i]);
  for (int j = 0; j < r->H; ++j) w2[j] = __float2bfloat16_rn(p[HF + r->H + j]);
  ROPE_HOST_CUDA(cudaMemcpy(r->master, p, r->P() * sizeof(float), cudaMemcpyHostToDevice));
  ROPE_HOST_CUDA(cudaMemcpy(r->w.W1, W1.data(), HF * sizeof(__nv_bfloat16), cudaMemcpyHostToDevice));
  ROPE_HOST_CUDA(cudaMemcpy(r->w.b1, p + HF, r->H * sizeof(float), cudaMemcpyHostToDevice));
  ROPE_HOST_CUDA(cudaMemcpy(r->w.w2, w2.data(), r->H * sizeof(__nv_bfloat16), cudaMemcpyHostToDevice));
  ROPE_HOST_CUDA(cudaMemcpy(r->w.b2, p + HF + 2 * r->H, sizeof(float), cudaMemcpyHostToDevice));
  return ROPE_OK;
}

// splitmix64 -> uniform in (-1, 1): seeded initial weights
double init_uniform(uint64_t& x) {
  uint64_t z = (x += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return ((double)(z >> 11) * (1.0 / 9007199254740992.0)) * 2.0 - 1.0;
}

}  // namespace

extern "C" rope_status rope_reranker_create(int32_t n_features, int32_t hidden, uint64_t seed, rope_reranker** out) {
  if (!out) return host_fail(ROPE_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (n_features < 1 || n_features > kMaxFeatures) return host_fail(ROPE_ERR_INVALID_ARG, "n_features outside [1,32]");
  if (hidden < 1 || hidden > 1024) return host_fail(ROPE_ERR_INVALID_ARG, "hidden outside [1,1024]");
  rope_reranker* r = new rope_reranker();
  ROPE_HOST_CUDA(cudaGetDevice(&r->device));
  r->F = n_features;
  r->H = hidden;
  r->w.F = n_features;
  r->w.H = hidden;
  const int64_t P = r->P();
  rope_status st;
  auto bail = [&](rope_status s) {
    rope_reranker_free(r);
    return s;
  };
  if ((st = dalloc(r, &r->master, P)) != ROPE_OK) return bail(st);
  if ((st = dalloc(r, &r->m1, P)) != ROPE_OK) return bail(st);
  if ((st = dalloc(r, &r->m2, P)) != ROPE_OK) return bail(st);
  if ((st = dalloc(r, &r->grad, P)) != ROPE_OK) return bail(st);
  if ((st = dalloc(r, &r->loss, 1)) != ROPE_OK) return bail(st);
  if ((st = dalloc(r, &r->w.W1, (size_t)hidden * n_features)) != ROPE_OK) return bail(st);
  if ((st = dalloc(r, &r->w.b1, hidden)) != ROPE_OK) return bail(st);
  if ((st = dalloc(r, &r->w.w2, hidden)) != ROPE_OK) return bail(st);
  if ((st = dalloc(r, &r->w.b2, 1)) != ROPE_OK) return bail(st);
  // Glorot-uniform weights, zero biases
  std::vector<float> p(P, 0.f);
  uint64_t x = seed;
  const double a1 = std::sqrt(6.0 / (n_features + hidden)), a2 = std::sqrt(6.0 / (hidden + 1));
  for (int64_t i = 0; i < (int64_t)hidden * n_features; ++i) p[i] = (float)(a1 * init_uniform(x));
  for (int j = 0; j < hidden; ++j) p[(int64_t)hidden * n_features + hidden + j] = (float)(a2 * init_uniform(x));
  if ((st = upload_params(r, p.data())) != ROPE_OK) return bail(st);
  if (cudaMemset(r->m1, 0, P * sizeof(float)) != cudaSuccess || cudaMemset(r->m2, 0, P * sizeof(float)) != cudaSuccess)
    return bail(host_fail(ROPE_ERR_CUDA, "cudaMemset"));
  *out = r;
  return ROPE_OK;
}

extern "C" void rope_reranker_free(rope_reranker* r) {
  if (!r) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(r->device);
  cudaDeviceSynchronize();
  for (void* q : r->owned) cudaFree(q);
  cudaSetDevice(prev);
  delete r;
}

extern "C" rope_status rope_reranker_get(const rope_reranker* r, float* params_host, int64_t* step) {
  if (!r || !params_host) return host_fail(ROPE_ERR_INVALID_ARG, "NULL argument");
  ROPE_HOST_CUDA(cudaDeviceSynchronize());
  ROPE_HOST_CUDA(cudaMemcpy(params_host, r->master, r->P() * sizeof(float), cudaMemcpyDeviceToHost));
  if (step) *step = r->step;
  return ROPE_OK;
}

extern "C" rope_status rope_reranker_set(rope_reranker* r, const float* params_host, int32_t reset_optimizer) {
  if (!r || !params_host) return host_fail(ROPE_ERR_INVALID_ARG, "NULL argument");
  ROPE_HOST_CUDA(cudaDeviceSynchronize());
  rope_status st = upload_params(r, params_host);
  if (st != ROPE_OK) return st;
  if (reset_optimizer) {
    ROPE_HOST_CUDA(cudaMemset(r->m1, 0, r->P() * sizeof(float)));
    ROPE_HOST_CUDA(cudaMemset(r->m2, 0, r->P() * sizeof(float)));
    r->step = 0;
  }
  return ROPE_OK;
}

extern "C" rope_status rope_reranker_grad(rope_reranker* r, const float* X, const float* t, const int64_t* sample_idx,
                                          int64_t B, float* grad, float* loss, cudaStream_t stream) {
  if (!r || !X || !t || !grad || B < 1) return host_fail(ROPE_ERR_INVALID_ARG, "bad gradient arguments");
  rope_status st = reserve(r, B);
  if (st != ROPE_OK) return st;
  ROPE_HOST_CUDA(launch_mlp_forward(r->w, X, sample_idx, B, nullptr, r->pre, t, r->dy, r->sq, stream));
  ROPE_HOST_CUDA(launch_mlp_backward(r->w, X, sample_idx, B, r->pre, r->dy, r->sq, grad, loss, 0, stream));
  return ROPE_OK;
}

extern "C" rope_status rope_reranker_train_step(rope_reranker* r, const float* X, const float* t,
                                                const int64_t* sample_idx, int64_t B, float lr, float weight_decay,
                                                float* loss_sum, cudaStream_t stream) {
  if (!r || !X || !t || B < 1) return host_fail(ROPE_ERR_INVALID_ARG, "bad training arguments");
  if (!(lr > 0.f) || weight_decay < 0.f) return host_fail(ROPE_ERR_INVALID_ARG, "lr must be > 0, weight_decay >= 0");
  rope_status st = reserve(r, B);
  if (st != ROPE_OK) return st;
  ROPE_HOST_CUDA(launch_mlp_forward(r->w, X, sample_idx, B, nullptr, r->pre, t, r->dy, r->sq, stream));
  ROPE_HOST_CUDA(launch_mlp_backward(r->w, X, sample_idx, B, r->pre, r->dy, r->sq, r->grad,
                                     loss_sum ? loss_sum : r->loss, loss_sum ? 1 : 0, stream));
  r->step += 1;
  ROPE_HOST_CUDA(launch_adamw(r->w, r->grad, r->master, r->m1, r->m2, r->step, lr, 0.9f, 0.999f, 1e-8f, weight_decay,
                              stream));
  return ROPE_OK;
}

extern "C" rope_status rope_reranker_predict(const rope_reranker* r, const float* X, int64_t B, float* y,
                                             cudaStream_t stream) {
  if (!r || !X || !y || B < 0) return host_fail(ROPE_ERR_INVALID_ARG, "bad prediction arguments");
  ROPE_HOST_CUDA(launch_mlp_forward(r->w, X, nullptr, B, y, nullptr, nullptr, nullptr, nullptr, stream));
  return ROPE_OK;
}

// Checkpoint: little-endian binary "ROPERR01", int32 F, int32 H, int64 step,
// then P floats each of the parameters, first and second moments.
extern "C" rope_status rope_reranker_save(const rope_reranker* r, const char* path) {
  if (!r || !path) return host_fail(ROPE_ERR_INVALID_ARG, "NULL argument");
  const int64_t P = r->P();
  std::vector<float> buf(3 * P);
  ROPE_HOST_CUDA(cudaDeviceSynchronize());
  ROPE_HOST_CUDA(cudaMemcpy(buf.data(), r->master, P * sizeof(float), cudaMemcpyDeviceToHost));
  ROPE_HOST_CUDA(cudaMemcpy(buf.data() + P, r->m1, P * sizeof(float), cudaMemcpyDeviceToHost));
  ROPE_HOST_CUDA(cudaMemcpy(buf.data() + 2 * P, r->m2, P * sizeof(float), cudaMemcpyDeviceToHost));
  FILE* f = fopen(path, "wb");
  if (!f) return host_fail(ROPE_ERR_INVALID_ARG, "cannot open %s for writing", path);
  const char magic[8] = {'R', 'O', 'P', 'E', 'R', 'R', '0', '1'};
  bool ok = fwrite(magic, 1, 8, f) == 8 && fwrite(&r->F, 4, 1, f) == 1 && fwrite(&r->H, 4, 1, f) == 1 &&
            fwrite(&r->step, 8, 1, f) == 1 && fwrite(buf.data(), sizeof(float), buf.size(), f) == buf.size();
  ok = (fclose(f) == 0) && ok;
  return ok ? ROPE_OK : host_fail(ROPE_ERR_INVALID_ARG, "write to %s failed", path);
}

extern "C" rope_status rope_reranker_load(rope_reranker* r, const char* path) {
  if (!r || !path) return host_fail(ROPE_ERR_INVALID_ARG, "NULL argument");
  FILE* f = fopen(path, "rb");
  if (!f) return host_fail(ROPE_ERR_INVALID_ARG, "cannot open %s", path);
  char magic[8];
  int32_t F = 0, H = 0;
  int64_t step = 0;
  bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, "ROPERR01", 8) == 0 && fread(&F, 4, 1, f) == 1 &&
            fread(&H, 4, 1, f) == 1 && fread(&step, 8, 1, f) == 1 && F == r->F && H == r->H;
  std::vector<float> buf;
  if (ok) {
    buf.resize(3 * r->P());
    ok = fread(buf.data(), sizeof(float), buf.size(), f) == buf.size();
  }
  fclose(f);
  if (!ok) return host_fail(ROPE_ERR_INVALID_ARG, "%s is not a checkpoint of a %dx%d reranker", path, r->F, r->H);
  ROPE_HOST_CUDA(cudaDeviceSynchronize());
  rope_status st = upload_params(r, buf.data());
  if (st != ROPE_OK) return st;
  const int64_t P = r->P();
  ROPE_HOST_CUDA(cudaMemcpy(r->m1, buf.data() + P, P * sizeof(float), cudaMemcpyHostToDevice));
  ROPE_HOST_CUDA(cudaMemcpy(r->m2, buf.data() + 2 * P, P * sizeof(float), cudaMemcpyHostToDevice));
  r->step = step;
  return ROPE_OK;
}

extern "C" rope_status rope_levenshtein(const rope_index* idx, const uint8_t* seqs, const int64_t* offsets,
                                        const int64_t* read_idx, const int64_t* win_start, int64_t n_pairs,
                                        int32_t* out_ld, float* out_frac, cudaStream_t stream) {
  if (!idx || n_pairs < 0) return host_fail(ROPE_ERR_INVALID_ARG, "bad arguments");
  if (n_pairs == 0) return ROPE_OK;
  if (!seqs || !offsets || !read_idx || !win_start || !out_ld) return host_fail(ROPE_ERR_INVALID_ARG, "NULL pointer");
  const DevIndex& ix = idx->ix;
  if (ix.N > 256) return host_fail(ROPE_ERR_UNSUPPORTED, "Levenshtein kernel built for N <= 256");
  ROPE_HOST_CUDA(launch_levenshtein(ix.packed, seqs, offsets, read_idx, win_start, n_pairs, ix.N, out_ld, stream));
  if (out_frac) ROPE_HOST_CUDA(launch_ld_fraction(out_ld, n_pairs, ix.N, out_frac, stream));
  return ROPE_OK;
}

extern "C" rope_status rope_rerank_features(const rope_index* idx, const uint8_t* seqs, const int64_t* offsets,
                                            const float* emb_f32, const float* norms, const int64_t* cand_win,
                                            const float* cand_score, int64_t n_reads, int32_t K, float* X,
                                            cudaStream_t stream) {
  if (!idx || n_reads < 0 || K < 1) return host_fail(ROPE_ERR_INVALID_ARG, "bad arguments");
  if (n_reads == 0) return ROPE_OK;
  const int F = K + 6 + idx->ix.m;
  if (F > kMaxFeatures) return host_fail(ROPE_ERR_INVALID_ARG, "K + 6 + m = %d > %d features", F, kMaxFeatures);
  if (!seqs || !offsets || !emb_f32 || !norms || !cand_win || !cand_score || !X)
    return host_fail(ROPE_ERR_INVALID_ARG, "NULL pointer");
  ROPE_HOST_CUDA(launch_features(idx->ix, seqs, offsets, emb_f32, norms, cand_win, cand_score, n_reads, K, F, X,
                                 stream));
  return ROPE_OK;
}

extern "C" rope_status rope_rerank_prune(const int64_t* cand_win, const float* cand_score, const float* pred,
                                         int64_t n_reads, int32_t K, int32_t keep, int64_t* out_win, float* out_score,
                                         float* out_pred, cudaStream_t stream) {
  if (n_reads < 0 || K < 1 || K > 64 || keep < 1 || keep > K) return host_fail(ROPE_ERR_INVALID_ARG, "bad arguments");
  if (n_reads == 0) return ROPE_OK;
  if (!cand_win || !cand_score || !pred || !out_win || !out_score) return host_fail(ROPE_ERR_INVALID_ARG, "NULL pointer");
  ROPE_HOST_CUDA(launch_prune(cand_win, cand_score, pred, n_reads, K, keep, out_win, out_score, out_pred, stream));
  return ROPE_OK;
}

extern "C" rope_status rope_map_rerank(const rope_index* idx, const uint8_t* seqs, const int64_t* offsets,
                                       int64_t n_reads, const rope_score_opts* opts, const rope_reranker* rr,
                                       int32_t keep, int64_t* out_win, float* out_score, float* out_pred,
                                       cudaStream_t stream) {
  if (!idx || !opts) return host_fail(ROPE_ERR_INVALID_ARG, "NULL argument");
  const int K = opts->k;
  if (keep < 1 || keep > K) return host_fail(ROPE_ERR_INVALID_ARG, "keep outside [1, k]");
  if (n_reads < 0) return host_fail(ROPE_ERR_INVALID_ARG, "n_reads < 0");
  if (n_reads == 0) return ROPE_OK;
  if (!seqs || !offsets || !out_win || !out_score) return host_fail(ROPE_ERR_INVALID_ARG, "NULL pointer");
  const int D = idx->ix.D, m = idx->ix.m;
  const int F = K + 6 + m;
  if (rr && rr->F != F) return host_fail(ROPE_ERR_INVALID_ARG, "reranker takes %d features, k=%d gives %d", rr->F, K, F);
  DeviceCtx* c;
  rope_status st = host_ctx(&c);
  if (st != ROPE_OK) return st;
  float *emb = nullptr, *norms = nullptr, *cs = nullptr, *X = nullptr, *pred = nullptr;
  uint16_t* embh = nullptr;
  int64_t* cw = nullptr;
  const size_t n = (size_t)n_reads;
  void** bufs[] = {(void**)&emb, (void**)&embh, (void**)&norms, (void**)&cw, (void**)&cs, (void**)&X, (void**)&pred};
  const size_t sizes[] = {n * 2 * D * 4, n * 2 * D * 2, n * (1 + m) * 4, n * K * 8, n * K * 4, n * K * F * 4, n * K * 4};
  int got = 0;
  for (; got < 7 && st == ROPE_OK; ++got) st = host_pool_alloc(c, bufs[got], sizes[got], stream);
  if (st == ROPE_OK) {
    cudaError_t e = launch_encode_reads(idx->enc, seqs, offsets, n_reads, emb, embh, norms, c->status, stream);
    if (e != cudaSuccess) st = host_fail(ROPE_ERR_CUDA, "encode launch: %s", cudaGetErrorString(e));
  }
  if (st == ROPE_OK) {
    rope_score_opts o = *opts;
    o.j_begin = o.j_end = 0;
    st = rope_score_topk(idx, emb, embh, norms, n_reads, &o, cw, cs, stream);
  }
  if (st == ROPE_OK && rr) {
    cudaError_t e = launch_features(idx->ix, seqs, offsets, emb, norms, cw, cs, n_reads, K, F, X, stream);
    if (e == cudaSuccess) e = launch_mlp_forward(rr->w, X, nullptr, n * K, pred, nullptr, nullptr, nullptr, nullptr, stream);
    if (e != cudaSuccess) st = host_fail(ROPE_ERR_CUDA, "rerank launch: %s", cudaGetErrorString(e));
  }
  if (st == ROPE_OK && !rr) {
    // fallback: the plain score ranking, i.e. a predicted distance increasing with rank
    cudaError_t e = launch_rank_as_prediction(n_reads, K, pred, stream);
    if (e != cudaSuccess) st = host_fail(ROPE_ERR_CUDA, "fallback launch: %s", cudaGetErrorString(e));
  }
  if (st == ROPE_OK) {
    cudaError_t e = launch_prune(cw, cs, pred, n_reads, K, keep, out_win, out_score, out_pred, stream);
    if (e != cudaSuccess) st = host_fail(ROPE_ERR_CUDA, "prune launch: %s", cudaGetErrorString(e));
  }
  for (int i = 0; i < got; ++i)
    if (*bufs[i]) cudaFreeAsync(*bufs[i], stream);
  return st;
}
