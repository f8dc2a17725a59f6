// Learned candidate reranker: exact Levenshtein labels, per-candidate
// features, a two-layer MLP (BF16 weights, FP32 arithmetic) with its forward,
// backward and AdamW kernels, and the pruning of each read's candidates to the
// ones with the smallest predicted edit distance.
//
// The paper has no reranker; it relates fidelity to Levenshtein distance (§1,
// §2.4 fitting curve) and thresholds fidelities per fragment (§3.3, §3.5).
// This network learns that relation from the scan's own score features.
#include <cuda_bf16.h>

#include "rope_internal.h"

namespace rope {

// ---------------------------------------------------------------- Levenshtein

// Global edit distance between the read head P (length N, letters from ASCII)
// and the reference window T (length N, from the 2-bit packed reference), by
// the bit-parallel recurrence of Myers (1999) in Hyyro's global form: bit i of
// Pv/Mv holds the vertical delta +1/-1 between rows i and i+1 of the DP
// column; for each text letter the column advances with one carry-propagating
// addition; the top row grows by one per column (global distance), so a 1 is
// shifted into the horizontal positive deltas. W 64-bit words hold N <= 64W.
template <int W>
__global__ void levenshtein_kernel(const uint32_t* __restrict__ packed, const uint8_t* __restrict__ seqs,
                                   const int64_t* __restrict__ offsets, const int64_t* __restrict__ read_idx,
                                   const int64_t* __restrict__ win_start, int64_t n_pairs, int N,
                                   int32_t* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_pairs; i += (int64_t)gridDim.x * blockDim.x) {
    const uint8_t* P = seqs + offsets[read_idx[i]];
    const int64_t w = win_start[i];
    uint64_t peq[4][W];
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int k = 0; k < W; ++k) peq[c][k] = 0;
    for (int p = 0; p < N; ++p) {
      const uint32_t c = letter_code(P[p]) & 3u;
#pragma unroll
      for (int k = 0; k < W; ++k)
        if (k == (p >> 6)) peq[c][k] |= 1ull << (p & 63);
    }
    uint64_t pv[W], mv[W];
#pragma unroll
    for (int k = 0; k < W; ++k) {
      pv[k] = ~0ull;
      mv[k] = 0;
    }
    const int top = N - 1 - 64 * (W - 1);  // bit of row N-1 in the last word
    int score = N;
    for (int j = 0; j < N; ++j) {
      const int64_t q = w + j;
      const uint32_t c = (packed[q >> 4] >> (2 * (q & 15))) & 3u;
      uint64_t carry = 0, hp_in = 1, hn_in = 0;
#pragma unroll
      for (int k = 0; k < W; ++k) {
        const uint64_t eq = peq[c][k];
        const uint64_t xv = eq | mv[k];
        const uint64_t a = eq & pv[k];
        const uint64_t s1 = a + pv[k];
        const uint64_t c1 = s1 < a;
        const uint64_t sum = s1 + carry;
        carry = c1 | (sum < s1);
        const uint64_t xh = (sum ^ pv[k]) | eq;
        uint64_t ph = mv[k] | ~(xh | pv[k]);
        uint64_t mh = pv[k] & xh;
        if (k == W - 1) {
          score += (int)((ph >> top) & 1ull) - (int)((mh >> top) & 1ull);
        }
        const uint64_t hp_out = ph >> 63, hn_out = mh >> 63;
        ph = (ph << 1) | hp_in;
        mh = (mh << 1) | hn_in;
        hp_in = hp_out;
        hn_in = hn_out;
        pv[k] = mh | ~(xv | ph);
        mv[k] = ph & xv;
      }
    }
    out[i] = score;
  }
}

cudaError_t launch_levenshtein(const uint32_t* packed, const uint8_t* seqs, const int64_t* offsets,
                               const int64_t* read_idx, const int64_t* win_start, int64_t n_pairs, int N, int32_t* out,
                               cudaStream_t st) {
  if (n_pairs <= 0) return cudaSuccess;
  const int threads = 128;
  int64_t blocks = (n_pairs + threads - 1) / threads;
  if (blocks > 152 * 64) blocks = 152 * 64;
  const int W = (N + 63) / 64;
  switch (W) {
    case 1: levenshtein_kernel<1><<<(unsigned)blocks, threads, 0, st>>>(packed, seqs, offsets, read_idx, win_start, n_pairs, N, out); break;
    case 2: levenshtein_kernel<2><<<(unsigned)blocks, threads, 0, st>>>(packed, seqs, offsets, read_idx, win_start, n_pairs, N, out); break;
    case 3: levenshtein_kernel<3><<<(unsigned)blocks, threads, 0, st>>>(packed, seqs, offsets, read_idx, win_start, n_pairs, N, out); break;
    case 4: levenshtein_kernel<4><<<(unsigned)blocks, threads, 0, st>>>(packed, seqs, offsets, read_idx, win_start, n_pairs, N, out); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------- features

// Per (read, candidate) feature row, F = K + 2 + m (<= kMaxFeatures):
//   [0, K)       the read's K candidate scores, best first (missing -> 0)
//   K            this candidate's fidelity
//   K+1 .. K+m   this candidate's per-band fidelities |<x_k|c_k>|^2/(X_k C_k)
//   K+m+1        rank / K
// One warp per read; each candidate window is summed directly in FP32
// (location order), as the re-scoring does. Missing candidates get a zero row.
// letter (0..3) at reference position p, or 4 outside [0, L)
__device__ __forceinline__ uint32_t ref_letter(const uint32_t* __restrict__ packed, int64_t L, int64_t p) {
  return (p >= 0 && p < L) ? (packed[p >> 4] >> ((p & 15) * 2)) & 3u : 4u;
}

__global__ void features_kernel(DevIndex ix, const uint8_t* __restrict__ seqs, const int64_t* __restrict__ offsets,
                                const float* __restrict__ emb_f32, const float* __restrict__ norms,
                                const int64_t* __restrict__ cand_win, const float* __restrict__ cand_score,
                                int64_t n_reads, int K, int F, float* __restrict__ X) {
  extern __shared__ float2 feat_acc[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int wpb = blockDim.x >> 5;
  float2* acc = feat_acc + (size_t)warp * ix.D;
  const int n_loc = ix.N - ix.s + 1;
  const int D = ix.D;
  for (int64_t r = (int64_t)blockIdx.x * wpb + warp; r < n_reads; r += (int64_t)gridDim.x * wpb) {
    const float* x = emb_f32 + (size_t)r * 2 * D;
    const float* nr = norms + (size_t)r * (1 + ix.m);
    for (int c = 0; c < K; ++c) {
      float* row = X + ((size_t)r * K + c) * F;
      const int64_t w0 = cand_win[r * K + c];
      if (w0 < 0) {
        for (int f = lane; f < F; f += 32) row[f] = 0.f;
        continue;
      }
      for (int g = lane; g < D; g += 32) acc[g] = make_float2(0.f, 0.f);
      __syncwarp();
      for (int loc0 = 0; loc0 < n_loc; loc0 += 32) {
        const int loc = loc0 + lane;
        const uint32_t b = loc < n_loc ? bin_at(ix.packed, w0 + loc, ix.s, ix.map_lsb) : 0u;
        const int cnt = min(32, n_loc - loc0);
        for (int jj = 0; jj < cnt; ++jj) {
          const uint32_t bj = __shfl_sync(0xffffffffu, b, jj);
          if (lane < ix.m) {
            const float2 ph = ix.phase[lane * n_loc + loc0 + jj];
            float2& v = acc[lane * ix.nb + bj];
            v.x += ph.x;
            v.y += ph.y;
          }
          __syncwarp();
        }
      }
      for (int k = 0; k < ix.m; ++k) {
        float re = 0.f, im = 0.f, C = 0.f;
        for (int b = lane; b < ix.nb; b += 32) {
          const int g = k * ix.nb + b;
          const float xr = x[g], xi = x[D + g];
          const float2 cc = acc[g];
          re = fmaf(xr, cc.x, fmaf(xi, cc.y, re));
          im = fmaf(xr, cc.y, fmaf(-xi, cc.x, im));
          C = fmaf(cc.x, cc.x, fmaf(cc.y, cc.y, C));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          re += __shfl_xor_sync(0xffffffffu, re, o);
          im += __shfl_xor_sync(0xffffffffu, im, o);
          C += __shfl_xor_sync(0xffffffffu, C, o);
        }
        const float Xk = nr[1 + k];
        if (lane == 0) row[K + 1 + k] = (Xk > kZeroNorm2 && C > kZeroNorm2) ? fmaf(re, re, im * im) / (Xk * C) : 0.f;
      }
      for (int f = lane; f < K; f += 32) {
        const float sc = cand_score[r * K + f];
        row[f] = cand_win[r * K + f] >= 0 ? sc : 0.f;
      }
      // Hamming fingerprint fidelities ((n - d) / n)^2 (§1) of the read head
      // against the window and the windows shifted by up to kShift letters
      // (letters outside the reference count as mismatches), and of the two
      // halves of the head at no shift
      {
        const uint8_t* head = seqs + offsets[r];
        const int N = ix.N, n1 = N / 2;
        int mm[2 * kShift + 1], mm1 = 0;
#pragma unroll
        for (int d = 0; d <= 2 * kShift; ++d) mm[d] = 0;
        for (int i = lane; i < N; i += 32) {
          const uint32_t q = letter_code(head[i]);
#pragma unroll
          for (int d = 0; d <= 2 * kShift; ++d) mm[d] += q != ref_letter(ix.packed, ix.L, w0 + i + d - kShift);
          if (i < n1) mm1 += q != ref_letter(ix.packed, ix.L, w0 + i);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
          for (int d = 0; d <= 2 * kShift; ++d) mm[d] += __shfl_xor_sync(0xffffffffu, mm[d], o);
          mm1 += __shfl_xor_sync(0xffffffffu, mm1, o);
        }
        if (lane == 0) {
          auto hf = [](int n, int d) {
            const float v = (float)(n - d) / (float)n;
            return v * v;
          };
          float best = 0.f;
#pragma unroll
          for (int d = 0; d <= 2 * kShift; ++d) best = fmaxf(best, hf(N, mm[d]));
          row[K] = cand_score[r * K + c];
          row[K + 1 + ix.m] = (float)c / (float)K;
          row[K + 2 + ix.m] = hf(N, mm[kShift]);
          row[K + 3 + ix.m] = best;
          row[K + 4 + ix.m] = hf(n1, mm1);
          row[K + 5 + ix.m] = hf(N - n1, mm[kShift] - mm1);
        }
      }
      for (int f = K + 6 + ix.m + lane; f < F; f += 32) row[f] = 0.f;
      __syncwarp();
    }
  }
}

cudaError_t launch_features(const DevIndex& ix, const uint8_t* seqs, const int64_t* offsets, const float* emb_f32,
                            const float* norms, const int64_t* cand_win, const float* cand_score, int64_t n_reads,
                            int K, int F, float* X, cudaStream_t st) {
  if (n_reads <= 0) return cudaSuccess;
  const int wpb = 8;
  int64_t blocks = (n_reads + wpb - 1) / wpb;
  if (blocks > 152 * 32) blocks = 152 * 32;
  features_kernel<<<(unsigned)blocks, wpb * 32, (size_t)wpb * ix.D * sizeof(float2), st>>>(
      ix, seqs, offsets, emb_f32, norms, cand_win, cand_score, n_reads, K, F, X);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- MLP

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.3989422804014327f * expf(-0.5f * z * z);
}

// Forward: one thread per sample; BF16 weights staged in shared memory as FP32.
// pre[s][j] is stored when `pre` is non-null (training), and with targets the
// per-sample residual gradient dy = 2 (y - t) / B and squared error.
// Sample s of the batch is row idx[s] of X and t (row s when idx is null).
__global__ void mlp_forward_kernel(MlpWeights w, const float* __restrict__ X, const int64_t* __restrict__ idx,
                                   int64_t B, float* __restrict__ y, float* __restrict__ pre,
                                   const float* __restrict__ t, float* __restrict__ dy, float* __restrict__ sq) {
  extern __shared__ float mlp_smem[];
  float* W1 = mlp_smem;                  // H x F
  float* b1 = W1 + w.H * w.F;            // H
  float* w2 = b1 + w.H;                  // H
  for (int i = threadIdx.x; i < w.H * w.F; i += blockDim.x) W1[i] = __bfloat162float(w.W1[i]);
  for (int i = threadIdx.x; i < w.H; i += blockDim.x) {
    b1[i] = w.b1[i];
    w2[i] = __bfloat162float(w.w2[i]);
  }
  __syncthreads();
  const float b2 = w.b2[0];
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < B; s += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = idx ? idx[s] : s;
    float xs[kMaxFeatures];
#pragma unroll
    for (int f = 0; f < kMaxFeatures; ++f) xs[f] = f < w.F ? X[row * w.F + f] : 0.f;
    float acc = b2;
    for (int j = 0; j < w.H; ++j) {
      float z = b1[j];
#pragma unroll
      for (int f = 0; f < kMaxFeatures; ++f)
        if (f < w.F) z = fmaf(W1[j * w.F + f], xs[f], z);
      if (pre) pre[s * w.H + j] = z;
      acc = fmaf(w2[j], gelu_f(z), acc);
    }
    if (y) y[s] = acc;
    if (t) {
      const float r = acc - t[row];
      dy[s] = 2.0f * r / (float)B;
      sq[s] = r * r;
    }
  }
}

// Backward: one block per hidden unit j; its threads split the samples and the
// block reduces in a fixed order (deterministic):
//   dW1[j][f] = sum_s dy_s w2_j GELU'(pre_sj) x_sf,  db1[j] = sum_s dy_s w2_j GELU'(pre_sj)
//   dw2[j]    = sum_s dy_s GELU(pre_sj);  block H also forms db2 = sum_s dy_s and the loss.
// `loss` receives the batch mean squared error, or has it added when
// accumulate != 0.
__global__ void mlp_backward_kernel(MlpWeights w, const float* __restrict__ X, const int64_t* __restrict__ idx,
                                    int64_t B, const float* __restrict__ pre, const float* __restrict__ dy,
                                    const float* __restrict__ sq, float* __restrict__ grad, float* __restrict__ loss,
                                    int accumulate) {
  constexpr int kT = 256;
  __shared__ float red[kT];
  const int j = blockIdx.x;
  const int tid = threadIdx.x;
  if (j < w.H) {
    const float w2j = __bfloat162float(w.w2[j]);
    float gW[kMaxFeatures];
#pragma unroll
    for (int f = 0; f < kMaxFeatures; ++f) gW[f] = 0.f;
    float gb1 = 0.f, gw2 = 0.f;
    for (int64_t s = tid; s < B; s += kT) {
      const float z = pre[s * w.H + j];
      const float d = dy[s];
      const float dz = d * w2j * gelu_grad_f(z);
      const int64_t row = idx ? idx[s] : s;
      gb1 += dz;
      gw2 = fmaf(d, gelu_f(z), gw2);
#pragma unroll
      for (int f = 0; f < kMaxFeatures; ++f)
        if (f < w.F) gW[f] = fmaf(dz, X[row * w.F + f], gW[f]);
    }
    // fixed-order tree reductions: F entries of W1's row, then b1, then w2
    for (int f = 0; f < w.F + 2; ++f) {
      float v = f == w.F ? gb1 : gw2;
      if (f < w.F) {
#pragma unroll
        for (int ff = 0; ff < kMaxFeatures; ++ff)
          if (ff == f) v = gW[ff];
      }
      red[tid] = v;
      __syncthreads();
      for (int o = kT / 2; o > 0; o >>= 1) {
        if (tid < o) red[tid] += red[tid + o];
        __syncthreads();
      }
      if (tid == 0) {
        if (f < w.F) grad[j * w.F + f] = red[0];
        else if (f == w.F) grad[w.H * w.F + j] = red[0];
        else grad[w.H * w.F + w.H + j] = red[0];
      }
      __syncthreads();
    }
  } else {
    // last block: db2 and the mean squared error
    for (int pass = 0; pass < 2; ++pass) {
      float v = 0.f;
      for (int64_t s = tid; s < B; s += kT) v += pass == 0 ? dy[s] : sq[s];
      red[tid] = v;
      __syncthreads();
      for (int o = kT / 2; o > 0; o >>= 1) {
        if (tid < o) red[tid] += red[tid + o];
        __syncthreads();
      }
      if (tid == 0) {
        if (pass == 0) grad[w.H * w.F + 2 * w.H] = red[0];
        else if (loss) loss[0] = (accumulate ? loss[0] : 0.f) + red[0] / (float)B;
      }
      __syncthreads();
    }
  }
}

// AdamW on the FP32 master parameters (flat: W1, b1, w2, b2), then the BF16
// copies of W1 and w2 the forward reads.
__global__ void adamw_kernel(MlpWeights w, const float* __restrict__ grad, float* __restrict__ master,
                             float* __restrict__ m1, float* __restrict__ m2, int64_t step, float lr, float beta1,
                             float beta2, float eps, float wd) {
  const int P = w.H * w.F + 2 * w.H + 1;
  const float c1 = 1.0f - powf(beta1, (float)step), c2 = 1.0f - powf(beta2, (float)step);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P; i += gridDim.x * blockDim.x) {
    const float g = grad[i];
    const float a = beta1 * m1[i] + (1.0f - beta1) * g;
    const float b = beta2 * m2[i] + (1.0f - beta2) * g * g;
    m1[i] = a;
    m2[i] = b;
    const float p = master[i] * (1.0f - lr * wd) - lr * (a / c1) / (sqrtf(b / c2) + eps);
    master[i] = p;
    if (i < w.H * w.F) w.W1[i] = __float2bfloat16_rn(p);
    else if (i < w.H * w.F + w.H) w.b1[i - w.H * w.F] = p;
    else if (i < w.H * w.F + 2 * w.H) w.w2[i - w.H * w.F - w.H] = __float2bfloat16_rn(p);
    else w.b2[0] = p;
  }
}

cudaError_t launch_mlp_forward(const MlpWeights& w, const float* X, const int64_t* idx, int64_t B, float* y, float* pre,
                               const float* t, float* dy, float* sq, cudaStream_t st) {
  if (B <= 0) return cudaSuccess;
  const int threads = 128;
  int64_t blocks = (B + threads - 1) / threads;
  if (blocks > 152 * 16) blocks = 152 * 16;
  const size_t smem = (size_t)(w.H * w.F + 2 * w.H) * sizeof(float);
  mlp_forward_kernel<<<(unsigned)blocks, threads, smem, st>>>(w, X, idx, B, y, pre, t, dy, sq);
  return cudaGetLastError();
}

cudaError_t launch_mlp_backward(const MlpWeights& w, const float* X, const int64_t* idx, int64_t B, const float* pre,
                                const float* dy, const float* sq, float* grad, float* loss, int accumulate,
                                cudaStream_t st) {
  mlp_backward_kernel<<<w.H + 1, 256, 0, st>>>(w, X, idx, B, pre, dy, sq, grad, loss, accumulate);
  return cudaGetLastError();
}

cudaError_t launch_adamw(const MlpWeights& w, const float* grad, float* master, float* m1, float* m2, int64_t step,
                         float lr, float beta1, float beta2, float eps, float wd, cudaStream_t st) {
  const int P = w.H * w.F + 2 * w.H + 1;
  adamw_kernel<<<(P + 255) / 256, 256, 0, st>>>(w, grad, master, m1, m2, step, lr, beta1, beta2, eps, wd);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- pruning

// Per read, keep the `keep` candidates with the smallest predicted distance
// (ties: better scan score, then lower start). Missing candidates are skipped.
__global__ void prune_kernel(const int64_t* __restrict__ cand_win, const float* __restrict__ cand_score,
                             const float* __restrict__ pred, int64_t n_reads, int K, int keep,
                             int64_t* __restrict__ out_win, float* __restrict__ out_score,
                             float* __restrict__ out_pred) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n_reads; r += (int64_t)gridDim.x * blockDim.x) {
    uint64_t taken = 0;
    for (int q = 0; q < keep; ++q) {
      int best = -1;
      for (int c = 0; c < K; ++c) {
        if ((taken >> c) & 1ull) continue;
        const int64_t wc = cand_win[r * K + c];
        if (wc < 0) continue;
        if (best < 0) {
          best = c;
          continue;
        }
        const float pc = pred[r * K + c], pb = pred[r * K + best];
        const float sc = cand_score[r * K + c], sb = cand_score[r * K + best];
        if (pc < pb || (pc == pb && (sc > sb || (sc == sb && wc < cand_win[r * K + best])))) best = c;
      }
      if (best >= 0) {
        taken |= 1ull << best;
        out_win[r * keep + q] = cand_win[r * K + best];
        out_score[r * keep + q] = cand_score[r * K + best];
        if (out_pred) out_pred[r * keep + q] = pred[r * K + best];
      } else {
        out_win[r * keep + q] = -1;
        out_score[r * keep + q] = -INFINITY;
        if (out_pred) out_pred[r * keep + q] = INFINITY;
      }
    }
  }
}

cudaError_t launch_prune(const int64_t* cand_win, const float* cand_score, const float* pred, int64_t n_reads, int K,
                         int keep, int64_t* out_win, float* out_score, float* out_pred, cudaStream_t st) {
  if (n_reads <= 0) return cudaSuccess;
  int64_t blocks = (n_reads + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  prune_kernel<<<(unsigned)blocks, 256, 0, st>>>(cand_win, cand_score, pred, n_reads, K, keep, out_win, out_score,
                                                  out_pred);
  return cudaGetLastError();
}

}  // namespace rope

namespace rope {

__global__ void ld_fraction_kernel(const int32_t* __restrict__ ld, int64_t n, float inv_n, float* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (float)ld[i] * inv_n;
}

cudaError_t launch_ld_fraction(const int32_t* ld, int64_t n, int N, float* out, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int64_t blocks = (n + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  ld_fraction_kernel<<<(unsigned)blocks, 256, 0, st>>>(ld, n, 1.0f / (float)N, out);
  return cudaGetLastError();
}

// The fallback without a network: candidate c of every read is given the
// "prediction" c, so pruning keeps the scan's own ranking.
__global__ void rank_prediction_kernel(int64_t n_reads, int K, float* __restrict__ pred) {
  const int64_t n = n_reads * K;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    pred[i] = (float)(i % K);
}

cudaError_t launch_rank_as_prediction(int64_t n_reads, int K, float* pred, cudaStream_t st) {
  const int64_t n = n_reads * K;
  if (n <= 0) return cudaSuccess;
  int64_t blocks = (n + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  rank_prediction_kernel<<<(unsigned)blocks, 256, 0, st>>>(n_reads, K, pred);
  return cudaGetLastError();
}

}  // namespace rope
