// Mutated copies on the GPU and the fidelities built on them: the §2.4
// scoring of correlations (random strings against their mutated copies, the
// samples behind the fitting curve) and the §3.4 per-window thresholds of the
// materialised index.
//
// A copy is the first N letters of a walk over a source string in which each
// letter is mutated with probability err: deleted, preceded by a random
// inserted letter, or substituted by one of the three other letters, each
// with probability 1/3 (past the end of the source the walk reads A). Its
// draws are SplitMix64 outputs: the stream keyed by output `stream` of the
// generator started at `seed`, outputs 3d, 3d+1, 3d+2 of that stream for
// source letter d (mutated?, kind, letter), compared in double precision --
// the walk of the threshold regime (rope_threshold.cu), so a copy is fixed by
// (seed, stream) alone.
#include <cuda_runtime.h>

#include "rope_internal.h"

namespace rope {

// One thread per copy. Strings mode (seqs != null): copy i walks string i with
// errs[i], stream i. Windows mode: copy i = (window j0 + i / n_samples, copy
// t = i % n_samples) walks the packed reference from the window's start with
// err, stream j * n_samples + t.
__global__ void mutate_kernel(MutArgs a) {
  static const char kAcgt[4] = {'A', 'C', 'G', 'T'};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint8_t* str = nullptr;
    int64_t len = 0, pos0 = 0;
    uint64_t stream;
    double err;
    if (a.seqs) {
      str = a.seqs + a.offsets[i];
      len = a.offsets[i + 1] - a.offsets[i];
      stream = (uint64_t)i;
      err = a.errs[i];
    } else {
      const int64_t j = a.j0 + i / a.n_samples;
      pos0 = j * a.stride;
      len = a.L - pos0;
      stream = (uint64_t)j * a.n_samples + (uint64_t)(i % a.n_samples);
      err = a.err;
    }
    const uint64_t key = sm64_out(a.seed, stream);
    uint8_t* out = a.out + (size_t)i * a.N;
    int bad = 0;
    int n = 0;
    for (int64_t d = 0; n < a.N; ++d) {
      uint32_t c = 0;  // 'A' past the end
      if (d < len) {
        if (str) {
          c = letter_code(str[d]);
          if (c > 3) {
            bad = 1;
            c = 0;
          }
        } else {
          const int64_t p = pos0 + d;
          c = (__ldg(a.packed + (p >> 4)) >> ((p & 15) * 2)) & 3u;
        }
      }
      if (sm64_unit(sm64_out(key, 3 * (uint64_t)d)) < err) {
        const int kind = (int)(sm64_unit(sm64_out(key, 3 * (uint64_t)d + 1)) * 3.0);
        const uint64_t z2 = sm64_out(key, 3 * (uint64_t)d + 2);
        if (kind == 0) continue;  // deletion
        if (kind == 1) {          // a random letter, then the source letter
          out[n++] = (uint8_t)kAcgt[z2 >> 62];
          if (n < a.N) out[n++] = (uint8_t)kAcgt[c];
          continue;
        }
        c = (c + 1u + (uint32_t)(int)(sm64_unit(z2) * 3.0)) & 3u;  // substitution
      }
      out[n++] = (uint8_t)kAcgt[c];
    }
    if (bad) set_status(a.status, kStatusBadBase);
  }
}

cudaError_t launch_mutate(const MutArgs& a, cudaStream_t st) {
  if (a.n <= 0) return cudaSuccess;
  int64_t blocks = (a.n + 127) / 128;
  if (blocks > 152 * 32) blocks = 152 * 32;
  mutate_kernel<<<(unsigned)blocks, 128, 0, st>>>(a);
  return cudaGetLastError();
}

// fidelity (score mode 0: concatenated, §2.4; 1: per-band mean, §2.5) of two
// FP32 encodings x, y [2D] with squared norms nx, ny [1 + m]; warp-wide,
// fixed-order reduction; every lane returns the result
__device__ float warp_fidelity(const float* __restrict__ x, const float* __restrict__ y, const float* nx,
                               const float* ny, int D, int m, int nb, int score_mode) {
  const int lane = threadIdx.x & 31;
  const int parts = score_mode == 1 ? m : 1;
  const int span = score_mode == 1 ? nb : D;
  float fid = 0.f;
  for (int k = 0; k < parts; ++k) {
    float re = 0.f, im = 0.f;
    for (int g = k * span + lane; g < (k + 1) * span; g += 32) {
      const float xr = x[g], xi = x[D + g], yr = y[g], yi = y[D + g];
      re = fmaf(xr, yr, fmaf(xi, yi, re));
      im = fmaf(xr, yi, fmaf(-xi, yr, im));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      re += __shfl_xor_sync(0xffffffffu, re, o);
      im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    const float X = score_mode == 1 ? nx[1 + k] : nx[0], Y = score_mode == 1 ? ny[1 + k] : ny[0];
    fid += (X > kZeroNorm2 && Y > kZeroNorm2) ? fmaf(re, re, im * im) / (X * Y) : 0.f;
  }
  return score_mode == 1 ? fid / m : fid;
}

// One warp per pair: string i (row i) against its copy (row n + i).
__global__ void pair_fidelity_kernel(const float* __restrict__ emb, const float* __restrict__ norms, int64_t n,
                                     int D, int m, int nb, int score_mode, float* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps) {
    const float f = warp_fidelity(emb + (size_t)i * 2 * D, emb + (size_t)(n + i) * 2 * D, norms + i * (1 + m),
                                  norms + (n + i) * (1 + m), D, m, nb, score_mode);
    if (lane == 0) out[i] = f;
  }
}

cudaError_t launch_pair_fidelity(const float* emb, const float* norms, int64_t n, int D, int m, int nb,
                                 int score_mode, float* out, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int64_t blocks = (n + 7) / 8;
  if (blocks > 152 * 32) blocks = 152 * 32;
  pair_fidelity_kernel<<<(unsigned)blocks, 256, 0, st>>>(emb, norms, n, D, m, nb, score_mode, out);
  return cudaGetLastError();
}

// Per-window threshold of the materialised index: the mean, in copy order, of
// the fidelities between window j's stored FP32 row and its n_samples copies
// (rows (j - j0) * n_samples + t of emb), one warp per window, FP64 mean.
__global__ void window_threshold_kernel(DevIndex ix, const float* __restrict__ emb, const float* __restrict__ norms,
                                        int64_t j0, int64_t count, int n_samples, float* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int D = ix.D, m = ix.m;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < count; w += warps) {
    const int64_t j = j0 + w;
    const float* c = ix.win_f32 + (size_t)j * 2 * D;
    // the window's squared norm (score mode 0: the materialised index's only mode)
    float C = 0.f;
    for (int g = lane; g < D; g += 32) C = fmaf(c[g], c[g], fmaf(c[D + g], c[D + g], C));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) C += __shfl_xor_sync(0xffffffffu, C, o);
    float nc[1] = {C};
    double sum = 0.0;
    for (int t = 0; t < n_samples; ++t) {
      const int64_t row = w * n_samples + t;
      sum += (double)warp_fidelity(emb + (size_t)row * 2 * D, c, norms + row * (1 + m), nc, D, m, ix.nb, 0);
    }
    if (lane == 0) out[w] = (float)(sum / n_samples);
  }
}

cudaError_t launch_window_thresholds(const DevIndex& ix, const float* emb, const float* norms, int64_t j0,
                                     int64_t count, int n_samples, float* out, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  int64_t blocks = (count + 7) / 8;
  if (blocks > 152 * 32) blocks = 152 * 32;
  window_threshold_kernel<<<(unsigned)blocks, 256, 0, st>>>(ix, emb, norms, j0, count, n_samples, out);
  return cudaGetLastError();
}

// offsets[i] = i * N for i <= n (copies laid out back to back)
__global__ void iota_offsets_kernel(int64_t* __restrict__ off, int64_t n, int64_t N) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += (int64_t)gridDim.x * blockDim.x)
    off[i] = i * N;
}

cudaError_t launch_iota_offsets(int64_t* off, int64_t n, int64_t N, cudaStream_t st) {
  int64_t blocks = (n + 1 + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  iota_offsets_kernel<<<(unsigned)blocks, 256, 0, st>>>(off, n, N);
  return cudaGetLastError();
}

}  // namespace rope
