// Materialised window index and its tensor-core scan (wide encodings).
//
// §3.1 builds an index of window encodings -- a database of vectors -- and
// scores a read against it by a matrix product; §3.2 sizes it for 20 kbp reads
// (window N = 20,000, step 1,250, 1024 complex dimensions: ~2.5M vectors for a
// 3.1 Gbp genome). At that width regenerating windows per read tile (the
// on-the-fly scan of the narrow encodings) would cost more than scoring them,
// so this index stores every window once, in BF16 for the tensor cores and in
// FP32 for re-scoring, and the scan is a GEMM.
//
// Index build, exact up to FP32 rounding (no recurrence, so no drift). With
// stride S, the s-mer starts of the reference fall into blocks of S starts;
// block q's sums B_q[k][b] = sum_{i<S} [bin(qS+i) = b] w_k^{f_k i} use
// block-relative phases. Window j (start jS) covers starts jS .. jS+N-s, i.e.
// blocks j .. j+n_blk-1 with block u's phases shifted by w_k^{f_k u S}:
//     c_j[k][b] = sum_u w_k^{f_k u S} B_{j+u}[k][b]  (+/- a short tail)
// where the tail adds the starts of a partial last block, or removes the
// starts past N-s that a whole last block over-covers (§2.1-§2.3 definition,
// summed in another order).
//
// Scan: C[read][window] = <x|c> as a real GEMM on tcgen05 (BF16 in, FP32 in
// tensor memory). Per tile 128 reads x 128 windows and per 64-wide K block, TMA
// brings three 128-row boxes into shared memory: the reads' [xr | xi] rows (A)
// and, back to back as one 256-row B operand, the windows' [cr | ci] rows and
// their [ci | -cr] rows (both stored by the index). One MMA of N = 256 per K
// step then writes Re<x|c> = xr.cr + xi.ci to columns [0, 128) and
// Im<x|c> = xr.ci - xi.cr to columns [128, 256) of the read's tensor-memory
// lane: the epilogue thread of a read forms |.|^2 with no data exchange (§4's
// real identity). Against two N = 128 MMAs (a [-xi | xr] A tile for Im) this
// reads 12 KB of shared memory per 128 tensor cycles instead of 16 KB.
#include <cuda.h>
#include <cuda_bf16.h>

#include "rope_internal.h"
#include "rope_topk.cuh"

namespace rope {

// ---------------------------------------------------------------- index build

// One warp per block of S s-mer starts: lanes compute 32 bins at a time from
// the packed letters, then the lane of each band adds the block-relative
// phase of every start to its bin, in start order (deterministic FP32 sums).
__global__ void block_sums_kernel(DevIndex ix, DenseTables dt, float2* __restrict__ out) {
  extern __shared__ float2 bs_acc[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int wpb = blockDim.x >> 5;
  float2* acc = bs_acc + (size_t)warp * ix.D;
  const int S = ix.stride;
  for (int64_t q = (int64_t)blockIdx.x * wpb + warp; q < dt.n_blocks; q += (int64_t)gridDim.x * wpb) {
    for (int g = lane; g < ix.D; g += 32) acc[g] = make_float2(0.f, 0.f);
    __syncwarp();
    const int64_t p0 = q * S;
    for (int i0 = 0; i0 < S; i0 += 32) {
      const int i = i0 + lane;
      const uint32_t b = i < S ? bin_at(ix.packed, p0 + i, ix.s, ix.map_lsb) : 0u;
      const int cnt = min(32, S - i0);
      for (int jj = 0; jj < cnt; ++jj) {
        const uint32_t bj = __shfl_sync(0xffffffffu, b, jj);
        if (lane < ix.m) {
          const float2 ph = __ldg(dt.bph + (size_t)lane * S + i0 + jj);
          float2& a = acc[lane * ix.nb + bj];
          a.x += ph.x;
          a.y += ph.y;
        }
        __syncwarp();
      }
    }
    float2* o = out + (size_t)q * ix.D;
    for (int g = lane; g < ix.D; g += 32) o[g] = acc[g];
    __syncwarp();
  }
}

// One block of 256 threads per run of consecutive windows; thread t holds
// entries t, t+256, ... (EPT of them). Per window: the tail sums (one warp, in
// start order, into shared memory), the block combination, the squared norm
// (fixed-order block reduction), then the FP32 row, the normalised BF16 rows
// [cr | ci] and [ci | -cr] (the scan's two B operands) and 1/|c|.
template <int EPT>
__global__ void __launch_bounds__(256) dense_windows_kernel(DevIndex ix, DenseTables dt,
                                                            const float2* __restrict__ bsum,
                                                            float* __restrict__ out_f32,
                                                            __nv_bfloat16* __restrict__ out_bf16,
                                                            __nv_bfloat16* __restrict__ out_bf16_im,
                                                            float* __restrict__ inv_norm, int64_t run) {
  extern __shared__ float2 dw_tail[];  // [D]
  __shared__ float red[8];
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const int D = ix.D;
  int band[EPT];
#pragma unroll
  for (int i = 0; i < EPT; ++i) {
    const int e = tid + 256 * i;
    band[i] = e < D ? e / ix.nb : 0;
  }
  const int64_t j_lo = (int64_t)blockIdx.x * run;
  const int64_t j_hi = min(ix.W, j_lo + run);
  for (int64_t j = j_lo; j < j_hi; ++j) {
    if (dt.n_t > 0) {
      for (int e = tid; e < D; e += 256) dw_tail[e] = make_float2(0.f, 0.f);
      __syncthreads();
      if (warp == 0) {
        const int64_t p0 = j * ix.stride + dt.t0;
        for (int i0 = 0; i0 < dt.n_t; i0 += 32) {
          const int i = i0 + lane;
          const uint32_t b = i < dt.n_t ? bin_at(ix.packed, p0 + i, ix.s, ix.map_lsb) : 0u;
          const int cnt = min(32, dt.n_t - i0);
          for (int jj = 0; jj < cnt; ++jj) {
            const uint32_t bj = __shfl_sync(0xffffffffu, b, jj);
            if (lane < ix.m) {
              const float2 ph = __ldg(dt.tph + (size_t)lane * dt.n_t + i0 + jj);
              float2& a = dw_tail[lane * ix.nb + bj];
              a.x += ph.x;
              a.y += ph.y;
            }
            __syncwarp();
          }
        }
      }
      __syncthreads();
    }
    float cr[EPT], ci[EPT];
#pragma unroll
    for (int i = 0; i < EPT; ++i) cr[i] = ci[i] = 0.f;
    for (int u = 0; u < dt.n_blk; ++u) {
      const float2* row = bsum + (size_t)(j + u) * D;
#pragma unroll
      for (int i = 0; i < EPT; ++i) {
        const int e = tid + 256 * i;
        if (e < D) {
          const float2 v = __ldg(row + e);
          const float2 r = __ldg(dt.rotu + (size_t)u * ix.m + band[i]);
          cr[i] = fmaf(v.x, r.x, fmaf(-v.y, r.y, cr[i]));
          ci[i] = fmaf(v.x, r.y, fmaf(v.y, r.x, ci[i]));
        }
      }
    }
    float part = 0.f;
#pragma unroll
    for (int i = 0; i < EPT; ++i) {
      const int e = tid + 256 * i;
      if (e < D) {
        if (dt.n_t > 0) {
          cr[i] += dw_tail[e].x;
          ci[i] += dw_tail[e].y;
        }
        part = fmaf(cr[i], cr[i], fmaf(ci[i], ci[i], part));
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if (lane == 0) red[warp] = part;
    __syncthreads();
    float tot = 0.f;
#pragma unroll
    for (int w = 0; w < 8; ++w) tot += red[w];
    const float inv = tot > kZeroNorm2 ? (float)(1.0 / sqrt((double)tot)) : 0.f;
    float* of = out_f32 + (size_t)j * 2 * D;
    __nv_bfloat16* ob = out_bf16 + (size_t)j * 2 * D;
    __nv_bfloat16* obi = out_bf16_im + (size_t)j * 2 * D;
#pragma unroll
    for (int i = 0; i < EPT; ++i) {
      const int e = tid + 256 * i;
      if (e < D) {
        of[e] = cr[i];
        of[D + e] = ci[i];
        const __nv_bfloat16 br = __float2bfloat16_rn(cr[i] * inv), bi = __float2bfloat16_rn(ci[i] * inv);
        ob[e] = br;
        ob[D + e] = bi;
        obi[e] = bi;
        obi[D + e] = __hneg(br);  // exact: the sign bit
      }
    }
    if (tid == 0) inv_norm[j] = inv;
    __syncthreads();  // red and the tail buffer are reused by the next window
  }
}

cudaError_t launch_dense_index(const DevIndex& ix, const DenseTables& dt, float2* bsum, float* win_f32,
                               uint16_t* win_bf16, uint16_t* win_bf16_im, float* inv_norm, cudaStream_t st) {
  if (dt.n_blocks > 0) {
    int wpb = (int)((96 * 1024) / ((size_t)ix.D * sizeof(float2)));  // accumulators within 96 KB
    wpb = wpb < 1 ? 1 : wpb > 8 ? 8 : wpb;
    const size_t smem = (size_t)wpb * ix.D * sizeof(float2);
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(block_sums_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    int64_t blocks = (dt.n_blocks + wpb - 1) / wpb;
    if (blocks > 152 * 32) blocks = 152 * 32;
    block_sums_kernel<<<(unsigned)blocks, wpb * 32, smem, st>>>(ix, dt, bsum);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const int64_t run = 32;
  const int64_t grid = (ix.W + run - 1) / run;
  const size_t smem = (size_t)ix.D * sizeof(float2);
  auto go = [&](auto kern) -> cudaError_t {
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    kern<<<(unsigned)grid, 256, smem, st>>>(ix, dt, bsum, win_f32, reinterpret_cast<__nv_bfloat16*>(win_bf16),
                                            reinterpret_cast<__nv_bfloat16*>(win_bf16_im), inv_norm, run);
    return cudaGetLastError();
  };
  const int ept = (ix.D + 255) / 256;
  if (ept <= 1) return go(dense_windows_kernel<1>);
  if (ept <= 2) return go(dense_windows_kernel<2>);
  if (ept <= 4) return go(dense_windows_kernel<4>);
  if (ept <= 8) return go(dense_windows_kernel<8>);
  if (ept <= 16) return go(dense_windows_kernel<16>);
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------- scan operands

// A operand of the scan: rows [0, n_pad) are the reads' normalised [xr | xi]
// rows, zero past n (an aligned, padded copy the tensor map can address).
// Eight BF16 entries per thread (2D is a multiple of 64).
__global__ void gemm_a_kernel(const uint16_t* __restrict__ emb, int64_t n, int64_t n_pad, int D,
                              uint16_t* __restrict__ a) {
  const int q8 = 2 * D / 8;
  const int64_t total = n_pad * q8;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = idx / q8;
    const int g = (int)(idx % q8) * 8;
    uint2 lo = make_uint2(0, 0), hi = make_uint2(0, 0);
    if (r < n) {
      lo = *reinterpret_cast<const uint2*>(emb + r * 2 * D + g);
      hi = *reinterpret_cast<const uint2*>(emb + r * 2 * D + g + 4);
    }
    *reinterpret_cast<uint4*>(a + r * 2 * D + g) = make_uint4(lo.x, lo.y, hi.x, hi.y);
  }
}

cudaError_t launch_gemm_a(const uint16_t* emb, int64_t n, int64_t n_pad, int D, uint16_t* a, cudaStream_t st) {
  const int64_t total = n_pad * (2 * D / 8);
  int64_t blocks = (total + 255) / 256;
  if (blocks > 152 * 64) blocks = 152 * 64;
  if (blocks < 1) return cudaSuccess;
  gemm_a_kernel<<<(unsigned)blocks, 256, 0, st>>>(emb, n, n_pad, D, a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- tensor-core scan

// Two shapes of the same scan. Long K (2D > 128, e.g. the long-read 2D = 2048):
// every stage brings one K block of A, B_re and B_im; one epilogue warp per
// tensor-memory lane quarter. Short K (2D <= 128: the d = 64 and d = 128
// encodings): the read tile's A (at most two K blocks) stays resident in shared
// memory for the whole work item, stages carry only the window boxes, and two
// epilogue warps share each lane quarter (half of the tile's columns and their
// own candidate list each): with so few MMAs per tile, the epilogue, not the
// tensor pipe, would otherwise set the pace.
template <bool kShort>
struct GemmShape {
  static constexpr int BM = 128;                 // reads per tile (tensor-memory lanes)
  static constexpr int BN = 128;                 // windows per tile (MMA N = 2 BN: Re and Im rows)
  static constexpr int BK = 64;                  // K per stage: one 128-byte swizzled BF16 row
  static constexpr int BOX_BYTES = 128 * BK * 2;           // one 128-row box: 16 KB
  static constexpr int STAGE_BYTES = (kShort ? 2 : 3) * BOX_BYTES;  // [A,] B_re, B_im
  static constexpr int MAX_STAGES = kShort ? 6 : 4;
  static constexpr int MAX_RES_KB = 2;           // short K: resident A of at most 2 K blocks
  static constexpr int EQ = kShort ? 2 : 1;      // epilogue warps per lane quarter
  static constexpr int WCOLS = BN / EQ;          // windows per epilogue warp per tile
  static constexpr int ACC_COLS = 2 * BN;                  // Re and Im accumulators of a tile
  static constexpr int TMEM_COLS = 512;                    // two accumulator buffers
  static constexpr int EPI_WARPS = 4 * EQ;
  static constexpr int NTHREADS = 32 * (2 + EPI_WARPS);    // producer, MMA, epilogue
  static constexpr uint32_t IDESC = idesc_bf16_f32(BM, 2 * BN);
  static_assert(2 * ACC_COLS <= TMEM_COLS, "tensor memory");
  static_assert(2 * BN <= 256 && BOX_BYTES % 1024 == 0, "B_re and B_im form one swizzled 256-row operand");
  static_assert(WCOLS % 16 == 0, "the epilogue loads 16-column chunks");
  // dynamic shared memory: [resident A][stages][lists], 1024-aligned
  static size_t smem_bytes(int stages, int cand_depth, int k_blocks) {
    return 1024 + (kShort ? (size_t)k_blocks * BOX_BYTES : 0) + (size_t)stages * STAGE_BYTES +
           (size_t)cand_depth * BM * EQ * 8;
  }
};

// largest of 16 scores: a depth-3 tree of 3-input maxima (short dependency
// chains for the latency-bound epilogue)
__device__ __forceinline__ float max3f(float a, float b, float c) {
  float d;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}
__device__ __forceinline__ float max16(const float (&v)[16]) {
  const float m0 = max3f(v[0], v[1], v[2]), m1 = max3f(v[3], v[4], v[5]), m2 = max3f(v[6], v[7], v[8]);
  const float m3 = max3f(v[9], v[10], v[11]), m4 = max3f(v[12], v[13], v[14]);
  return fmaxf(max3f(m0, m1, m2), max3f(m3, m4, v[15]));
}

// (read tile, window range) of item `it`; false for the padding items of the
// last wave. Items come in waves of grp read tiles x n_ranges ranges, range
// by range, so that a wave's blocks share each window tile in L2 while its
// grp read tiles stay resident there.
__device__ __forceinline__ bool gemm_item(const GemmArgs& g, int64_t it, int& rt, int& rg, int64_t& w_lo,
                                          int64_t& w_hi) {
  const int64_t per_wave = (int64_t)g.grp * g.n_ranges;
  const int64_t wv = it / per_wave;
  const int64_t in = it % per_wave;
  rg = (int)(in / g.grp);
  rt = (int)(wv * g.grp + in % g.grp);
  w_lo = g.jb + (int64_t)rg * g.range_len;
  w_hi = min(w_lo + g.range_len, g.je);
  return rt < g.n_rt;
}

// kMode 0: per-read candidate lists (top-k); 1: every score into g.dense;
// 2: every pair whose score reaches its window's threshold g.thr.thr[j],
// appended at an atomically taken index of g.thr's bounded arrays.
template <int kMode, bool kShort>
__global__ void __launch_bounds__(GemmShape<kShort>::NTHREADS, 1)
    gemm_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const __grid_constant__ CUtensorMap tmBi, GemmArgs g) {
  using Sh = GemmShape<kShort>;
  constexpr bool kDense = kMode == 1, kThr = kMode == 2, kLists = kMode == 0;
  extern __shared__ __align__(1024) uint8_t gm_raw[];
  __shared__ __align__(8) uint64_t bar_full[Sh::MAX_STAGES], bar_empty[Sh::MAX_STAGES];
  __shared__ __align__(8) uint64_t bar_accfull[2], bar_accempty[2], bar_drain, bar_afull, bar_aempty;
  __shared__ uint32_t tmem_base_s;
  __shared__ int abort_s;
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(gm_raw) + 1023) & ~uintptr_t(1023));
  const int kbl = g.k_blocks;
  uint8_t* a_res = smem;  // short K: the item's A tile, kbl K blocks
  uint8_t* stages = smem + (kShort ? (size_t)kbl * Sh::BOX_BYTES : 0);
  float* list_s = reinterpret_cast<float*>(stages + (size_t)g.stages * Sh::STAGE_BYTES);
  uint32_t* list_w = reinterpret_cast<uint32_t*>(list_s + (size_t)g.cand_depth * Sh::BM * Sh::EQ);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint64_t wlim = g.wait_limit_ns;
  volatile int* abort_flag = &abort_s;
  const int ns = g.stages;

  if (tid == 0) {
    for (int i = 0; i < ns; ++i) {
      mbar_init(&bar_full[i], 1);
      mbar_init(&bar_empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&bar_accfull[i], 1);
      mbar_init(&bar_accempty[i], Sh::EPI_WARPS);
    }
    mbar_init(&bar_drain, 1);
    mbar_init(&bar_afull, 1);
    mbar_init(&bar_aempty, 1);
    abort_s = 0;
    fence_barrier_init();
    prefetch_tensor_map(&tmA);
    prefetch_tensor_map(&tmB);
    prefetch_tensor_map(&tmBi);
  }
  if (warp == 1) {
    tmem_alloc(&tmem_base_s, Sh::TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tmem_base_s;
  const int64_t n_items = (int64_t)((g.n_rt + g.grp - 1) / g.grp) * g.grp * g.n_ranges;

  if (warp == 0) {
    // ================================================================ TMA producer
    if (lane == 0) {
      uint32_t stage = 0, phase = 0, a_par = 0;
      int64_t issued = 0, a_issued = 0;
      for (int64_t it = blockIdx.x; it < n_items; it += gridDim.x) {
        int rt, rg;
        int64_t w_lo, w_hi;
        if (!gemm_item(g, it, rt, rg, w_lo, w_hi)) continue;
        bool ok = true;
        if constexpr (kShort) {
          // the resident A tile: free once the previous item's MMAs completed
          if (!mbar_wait(&bar_aempty, a_par ^ 1u, abort_flag, g.status, wlim)) break;
          mbar_expect_tx(&bar_afull, (uint32_t)(kbl * Sh::BOX_BYTES));
          for (int kb = 0; kb < kbl; ++kb)
            tma_load_2d(a_res + (size_t)kb * Sh::BOX_BYTES, &tmA, kb * Sh::BK, rt * Sh::BM, &bar_afull);
          a_par ^= 1u;
          ++a_issued;
        }
        for (int64_t w0 = w_lo; w0 < w_hi && ok; w0 += Sh::BN) {
          for (int kb = 0; kb < kbl; ++kb) {
            if (!mbar_wait(&bar_empty[stage], phase ^ 1u, abort_flag, g.status, wlim)) {
              ok = false;
              break;
            }
            uint8_t* st = stages + (size_t)stage * Sh::STAGE_BYTES;
            mbar_expect_tx(&bar_full[stage], Sh::STAGE_BYTES);
            if constexpr (!kShort) {
              tma_load_2d(st, &tmA, kb * Sh::BK, rt * Sh::BM, &bar_full[stage]);
              st += Sh::BOX_BYTES;
            }
            tma_load_2d(st, &tmB, kb * Sh::BK, (int32_t)w0, &bar_full[stage]);
            tma_load_2d(st + Sh::BOX_BYTES, &tmBi, kb * Sh::BK, (int32_t)w0, &bar_full[stage]);
            ++issued;
            if (++stage == (uint32_t)ns) {
              stage = 0;
              phase ^= 1u;
            }
          }
        }
        if (!ok) break;
      }
      // the latest copy into each stage (and into the A tile) may still be in
      // flight (after an abort)
      for (int64_t i = issued > ns ? issued - ns : 0; i < issued; ++i)
        mbar_drain_wait(&bar_full[i % ns], (uint32_t)((i / ns) & 1), g.status, wlim);
      if (kShort && a_issued > 0) mbar_drain_wait(&bar_afull, (uint32_t)((a_issued - 1) & 1), g.status, wlim);
    }
  } else if (warp == 1) {
    // ================================================================ MMA issue
    if (lane == 0) {
      uint32_t stage = 0, phase = 0, t = 0, a_par = 0;
      bool ok = true;
      for (int64_t it = blockIdx.x; it < n_items && ok; it += gridDim.x) {
        int rt, rg;
        int64_t w_lo, w_hi;
        if (!gemm_item(g, it, rt, rg, w_lo, w_hi)) continue;
        if constexpr (kShort) {
          if (!mbar_wait(&bar_afull, a_par, abort_flag, g.status, wlim)) break;
          a_par ^= 1u;
          tc_fence_after();
        }
        for (int64_t w0 = w_lo; w0 < w_hi && ok; w0 += Sh::BN, ++t) {
          const uint32_t buf = t & 1u;
          if (!mbar_wait(&bar_accempty[buf], ((t >> 1) & 1u) ^ 1u, abort_flag, g.status, wlim)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t d = tbase + buf * Sh::ACC_COLS;  // Re: columns [0, BN), Im: [BN, 2 BN)
          for (int kb = 0; kb < kbl; ++kb) {
            if (!mbar_wait(&bar_full[stage], phase, abort_flag, g.status, wlim)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t base = smem_u32(stages + (size_t)stage * Sh::STAGE_BYTES);
            const uint64_t a = kShort ? smem_desc_sw128(smem_u32(a_res) + (uint32_t)kb * Sh::BOX_BYTES)
                                      : smem_desc_sw128(base);
            // 256 rows: B_re then B_im
            const uint64_t b = smem_desc_sw128(base + (kShort ? 0u : (uint32_t)Sh::BOX_BYTES));
#pragma unroll
            for (int kk = 0; kk < Sh::BK / 16; ++kk) {
              const uint32_t acc = (kb > 0 || kk > 0) ? 1u : 0u;
              // K step kk: 32 bytes further along the 128-byte rows (16-byte units)
              tc_mma_ss(d, a + 2 * kk, b + 2 * kk, Sh::IDESC, acc);
            }
            tc_commit(&bar_empty[stage]);
            if (++stage == (uint32_t)ns) {
              stage = 0;
              phase ^= 1u;
            }
          }
          if (ok) tc_commit(&bar_accfull[buf]);
        }
        // the resident A tile is free once this item's MMAs have completed
        if (kShort) tc_commit(&bar_aempty);
      }
      // every MMA issued by this thread has completed (also after an abort)
      tc_commit(&bar_drain);
      mbar_drain_wait(&bar_drain, 0, g.status, wlim);
    }
  } else {
    // ================================================================ epilogue
    // thread = one read (tensor-memory lane 32q + lane of its warp's quarter);
    // with EQ warps per quarter, warp h of a quarter takes the tile's columns
    // [h WCOLS, (h + 1) WCOLS) and keeps its own list for them
    const int q = warp & 3;
    const int h = (warp - 2) >> 2;
    const int row = 32 * q + lane;
    const uint32_t lane_base = (uint32_t)(32 * q) << 16;
    constexpr int LSTR = Sh::BM * Sh::EQ;  // list entry stride
    float* ls = list_s + h * Sh::BM + row;
    uint32_t* lw = list_w + h * Sh::BM + row;
    uint32_t t = 0;
    const int64_t n_dense = g.je - g.jb;
    for (int64_t it = blockIdx.x; it < n_items; it += gridDim.x) {
      int rt, rg;
      int64_t w_lo, w_hi;
      if (!gemm_item(g, it, rt, rg, w_lo, w_hi)) continue;
      const int64_t r = (int64_t)rt * Sh::BM + row;
      const bool have = r < g.n_reads;
      float thr = -INFINITY;
      int worst = 0;
      if (kLists) {
        for (int e = 0; e < g.cand_depth; ++e) {
          ls[e * LSTR] = -INFINITY;
          lw[e * LSTR] = kEmptyWin;
        }
      }
      for (int64_t w0 = w_lo; w0 < w_hi; w0 += Sh::BN, ++t) {
        const uint32_t buf = t & 1u;
        if (!mbar_wait_warp(&bar_accfull[buf], (t >> 1) & 1u, abort_flag, g.status, wlim)) goto epi_done;
        tc_fence_after();
        const int64_t wc = w0 + h * Sh::WCOLS;  // this warp's first window
        const bool full = wc + Sh::WCOLS <= w_hi;
        const uint32_t tcol = tbase + lane_base + buf * Sh::ACC_COLS + (uint32_t)(h * Sh::WCOLS);
        // the 16 windows from column c0 of this warp's share: Re in vr, Im in vi
        auto chunk = [&](const uint32_t* vr, const uint32_t* vi, int c0) {
          float sc[16];
#pragma unroll
          for (int n = 0; n < 16; n += 2) abs2_pair(vr[n], vr[n + 1], vi[n], vi[n + 1], sc[n], sc[n + 1]);
          const int64_t jc = wc + c0;
          if constexpr (kThr) {
            // lane l holds the threshold of window jc + (l & 15) (+inf outside
            // the range); the chunk's smallest threshold decides whether any
            // of its 16 scores needs a look
            const float tl = (jc + (lane & 15) < w_hi) ? __ldg(g.thr.thr + jc + (lane & 15)) : INFINITY;
            float mn = tl;
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
            const float mx = max16(sc);
            if (__any_sync(0xffffffffu, have && mx >= mn)) {
#pragma unroll
              for (int n = 0; n < 16; ++n) {
                const float th = __shfl_sync(0xffffffffu, tl, n);
                if (have && sc[n] >= th) {
                  const unsigned long long slot = atomicAdd(g.thr.count, 1ull);
                  if (slot < (unsigned long long)g.thr.cap) {
                    g.thr.read[slot] = r;
                    g.thr.win[slot] = jc + n;
                    g.thr.score[slot] = sc[n];
                  }
                }
              }
            }
          } else if constexpr (kDense) {
            if (have) {
#pragma unroll
              for (int n = 0; n < 16; ++n)
                if (jc + n < w_hi) g.dense[r * n_dense + (jc + n - g.jb)] = sc[n];
            }
          } else {
            float mx = -INFINITY;
            if (full) {
              mx = max16(sc);
            } else {
#pragma unroll
              for (int n = 0; n < 16; ++n)
                if (jc + n < w_hi) mx = fmaxf(mx, sc[n]);
            }
            if (have && mx >= thr) {
              for (int n = 0; n < 16; ++n) {
                if (jc + n >= w_hi || !(sc[n] >= thr)) continue;
                const ListState nsl = list_insert(ls, lw, LSTR, g.cand_depth, worst, sc[n], (uint32_t)(jc + n),
                                                  g.sep, g.stride);
                thr = nsl.thr;
                worst = nsl.worst;
              }
            }
          }
        };
        if constexpr (kShort) {
          // every column of this warp's share in registers at once: one exposed
          // tensor-memory load latency per tile instead of one per chunk
          uint32_t vr[Sh::WCOLS], vi[Sh::WCOLS];
#pragma unroll
          for (int u = 0; u < Sh::WCOLS; u += 16) {
            tmem_ld16(tcol + u, *reinterpret_cast<uint32_t(*)[16]>(&vr[u]));
            tmem_ld16(tcol + Sh::BN + u, *reinterpret_cast<uint32_t(*)[16]>(&vi[u]));
          }
          tc_wait_ld();
          reg_fence(vr);
          reg_fence(vi);
          // all of this warp's columns are in registers: hand the buffer back
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&bar_accempty[buf]);
#pragma unroll
          for (int c0 = 0; c0 < Sh::WCOLS; c0 += 16) chunk(vr + c0, vi + c0, c0);
        } else {
#pragma unroll 1
          for (int c0 = 0; c0 < Sh::WCOLS; c0 += 16) {
            uint32_t vr[16], vi[16];
            tmem_ld16(tcol + c0, vr);
            tmem_ld16(tcol + Sh::BN + c0, vi);
            tc_wait_ld();
            reg_fence(vr);
            reg_fence(vi);
            if (c0 + 16 == Sh::WCOLS) {
              // this warp's last columns are in registers: hand the buffer back
              tc_fence_before();
              __syncwarp();
              if (lane == 0) mbar_arrive(&bar_accempty[buf]);
            }
            chunk(vr, vi, c0);
          }
        }
      }
      if (kLists && have) {
        Candidate* out = g.cand + (((size_t)r * g.n_ranges + rg) * Sh::EQ + h) * g.cand_depth;
        for (int e = 0; e < g.cand_depth; ++e) out[e] = Candidate{ls[e * LSTR], lw[e * LSTR]};
      }
    }
  epi_done:;
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tbase, Sh::TMEM_COLS);
  }
}

// ---------------------------------------------------------------- FP32 plain scan

// The plain path of the materialised index: FP32 inner products of the reads'
// unnormalised FP32 encodings with the stored FP32 window rows on the CUDA
// cores. A block of 256 threads computes a 64-read x 64-window tile, each
// thread a 4 x 4 sub-tile of (Re, Im) accumulators, over K in chunks of 32
// complex entries staged in shared memory; the tile's fidelities
// |ip|^2 / (|x|^2 |c|^2) go to shared memory and one thread per read offers
// them, in window order, to its read's candidate list. Work items are
// (read tile, window range) as in the GEMM scan.
constexpr int kF32Tile = 64;
constexpr int kF32Kc = 32;  // complex entries per K chunk

__global__ void __launch_bounds__(256) dense_fp32_kernel(DevIndex ix, GemmArgs g, const float* __restrict__ emb,
                                                         const float* __restrict__ norms) {
  __shared__ float2 xs[kF32Kc][kF32Tile + 1];   // [k][read]: (xr, xi); the score tile after the K loop
  __shared__ float2 cs[kF32Kc][kF32Tile + 1];   // [k][window]: (cr, ci)
  static_assert(sizeof(xs) >= sizeof(float) * kF32Tile * (kF32Tile + 1), "score tile overlays xs");
  float (*tile_s)[kF32Tile + 1] = reinterpret_cast<float (*)[kF32Tile + 1]>(&xs[0][0]);
  extern __shared__ float f32_lists[];          // [cand_depth][64] scores, then windows
  float* ls_all = f32_lists;
  uint32_t* lw_all = reinterpret_cast<uint32_t*>(f32_lists + (size_t)g.cand_depth * kF32Tile);
  const int tid = threadIdx.x;
  const int tr = tid / 16, tc = tid % 16;  // sub-tile: reads 4tr..4tr+3, windows 4tc..4tc+3
  const int D = ix.D, m = ix.m;
  const int64_t n_items = (int64_t)((g.n_rt + g.grp - 1) / g.grp) * g.grp * g.n_ranges;
  for (int64_t it = blockIdx.x; it < n_items; it += gridDim.x) {
    int rt, rg;
    int64_t w_lo, w_hi;
    if (!gemm_item(g, it, rt, rg, w_lo, w_hi)) continue;
    const int64_t r0 = (int64_t)rt * kF32Tile;
    float thr = -INFINITY;
    int worst = 0;
    float* ls = ls_all + (tid < kF32Tile ? tid : 0);
    uint32_t* lw = lw_all + (tid < kF32Tile ? tid : 0);
    if (tid < kF32Tile)
      for (int e = 0; e < g.cand_depth; ++e) {
        ls[e * kF32Tile] = -INFINITY;
        lw[e * kF32Tile] = kEmptyWin;
      }
    for (int64_t w0 = w_lo; w0 < w_hi; w0 += kF32Tile) {
      float re[4][4], im[4][4];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) re[a][b] = im[a][b] = 0.f;
      for (int k0 = 0; k0 < D; k0 += kF32Kc) {
        __syncthreads();  // the previous chunk (or tile) is consumed
        for (int q = tid; q < kF32Kc * kF32Tile; q += 256) {
          const int k = q % kF32Kc, i = q / kF32Kc;
          const int64_t r = r0 + i, j = w0 + i;
          const float* xrow = emb + (size_t)r * 2 * D;
          const float* crow = ix.win_f32 + (size_t)j * 2 * D;
          xs[k][i] = r < g.n_reads ? make_float2(xrow[k0 + k], xrow[D + k0 + k]) : make_float2(0.f, 0.f);
          cs[k][i] = j < w_hi ? make_float2(crow[k0 + k], crow[D + k0 + k]) : make_float2(0.f, 0.f);
        }
        __syncthreads();
#pragma unroll 4
        for (int k = 0; k < kF32Kc; ++k) {
          float2 x[4], c[4];
#pragma unroll
          for (int a = 0; a < 4; ++a) x[a] = xs[k][4 * tr + a];
#pragma unroll
          for (int b = 0; b < 4; ++b) c[b] = cs[k][4 * tc + b];
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) {
              // Re += xr cr + xi ci, Im += xr ci - xi cr (conj(x) . c, §4)
              re[a][b] = fmaf(x[a].x, c[b].x, fmaf(x[a].y, c[b].y, re[a][b]));
              im[a][b] = fmaf(x[a].x, c[b].y, fmaf(-x[a].y, c[b].x, im[a][b]));
            }
        }
      }
      // fidelities of the tile (over the staged x chunk: every thread is past it)
      __syncthreads();
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const int64_t r = r0 + 4 * tr + a;
        const float X = r < g.n_reads ? norms[r * (1 + m)] : 0.f;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int64_t j = w0 + 4 * tc + b;
          const float inv = j < w_hi ? __ldg(ix.inv_norm + j) : 0.f;  // 1/|c|, 0 for a zero vector
          const float num = fmaf(re[a][b], re[a][b], im[a][b] * im[a][b]);
          tile_s[4 * tr + a][4 * tc + b] = (X > kZeroNorm2 && inv > 0.f) ? num / X * (inv * inv) : 0.f;
        }
      }
      __syncthreads();
      if (tid < kF32Tile && r0 + tid < g.n_reads) {
        const int n_w = (int)(w_hi - w0 < kF32Tile ? w_hi - w0 : kF32Tile);
        for (int n = 0; n < n_w; ++n) {
          const float v = tile_s[tid][n];
          if (v >= thr) {
            const ListState ns = list_insert(ls, lw, kF32Tile, g.cand_depth, worst, v, (uint32_t)(w0 + n), g.sep,
                                             g.stride);
            thr = ns.thr;
            worst = ns.worst;
          }
        }
      }
    }
    if (tid < kF32Tile && r0 + tid < g.n_reads) {
      Candidate* out = g.cand + ((size_t)(r0 + tid) * g.n_ranges + rg) * g.cand_depth;
      for (int e = 0; e < g.cand_depth; ++e) out[e] = Candidate{ls[e * kF32Tile], lw[e * kF32Tile]};
    }
    __syncthreads();  // the lists are reused by the next item
  }
}

int dense_fp32_group() { return kF32Tile; }

cudaError_t launch_dense_fp32(const DevIndex& ix, const GemmArgs& g, const float* emb, const float* norms, int num_sms,
                              cudaStream_t st) {
  const int64_t n_items = (int64_t)((g.n_rt + g.grp - 1) / g.grp) * g.grp * g.n_ranges;
  int64_t grid = n_items < (int64_t)num_sms * 2 ? n_items : (int64_t)num_sms * 2;
  if (grid < 1) return cudaSuccess;
  const size_t smem = (size_t)g.cand_depth * kF32Tile * 8;
  // lists of up to 32 entries (16 KB) beside 33 KB of static tiles: past the
  // default 48 KB per block
  const cudaError_t attr =
      cudaFuncSetAttribute(dense_fp32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (attr != cudaSuccess) return attr;
  dense_fp32_kernel<<<(unsigned)grid, 256, smem, st>>>(ix, g, emb, norms);
  return cudaGetLastError();
}

int gemm_tc_group() { return GemmShape<false>::BM; }
int gemm_tc_window_tile() { return GemmShape<false>::BN; }
int gemm_tc_lists(int k_blocks) { return k_blocks <= GemmShape<true>::MAX_RES_KB ? GemmShape<true>::EQ : 1; }

// Deepest pipeline of the shape for k_blocks whose shared memory fits with
// lists of cand_depth (0: none fits).
int gemm_tc_stages(int cand_depth, int k_blocks) {
  int optin = 0, dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const size_t avail = (size_t)optin > 2048 ? (size_t)optin - 2048 : 0;  // static shared memory
  auto deepest = [&](auto shape) {
    using Sh = decltype(shape);
    for (int s = Sh::MAX_STAGES; s >= 2; --s)
      if (Sh::smem_bytes(s, cand_depth, k_blocks) <= avail) return s;
    return 0;
  };
  return k_blocks <= GemmShape<true>::MAX_RES_KB ? deepest(GemmShape<true>{}) : deepest(GemmShape<false>{});
}

cudaError_t launch_gemm_tc(const CUtensorMap& tmA, const CUtensorMap& tmB, const CUtensorMap& tmBi,
                           const GemmArgs& g, int mode, int num_sms, cudaStream_t st) {
  const int64_t n_items = (int64_t)((g.n_rt + g.grp - 1) / g.grp) * g.grp * g.n_ranges;
  const int grid = (int)(n_items < num_sms ? n_items : num_sms);
  if (grid < 1) return cudaSuccess;
  const bool short_k = g.k_blocks <= GemmShape<true>::MAX_RES_KB;
  const size_t smem = short_k ? GemmShape<true>::smem_bytes(g.stages, mode == 0 ? g.cand_depth : 0, g.k_blocks)
                              : GemmShape<false>::smem_bytes(g.stages, mode == 0 ? g.cand_depth : 0, g.k_blocks);
  auto go = [&](auto kern, int threads) -> cudaError_t {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return e;
    }
    kern<<<grid, threads, smem, st>>>(tmA, tmB, tmBi, g);
    return cudaGetLastError();
  };
  if (short_k) {
    constexpr int T = GemmShape<true>::NTHREADS;
    return mode == 1 ? go(gemm_tc_kernel<1, true>, T) : mode == 2 ? go(gemm_tc_kernel<2, true>, T)
                                                                 : go(gemm_tc_kernel<0, true>, T);
  }
  constexpr int T = GemmShape<false>::NTHREADS;
  return mode == 1 ? go(gemm_tc_kernel<1, false>, T) : mode == 2 ? go(gemm_tc_kernel<2, false>, T)
                                                                : go(gemm_tc_kernel<0, false>, T);
}

}  // namespace rope
