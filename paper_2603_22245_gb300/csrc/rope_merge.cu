// Merge of the per-range candidate lists, optional FP32 re-scoring by direct
// summation, and the final per-read top-k (§3.5, generalised from top-1).
//
// One warp per read. Candidates are ordered by the 64-bit key
// (orderable score << 32 | ~window), so the best entry is the key maximum and
// ties in score go to the lower window. The warp extracts the best
// `depth` candidates one at a time (with sep > 0, skipping windows whose
// bucket is already taken); if re-scoring is on, each kept window's
// encoding is rebuilt by direct summation over its N-s+1 locations (§2.1-§2.3,
// FP32, location order) and its fidelity recomputed against the read's FP32
// encoding; the kept entries are then sorted across the warp (bitonic) and the
// first k written.
#include "rope_internal.h"
#include "rope_topk.cuh"

namespace rope {

__device__ __forceinline__ uint32_t ord_float(float f) {
  const uint32_t b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float unord_float(uint32_t u) {
  return __uint_as_float((u & 0x80000000u) ? (u ^ 0x80000000u) : ~u);
}
__device__ __forceinline__ uint64_t cand_key(float s, uint32_t w) {
  return ((uint64_t)ord_float(s) << 32) | (uint64_t)(0xFFFFFFFFu - w);
}

__device__ __forceinline__ uint64_t warp_max_u64(uint64_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const uint64_t u = __shfl_xor_sync(0xffffffffu, v, o);
    v = u > v ? u : v;
  }
  return v;
}

__global__ void merge_kernel(DevIndex ix, MergeArgs a) {
  extern __shared__ float2 merge_acc[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int wpb = blockDim.x >> 5;
  float2* acc = merge_acc + (size_t)warp * ix.D;
  const int total = a.n_ranges * a.cand_depth;
  const int depth = a.rescore ? a.rescore_depth : a.k;
  const int n_loc = ix.N - ix.s + 1;
  const int D = ix.D;
  // the scan's lists are incomplete after a timeout: report nothing rather than part
  const int scan_bits = *reinterpret_cast<volatile int*>(a.status);
  const bool give_up = a.empty_on_timeout && (scan_bits & kStatusTimeout);
  if (a.sticky_status && blockIdx.x == 0 && threadIdx.x == 0 && scan_bits) atomicOr(a.sticky_status, scan_bits);

  for (int64_t r = (int64_t)blockIdx.x * wpb + warp; r < a.n_reads; r += (int64_t)gridDim.x * wpb) {
    if (give_up) {
      const int64_t orow = a.out_row ? a.out_row[r] : r;
      for (int e = lane; e < a.k; e += 32) {
        a.out_win[orow * a.k + e] = -1;
        a.out_score[orow * a.k + e] = -INFINITY;
      }
      continue;
    }
    const Candidate* cands = a.cand + (size_t)r * total;
    uint64_t last = ~0ull;
    int n_sel = 0;
    uint64_t my_key = 0;  // entry `lane` of the kept list
    while (n_sel < depth) {
      uint64_t best = 0;
      for (int e = lane; e < total; e += 32) {
        const Candidate c = cands[e];
        if (c.win >= kUnusedWin) continue;  // empty entry, or the mark of an unused slot
        if (cands[e - e % a.cand_depth].win == kUnusedWin) continue;  // rest of an unused slot
        if (c.win >= ix.W) {
          // no scan writes a window past the index: a corrupt slot, never dereferenced
          set_status(a.status, kStatusBadArg);
          set_status(a.sticky_status, kStatusBadArg);
          continue;
        }
        const uint64_t key = cand_key(c.score, c.win);
        if (key < last && key > best) best = key;
      }
      best = warp_max_u64(best);
      if (best == 0) break;
      last = best;
      if (a.sep > 0) {
        const uint32_t w = 0xFFFFFFFFu - (uint32_t)best;
        const int64_t bucket = (int64_t)w * ix.stride / a.sep;
        const uint32_t mine = 0xFFFFFFFFu - (uint32_t)my_key;
        const bool dup = lane < n_sel && (int64_t)mine * ix.stride / a.sep == bucket;
        if (__any_sync(0xffffffffu, dup)) continue;
      }
      if (lane == n_sel) my_key = best;
      ++n_sel;
    }

    if (a.rescore && n_sel > 0) {
      const float* x = a.emb_f32 + (size_t)r * 2 * D;
      const float* nr = a.norms + (size_t)r * (1 + ix.m);
      for (int i = 0; i < n_sel; ++i) {
        const uint64_t key = __shfl_sync(0xffffffffu, my_key, i);
        const uint32_t jw = 0xFFFFFFFFu - (uint32_t)key;
        const int64_t w0 = (int64_t)jw * ix.stride;
        if (ix.win_f32) {
          // materialised index: the window's stored FP32 encoding (§2.1-§2.3
          // sums, built once) against the read's FP32 encoding
          const float* cw = ix.win_f32 + (size_t)jw * 2 * D;
          float re = 0.f, im = 0.f, C = 0.f;
          for (int g = lane; g < D; g += 32) {
            const float xr = x[g], xi = x[D + g];
            const float cr = cw[g], ci = cw[D + g];
            re = fmaf(xr, cr, fmaf(xi, ci, re));
            im = fmaf(xr, ci, fmaf(-xi, cr, im));
            C = fmaf(cr, cr, fmaf(ci, ci, C));
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            re += __shfl_xor_sync(0xffffffffu, re, o);
            im += __shfl_xor_sync(0xffffffffu, im, o);
            C += __shfl_xor_sync(0xffffffffu, C, o);
          }
          const float X = nr[0];
          const float fid = (X > kZeroNorm2 && C > kZeroNorm2) ? fmaf(re, re, im * im) / (X * C) : 0.f;
          if (lane == i) my_key = cand_key(fid, jw);
          __syncwarp();
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
        float fid = 0.f;
        if (ix.score_mode == 0) {
          float re = 0.f, im = 0.f, C = 0.f;
          for (int g = lane; g < D; g += 32) {
            const float xr = x[g], xi = x[D + g];
            const float2 c = acc[g];
            re = fmaf(xr, c.x, fmaf(xi, c.y, re));
            im = fmaf(xr, c.y, fmaf(-xi, c.x, im));
            C = fmaf(c.x, c.x, fmaf(c.y, c.y, C));
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            re += __shfl_xor_sync(0xffffffffu, re, o);
            im += __shfl_xor_sync(0xffffffffu, im, o);
            C += __shfl_xor_sync(0xffffffffu, C, o);
          }
          const float X = nr[0];
          fid = (X > kZeroNorm2 && C > kZeroNorm2) ? fmaf(re, re, im * im) / (X * C) : 0.f;
        } else {
          for (int k = 0; k < ix.m; ++k) {
            float re = 0.f, im = 0.f, C = 0.f;
            for (int b = lane; b < ix.nb; b += 32) {
              const int g = k * ix.nb + b;
              const float xr = x[g], xi = x[D + g];
              const float2 c = acc[g];
              re = fmaf(xr, c.x, fmaf(xi, c.y, re));
              im = fmaf(xr, c.y, fmaf(-xi, c.x, im));
              C = fmaf(c.x, c.x, fmaf(c.y, c.y, C));
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
              re += __shfl_xor_sync(0xffffffffu, re, o);
              im += __shfl_xor_sync(0xffffffffu, im, o);
              C += __shfl_xor_sync(0xffffffffu, C, o);
            }
            const float Xk = nr[1 + k];
            fid += (Xk > kZeroNorm2 && C > kZeroNorm2) ? fmaf(re, re, im * im) / (Xk * C) : 0.f;
          }
          fid /= ix.m;
        }
        if (lane == i) my_key = cand_key(fid, jw);
        __syncwarp();
      }
    }

    // bitonic sort of the kept keys across the warp, descending
#pragma unroll
    for (int k2 = 2; k2 <= 32; k2 <<= 1) {
#pragma unroll
      for (int j2 = k2 >> 1; j2 > 0; j2 >>= 1) {
        const uint64_t other = __shfl_xor_sync(0xffffffffu, my_key, j2);
        const int p = lane ^ j2;
        const bool take_max = (((lane & k2) == 0) == (lane < p));
        my_key = take_max ? (other > my_key ? other : my_key) : (other < my_key ? other : my_key);
      }
    }
    if (lane < a.k) {
      int64_t ow = -1;
      float os = -INFINITY;
      if (lane < n_sel && my_key != 0) {
        ow = (int64_t)(0xFFFFFFFFu - (uint32_t)my_key) * ix.stride;
        os = unord_float((uint32_t)(my_key >> 32));
      }
      const int64_t orow = a.out_row ? a.out_row[r] : r;
      a.out_win[orow * a.k + lane] = ow;
      a.out_score[orow * a.k + lane] = os;
    }
  }
}

cudaError_t launch_merge(const DevIndex& ix, const MergeArgs& a, cudaStream_t st) {
  if (a.n_reads <= 0) return cudaSuccess;
  const int wpb = 8;
  int64_t blocks = (a.n_reads + wpb - 1) / wpb;
  if (blocks > 152 * 32) blocks = 152 * 32;
  const size_t smem = ix.win_f32 ? 0 : (size_t)wpb * ix.D * sizeof(float2);
  merge_kernel<<<(unsigned)blocks, wpb * 32, smem, st>>>(ix, a);
  return cudaGetLastError();
}

}  // namespace rope

namespace rope {

// Two sorted top-k lists per read (forward row r, reverse row n + r, each by
// score descending and start ascending, missing entries (-1, -inf) last)
// merged into one: score descending, the forward strand first on equal
// scores, then the lower start.
__global__ void strand_merge_kernel(const int64_t* __restrict__ win2, const float* __restrict__ score2, int64_t n,
                                    int k, int64_t* __restrict__ out_win, float* __restrict__ out_score,
                                    int8_t* __restrict__ out_strand) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t* wf = win2 + r * k;
    const int64_t* wr = win2 + (n + r) * k;
    const float* sf = score2 + r * k;
    const float* sr = score2 + (n + r) * k;
    int i = 0, j = 0;
    for (int o = 0; o < k; ++o) {
      const bool okf = i < k && wf[i] >= 0, okr = j < k && wr[j] >= 0;
      int8_t strand = -1;
      if (okf && okr) {
        strand = sr[j] > sf[i] ? 1 : 0;  // equal scores: forward first
      } else if (okf) {
        strand = 0;
      } else if (okr) {
        strand = 1;
      }
      int64_t w = -1;
      float sc = -INFINITY;
      if (strand == 0) {
        w = wf[i];
        sc = sf[i++];
      } else if (strand == 1) {
        w = wr[j];
        sc = sr[j++];
      }
      out_win[r * k + o] = w;
      out_score[r * k + o] = sc;
      out_strand[r * k + o] = strand;
    }
  }
}

cudaError_t launch_strand_merge(const int64_t* win2, const float* score2, int64_t n, int k, int64_t* out_win,
                                float* out_score, int8_t* out_strand, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int64_t blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  strand_merge_kernel<<<(unsigned)blocks, 256, 0, st>>>(win2, score2, n, k, out_win, out_score, out_strand);
  return cudaGetLastError();
}

}  // namespace rope
