// Refinement (§3.4, increasing the accuracy): around a candidate start found
// at a coarse window stride, the window is slid one letter at a time and each
// position is scored against the read head, typically with a richer encoding
// (up to 4^8 bins per band) than the scan's.
//
// The per-step update is the paper's inner-product recurrence written in the
// frame of the first position p0 of the range: with S_{k,b} = sum over the
// window's locations d (absolute offset from p0) whose s-mer falls in bin b of
// w_k^d (w_k = e^{2 pi i f_k / N}), the window's encoding is
// c_{k,b}(p) = w_k^{-(p-p0)} S_{k,b}, so
//   ip_k(p) = w_k^{-(p-p0)} J_k,   J_k = sum_b conj(x_{k,b}) S_{k,b},
//   C_k(p)  = sum_b |S_{k,b}|^2.
// Sliding by one letter removes location d = p-p0 from its bin and adds
// d + N-s+1 to another: J_k and C_k change by O(m) terms (the leaving and
// entering s-mers only), and no entry is rotated, so no rounding drift builds
// up in the rotated entries. The window norm is tracked exactly (every bin's
// S kept in a hash table), not skipped.
//
// One block per read: warp 0 builds the read's sparse encoding (bins it
// touches, x_{k,b} summed in location order) in a shared hash table; each warp
// then takes candidates in turn: the bins and phases of its range are computed
// by all lanes, the window hash table is filled and slid by lane 0 (the steps
// are sequential), and the best position (ties: the lower) is written.
#include <cuda_runtime.h>

#include "rope_internal.h"

namespace rope {

constexpr int kRefMaxBands = 8;
constexpr int32_t kEmptyKey = -1;

struct RefineArgs {
  EncTables tb;                  // map [4^s] (first letter most significant), read-frame phases [m * n_loc]
  int64_t a[kRefMaxBands];       // f_k = a_k / q
  int64_t Q;                     // q * N
  int32_t score_mode;
  const uint32_t* packed;        // 2-bit packed reference
  int64_t L;
  const uint8_t* seqs;
  const int64_t* offsets;
  int64_t n_reads;
  const int64_t* cand;           // [n_reads, n_cand]
  int32_t n_cand, radius;
  int64_t* out_pos;              // [n_reads, n_cand]
  float* out_fid;
  int* status;
  int32_t cap_r_log2, cap_w_log2;  // hash table capacities (powers of two)
  int32_t n_w_max;                 // window locations of the longest range: 2*radius + N-s+1
  uint32_t warp_bytes;             // shared memory per warp
};

__device__ __forceinline__ uint32_t ref_hash(int32_t key, int cap_log2) {
  return ((uint32_t)key * 0x9E3779B1u) >> (32 - cap_log2);
}

// slot of key (inserted, zero-valued, if absent); the table never fills: its
// capacity is at least twice the number of keys a read or a range can hold
__device__ __forceinline__ int table_slot(int32_t* keys, float2* vals, int m, int cap_log2, int32_t key) {
  const uint32_t mask = (1u << cap_log2) - 1u;
  uint32_t h = ref_hash(key, cap_log2);
  while (true) {
    const int32_t k = keys[h];
    if (k == key) return (int)h;
    if (k == kEmptyKey) {
      keys[h] = key;
      for (int b = 0; b < m; ++b) vals[h * m + b] = make_float2(0.f, 0.f);
      return (int)h;
    }
    h = (h + 1u) & mask;
  }
}

// slot of key, or -1
__device__ __forceinline__ int table_find(const int32_t* keys, int cap_log2, int32_t key) {
  const uint32_t mask = (1u << cap_log2) - 1u;
  uint32_t h = ref_hash(key, cap_log2);
  while (true) {
    const int32_t k = keys[h];
    if (k == key) return (int)h;
    if (k == kEmptyKey) return -1;
    h = (h + 1u) & mask;
  }
}

// e^{2 pi i a d / Q} with the exponent reduced in integers, rounded to FP32
__device__ __forceinline__ float2 ref_unit(int64_t a, int64_t Q, int64_t d) {
  int64_t r = (a * d) % Q;
  if (r < 0) r += Q;
  double sn, cs;
  sincospi(2.0 * (double)r / (double)Q, &sn, &cs);
  return make_float2((float)cs, (float)sn);
}

__device__ __forceinline__ uint32_t packed_letter(const uint32_t* __restrict__ packed, int64_t pos) {
  return (__ldg(packed + (pos >> 4)) >> ((pos & 15) * 2)) & 3u;
}

__global__ void refine_kernel(RefineArgs a) {
  extern __shared__ __align__(16) uint8_t ref_smem[];
  const int m = a.tb.m, N = a.tb.N, s = a.tb.s;
  const int n_loc = N - s + 1;
  const int cap_r = 1 << a.cap_r_log2, cap_w = 1 << a.cap_w_log2;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int64_t r = blockIdx.x;

  // block: read table [keys cap_r | vals cap_r*m], read bins [n_loc], X_k [m], flag
  int32_t* rkeys = reinterpret_cast<int32_t*>(ref_smem);
  float2* rvals = reinterpret_cast<float2*>(rkeys + cap_r);
  int32_t* rbins = reinterpret_cast<int32_t*>(rvals + (size_t)cap_r * m);
  float* xnorm = reinterpret_cast<float*>(rbins + n_loc);  // [m] per band, then the total
  int* ok_s = reinterpret_cast<int*>(xnorm + kRefMaxBands + 1);
  uint8_t* warp_base = ref_smem + (((size_t)cap_r * (4 + 8 * m) + (size_t)n_loc * 4 + 4 * (kRefMaxBands + 2) + 15) & ~size_t(15));

  const int64_t start = a.offsets[r];
  const int64_t len = a.offsets[r + 1] - start;
  const uint8_t* seq = a.seqs + start;
  if (threadIdx.x == 0) *ok_s = 1;
  __syncthreads();
  if (len < N) {
    if (threadIdx.x == 0) {
      set_status(a.status, kStatusShortRead);
      *ok_s = 0;
    }
  } else {
    for (int l = threadIdx.x; l < n_loc; l += blockDim.x) {
      uint32_t code = 0;
      bool bad = false;
      for (int i = 0; i < s; ++i) {
        const uint32_t c = letter_code(seq[l + i]);
        bad |= c > 3;
        code = code * 4u + (c & 3u);
      }
      if (bad) {
        set_status(a.status, kStatusBadBase);
        *ok_s = 0;
      }
      rbins[l] = a.tb.map[code];
    }
    for (int i = threadIdx.x; i < cap_r; i += blockDim.x) rkeys[i] = kEmptyKey;
  }
  __syncthreads();
  const bool ok = *ok_s != 0;
  if (ok && threadIdx.x == 0) {
    // x_{k,b}: each bin's phases summed in location order
    for (int l = 0; l < n_loc; ++l) {
      const int h = table_slot(rkeys, rvals, m, a.cap_r_log2, rbins[l]);
      for (int k = 0; k < m; ++k) {
        const float2 ph = a.tb.phase[(size_t)k * n_loc + l];
        rvals[h * m + k].x += ph.x;
        rvals[h * m + k].y += ph.y;
      }
    }
    float tot = 0.f;
    for (int k = 0; k < m; ++k) {
      float xk = 0.f;
      for (int h = 0; h < cap_r; ++h)
        if (rkeys[h] != kEmptyKey) xk = fmaf(rvals[h * m + k].x, rvals[h * m + k].x, fmaf(rvals[h * m + k].y, rvals[h * m + k].y, xk));
      xnorm[k] = xk;
      tot += xk;
    }
    xnorm[kRefMaxBands] = tot;
  }
  __syncthreads();

  // warp: window table [keys cap_w | vals cap_w*m], bins [n_w_max], phases [n_w_max*m]
  uint8_t* wb = warp_base + (size_t)warp * a.warp_bytes;
  int32_t* wkeys = reinterpret_cast<int32_t*>(wb);
  float2* wvals = reinterpret_cast<float2*>(wkeys + cap_w);
  int32_t* wbins = reinterpret_cast<int32_t*>(wvals + (size_t)cap_w * m);
  float2* wph = reinterpret_cast<float2*>(((uintptr_t)(wbins + a.n_w_max) + 7) & ~uintptr_t(7));
  const int64_t last = a.L - N;  // last window start

  for (int c = warp; c < a.n_cand; c += nwarps) {
    const size_t o = (size_t)r * a.n_cand + c;
    const int64_t pos = a.cand[o];
    if (!ok || pos < 0 || last < 0) {
      if (lane == 0) {
        a.out_pos[o] = -1;
        a.out_fid[o] = -INFINITY;
      }
      continue;
    }
    const int64_t cpos = pos < last ? pos : last;
    const int64_t p0 = cpos - a.radius > 0 ? cpos - a.radius : 0;
    const int64_t p1 = cpos + a.radius < last ? cpos + a.radius : last;
    const int n_steps = (int)(p1 - p0);
    const int n_w = n_steps + n_loc;
    for (int d = lane; d < n_w; d += 32) {
      uint32_t code = 0;
      for (int i = 0; i < s; ++i) code = code * 4u + packed_letter(a.packed, p0 + d + i);
      wbins[d] = a.tb.map[code];
      for (int k = 0; k < m; ++k) wph[(size_t)d * m + k] = ref_unit(a.a[k], a.Q, d);
    }
    for (int i = lane; i < cap_w; i += 32) wkeys[i] = kEmptyKey;
    __syncwarp();
    if (lane == 0) {
      double Jr[kRefMaxBands], Ji[kRefMaxBands], C[kRefMaxBands];
      for (int k = 0; k < m; ++k) Jr[k] = Ji[k] = C[k] = 0.0;
      // location d of the window enters (sgn = +1) or leaves (sgn = -1) its bin
      auto move = [&](int d, float sgn) {
        const int32_t b = wbins[d];
        const int h = table_slot(wkeys, wvals, m, a.cap_w_log2, b);
        const int hx = table_find(rkeys, a.cap_r_log2, b);
        for (int k = 0; k < m; ++k) {
          const float2 ph = wph[(size_t)d * m + k];
          const float2 old = wvals[h * m + k];
          const float2 nw = make_float2(old.x + sgn * ph.x, old.y + sgn * ph.y);
          wvals[h * m + k] = nw;
          C[k] += ((double)nw.x * nw.x + (double)nw.y * nw.y) - ((double)old.x * old.x + (double)old.y * old.y);
          if (hx >= 0) {
            // conj(x) * (sgn * ph)
            const float2 x = rvals[hx * m + k];
            Jr[k] += sgn * ((double)x.x * ph.x + (double)x.y * ph.y);
            Ji[k] += sgn * ((double)x.x * ph.y - (double)x.y * ph.x);
          }
        }
      };
      auto fid_at = [&](int i) -> double {
        if (a.score_mode == 0) {
          double ir = 0.0, ii = 0.0, ct = 0.0;
          for (int k = 0; k < m; ++k) {
            // ip_k = conj(w_k^i) J_k
            const float2 ph = wph[(size_t)i * m + k];
            ir += (double)ph.x * Jr[k] + (double)ph.y * Ji[k];
            ii += (double)ph.x * Ji[k] - (double)ph.y * Jr[k];
            ct += C[k];
          }
          const double den = (double)xnorm[kRefMaxBands] * ct;
          return den > (double)kZeroNorm2 ? (ir * ir + ii * ii) / den : 0.0;
        }
        double f = 0.0;
        for (int k = 0; k < m; ++k) {
          const double den = (double)xnorm[k] * C[k];
          if (den > (double)kZeroNorm2) f += (Jr[k] * Jr[k] + Ji[k] * Ji[k]) / den;
        }
        return f / m;
      };
      for (int d = 0; d < n_loc; ++d) move(d, 1.f);
      double best = fid_at(0);
      int best_i = 0;
      for (int i = 1; i <= n_steps; ++i) {
        move(i - 1, -1.f);
        move(i - 1 + n_loc, 1.f);
        const double f = fid_at(i);
        if (f > best) {
          best = f;
          best_i = i;
        }
      }
      a.out_pos[o] = p0 + best_i;
      a.out_fid[o] = (float)best;
    }
    __syncwarp();
  }
}

// shared memory of a block with `warps` warps
static size_t refine_smem(const RefineArgs& a, int warps) {
  const int m = a.tb.m, n_loc = a.tb.N - a.tb.s + 1;
  const size_t block = (((size_t)(1 << a.cap_r_log2) * (4 + 8 * m) + (size_t)n_loc * 4 + 4 * (kRefMaxBands + 2) + 15) &
                        ~size_t(15));
  return block + (size_t)warps * a.warp_bytes;
}

static int ceil_log2(int64_t v) {
  int r = 0;
  while ((int64_t(1) << r) < v) ++r;
  return r;
}

cudaError_t launch_refine(RefineArgs a, int max_warps, cudaStream_t st) {
  if (a.n_reads <= 0 || a.n_cand <= 0) return cudaSuccess;
  const int m = a.tb.m, n_loc = a.tb.N - a.tb.s + 1;
  a.n_w_max = 2 * a.radius + n_loc;
  a.cap_r_log2 = ceil_log2(2 * (int64_t)n_loc) < 5 ? 5 : ceil_log2(2 * (int64_t)n_loc);
  a.cap_w_log2 = ceil_log2(2 * (int64_t)a.n_w_max) < 5 ? 5 : ceil_log2(2 * (int64_t)a.n_w_max);
  const size_t wbytes = (size_t)(1 << a.cap_w_log2) * (4 + 8 * m) + (size_t)a.n_w_max * 4 + 8 +
                        (size_t)a.n_w_max * m * 8;
  a.warp_bytes = (uint32_t)((wbytes + 15) & ~size_t(15));
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  int warps = a.n_cand < max_warps ? a.n_cand : max_warps;
  while (warps > 1 && refine_smem(a, warps) > (size_t)optin) --warps;
  const size_t smem = refine_smem(a, warps);
  if (smem > (size_t)optin) return cudaErrorInvalidValue;
  e = cudaFuncSetAttribute(refine_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  refine_kernel<<<(unsigned)a.n_reads, warps * 32, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace rope

// ---------------------------------------------------------------- C ABI

#include "rope_host.h"

extern "C" rope_status rope_refine(const rope_index* idx, const rope_params* p, const uint8_t* seqs,
                                   const int64_t* offsets, int64_t n_reads, const int64_t* cand_pos, int32_t n_cand,
                                   int32_t radius, int64_t* out_pos, float* out_fid, cudaStream_t stream) {
  using namespace rope;
  if (!idx) return host_fail(ROPE_ERR_INVALID_ARG, "index is NULL");
  if (n_reads < 0 || n_reads > 0x7FFFFFFFLL) return host_fail(ROPE_ERR_INVALID_ARG, "n_reads outside [0, 2^31)");
  if (n_cand < 1 || n_cand > 64) return host_fail(ROPE_ERR_INVALID_ARG, "n_cand=%d outside [1,64]", n_cand);
  if (radius < 0 || radius > 4096) return host_fail(ROPE_ERR_INVALID_ARG, "radius=%d outside [0,4096]", radius);
  if (n_reads == 0) return ROPE_OK;
  if (!seqs || !offsets || !cand_pos || !out_pos || !out_fid) return host_fail(ROPE_ERR_INVALID_ARG, "NULL pointer");
  RefineArgs a{};
  rope_status st = host_refine_tables(p, &a.tb);
  if (st != ROPE_OK) return st;
  if (p->window_len > idx->ix.L) return host_fail(ROPE_ERR_INVALID_ARG, "window_len beyond the reference");
  DeviceCtx* c;
  if ((st = host_ctx(&c)) != ROPE_OK) return st;
  for (int k = 1; k <= p->m; ++k) {
    int64_t q;
    host_factor(p, k, &a.a[k - 1], &q);
    a.Q = q * p->window_len;
  }
  a.score_mode = p->score_mode;
  a.packed = idx->ix.packed;
  a.L = idx->ix.L;
  a.seqs = seqs;
  a.offsets = offsets;
  a.n_reads = n_reads;
  a.cand = cand_pos;
  a.n_cand = n_cand;
  a.radius = radius;
  a.out_pos = out_pos;
  a.out_fid = out_fid;
  a.status = c->status;
  const cudaError_t e = launch_refine(a, 8, stream);
  if (e == cudaErrorInvalidValue)
    return host_fail(ROPE_ERR_UNSUPPORTED, "refinement tables for N=%d, m=%d, radius=%d exceed shared memory",
                     p->window_len, p->m, radius);
  if (e != cudaSuccess) return host_fail(ROPE_ERR_CUDA, "refine launch: %s", cudaGetErrorString(e));
  return ROPE_OK;
}
