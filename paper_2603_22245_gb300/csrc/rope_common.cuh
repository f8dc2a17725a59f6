// Shared device-side definitions of the RotorMap GB300 library.
//
// The device view of a reference index (DevIndex), the status word that kernels
// report errors through, bounded waits, the s-mer bin lookup on packed words,
// the window generator (the slide-by-one recurrence of §3.4) and thin inline
// PTX wrappers for mbarrier, bulk copies and tcgen05.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace rope {

// Bits of the device status word (OR-ed by kernels, read by rope_sync_status).
enum : int {
  kStatusBadBase = 1,     // letter outside {A,C,G,T,a,c,g,t}
  kStatusShortRead = 2,   // read shorter than N
  kStatusTimeout = 4,     // a bounded wait ran out
  kStatusBadArg = 8,      // a kernel saw an out-of-range argument
};

constexpr int kAnchorPeriod = 64;  // windows between exact anchors
constexpr int kMaxScanDim = 128;   // largest complex dimension the scans take
constexpr int kPackPadWords = 64;  // zero words after the packed reference
// A vector whose squared norm is at most this is the zero vector (§3.3: evenly
// spaced unit phases sum to zero exactly; rounding leaves ~1e-28 in FP64 and
// ~1e-12 in FP32, while a nonzero encoding has a squared norm of order N).
// Its fidelity with anything is 0.
constexpr float kZeroNorm2 = 1e-6f;

// Device view of a reference index. All pointers are device pointers.
struct DevIndex {
  const uint32_t* packed;  // 2-bit letters, + kPackPadWords zero words
  int64_t L;               // letters
  int64_t W;               // windows
  int32_t N, s, m, t, nb, D, stride, A;
  int32_t variant, score_mode;
  const float* inv_norm;    // [W] 1/sqrt(|c_j|^2), 0 for a zero vector
  const float* band_norm;   // [W*m] |c_j,k|^2 (score_mode 1), else null
  const float2* anchors;    // [ceil(W/A) * D] c(a*A) in FP32
  const uint16_t* map_lsb;  // [4^s] bin of the little-endian 2s-bit letter field
  const float2* phase;      // [m * (N-s+1)] exp(2 pi i f_k loc / N)
  const float2* rot;        // [m] exp(-2 pi i f_k stride / N)
  const float2* eout;       // [m * stride] exp(2 pi i f_k j / N), j < stride
  const float2* ein;        // [m * stride] exp(2 pi i f_k (N-s+1+j) / N), j < stride
  // materialised index (the window matrix of §3.1; null for the on-the-fly index)
  const float* win_f32;     // [W, 2D] unnormalised [cr | ci]
  const uint16_t* win_bf16; // [W, 2D] BF16 [cr | ci] / |c|
};

// ---------------------------------------------------------------- status

__device__ __forceinline__ void set_status(int* status, int bits) {
  if (status) atomicOr(status, bits);
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s per wait

// ---------------------------------------------------------------- SplitMix64

// Output i (0-based) of the SplitMix64 generator started at `seed` (Steele,
// Lea and Flood, 2014): the state advances by the golden-ratio increment and
// each output is the state passed through the published 64-bit finaliser.
__device__ __forceinline__ uint64_t sm64_out(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
// the top 53 bits as a double in [0, 1)
__device__ __forceinline__ double sm64_unit(uint64_t z) { return (double)(z >> 11) * (1.0 / 9007199254740992.0); }

// ---------------------------------------------------------------- letters

// A,C,G,T (either case) -> 0..3, else 4
__device__ __forceinline__ uint32_t letter_code(uint32_t c) {
  c |= 0x20u;  // lower case
  return c == 'a' ? 0u : c == 'c' ? 1u : c == 'g' ? 2u : c == 't' ? 3u : 4u;
}

// bin of the s-mer at position p, read from 2-bit packed words
__device__ __forceinline__ uint32_t bin_at(const uint32_t* __restrict__ packed, int64_t p, int s,
                                           const uint16_t* __restrict__ map_lsb) {
  const int64_t wi = p >> 4;
  const int sh = (int)(p & 15) * 2;
  const uint64_t v = ((uint64_t)__ldg(packed + wi + 1) << 32) | __ldg(packed + wi);
  const uint32_t field = (uint32_t)(v >> sh) & ((1u << (2 * s)) - 1u);
  return __ldg(map_lsb + field);
}

// ---------------------------------------------------------------- generator

// One chain of the window generator: lanes hold the D complex entries of c(j),
// BPL consecutive entries per lane (entries BPL*l .. BPL*l+BPL-1 of lane l, all
// in one band since 4^t is a multiple of BPL). A step moves c(j) to c(j+1) by
// the slide relations of §3.4, for stride S:
//   c_b <- c_b - sum_{i<S} [bin(w+i) = b] e^{2 pi i f i/N}
//   c_b <- c_b + sum_{i<S} [bin(w+N-s+1+i) = b] e^{2 pi i f (N-s+1+i)/N}
//   c   <- c * e^{-2 pi i f S/N}
// (for S = 1 these are exactly the paper's relations: every entry rotates by
// w^{-f}, the leaving s-mer loses w^{-f}, the entering one gains w^{f(N-s)}).
template <int BPL>
struct ChainB {
  float cr[BPL], ci[BPL];
  int band;   // band k-1 of this lane's entries
  int b0;     // bin of entry 0 of this lane
  float rc, rs;  // rotation e^{-2 pi i f S / N}
  float ec, es;  // stride-1 entering phase e^{2 pi i f (N-s+1) / N}

  __device__ __forceinline__ void setup(const DevIndex& ix, int lane_in_chain) {
    const int g0 = BPL * lane_in_chain;
    band = g0 / ix.nb;
    b0 = g0 - band * ix.nb;
    const float2 r = ix.rot[band];
    rc = r.x;
    rs = r.y;
    const float2 e = ix.ein[band * ix.stride];
    ec = e.x;
    es = e.y;
  }

  __device__ __forceinline__ void load(const float2* __restrict__ anchor, int lane_in_chain) {
#pragma unroll
    for (int i = 0; i < BPL; ++i) {
      const float2 v = anchor[BPL * lane_in_chain + i];
      cr[i] = v.x;
      ci[i] = v.y;
    }
  }

  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int i = 0; i < BPL; ++i) cr[i] = ci[i] = 0.f;
  }

  __device__ __forceinline__ void rotate() {
#pragma unroll
    for (int i = 0; i < BPL; ++i) {
      const float xr = cr[i], xi = ci[i];
      cr[i] = fmaf(xr, rc, -xi * rs);
      ci[i] = fmaf(xr, rs, xi * rc);
    }
  }

  // stride 1: bout = bin leaving at the start, bin_in = bin entering at the end
  __device__ __forceinline__ void step1(uint32_t bout, uint32_t bin_in) {
#pragma unroll
    for (int i = 0; i < BPL; ++i) {
      if ((uint32_t)(b0 + i) == bout) cr[i] -= 1.0f;
      if ((uint32_t)(b0 + i) == bin_in) {
        cr[i] += ec;
        ci[i] += es;
      }
    }
    rotate();
  }

  // general stride: one leaving (sub_at) or entering (add_at) location
  __device__ __forceinline__ void sub_at(uint32_t b, float2 v) {
#pragma unroll
    for (int i = 0; i < BPL; ++i)
      if ((uint32_t)(b0 + i) == b) {
        cr[i] -= v.x;
        ci[i] -= v.y;
      }
  }
  __device__ __forceinline__ void add_at(uint32_t b, float2 v) {
#pragma unroll
    for (int i = 0; i < BPL; ++i)
      if ((uint32_t)(b0 + i) == b) {
        cr[i] += v.x;
        ci[i] += v.y;
      }
  }
};

// Chains of D/4 lanes, four entries per lane (FP32 scan, window inspection).
template <int D>
struct Chain : ChainB<4> {
  static constexpr int LPC = D / 4;
};

// ---------------------------------------------------------------- packed FP32 pairs

// (re0^2 + im0^2, re1^2 + im1^2) with the FP32x2 instructions of sm_100+: one
// packed multiply and one packed fma for two scores, each lane of the pair
// rounded exactly as fmaf(re, re, im * im).
__device__ __forceinline__ void abs2_pair(uint32_t re0, uint32_t re1, uint32_t im0, uint32_t im1, float& s0,
                                          float& s1) {
  uint64_t re, im, r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(re) : "r"(re0), "r"(re1));
  asm("mov.b64 %0, {%1, %2};" : "=l"(im) : "r"(im0), "r"(im1));
  asm("mul.rn.f32x2 %0, %1, %1;" : "=l"(r) : "l"(im));
  asm("fma.rn.f32x2 %0, %1, %1, %2;" : "=l"(r) : "l"(re), "l"(r));
  asm("mov.b64 {%0, %1}, %2;" : "=f"(s0), "=f"(s1) : "l"(r));
}

// ---------------------------------------------------------------- PTX: mbarrier

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// try_wait that may park the thread until the phase completes or about
// kSuspendHintNs pass, so a waiting warp takes no issue slots from the warps
// doing the work.
constexpr uint32_t kSuspendHintNs = 200000;
__device__ __forceinline__ bool mbar_try_wait_suspend(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "n"(kSuspendHintNs)
      : "memory");
  return ok != 0;
}

// Bounded wait on a phase parity. Returns false (and sets the timeout bit and
// the block's abort flag) if the phase did not complete within limit_ns, or
// if another role of the block has already aborted. Limits shorter than the
// suspend hint poll without suspending, so that a short limit is kept.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int* status,
                                          uint64_t limit_ns = kWaitLimitNs) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  const bool suspend = limit_ns >= 4ull * kSuspendHintNs;
  for (;;) {
    if (suspend ? mbar_try_wait_suspend(bar, parity) : mbar_try_wait(bar, parity)) return true;
    if (*abort_flag) return false;
    if (globaltimer_ns() - t0 > limit_ns) {
      *abort_flag = 1;
      set_status(status, kStatusTimeout);
      return false;
    }
  }
}

// Bound of a drain wait: at least one second, whatever the ordinary limit.
constexpr uint64_t kDrainLimitNs = 1000000000ull;

// Wait for this block's own asynchronous work in flight (bulk copies, MMAs)
// before it frees tensor memory and exits: unlike mbar_wait it does not give
// up when the block has aborted, only when max(limit_ns, kDrainLimitNs) has
// passed (then it sets the timeout bit and returns false).
__device__ __forceinline__ bool mbar_drain_wait(uint64_t* bar, uint32_t parity, int* status, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t lim = limit_ns > kDrainLimitNs ? limit_ns : kDrainLimitNs;
  const uint64_t t0 = globaltimer_ns();
  for (;;) {
    if (mbar_try_wait_suspend(bar, parity)) return true;
    if (globaltimer_ns() - t0 > lim) {
      set_status(status, kStatusTimeout);
      return false;
    }
  }
}

// Warp-uniform bounded wait: every lane waits, then the warp agrees (and
// reconverges) before any .sync.aligned instruction that follows.
__device__ __forceinline__ bool mbar_wait_warp(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                               int* status, uint64_t limit_ns = kWaitLimitNs) {
  const bool ok = mbar_wait(bar, parity, abort_flag, status, limit_ns);
  return __all_sync(0xffffffffu, ok);
}

// ---------------------------------------------------------------- PTX: bulk copy

// 1-D bulk copy global -> shared, completion signalled on `bar` (tx bytes).
// Both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst_smem, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst_smem)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// 2-D tiled tensor copy global -> shared (TMA), completion signalled on `bar`
// (tx bytes = the whole box, out-of-bounds elements filled with zero). x is the
// innermost coordinate in elements (x * element size a multiple of 16 bytes),
// y the row; dst 1024-byte aligned for the 128-byte swizzle.
__device__ __forceinline__ void tma_load_2d(void* dst_smem, const void* tensor_map, int32_t x, int32_t y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(smem_u32(dst_smem)),
      "l"(tensor_map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void prefetch_tensor_map(const void* tensor_map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(tensor_map) : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void fence_barrier_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// ---------------------------------------------------------------- PTX: tcgen05

__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D[tmem] (+)= A[tmem] * B[smem desc], kind::f16 (BF16 inputs, FP32 accumulate)
__device__ __forceinline__ void tc_mma_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}" ::"r"(d_tmem),
      "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// D[tmem] (+)= A[smem desc] * B[smem desc], kind::f16 (BF16 inputs, FP32 accumulate)
__device__ __forceinline__ void tc_mma_ss(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// D[tmem] (+)= A[smem desc] * B[smem desc], kind::f8f6f4 (8-bit inputs given
// by the instruction descriptor, FP32 accumulate; K = 32 per instruction)
__device__ __forceinline__ void tc_mma_ss_f8(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                             uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// arrive on `bar` once all prior tcgen05 async ops of this thread complete
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tc_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Orders the use of registers written by tcgen05.ld after tcgen05.wait::ld:
// an empty volatile asm that reads and writes each register.
template <int N>
__device__ __forceinline__ void reg_fence(uint32_t (&r)[N]) {
#pragma unroll
  for (int i = 0; i < N; ++i) asm volatile("" : "+r"(r[i]));
}

// 32 lanes x 16 consecutive 32-bit columns -> 16 registers per thread
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

// 32 lanes x 8 consecutive 32-bit columns from 8 registers per thread
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&r)[8]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr), "r"(r[0]), "r"(r[1]),
      "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
      : "memory");
}

// Shared-memory matrix descriptor (tcgen05): K-major, 128-byte swizzle, rows of
// 128 bytes in 8-row (1024-byte) groups. Start address and group stride in
// 16-byte units; bits 46-47 hold the descriptor version (1), bits 61-63 the
// layout (2 = 128-byte swizzle).
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;                 // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;       // stride byte offset: next 8-row group
  d |= (uint64_t)1 << 46;                 // version
  d |= (uint64_t)2 << 61;                 // 128-byte swizzle
  return d;
}

// Same for a 64-byte swizzle: rows of 64 bytes in 8-row (512-byte) groups,
// layout code 4.
__device__ __forceinline__ uint64_t smem_desc_sw64(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;                 // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(512 >> 4) << 32;        // stride byte offset: next 8-row group
  d |= (uint64_t)1 << 46;                 // version
  d |= (uint64_t)4 << 61;                 // 64-byte swizzle
  return d;
}

// Instruction descriptor, kind::f8f6f4: E4M3 A and B (format code 0, K-major),
// FP32 D, shape M x N.
__host__ __device__ constexpr uint32_t idesc_e4m3_f32(int M, int N) {
  return (1u << 4)                       // D format FP32
         | ((uint32_t)(N >> 3) << 17)    // N / 8
         | ((uint32_t)(M >> 4) << 24);   // M / 16
}

// Instruction descriptor, kind::f16: BF16 A and B (K-major), FP32 D, shape M x N.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
  return (1u << 4)                       // D format FP32
         | (1u << 7)                     // A format BF16
         | (1u << 10)                    // B format BF16
         | ((uint32_t)(N >> 3) << 17)    // N / 8
         | ((uint32_t)(M >> 4) << 24);   // M / 16
}

// byte offset of (row r, byte o of the 128-byte row) in a 128-byte-swizzled
// K-major tile: 16-byte chunk index XOR (row mod 8), 8-row groups 1024 B apart
__host__ __device__ __forceinline__ uint32_t sw128_offset(uint32_t r, uint32_t o) {
  return (r >> 3) * 1024u + (r & 7u) * 128u + ((((o >> 4) ^ (r & 7u)) & 7u) << 4) + (o & 15u);
}

// byte offset of (row r, byte o of the 64-byte row) in a 64-byte-swizzled
// K-major tile: 16-byte chunk index XOR ((row / 2) mod 4), 8-row groups 512 B apart
__host__ __device__ __forceinline__ uint32_t sw64_offset(uint32_t r, uint32_t o) {
  return (r >> 3) * 512u + (r & 7u) * 64u + ((((o >> 4) ^ (r >> 1)) & 3u) << 4) + (o & 15u);
}

}  // namespace rope
