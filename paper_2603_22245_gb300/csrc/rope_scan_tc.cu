// Tensor-core scan (BF16 in, FP32 accumulate) on sm_103a with tcgen05.
//
// The fidelity of a read x against a window c is |<x|c>|^2 for normalised
// vectors (§2.4); with x = xr + i xi and c = cr + i ci, Re<x|c> = xr.cr + xi.ci
// and Im<x|c> = xr.ci - xi.cr (the real identity of §4). Per block (one per SM):
//   * A operand (shared memory, 128-byte swizzled K-major): NT tiles of 128
//     reads, row = the read's normalised [xr | xi] in BF16 (K = 2D), written
//     once per work item by the epilogue warps.
//   * B operand (shared memory, same layout): per stage T windows as 2T rows,
//     row n = [cr | ci] and row T+n = [ci | -cr] of window n. The generator
//     warps produce them: each chain of LPC lanes runs the §3.4 recurrence from
//     an exact anchor through 64 consecutive windows and emits one window per
//     stage, scaled by the stored 1/sqrt(C_j) and rounded to BF16.
//   * D (tensor memory): per stage and tile a 128 x 2T FP32 accumulator whose
//     columns are Re (0..T-1) and Im (T..2T-1).
//   * One thread issues tcgen05.mma (M = 128, N = 2T = 128, K = 16 per
//     instruction; an MMA costs at least ~45 cycles whatever N is, so N = 128
//     keeps the tensor pipe saturated) and commits to mbarriers; a producer
//     warp streams the 2-bit packed reference of each super-tile into shared
//     memory with bulk copies (TMA); epilogue warps (thread = read; HALVES
//     warps split an accumulator's windows) load the accumulators with
//     tcgen05.ld in 16-column chunks, form Re^2 + Im^2 and keep the read's best
//     windows in a list per (read, half).
// Every wait is bounded; a wait that runs out sets the timeout status bit and
// the block drains its in-flight copies and MMAs, frees tensor memory and exits.
#include <cuda_bf16.h>

#include "rope_internal.h"
#include "rope_topk.cuh"

namespace rope {

// Scale of both operands in the E4M3 scan (a power of two, so exact): the
// normalised entries (|.| <= 1, typically 1/sqrt(2D)) land in [2^-6, 448],
// the normal range of E4M3, except for entries near 0.
constexpr float kFp8Scale = 32.f;

template <int D_, int NT_, int T_, int STAGES_, int NB_, int LPC_, int HALVES_, bool ISOLATE_MMA_, bool FP8_ = false>
struct TcShape {
  static constexpr int D = D_, NT = NT_, T = T_, STAGES = STAGES_, NB = NB_;  // NB: most B ring slots
  static constexpr int A = kAnchorPeriod;
  static constexpr int LPC = LPC_;               // lanes per chain
  static constexpr int BPL = D / LPC;            // complex entries per generator lane
  static constexpr int CPW = 32 / LPC;           // chains per warp
  static constexpr int GEN_WARPS = T / CPW;
  static constexpr int HALVES = HALVES_;         // epilogue warps sharing one accumulator's columns
  static constexpr int WPH = T / HALVES;         // windows per epilogue warp per stage
  static constexpr int EPI_WARPS = 4 * NT * HALVES;
  static constexpr int EPI_THREADS = 32 * EPI_WARPS;
  static constexpr int WARP_MMA = EPI_WARPS;      // on scheduler 0 (EPI_WARPS is a multiple of 4)
  static constexpr int WARP_PROD = EPI_WARPS + 1;
  static constexpr int WARP_GEN0 = EPI_WARPS + 2;
  // With ISOLATE_MMA the warps after the producer whose number is a multiple
  // of 4 stay idle, so that the single MMA-issuing thread shares scheduler 0
  // with the epilogue warps only and gets its instructions issued promptly.
  static constexpr bool ISOLATE_MMA = ISOLATE_MMA_;
  __host__ __device__ static constexpr int idle_before(int w) { return ISOLATE_MMA ? (w - 1) / 4 - (WARP_GEN0 - 1) / 4 : 0; }
  __host__ __device__ static constexpr int nwarps_for(int w) { return (w - WARP_GEN0) - idle_before(w) >= GEN_WARPS ? w : nwarps_for(w + 1); }
  static constexpr int NWARPS = nwarps_for(WARP_GEN0);
  static constexpr int NTHREADS = 32 * NWARPS;
  static constexpr int SUP = T * A;                   // windows per super-tile
  static constexpr int GROUP = NT * 128;              // reads per work item
  // operands: BF16, or E4M3 scaled by kFp8Scale (scores then carry kFp8Scale^4)
  static constexpr bool FP8 = FP8_;
  static constexpr int EB = FP8 ? 1 : 2;               // bytes per operand element
  static constexpr int ROW_BYTES = 2 * D * EB;         // one operand row, K = 2D
  static constexpr int KBLK = ROW_BYTES < 128 ? ROW_BYTES : 128;  // swizzle row: 64 or 128 bytes
  static constexpr int KSTEPS = ROW_BYTES / 32;        // 32 bytes of K per MMA (16 BF16 or 32 E4M3)
  static constexpr int STEPS_PER_KBLK = KBLK / 32;
  static constexpr int KBLOCKS = ROW_BYTES / KBLK;     // swizzled K blocks per row
  static constexpr int A_KBLK_BYTES = 128 * KBLK;      // one K block of an A tile
  static constexpr int A_TILE_BYTES = KBLOCKS * A_KBLK_BYTES;
  static constexpr int B_KBLK_BYTES = 2 * T * KBLK;    // one K block of a B tile
  static constexpr int B_SLOT_BYTES = KBLOCKS * B_KBLK_BYTES;
  static constexpr int TMEM_COLS = 512;
  static constexpr uint32_t IDESC = FP8 ? idesc_e4m3_f32(128, 2 * T) : idesc_bf16_f32(128, 2 * T);
  static constexpr float SCORE_SCALE = FP8 ? 1.f / (kFp8Scale * kFp8Scale * kFp8Scale * kFp8Scale) : 1.f;
  static constexpr int PIECE = BPL * EB == 8 ? 8 : 16;  // bytes of one generator store
  static constexpr int NPC = BPL * EB / PIECE;           // generator stores per half-row
  static constexpr int WPC = PIECE / 4;                  // 32-bit words per store
  // byte offset of (row r, byte o) of a K block
  __host__ __device__ static uint32_t swz(uint32_t r, uint32_t o) {
    return KBLK == 128 ? sw128_offset(r, o) : sw64_offset(r, o);
  }
  __device__ static uint64_t desc(uint32_t saddr) { return KBLK == 128 ? smem_desc_sw128(saddr) : smem_desc_sw64(saddr); }
  static_assert(D == 32 || D == 64, "complex dimension");
  static_assert(GEN_WARPS * CPW == T, "T must be a multiple of chains per warp");
  static_assert(STAGES * NT * 2 * T <= TMEM_COLS, "tensor memory budget");
  static_assert(WPH % 16 == 0, "the epilogue loads 16-column chunks");
  static_assert(BPL * EB == 8 || (BPL * EB) % 16 == 0, "generator lanes write 8-byte or whole 16-byte pieces");
  static_assert(KBLK == 64 || KBLK == 128, "swizzle row");
  static_assert((2 * T) % 16 == 0 && 2 * T <= 256, "MMA N");
  static_assert(NTHREADS <= 1024, "block size");
};

constexpr int kMaxPhaseTab = 16 * 8;  // m * stride <= 16 * 8 (D <= 64 complex, t >= 1)

// two floats rounded to E4M3 (nearest, saturating), lo in the low byte
__device__ __forceinline__ uint32_t e4m3x2(float lo, float hi) {
  uint16_t r;
  asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(r) : "f"(hi), "f"(lo));
  return r;
}
__device__ __forceinline__ uint32_t f32x4_to_e4m3(float a, float b, float c, float d) {
  return e4m3x2(a, b) | (e4m3x2(c, d) << 16);
}
// four BF16 (two packed pairs, first entry in the low half) times kFp8Scale, as E4M3
__device__ __forceinline__ uint32_t bf16x4_to_e4m3(uint32_t p, uint32_t q) {
  return f32x4_to_e4m3(__uint_as_float(p << 16) * kFp8Scale, __uint_as_float(p & 0xFFFF0000u) * kFp8Scale,
                       __uint_as_float(q << 16) * kFp8Scale, __uint_as_float(q & 0xFFFF0000u) * kFp8Scale);
}

struct TcLaunch {
  int32_t nb;              // B ring slots in use (1..NB, the most that fit in shared memory)
  int32_t words_per_slot;  // packed words staged per super-tile (multiple of 4)
  int32_t st_slot_bytes;   // bytes of one super-tile data slot
  int32_t bins_bytes;      // bytes of the bin arrays (per chain at stride 1, per location otherwise)
  int32_t inv_bytes;       // bytes of the chain-interleaved window norms
  ThrOut thr;              // threshold mode's output (unused otherwise)
};

__device__ __forceinline__ float fmax3(float a, float b, float c) {
  float d;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}

// bin of position p from the super-tile's staged words (word index relative to word0)
__device__ __forceinline__ uint32_t bin_staged(const uint32_t* words, int64_t word0, int64_t p, int s,
                                               const uint16_t* __restrict__ map_lsb) {
  const int64_t wi = (p >> 4) - word0;
  const uint64_t v = ((uint64_t)words[wi + 1] << 32) | words[wi];
  const uint32_t field = (uint32_t)(v >> ((p & 15) * 2)) & ((1u << (2 * s)) - 1u);
  return __ldg(map_lsb + field);
}

// kDense: every score written to a.dense. kThr: every score at or above its
// window's threshold L.thr.thr[j] appended to the L.thr pair arrays.
// Otherwise: per-read candidate lists (top-k).
template <class Sh, bool kDense, bool kThr = false>
__global__ void __launch_bounds__(Sh::NTHREADS, 1) scan_tc_kernel(DevIndex ix, ScanArgs a, TcLaunch L) {
  constexpr bool kLists = !kDense && !kThr;
  constexpr int D = Sh::D, NT = Sh::NT, T = Sh::T, STAGES = Sh::STAGES, NB = Sh::NB, A = Sh::A, BPL = Sh::BPL;
  extern __shared__ __align__(1024) uint8_t tc_smem_raw[];
  __shared__ __align__(8) uint64_t bar_bfull[NB], bar_bempty[NB];
  __shared__ __align__(8) uint64_t bar_afull[STAGES], bar_aempty[STAGES];
  __shared__ __align__(8) uint64_t bar_stfull[2], bar_stempty[2];
  __shared__ __align__(8) uint64_t bar_aready, bar_drain;
  __shared__ __align__(8) uint64_t bar_gsync;  // generator warps, stride > 1 super-tile bins
  __shared__ float2 e_tab[2][kMaxPhaseTab];     // leaving / entering phases [band * S + u]
  __shared__ uint32_t tmem_base_s;
  __shared__ int abort_s;

  // dynamic shared memory:
  //   [A tiles | B ring | 2 packed-word slots | window norms [A][T] | bins [2][A][T] | lists]
  // (norms and bins are chain-interleaved: entry (step i, chain c) at i*T + c,
  // so the chains of a warp read consecutive addresses)
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* a_tiles = smem;
  uint8_t* b_ring = a_tiles + NT * Sh::A_TILE_BYTES;
  uint8_t* st_slots = b_ring + L.nb * Sh::B_SLOT_BYTES;
  float* inv_t = reinterpret_cast<float*>(st_slots + 2 * L.st_slot_bytes);
  uint8_t* bins_t = reinterpret_cast<uint8_t*>(inv_t) + L.inv_bytes;
  float* list_s = reinterpret_cast<float*>(bins_t + L.bins_bytes);
  uint32_t* list_w = reinterpret_cast<uint32_t*>(list_s + (size_t)a.cand_depth * Sh::GROUP * Sh::HALVES);
  const uint64_t wlim = a.wait_limit_ns;

  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int lane = tid & 31;
  const int S = ix.stride;
  volatile int* abort_flag = &abort_s;

  if (tid == 0) {
    for (int i = 0; i < L.nb; ++i) {
      mbar_init(&bar_bfull[i], Sh::GEN_WARPS);
      mbar_init(&bar_bempty[i], 1);
    }
    for (int i = 0; i < STAGES; ++i) {
      mbar_init(&bar_afull[i], 1);
      mbar_init(&bar_aempty[i], Sh::EPI_WARPS);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&bar_stfull[i], 1);
      mbar_init(&bar_stempty[i], Sh::GEN_WARPS);
    }
    mbar_init(&bar_aready, Sh::EPI_WARPS);
    mbar_init(&bar_gsync, Sh::GEN_WARPS * 32);
    mbar_init(&bar_drain, 1);
    abort_s = 0;
    fence_barrier_init();
  }
  for (int q = tid; q < ix.m * S; q += Sh::NTHREADS) {
    e_tab[0][q] = ix.eout[q];
    e_tab[1][q] = ix.ein[q];
  }
  if (warp == Sh::WARP_MMA) {
    tmem_alloc(&tmem_base_s, Sh::TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tmem_base_s;
  // items (read group, window range) in group-major order; each block takes a
  // contiguous run, so consecutive items of one group reuse the A operand and
  // keep one candidate list per read across their ranges
  const int64_t n_items = (int64_t)a.n_groups * a.n_ranges;
  const int64_t it_lo = n_items * blockIdx.x / gridDim.x;
  const int64_t it_hi = n_items * (blockIdx.x + 1) / gridDim.x;

  if (warp < Sh::EPI_WARPS) {
    // ================================================================ epilogue
    // warp = (half h, tile, lane quarter q); h selects windows [h*WPH, (h+1)*WPH)
    // of each stage. Each (read, half) keeps its own candidate list.
    const int q = warp & 3;
    const int tile = (warp >> 2) % NT;
    const int h = warp / (4 * NT);
    const int rs = tile * 128 + 32 * q + lane;  // read slot in the group
    const int arow = 32 * q + lane;             // its row in the A tile
    const int lstride = Sh::GROUP * Sh::HALVES;
    float* ls = list_s + h * Sh::GROUP + rs;
    uint32_t* lw = list_w + h * Sh::GROUP + rs;
    const uint32_t lane_base = (uint32_t)(32 * q) << 16;
    uint8_t* arow_base = a_tiles + tile * Sh::A_TILE_BYTES;
    uint32_t gs = 0;
    int prev_grp = -1;     // read group of the list being kept
    int seg_rng = 0;       // range whose slot receives that list
    float thr = -INFINITY;  // worst kept score, kept in a register
    int worst = 0;
    // writes the kept list of read r to the slot of range rng
    auto flush = [&](int64_t r, int rng) {
      Candidate* out = a.cand + (((size_t)r * a.n_ranges + rng) * Sh::HALVES + h) * a.cand_depth;
      for (int e = 0; e < a.cand_depth; ++e) out[e] = Candidate{ls[e * lstride] * Sh::SCORE_SCALE, lw[e * lstride]};
    };
    for (int64_t item = it_lo; item < it_hi; ++item) {
      const int grp = (int)(item / a.n_ranges);
      const int rng = (int)(item % a.n_ranges);
      const int64_t r = (int64_t)grp * Sh::GROUP + rs;
      const bool have_read = r < a.n_reads;
      const int64_t st_begin = a.st0 + (int64_t)rng * a.range_len;
      const int64_t j_lo = max(st_begin, a.jb);
      const int64_t j_hi = min(st_begin + a.range_len, a.je);
      const int64_t n_st = (j_hi - st_begin + Sh::SUP - 1) / Sh::SUP;
      // window numbers fit in 32 bits with room for a super-tile past the last
      // window (the index refuses W > 2^32 - 2^16)
      const uint32_t jlo = (uint32_t)j_lo, jhi = (uint32_t)j_hi;
      if (grp != prev_grp) {
        // a new read group: hand over the previous group's list, load the A
        // operand and start an empty list. The previous item's MMAs have all
        // completed: this thread consumed every accumulator they wrote.
        if (kLists && prev_grp >= 0) {
          const int64_t pr = (int64_t)prev_grp * Sh::GROUP + rs;
          if (pr < a.n_reads) flush(pr, seg_rng);
        }
        if (h == 0) {
          // this read's normalised BF16 row, 16-byte chunks into the swizzled
          // tile (E4M3: each chunk of 8 entries scaled, rounded and written as 8 bytes)
          const uint4* src = reinterpret_cast<const uint4*>(a.emb_bf16 + (have_read ? r : 0) * 2 * D);
#pragma unroll
          for (int c = 0; c < 2 * D / 8; ++c) {
            const uint4 v = have_read ? __ldg(src + c) : make_uint4(0, 0, 0, 0);
            const int byte = c * 8 * Sh::EB;  // first byte of the chunk in the operand row
            uint8_t* dst = arow_base + (byte / Sh::KBLK) * Sh::A_KBLK_BYTES +
                           Sh::swz((uint32_t)arow, (uint32_t)(byte % Sh::KBLK));
            if constexpr (Sh::FP8) {
              *reinterpret_cast<uint2*>(dst) = make_uint2(bf16x4_to_e4m3(v.x, v.y), bf16x4_to_e4m3(v.z, v.w));
            } else {
              *reinterpret_cast<uint4*>(dst) = v;
            }
          }
          fence_proxy_async_smem();
        }
        thr = -INFINITY;
        worst = 0;
        if (kLists) {
          for (int e = 0; e < a.cand_depth; ++e) {
            ls[e * lstride] = -INFINITY;
            lw[e * lstride] = kEmptyWin;
          }
        }
        prev_grp = grp;
        seg_rng = rng;
      } else if (kLists && have_read) {
        // the list carries on: this range's own slot holds no list
        a.cand[(((size_t)r * a.n_ranges + rng) * Sh::HALVES + h) * a.cand_depth].win = kUnusedWin;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&bar_aready);
      for (int64_t sti = 0; sti < n_st; ++sti) {
        const uint32_t st = (uint32_t)(st_begin + sti * Sh::SUP);
        for (int i = 0; i < A; ++i, ++gs) {
          const uint32_t s = gs % STAGES;
          if (!mbar_wait_warp(&bar_afull[s], (gs / STAGES) & 1, abort_flag, a.status, wlim)) goto epi_done;
          tc_fence_after();
          const uint32_t col = (uint32_t)(((int)s * NT + tile) * 2 * T);
          const uint32_t jbase = st + (uint32_t)i;  // column n holds window jbase + n*A
          const bool full = jbase >= jlo && jbase + (uint32_t)((T - 1) * A) < jhi;
          // threshold mode: lane l holds the thresholds of this warp's
          // columns h*WPH + 32u + l (+inf outside the scanned range), and each
          // 16-column chunk's smallest threshold is known to all lanes
          constexpr int TPL = kThr ? Sh::WPH / 32 : 1;
          float thr_lane[TPL], thr_min[2 * TPL];
          if constexpr (kThr) {
            static_assert(Sh::WPH % 32 == 0, "threshold mode: whole columns per lane");
#pragma unroll
            for (int u = 0; u < TPL; ++u) {
              const uint32_t jl = jbase + (uint32_t)((h * Sh::WPH + 32 * u + lane) * A);
              thr_lane[u] = (jl >= jlo && jl < jhi) ? __ldg(L.thr.thr + jl) : INFINITY;
              float mn = thr_lane[u];
#pragma unroll
              for (int o = 8; o > 0; o >>= 1) mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
              thr_min[2 * u] = __shfl_sync(0xffffffffu, mn, 0);
              thr_min[2 * u + 1] = __shfl_sync(0xffffffffu, mn, 16);
            }
          }
#pragma unroll
          for (int c0 = h * Sh::WPH; c0 < (h + 1) * Sh::WPH; c0 += 16) {
            const uint32_t taddr = tbase + lane_base + col + c0;
            uint32_t vr[16], vi[16];
            tmem_ld16(taddr, vr);
            tmem_ld16(taddr + T, vi);
            tc_wait_ld();
            if (c0 + 16 == (h + 1) * Sh::WPH) {
              // this warp's last chunk is in registers: hand the accumulator back
              tc_fence_before();
              __syncwarp();
              if (lane == 0) mbar_arrive(&bar_aempty[s]);
            }
            float sc[16];
#pragma unroll
            for (int n = 0; n < 16; n += 2) abs2_pair(vr[n], vr[n + 1], vi[n], vi[n + 1], sc[n], sc[n + 1]);
            const uint32_t jc = jbase + (uint32_t)(c0 * A);
            if constexpr (kThr) {
              // the chunk's scores against their windows' thresholds
              const float m0 = fmax3(sc[0], sc[1], sc[2]), m1 = fmax3(sc[3], sc[4], sc[5]);
              const float m2 = fmax3(sc[6], sc[7], sc[8]), m3 = fmax3(sc[9], sc[10], sc[11]);
              const float m4 = fmax3(sc[12], sc[13], sc[14]);
              const float mx = fmaxf(fmax3(m0, m1, m2), fmax3(m3, m4, sc[15]));
              const int rel = c0 - h * Sh::WPH;  // the chunk's first column in this warp's share
              const bool any = have_read && mx * Sh::SCORE_SCALE >= thr_min[rel >> 4];
              if (__any_sync(0xffffffffu, any)) {
#pragma unroll
                for (int n = 0; n < 16; ++n) {
                  const float th = __shfl_sync(0xffffffffu, thr_lane[rel >> 5], (rel & 31) + n);
                  const float v = sc[n] * Sh::SCORE_SCALE;
                  if (have_read && v >= th) {
                    const unsigned long long slot = atomicAdd(L.thr.count, 1ull);
                    if (slot < (unsigned long long)L.thr.cap) {
                      L.thr.read[slot] = r;
                      L.thr.win[slot] = (int64_t)(jc + (uint32_t)(n * A));
                      L.thr.score[slot] = v;
                    }
                  }
                }
              }
            } else if (kDense) {
              if (have_read) {
#pragma unroll
                for (int n = 0; n < 16; ++n) {
                  const uint32_t j = jc + (uint32_t)(n * A);
                  if (j >= jlo && j < jhi) a.dense[r * (a.je - a.jb) + ((int64_t)j - a.jb)] = sc[n] * Sh::SCORE_SCALE;
                }
              }
            } else {
              float mx;
              if (full) {
                // depth-3 tree of 3-input maxima
                const float m0 = fmax3(sc[0], sc[1], sc[2]), m1 = fmax3(sc[3], sc[4], sc[5]);
                const float m2 = fmax3(sc[6], sc[7], sc[8]), m3 = fmax3(sc[9], sc[10], sc[11]);
                const float m4 = fmax3(sc[12], sc[13], sc[14]);
                mx = fmaxf(fmax3(m0, m1, m2), fmax3(m3, m4, sc[15]));
              } else {
                mx = -INFINITY;
#pragma unroll
                for (int n = 0; n < 16; ++n) {
                  const uint32_t j = jc + (uint32_t)(n * A);
                  if (j >= jlo && j < jhi) mx = fmaxf(mx, sc[n]);
                }
              }
              if (have_read && mx >= thr) {
                // rare: the windows of this chunk at or above the threshold, in
                // column order, each offered to the out-of-line list update
                uint32_t pass = 0;
#pragma unroll
                for (int n = 0; n < 16; ++n) {
                  const uint32_t j = jc + (uint32_t)(n * A);
                  pass |= (j >= jlo && j < jhi && sc[n] >= thr) ? (1u << n) : 0u;
                }
                while (pass) {
                  const int n = __ffs(pass) - 1;
                  pass &= pass - 1;
                  float v = sc[0];
#pragma unroll
                  for (int k2 = 1; k2 < 16; ++k2) v = n == k2 ? sc[k2] : v;
                  if (v >= thr) {
                    const ListState ns =
                        list_insert(ls, lw, lstride, a.cand_depth, worst, v, jc + (uint32_t)(n * A), a.sep, S);
                    thr = ns.thr;
                    worst = ns.worst;
                  }
                }
              }
            }
          }
        }
      }
    }
    if (kLists && prev_grp >= 0) {
      const int64_t pr = (int64_t)prev_grp * Sh::GROUP + rs;
      if (pr < a.n_reads) flush(pr, seg_rng);
    }
  epi_done:;
  } else if (warp == Sh::WARP_MMA) {
    // ================================================================ MMA issue
    if (lane == 0) {
      uint32_t gs = 0, it = 0, bslot = 0, bphase = 0;
      bool ok = true;
      const uint64_t a_desc0 = Sh::desc(smem_u32(a_tiles));
      const uint64_t b_desc0 = Sh::desc(smem_u32(b_ring));
      for (int64_t item = it_lo; item < it_hi && ok; ++item, ++it) {
        const int rng = (int)(item % a.n_ranges);
        const int64_t st_begin = a.st0 + (int64_t)rng * a.range_len;
        const int64_t j_hi = min(st_begin + a.range_len, a.je);
        const int64_t n_stage = (j_hi - st_begin + Sh::SUP - 1) / Sh::SUP * A;
        if (!mbar_wait(&bar_aready, it & 1, abort_flag, a.status, wlim)) break;
        for (int64_t k = 0; k < n_stage; ++k, ++gs) {
          const uint32_t slot = bslot;
          const uint32_t s = gs % STAGES;
          if (!mbar_wait(&bar_bfull[slot], bphase, abort_flag, a.status, wlim)) { ok = false; break; }
          if (!mbar_wait(&bar_aempty[s], ((gs / STAGES) & 1) ^ 1, abort_flag, a.status, wlim)) { ok = false; break; }
          tc_fence_after();
          // descriptors differ only in the start-address field (16-byte units)
          const uint64_t slot_desc = b_desc0 + (uint64_t)((slot * Sh::B_SLOT_BYTES) >> 4);
#pragma unroll
          for (int t = 0; t < NT; ++t) {
            const uint32_t d_tmem = tbase + (uint32_t)(((int)s * NT + t) * 2 * T);
            const uint64_t tile_desc = a_desc0 + (uint64_t)((t * Sh::A_TILE_BYTES) >> 4);
#pragma unroll
            for (int kk = 0; kk < Sh::KSTEPS; ++kk) {
              const uint32_t kb = kk / Sh::STEPS_PER_KBLK, ko = (kk % Sh::STEPS_PER_KBLK) * 32;
              const uint64_t ad = tile_desc + (uint64_t)((kb * Sh::A_KBLK_BYTES + ko) >> 4);
              const uint64_t bd = slot_desc + (uint64_t)((kb * Sh::B_KBLK_BYTES + ko) >> 4);
              if constexpr (Sh::FP8) {
                tc_mma_ss_f8(d_tmem, ad, bd, Sh::IDESC, kk > 0 ? 1u : 0u);
              } else {
                tc_mma_ss(d_tmem, ad, bd, Sh::IDESC, kk > 0 ? 1u : 0u);
              }
            }
          }
          tc_commit(&bar_bempty[slot]);
          tc_commit(&bar_afull[s]);
          if (++bslot == (uint32_t)L.nb) {
            bslot = 0;
            bphase ^= 1u;
          }
        }
      }
      // drain: every MMA issued by this thread has completed (waited for even
      // after an abort, so that tensor memory is freed with no MMA in flight)
      tc_commit(&bar_drain);
      mbar_drain_wait(&bar_drain, 0, a.status, wlim);
    }
  } else if (warp == Sh::WARP_PROD) {
    // ================================================================ bulk-copy producer
    if (lane == 0) {
      uint32_t g = 0;
      for (int64_t item = it_lo; item < it_hi; ++item) {
        const int rng = (int)(item % a.n_ranges);
        const int64_t st_begin = a.st0 + (int64_t)rng * a.range_len;
        const int64_t j_hi = min(st_begin + a.range_len, a.je);
        const int64_t n_st = (j_hi - st_begin + Sh::SUP - 1) / Sh::SUP;
        bool ok = true;
        for (int64_t sti = 0; sti < n_st; ++sti, ++g) {
          const int64_t st = st_begin + sti * Sh::SUP;
          const uint32_t slot = g & 1;
          if (!mbar_wait(&bar_stempty[slot], ((g >> 1) & 1) ^ 1, abort_flag, a.status, wlim)) { ok = false; break; }
          uint8_t* dst = st_slots + slot * L.st_slot_bytes;
          const int64_t word0 = ((st * S) >> 4) & ~int64_t(3);
          const uint32_t wbytes = (uint32_t)L.words_per_slot * 4u;
          mbar_expect_tx(&bar_stfull[slot], wbytes);
          bulk_g2s(dst, ix.packed + word0, wbytes, &bar_stfull[slot]);
        }
        if (!ok) break;
      }
      // wait for the copies still in flight into either slot (the latest phase
      // of each), also after an abort: the block's shared memory must not be
      // released with a copy still writing to it
      for (uint32_t h = (g >= 2 ? g - 2 : 0); h < g; ++h)
        mbar_drain_wait(&bar_stfull[h & 1], (h >> 1) & 1, a.status, wlim);
    }
  } else if (!Sh::ISOLATE_MMA || (warp & 3) != 0) {
    // ================================================================ window generators
    const int gw = warp - Sh::WARP_GEN0 - Sh::idle_before(warp);
    const int chain = gw * Sh::CPW + lane / Sh::LPC;  // B row (Re) and column of its windows
    const int lic = lane % Sh::LPC;
    ChainB<BPL> ch;
    ch.setup(ix, lic);
    // byte offsets of this lane's pieces in a B slot: row chain = [cr | ci],
    // row T+chain = [ci | -cr]; BPL entries = BPL*EB bytes per half-row,
    // written as one 8-byte piece or 16-byte pieces
    constexpr int NPC = Sh::NPC;
    uint32_t off_re_cr[NPC], off_re_ci[NPC], off_im_ci[NPC], off_im_cr[NPC];
    {
      auto off = [&](int row, int e) -> uint32_t {
        const int byte = e * Sh::EB;
        return (uint32_t)((byte / Sh::KBLK) * Sh::B_KBLK_BYTES) + Sh::swz((uint32_t)row, (uint32_t)(byte % Sh::KBLK));
      };
#pragma unroll
      for (int pc = 0; pc < NPC; ++pc) {
        const int e_lo = BPL * lic + pc * Sh::PIECE / Sh::EB, e_hi = D + e_lo;
        off_re_cr[pc] = off(chain, e_lo);
        off_re_ci[pc] = off(chain, e_hi);
        off_im_ci[pc] = off(T + chain, e_lo);
        off_im_cr[pc] = off(T + chain, e_hi);
      }
    }
    uint32_t g = 0, bslot = 0, bphase = 0, gsp = 0;
    // all generator threads meet (bounded wait) around the stride > 1 bin fill
    auto gen_sync = [&]() -> bool {
      mbar_arrive(&bar_gsync);
      return mbar_wait_warp(&bar_gsync, (gsp++) & 1, abort_flag, a.status, wlim);
    };
    const int in_off = ix.N - ix.s + 1;  // entering location relative to the leaving one
    for (int64_t item = it_lo; item < it_hi; ++item) {
      const int rng = (int)(item % a.n_ranges);
      const int64_t st_begin = a.st0 + (int64_t)rng * a.range_len;
      const int64_t j_hi = min(st_begin + a.range_len, a.je);
      const int64_t n_st = (j_hi - st_begin + Sh::SUP - 1) / Sh::SUP;
      for (int64_t sti = 0; sti < n_st; ++sti, ++g) {
        const int64_t st = st_begin + sti * Sh::SUP;
        const uint32_t slot = g & 1;
        if (!mbar_wait_warp(&bar_stfull[slot], (g >> 1) & 1, abort_flag, a.status, wlim)) goto gen_done;
        const uint32_t* words = reinterpret_cast<const uint32_t*>(st_slots + slot * L.st_slot_bytes);
        const int64_t word0 = ((st * S) >> 4) & ~int64_t(3);
        const int64_t a_idx = st / A + chain;  // this chain's anchor (padded past the last window)
        const int64_t p_out0 = (st + (int64_t)chain * A) * S;
        const int64_t p_in0 = p_out0 + ix.N - ix.s + 1;
        // this chain's window norms and (stride 1) bins, chain-interleaved
        for (int u = lic; u < A; u += Sh::LPC) {
          inv_t[u * T + chain] = __ldg(ix.inv_norm + st + (int64_t)chain * A + u);
          if (S == 1) {
            bins_t[u * T + chain] = (uint8_t)bin_staged(words, word0, p_out0 + u, ix.s, ix.map_lsb);
            bins_t[(A + u) * T + chain] = (uint8_t)bin_staged(words, word0, p_in0 + u, ix.s, ix.map_lsb);
          }
        }
        if (S > 1) {
          // the bins of every location of the super-tile, each computed once
          // and shared by all chains (the previous super-tile's are all used)
          if (!gen_sync()) goto gen_done;
          const int n_pos = Sh::SUP * S + in_off;
          const int64_t pos0 = st * S;
          for (int t = gw * 32 + lane; t < n_pos; t += Sh::GEN_WARPS * 32)
            bins_t[t] = (uint8_t)bin_staged(words, word0, pos0 + t, ix.s, ix.map_lsb);
          if (!gen_sync()) goto gen_done;
        }
        ch.load(ix.anchors + a_idx * D, lic);
        __syncwarp();
        for (int i = 0; i < A; ++i) {
          const float nv = inv_t[i * T + chain] * (Sh::FP8 ? kFp8Scale : 1.f);
          if (!mbar_wait_warp(&bar_bempty[bslot], bphase ^ 1u, abort_flag, a.status, wlim)) goto gen_done;
          {
            uint8_t* bt = b_ring + bslot * Sh::B_SLOT_BYTES;
            // packed operand words of cr, ci and -cr (sign bits flipped)
            constexpr int NW = BPL * Sh::EB / 4;
            uint32_t pr[NW], pi[NW], pn[NW];
#pragma unroll
            for (int hh = 0; hh < NW; ++hh) {
              if constexpr (Sh::FP8) {
                pr[hh] = f32x4_to_e4m3(ch.cr[4 * hh] * nv, ch.cr[4 * hh + 1] * nv, ch.cr[4 * hh + 2] * nv,
                                       ch.cr[4 * hh + 3] * nv);
                pi[hh] = f32x4_to_e4m3(ch.ci[4 * hh] * nv, ch.ci[4 * hh + 1] * nv, ch.ci[4 * hh + 2] * nv,
                                       ch.ci[4 * hh + 3] * nv);
                pn[hh] = pr[hh] ^ 0x80808080u;
              } else {
                const __nv_bfloat162 rr = __floats2bfloat162_rn(ch.cr[2 * hh] * nv, ch.cr[2 * hh + 1] * nv);
                const __nv_bfloat162 ii = __floats2bfloat162_rn(ch.ci[2 * hh] * nv, ch.ci[2 * hh + 1] * nv);
                pr[hh] = *reinterpret_cast<const uint32_t*>(&rr);
                pi[hh] = *reinterpret_cast<const uint32_t*>(&ii);
                pn[hh] = pr[hh] ^ 0x80008000u;
              }
            }
            if constexpr (Sh::PIECE == 8) {
              *reinterpret_cast<uint2*>(bt + off_re_cr[0]) = make_uint2(pr[0], pr[1]);
              *reinterpret_cast<uint2*>(bt + off_re_ci[0]) = make_uint2(pi[0], pi[1]);
              *reinterpret_cast<uint2*>(bt + off_im_ci[0]) = make_uint2(pi[0], pi[1]);
              *reinterpret_cast<uint2*>(bt + off_im_cr[0]) = make_uint2(pn[0], pn[1]);
            } else {
#pragma unroll
              for (int pc = 0; pc < NPC; ++pc) {
                const int o = 4 * pc;
                *reinterpret_cast<uint4*>(bt + off_re_cr[pc]) = make_uint4(pr[o], pr[o + 1], pr[o + 2], pr[o + 3]);
                *reinterpret_cast<uint4*>(bt + off_re_ci[pc]) = make_uint4(pi[o], pi[o + 1], pi[o + 2], pi[o + 3]);
                *reinterpret_cast<uint4*>(bt + off_im_ci[pc]) = make_uint4(pi[o], pi[o + 1], pi[o + 2], pi[o + 3]);
                *reinterpret_cast<uint4*>(bt + off_im_cr[pc]) = make_uint4(pn[o], pn[o + 1], pn[o + 2], pn[o + 3]);
              }
            }
          }
          fence_proxy_async_smem();
          __syncwarp();
          if (lane == 0) mbar_arrive(&bar_bfull[bslot]);
          if (++bslot == (uint32_t)L.nb) {
            bslot = 0;
            bphase ^= 1u;
          }
          // advance the recurrence to the next window
          if (S == 1) {
            ch.step1(bins_t[i * T + chain], bins_t[(A + i) * T + chain]);
          } else {
            const int base = (chain * A + i) * S;
            const float2* eo = e_tab[0] + ch.band * S;
            const float2* ei = e_tab[1] + ch.band * S;
            for (int u = 0; u < S; ++u) {
              ch.sub_at(bins_t[base + u], eo[u]);
              ch.add_at(bins_t[base + in_off + u], ei[u]);
            }
            ch.rotate();
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&bar_stempty[slot]);
      }
    }
  gen_done:;
  }

  tc_fence_before();
  __syncthreads();
  if (warp == Sh::WARP_MMA) {
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tbase, Sh::TMEM_COLS);
  }
}

// ---------------------------------------------------------------- configurations

// d = 64:  256 reads x 64 windows per stage, MMA N = 128; 16 epilogue warps (two
//          per accumulator quarter), 8 generator warps (chains of 4 lanes x 8
//          entries), the MMA warp alone with epilogue warps on its scheduler;
//          up to 6 window slots between the generators and the MMA warp.
using TcShape32 = TcShape<32, 2, 64, 2, 6, 4, 2, true>;
// d = 64, second tile variant: one epilogue warp per accumulator quarter and
//          tile (8 warps, each reading all 64 windows of a stage; one candidate
//          list per read), more registers per thread. Faster at large strides.
using TcShape32b = TcShape<32, 2, 64, 2, 4, 4, 1, true>;
// d = 64, third tile variant: 512 reads (4 tiles) x 32 windows per stage, MMA
//          N = 64 (twice the MMA instructions per score, on a tensor pipe that
//          is a quarter busy) so that each generated window serves twice as
//          many reads: half the window-generation work per score.
using TcShape32c = TcShape<32, 4, 32, 2, 4, 4, 1, true>;
// d = 128: 256 reads x 64 windows per stage, MMA N = 128 (twice the tensor time
//          per stage); 8 epilogue warps, 16 generator warps (chains of 8 lanes x 8 entries)
using TcShape64 = TcShape<64, 2, 64, 2, 2, 8, 1, false>;
// the same tiles with E4M3 operands (kind::f8f6f4): half the operand bytes,
// half the MMA instructions per stage; 64-byte swizzled rows at d = 64
using TcShape32f8 = TcShape<32, 2, 64, 2, 4, 4, 2, true, true>;
using TcShape32bf8 = TcShape<32, 2, 64, 2, 4, 4, 1, true, true>;
using TcShape32cf8 = TcShape<32, 4, 32, 2, 4, 4, 1, true, true>;
using TcShape64f8 = TcShape<64, 2, 64, 2, 2, 8, 1, false, true>;

// Dynamic shared memory one block of this kernel may take: the device's
// opt-in maximum per block less the kernel's static shared memory (barriers,
// phase tables). 0 if the attributes cannot be read.
// Read once per device and kept (so that launches made while a stream is
// being captured into a graph query nothing).
constexpr int kMaxDevices = 64;

template <class Sh, bool kDense, bool kThr = false>
static size_t tc_dyn_limit() {
  static size_t cached[kMaxDevices] = {};  // value + 1, 0 = not read yet
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return 0;
  }
  if (cached[dev]) return cached[dev] - 1;
  cudaFuncAttributes fa{};
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
      cudaFuncGetAttributes(&fa, scan_tc_kernel<Sh, kDense, kThr>) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const size_t v = optin > (int)fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes : 0;
  cached[dev] = v + 1;
  return v;
}

// Raises the kernel's dynamic shared-memory limit on the current device when
// a launch needs more than it was last set to (once per size increase).
template <class Sh, bool kDense, bool kThr = false>
static cudaError_t tc_reserve_smem(size_t smem) {
  static size_t set[kMaxDevices] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < kMaxDevices && set[dev] >= smem) return cudaSuccess;
  e = cudaFuncSetAttribute(scan_tc_kernel<Sh, kDense, kThr>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess && dev >= 0 && dev < kMaxDevices) set[dev] = smem;
  return e;
}

int scan_tc_supported(int D) { return D == 32 || D == 64; }

int64_t scan_tc_super_tile(int D, int variant) {
  if (D == 32) return variant == 2 ? TcShape32c::SUP : TcShape32::SUP;
  return D == 64 ? TcShape64::SUP : 0;
}

int scan_tc_group(int D, int variant) {
  if (D == 32) return variant == 2 ? TcShape32c::GROUP : TcShape32::GROUP;
  return D == 64 ? TcShape64::GROUP : 0;
}

int scan_tc_max_stride() { return 8; }

int scan_tc_variants(int D) { return D == 32 ? 3 : D == 64 ? 1 : 0; }

int scan_tc_lists_per_range(int D, int variant) {
  if (D == 32) return variant == 1 ? TcShape32b::HALVES : variant == 2 ? TcShape32c::HALVES : TcShape32::HALVES;
  return D == 64 ? TcShape64::HALVES : 1;
}

template <class Sh>
static size_t tc_smem_bytes(const DevIndex& ix, int cand_depth, bool dense, int nb, TcLaunch* Lout) {
  TcLaunch L;
  L.nb = nb;
  const int S = ix.stride;
  int64_t words = ((int64_t)Sh::SUP * S + ix.N + 64) / 16 + 8;
  words = (words + 3) & ~int64_t(3);
  L.words_per_slot = (int32_t)words;
  int64_t slot = words * 4;
  slot = (slot + 127) & ~int64_t(127);
  L.st_slot_bytes = (int32_t)slot;
  L.inv_bytes = Sh::A * Sh::T * 4;
  // stride 1: per-chain bins, chain-interleaved; stride > 1: one bin per
  // location of the super-tile, shared by the chains
  L.bins_bytes = S == 1 ? (int32_t)(Sh::T * 2 * Sh::A) : (int32_t)((Sh::SUP * S + ix.N - ix.s + 1 + 15) & ~15);
  const size_t lists = dense ? 0 : (size_t)cand_depth * Sh::GROUP * Sh::HALVES * 8;
  if (Lout) *Lout = L;
  return 1024 + (size_t)Sh::NT * Sh::A_TILE_BYTES + (size_t)nb * Sh::B_SLOT_BYTES + 2 * (size_t)L.st_slot_bytes +
         L.inv_bytes + L.bins_bytes + lists;
}

template <class Sh>
static int tc_fits(const DevIndex& ix, int cand_depth) {
  TcLaunch L;
  return tc_smem_bytes<Sh>(ix, cand_depth, false, 1, &L) <= tc_dyn_limit<Sh, false>();
}

int scan_tc_fits(const DevIndex& ix, int cand_depth, int variant, int fp8) {
  if (ix.D == 32 && variant == 1) return fp8 ? tc_fits<TcShape32bf8>(ix, cand_depth) : tc_fits<TcShape32b>(ix, cand_depth);
  if (ix.D == 32 && variant == 2) return fp8 ? tc_fits<TcShape32cf8>(ix, cand_depth) : tc_fits<TcShape32c>(ix, cand_depth);
  if (ix.D == 32) return fp8 ? tc_fits<TcShape32f8>(ix, cand_depth) : tc_fits<TcShape32>(ix, cand_depth);
  if (ix.D == 64) return fp8 ? tc_fits<TcShape64f8>(ix, cand_depth) : tc_fits<TcShape64>(ix, cand_depth);
  return 0;
}

template <class Sh, bool kDense, bool kThr = false>
static cudaError_t launch_tc(const DevIndex& ix, const ScanArgs& a, int num_sms, cudaStream_t st,
                             const ThrOut* thr = nullptr) {
  // the deepest B ring that fits (long windows at large strides and deep
  // candidate lists leave room for fewer slots)
  TcLaunch L;
  const size_t limit = tc_dyn_limit<Sh, kDense, kThr>();
  int nb = Sh::NB;
  constexpr bool kNoLists = kDense || kThr;
  size_t smem = tc_smem_bytes<Sh>(ix, a.cand_depth, kNoLists, nb, &L);
  while (smem > limit && nb > 1) smem = tc_smem_bytes<Sh>(ix, a.cand_depth, kNoLists, nb >>= 1, &L);
  if (smem > limit) return cudaErrorInvalidValue;
  L.thr = thr ? *thr : ThrOut{};
  auto kern = scan_tc_kernel<Sh, kDense, kThr>;
  cudaError_t e = tc_reserve_smem<Sh, kDense, kThr>(smem);
  if (e != cudaSuccess) {
    cudaGetLastError();  // not sticky: leave no pending error for later launches
    return e;
  }
  const int64_t n_items = (int64_t)a.n_groups * a.n_ranges;
  const int grid = (int)(num_sms < n_items ? num_sms : n_items);
  if (grid < 1) return cudaSuccess;
  kern<<<grid, Sh::NTHREADS, smem, st>>>(ix, a, L);
  return cudaGetLastError();
}

template <class Sh>
static cudaError_t launch_tc_any(const DevIndex& ix, const ScanArgs& a, bool dense, int num_sms, cudaStream_t st) {
  return dense ? launch_tc<Sh, true>(ix, a, num_sms, st) : launch_tc<Sh, false>(ix, a, num_sms, st);
}

cudaError_t launch_scan_tc(const DevIndex& ix, const ScanArgs& a, bool dense, int num_sms, cudaStream_t st) {
  if (ix.stride > scan_tc_max_stride()) return cudaErrorInvalidValue;
  if (ix.D == 32 && a.tc_variant == 1)
    return a.fp8 ? launch_tc_any<TcShape32bf8>(ix, a, dense, num_sms, st)
                 : launch_tc_any<TcShape32b>(ix, a, dense, num_sms, st);
  if (ix.D == 32 && a.tc_variant == 2)
    return a.fp8 ? launch_tc_any<TcShape32cf8>(ix, a, dense, num_sms, st)
                 : launch_tc_any<TcShape32c>(ix, a, dense, num_sms, st);
  if (ix.D == 32)
    return a.fp8 ? launch_tc_any<TcShape32f8>(ix, a, dense, num_sms, st)
                 : launch_tc_any<TcShape32>(ix, a, dense, num_sms, st);
  if (ix.D == 64)
    return a.fp8 ? launch_tc_any<TcShape64f8>(ix, a, dense, num_sms, st)
                 : launch_tc_any<TcShape64>(ix, a, dense, num_sms, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_scan_tc_threshold(const DevIndex& ix, const ScanArgs& a, const ThrOut& out, int num_sms,
                                     cudaStream_t st) {
  if (ix.stride > scan_tc_max_stride() || a.fp8) return cudaErrorInvalidValue;
  if (ix.D == 32) return launch_tc<TcShape32, false, true>(ix, a, num_sms, st, &out);
  if (ix.D == 64) return launch_tc<TcShape64, false, true>(ix, a, num_sms, st, &out);
  return cudaErrorInvalidValue;
}

}  // namespace rope
