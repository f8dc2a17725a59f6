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
//     warps produce them: each chain of 8 lanes runs the §3.4 recurrence from
//     an exact anchor through 64 consecutive windows and emits one window per
//     stage, scaled by the stored 1/sqrt(C_j) and rounded to BF16.
//   * D (tensor memory): per stage and tile a 128 x 2T FP32 accumulator whose
//     columns are Re (0..T-1) and Im (T..2T-1).
//   * One thread issues tcgen05.mma (M = 128, N = 2T = 128, K = 16 per
//     instruction; an MMA costs at least ~45 cycles whatever N is, so N = 128
//     keeps the tensor pipe saturated) and commits to mbarriers; a producer
//     warp streams the 2-bit packed reference and the window norms of each
//     super-tile into shared memory with bulk copies (TMA); epilogue warps
//     (thread = read) load the accumulators with tcgen05.ld in 16-column
//     chunks, form Re^2 + Im^2 and keep the read's best windows.
// Every wait is bounded; a wait that runs out sets the timeout status bit and
// the block drains its in-flight copies and MMAs, frees tensor memory and exits.
#include <cuda_bf16.h>

#include "rope_internal.h"
#include "rope_topk.cuh"

namespace rope {

template <int D_, int NT_, int T_, int STAGES_, int NB_>
struct TcShape {
  static constexpr int D = D_, NT = NT_, T = T_, STAGES = STAGES_, NB = NB_;
  static constexpr int A = kAnchorPeriod;
  static constexpr int BPL = D / 8;              // complex entries per generator lane
  static constexpr int LPC = 8;                  // lanes per chain
  static constexpr int CPW = 32 / LPC;           // chains per warp
  static constexpr int GEN_WARPS = T / CPW;
  static constexpr int EPI_WARPS = 4 * NT;
  static constexpr int WARP_MMA = EPI_WARPS;
  static constexpr int WARP_PROD = EPI_WARPS + 1;
  static constexpr int WARP_GEN0 = EPI_WARPS + 2;
  static constexpr int NWARPS = EPI_WARPS + 2 + GEN_WARPS;
  static constexpr int NTHREADS = 32 * NWARPS;
  static constexpr int SUP = T * A;                   // windows per super-tile
  static constexpr int GROUP = NT * 128;              // reads per work item
  static constexpr int KSTEPS = 2 * D / 16;           // K = 2D in steps of 16
  static constexpr int KBLOCKS = 2 * D / 64;          // 64-element (128-byte) K blocks
  static constexpr int A_KBLK_BYTES = 128 * 128;      // one K block of an A tile
  static constexpr int A_TILE_BYTES = KBLOCKS * A_KBLK_BYTES;
  static constexpr int B_KBLK_BYTES = 2 * T * 128;    // one K block of a B tile
  static constexpr int B_SLOT_BYTES = KBLOCKS * B_KBLK_BYTES;
  static constexpr int TMEM_COLS = 512;
  static constexpr uint32_t IDESC = idesc_bf16_f32(128, 2 * T);
  static_assert(D == 32 || D == 64, "complex dimension");
  static_assert(GEN_WARPS * CPW == T, "T must be a multiple of chains per warp");
  static_assert(STAGES * NT * 2 * T <= TMEM_COLS, "tensor memory budget");
  static_assert(T % 16 == 0, "the epilogue loads 16-column chunks");
  static_assert((2 * T) % 16 == 0 && 2 * T <= 256, "MMA N");
  static_assert(NTHREADS <= 1024, "block size");
};

struct TcLaunch {
  int32_t words_per_slot;  // packed words staged per super-tile (multiple of 4)
  int32_t st_slot_bytes;   // bytes of one super-tile data slot
  int32_t bins_bytes;      // bytes of the per-chain bin arrays (stride 1)
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

template <class Sh, bool kDense>
__global__ void __launch_bounds__(Sh::NTHREADS, 1) scan_tc_kernel(DevIndex ix, ScanArgs a, TcLaunch L) {
  constexpr int D = Sh::D, NT = Sh::NT, T = Sh::T, STAGES = Sh::STAGES, NB = Sh::NB, A = Sh::A, BPL = Sh::BPL;
  extern __shared__ __align__(1024) uint8_t tc_smem_raw[];
  __shared__ __align__(8) uint64_t bar_bfull[NB], bar_bempty[NB];
  __shared__ __align__(8) uint64_t bar_afull[STAGES], bar_aempty[STAGES];
  __shared__ __align__(8) uint64_t bar_stfull[2], bar_stempty[2];
  __shared__ __align__(8) uint64_t bar_aready, bar_drain;
  __shared__ uint32_t tmem_base_s;
  __shared__ int abort_s;

  // dynamic shared memory: [A tiles | B ring | 2 super-tile slots | chain bins | lists]
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* a_tiles = smem;
  uint8_t* b_ring = a_tiles + NT * Sh::A_TILE_BYTES;
  uint8_t* st_slots = b_ring + NB * Sh::B_SLOT_BYTES;
  uint8_t* chain_bins = st_slots + 2 * L.st_slot_bytes;
  float* list_s = reinterpret_cast<float*>(chain_bins + L.bins_bytes);
  uint32_t* list_w = reinterpret_cast<uint32_t*>(list_s + (size_t)a.cand_depth * Sh::GROUP);

  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int lane = tid & 31;
  const int S = ix.stride;
  volatile int* abort_flag = &abort_s;

  if (tid == 0) {
    for (int i = 0; i < NB; ++i) {
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
    mbar_init(&bar_drain, 1);
    abort_s = 0;
    fence_barrier_init();
  }
  if (warp == Sh::WARP_MMA) {
    tmem_alloc(&tmem_base_s, Sh::TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tmem_base_s;
  const int n_items = a.n_groups * a.n_ranges;

  if (warp < Sh::EPI_WARPS) {
    // ================================================================ epilogue
    const int q = warp & 3;
    const int tile = warp >> 2;
    const int rs = tile * 128 + 32 * q + lane;  // read slot in the group
    const int arow = 32 * q + lane;             // its row in the A tile
    ThreadList lst;
    lst.s = list_s + rs;
    lst.w = list_w + rs;
    lst.stride = Sh::GROUP;
    lst.depth = a.cand_depth;
    const uint32_t lane_base = (uint32_t)(32 * q) << 16;
    uint8_t* arow_base = a_tiles + tile * Sh::A_TILE_BYTES;
    uint32_t gs = 0;
    for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
      const int grp = item % a.n_groups;
      const int rng = item / a.n_groups;
      const int64_t r = (int64_t)grp * Sh::GROUP + rs;
      const bool have_read = r < a.n_reads;
      const int64_t st_begin = a.st0 + (int64_t)rng * a.range_len;
      const int64_t j_lo = max(st_begin, a.jb);
      const int64_t j_hi = min(st_begin + a.range_len, a.je);
      const int64_t n_st = (j_hi - st_begin + Sh::SUP - 1) / Sh::SUP;
      // A operand: this read's normalised BF16 row, 16-byte chunks into the
      // swizzled tile. The previous item's MMAs have all completed: this
      // thread consumed every accumulator they wrote.
      {
        const uint4* src = reinterpret_cast<const uint4*>(a.emb_bf16 + (have_read ? r : 0) * 2 * D);
#pragma unroll
        for (int c = 0; c < 2 * D / 8; ++c) {
          const uint4 v = have_read ? __ldg(src + c) : make_uint4(0, 0, 0, 0);
          const int kb = c >> 3;
          *reinterpret_cast<uint4*>(arow_base + kb * Sh::A_KBLK_BYTES +
                                    sw128_offset((uint32_t)arow, (uint32_t)((c & 7) * 16))) = v;
        }
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(&bar_aready);
      }
      if (!kDense) lst.reset();
      for (int64_t sti = 0; sti < n_st; ++sti) {
        const int64_t st = st_begin + sti * Sh::SUP;
        for (int i = 0; i < A; ++i, ++gs) {
          const uint32_t s = gs % STAGES;
          if (!mbar_wait_warp(&bar_afull[s], (gs / STAGES) & 1, abort_flag, a.status)) goto epi_done;
          tc_fence_after();
          const uint32_t col = (uint32_t)(((int)s * NT + tile) * 2 * T);
          const int64_t jbase = st + i;  // column n holds window jbase + n*A
          const bool full = jbase >= j_lo && jbase + (int64_t)(T - 1) * A < j_hi;
#pragma unroll
          for (int c0 = 0; c0 < T; c0 += 16) {
            uint32_t vr[16], vi[16];
            tmem_ld16(tbase + lane_base + col + c0, vr);
            tmem_ld16(tbase + lane_base + col + T + c0, vi);
            tc_wait_ld();
            if (c0 + 16 == T) {
              // the last chunk is in registers: hand the accumulator back
              tc_fence_before();
              __syncwarp();
              if (lane == 0) mbar_arrive(&bar_aempty[s]);
            }
            float sc[16];
#pragma unroll
            for (int n = 0; n < 16; ++n) {
              const float re = __uint_as_float(vr[n]);
              const float im = __uint_as_float(vi[n]);
              sc[n] = fmaf(re, re, im * im);
            }
            const int64_t jc = jbase + (int64_t)c0 * A;
            if (kDense) {
              if (have_read) {
#pragma unroll
                for (int n = 0; n < 16; ++n) {
                  const int64_t j = jc + (int64_t)n * A;
                  if (j >= j_lo && j < j_hi) a.dense[r * (a.je - a.jb) + (j - a.jb)] = sc[n];
                }
              }
            } else {
              float mx;
              if (full) {
                mx = fmax3(sc[0], sc[1], sc[2]);
#pragma unroll
                for (int n = 3; n + 1 < 16; n += 2) mx = fmax3(mx, sc[n], sc[n + 1]);
                mx = fmaxf(mx, sc[15]);
              } else {
                mx = -INFINITY;
#pragma unroll
                for (int n = 0; n < 16; ++n) {
                  const int64_t j = jc + (int64_t)n * A;
                  if (j >= j_lo && j < j_hi) mx = fmaxf(mx, sc[n]);
                }
              }
              if (have_read && mx >= lst.thr) {
#pragma unroll
                for (int n = 0; n < 16; ++n) {
                  const int64_t j = jc + (int64_t)n * A;
                  if (j >= j_lo && j < j_hi && sc[n] >= lst.thr) lst.insert(sc[n], (uint32_t)j, a.sep, S);
                }
              }
            }
          }
        }
      }
      if (!kDense && have_read) {
        Candidate* out = a.cand + ((size_t)r * a.n_ranges + rng) * a.cand_depth;
        for (int e = 0; e < a.cand_depth; ++e) out[e] = Candidate{lst.S(e), lst.Wn(e)};
      }
    }
  epi_done:;
  } else if (warp == Sh::WARP_MMA) {
    // ================================================================ MMA issue
    if (lane == 0) {
      uint32_t gs = 0, gb = 0, it = 0;
      bool ok = true;
      const uint64_t a_desc0 = smem_desc_sw128(smem_u32(a_tiles));
      const uint64_t b_desc0 = smem_desc_sw128(smem_u32(b_ring));
      for (int item = blockIdx.x; item < n_items && ok; item += gridDim.x, ++it) {
        const int rng = item / a.n_groups;
        const int64_t st_begin = a.st0 + (int64_t)rng * a.range_len;
        const int64_t j_hi = min(st_begin + a.range_len, a.je);
        const int64_t n_stage = (j_hi - st_begin + Sh::SUP - 1) / Sh::SUP * A;
        if (!mbar_wait(&bar_aready, it & 1, abort_flag, a.status)) break;
        for (int64_t k = 0; k < n_stage; ++k, ++gs, ++gb) {
          const uint32_t slot = gb % NB;
          const uint32_t s = gs % STAGES;
          if (!mbar_wait(&bar_bfull[slot], (gb / NB) & 1, abort_flag, a.status)) { ok = false; break; }
          if (!mbar_wait(&bar_aempty[s], ((gs / STAGES) & 1) ^ 1, abort_flag, a.status)) { ok = false; break; }
          tc_fence_after();
          // descriptors differ only in the start-address field (16-byte units)
          const uint64_t slot_desc = b_desc0 + (uint64_t)((slot * Sh::B_SLOT_BYTES) >> 4);
#pragma unroll
          for (int t = 0; t < NT; ++t) {
            const uint32_t d_tmem = tbase + (uint32_t)(((int)s * NT + t) * 2 * T);
            const uint64_t tile_desc = a_desc0 + (uint64_t)((t * Sh::A_TILE_BYTES) >> 4);
#pragma unroll
            for (int kk = 0; kk < Sh::KSTEPS; ++kk) {
              const uint32_t kb = kk >> 2, ko = (kk & 3) * 32;
              const uint64_t ad = tile_desc + (uint64_t)((kb * Sh::A_KBLK_BYTES + ko) >> 4);
              const uint64_t bd = slot_desc + (uint64_t)((kb * Sh::B_KBLK_BYTES + ko) >> 4);
              tc_mma_ss(d_tmem, ad, bd, Sh::IDESC, kk > 0 ? 1u : 0u);
            }
          }
          tc_commit(&bar_bempty[slot]);
          tc_commit(&bar_afull[s]);
        }
      }
      // drain: every MMA issued by this thread has completed
      tc_commit(&bar_drain);
      mbar_wait(&bar_drain, 0, abort_flag, a.status);
    }
  } else if (warp == Sh::WARP_PROD) {
    // ================================================================ bulk-copy producer
    if (lane == 0) {
      uint32_t g = 0;
      for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int rng = item / a.n_groups;
        const int64_t st_begin = a.st0 + (int64_t)rng * a.range_len;
        const int64_t j_hi = min(st_begin + a.range_len, a.je);
        const int64_t n_st = (j_hi - st_begin + Sh::SUP - 1) / Sh::SUP;
        bool ok = true;
        for (int64_t sti = 0; sti < n_st; ++sti, ++g) {
          const int64_t st = st_begin + sti * Sh::SUP;
          const uint32_t slot = g & 1;
          if (!mbar_wait(&bar_stempty[slot], ((g >> 1) & 1) ^ 1, abort_flag, a.status)) { ok = false; break; }
          uint8_t* dst = st_slots + slot * L.st_slot_bytes;
          const int64_t word0 = ((st * S) >> 4) & ~int64_t(3);
          const uint32_t wbytes = (uint32_t)L.words_per_slot * 4u;
          const uint32_t nbytes = (uint32_t)Sh::SUP * 4u;
          mbar_expect_tx(&bar_stfull[slot], wbytes + nbytes);
          bulk_g2s(dst, ix.packed + word0, wbytes, &bar_stfull[slot]);
          bulk_g2s(dst + wbytes, ix.inv_norm + st, nbytes, &bar_stfull[slot]);
        }
        if (!ok) break;
      }
      // wait for the copies still in flight into either slot (the latest phase of each)
      for (uint32_t h = (g >= 2 ? g - 2 : 0); h < g; ++h)
        mbar_wait(&bar_stfull[h & 1], (h >> 1) & 1, abort_flag, a.status);
    }
  } else {
    // ================================================================ window generators
    const int gw = warp - Sh::WARP_GEN0;
    const int chain = gw * Sh::CPW + lane / Sh::LPC;  // B row (Re) and column of its windows
    const int lic = lane % Sh::LPC;
    uint8_t* bins_out = chain_bins + (size_t)chain * 2 * A;
    uint8_t* bins_in = bins_out + A;
    ChainB<BPL> ch;
    ch.setup(ix, lic);
    // byte offsets of this lane's pieces in a B slot: row chain = [cr | ci],
    // row T+chain = [ci | -cr]; BPL bf16 (2*BPL bytes) each
    uint32_t off_re_cr, off_re_ci, off_im_ci, off_im_cr;
    {
      const int e_lo = BPL * lic, e_hi = D + BPL * lic;
      auto off = [&](int row, int e) -> uint32_t {
        return (uint32_t)((e >> 6) * Sh::B_KBLK_BYTES) + sw128_offset((uint32_t)row, (uint32_t)((e & 63) * 2));
      };
      off_re_cr = off(chain, e_lo);
      off_re_ci = off(chain, e_hi);
      off_im_ci = off(T + chain, e_lo);
      off_im_cr = off(T + chain, e_hi);
    }
    uint32_t g = 0, gb = 0;
    for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
      const int rng = item / a.n_groups;
      const int64_t st_begin = a.st0 + (int64_t)rng * a.range_len;
      const int64_t j_hi = min(st_begin + a.range_len, a.je);
      const int64_t n_st = (j_hi - st_begin + Sh::SUP - 1) / Sh::SUP;
      for (int64_t sti = 0; sti < n_st; ++sti, ++g) {
        const int64_t st = st_begin + sti * Sh::SUP;
        const uint32_t slot = g & 1;
        if (!mbar_wait_warp(&bar_stfull[slot], (g >> 1) & 1, abort_flag, a.status)) goto gen_done;
        const uint8_t* src = st_slots + slot * L.st_slot_bytes;
        const uint32_t* words = reinterpret_cast<const uint32_t*>(src);
        const float* inv = reinterpret_cast<const float*>(src + (size_t)L.words_per_slot * 4);
        const int64_t word0 = ((st * S) >> 4) & ~int64_t(3);
        const int64_t a_idx = st / A + chain;  // this chain's anchor (padded past the last window)
        const int64_t p_out0 = (st + (int64_t)chain * A) * S;
        const int64_t p_in0 = p_out0 + ix.N - ix.s + 1;
        if (S == 1) {
          for (int u = lic; u < 2 * A; u += Sh::LPC) {
            const int64_t p = u < A ? p_out0 + u : p_in0 + (u - A);
            bins_out[u] = (uint8_t)bin_staged(words, word0, p, ix.s, ix.map_lsb);
          }
        }
        ch.load(ix.anchors + a_idx * D, lic);
        __syncwarp();
        for (int i = 0; i < A; ++i, ++gb) {
          const uint32_t bslot = gb % NB;
          const float nv = inv[chain * A + i];
          if (!mbar_wait_warp(&bar_bempty[bslot], ((gb / NB) & 1) ^ 1, abort_flag, a.status)) goto gen_done;
          {
            uint8_t* bt = b_ring + bslot * Sh::B_SLOT_BYTES;
            uint32_t pr[BPL / 2], pi[BPL / 2], pn[BPL / 2];
#pragma unroll
            for (int h = 0; h < BPL / 2; ++h) {
              const __nv_bfloat162 rr = __floats2bfloat162_rn(ch.cr[2 * h] * nv, ch.cr[2 * h + 1] * nv);
              const __nv_bfloat162 ii = __floats2bfloat162_rn(ch.ci[2 * h] * nv, ch.ci[2 * h + 1] * nv);
              pr[h] = *reinterpret_cast<const uint32_t*>(&rr);
              pi[h] = *reinterpret_cast<const uint32_t*>(&ii);
              pn[h] = pr[h] ^ 0x80008000u;
            }
            if constexpr (BPL == 4) {
              *reinterpret_cast<uint2*>(bt + off_re_cr) = make_uint2(pr[0], pr[1]);
              *reinterpret_cast<uint2*>(bt + off_re_ci) = make_uint2(pi[0], pi[1]);
              *reinterpret_cast<uint2*>(bt + off_im_ci) = make_uint2(pi[0], pi[1]);
              *reinterpret_cast<uint2*>(bt + off_im_cr) = make_uint2(pn[0], pn[1]);
            } else {
              *reinterpret_cast<uint4*>(bt + off_re_cr) = make_uint4(pr[0], pr[1], pr[2], pr[3]);
              *reinterpret_cast<uint4*>(bt + off_re_ci) = make_uint4(pi[0], pi[1], pi[2], pi[3]);
              *reinterpret_cast<uint4*>(bt + off_im_ci) = make_uint4(pi[0], pi[1], pi[2], pi[3]);
              *reinterpret_cast<uint4*>(bt + off_im_cr) = make_uint4(pn[0], pn[1], pn[2], pn[3]);
            }
          }
          fence_proxy_async_smem();
          __syncwarp();
          if (lane == 0) mbar_arrive(&bar_bfull[bslot]);
          // advance the recurrence to the next window
          if (S == 1) {
            ch.step1(bins_out[i], bins_in[i]);
          } else {
            const int64_t po = p_out0 + (int64_t)i * S;
            for (int u = 0; u < S; ++u) {
              ch.sub_at(bin_staged(words, word0, po + u, ix.s, ix.map_lsb), ix.eout[ch.band * S + u]);
              ch.add_at(bin_staged(words, word0, po + ix.N - ix.s + 1 + u, ix.s, ix.map_lsb),
                        ix.ein[ch.band * S + u]);
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

using TcShape32 = TcShape<32, 2, 64, 2, 4>;  // d = 64:  256 reads x 64 windows per stage, MMA N = 128
using TcShape64 = TcShape<64, 2, 64, 2, 2>;  // d = 128: 256 reads x 64 windows per stage, MMA N = 128

int scan_tc_supported(int D) { return D == 32 || D == 64; }

int64_t scan_tc_super_tile(int D) { return D == 32 ? TcShape32::SUP : D == 64 ? TcShape64::SUP : 0; }

int scan_tc_group(int D) { return D == 32 ? TcShape32::GROUP : D == 64 ? TcShape64::GROUP : 0; }

int scan_tc_max_stride() { return 8; }

template <class Sh>
static size_t tc_smem_bytes(const DevIndex& ix, int cand_depth, bool dense, TcLaunch* Lout) {
  TcLaunch L;
  const int S = ix.stride;
  int64_t words = ((int64_t)Sh::SUP * S + ix.N + 64) / 16 + 8;
  words = (words + 3) & ~int64_t(3);
  L.words_per_slot = (int32_t)words;
  int64_t slot = words * 4 + (int64_t)Sh::SUP * 4;
  slot = (slot + 127) & ~int64_t(127);
  L.st_slot_bytes = (int32_t)slot;
  L.bins_bytes = S == 1 ? (int32_t)(Sh::T * 2 * Sh::A) : 0;
  const size_t lists = dense ? 0 : (size_t)cand_depth * Sh::GROUP * 8;
  if (Lout) *Lout = L;
  return 1024 + (size_t)Sh::NT * Sh::A_TILE_BYTES + (size_t)Sh::NB * Sh::B_SLOT_BYTES + 2 * (size_t)L.st_slot_bytes +
         L.bins_bytes + lists;
}

template <class Sh, bool kDense>
static cudaError_t launch_tc(const DevIndex& ix, const ScanArgs& a, int num_sms, cudaStream_t st) {
  TcLaunch L;
  const size_t smem = tc_smem_bytes<Sh>(ix, a.cand_depth, kDense, &L);
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  auto kern = scan_tc_kernel<Sh, kDense>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int n_items = a.n_groups * a.n_ranges;
  int grid = num_sms < n_items ? num_sms : n_items;
  if (grid < 1) return cudaSuccess;
  kern<<<grid, Sh::NTHREADS, smem, st>>>(ix, a, L);
  return cudaGetLastError();
}

cudaError_t launch_scan_tc(const DevIndex& ix, const ScanArgs& a, bool dense, int num_sms, cudaStream_t st) {
  if (ix.stride > scan_tc_max_stride()) return cudaErrorInvalidValue;
  if (ix.D == 32)
    return dense ? launch_tc<TcShape32, true>(ix, a, num_sms, st) : launch_tc<TcShape32, false>(ix, a, num_sms, st);
  if (ix.D == 64)
    return dense ? launch_tc<TcShape64, true>(ix, a, num_sms, st) : launch_tc<TcShape64, false>(ix, a, num_sms, st);
  return cudaErrorInvalidValue;
}

}  // namespace rope
