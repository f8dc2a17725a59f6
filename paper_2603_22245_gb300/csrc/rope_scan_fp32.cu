// FP32 CUDA-core scan ("plain" path).
//
// One thread per read: the read's normalised vector sits in registers; the
// block's eight warps generate tiles of window vectors on chip (chains of D/4
// lanes running the §3.4 recurrence from exact anchors), normalise them by the
// stored 1/sqrt(C_j) and stage them in shared memory; every thread then forms
// Re and Im of <x|c> for each window (the §4 real identity) and the fidelity
// Re^2 + Im^2, keeping its read's best windows in a shared-memory list.
#include "rope_internal.h"
#include "rope_topk.cuh"

namespace rope {

constexpr int kF32Threads = 256;  // reads per group
constexpr int kF32Steps = 8;      // windows per chain per tile

template <int D>
struct F32Shape {
  static constexpr int LPC = D / 4;
  static constexpr int CPW = 32 / LPC;
  static constexpr int C = (kF32Threads / 32) * CPW;  // chains per block
  static constexpr int TW = C * kF32Steps;            // windows per tile
  static constexpr int SUP = C * kAnchorPeriod;       // windows per super-tile
  static constexpr size_t kTileBytes = (size_t)TW * 2 * D * sizeof(float);
};

template <int D, bool kDense, bool kPerBand>
__global__ void __launch_bounds__(kF32Threads) scan_fp32_kernel(DevIndex ix, ScanArgs a) {
  using Sh = F32Shape<D>;
  extern __shared__ __align__(16) uint8_t f32_smem[];
  float* tile = reinterpret_cast<float*>(f32_smem);
  float* list_s = reinterpret_cast<float*>(f32_smem + Sh::kTileBytes);
  uint32_t* list_w = reinterpret_cast<uint32_t*>(list_s + (size_t)a.cand_depth * kF32Threads);

  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const int lic = lane % Sh::LPC;
  const int chain = warp * Sh::CPW + lane / Sh::LPC;
  const int S = ix.stride;
  const int n_items = a.n_groups * a.n_ranges;

  ThreadList lst;
  lst.s = list_s + tid;
  lst.w = list_w + tid;
  lst.stride = kF32Threads;
  lst.depth = a.cand_depth;

  Chain<D> ch;
  ch.setup(ix, lic);

  for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
    const int grp = item % a.n_groups;
    const int rng = item / a.n_groups;
    const int64_t r = (int64_t)grp * kF32Threads + tid;
    const bool have_read = r < a.n_reads;
    const int64_t st_begin = a.st0 + (int64_t)rng * a.range_len;
    const int64_t j_lo = max(st_begin, a.jb);
    const int64_t j_hi = min(st_begin + a.range_len, a.je);

    // the read's vector, normalised (per band in score mode 1)
    float xr[D], xi[D];
    {
      const float* e = a.emb_f32 + (have_read ? r : 0) * 2 * D;
      const float* nr = a.norms + (have_read ? r : 0) * (1 + ix.m);
      float inv = 0.f;
      if (!kPerBand) {
        const float X = nr[0];
        inv = (have_read && X > kZeroNorm2) ? rsqrtf(X) : 0.f;
      }
#pragma unroll
      for (int g = 0; g < D; ++g) {
        float sc = inv;
        if (kPerBand) {
          const float Xk = nr[1 + g / ix.nb];
          sc = (have_read && Xk > kZeroNorm2) ? rsqrtf(Xk) : 0.f;
        }
        xr[g] = e[g] * sc;
        xi[g] = e[D + g] * sc;
      }
    }
    if (!kDense) lst.reset();

    for (int64_t st = st_begin; st < j_hi; st += Sh::SUP) {
      const int64_t a_idx = st / ix.A + chain;
      const bool chain_live = a_idx * ix.A < ix.W;
      if (chain_live) {
        ch.load(ix.anchors + a_idx * D, lic);
      } else {
#pragma unroll
        for (int i = 0; i < 4; ++i) ch.cr[i] = ch.ci[i] = 0.f;
      }
      for (int rd = 0; rd < kAnchorPeriod / kF32Steps; ++rd) {
        // ---- generate kF32Steps windows per chain into the tile
#pragma unroll 1
        for (int u = 0; u < kF32Steps; ++u) {
          const int64_t j = st + (int64_t)chain * ix.A + rd * kF32Steps + u;
          const bool live = chain_live && j < ix.W;
          float* row = tile + (size_t)(chain * kF32Steps + u) * 2 * D;
          float4 vr, vi;
          if (!kPerBand) {
            const float inv = live ? ix.inv_norm[j] : 0.f;
            vr = make_float4(ch.cr[0] * inv, ch.cr[1] * inv, ch.cr[2] * inv, ch.cr[3] * inv);
            vi = make_float4(ch.ci[0] * inv, ch.ci[1] * inv, ch.ci[2] * inv, ch.ci[3] * inv);
          } else {
            const float Ck = live ? ix.band_norm[j * ix.m + ch.band] : 0.f;
            const float inv = Ck > kZeroNorm2 ? rsqrtf(Ck) : 0.f;
            vr = make_float4(ch.cr[0] * inv, ch.cr[1] * inv, ch.cr[2] * inv, ch.cr[3] * inv);
            vi = make_float4(ch.ci[0] * inv, ch.ci[1] * inv, ch.ci[2] * inv, ch.ci[3] * inv);
          }
          reinterpret_cast<float4*>(row)[lic] = vr;
          reinterpret_cast<float4*>(row + D)[lic] = vi;
          if (live) {
            const int64_t w = j * S;
            if (S == 1) {
              ch.step1(bin_at(ix.packed, w, ix.s, ix.map_lsb),
                       bin_at(ix.packed, w + ix.N - ix.s + 1, ix.s, ix.map_lsb));
            } else {
              for (int q = 0; q < S; ++q) {
                ch.sub_at(bin_at(ix.packed, w + q, ix.s, ix.map_lsb), ix.eout[ch.band * S + q]);
                ch.add_at(bin_at(ix.packed, w + ix.N - ix.s + 1 + q, ix.s, ix.map_lsb), ix.ein[ch.band * S + q]);
              }
              ch.rotate();
            }
          }
        }
        __syncthreads();
        // ---- score every window of the tile against this thread's read
        if (have_read) {
#pragma unroll 1
          for (int q = 0; q < Sh::TW; q += 2) {
            const float4* c0r = reinterpret_cast<const float4*>(tile + (size_t)q * 2 * D);
            const float4* c0i = c0r + D / 4;
            const float4* c1r = c0r + 2 * D / 4;
            const float4* c1i = c1r + D / 4;
            float sc0 = 0.f, sc1 = 0.f;
            if (!kPerBand) {
              float re0a = 0.f, re0b = 0.f, im0a = 0.f, im0b = 0.f;
              float re1a = 0.f, re1b = 0.f, im1a = 0.f, im1b = 0.f;
#pragma unroll
              for (int e4 = 0; e4 < D / 4; ++e4) {
                const float4 ar = c0r[e4], ai = c0i[e4], br = c1r[e4], bi = c1i[e4];
                const float xa[4] = {xr[4 * e4], xr[4 * e4 + 1], xr[4 * e4 + 2], xr[4 * e4 + 3]};
                const float ya[4] = {xi[4 * e4], xi[4 * e4 + 1], xi[4 * e4 + 2], xi[4 * e4 + 3]};
                const float car[4] = {ar.x, ar.y, ar.z, ar.w}, cai[4] = {ai.x, ai.y, ai.z, ai.w};
                const float cbr[4] = {br.x, br.y, br.z, br.w}, cbi[4] = {bi.x, bi.y, bi.z, bi.w};
#pragma unroll
                for (int h = 0; h < 4; h += 2) {
                  re0a = fmaf(xa[h], car[h], fmaf(ya[h], cai[h], re0a));
                  im0a = fmaf(xa[h], cai[h], fmaf(-ya[h], car[h], im0a));
                  re1a = fmaf(xa[h], cbr[h], fmaf(ya[h], cbi[h], re1a));
                  im1a = fmaf(xa[h], cbi[h], fmaf(-ya[h], cbr[h], im1a));
                  re0b = fmaf(xa[h + 1], car[h + 1], fmaf(ya[h + 1], cai[h + 1], re0b));
                  im0b = fmaf(xa[h + 1], cai[h + 1], fmaf(-ya[h + 1], car[h + 1], im0b));
                  re1b = fmaf(xa[h + 1], cbr[h + 1], fmaf(ya[h + 1], cbi[h + 1], re1b));
                  im1b = fmaf(xa[h + 1], cbi[h + 1], fmaf(-ya[h + 1], cbr[h + 1], im1b));
                }
              }
              const float re0 = re0a + re0b, im0 = im0a + im0b, re1 = re1a + re1b, im1 = im1a + im1b;
              sc0 = fmaf(re0, re0, im0 * im0);
              sc1 = fmaf(re1, re1, im1 * im1);
            } else {
              const float* t0 = tile + (size_t)q * 2 * D;
              const float* t1 = t0 + 2 * D;
              for (int k = 0; k < ix.m; ++k) {
                float re0 = 0.f, im0 = 0.f, re1 = 0.f, im1 = 0.f;
#pragma unroll
                for (int g = 0; g < D; ++g) {
                  if (g / ix.nb != k) continue;
                  re0 = fmaf(xr[g], t0[g], fmaf(xi[g], t0[D + g], re0));
                  im0 = fmaf(xr[g], t0[D + g], fmaf(-xi[g], t0[g], im0));
                  re1 = fmaf(xr[g], t1[g], fmaf(xi[g], t1[D + g], re1));
                  im1 = fmaf(xr[g], t1[D + g], fmaf(-xi[g], t1[g], im1));
                }
                sc0 += fmaf(re0, re0, im0 * im0);
                sc1 += fmaf(re1, re1, im1 * im1);
              }
              sc0 /= ix.m;
              sc1 /= ix.m;
            }
            // window numbers of tile slots q, q+1
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int qq = q + h;
              const int64_t j = st + (int64_t)(qq / kF32Steps) * ix.A + rd * kF32Steps + (qq % kF32Steps);
              const float sc = h == 0 ? sc0 : sc1;
              if (j < j_lo || j >= j_hi) continue;
              if (kDense) {
                a.dense[r * (a.je - a.jb) + (j - a.jb)] = sc;
              } else if (sc >= lst.thr) {
                lst.insert(sc, (uint32_t)j, a.sep, S);
              }
            }
          }
        }
        __syncthreads();
      }
    }
    if (!kDense && have_read) {
      Candidate* out = a.cand + ((size_t)r * a.n_ranges + rng) * a.cand_depth;
      for (int e = 0; e < a.cand_depth; ++e) out[e] = Candidate{lst.S(e), lst.Wn(e)};
    }
  }
}

int scan_fp32_supported(int D) { return D == 4 || D == 8 || D == 16 || D == 32 || D == 64; }

int64_t scan_fp32_super_tile(int D) {
  switch (D) {
    case 4: return F32Shape<4>::SUP;
    case 8: return F32Shape<8>::SUP;
    case 16: return F32Shape<16>::SUP;
    case 32: return F32Shape<32>::SUP;
    case 64: return F32Shape<64>::SUP;
  }
  return 0;
}

int scan_fp32_group(int) { return kF32Threads; }

template <int D, bool kDense, bool kPerBand>
static cudaError_t launch_one(const DevIndex& ix, const ScanArgs& a, int num_sms, cudaStream_t st) {
  using Sh = F32Shape<D>;
  const size_t smem = Sh::kTileBytes + (kDense ? 0 : (size_t)a.cand_depth * kF32Threads * 8);
  auto kern = scan_fp32_kernel<D, kDense, kPerBand>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 1;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kF32Threads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  const int n_items = a.n_groups * a.n_ranges;
  int grid = num_sms * per_sm;
  if (grid > n_items) grid = n_items;
  if (grid < 1) return cudaSuccess;
  kern<<<grid, kF32Threads, smem, st>>>(ix, a);
  return cudaGetLastError();
}

template <bool kDense, bool kPerBand>
static cudaError_t dispatch(const DevIndex& ix, const ScanArgs& a, int num_sms, cudaStream_t st) {
  switch (ix.D) {
    case 4: return launch_one<4, kDense, kPerBand>(ix, a, num_sms, st);
    case 8: return launch_one<8, kDense, kPerBand>(ix, a, num_sms, st);
    case 16: return launch_one<16, kDense, kPerBand>(ix, a, num_sms, st);
    case 32: return launch_one<32, kDense, kPerBand>(ix, a, num_sms, st);
    case 64: return launch_one<64, kDense, kPerBand>(ix, a, num_sms, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_scan_fp32(const DevIndex& ix, const ScanArgs& a, bool dense, int num_sms, cudaStream_t st) {
  const bool pb = ix.score_mode == 1;
  if (dense) return pb ? dispatch<true, true>(ix, a, num_sms, st) : dispatch<true, false>(ix, a, num_sms, st);
  return pb ? dispatch<false, true>(ix, a, num_sms, st) : dispatch<false, false>(ix, a, num_sms, st);
}

}  // namespace rope
