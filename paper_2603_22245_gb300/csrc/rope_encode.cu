// Encoding kernels: 2-bit packing, s-mer bins, read-head encodings (direct
// summation), the FP64 reference pre-pass (anchors and exact window norms) and
// the window-embedding inspection kernel.
#include <cuda_bf16.h>

#include "rope_internal.h"

namespace rope {

// ---------------------------------------------------------------- a1: packing

// Four letters (one byte each) to four 2-bit codes in one byte, a word at a
// time. Bits 1-2 of an ASCII letter are 0,1,3,2 for A,C,G,T (either case), a
// Gray code: x ^ (x >> 1) turns them into 0,1,2,3. The letters are then
// checked by rebuilding each byte's lower-case letter from its code
// ('a' + {0, 2, 6, 19}) and comparing with the input folded to lower case;
// any difference, accumulated in `bad`, marks a letter outside ACGTacgt. The
// multiply gathers the byte-spaced codes into the top byte (the partial
// products of different bytes land in disjoint bits below it).
__device__ __forceinline__ uint32_t pack4(uint32_t x, uint32_t& bad) {
  const uint32_t g = (x >> 1) & 0x03030303u;
  const uint32_t code = g ^ ((g >> 1) & 0x01010101u);
  const uint32_t hi = (code >> 1) & 0x01010101u;           // code >= 2
  const uint32_t three = hi & code;                         // code == 3
  const uint32_t letter = 0x61616161u + ((code + hi) << 1) + three * 11u;
  bad |= (x | 0x20202020u) ^ letter;
  return (code * 0x01041040u) >> 24;
}

// One output word (16 letters) per thread; 16-byte vector loads when aligned.
// HBM-bound: 1 byte in and 1/4 byte out per letter.
// One thread packs kPackWords consecutive 16-letter words per step: their
// four 16-byte loads are issued together, so enough bytes are in flight to
// keep HBM busy; the ragged tail and unaligned inputs take the byte path.
constexpr int kPackWords = 4;

__device__ __forceinline__ uint32_t pack_bytes(const uint8_t* seq, int64_t base, int64_t len, uint32_t& bad) {
  uint32_t word = 0;
  for (int i = 0; i < 16 && base + i < len; ++i) {
    const uint32_t c = letter_code(seq[base + i]);
    bad |= (c > 3);
    word |= (c & 3u) << (2 * i);
  }
  return word;
}

__global__ void pack_kernel(const uint8_t* __restrict__ seq, int64_t len, uint32_t* __restrict__ out,
                            int64_t n_words, int* status) {
  // vector loads and stores need 16-byte aligned input and output
  const bool aligned = ((((uintptr_t)seq) | ((uintptr_t)out)) & 15u) == 0;
  uint32_t bad = 0;
  const int64_t n_groups = (n_words + kPackWords - 1) / kPackWords;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n_groups;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t w0 = g * kPackWords;
    if (aligned && (w0 + kPackWords) * 16 <= len) {
      uint4 v[kPackWords];
#pragma unroll
      for (int q = 0; q < kPackWords; ++q) v[q] = __ldg(reinterpret_cast<const uint4*>(seq + (w0 + q) * 16));
      uint32_t wd[kPackWords];
#pragma unroll
      for (int q = 0; q < kPackWords; ++q)
        wd[q] = pack4(v[q].x, bad) | (pack4(v[q].y, bad) << 8) | (pack4(v[q].z, bad) << 16) |
                (pack4(v[q].w, bad) << 24);
      *reinterpret_cast<uint4*>(out + w0) = make_uint4(wd[0], wd[1], wd[2], wd[3]);
    } else {
      for (int q = 0; q < kPackWords && w0 + q < n_words; ++q) out[w0 + q] = pack_bytes(seq, (w0 + q) * 16, len, bad);
    }
  }
  if (bad) set_status(status, kStatusBadBase);
}

cudaError_t launch_pack(const uint8_t* seq, int64_t len, uint32_t* out, int* status, cudaStream_t st) {
  const int64_t n_words = (len + 15) / 16;
  if (n_words == 0) return cudaSuccess;
  const int threads = 256;
  const int64_t n_groups = (n_words + kPackWords - 1) / kPackWords;
  int64_t blocks = (n_groups + threads - 1) / threads;
  if (blocks > 152 * 32) blocks = 152 * 32;
  pack_kernel<<<(unsigned)blocks, threads, 0, st>>>(seq, len, out, n_words, status);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- a2: bins

__global__ void mer_bins_kernel(const uint32_t* __restrict__ packed, int64_t n_pos, int64_t n_words, int s,
                                const uint16_t* __restrict__ map_lsb, uint16_t* __restrict__ out) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n_pos; p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t wi = p >> 4;
    const uint32_t lo = packed[wi];
    const uint32_t hi = wi + 1 < n_words ? packed[wi + 1] : 0u;
    const uint64_t v = ((uint64_t)hi << 32) | lo;
    const uint32_t field = (uint32_t)(v >> ((p & 15) * 2)) & ((1u << (2 * s)) - 1u);
    out[p] = map_lsb[field];
  }
}

cudaError_t launch_mer_bins(const uint32_t* packed, int64_t len, int64_t n_words, int s, const uint16_t* map_lsb,
                            uint16_t* out, cudaStream_t st) {
  const int64_t n_pos = len - s + 1;
  if (n_pos <= 0) return cudaSuccess;
  int64_t blocks = (n_pos + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  mer_bins_kernel<<<(unsigned)blocks, 256, 0, st>>>(packed, n_pos, n_words, s, map_lsb, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- a3: read heads

// One warp per read. Locations are taken in order; for each location the
// lanes k < m add exp(2 pi i f_k loc / N) to entry (k, bin) of a per-warp
// shared accumulator, so every entry is summed in location order (the direct
// sum of §2.1-§2.3 in FP32, deterministic).
// Letter q (0..3, 4 if not ACGT) of the head of a read of length len: the read
// itself, or (rc) its reverse complement, whose head is the complement of the
// read's last letters read backwards.
__device__ __forceinline__ uint32_t head_letter(const uint8_t* seq, int64_t len, int q, bool rc) {
  if (!rc) return letter_code(seq[q]);
  const uint32_t c = letter_code(seq[len - 1 - q]);
  return c > 3 ? c : 3u - c;  // A<->T, C<->G
}

// One warp per read; lane l owns entries g = l, l + 32, ... of the D complex
// entries (band g / 4^t, bin g % 4^t) in registers. The locations are taken 32
// at a time, one per lane; warp ballots of the bits of their bins tell each
// lane which of the 32 locations fall in its entries' bins, and the lane adds
// e^{2 pi i f_k loc / N} (phase table staged in shared memory) for those
// locations in increasing order. Every entry is thus summed in location order
// (the direct sum of §2.1-§2.3 in FP32, deterministic), with a warp cost per
// 32 locations of a few ballots plus the largest bin's count.
constexpr int kEncMaxPerLane = kMaxScanDim / 32;
constexpr int kEncMaxBinBits = 8;  // bins per band up to 256

__global__ void encode_reads_kernel(EncTables tb, const uint8_t* __restrict__ seqs,
                                    const int64_t* __restrict__ offsets, int64_t n, float* __restrict__ emb_f32,
                                    __nv_bfloat16* __restrict__ emb_bf16, float* __restrict__ norms, int* status,
                                    const int64_t* __restrict__ perm, bool rc) {
  extern __shared__ float2 enc_phase[];  // [m * n_loc] phases, staged once per block
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int wpb = blockDim.x >> 5;
  const int n_loc = tb.N - tb.s + 1;
  const int E = (tb.D + 31) / 32;  // entries per lane
  const int bin_bits = 32 - __clz(tb.nb > 1 ? tb.nb - 1 : 1);
  for (int i = threadIdx.x; i < tb.m * n_loc; i += blockDim.x) enc_phase[i] = tb.phase[i];
  __syncthreads();
  int band[kEncMaxPerLane], bin[kEncMaxPerLane];
#pragma unroll
  for (int e = 0; e < kEncMaxPerLane; ++e) {
    const int g = lane + 32 * e;
    band[e] = g < tb.D ? g / tb.nb : 0;
    bin[e] = g < tb.D ? g % tb.nb : -1;  // -1: no entry
  }
  for (int64_t r = (int64_t)blockIdx.x * wpb + warp; r < n; r += (int64_t)gridDim.x * wpb) {
    const int64_t src = perm ? perm[r] : r;
    const int64_t start = offsets[src];
    const int64_t len = offsets[src + 1] - start;
    const uint8_t* seq = seqs + start;
    float ar[kEncMaxPerLane], ai[kEncMaxPerLane];
#pragma unroll
    for (int e = 0; e < kEncMaxPerLane; ++e) ar[e] = ai[e] = 0.f;
    bool ok = len >= tb.N;
    if (!ok) {
      if (lane == 0) set_status(status, kStatusShortRead);
    } else {
      int bad = 0;
      for (int i = lane; i < tb.N; i += 32) bad |= head_letter(seq, len, i, rc) > 3;
      if (__any_sync(0xffffffffu, bad)) {
        ok = false;
        if (lane == 0) set_status(status, kStatusBadBase);
      }
    }
    if (ok) {
      for (int loc0 = 0; loc0 < n_loc; loc0 += 32) {
        const int loc = loc0 + lane;
        uint32_t b = 0;
        if (loc < n_loc) {
          uint32_t code = 0;
          for (int i = 0; i < tb.s; ++i) code = code * 4u + (head_letter(seq, len, loc + i, rc) & 3u);
          b = (uint32_t)tb.map[code];
        }
        // bit planes of the 32 locations' bins: the locations whose bin is
        // B are the lanes that agree with B on every plane
        const uint32_t valid = __ballot_sync(0xffffffffu, loc < n_loc);
        uint32_t plane[kEncMaxBinBits];
#pragma unroll
        for (int i = 0; i < kEncMaxBinBits; ++i)
          plane[i] = i < bin_bits ? __ballot_sync(0xffffffffu, (b >> i) & 1u) : 0u;
#pragma unroll
        for (int e = 0; e < kEncMaxPerLane; ++e) {
          if (e >= E || bin[e] < 0) continue;
          uint32_t hit = valid;
#pragma unroll
          for (int i = 0; i < kEncMaxBinBits; ++i)
            if (i < bin_bits) hit &= ((bin[e] >> i) & 1) ? plane[i] : ~plane[i];
          const float2* ph_row = enc_phase + band[e] * n_loc + loc0;
          while (hit) {  // the matching locations in increasing order
            const int j = __ffs(hit) - 1;
            hit &= hit - 1u;
            const float2 ph = ph_row[j];
            ar[e] += ph.x;
            ai[e] += ph.y;
          }
        }
      }
    }
    // per-band squared norms, then the total
    float total = 0.f;
    for (int k = 0; k < tb.m; ++k) {
      float part = 0.f;
#pragma unroll
      for (int e = 0; e < kEncMaxPerLane; ++e)
        if (e < E && bin[e] >= 0 && band[e] == k) part = fmaf(ar[e], ar[e], fmaf(ai[e], ai[e], part));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
      if (lane == 0) norms[r * (1 + tb.m) + 1 + k] = part;
      total += part;
    }
    if (lane == 0) norms[r * (1 + tb.m)] = total;
    const float inv = total > kZeroNorm2 ? rsqrtf(total) : 0.f;
#pragma unroll
    for (int e = 0; e < kEncMaxPerLane; ++e) {
      const int g = lane + 32 * e;
      if (e >= E || g >= tb.D) continue;
      if (emb_f32) {
        emb_f32[r * 2 * tb.D + g] = ar[e];
        emb_f32[r * 2 * tb.D + tb.D + g] = ai[e];
      }
      if (emb_bf16) {
        emb_bf16[r * 2 * tb.D + g] = __float2bfloat16_rn(ar[e] * inv);
        emb_bf16[r * 2 * tb.D + tb.D + g] = __float2bfloat16_rn(ai[e] * inv);
      }
    }
  }
}

// Encodings wider than kMaxScanDim complex entries, or heads whose phase table
// exceeds what one block stages: one warp per read head, its D complex entries
// in shared memory. Locations are taken 32 at a time, one per lane; lanes whose
// locations fall in the same bin form a group (__match_any_sync), and the
// group's lowest lane (its first location) sums the group's phases in
// location order and adds that sum to the entry, so each entry receives one
// update per 32 locations, in location order (deterministic FP32 sums of the
// §2.1-§2.3 direct sum). The phases of kEncChunk locations are staged in
// shared memory once per block for all of its warps.
constexpr int kEncChunk = 1024;

__global__ void encode_reads_wide_kernel(EncTables tb, const uint8_t* __restrict__ seqs,
                                    const int64_t* __restrict__ offsets, int64_t n, float* __restrict__ emb_f32,
                                    __nv_bfloat16* __restrict__ emb_bf16, float* __restrict__ norms, int* status,
                                    const int64_t* __restrict__ perm, bool rc) {
  extern __shared__ float2 enc_sm[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int wpb = blockDim.x >> 5;
  const int n_loc = tb.N - tb.s + 1;
  float2* ph = enc_sm;                                              // [m][kEncChunk]
  float2* acc = enc_sm + (size_t)tb.m * kEncChunk + (size_t)warp * tb.D;  // this warp's entries
  for (int64_t r0 = (int64_t)blockIdx.x * wpb; r0 < n; r0 += (int64_t)gridDim.x * wpb) {
    const int64_t r = r0 + warp;
    const bool live = r < n;
    const int64_t src = live ? (perm ? perm[r] : r) : 0;
    const int64_t start = live ? offsets[src] : 0;
    const int64_t len = live ? offsets[src + 1] - start : 0;
    const uint8_t* seq = seqs + start;
    for (int g = lane; g < tb.D; g += 32) acc[g] = make_float2(0.f, 0.f);
    bool ok = live && len >= tb.N;
    if (live && !ok) {
      if (lane == 0) set_status(status, kStatusShortRead);
    } else if (ok) {
      int bad = 0;
      for (int i = lane; i < tb.N; i += 32) bad |= head_letter(seq, len, i, rc) > 3;
      if (__any_sync(0xffffffffu, bad)) {
        ok = false;
        if (lane == 0) set_status(status, kStatusBadBase);
      }
    }
    for (int c0 = 0; c0 < n_loc; c0 += kEncChunk) {
      const int c1 = min(c0 + kEncChunk, n_loc);
      __syncthreads();  // every warp is done with the previous chunk's phases
      for (int i = threadIdx.x; i < tb.m * kEncChunk; i += blockDim.x) {
        const int k = i / kEncChunk, u = i - k * kEncChunk;
        if (c0 + u < c1) ph[i] = tb.phase[(size_t)k * n_loc + c0 + u];
      }
      __syncthreads();
      if (!ok) continue;
      for (int l0 = c0; l0 < c1; l0 += 32) {
        const int loc = l0 + lane;
        const bool valid = loc < c1;
        // s-mer code of this lane's location from the letters of lanes
        // loc .. loc+s-1 (two 32-letter rows held across the warp)
        // every letter of the head is loaded, also past the chunk's last
        // location: the s-mers of the chunk's last locations read them
        const uint32_t lo = loc < tb.N ? head_letter(seq, len, loc, rc) & 3u : 0u;
        const uint32_t hi = (l0 + 32 + lane < tb.N) ? head_letter(seq, len, l0 + 32 + lane, rc) & 3u : 0u;
        uint32_t code = 0;
        for (int i = 0; i < tb.s; ++i) {
          const int sl = lane + i;
          const uint32_t a = __shfl_sync(0xffffffffu, lo, sl & 31);
          const uint32_t b = __shfl_sync(0xffffffffu, hi, sl & 31);
          code = code * 4u + (sl < 32 ? a : b);
        }
        const uint32_t bin = valid ? (uint32_t)__ldg(tb.map + code) : 0xFFFFFFFFu;
        const uint32_t grp = __match_any_sync(0xffffffffu, bin);
        const int size = __popc(grp);
        const int gmax = (int)__reduce_max_sync(0xffffffffu, (unsigned)size);
        const bool leader = valid && (__ffs(grp) - 1) == lane;
        for (int k = 0; k < tb.m; ++k) {
          const float2 p = valid ? ph[k * kEncChunk + (loc - c0)] : make_float2(0.f, 0.f);
          float sx = 0.f, sy = 0.f;
          uint32_t rest = grp;
          for (int it = 0; it < gmax; ++it) {  // the group's members in location order
            const int m_lane = rest ? __ffs(rest) - 1 : lane;
            rest &= rest - 1u;
            const float qx = __shfl_sync(0xffffffffu, p.x, m_lane);
            const float qy = __shfl_sync(0xffffffffu, p.y, m_lane);
            if (it < size) {
              sx += qx;
              sy += qy;
            }
          }
          if (leader) {
            float2& e = acc[k * tb.nb + bin];
            e.x += sx;
            e.y += sy;
          }
        }
      }
    }
    __syncwarp();
    if (live) {
      // per-band squared norms, then the total
      float total = 0.f;
      for (int k = 0; k < tb.m; ++k) {
        float part = 0.f;
        for (int b = lane; b < tb.nb; b += 32) {
          const float2 a = acc[k * tb.nb + b];
          part = fmaf(a.x, a.x, fmaf(a.y, a.y, part));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if (lane == 0) norms[r * (1 + tb.m) + 1 + k] = part;
        total += part;
      }
      if (lane == 0) norms[r * (1 + tb.m)] = total;
      const float inv = total > kZeroNorm2 ? rsqrtf(total) : 0.f;
      for (int g = lane; g < tb.D; g += 32) {
        const float2 a = acc[g];
        if (emb_f32) {
          emb_f32[r * 2 * tb.D + g] = a.x;
          emb_f32[r * 2 * tb.D + tb.D + g] = a.y;
        }
        if (emb_bf16) {
          emb_bf16[r * 2 * tb.D + g] = __float2bfloat16_rn(a.x * inv);
          emb_bf16[r * 2 * tb.D + tb.D + g] = __float2bfloat16_rn(a.y * inv);
        }
      }
    }
    __syncwarp();
  }
}

cudaError_t launch_encode_reads(const EncTables& tb, const uint8_t* seqs, const int64_t* offsets, int64_t n,
                                float* emb_f32, uint16_t* emb_bf16, float* norms, int* status, cudaStream_t st,
                                const int64_t* perm, bool rc) {
  if (n <= 0) return cudaSuccess;
  const size_t phase_bytes = (size_t)tb.m * (tb.N - tb.s + 1) * sizeof(float2);
  if (tb.D <= kMaxScanDim && phase_bytes <= 48 * 1024) {
    const int wpb = 8;
    int64_t blocks = (n + wpb - 1) / wpb;
    if (blocks > 152 * 16) blocks = 152 * 16;  // each block stages the phase table once
    encode_reads_kernel<<<(unsigned)blocks, wpb * 32, phase_bytes, st>>>(tb, seqs, offsets, n, emb_f32,
                                                                 reinterpret_cast<__nv_bfloat16*>(emb_bf16), norms,
                                                                 status, perm, rc);
    return cudaGetLastError();
  }
  // phase chunk + one accumulator per warp, within 100 KB (two blocks per SM)
  const size_t chunk_bytes = (size_t)tb.m * kEncChunk * sizeof(float2);
  int wpb = (int)((100 * 1024 - chunk_bytes) / (tb.D * sizeof(float2)));
  if (wpb > 8) wpb = 8;
  if (wpb < 1) wpb = 1;
  const size_t smem = chunk_bytes + (size_t)wpb * tb.D * sizeof(float2);
  static int attr_set[64] = {};  // per device: bytes the attribute was last raised to
  int dev = 0;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || (int)smem > attr_set[dev]) {
      e = cudaFuncSetAttribute(encode_reads_wide_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      if (dev >= 0 && dev < 64) attr_set[dev] = (int)smem;
    }
  }
  int64_t blocks = (n + wpb - 1) / wpb;
  if (blocks > 152 * 16) blocks = 152 * 16;
  encode_reads_wide_kernel<<<(unsigned)blocks, wpb * 32, smem, st>>>(tb, seqs, offsets, n, emb_f32,
                                                                       reinterpret_cast<__nv_bfloat16*>(emb_bf16),
                                                                       norms, status, perm, rc);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- reference pre-pass

// One warp per anchor chunk of A windows, in FP64. The chunk's first window is
// summed directly (§2.1-§2.3); it is stored in FP32 as the anchor that seeds
// the on-chip FP32 recurrence. The chunk is then walked with the slide
// relations of §3.4 in FP64 and every window's squared norm (and per-band
// norms for score_mode 1) is reduced across the warp, so the stored
// 1/sqrt(C_j) does not inherit the FP32 recurrence's drift.
__global__ void prepass_kernel(DevIndex ix, PrepassTables pt, float2* __restrict__ anchors,
                               float* __restrict__ inv_norm, float* __restrict__ band_norm) {
  extern __shared__ double2 pre_acc[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int wpb = blockDim.x >> 5;
  double2* acc = pre_acc + (size_t)warp * ix.D;
  const int64_t n_chunks = (ix.W + ix.A - 1) / ix.A;
  const int n_loc = ix.N - ix.s + 1;
  const int S = ix.stride;
  for (int64_t a = (int64_t)blockIdx.x * wpb + warp; a < n_chunks; a += (int64_t)gridDim.x * wpb) {
    const int64_t j0 = a * ix.A;
    const int64_t w0 = j0 * S;
    for (int g = lane; g < ix.D; g += 32) acc[g] = make_double2(0.0, 0.0);
    __syncwarp();
    for (int loc0 = 0; loc0 < n_loc; loc0 += 32) {
      const int loc = loc0 + lane;
      const uint32_t b = loc < n_loc ? bin_at(ix.packed, w0 + loc, ix.s, ix.map_lsb) : 0u;
      const int cnt = min(32, n_loc - loc0);
      for (int jj = 0; jj < cnt; ++jj) {
        const uint32_t bj = __shfl_sync(0xffffffffu, b, jj);
        if (lane < ix.m) {
          const double2 ph = pt.phase[lane * n_loc + loc0 + jj];
          double2& v = acc[lane * ix.nb + bj];
          v.x += ph.x;
          v.y += ph.y;
        }
        __syncwarp();
      }
    }
    // registers: entries g = lane + 32*i
    double cr[4], ci[4];
    int kb[4], bb[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int g = lane + 32 * i;
      const bool v = g < ix.D;
      cr[i] = v ? acc[g].x : 0.0;
      ci[i] = v ? acc[g].y : 0.0;
      kb[i] = v ? g / ix.nb : 0;
      bb[i] = v ? g % ix.nb : -1;
      if (v) anchors[a * ix.D + g] = make_float2((float)cr[i], (float)ci[i]);
    }
    __syncwarp();
    const int64_t j_end = min(ix.W, j0 + ix.A);
    for (int64_t j = j0; j < j_end; ++j) {
      double part = 0.0;
#pragma unroll
      for (int i = 0; i < 4; ++i) part = fma(cr[i], cr[i], fma(ci[i], ci[i], part));
      double tot = part;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
      if (lane == 0) inv_norm[j] = tot > (double)kZeroNorm2 ? (float)(1.0 / sqrt(tot)) : 0.f;
      if (band_norm) {
        for (int k = 0; k < ix.m; ++k) {
          double pk = 0.0;
#pragma unroll
          for (int i = 0; i < 4; ++i)
            if (bb[i] >= 0 && kb[i] == k) pk = fma(cr[i], cr[i], fma(ci[i], ci[i], pk));
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) pk += __shfl_xor_sync(0xffffffffu, pk, o);
          if (lane == 0) band_norm[j * ix.m + k] = (float)pk;
        }
      }
      if (j + 1 < j_end) {
        const int64_t w = j * S;
        for (int u = 0; u < S; ++u) {
          const uint32_t bo = bin_at(ix.packed, w + u, ix.s, ix.map_lsb);
          const uint32_t bi = bin_at(ix.packed, w + ix.N - ix.s + 1 + u, ix.s, ix.map_lsb);
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            if (bb[i] == (int)bo) {
              const double2 e = pt.eout[kb[i] * S + u];
              cr[i] -= e.x;
              ci[i] -= e.y;
            }
            if (bb[i] == (int)bi) {
              const double2 e = pt.ein[kb[i] * S + u];
              cr[i] += e.x;
              ci[i] += e.y;
            }
          }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const double2 r = pt.rot[kb[i]];
          const double xr = cr[i], xi = ci[i];
          cr[i] = xr * r.x - xi * r.y;
          ci[i] = xr * r.y + xi * r.x;
        }
      }
    }
  }
}

cudaError_t launch_prepass(const DevIndex& ix, const PrepassTables& pt, float2* anchors, float* inv_norm,
                           float* band_norm, int* status, cudaStream_t st) {
  (void)status;
  const int64_t n_chunks = (ix.W + ix.A - 1) / ix.A;
  const int wpb = 4;
  int64_t blocks = (n_chunks + wpb - 1) / wpb;
  if (blocks > 152 * 64) blocks = 152 * 64;
  const size_t smem = (size_t)wpb * ix.D * sizeof(double2);
  prepass_kernel<<<(unsigned)blocks, wpb * 32, smem, st>>>(ix, pt, anchors, inv_norm, band_norm);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- a4: windows

// Each chain of D/4 lanes starts at one anchor and runs the FP32 recurrence
// through its chunk of A windows, storing the unnormalised c(j) of the
// requested windows. This is the generator the scans run, exposed for checks.
template <int D>
__global__ void window_embeddings_kernel(DevIndex ix, int64_t j_begin, int64_t count, float* __restrict__ out) {
  constexpr int LPC = Chain<D>::LPC;
  constexpr int CPW = 32 / LPC;
  const int lane = threadIdx.x & 31;
  const int lic = lane % LPC;
  const int64_t chain = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * CPW + lane / LPC;
  const int64_t a0 = j_begin / ix.A;
  const int64_t a = a0 + chain;
  const int64_t j_end = min(ix.W, j_begin + count);
  if (a * ix.A >= j_end) return;
  Chain<D> ch;
  ch.setup(ix, lic);
  ch.load(ix.anchors + a * ix.D, lic);
  const int S = ix.stride;
  const int64_t jlast = min(j_end, (a + 1) * ix.A);
  for (int64_t j = a * ix.A; j < jlast; ++j) {
    if (j >= j_begin) {
      float* o = out + (j - j_begin) * 2 * D;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        o[4 * lic + i] = ch.cr[i];
        o[D + 4 * lic + i] = ch.ci[i];
      }
    }
    const int64_t w = j * S;
    if (S == 1) {
      ch.step1(bin_at(ix.packed, w, ix.s, ix.map_lsb), bin_at(ix.packed, w + ix.N - ix.s + 1, ix.s, ix.map_lsb));
    } else {
      for (int u = 0; u < S; ++u) {
        ch.sub_at(bin_at(ix.packed, w + u, ix.s, ix.map_lsb), ix.eout[ch.band * S + u]);
        ch.add_at(bin_at(ix.packed, w + ix.N - ix.s + 1 + u, ix.s, ix.map_lsb), ix.ein[ch.band * S + u]);
      }
      ch.rotate();
    }
  }
}

cudaError_t launch_window_embeddings(const DevIndex& ix, int64_t j_begin, int64_t count, float* out,
                                     cudaStream_t st) {
  const int64_t j_end = min(ix.W, j_begin + count);
  if (j_end <= j_begin) return cudaSuccess;
  const int64_t n_chains = (j_end - 1) / ix.A - j_begin / ix.A + 1;
  const int LPC = ix.D / 4;
  const int cpb = 4 * (32 / LPC);  // 4 warps per block
  const unsigned blocks = (unsigned)((n_chains + cpb - 1) / cpb);
  switch (ix.D) {
    case 4: window_embeddings_kernel<4><<<blocks, 128, 0, st>>>(ix, j_begin, count, out); break;
    case 8: window_embeddings_kernel<8><<<blocks, 128, 0, st>>>(ix, j_begin, count, out); break;
    case 16: window_embeddings_kernel<16><<<blocks, 128, 0, st>>>(ix, j_begin, count, out); break;
    case 32: window_embeddings_kernel<32><<<blocks, 128, 0, st>>>(ix, j_begin, count, out); break;
    case 64: window_embeddings_kernel<64><<<blocks, 128, 0, st>>>(ix, j_begin, count, out); break;
    case 128: window_embeddings_kernel<128><<<blocks, 128, 0, st>>>(ix, j_begin, count, out); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace rope
