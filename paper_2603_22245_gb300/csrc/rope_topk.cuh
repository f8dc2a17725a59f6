// Per-thread candidate list used by the scan epilogues: cand_depth entries of
// (score, window number) held in shared memory, entry-major ([e][thread]) so
// that a warp's accesses fall in distinct banks. The list keeps the best
// entries by (score descending, window ascending); with sep > 0 it keeps at
// most one window per bucket floor(start/sep), the best one. The worst entry
// and its score (thr) are cached so that the scan compares each score with
// one register and enters this code only on an improvement.
#pragma once

#include <stdint.h>

namespace rope {

constexpr uint32_t kEmptyWin = 0xFFFFFFFFu;
// First entry of a candidate slot that holds no list: the tensor-core scan
// keeps one list across consecutive ranges of a read group and writes it to
// the slot of the first range; the later ranges' slots carry this mark.
constexpr uint32_t kUnusedWin = 0xFFFFFFFEu;

__device__ __forceinline__ bool cand_better(float s1, uint32_t j1, float s2, uint32_t j2) {
  return s1 > s2 || (s1 == s2 && j1 < j2);
}

struct ThreadList {
  float* s;       // &list_s[thread]
  uint32_t* w;    // &list_w[thread]
  int stride;     // threads per entry row
  int depth;
  int worst;
  float thr;

  __device__ __forceinline__ float S(int e) const { return s[e * stride]; }
  __device__ __forceinline__ uint32_t Wn(int e) const { return w[e * stride]; }

  __device__ __forceinline__ void reset() {
    for (int e = 0; e < depth; ++e) {
      s[e * stride] = -INFINITY;
      w[e * stride] = kEmptyWin;
    }
    worst = 0;
    thr = -INFINITY;
  }

  // new worst entry: the lowest score, the highest window among equal scores;
  // scores read 8 at a time so the loads' latencies overlap
  __device__ __forceinline__ void rescan() {
    int wi = 0;
    float ws = INFINITY;
    uint32_t ww = 0;
    for (int e0 = 0; e0 < depth; e0 += 8) {
      float se[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) se[u] = e0 + u < depth ? S(e0 + u) : INFINITY;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if (se[u] > ws) continue;
        const uint32_t we = Wn(e0 + u);
        if (se[u] < ws || we > ww) {
          wi = e0 + u;
          ws = se[u];
          ww = we;
        }
      }
    }
    worst = wi;
    thr = ws;
  }

  // window number j starts at j*stride_pos; buckets are floor(start / sep).
  __device__ __forceinline__ void insert(float sc, uint32_t j, int sep, int stride_pos) {
    if (sep > 0) {
      const int64_t bucket = (int64_t)j * stride_pos / sep;
      for (int e = 0; e < depth; ++e) {
        const uint32_t we = Wn(e);
        if (we != kEmptyWin && (int64_t)we * stride_pos / sep == bucket) {
          if (cand_better(sc, j, S(e), we)) {
            s[e * stride] = sc;
            w[e * stride] = j;
            rescan();
          }
          return;
        }
      }
    }
    if (!cand_better(sc, j, S(worst), Wn(worst))) return;
    s[worst * stride] = sc;
    w[worst * stride] = j;
    rescan();
  }
};

// The same list update as a free function for the tensor-core epilogue: it is
// out of line (called rarely; inlining it at every score position would bloat
// the hot loop's instruction stream) and returns the new worst entry and its
// score by value, so the caller keeps the filter threshold in a register.
struct ListState {
  float thr;
  int worst;
};

static __device__ __noinline__ ListState list_insert(float* ls, uint32_t* lw, int stride, int depth, int worst, float sc,
                                             uint32_t j, int sep, int stride_pos) {
  ThreadList t;
  t.s = ls;
  t.w = lw;
  t.stride = stride;
  t.depth = depth;
  t.worst = worst;
  t.thr = ls[worst * stride];
  t.insert(sc, j, sep, stride_pos);
  return ListState{t.thr, t.worst};
}

}  // namespace rope
