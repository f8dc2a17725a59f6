// Host-side merge of per-shard top-k lists (window-range sharding across
// GPUs). Each shard scanned a disjoint window range and reported, per read,
// its best k windows by (score descending, start ascending), missing entries
// as (-1, -inf). The merge keeps, per read, the best k over all shards with the
// same order; with sep > 0 it keeps at most one window per bucket
// floor(start/sep), the best, which is exact as long as every shard kept its
// own best k buckets (a bucket split by a shard boundary appears in both lists
// and is collapsed here).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "rotormap.h"

extern "C" rope_status rope_merge_shards_host(const int64_t* win_host, const float* score_host, int32_t n_shards,
                                              int64_t n_reads, int32_t k_in, int32_t k_out, int32_t sep,
                                              int64_t* out_win_host, float* out_score_host) {
  if (n_shards < 1 || n_reads < 0 || k_in < 1 || k_out < 1 || sep < 0) return ROPE_ERR_INVALID_ARG;
  if (n_reads > 0 && (!win_host || !score_host || !out_win_host || !out_score_host)) return ROPE_ERR_INVALID_ARG;
  struct E {
    float s;
    int64_t w;
  };
  std::vector<E> all;
  for (int64_t r = 0; r < n_reads; ++r) {
    all.clear();
    for (int32_t sh = 0; sh < n_shards; ++sh) {
      const size_t base = ((size_t)sh * n_reads + r) * k_in;
      for (int32_t e = 0; e < k_in; ++e)
        if (win_host[base + e] >= 0) all.push_back(E{score_host[base + e], win_host[base + e]});
    }
    std::sort(all.begin(), all.end(), [](const E& a, const E& b) { return a.s > b.s || (a.s == b.s && a.w < b.w); });
    int32_t got = 0;
    std::vector<int64_t> taken;
    for (const E& e : all) {
      if (got == k_out) break;
      if (sep > 0) {
        const int64_t b = e.w / sep;
        if (std::find(taken.begin(), taken.end(), b) != taken.end()) continue;
        taken.push_back(b);
      }
      out_win_host[r * k_out + got] = e.w;
      out_score_host[r * k_out + got] = e.s;
      ++got;
    }
    for (; got < k_out; ++got) {
      out_win_host[r * k_out + got] = -1;
      out_score_host[r * k_out + got] = -INFINITY;
    }
  }
  return ROPE_OK;
}
