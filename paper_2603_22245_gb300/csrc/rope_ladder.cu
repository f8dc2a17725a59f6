// Length ladder: reads of different lengths are mapped by their heads, each
// read with the longest window length of the ladder that it covers (§3.5 fixes
// one window length N shorter than the reads and maps the read head; a ladder
// of lengths applies that per read). These kernels bucket the reads and sort
// them stably by bucket, so the reads of one bucket occupy consecutive rows in
// input order and are scanned as one batch against that bucket's index.
//
//   ladder_hist_kernel     bucket of each read; per-block bucket histograms
//   ladder_offsets_kernel  exclusive scan of the histograms (bucket-major):
//                          first row of (bucket, block), bucket sizes
//   ladder_scatter_kernel  stable rank of each read inside its block -> row
#include "rope_internal.h"

namespace rope {

namespace {

constexpr int kLadderThreads = 1024;

__global__ void ladder_hist_kernel(const int64_t* __restrict__ offsets, int64_t n, const int32_t* __restrict__ lens,
                                   int nbk, int32_t* __restrict__ bucket, int32_t* __restrict__ out_len,
                                   int64_t* __restrict__ hist) {
  __shared__ int32_t h[kLadderMaxBuckets];
  for (int i = threadIdx.x; i < nbk; i += blockDim.x) h[i] = 0;
  __syncthreads();
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n) {
    const int64_t len = offsets[r + 1] - offsets[r];
    int lo = 0, hi = nbk;  // number of ladder lengths <= len
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if ((int64_t)lens[mid] <= len)
        lo = mid + 1;
      else
        hi = mid;
    }
    const int b = lo - 1;
    bucket[r] = b;
    if (out_len) out_len[r] = b >= 0 ? lens[b] : -1;
    if (b >= 0) atomicAdd(&h[b], 1);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nbk; i += blockDim.x) hist[(size_t)i * gridDim.x + blockIdx.x] = h[i];
}

// One block. hist[b * n_blk + blk] -> first row of (bucket b, block blk);
// base[b] = first row of bucket b, count[b] = its size.
__global__ void ladder_offsets_kernel(int64_t* __restrict__ hist, int64_t n_entries, int nbk, int64_t n_blk,
                                      int64_t* __restrict__ base, int64_t* __restrict__ count) {
  __shared__ int64_t part[kLadderThreads];
  const int t = threadIdx.x;
  const int64_t seg = (n_entries + blockDim.x - 1) / blockDim.x;
  const int64_t e0 = t * seg < n_entries ? t * seg : n_entries;
  const int64_t e1 = e0 + seg < n_entries ? e0 + seg : n_entries;
  int64_t sum = 0;
  for (int64_t e = e0; e < e1; ++e) sum += hist[e];
  part[t] = sum;
  __syncthreads();
  // inclusive scan of the segment sums (Hillis-Steele)
  for (int o = 1; o < (int)blockDim.x; o <<= 1) {
    const int64_t v = t >= o ? part[t - o] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  int64_t run = part[t] - sum;  // exclusive prefix of this segment
  for (int64_t e = e0; e < e1; ++e) {
    const int64_t v = hist[e];
    hist[e] = run;
    run += v;
  }
  __syncthreads();
  const int64_t total = part[blockDim.x - 1];
  for (int b = t; b < nbk; b += blockDim.x) {
    const int64_t first = hist[(size_t)b * n_blk];
    const int64_t next = b + 1 < nbk ? hist[(size_t)(b + 1) * n_blk] : total;
    base[b] = first;
    count[b] = next - first;
  }
}

__global__ void ladder_scatter_kernel(const int32_t* __restrict__ bucket, int64_t n, int nbk,
                                      const int64_t* __restrict__ first, int64_t* __restrict__ perm) {
  __shared__ int32_t wc[kLadderThreads / 32][kLadderMaxBuckets];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < (kLadderThreads / 32) * kLadderMaxBuckets; i += blockDim.x) (&wc[0][0])[i] = 0;
  __syncthreads();
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int b = r < n ? bucket[r] : -1;
  const uint32_t same = __match_any_sync(0xffffffffu, b);
  const int rank = __popc(same & ((1u << lane) - 1u));
  if (b >= 0 && rank == 0) wc[warp][b] = __popc(same);
  __syncthreads();
  if (b >= 0) {
    int before = rank;
    for (int w = 0; w < warp; ++w) before += wc[w][b];
    perm[first[(size_t)b * gridDim.x + blockIdx.x] + before] = r;
  }
}

}  // namespace

int64_t ladder_hist_entries(int64_t n_reads, int nbk) {
  return ((n_reads + kLadderThreads - 1) / kLadderThreads) * (int64_t)nbk;
}

cudaError_t launch_ladder_sort(const int64_t* offsets, int64_t n, const int32_t* lens, int nbk, int32_t* bucket,
                               int32_t* out_len, int64_t* hist, int64_t* base, int64_t* count, int64_t* perm,
                               cudaStream_t st) {
  if (nbk < 1 || nbk > kLadderMaxBuckets) return cudaErrorInvalidValue;
  const int64_t n_blk = (n + kLadderThreads - 1) / kLadderThreads;
  if (n_blk == 0) return cudaMemsetAsync(count, 0, sizeof(int64_t) * nbk, st);
  ladder_hist_kernel<<<(unsigned)n_blk, kLadderThreads, 0, st>>>(offsets, n, lens, nbk, bucket, out_len, hist);
  ladder_offsets_kernel<<<1, kLadderThreads, 0, st>>>(hist, n_blk * nbk, nbk, n_blk, base, count);
  ladder_scatter_kernel<<<(unsigned)n_blk, kLadderThreads, 0, st>>>(bucket, n, nbk, hist, perm);
  return cudaGetLastError();
}

__global__ void fill_empty_kernel(int64_t* __restrict__ win, float* __restrict__ score, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    win[i] = -1;
    score[i] = -INFINITY;
  }
}

cudaError_t launch_fill_empty(int64_t* win, float* score, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int64_t blocks = (n + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  fill_empty_kernel<<<(unsigned)blocks, 256, 0, st>>>(win, score, n);
  return cudaGetLastError();
}

}  // namespace rope
