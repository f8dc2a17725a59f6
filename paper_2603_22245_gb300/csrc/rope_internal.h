// Host-side interface between the C ABI (rope_api.cu) and the kernel
// launchers of the other translation units.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "rope_common.cuh"

namespace rope {

// Tables a read encoder needs (device pointers).
struct EncTables {
  int32_t N, s, m, t, nb, D;
  const uint16_t* map;   // [4^s] bin of the s-mer code (first letter most significant)
  const float2* phase;   // [m * (N-s+1)] exp(2 pi i f_k loc / N)
};

struct Candidate {
  float score;
  uint32_t win;  // window number; 0xFFFFFFFF = empty
};

// Arguments shared by the scan kernels.
struct ScanArgs {
  const float* emb_f32;      // [n_reads, 2D] unnormalised (FP32 scan)
  const uint16_t* emb_bf16;  // [n_reads, 2D] normalised bf16 (tensor-core scan)
  const float* norms;        // [n_reads, 1+m]
  int64_t n_reads;
  int64_t jb, je;            // scanned windows [jb, je)
  int64_t st0;               // first super-tile start (multiple of the super-tile)
  int64_t range_len;         // windows per range (multiple of the super-tile)
  int32_t n_ranges;
  int32_t n_groups;
  int32_t cand_depth;        // candidates kept per read per range
  int32_t sep;
  Candidate* cand;           // [n_reads, n_ranges * lists_per_range, cand_depth]
  float* dense;              // [n_reads, je-jb] (dense mode)
  int* status;
  int32_t lists_per_range;   // candidate lists a scan keeps per read and range
  uint64_t wait_limit_ns;    // bound of every in-kernel wait
  int32_t tc_variant;        // tile variant of the tensor-core scan (< scan_tc_variants(D))
  int32_t fp8;               // tensor-core scan with E4M3 operands instead of BF16
};

struct MergeArgs {
  const Candidate* cand;
  int64_t n_reads;
  int32_t n_ranges, cand_depth, k, sep, rescore, rescore_depth;
  const float* emb_f32;
  const float* norms;
  int64_t* out_win;
  float* out_score;
  const int64_t* out_row;  // output row of read r (null: row r)
  int* status;
  // when the status word already carries the timeout bit (a scan of this call
  // gave up), write (-1, -inf) for every read instead of merging
  int32_t empty_on_timeout;
  // if not null, the status bits of this call (the scan's and the merge's)
  // are also OR-ed into this word
  int* sticky_status;
};

// rope_ladder.cu
constexpr int kLadderMaxBuckets = 64;
// entries of the per-block histogram scratch (int64) for n_reads reads
int64_t ladder_hist_entries(int64_t n_reads, int nbk);
// bucket of each read (largest lens[j] <= length, -1 if none; out_len = that
// length, may be null) and a stable sort of the bucketed reads by bucket:
// perm[base[b] + i] = i-th read of bucket b, count[b] = size of bucket b
cudaError_t launch_ladder_sort(const int64_t* offsets, int64_t n, const int32_t* lens, int nbk, int32_t* bucket,
                               int32_t* out_len, int64_t* hist, int64_t* base, int64_t* count, int64_t* perm,
                               cudaStream_t st);
cudaError_t launch_fill_empty(int64_t* win, float* score, int64_t n, cudaStream_t st);

// rope_encode.cu
cudaError_t launch_pack(const uint8_t* seq, int64_t len, uint32_t* out, int* status, cudaStream_t st);
cudaError_t launch_mer_bins(const uint32_t* packed, int64_t len, int64_t n_words, int s, const uint16_t* map_lsb,
                            uint16_t* out, cudaStream_t st);
// Row r encodes read perm[r] (perm null: read r); with rc, the head of the
// read's reverse complement.
cudaError_t launch_encode_reads(const EncTables& tb, const uint8_t* seqs, const int64_t* offsets, int64_t n,
                                float* emb_f32, uint16_t* emb_bf16, float* norms, int* status, cudaStream_t st,
                                const int64_t* perm = nullptr, bool rc = false);
// Per read, the best k of its forward-strand row r and reverse-strand row
// n + r of (win, score) [2n, k] by (score desc, forward first, start asc);
// strand 0 forward, 1 reverse, -1 for a missing entry.
cudaError_t launch_strand_merge(const int64_t* win2, const float* score2, int64_t n, int k, int64_t* out_win,
                                float* out_score, int8_t* out_strand, cudaStream_t st);
struct PrepassTables {
  const double2* phase;  // [m*(N-s+1)]
  const double2* rot;    // [m]
  const double2* eout;   // [m*stride]
  const double2* ein;    // [m*stride]
};
cudaError_t launch_prepass(const DevIndex& ix, const PrepassTables& pt, float2* anchors, float* inv_norm,
                           float* band_norm, int* status, cudaStream_t st);
cudaError_t launch_window_embeddings(const DevIndex& ix, int64_t j_begin, int64_t count, float* out,
                                     cudaStream_t st);

// rope_scan_fp32.cu
int scan_fp32_supported(int D);
int64_t scan_fp32_super_tile(int D);
int scan_fp32_group(int D);
cudaError_t launch_scan_fp32(const DevIndex& ix, const ScanArgs& a, bool dense, int num_sms, cudaStream_t st);

// rope_scan_tc.cu
int scan_tc_supported(int D);
int64_t scan_tc_super_tile(int D, int variant = 0);
int scan_tc_group(int D, int variant = 0);
int scan_tc_max_stride();
int scan_tc_variants(int D);
int scan_tc_lists_per_range(int D, int variant);
uint64_t wait_limit_ns();
cudaError_t launch_scan_tc(const DevIndex& ix, const ScanArgs& a, bool dense, int num_sms, cudaStream_t st);
// Output of the tensor-core scan's threshold mode: every pair with score >=
// thr[j] is appended at index atomicAdd(count, 1) when that index is < cap.
struct ThrOut {
  const float* thr;  // [W] per-window thresholds
  unsigned long long* count;
  int64_t cap;
  int64_t* read;
  int64_t* win;      // window number j
  float* score;
};
// threshold mode of the tensor-core scan (BF16, tile variant 0 at d = 64, or d = 128)
cudaError_t launch_scan_tc_threshold(const DevIndex& ix, const ScanArgs& a, const ThrOut& out, int num_sms,
                                     cudaStream_t st);
// whether the tensor-core scan's shared memory holds candidate lists of this depth
int scan_tc_fits(const DevIndex& ix, int cand_depth, int variant, int fp8);

// rope_merge.cu
cudaError_t launch_merge(const DevIndex& ix, const MergeArgs& a, cudaStream_t st);

// rope_dense.cu: materialised window index (wide encodings) and its GEMM scan
struct DenseTables {
  int32_t n_blk;         // whole blocks of `stride` starts summed per window
  int32_t t0, n_t;       // tail: window-relative starts [t0, t0 + n_t), signs folded into tph
  int64_t n_blocks;      // block sums built (W + n_blk - 1)
  const float2* bph;     // [m * stride] exp(2 pi i f_k i / N), i < stride
  const float2* rotu;    // [n_blk * m] exp(2 pi i f_k u stride / N)
  const float2* tph;     // [m * n_t] +-exp(2 pi i f_k (t0 + i) / N)
};
// block sums into bsum [n_blocks, D] (scratch), then every window's FP32 row
// [W, 2D], normalised BF16 rows [cr | ci] and [ci | -cr] ([W, 2D] each) and
// 1/|c| [W]
cudaError_t launch_dense_index(const DevIndex& ix, const DenseTables& dt, float2* bsum, float* win_f32,
                               uint16_t* win_bf16, uint16_t* win_bf16_im, float* inv_norm, cudaStream_t st);
// the scan's A operand [n_pad, 2D]: the reads' [xr | xi] rows, zero past n
cudaError_t launch_gemm_a(const uint16_t* emb, int64_t n, int64_t n_pad, int D, uint16_t* a, cudaStream_t st);
struct GemmArgs {
  int64_t n_reads;
  int32_t n_rt;          // read tiles of 128
  int32_t grp;           // read tiles per wave
  int32_t n_ranges;      // window ranges (candidate lists per read)
  int32_t k_blocks;      // 2D / 64
  int32_t stages;        // shared-memory pipeline depth
  int64_t jb, je;        // scanned windows [jb, je)
  int64_t range_len;     // windows per range (multiple of 128)
  int32_t cand_depth, sep, stride;
  Candidate* cand;       // [n_reads, n_ranges, cand_depth]
  float* dense;          // [n_reads, je - jb] (dense mode)
  int* status;
  uint64_t wait_limit_ns;
  ThrOut thr;            // threshold mode: every score >= thr.thr[j] appended
};
// rope_pairs.cu: mutated copies (the threshold regime's walk), §2.4 pair
// fidelities, per-window thresholds of the materialised index
struct MutArgs {
  const uint8_t* seqs;      // strings mode: ASCII strings seqs[offsets[i], offsets[i+1]) (null: windows mode)
  const int64_t* offsets;
  const double* errs;       // strings mode: rate of copy i
  const uint32_t* packed;   // windows mode: packed reference, windows j0 + i / n_samples
  int64_t L, j0;
  int32_t stride, n_samples;
  double err;               // windows mode: rate
  int64_t n;                // copies
  int32_t N;                // letters per copy
  uint64_t seed;
  uint8_t* out;             // [n, N] ASCII
  int* status;
};
cudaError_t launch_mutate(const MutArgs& a, cudaStream_t st);
// out[i] = fidelity of rows i and n + i of emb [2n, 2D] (FP32 encodings, norms [2n, 1 + m])
cudaError_t launch_pair_fidelity(const float* emb, const float* norms, int64_t n, int D, int m, int nb,
                                 int score_mode, float* out, cudaStream_t st);
// out[w] = mean over t of the fidelity between window j0 + w's stored FP32 row
// and row w * n_samples + t of emb (materialised index)
cudaError_t launch_window_thresholds(const DevIndex& ix, const float* emb, const float* norms, int64_t j0,
                                     int64_t count, int n_samples, float* out, cudaStream_t st);
cudaError_t launch_iota_offsets(int64_t* off, int64_t n, int64_t N, cudaStream_t st);

// FP32 plain scan of a materialised index (reads' FP32 encodings against the
// stored FP32 rows, CUDA cores): per-read lists into g.cand, items as the GEMM's
int dense_fp32_group();    // reads per tile (64)
cudaError_t launch_dense_fp32(const DevIndex& ix, const GemmArgs& g, const float* emb, const float* norms, int num_sms,
                              cudaStream_t st);
int gemm_tc_group();       // reads per tile
int gemm_tc_window_tile(); // windows per tile
int gemm_tc_stages(int cand_depth, int k_blocks);  // deepest pipeline that fits (0: none)
int gemm_tc_lists(int k_blocks);     // candidate lists per (read, window range)
// mode 0: top-k lists, 1: every score (dense), 2: threshold pairs
cudaError_t launch_gemm_tc(const CUtensorMap& tmA, const CUtensorMap& tmB, const CUtensorMap& tmBi,
                           const GemmArgs& g, int mode, int num_sms, cudaStream_t st);

// rope_rerank.cu
constexpr int kMaxFeatures = 32;
struct MlpWeights {
  int32_t F, H;
  __nv_bfloat16* W1;  // [H, F]
  float* b1;          // [H]
  __nv_bfloat16* w2;  // [H]
  float* b2;          // [1]
};
cudaError_t launch_levenshtein(const uint32_t* packed, const uint8_t* seqs, const int64_t* offsets,
                               const int64_t* read_idx, const int64_t* win_start, int64_t n_pairs, int N, int32_t* out,
                               cudaStream_t st);
// kShift: largest letter shift of the Hamming features
constexpr int kShift = 4;
cudaError_t launch_features(const DevIndex& ix, const uint8_t* seqs, const int64_t* offsets, const float* emb_f32,
                            const float* norms, const int64_t* cand_win, const float* cand_score, int64_t n_reads,
                            int K, int F, float* X, cudaStream_t st);
cudaError_t launch_mlp_forward(const MlpWeights& w, const float* X, const int64_t* idx, int64_t B, float* y, float* pre,
                               const float* t, float* dy, float* sq, cudaStream_t st);
cudaError_t launch_mlp_backward(const MlpWeights& w, const float* X, const int64_t* idx, int64_t B, const float* pre,
                                const float* dy, const float* sq, float* grad, float* loss, int accumulate,
                                cudaStream_t st);
cudaError_t launch_adamw(const MlpWeights& w, const float* grad, float* master, float* m1, float* m2, int64_t step,
                         float lr, float beta1, float beta2, float eps, float wd, cudaStream_t st);
cudaError_t launch_ld_fraction(const int32_t* ld, int64_t n, int N, float* out, cudaStream_t st);
cudaError_t launch_rank_as_prediction(int64_t n_reads, int K, float* pred, cudaStream_t st);
cudaError_t launch_prune(const int64_t* cand_win, const float* cand_score, const float* pred, int64_t n_reads, int K,
                         int keep, int64_t* out_win, float* out_score, float* out_pred, cudaStream_t st);

}  // namespace rope
