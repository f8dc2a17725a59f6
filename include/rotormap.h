/*
 * rotormap.h — C ABI of the GB300 (sm_103a) RotorMap hot path.
 *
 * RotorMap (§3) maps a DNA read to a reference by encoding the read's head of
 * length N with the RoPE encoding (§2) and scoring it against the encoding of
 * every length-N window of the reference (§3.1), keeping the best loci
 * (§3.5). This library computes, on one GPU:
 *   - the 2-bit packing of letters and the s-mer bin codes (§2.1, §2.6),
 *   - the RoPE encodings of read heads by direct summation (§2.1-§2.3, §3.3),
 *   - the encodings of all reference windows, generated on chip by the
 *     slide-by-one recurrence of §3.4 from periodic exact anchors (never stored),
 *   - the read x window fidelity |<x|c>|^2/(|x|^2 |c|^2) (§2.4) as a real
 *     contraction (§4 identity) on the tensor cores (BF16 in, FP32 accumulate)
 *     or on the CUDA cores in FP32, fused with a per-read top-k (§3.5),
 *   - an FP32 re-scoring of the best candidates by direct summation.
 *
 * Conventions
 *   - Pointers are DEVICE pointers unless the name ends in _host.
 *   - Outputs are allocated by the caller. The library owns only rope_index
 *     objects and the per-call scratch it takes from its own stream-ordered
 *     memory pool (released back to the pool on the same stream).
 *   - Calls are asynchronous on `stream` unless stated otherwise. Errors found
 *     on the host are returned at once; errors found by a kernel (a letter
 *     outside {A,C,G,T}, a read shorter than N, a wait that ran out) are
 *     recorded in a device status word and returned by rope_sync_status().
 *   - Nothing is thrown across the ABI. rope_last_error() gives a per-thread
 *     message for the last failing call.
 *   - Letters: A,C,G,T in either case map to 0,1,2,3. Window j starts at
 *     reference position j*stride; window starts and counts are int64.
 *   - Vectors: an encoding has D = m*4^t complex entries, band-major (entry
 *     (k-1)*4^t + b for factor k and bin b). As reals it is stored
 *     [re_0..re_{D-1}, im_0..im_{D-1}] (2D floats).
 */
#ifndef ROTORMAP_H
#define ROTORMAP_H

#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  ROPE_OK = 0,
  ROPE_ERR_INVALID_ARG = 1,   /* bad parameter, size or pointer                  */
  ROPE_ERR_INVALID_BASE = 2,  /* a letter outside {A,C,G,T,a,c,g,t}              */
  ROPE_ERR_OOM = 3,           /* device allocation failed                        */
  ROPE_ERR_CUDA = 4,          /* a CUDA runtime call failed                      */
  ROPE_ERR_TIMEOUT = 5,       /* a bounded in-kernel wait ran out                */
  ROPE_ERR_UNSUPPORTED = 6    /* parameters valid but not built for this path    */
} rope_status;

/* Encoding and window parameters.
 *   s        s-mer length, 1 <= s <= 8 (§2.1)
 *   m        number of multiplicity factors, 1 <= m <= 8 (§2.2, §2.3)
 *   t        compact bin exponent, 1 <= t <= s: 4^s s-mers fold onto 4^t bins
 *            (§2.6); m*4^t <= 4096
 *   variant  0 = default factors f_k = k (§2.2 Eq. mult-factor),
 *            1 = fine-tuned f_k = 2(k-1)/(m-1)+1 (§3.3 Eq. mult-factor-finetune;
 *                f_1 = 1 when m = 1)
 *   score_mode 0 = fidelity of the concatenated normalised vector (§2.3, §2.4);
 *            1 = mean over k of per-band fidelities (§2.5)
 *   window_len N, the window and read-head length (§3.1), s <= N <= 65536
 *   stride   window step (§3.1), 1 <= stride <= 64
 *   bin_of_mer_host  4^s entries in [0, 4^t) mapping s-mer code
 *            sum_i base(p+i) 4^(s-1-i) to its bin; NULL selects the identity
 *            when s == t and Knuth's multiplicative hash
 *            (code * 0x9E3779B97F4A7C15 mod 2^64) >> (64-2t) otherwise. Copied
 *            at the call; the caller keeps ownership. */
typedef struct {
  int32_t s, m, t;
  int32_t variant;
  int32_t score_mode;
  int32_t window_len;
  int32_t stride;
  int32_t reserved0;
  const uint16_t* bin_of_mer_host;
} rope_params;

/* Scoring precision. ROPE_PREC_FP8 is the tensor-core scan with E4M3
 * operands (kind::f8f6f4, FP32 accumulation): the read's BF16 encoding and the
 * window's normalised encoding are each scaled by 2^5 and rounded to E4M3, and
 * the scores are scaled back by 2^-20 (exact); it takes emb_bf16 like
 * ROPE_PREC_BF16. Its raw scores carry the E4M3 rounding (3 mantissa bits);
 * with rescore = 1 the reported scores are the FP32 re-scores as for BF16. */
enum { ROPE_PREC_FP32 = 0, ROPE_PREC_BF16 = 1, ROPE_PREC_FP8 = 2 };

/* Options of rope_score_topk.
 *   k          results per read, 1 <= k <= 32
 *   sep        0: plain top-k. sep > 0: at most one window per bucket
 *              floor(start/sep) (the best), then the best k buckets
 *   precision  ROPE_PREC_FP32 (CUDA cores), ROPE_PREC_BF16 or ROPE_PREC_FP8
 *              (tensor cores)
 *   rescore    1: re-score the kept candidates by direct FP32 summation before
 *              the final ranking; 0: report the scan's own scores
 *   cand_depth candidates kept per read per window range and list (0 = 8,
 *              raised to k); k..32
 *   rescore_depth candidates re-scored per read (0 = 2*k, capped at 32)
 *   j_begin, j_end  window-number range [j_begin, j_end) scanned; j_end <= 0
 *              means all windows
 *   n_ranges   window ranges the scan is split into (0 = automatic) */
typedef struct {
  int32_t k;
  int32_t sep;
  int32_t precision;
  int32_t rescore;
  int32_t cand_depth;
  int32_t rescore_depth;
  int32_t n_ranges;
  int32_t reserved0;
  int64_t j_begin;
  int64_t j_end;
} rope_score_opts;

typedef struct rope_index rope_index;

/* Name of a status code (static string). */
const char* rope_status_string(rope_status st);

/* Message of the last failing call on this host thread (static storage). */
const char* rope_last_error(void);

/* Complex dimension m*4^t of valid params, else -1. */
int32_t rope_dim(const rope_params* p);

/* Synchronises `stream`, then returns and clears the device status word of
 * the current device: ROPE_OK, ROPE_ERR_INVALID_BASE, ROPE_ERR_INVALID_ARG
 * (a read shorter than N) or ROPE_ERR_TIMEOUT. */
rope_status rope_sync_status(cudaStream_t stream);

/* Bound of every in-kernel wait of later launches on any device, in seconds
 * (the paper has no counterpart: this is part of failure detection). The
 * default is 2 s, or the environment's ROPE_WAIT_LIMIT_S (clamped to
 * [0.05, 120]) for runs that slow kernels down on purpose, such as a profiler
 * replaying them. `seconds` in [1e-9, 120] sets the bound, 0 restores the
 * default; else ROPE_ERR_INVALID_ARG. A wait that runs out sets the timeout
 * bit (ROPE_ERR_TIMEOUT from rope_sync_status); the kernel then waits (at
 * least 1 s more) for its own copies and tensor-core operations in flight,
 * frees its tensor memory and returns, so the context stays usable. Bounds of
 * nanoseconds make every wait that is not satisfied at once run out: the
 * tests of this path use them. Launches captured in a CUDA graph keep the
 * bound in force when they were captured. */
rope_status rope_set_wait_limit(double seconds);

/* ---- step a1: 2-bit packing (§2.1 alphabet) ------------------------------
 * seq: len letters (uint8). out_words: ceil(len/16) uint32; base i goes to
 * bits 2*(i mod 16) of word i/16, unused high bits of the last word are 0.
 * An invalid letter sets ROPE_ERR_INVALID_BASE in the status word. */
rope_status rope_pack_2bit(const uint8_t* seq, int64_t len, uint32_t* out_words, cudaStream_t stream);

/* ---- step a2: s-mer bins (§2.1 locations, §2.6 compact map) -------------
 * packed: words from rope_pack_2bit for a sequence of `len` letters.
 * out_bins: len-s+1 uint16, out_bins[p] = bin of the s-mer at location p. */
rope_status rope_mer_bins(const rope_params* p, const uint32_t* packed, int64_t len, uint16_t* out_bins,
                          cudaStream_t stream);

/* ---- reference index (§3.1) ---------------------------------------------
 * ref: len letters on the device. Packs the reference, and for every window
 * j < W = floor((len-N)/stride)+1 computes its squared norm exactly enough
 * (FP64 recurrence from FP64 anchors) to store 1/sqrt(C_j) in FP32 (0 for a
 * zero vector, whose fidelity is 0), per-band norms when score_mode = 1, and
 * the FP32 anchors c(j) every 64 windows that seed the on-chip recurrence
 * (the on-the-fly index: stride <= 64, complex dimension m*4^t <= 128; the
 * scans regenerate every window on chip). Encodings wider than 128 complex
 * dimensions get the materialised index of rope_encode_reference_dense
 * instead. Requires 1 <= W < 2^32. Synchronous: returns after the index is
 * built. *out receives a new index owned by the caller (free with
 * rope_index_free). */
rope_status rope_encode_reference(const rope_params* p, const uint8_t* ref, int64_t len, rope_index** out,
                                  cudaStream_t stream);

/* Materialised index (§3.1's "database of vectors", sized in §3.2 for 20 kbp
 * reads: window 20,000, step 1,250, 1024 complex dimensions). Stores every
 * window's encoding on the device -- FP32 [W, 2D] unnormalised (re block, im
 * block; for re-scoring and the FP32 scan) and, divided by its norm, the two
 * BF16 [W, 2D] tensor-core operands [cr | ci] and [ci | -cr] -- plus 1/|c_j|
 * in FP32: W * 2D * 8 bytes (41 GB for a 3.1 Gbp genome at those settings),
 * and 8 * D bytes per window of scratch during the build. Each window is
 * summed exactly from per-block sums over blocks of `stride` s-mer starts (no
 * recurrence, no drift; FP32). Any stride (1..65536); D = m*4^t a multiple of
 * 32, at most 4096; score_mode 0; W < 2^31. rope_score_topk / rope_map /
 * rope_map_strands / rope_score_dense / rope_score_threshold on it run the
 * BF16 tensor-core GEMM (ROPE_PREC_BF16) with the top-k fused into its
 * epilogue and re-score in FP32 from the stored rows; the top-k calls also
 * take ROPE_PREC_FP32 (a plain CUDA-core scan over the FP32 rows). Other
 * precisions and the other scans refuse it (ROPE_ERR_UNSUPPORTED). Synchronous. */
rope_status rope_encode_reference_dense(const rope_params* p, const uint8_t* ref, int64_t len, rope_index** out,
                                        cudaStream_t stream);

/* Frees an index (NULL is allowed). Synchronises the device first. */
void rope_index_free(rope_index* idx);

/* Index facts: number of windows, reference length, anchor period, and the
 * device arrays (packed words, 1/sqrt(C_j)); any output pointer may be NULL. */
rope_status rope_index_info(const rope_index* idx, int64_t* n_windows, int64_t* ref_len, int32_t* anchor_period,
                            const uint32_t** packed, const float** inv_norm);

/* ---- step a4: window encodings (§3.4 recurrence), for inspection --------
 * Writes c(j) for j in [j_begin, j_begin+count) as count x 2D floats,
 * unnormalised, generated by the same on-chip recurrence the scans use. */
rope_status rope_window_embeddings(const rope_index* idx, int64_t j_begin, int64_t count, float* out,
                                   cudaStream_t stream);

/* ---- step a3: read encoding (§2.1-§2.3, §3.3) ---------------------------
 * seqs: concatenated reads (uint8 letters); offsets: n_reads+1 int64 (read r
 * is seqs[offsets[r], offsets[r+1])); only the head of length N is encoded
 * and every read must have at least N letters.
 *   emb_f32  n_reads x 2D floats, the unnormalised encoding (may be NULL)
 *   emb_bf16 n_reads x 2D bf16 (uint16 bits), the encoding divided by its norm
 *            (zero for a zero vector); the tensor-core operand (may be NULL)
 *   norms    n_reads x (1+m) floats: |x|^2, then |x_k|^2 per band (required) */
rope_status rope_encode_reads(const rope_params* p, const uint8_t* seqs, const int64_t* offsets, int64_t n_reads,
                              float* emb_f32, uint16_t* emb_bf16, float* norms, cudaStream_t stream);

/* ---- steps a4-a7: scan, fidelity, top-k, re-scoring (§3.1, §3.4, §3.5) --
 * Scores every read against every window in the range and writes, per read,
 * k window starts (int64, j*stride) and fidelities (float), best first
 * (score descending, start ascending); missing entries are (-1, -inf).
 * emb_f32/norms come from rope_encode_reads; emb_bf16 is required for
 * ROPE_PREC_BF16 and ROPE_PREC_FP8. Uses scratch from the library's stream-ordered pool. */
rope_status rope_score_topk(const rope_index* idx, const float* emb_f32, const uint16_t* emb_bf16,
                            const float* norms, int64_t n_reads, const rope_score_opts* opts, int64_t* out_win,
                            float* out_score, cudaStream_t stream);

/* Allocation-free variant of rope_score_topk (the paper has no counterpart:
 * this is for callers, not for the method). For callers that must not have
 * the library allocate device memory during the call -- e.g. a process that
 * gives nearly all device memory to its own arena at start-up, or a
 * latency-critical loop that cannot take the device-wide synchronisation of
 * cudaMalloc/cudaFree. Same arguments, results and kernels as
 * rope_score_topk (the split of the windows into ranges may differ, which
 * does not change the result: the union of per-range top lists always holds
 * the overall top list); the caller still passes the inputs and outputs. The
 * scratch (status words + candidate lists) is a 16 MiB array inside the
 * library that every GPU which loads the library holds until exit; a call
 * needing more (n_reads * n_ranges * cand_depth * 8 bytes beyond 16 MiB - 256 B)
 * is rejected with ROPE_ERR_INVALID_ARG and a message giving the limit
 * (n_ranges = 0 picks the largest split that fits). No cudaMalloc, cudaFree
 * or pool allocation happens; every call sets its candidate lists empty
 * (cudaMemsetAsync, at most 16 MiB) before the scan. The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress), so make
 * that first call before any stream capture on that device. All calls on a
 * device share the one array: calls that overlap on the GPU (e.g. on two
 * streams at once) race and corrupt each other's results; serialise them. A
 * bounded in-kernel wait that runs out during a call makes that call's
 * output (-1, -inf) for every read, and is recorded in the array's own status
 * word, which rope_noalloc_sync_status reads (not rope_sync_status). */
rope_status rope_score_topk_noalloc(const rope_index* idx, const float* emb_f32, const uint16_t* emb_bf16,
                                    const float* norms, int64_t n_reads, const rope_score_opts* opts,
                                    int64_t* out_win, float* out_score, cudaStream_t stream);

/* Status of the allocation-free calls on the current device: synchronises
 * `stream`, then returns and clears the bits every rope_score_topk_noalloc
 * call since the last read has recorded -- ROPE_OK, ROPE_ERR_TIMEOUT (a
 * bounded wait ran out; that call's output is (-1, -inf)) or
 * ROPE_ERR_INVALID_ARG (the merge found a corrupt candidate slot and skipped
 * it). Allocates nothing; no counterpart in the paper. */
rope_status rope_noalloc_sync_status(cudaStream_t stream);

/* ---- tuner (no counterpart in the paper) --------------------------------
 * The BF16 scan has tile variants and a free split of the work into
 * (read group, window range) items. On the first BF16 rope_score_topk /
 * rope_map call of a shape class (device, complex dimension, stride, window
 * length, read groups and scanned windows rounded up to powers of two,
 * cand_depth, sep on/off) with opts->n_ranges == 0, the library times each
 * variant with 8, 16 and 32 items per SM on that call's reads and windows and
 * keeps the fastest for the class; later calls of the class use it. Only
 * scans of at most 2^22 windows are timed (short samples of a longer scan
 * mispredict it: the cost per window falls with the scan's length); longer
 * ones keep the defaults (variant 0, 16 items per SM) unless set by hand.
 * Results do not depend on the choice.
 * Tuning is on unless the environment sets ROPE_AUTOTUNE=0; the
 * allocation-free entry point only reads earlier choices. */
rope_status rope_autotune_enable(int32_t enabled);  /* 0 also forgets earlier choices */
/* Records (variant, items per SM) for the class of (idx, n_reads, opts), as if
 * tuned: later calls of the class use it. variant < 2 at d = 64, 0 at d = 128. */
rope_status rope_autotune_set(const rope_index* idx, int64_t n_reads, const rope_score_opts* opts, int32_t variant,
                              int32_t items_per_sm);
/* The choice recorded for the class of (idx, n_reads, opts): tile variant,
 * items per SM and its measured scan time (ms; 0 if set by hand or kept as
 * the default);
 * ROPE_ERR_INVALID_ARG if none yet. */
rope_status rope_autotune_query(const rope_index* idx, int64_t n_reads, const rope_score_opts* opts,
                                int32_t* variant, int32_t* items_per_sm, float* sample_ms);

/* Every score of every read against windows [j_begin, j_begin+count), as
 * n_reads x count floats, computed by the same scan kernel as rope_score_topk
 * (FP32 or BF16 tensor-core path) with its top-k stage replaced by a store.
 * For parity checks on small cases. */
rope_status rope_score_dense(const rope_index* idx, const float* emb_f32, const uint16_t* emb_bf16,
                             const float* norms, int64_t n_reads, int32_t precision, int64_t j_begin, int64_t count,
                             float* out, cudaStream_t stream);

/* ---- the whole path (§3.1, §3.5) ----------------------------------------
 * Encodes the heads of the reads and scans them against the index; writes k
 * window starts and fidelities per read as rope_score_topk does. `opts` as
 * for rope_score_topk (j range ignored). Reads shorter than N are an error. */
rope_status rope_map(const rope_index* idx, const uint8_t* seqs, const int64_t* offsets, int64_t n_reads,
                     const rope_score_opts* opts, int64_t* out_win, float* out_score, cudaStream_t stream);

/* ---- threshold regime (§3.4 per-fragment thresholds, §3.5 multi-locus output)
 * rope_fragment_thresholds: for windows [j_begin, j_begin + count) of the
 * index, the threshold of window j for mutation rate err: the mean fidelity
 * (the index's score mode, FP32 sums) between the window and n_samples
 * mutated copies of it. A copy is the first N letters of a walk from the
 * window's start in which each reference letter is mutated with probability
 * err: deleted, preceded by a random inserted letter, or substituted by one
 * of the three other letters, each with probability 1/3 (past the reference
 * end the walk reads A). Its draws are SplitMix64 outputs: the stream keyed
 * by output j*n_samples + t of the generator started at `seed` (copy t),
 * outputs 3d, 3d+1, 3d+2 of that stream for reference letter d of the walk,
 * so the copies are fixed by (seed, j, t). n_samples: a power of two in
 * [1, 32]; complex dimension <= 64. out: count floats (device).
 *
 * rope_score_threshold: every (read, window) pair of windows [j_begin, j_end)
 * (j_end <= 0: all) whose BF16 tensor-core score (normalised operands, FP32
 * accumulation, as rope_score_topk's scan) is >= thr[j] (device, one float
 * per window of the index). The count of such pairs is written to
 * *out_count (device); the first min(count, cap) of them, in no particular
 * order, to out_read / out_win (window number j; start j*stride) /
 * out_score (device). A count above cap means pairs were dropped: call
 * again with a larger cap. Score mode 0, d = 64 (tile variant 0) or 128, or
 * a materialised index of any dimension. */
rope_status rope_fragment_thresholds(const rope_index* idx, double err, int32_t n_samples, uint64_t seed,
                                     int64_t j_begin, int64_t count, float* out, cudaStream_t stream);
/* On a materialised index (rope_encode_reference_dense) both calls take any
 * complex dimension: the copies are walked on the GPU, encoded by the read
 * encoder and compared with the windows' stored FP32 rows (pool scratch of
 * at most about 2 GB, a chunk of windows at a time), and the pairs come from
 * the GEMM scan's threshold mode. */
rope_status rope_score_threshold(const rope_index* idx, const uint16_t* emb_bf16, int64_t n_reads, const float* thr,
                                 int64_t j_begin, int64_t j_end, int64_t cap, int64_t* out_read, int64_t* out_win,
                                 float* out_score, unsigned long long* out_count, cudaStream_t stream);

/* ---- scoring of correlations (§2.4) ---------------------------------------
 * For each string i (seqs[offsets[i], offsets[i+1]) on the device, at least
 * N = p->window_len letters of A,C,G,T): the fidelity (p's score mode) between
 * the encoding of its first N letters and the encoding of its mutated copy at
 * rate errs[i] (double, device). The copy is the first N letters of the walk
 * of the threshold regime over the string (each letter mutated with
 * probability errs[i]: deleted, preceded by a random inserted letter, or
 * substituted, 1/3 each; A past the string's end), its draws the SplitMix64
 * stream keyed by output i of the generator started at `seed`. These are the
 * samples of the paper's fitting curve (mean fidelity per mutation rate,
 * inverted to predict the rate). Any complex dimension; FP32 encodings and
 * products. out_fid: n floats (device). Pool scratch: n*(N + 16*D + 8) bytes. */
rope_status rope_pair_fidelities(const rope_params* p, const uint8_t* seqs, const int64_t* offsets, int64_t n,
                                 const double* errs, uint64_t seed, float* out_fid, cudaStream_t stream);

/* ---- refinement (§3.4, increasing the accuracy) -------------------------
 * Slides the window one letter at a time around coarse candidates and scores
 * each position with the encoding p (which may differ from the index's: e.g.
 * s = t = 8, up to 4^8 bins per band, m <= 8), using the paper's O(1)-per-step
 * update of the inner product and an exactly tracked window norm (every bin's
 * sum kept on chip; the norm is not skipped).
 *   idx       supplies the 2-bit packed reference only (its own encoding is
 *             not used)
 *   p         s, m, t, variant, score_mode, bin map and window_len = N (the
 *             read head length); stride is ignored. N <= reference length.
 *   seqs, offsets, n_reads  reads as for rope_encode_reads (each >= N letters)
 *   cand_pos  n_reads x n_cand int64 window starts (device), 1 <= n_cand <= 64;
 *             a negative entry means no candidate; a start past the last
 *             window is taken as the last window
 *   radius    positions [c - radius, c + radius] clipped to [0, L - N] are
 *             scored, 0 <= radius <= 4096
 *   out_pos, out_fid  n_reads x n_cand (device): per candidate, the best
 *             position of its range (ties: the lower) and its fidelity (FP32;
 *             FP64 accumulation of the updates); (-1, -inf) where there is no
 *             candidate or the read is invalid (status word set as for
 *             rope_encode_reads)
 * Returns ROPE_ERR_UNSUPPORTED when the on-chip tables for (N, m, radius) do
 * not fit in one block's shared memory. */
rope_status rope_refine(const rope_index* idx, const rope_params* p, const uint8_t* seqs, const int64_t* offsets,
                        int64_t n_reads, const int64_t* cand_pos, int32_t n_cand, int32_t radius, int64_t* out_pos,
                        float* out_fid, cudaStream_t stream);

/* Both strands (§3.5 maps reads in both directions): each read is mapped by
 * its head and by the head of its reverse complement (the complement of its
 * last N letters, read backwards), both against the forward reference, and
 * the best k of the two candidate lists are kept by (score descending, the
 * forward strand first on equal scores, start ascending). out_strand int8
 * [n_reads, k]: 0 forward, 1 reverse complement, -1 for a missing entry. */
rope_status rope_map_strands(const rope_index* idx, const uint8_t* seqs, const int64_t* offsets, int64_t n_reads,
                             const rope_score_opts* opts, int64_t* out_win, float* out_score, int8_t* out_strand,
                             cudaStream_t stream);

/* ---- learned reranker (steps a8, a9) -------------------------------------
 * The paper relates fidelity to Levenshtein distance (§1, §2.4) and keeps
 * candidate loci by score or per-fragment thresholds (§3.3, §3.5). This
 * optional stage learns, from the scan's own score features, each candidate's
 * Levenshtein distance (§1) to the read head as a fraction of N, and keeps the
 * candidates with the smallest prediction. Network: y = w2 . GELU(W1 x + b1)
 * + b2 with exact GELU (z Phi(z)), W1 [hidden x F] and w2 stored in BF16, b1,
 * b2 and all arithmetic in FP32; FP32 master weights and AdamW state
 * (beta1 0.9, beta2 0.999, eps 1e-8, decoupled weight decay) for training.
 * Parameters are flattened as W1 (row-major), b1, w2, b2: P = H*F + 2H + 1. */
typedef struct rope_reranker rope_reranker;

/* New network on the current device: F in [1,32] features, H in [1,1024]
 * hidden units, Glorot-uniform weights from `seed`, zero biases. */
rope_status rope_reranker_create(int32_t n_features, int32_t hidden, uint64_t seed, rope_reranker** out);
void rope_reranker_free(rope_reranker* rr);
/* FP32 master parameters (P floats, host) and the number of training steps taken. Synchronising. */
rope_status rope_reranker_get(const rope_reranker* rr, float* params_host, int64_t* step);
/* Replaces the parameters (P floats, host); reset_optimizer zeroes the AdamW
 * moments and the step count. Synchronising. */
rope_status rope_reranker_set(rope_reranker* rr, const float* params_host, int32_t reset_optimizer);
/* Gradient (P floats, device) and mean squared error (device float) of the
 * batch {X[sample_idx[i]], t[sample_idx[i]] : i < B} (rows 0..B-1 when
 * sample_idx is NULL). X: rows of F floats. Deterministic reductions. */
rope_status rope_reranker_grad(rope_reranker* rr, const float* X, const float* t, const int64_t* sample_idx,
                               int64_t B, float* grad, float* loss, cudaStream_t stream);
/* One AdamW step on that batch; its mean squared error is added to *loss_sum
 * (device float) when loss_sum is not NULL. */
rope_status rope_reranker_train_step(rope_reranker* rr, const float* X, const float* t, const int64_t* sample_idx,
                                     int64_t B, float lr, float weight_decay, float* loss_sum, cudaStream_t stream);
/* y[b] for the B rows of X (device). */
rope_status rope_reranker_predict(const rope_reranker* rr, const float* X, int64_t B, float* y, cudaStream_t stream);
/* Checkpoint: "ROPERR01", int32 F, int32 H, int64 step, then P floats each of
 * parameters, first and second moments (little endian). Load requires the same
 * F and H and restores the training state exactly. */
rope_status rope_reranker_save(const rope_reranker* rr, const char* path);
rope_status rope_reranker_load(rope_reranker* rr, const char* path);

/* Exact Levenshtein distance (§1) between each read head (length N of the
 * index) and the reference window starting at win_start[i], for the pairs
 * (read_idx[i], win_start[i]); out_ld int32 [n_pairs], out_frac (may be NULL)
 * float distance / N. Bit-parallel DP (Myers; global form), N <= 256. */
rope_status rope_levenshtein(const rope_index* idx, const uint8_t* seqs, const int64_t* offsets,
                             const int64_t* read_idx, const int64_t* win_start, int64_t n_pairs, int32_t* out_ld,
                             float* out_frac, cudaStream_t stream);

/* Feature rows X [n_reads * K, F], F = K + 6 + m, for each read's K candidates
 * (cand_win/cand_score [n_reads, K] from rope_score_topk, best first):
 * the read's K scores (missing = 0), the candidate's fidelity, its m per-band
 * fidelities (§2.5, FP32 direct sums), rank / K, and four Hamming fingerprint
 * fidelities ((n - d)/n)^2 (§1) of the read head (seqs/offsets, the reads the
 * embeddings were made from): against the window, the best against the
 * windows shifted by -4..4 letters (letters outside the reference mismatch),
 * and of the head's first and second halves against the window's. Rows of
 * missing candidates (start -1) are zero. */
rope_status rope_rerank_features(const rope_index* idx, const uint8_t* seqs, const int64_t* offsets,
                                 const float* emb_f32, const float* norms, const int64_t* cand_win,
                                 const float* cand_score, int64_t n_reads, int32_t K, float* X, cudaStream_t stream);

/* Per read, the `keep` of its K candidates with the smallest pred (ties: higher
 * score, then lower start); out_* [n_reads, keep], missing (-1, -inf, +inf). */
rope_status rope_rerank_prune(const int64_t* cand_win, const float* cand_score, const float* pred, int64_t n_reads,
                              int32_t K, int32_t keep, int64_t* out_win, float* out_score, float* out_pred,
                              cudaStream_t stream);

/* rope_map with opts->k candidates per read (use opts->sep = N for one per
 * locus), then pruning to `keep` by the network's predicted distance; with
 * rr = NULL the plain score ranking is kept (the fallback). out_pred
 * [n_reads, keep] (may be NULL) receives the predicted distance / N (the rank
 * for the fallback). */
rope_status rope_map_rerank(const rope_index* idx, const uint8_t* seqs, const int64_t* offsets, int64_t n_reads,
                            const rope_score_opts* opts, const rope_reranker* rr, int32_t keep, int64_t* out_win,
                            float* out_score, float* out_pred, cudaStream_t stream);

/* ---- length ladder: reads of many lengths (§3.5) -------------------------
 * §3.5 maps a read by its head of one fixed window length N. For reads of
 * many lengths a ladder of window lengths N_j = floor(n_min * 2^(j/steps)),
 * j = 0, 1, ... while N_j <= min(n_max, reference length) (repeats dropped),
 * is indexed, and each read is mapped by its head of the largest N_j not
 * longer than the read. Every bucket j is a full index (window norms,
 * anchors) with window length N_j and the parameters' s, m, t, variant,
 * score_mode and stride, built over one shared packed copy of the
 * reference. */
typedef struct rope_ladder rope_ladder;

/* The ladder's lengths, host only: returns their number (or -1 for n_min < 1,
 * n_max < n_min or steps outside [1, 64]) and writes the first `cap` of them to
 * out_host (may be NULL). */
int32_t rope_ladder_lengths(int32_t n_min, int32_t n_max, int32_t steps_per_octave, int32_t* out_host, int32_t cap);

/* Builds the ladder over a device reference (as rope_encode_reference;
 * p->window_len is ignored). At most 64 lengths (ROPE_ERR_UNSUPPORTED above);
 * n_min must be >= p->s. Synchronises `stream`. */
rope_status rope_ladder_create(const rope_params* p, const uint8_t* ref, int64_t len, int32_t n_min, int32_t n_max,
                               int32_t steps_per_octave, rope_ladder** out, cudaStream_t stream);
void rope_ladder_free(rope_ladder* lad);
/* number of lengths; bucket j's index (owned by the ladder; NULL out of range) */
int32_t rope_ladder_size(const rope_ladder* lad);
/* number of captured CUDA graphs the ladder holds (one per repeated key of
 * bucket sizes, buffers and options; see rope_ladder_map) */
int32_t rope_ladder_graph_count(const rope_ladder* lad);
const rope_index* rope_ladder_bucket(const rope_ladder* lad, int32_t j);

/* Maps reads of any length: per read the bucket's k best window starts and
 * fidelities as rope_map gives for that bucket's index (opts as for
 * rope_score_topk; j_begin/j_end must be 0). out_len [n_reads] (may be NULL)
 * receives the window length used, -1 for a read shorter than n_min, whose
 * outputs are all (-1, -inf). Synchronises `stream` once (after bucketing the
 * reads on the device, to read back the bucket sizes); the buckets then run on
 * the ladder's own streams and `stream` waits for them before returning. The
 * ladder keeps the call's scratch; the second call with the same bucket sizes,
 * read and output buffers and options captures the buckets' work in a CUDA
 * graph, later such calls replay it (inputs may change in place). Not for
 * concurrent calls on one ladder from several host threads. */
rope_status rope_ladder_map(const rope_ladder* lad, const uint8_t* seqs, const int64_t* offsets, int64_t n_reads,
                            const rope_score_opts* opts, int64_t* out_win, float* out_score, int32_t* out_len,
                            cudaStream_t stream);

/* ---- multi-GPU: merge of window-range shards (host only) ---------------
 * The reference's windows can be split into disjoint ranges scanned on
 * different GPUs (segments are independent, §2.8). win_host/score_host hold
 * n_shards x n_reads x k_in results of rope_score_topk (shard-major); the
 * best k_out per read over all shards are written to out_* (n_reads x k_out)
 * by (score descending, start ascending), at most one per bucket
 * floor(start/sep) when sep > 0, missing entries (-1, -inf). Pure host code:
 * no device, no allocation visible to the caller. */
rope_status rope_merge_shards_host(const int64_t* win_host, const float* score_host, int32_t n_shards,
                                   int64_t n_reads, int32_t k_in, int32_t k_out, int32_t sep, int64_t* out_win_host,
                                   float* out_score_host);

/* ---- stage timing (tracing) ---------------------------------------------
 * rope_profile_enable(max_calls) starts recording: every following
 * rope_score_topk / rope_map call (up to max_calls) records CUDA events on its
 * stream around its three stages (read encoding, scan, merge/re-score);
 * max_calls = 0 stops recording and frees the events.
 * rope_profile_read() synchronises those events and writes, per recorded
 * call, the milliseconds of [encode, scan, merge] (encode is 0 for
 * rope_score_topk) into ms[3*i .. 3*i+2]; *n_calls receives the number of
 * calls recorded (at most `capacity`). Host-thread-safe; one recorder per
 * process. */
rope_status rope_profile_enable(int32_t max_calls);
rope_status rope_profile_read(float* ms_host, int32_t capacity, int32_t* n_calls);

#ifdef __cplusplus
}
#endif

#endif /* ROTORMAP_H */
