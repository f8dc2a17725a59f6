// Host-side helpers shared by the C-ABI translation units: the per-device
// context (status word, scratch pool), the thread-local error message, and the
// definition of rope_index.
#pragma once

#include <vector>

#include "rope_internal.h"
#include "rotormap.h"

namespace rope {

// precisions scored by the tensor-core scan (BF16 or E4M3 operands)
inline bool prec_tc(int32_t precision) { return precision == ROPE_PREC_BF16 || precision == ROPE_PREC_FP8; }

struct DeviceCtx {
  int* status = nullptr;  // device status word
  cudaMemPool_t pool = nullptr;
  int num_sms = 0;
};

// Records a message for rope_last_error() and returns st.
rope_status host_fail(rope_status st, const char* fmt, ...);
// The current device's context (created on first use).
rope_status host_ctx(DeviceCtx** out);
// Stream-ordered scratch from the context's pool.
rope_status host_pool_alloc(DeviceCtx* c, void** p, size_t bytes, cudaStream_t st);
// Stage timing of one call (rope_profile_enable): a slot (or -1 when off or
// full) and its marks 1..3.
int host_prof_begin(cudaStream_t st);
void host_prof_mark(int slot, int which, cudaStream_t st);
// Map and read-frame phase tables of a refinement encoding (validated; any
// m*4^t), cached per device and parameter set.
rope_status host_refine_tables(const rope_params* p, EncTables* out);
// f_k = a / q of band k (1-based) of the encoding p.
void host_factor(const rope_params* p, int k, int64_t* a, int64_t* q);
// Index build; with shared_packed set, the index borrows that packed
// reference (same letters, owned by another index) instead of packing ref.
rope_status encode_reference_impl(const rope_params* p, const uint8_t* ref, int64_t len,
                                  const uint32_t* shared_packed, rope_index** out, cudaStream_t stream);
// Materialised index (every window's encoding stored; any stride).
rope_status encode_reference_dense_impl(const rope_params* p, const uint8_t* ref, int64_t len, rope_index** out,
                                        cudaStream_t stream);
// Scan + merge for n_reads encoded reads; the result of read r goes to output
// row out_row[r] (out_row null: row r). prof_slot < 0: no stage timing.
// A caller-provided candidate buffer for score_topk_impl: used instead of a
// pool block, and the call then never tunes (no timing, no synchronisation).
struct ExtCandidates {
  Candidate* cand;
  size_t bytes;
};
rope_status score_topk_impl(const rope_index* idx, const float* emb_f32, const uint16_t* emb_bf16,
                            const float* norms, int64_t n_reads, const rope_score_opts* opts, int64_t* out_win,
                            float* out_score, cudaStream_t stream, int prof_slot, const int64_t* out_row,
                            const ExtCandidates* ext);
// Candidate-buffer bytes such a call needs, with the configuration it would use
// now (the tuned one for its class, else the defaults).
rope_status topk_cand_bytes(const rope_index* idx, int64_t n_reads, const rope_score_opts* opts, size_t* bytes);

}  // namespace rope

#define ROPE_HOST_CUDA(call)                                                                                \
  do {                                                                                                      \
    cudaError_t e_ = (call);                                                                                \
    if (e_ != cudaSuccess)                                                                                  \
      return rope::host_fail(ROPE_ERR_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
  } while (0)

struct rope_index {
  int device = 0;
  rope_params p{};
  rope::DevIndex ix{};
  rope::EncTables enc{};
  std::vector<void*> owned;
  // materialised index (rope_encode_reference_dense, or any encoding wider
  // than the on-the-fly scans take): TMA descriptors of the window matrices
  // [cr | ci] and [ci | -cr]
  bool dense = false;
  CUtensorMap tm_win{}, tm_win_im{};
};
