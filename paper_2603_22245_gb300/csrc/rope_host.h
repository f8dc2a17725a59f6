// Host-side helpers shared by the C-ABI translation units: the per-device
// context (status word, scratch pool), the thread-local error message, and the
// definition of rope_index.
#pragma once

#include <vector>

#include "rope_internal.h"
#include "rotormap.h"

namespace rope {

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
};
