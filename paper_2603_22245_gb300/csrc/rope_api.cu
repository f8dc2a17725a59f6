// C ABI of the RotorMap GB300 library (see include/rotormap.h).
//
// Host responsibilities: validation, the exact phase tables (factor f_k held as
// the fraction a_k/q so that every exponent is reduced in integers before the
// FP64 trigonometric call), the default 4^s -> 4^t map, index construction,
// per-call scratch from a stream-ordered memory pool, and launch geometry.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <atomic>
#include <tuple>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "rope_host.h"

using namespace rope;

// ---------------------------------------------------------------- errors

static thread_local char g_last_error[512] = "";

static rope_status fail(rope_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
  va_end(ap);
  return st;
}

rope_status rope::host_fail(rope_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
  va_end(ap);
  return st;
}

#define ROPE_CUDA(call)                                                                               \
  do {                                                                                                \
    cudaError_t e_ = (call);                                                                          \
    if (e_ != cudaSuccess) return fail(ROPE_ERR_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                                       __FILE__, __LINE__);                                           \
  } while (0)

extern "C" const char* rope_status_string(rope_status st) {
  switch (st) {
    case ROPE_OK: return "ROPE_OK";
    case ROPE_ERR_INVALID_ARG: return "ROPE_ERR_INVALID_ARG";
    case ROPE_ERR_INVALID_BASE: return "ROPE_ERR_INVALID_BASE";
    case ROPE_ERR_OOM: return "ROPE_ERR_OOM";
    case ROPE_ERR_CUDA: return "ROPE_ERR_CUDA";
    case ROPE_ERR_TIMEOUT: return "ROPE_ERR_TIMEOUT";
    case ROPE_ERR_UNSUPPORTED: return "ROPE_ERR_UNSUPPORTED";
  }
  return "ROPE_ERR_UNKNOWN";
}

extern "C" const char* rope_last_error(void) { return g_last_error; }

// Bound of every in-kernel wait: 2 s, or ROPE_WAIT_LIMIT_S seconds (clamped to
// [0.05, 120]) for runs that slow kernels down on purpose, such as profilers
// replaying a kernel under instrumentation; rope_set_wait_limit overrides it
// for later launches (tests of the timeout path use a limit of nanoseconds).
static uint64_t default_wait_limit_ns() {
  static const uint64_t v = [] {
    const char* e = getenv("ROPE_WAIT_LIMIT_S");
    double s = e ? atof(e) : 2.0;
    if (!(s >= 0.05)) s = 0.05;
    if (s > 120.0) s = 120.0;
    return (uint64_t)(s * 1e9);
  }();
  return v;
}

static std::atomic<uint64_t> g_wait_limit_override{0};

uint64_t rope::wait_limit_ns() {
  const uint64_t o = g_wait_limit_override.load(std::memory_order_relaxed);
  return o ? o : default_wait_limit_ns();
}

extern "C" rope_status rope_set_wait_limit(double seconds) {
  if (seconds == 0.0) {
    g_wait_limit_override.store(0, std::memory_order_relaxed);
    return ROPE_OK;
  }
  if (!(seconds >= 1e-9 && seconds <= 120.0))
    return fail(ROPE_ERR_INVALID_ARG, "wait limit %g s outside [1e-9, 120] (0 restores the default)", seconds);
  g_wait_limit_override.store((uint64_t)(seconds * 1e9 + 0.5), std::memory_order_relaxed);
  return ROPE_OK;
}

// ---------------------------------------------------------------- per-device context

namespace {

std::mutex g_mu;
std::map<int, DeviceCtx> g_ctx;

rope_status get_ctx(DeviceCtx** out) {
  int dev = 0;
  ROPE_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_ctx.find(dev);
  if (it != g_ctx.end()) {
    *out = &it->second;
    return ROPE_OK;
  }
  DeviceCtx c;
  ROPE_CUDA(cudaDeviceGetAttribute(&c.num_sms, cudaDevAttrMultiProcessorCount, dev));
  ROPE_CUDA(cudaMalloc(&c.status, sizeof(int)));
  ROPE_CUDA(cudaMemset(c.status, 0, sizeof(int)));
  cudaMemPoolProps props;
  memset(&props, 0, sizeof(props));
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  ROPE_CUDA(cudaMemPoolCreate(&c.pool, &props));
  uint64_t keep = ~0ull;  // keep freed blocks in the pool for reuse
  ROPE_CUDA(cudaMemPoolSetAttribute(c.pool, cudaMemPoolAttrReleaseThreshold, &keep));
  auto res = g_ctx.emplace(dev, c);
  *out = &res.first->second;
  return ROPE_OK;
}

rope_status pool_alloc(DeviceCtx* c, void** p, size_t bytes, cudaStream_t st) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMallocFromPoolAsync(p, bytes, c->pool, st);
  if (e == cudaErrorMemoryAllocation) return fail(ROPE_ERR_OOM, "scratch allocation of %zu bytes failed", bytes);
  if (e != cudaSuccess) return fail(ROPE_ERR_CUDA, "cudaMallocFromPoolAsync: %s", cudaGetErrorString(e));
  return ROPE_OK;
}

}  // namespace

rope_status rope::host_ctx(DeviceCtx** out) { return get_ctx(out); }
rope_status rope::host_pool_alloc(DeviceCtx* c, void** p, size_t bytes, cudaStream_t st) {
  return pool_alloc(c, p, bytes, st);
}

namespace {

// ---------------------------------------------------------------- parameters and tables

rope_status check_params(const rope_params* p) {
  if (!p) return fail(ROPE_ERR_INVALID_ARG, "params is NULL");
  if (p->s < 1 || p->s > 8) return fail(ROPE_ERR_INVALID_ARG, "s=%d outside [1,8]", p->s);
  if (p->t < 1 || p->t > p->s) return fail(ROPE_ERR_INVALID_ARG, "t=%d outside [1,s]", p->t);
  if (p->m < 1 || p->m > 8) return fail(ROPE_ERR_INVALID_ARG, "m=%d outside [1,8]", p->m);
  if ((int64_t)p->m << (2 * p->t) > 4096) return fail(ROPE_ERR_INVALID_ARG, "m*4^t > 4096");
  if (p->variant != 0 && p->variant != 1) return fail(ROPE_ERR_INVALID_ARG, "variant=%d", p->variant);
  if (p->score_mode != 0 && p->score_mode != 1) return fail(ROPE_ERR_INVALID_ARG, "score_mode=%d", p->score_mode);
  if (p->window_len < p->s || p->window_len > 65536)
    return fail(ROPE_ERR_INVALID_ARG, "window_len=%d outside [s,65536]", p->window_len);
  if (p->stride < 1 || p->stride > 65536) return fail(ROPE_ERR_INVALID_ARG, "stride=%d outside [1,65536]", p->stride);
  if (p->bin_of_mer_host) {
    const int nb = 1 << (2 * p->t);
    for (int i = 0; i < (1 << (2 * p->s)); ++i)
      if (p->bin_of_mer_host[i] >= nb) return fail(ROPE_ERR_INVALID_ARG, "bin_of_mer[%d] >= 4^t", i);
  }
  return ROPE_OK;
}

// f_k = a_k / q (default: k/1; fine-tuned: (2k+m-3)/(m-1), f = 1 when m = 1)
void factor(const rope_params& p, int k, int64_t* a, int64_t* q) {
  if (p.variant == 1 && p.m > 1) {
    *a = 2 * (int64_t)k + p.m - 3;
    *q = p.m - 1;
  } else {
    *a = k;
    *q = 1;
  }
}

// exp(2 pi i a x / (q N)) with the exponent reduced modulo qN in integers
double2 unit(int64_t a, int64_t q, int64_t N, int64_t x) {
  const int64_t Q = q * N;
  int64_t r = (a * x) % Q;
  if (r < 0) r += Q;
  const double ang = 6.283185307179586476925286766559 * (double)r / (double)Q;
  return make_double2(std::cos(ang), std::sin(ang));
}

struct HostTables {
  std::vector<uint16_t> map;      // 4^s, code with the first letter most significant
  std::vector<uint16_t> map_lsb;  // 4^s, little-endian 2-bit letter field
  std::vector<double2> phase, rot, eout, ein;
  int nb = 0, D = 0, n_loc = 0;
};

void build_tables(const rope_params& p, HostTables& h) {
  const int n_codes = 1 << (2 * p.s);
  h.nb = 1 << (2 * p.t);
  h.D = p.m * h.nb;
  h.n_loc = p.window_len - p.s + 1;
  h.map.resize(n_codes);
  for (int c = 0; c < n_codes; ++c) {
    if (p.bin_of_mer_host) {
      h.map[c] = p.bin_of_mer_host[c];
    } else if (p.s == p.t) {
      h.map[c] = (uint16_t)c;
    } else {
      const uint64_t x = (uint64_t)c * 0x9E3779B97F4A7C15ull;
      h.map[c] = (uint16_t)(x >> (64 - 2 * p.t));
    }
  }
  h.map_lsb.resize(n_codes);
  for (int v = 0; v < n_codes; ++v) {
    int code = 0;
    for (int i = 0; i < p.s; ++i) code = code * 4 + ((v >> (2 * i)) & 3);  // letter i at bits 2i
    h.map_lsb[v] = h.map[code];
  }
  const int S = p.stride, N = p.window_len;
  h.phase.resize((size_t)p.m * h.n_loc);
  h.rot.resize(p.m);
  h.eout.resize((size_t)p.m * S);
  h.ein.resize((size_t)p.m * S);
  for (int k = 1; k <= p.m; ++k) {
    int64_t a, q;
    factor(p, k, &a, &q);
    for (int loc = 0; loc < h.n_loc; ++loc) h.phase[(size_t)(k - 1) * h.n_loc + loc] = unit(a, q, N, loc);
    h.rot[k - 1] = unit(a, q, N, -S);
    for (int u = 0; u < S; ++u) {
      h.eout[(size_t)(k - 1) * S + u] = unit(a, q, N, u);
      h.ein[(size_t)(k - 1) * S + u] = unit(a, q, N, N - p.s + 1 + u);
    }
  }
}

std::vector<float2> to_f32(const std::vector<double2>& v) {
  std::vector<float2> o(v.size());
  for (size_t i = 0; i < v.size(); ++i) o[i] = make_float2((float)v[i].x, (float)v[i].y);
  return o;
}

template <class T>
rope_status upload(std::vector<void*>& owned, const std::vector<T>& v, T** out, size_t pad_elems = 0) {
  void* d = nullptr;
  const size_t bytes = (v.size() + pad_elems) * sizeof(T);
  cudaError_t e = cudaMalloc(&d, bytes ? bytes : 16);
  if (e != cudaSuccess) return fail(ROPE_ERR_OOM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
  owned.push_back(d);
  if (bytes) {
    ROPE_CUDA(cudaMemset(d, 0, bytes));
    if (!v.empty()) ROPE_CUDA(cudaMemcpy(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  }
  *out = static_cast<T*>(d);
  return ROPE_OK;
}

// Device tables for read encoding, cached per device and parameter set.
struct EncEntry {
  std::vector<void*> owned;
  EncTables tb;
};
std::map<std::string, EncEntry> g_enc_cache;

std::string enc_key(int dev, const rope_params& p) {
  std::string k = std::to_string(dev) + ":" + std::to_string(p.s) + "," + std::to_string(p.m) + "," +
                  std::to_string(p.t) + "," + std::to_string(p.variant) + "," + std::to_string(p.window_len) + ":";
  if (p.bin_of_mer_host) {
    uint64_t h = 1469598103934665603ull;
    for (int i = 0; i < (1 << (2 * p.s)); ++i) h = (h ^ p.bin_of_mer_host[i]) * 1099511628211ull;
    k += std::to_string(h);
  } else {
    k += "default";
  }
  return k;
}

rope_status get_enc_tables(const rope_params& p, EncTables* out) {
  int dev = 0;
  ROPE_CUDA(cudaGetDevice(&dev));
  const std::string key = enc_key(dev, p);
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_enc_cache.find(key);
  if (it != g_enc_cache.end()) {
    *out = it->second.tb;
    return ROPE_OK;
  }
  HostTables h;
  build_tables(p, h);
  EncEntry e;
  uint16_t* map = nullptr;
  float2* ph = nullptr;
  rope_status st = upload(e.owned, h.map, &map);
  if (st == ROPE_OK) st = upload(e.owned, to_f32(h.phase), &ph);
  if (st != ROPE_OK) {
    for (void* q : e.owned) cudaFree(q);
    return st;
  }
  e.tb = EncTables{p.window_len, p.s, p.m, p.t, h.nb, h.D, map, ph};
  g_enc_cache.emplace(key, e);
  *out = e.tb;
  return ROPE_OK;
}

}  // namespace

// Tables of an encoding used only for refinement: the s-mer map and the
// read-frame phases; unlike an index's encoding its dense dimension m*4^t is
// not bounded (up to 4^8 bins per band), since refinement stores only the
// bins a read or window touches.
rope_status rope::host_refine_tables(const rope_params* p, EncTables* out) {
  if (!p) return fail(ROPE_ERR_INVALID_ARG, "params is NULL");
  if (p->s < 1 || p->s > 8) return fail(ROPE_ERR_INVALID_ARG, "s=%d outside [1,8]", p->s);
  if (p->t < 1 || p->t > p->s) return fail(ROPE_ERR_INVALID_ARG, "t=%d outside [1,s]", p->t);
  if (p->m < 1 || p->m > 8) return fail(ROPE_ERR_INVALID_ARG, "m=%d outside [1,8]", p->m);
  if (p->variant != 0 && p->variant != 1) return fail(ROPE_ERR_INVALID_ARG, "variant=%d", p->variant);
  if (p->score_mode != 0 && p->score_mode != 1) return fail(ROPE_ERR_INVALID_ARG, "score_mode=%d", p->score_mode);
  if (p->window_len < p->s || p->window_len > 65536)
    return fail(ROPE_ERR_INVALID_ARG, "window_len=%d outside [s,65536]", p->window_len);
  if (p->bin_of_mer_host) {
    const int nb = 1 << (2 * p->t);
    for (int i = 0; i < (1 << (2 * p->s)); ++i)
      if (p->bin_of_mer_host[i] >= nb) return fail(ROPE_ERR_INVALID_ARG, "bin_of_mer[%d] >= 4^t", i);
  }
  return get_enc_tables(*p, out);
}

void rope::host_factor(const rope_params* p, int k, int64_t* a, int64_t* q) { factor(*p, k, a, q); }

namespace {

// Stage recorder: CUDA events around encode / scan / merge of each call.
struct Profiler {
  std::mutex mu;
  int cap = 0, used = 0;
  std::vector<cudaEvent_t> ev;  // 4 per call: start, encoded, scanned, merged
};
Profiler g_prof;

int prof_begin(cudaStream_t st) {
  std::lock_guard<std::mutex> lk(g_prof.mu);
  if (g_prof.used >= g_prof.cap) return -1;
  const int slot = g_prof.used++;
  cudaEventRecord(g_prof.ev[4 * slot], st);
  return slot;
}

void prof_mark(int slot, int which, cudaStream_t st) {
  if (slot >= 0) cudaEventRecord(g_prof.ev[4 * slot + which], st);
}

}  // namespace

int rope::host_prof_begin(cudaStream_t st) { return prof_begin(st); }
void rope::host_prof_mark(int slot, int which, cudaStream_t st) { prof_mark(slot, which, st); }

extern "C" rope_status rope_profile_enable(int32_t max_calls) {
  if (max_calls < 0) return fail(ROPE_ERR_INVALID_ARG, "max_calls < 0");
  std::lock_guard<std::mutex> lk(g_prof.mu);
  for (cudaEvent_t e : g_prof.ev) cudaEventDestroy(e);
  g_prof.ev.clear();
  g_prof.cap = g_prof.used = 0;
  for (int i = 0; i < 4 * max_calls; ++i) {
    cudaEvent_t e;
    ROPE_CUDA(cudaEventCreate(&e));
    g_prof.ev.push_back(e);
  }
  g_prof.cap = max_calls;
  return ROPE_OK;
}

extern "C" rope_status rope_profile_read(float* ms_host, int32_t capacity, int32_t* n_calls) {
  std::lock_guard<std::mutex> lk(g_prof.mu);
  const int n = g_prof.used < capacity ? g_prof.used : capacity;
  for (int i = 0; i < n; ++i) {
    ROPE_CUDA(cudaEventSynchronize(g_prof.ev[4 * i + 3]));
    for (int k = 0; k < 3; ++k) {
      float ms = 0.f;
      ROPE_CUDA(cudaEventElapsedTime(&ms, g_prof.ev[4 * i + k], g_prof.ev[4 * i + k + 1]));
      ms_host[3 * i + k] = ms;
    }
  }
  if (n_calls) *n_calls = n;
  return ROPE_OK;
}

// ---------------------------------------------------------------- index

extern "C" int32_t rope_dim(const rope_params* p) {
  if (check_params(p) != ROPE_OK) return -1;
  return p->m << (2 * p->t);
}

extern "C" rope_status rope_sync_status(cudaStream_t stream) {
  DeviceCtx* c;
  rope_status st = get_ctx(&c);
  if (st != ROPE_OK) return st;
  ROPE_CUDA(cudaStreamSynchronize(stream));
  int v = 0;
  ROPE_CUDA(cudaMemcpy(&v, c->status, sizeof(int), cudaMemcpyDeviceToHost));
  ROPE_CUDA(cudaMemset(c->status, 0, sizeof(int)));
  if (v & kStatusTimeout) return fail(ROPE_ERR_TIMEOUT, "a bounded in-kernel wait ran out");
  if (v & kStatusBadBase) return fail(ROPE_ERR_INVALID_BASE, "letter outside {A,C,G,T}");
  if (v & kStatusShortRead) return fail(ROPE_ERR_INVALID_ARG, "a read is shorter than the window length");
  if (v & kStatusBadArg) return fail(ROPE_ERR_INVALID_ARG, "a kernel saw an out-of-range argument");
  return ROPE_OK;
}

extern "C" rope_status rope_pack_2bit(const uint8_t* seq, int64_t len, uint32_t* out_words, cudaStream_t stream) {
  if (len < 0 || (len > 0 && (!seq || !out_words))) return fail(ROPE_ERR_INVALID_ARG, "bad pack arguments");
  DeviceCtx* c;
  rope_status st = get_ctx(&c);
  if (st != ROPE_OK) return st;
  ROPE_CUDA(launch_pack(seq, len, out_words, c->status, stream));
  return ROPE_OK;
}

extern "C" rope_status rope_mer_bins(const rope_params* p, const uint32_t* packed, int64_t len, uint16_t* out_bins,
                                     cudaStream_t stream) {
  rope_status st = check_params(p);
  if (st != ROPE_OK) return st;
  if (len < p->s) return fail(ROPE_ERR_INVALID_ARG, "len < s");
  if (!packed || !out_bins) return fail(ROPE_ERR_INVALID_ARG, "NULL pointer");
  HostTables h;
  build_tables(*p, h);
  uint16_t* d_map = nullptr;
  ROPE_CUDA(cudaMallocAsync((void**)&d_map, h.map_lsb.size() * sizeof(uint16_t), stream));
  ROPE_CUDA(cudaMemcpyAsync(d_map, h.map_lsb.data(), h.map_lsb.size() * sizeof(uint16_t), cudaMemcpyHostToDevice,
                            stream));
  ROPE_CUDA(launch_mer_bins(packed, len, (len + 15) / 16, p->s, d_map, out_bins, stream));
  ROPE_CUDA(cudaStreamSynchronize(stream));  // the host table must outlive the copy
  ROPE_CUDA(cudaFreeAsync(d_map, stream));
  return ROPE_OK;
}

extern "C" void rope_index_free(rope_index* idx) {
  if (!idx) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(idx->device);
  cudaDeviceSynchronize();
  for (void* q : idx->owned) cudaFree(q);
  cudaSetDevice(prev);
  delete idx;
}

// ---------------------------------------------------------------- materialised index

namespace {

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// TMA descriptor of a row-major BF16 matrix [rows, cols] read in boxes of
// 128 rows x 64 columns (128 bytes, the 128-byte swizzle of the MMA operands);
// rows past the end read as zero.
rope_status tensor_map_rows(CUtensorMap* m, const void* base, int64_t rows, int cols) {
  static EncodeTiledFn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      f = nullptr;
    }
    return reinterpret_cast<EncodeTiledFn>(f);
  }();
  if (!fn) return fail(ROPE_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
  if (rows < 1 || rows > 0x7FFFFFFF || cols % 64 != 0) return fail(ROPE_ERR_INVALID_ARG, "tensor map of %lld x %d", (long long)rows, cols);
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
  const cuuint32_t box[2] = {64, 128};
  const cuuint32_t es[2] = {1, 1};
  const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(ROPE_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return ROPE_OK;
}

}  // namespace

// The paper's index (§3.1): every window's encoding stored, FP32 and
// normalised BF16, built from per-block sums (see rope_dense.cu).
rope_status rope::encode_reference_dense_impl(const rope_params* p, const uint8_t* ref, int64_t len,
                                              rope_index** out, cudaStream_t stream) {
  rope_status st = check_params(p);
  if (st != ROPE_OK) return st;
  if (!out) return fail(ROPE_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!ref || len < p->window_len) return fail(ROPE_ERR_INVALID_ARG, "reference shorter than the window");
  const int D = p->m << (2 * p->t);
  if (D % 32 != 0 || D > 4096)
    return fail(ROPE_ERR_UNSUPPORTED, "materialised index: complex dimension %d is not a multiple of 32 up to 4096", D);
  if (p->score_mode != 0) return fail(ROPE_ERR_UNSUPPORTED, "materialised index takes score_mode 0");
  const int S = p->stride, N = p->window_len;
  const int64_t W = (len - N) / S + 1;
  if (W > 0x7FFFFFFF - 256) return fail(ROPE_ERR_UNSUPPORTED, "more than 2^31 windows");
  DeviceCtx* c;
  if ((st = get_ctx(&c)) != ROPE_OK) return st;

  rope_index* idx = new rope_index();
  ROPE_CUDA(cudaGetDevice(&idx->device));
  idx->p = *p;
  idx->p.bin_of_mer_host = nullptr;
  idx->dense = true;
  auto cleanup = [&](rope_status s) {
    rope_index_free(idx);
    return s;
  };
  HostTables h;
  build_tables(*p, h);
  // blocks of S starts: n_loc = full * S + rem; the partial block's starts are
  // added directly, or a whole block is summed and the over-covered starts
  // removed, whichever touches fewer starts
  const int n_loc = N - p->s + 1;
  const int full = n_loc / S, rem = n_loc - full * S;
  int n_blk = full, t0 = 0, n_t = 0;
  double sign = 1.0;
  if (rem > 0 && rem <= S - rem) {
    t0 = full * S;
    n_t = rem;
  } else if (rem > 0) {
    n_blk = full + 1;
    t0 = n_loc;
    n_t = S - rem;
    sign = -1.0;
  }
  std::vector<float2> bph((size_t)p->m * S), rotu((size_t)std::max(n_blk, 1) * p->m), tph((size_t)p->m * std::max(n_t, 1));
  for (int k = 1; k <= p->m; ++k) {
    int64_t a, q;
    factor(*p, k, &a, &q);
    for (int i = 0; i < S; ++i) {
      const double2 v = unit(a, q, N, i);
      bph[(size_t)(k - 1) * S + i] = make_float2((float)v.x, (float)v.y);
    }
    for (int u = 0; u < n_blk; ++u) {
      const double2 v = unit(a, q, N, (int64_t)u * S);
      rotu[(size_t)u * p->m + (k - 1)] = make_float2((float)v.x, (float)v.y);
    }
    for (int i = 0; i < n_t; ++i) {
      const double2 v = unit(a, q, N, (int64_t)t0 + i);
      tph[(size_t)(k - 1) * n_t + i] = make_float2((float)(sign * v.x), (float)(sign * v.y));
    }
  }
  const int64_t n_words = (len + 15) / 16;
  const int64_t pad_words = 16384 + kPackPadWords + ((int64_t)S + 15) / 16;
  const int64_t n_blocks = n_blk > 0 ? W + n_blk - 1 : 0;
  uint32_t* packed = nullptr;
  float *inv_norm = nullptr, *win_f32 = nullptr;
  uint16_t *win_bf16 = nullptr, *win_bf16_im = nullptr, *map_lsb = nullptr, *map = nullptr;
  float2 *phase = nullptr, *d_bph = nullptr, *d_rotu = nullptr, *d_tph = nullptr;
  if ((st = upload(idx->owned, std::vector<uint32_t>(), &packed, (size_t)(n_words + pad_words))) != ROPE_OK ||
      (st = upload(idx->owned, std::vector<float>(), &inv_norm, (size_t)W + 256)) != ROPE_OK ||
      (st = upload(idx->owned, std::vector<float>(), &win_f32, (size_t)W * 2 * D)) != ROPE_OK ||
      (st = upload(idx->owned, std::vector<uint16_t>(), &win_bf16, (size_t)W * 2 * D)) != ROPE_OK ||
      (st = upload(idx->owned, std::vector<uint16_t>(), &win_bf16_im, (size_t)W * 2 * D)) != ROPE_OK ||
      (st = upload(idx->owned, h.map_lsb, &map_lsb)) != ROPE_OK || (st = upload(idx->owned, h.map, &map)) != ROPE_OK ||
      (st = upload(idx->owned, to_f32(h.phase), &phase)) != ROPE_OK ||
      (st = upload(idx->owned, bph, &d_bph)) != ROPE_OK || (st = upload(idx->owned, rotu, &d_rotu)) != ROPE_OK ||
      (st = upload(idx->owned, tph, &d_tph)) != ROPE_OK)
    return cleanup(st);
  DevIndex& ix = idx->ix;
  ix.packed = packed;
  ix.L = len;
  ix.W = W;
  ix.N = N;
  ix.s = p->s;
  ix.m = p->m;
  ix.t = p->t;
  ix.nb = h.nb;
  ix.D = D;
  ix.stride = S;
  ix.A = 0;
  ix.variant = p->variant;
  ix.score_mode = p->score_mode;
  ix.inv_norm = inv_norm;
  ix.map_lsb = map_lsb;
  ix.phase = phase;
  ix.win_f32 = win_f32;
  ix.win_bf16 = win_bf16;
  idx->enc = EncTables{N, p->s, p->m, p->t, h.nb, D, map, phase};
  DenseTables dt{n_blk, t0, n_t, n_blocks, d_bph, d_rotu, d_tph};

  float2* bsum = nullptr;
  int zero = 0;
  cudaError_t e = cudaMemcpy(c->status, &zero, sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && n_blocks > 0) e = cudaMalloc(&bsum, (size_t)n_blocks * D * sizeof(float2));
  if (e == cudaErrorMemoryAllocation) return cleanup(fail(ROPE_ERR_OOM, "block sums: %s", cudaGetErrorString(e)));
  if (e == cudaSuccess) e = launch_pack(ref, len, packed, c->status, stream);
  if (e == cudaSuccess) e = launch_dense_index(ix, dt, bsum, win_f32, win_bf16, win_bf16_im, inv_norm, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (bsum) cudaFree(bsum);
  if (e != cudaSuccess) return cleanup(fail(ROPE_ERR_CUDA, "materialised index build: %s", cudaGetErrorString(e)));
  if ((st = rope_sync_status(stream)) != ROPE_OK) return cleanup(st);
  if ((st = tensor_map_rows(&idx->tm_win, win_bf16, W, 2 * D)) != ROPE_OK ||
      (st = tensor_map_rows(&idx->tm_win_im, win_bf16_im, W, 2 * D)) != ROPE_OK)
    return cleanup(st);
  *out = idx;
  return ROPE_OK;
}

extern "C" rope_status rope_encode_reference_dense(const rope_params* p, const uint8_t* ref, int64_t len,
                                                   rope_index** out, cudaStream_t stream) {
  return encode_reference_dense_impl(p, ref, len, out, stream);
}

rope_status rope::encode_reference_impl(const rope_params* p, const uint8_t* ref, int64_t len,
                                        const uint32_t* shared_packed, rope_index** out, cudaStream_t stream) {
  rope_status st = check_params(p);
  if (st != ROPE_OK) return st;
  if (!out) return fail(ROPE_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!ref || len < p->window_len) return fail(ROPE_ERR_INVALID_ARG, "reference shorter than the window");
  const int D = p->m << (2 * p->t);
  if (D > kMaxScanDim) {
    if (shared_packed) return fail(ROPE_ERR_UNSUPPORTED, "index dimension %d > %d in a ladder", D, kMaxScanDim);
    return encode_reference_dense_impl(p, ref, len, out, stream);
  }
  if (p->stride > 64) return fail(ROPE_ERR_UNSUPPORTED, "stride=%d: the on-the-fly index takes stride <= 64", p->stride);
  const int64_t W = (len - p->window_len) / p->stride + 1;
  // window numbers are 32-bit in the scans, with room for one super-tile past the end
  if (W > (int64_t)0xFFFFFFFF - 65536) return fail(ROPE_ERR_UNSUPPORTED, "more than 2^32 - 2^16 windows");
  DeviceCtx* c;
  st = get_ctx(&c);
  if (st != ROPE_OK) return st;

  rope_index* idx = new rope_index();
  ROPE_CUDA(cudaGetDevice(&idx->device));
  idx->p = *p;
  idx->p.bin_of_mer_host = nullptr;
  HostTables h;
  build_tables(*p, h);
  const int A = kAnchorPeriod;
  const int64_t n_words = (len + 15) / 16;
  const int64_t pad_words = 16384 + kPackPadWords;
  const int64_t n_anchor = (W + A - 1) / A;

  auto cleanup = [&](rope_status s) {
    rope_index_free(idx);
    return s;
  };
  std::vector<uint32_t> none;
  uint32_t* packed = nullptr;
  float* inv_norm = nullptr;
  float* band_norm = nullptr;
  float2* anchors = nullptr;
  uint16_t *map_lsb = nullptr, *map = nullptr;
  float2 *phase = nullptr, *rot = nullptr, *eout = nullptr, *ein = nullptr;
  double2 *phase64 = nullptr, *rot64 = nullptr, *eout64 = nullptr, *ein64 = nullptr;
  if (shared_packed) {
    packed = const_cast<uint32_t*>(shared_packed);  // borrowed: another index owns it
  } else if ((st = upload(idx->owned, std::vector<uint32_t>(), &packed, (size_t)(n_words + pad_words))) != ROPE_OK) {
    return cleanup(st);
  }
  if ((st = upload(idx->owned, std::vector<float>(), &inv_norm, (size_t)W + 8192)) != ROPE_OK) return cleanup(st);
  if (p->score_mode == 1 &&
      (st = upload(idx->owned, std::vector<float>(), &band_norm, (size_t)W * p->m + 8192)) != ROPE_OK)
    return cleanup(st);
  if ((st = upload(idx->owned, std::vector<float2>(), &anchors, (size_t)(n_anchor + 128) * D)) != ROPE_OK)
    return cleanup(st);
  if ((st = upload(idx->owned, h.map_lsb, &map_lsb)) != ROPE_OK) return cleanup(st);
  if ((st = upload(idx->owned, h.map, &map)) != ROPE_OK) return cleanup(st);
  if ((st = upload(idx->owned, to_f32(h.phase), &phase)) != ROPE_OK) return cleanup(st);
  if ((st = upload(idx->owned, to_f32(h.rot), &rot)) != ROPE_OK) return cleanup(st);
  if ((st = upload(idx->owned, to_f32(h.eout), &eout)) != ROPE_OK) return cleanup(st);
  if ((st = upload(idx->owned, to_f32(h.ein), &ein)) != ROPE_OK) return cleanup(st);
  if ((st = upload(idx->owned, h.phase, &phase64)) != ROPE_OK) return cleanup(st);
  if ((st = upload(idx->owned, h.rot, &rot64)) != ROPE_OK) return cleanup(st);
  if ((st = upload(idx->owned, h.eout, &eout64)) != ROPE_OK) return cleanup(st);
  if ((st = upload(idx->owned, h.ein, &ein64)) != ROPE_OK) return cleanup(st);

  DevIndex& ix = idx->ix;
  ix.packed = packed;
  ix.L = len;
  ix.W = W;
  ix.N = p->window_len;
  ix.s = p->s;
  ix.m = p->m;
  ix.t = p->t;
  ix.nb = h.nb;
  ix.D = D;
  ix.stride = p->stride;
  ix.A = A;
  ix.variant = p->variant;
  ix.score_mode = p->score_mode;
  ix.inv_norm = inv_norm;
  ix.band_norm = band_norm;
  ix.anchors = anchors;
  ix.map_lsb = map_lsb;
  ix.phase = phase;
  ix.rot = rot;
  ix.eout = eout;
  ix.ein = ein;
  idx->enc = EncTables{p->window_len, p->s, p->m, p->t, h.nb, D, map, phase};

  // clear stale status, pack, pre-pass
  int zero = 0;
  cudaError_t e = cudaMemcpy(c->status, &zero, sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !shared_packed) e = launch_pack(ref, len, packed, c->status, stream);
  if (e == cudaSuccess) {
    PrepassTables pt{phase64, rot64, eout64, ein64};
    e = launch_prepass(ix, pt, anchors, inv_norm, band_norm, c->status, stream);
  }
  if (e != cudaSuccess) return cleanup(fail(ROPE_ERR_CUDA, "index build launch: %s", cudaGetErrorString(e)));
  st = rope_sync_status(stream);
  if (st != ROPE_OK) return cleanup(st);
  *out = idx;
  return ROPE_OK;
}

extern "C" rope_status rope_encode_reference(const rope_params* p, const uint8_t* ref, int64_t len, rope_index** out,
                                             cudaStream_t stream) {
  return encode_reference_impl(p, ref, len, nullptr, out, stream);
}

extern "C" rope_status rope_index_info(const rope_index* idx, int64_t* n_windows, int64_t* ref_len,
                                       int32_t* anchor_period, const uint32_t** packed, const float** inv_norm) {
  if (!idx) return fail(ROPE_ERR_INVALID_ARG, "index is NULL");
  if (n_windows) *n_windows = idx->ix.W;
  if (ref_len) *ref_len = idx->ix.L;
  if (anchor_period) *anchor_period = idx->ix.A;
  if (packed) *packed = idx->ix.packed;
  if (inv_norm) *inv_norm = idx->ix.inv_norm;
  return ROPE_OK;
}

extern "C" rope_status rope_window_embeddings(const rope_index* idx, int64_t j_begin, int64_t count, float* out,
                                              cudaStream_t stream) {
  if (!idx || !out) return fail(ROPE_ERR_INVALID_ARG, "NULL argument");
  if (j_begin < 0 || count < 0 || j_begin + count > idx->ix.W) return fail(ROPE_ERR_INVALID_ARG, "window range");
  if (idx->dense) {
    const size_t row = (size_t)2 * idx->ix.D * sizeof(float);
    ROPE_CUDA(cudaMemcpyAsync(out, idx->ix.win_f32 + (size_t)j_begin * 2 * idx->ix.D, (size_t)count * row,
                              cudaMemcpyDeviceToDevice, stream));
    return ROPE_OK;
  }
  ROPE_CUDA(launch_window_embeddings(idx->ix, j_begin, count, out, stream));
  return ROPE_OK;
}

extern "C" rope_status rope_encode_reads(const rope_params* p, const uint8_t* seqs, const int64_t* offsets,
                                         int64_t n_reads, float* emb_f32, uint16_t* emb_bf16, float* norms,
                                         cudaStream_t stream) {
  rope_status st = check_params(p);
  if (st != ROPE_OK) return st;
  if (n_reads < 0) return fail(ROPE_ERR_INVALID_ARG, "n_reads < 0");
  if (n_reads == 0) return ROPE_OK;
  if (!seqs || !offsets || !norms) return fail(ROPE_ERR_INVALID_ARG, "NULL pointer");
  DeviceCtx* c;
  if ((st = get_ctx(&c)) != ROPE_OK) return st;
  EncTables tb;
  if ((st = get_enc_tables(*p, &tb)) != ROPE_OK) return st;
  ROPE_CUDA(launch_encode_reads(tb, seqs, offsets, n_reads, emb_f32, emb_bf16, norms, c->status, stream));
  return ROPE_OK;
}

// ---------------------------------------------------------------- §2.4 pair fidelities

extern "C" rope_status rope_pair_fidelities(const rope_params* p, const uint8_t* seqs, const int64_t* offsets,
                                            int64_t n, const double* errs, uint64_t seed, float* out_fid,
                                            cudaStream_t stream) {
  rope_status st = check_params(p);
  if (st != ROPE_OK) return st;
  if (n < 0) return fail(ROPE_ERR_INVALID_ARG, "n < 0");
  if (n == 0) return ROPE_OK;
  if (!seqs || !offsets || !errs || !out_fid) return fail(ROPE_ERR_INVALID_ARG, "NULL pointer");
  DeviceCtx* c;
  if ((st = get_ctx(&c)) != ROPE_OK) return st;
  EncTables tb;
  if ((st = get_enc_tables(*p, &tb)) != ROPE_OK) return st;
  const int N = p->window_len, D = tb.D, m = tb.m;
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  const size_t b_copy = al((size_t)n * N), b_off = al((size_t)(n + 1) * sizeof(int64_t));
  const size_t b_emb = al((size_t)2 * n * 2 * D * sizeof(float)), b_norm = al((size_t)2 * n * (1 + m) * sizeof(float));
  uint8_t* scratch = nullptr;
  if ((st = pool_alloc(c, (void**)&scratch, b_copy + b_off + b_emb + b_norm, stream)) != ROPE_OK) return st;
  uint8_t* copies = scratch;
  int64_t* coff = reinterpret_cast<int64_t*>(scratch + b_copy);
  float* emb = reinterpret_cast<float*>(scratch + b_copy + b_off);
  float* norms = reinterpret_cast<float*>(scratch + b_copy + b_off + b_emb);
  MutArgs ma{};
  ma.seqs = seqs;
  ma.offsets = offsets;
  ma.errs = errs;
  ma.n = n;
  ma.N = N;
  ma.seed = seed;
  ma.out = copies;
  ma.status = c->status;
  cudaError_t e = launch_mutate(ma, stream);
  if (e == cudaSuccess) e = launch_iota_offsets(coff, n, N, stream);
  if (e == cudaSuccess) e = launch_encode_reads(tb, seqs, offsets, n, emb, nullptr, norms, c->status, stream);
  if (e == cudaSuccess)
    e = launch_encode_reads(tb, copies, coff, n, emb + (size_t)n * 2 * D, nullptr, norms + (size_t)n * (1 + m),
                            c->status, stream);
  if (e == cudaSuccess) e = launch_pair_fidelity(emb, norms, n, D, m, tb.nb, p->score_mode, out_fid, stream);
  cudaFreeAsync(scratch, stream);
  if (e != cudaSuccess) return fail(ROPE_ERR_CUDA, "pair fidelities launch: %s", cudaGetErrorString(e));
  return ROPE_OK;
}

// ---------------------------------------------------------------- scan

namespace {

struct ScanPlan {
  ScanArgs a{};
  bool tc = false;
  size_t cand_bytes = 0;
};

rope_status plan_scan(const rope_index* idx, int32_t precision, int64_t n_reads, int64_t jb, int64_t je,
                      int32_t n_ranges_req, int num_sms, ScanPlan* out, int32_t tc_variant = 0) {
  const DevIndex& ix = idx->ix;
  if (idx->dense) return fail(ROPE_ERR_UNSUPPORTED, "a materialised index is scored by rope_score_topk / rope_map / rope_score_dense only");
  ScanPlan pl;
  pl.tc = prec_tc(precision);
  int64_t sup;
  int group;
  if (pl.tc) {
    if (!scan_tc_supported(ix.D))
      return fail(ROPE_ERR_UNSUPPORTED, "tensor-core scan built for complex dimension 32 or 64, not %d", ix.D);
    if (ix.score_mode != 0) return fail(ROPE_ERR_UNSUPPORTED, "tensor-core scan takes score_mode 0 only");
    if (ix.stride > scan_tc_max_stride())
      return fail(ROPE_ERR_UNSUPPORTED, "tensor-core scan takes stride <= %d", scan_tc_max_stride());
    sup = scan_tc_super_tile(ix.D, tc_variant);
    group = scan_tc_group(ix.D, tc_variant);
  } else if (precision == ROPE_PREC_FP32) {
    if (!scan_fp32_supported(ix.D))
      return fail(ROPE_ERR_UNSUPPORTED, "FP32 scan built for complex dimension <= 64, not %d", ix.D);
    sup = scan_fp32_super_tile(ix.D);
    group = scan_fp32_group(ix.D);
  } else {
    return fail(ROPE_ERR_INVALID_ARG, "precision %d", precision);
  }
  ScanArgs& a = pl.a;
  a.n_reads = n_reads;
  a.jb = jb;
  a.je = je;
  a.st0 = (jb / sup) * sup;
  const int64_t n_sup = (je - a.st0 + sup - 1) / sup;
  a.n_groups = (int32_t)((n_reads + group - 1) / group);
  int64_t nr = n_ranges_req > 0 ? n_ranges_req : (16LL * num_sms + a.n_groups - 1) / a.n_groups;
  if (nr < 1) nr = 1;
  if (nr > n_sup) nr = n_sup;
  if (nr > 4096) nr = 4096;
  const int64_t sup_per_range = (n_sup + nr - 1) / nr;
  a.range_len = sup_per_range * sup;
  a.n_ranges = (int32_t)((n_sup + sup_per_range - 1) / sup_per_range);
  a.tc_variant = pl.tc ? tc_variant : 0;
  a.fp8 = precision == ROPE_PREC_FP8;
  a.lists_per_range = pl.tc ? scan_tc_lists_per_range(ix.D, a.tc_variant) : 1;
  a.wait_limit_ns = wait_limit_ns();
  *out = pl;
  return ROPE_OK;
}

rope_status check_opts(const rope_score_opts* o, rope_score_opts* v) {
  if (!o) return fail(ROPE_ERR_INVALID_ARG, "opts is NULL");
  *v = *o;
  if (v->k < 1 || v->k > 32) return fail(ROPE_ERR_INVALID_ARG, "k=%d outside [1,32]", v->k);
  if (v->sep < 0) return fail(ROPE_ERR_INVALID_ARG, "sep < 0");
  // default: 8 candidates per list (k when k > 8); the union of a read's
  // lists (two halves x several window ranges) feeds the re-scoring
  if (v->cand_depth == 0) v->cand_depth = 8;
  if (v->cand_depth < v->k) v->cand_depth = v->k;
  if (v->cand_depth > 32) return fail(ROPE_ERR_INVALID_ARG, "cand_depth > 32");
  if (v->rescore_depth == 0) v->rescore_depth = v->k * 2 < 32 ? v->k * 2 : 32;
  if (v->rescore_depth < v->k) v->rescore_depth = v->k;
  if (v->rescore_depth > 32) return fail(ROPE_ERR_INVALID_ARG, "rescore_depth > 32");
  if (v->rescore != 0 && v->rescore != 1) return fail(ROPE_ERR_INVALID_ARG, "rescore must be 0 or 1");
  return ROPE_OK;
}

// ---------------------------------------------------------------- tuner
//
// The tensor-core scan has tile variants (scan_tc_variants) and a free work
// split (read-group x window-range items per SM). On the first BF16 call for
// a shape class (device, complex dimension, stride, window length and read
// groups to the nearest power of two, candidate depth, sep on/off) the tuner
// times every (variant, items per SM) pair on a sample of the call's own
// windows with the call's own reads and keeps the fastest for that class. The
// results of a scan do not depend on these choices (each window's score is
// the same product; the merge takes the best entries of all lists), only its
// speed does. ROPE_AUTOTUNE=0 (or rope_autotune_enable(0)) keeps the defaults.

struct TuneKey {
  int dev, D, stride, n_log2, g_log2, w_log2, cand_depth, sep_on, fp8;
  bool operator<(const TuneKey& o) const {
    return std::tie(dev, D, stride, n_log2, g_log2, w_log2, cand_depth, sep_on, fp8) <
           std::tie(o.dev, o.D, o.stride, o.n_log2, o.g_log2, o.w_log2, o.cand_depth, o.sep_on, o.fp8);
  }
};
struct TuneVal {
  int32_t variant = 0;
  int32_t items_per_sm = 16;
  float sample_ms = 0.f;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tune;
int g_autotune = -1;  // -1: from the environment on first use

bool autotune_on() {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  if (g_autotune < 0) {
    const char* e = getenv("ROPE_AUTOTUNE");
    g_autotune = (e && e[0] == '0') ? 0 : 1;
  }
  return g_autotune == 1;
}

// ROPE_AUTOTUNE_LOG=1 prints every candidate's predicted time to stderr.
bool tune_log() {
  static const bool on = [] {
    const char* e = getenv("ROPE_AUTOTUNE_LOG");
    return e && e[0] == '1';
  }();
  return on;
}

int ilog2_ceil(int64_t v) {
  int r = 0;
  while ((int64_t(1) << r) < v) ++r;
  return r;
}

// windows a call scans: [j_begin, j_end) clipped to the index as score_topk_impl does
int64_t scanned_windows(const rope_index* idx, const rope_score_opts& o) {
  const int64_t W = idx->ix.W;
  const int64_t jb = o.j_begin > 0 ? o.j_begin : 0;
  const int64_t je = o.j_end > 0 ? (o.j_end < W ? o.j_end : W) : W;
  return je > jb ? je - jb : 0;
}

TuneKey tune_key(const rope_index* idx, int64_t n_reads, const rope_score_opts& o) {
  const DevIndex& ix = idx->ix;
  const int64_t groups = (n_reads + scan_tc_group(ix.D) - 1) / scan_tc_group(ix.D);
  return TuneKey{idx->device,         ix.D,        ix.stride, ilog2_ceil(ix.N), ilog2_ceil(groups),
                 ilog2_ceil(scanned_windows(idx, o)), o.cand_depth, o.sep > 0,
                 o.precision == ROPE_PREC_FP8};
}

int32_t ranges_for(int items_per_sm, int num_sms, int64_t n_groups) {
  const int64_t nr = ((int64_t)items_per_sm * num_sms + n_groups - 1) / n_groups;
  return (int32_t)(nr < 1 ? 1 : nr > 4096 ? 4096 : nr);
}

// Times one candidate (variant, n_ranges) on windows [jb, jb + len).
rope_status time_candidate(const rope_index* idx, const uint16_t* emb_bf16, const float* emb_f32, const float* norms,
                           int64_t n_reads, int64_t jb, int64_t len, int32_t n_ranges, int variant,
                           const rope_score_opts& o, Candidate* cand, DeviceCtx* c, cudaStream_t stream,
                           cudaEvent_t e0, cudaEvent_t e1, int reps, float* ms) {
  ScanPlan pl;
  rope_status st = plan_scan(idx, o.precision, n_reads, jb, jb + len, n_ranges, c->num_sms, &pl, variant);
  if (st != ROPE_OK) return st;
  pl.a.emb_f32 = emb_f32;
  pl.a.emb_bf16 = emb_bf16;
  pl.a.norms = norms;
  pl.a.cand_depth = o.cand_depth;
  pl.a.sep = o.sep;
  pl.a.cand = cand;
  pl.a.status = c->status;
  cudaError_t e = cudaSuccess;
  for (int rep = 0; rep < reps && e == cudaSuccess; ++rep) {  // only the last launch is timed
    cudaEventRecord(e0, stream);
    e = launch_scan_tc(idx->ix, pl.a, false, c->num_sms, stream);
    cudaEventRecord(e1, stream);
  }
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  if (e != cudaSuccess) return fail(ROPE_ERR_CUDA, "tuning launch: %s", cudaGetErrorString(e));
  return ROPE_OK;
}

// Times each candidate on the call's own windows [jb, je) and records the
// fastest, when the scan is short enough to be timed whole (at most
// kTuneMaxWindows windows). A longer scan keeps the defaults: measured on this
// GPU, a scan's cost per window falls with its length (each candidate list
// takes about k*ln(n/k) updates over n windows, most of them early), by 2.2x
// from 2^20 to 10^8 windows, and unevenly across the tile variants, so timings
// of a short sample ranked the variants the wrong way round for a long scan.
constexpr int64_t kTuneMaxWindows = (int64_t)1 << 22;

rope_status tune_tc(const rope_index* idx, const uint16_t* emb_bf16, const float* emb_f32, const float* norms,
                    int64_t n_reads, int64_t jb, int64_t je, const rope_score_opts& o, DeviceCtx* c,
                    cudaStream_t stream, TuneVal* best) {
  const DevIndex& ix = idx->ix;
  auto n_groups = [&](int v) -> int64_t { return (n_reads + scan_tc_group(ix.D, v) - 1) / scan_tc_group(ix.D, v); };
  static const int kItems[] = {8, 16, 32};
  const int64_t total = je - jb;
  if (total > kTuneMaxWindows) {
    *best = TuneVal{0, 16, 0.f};
    return ROPE_OK;
  }
  size_t cand_bytes = 0;
  for (int v = 0; v < scan_tc_variants(ix.D); ++v)
    for (int items : kItems) {
      const size_t b = (size_t)n_reads * ranges_for(items, c->num_sms, n_groups(v)) * scan_tc_lists_per_range(ix.D, v) *
                       o.cand_depth * sizeof(Candidate);
      cand_bytes = std::max(cand_bytes, b);
    }
  Candidate* cand = nullptr;
  rope_status st = pool_alloc(c, (void**)&cand, cand_bytes, stream);
  if (st != ROPE_OK) return st;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  TuneVal b{0, 16, 1e30f};
  bool any = false;
  for (int v = 0; v < scan_tc_variants(ix.D) && st == ROPE_OK; ++v) {
    if (!scan_tc_fits(ix, o.cand_depth, v, o.precision == ROPE_PREC_FP8)) continue;
    for (int items : kItems) {
      const int32_t nr = ranges_for(items, c->num_sms, n_groups(v));
      const int reps = any ? 1 : 2;  // the very first launch warms up, untimed
      float ms = 0.f;
      st = time_candidate(idx, emb_bf16, emb_f32, norms, n_reads, jb, total, nr, v, o, cand, c, stream, e0, e1, reps,
                          &ms);
      if (st != ROPE_OK) break;
      if (tune_log())
        fprintf(stderr, "rotormap tuner: D=%d stride=%d N=%d reads=%lld windows=%lld variant=%d items/SM=%d %.3f ms\n",
                ix.D, ix.stride, ix.N, (long long)n_reads, (long long)total, v, items, ms);
      if (ms < b.sample_ms) b = TuneVal{v, items, ms};
      any = true;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(cand, stream);
  if (st == ROPE_OK && any) *best = b;
  return st;
}

// The variant and range split of a BF16 scan: the tuned ones for its class
// (tuned now if new and the call's n_ranges is 0), else the defaults.
rope_status choose_tc(const rope_index* idx, const uint16_t* emb_bf16, const float* emb_f32, const float* norms,
                      int64_t n_reads, int64_t jb, int64_t je, const rope_score_opts& o, DeviceCtx* c,
                      cudaStream_t stream, bool may_tune, int32_t* variant, int32_t* n_ranges) {
  *variant = 0;
  *n_ranges = o.n_ranges;
  if (!scan_tc_supported(idx->ix.D) || idx->ix.score_mode != 0 || idx->ix.stride > scan_tc_max_stride())
    return ROPE_OK;  // plan_scan reports why
  const TuneKey key = tune_key(idx, n_reads, o);
  TuneVal val;
  bool found;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    found = it != g_tune.end();
    if (found) val = it->second;
  }
  if (!found && may_tune && o.n_ranges == 0 && autotune_on()) {
    rope_status st = tune_tc(idx, emb_bf16, emb_f32, norms, n_reads, jb, je, o, c, stream, &val);
    if (st != ROPE_OK) return st;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = val;
    found = true;
  }
  if (found) {
    *variant = val.variant;
    const int g = scan_tc_group(idx->ix.D, val.variant);
    if (o.n_ranges == 0) *n_ranges = ranges_for(val.items_per_sm, c->num_sms, (n_reads + g - 1) / g);
  }
  return ROPE_OK;
}

}  // namespace

namespace {

// Scan of a materialised index: the A operand, the tcgen05 GEMM with its fused
// top-k (or every score into dense_out), then the merge with FP32 re-scoring
// from the stored FP32 window rows.
rope_status dense_scan(const rope_index* idx, const uint16_t* emb_bf16, const float* emb_f32, const float* norms,
                       int64_t n_reads, const rope_score_opts& o, int64_t jb, int64_t je, int64_t* out_win,
                       float* out_score, float* dense_out, cudaStream_t stream, int prof_slot,
                       const int64_t* out_row, const ThrOut* thr_out = nullptr) {
  const int mode = thr_out ? 2 : dense_out ? 1 : 0;
  const DevIndex& ix = idx->ix;
  // FP32: the plain CUDA-core scan over the stored FP32 rows (top-k only)
  const bool fp32 = o.precision == ROPE_PREC_FP32 && mode == 0;
  if (!fp32 && o.precision != ROPE_PREC_BF16)
    return fail(ROPE_ERR_UNSUPPORTED, "a materialised index is scored by the BF16 tensor-core GEMM or, for its top-k, "
                "the FP32 plain scan (precision %d)", o.precision);
  if (!fp32 && !emb_bf16) return fail(ROPE_ERR_INVALID_ARG, "the tensor-core scan needs emb_bf16");
  DeviceCtx* c;
  rope_status st = get_ctx(&c);
  if (st != ROPE_OK) return st;
  const int BM = fp32 ? dense_fp32_group() : gemm_tc_group(), BN = fp32 ? dense_fp32_group() : gemm_tc_window_tile();
  const int64_t n_pad = (n_reads + BM - 1) / BM * BM;
  if (2 * n_pad > 0x7FFFFFFF) return fail(ROPE_ERR_UNSUPPORTED, "more than 2^30 reads in one call");
  const int n_rt = (int)(n_pad / BM);
  const int64_t n_wt = je > jb ? (je - jb + BN - 1) / BN : 0;
  // waves of grp read tiles x n_ranges window ranges (one block each): the
  // grp read tiles' operands stay in L2 while each range's window tiles stream
  // past its grp blocks
  const int slots = fp32 ? 2 * c->num_sms : c->num_sms;  // blocks resident at once
  int grp, n_ranges;
  if ((int64_t)n_rt * 4 >= slots) {
    n_ranges = 4;
    grp = std::max(1, slots / 4);
  } else {
    grp = n_rt;
    n_ranges = std::max(1, slots / n_rt);
  }
  if (n_ranges > n_wt) n_ranges = (int)std::max<int64_t>(1, n_wt);
  const int64_t tiles_per_range = n_wt > 0 ? (n_wt + n_ranges - 1) / n_ranges : 1;
  if (n_wt > 0) n_ranges = (int)((n_wt + tiles_per_range - 1) / tiles_per_range);
  const int k_blocks = 2 * ix.D / 64;
  const int stages = fp32 ? 2 : gemm_tc_stages(mode == 0 ? o.cand_depth : 0, k_blocks);
  const int lists = fp32 ? 1 : gemm_tc_lists(k_blocks);  // candidate lists per (read, range)
  if (stages < 2) return fail(ROPE_ERR_UNSUPPORTED, "cand_depth=%d: the GEMM scan does not fit in shared memory", o.cand_depth);
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  const size_t a_bytes = fp32 ? 0 : al((size_t)n_pad * 2 * ix.D * sizeof(uint16_t));
  const size_t cand_bytes = mode != 0 ? 0 : (size_t)n_reads * n_ranges * lists * o.cand_depth * sizeof(Candidate);
  uint8_t* scratch = nullptr;
  if ((st = pool_alloc(c, (void**)&scratch, a_bytes + cand_bytes, stream)) != ROPE_OK) return st;
  uint16_t* a_op = reinterpret_cast<uint16_t*>(scratch);
  Candidate* cand = reinterpret_cast<Candidate*>(scratch + a_bytes);
  auto release = [&](rope_status r) {
    cudaFreeAsync(scratch, stream);
    return r;
  };
  cudaError_t e = cudaSuccess;
  if (n_wt > 0 && fp32) {
    GemmArgs g{};
    g.n_reads = n_reads;
    g.n_rt = n_rt;
    g.grp = grp;
    g.n_ranges = n_ranges;
    g.jb = jb;
    g.je = je;
    g.range_len = tiles_per_range * BN;
    g.cand_depth = o.cand_depth;
    g.sep = o.sep;
    g.stride = ix.stride;
    g.cand = cand;
    g.status = c->status;
    e = launch_dense_fp32(ix, g, emb_f32, norms, c->num_sms, stream);
    if (e != cudaSuccess) return release(fail(ROPE_ERR_CUDA, "FP32 scan launch: %s", cudaGetErrorString(e)));
  } else if (n_wt > 0) {
    CUtensorMap tmA;
    e = launch_gemm_a(emb_bf16, n_reads, n_pad, ix.D, a_op, stream);
    if (e != cudaSuccess) return release(fail(ROPE_ERR_CUDA, "A operand launch: %s", cudaGetErrorString(e)));
    if ((st = tensor_map_rows(&tmA, a_op, n_pad, 2 * ix.D)) != ROPE_OK) return release(st);
    GemmArgs g{};
    g.n_reads = n_reads;
    g.n_rt = n_rt;
    g.grp = grp;
    g.n_ranges = n_ranges;
    g.k_blocks = k_blocks;
    g.stages = stages;
    g.jb = jb;
    g.je = je;
    g.range_len = tiles_per_range * BN;
    g.cand_depth = mode == 0 ? o.cand_depth : 1;
    g.sep = o.sep;
    g.stride = ix.stride;
    g.cand = mode == 0 ? cand : nullptr;
    g.dense = dense_out;
    g.status = c->status;
    g.wait_limit_ns = wait_limit_ns();
    if (thr_out) g.thr = *thr_out;
    e = launch_gemm_tc(tmA, idx->tm_win, idx->tm_win_im, g, mode, c->num_sms, stream);
    if (e != cudaSuccess) return release(fail(ROPE_ERR_CUDA, "GEMM scan launch: %s", cudaGetErrorString(e)));
  } else if (mode == 0) {
    e = cudaMemsetAsync(cand, 0xFF, cand_bytes, stream);  // every slot empty
    if (e != cudaSuccess) return release(fail(ROPE_ERR_CUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e)));
  }
  if (mode != 0) return release(ROPE_OK);
  prof_mark(prof_slot, 2, stream);
  MergeArgs m{};
  m.cand = cand;
  m.n_reads = n_reads;
  m.n_ranges = n_ranges * lists;
  m.cand_depth = o.cand_depth;
  m.k = o.k;
  m.sep = o.sep;
  m.rescore = o.rescore;
  m.rescore_depth = o.rescore_depth;
  m.emb_f32 = emb_f32;
  m.norms = norms;
  m.out_win = out_win;
  m.out_score = out_score;
  m.out_row = out_row;
  m.status = c->status;
  e = launch_merge(ix, m, stream);
  prof_mark(prof_slot, 3, stream);
  if (e != cudaSuccess) return release(fail(ROPE_ERR_CUDA, "merge launch: %s", cudaGetErrorString(e)));
  return release(ROPE_OK);
}

}  // namespace

rope_status rope::score_topk_impl(const rope_index* idx, const float* emb_f32, const uint16_t* emb_bf16,
                                  const float* norms, int64_t n_reads, const rope_score_opts* opts, int64_t* out_win,
                                  float* out_score, cudaStream_t stream, int prof_slot, const int64_t* out_row, const ExtCandidates* ext) {
  if (!idx) return fail(ROPE_ERR_INVALID_ARG, "index is NULL");
  rope_score_opts o;
  rope_status st = check_opts(opts, &o);
  if (st != ROPE_OK) return st;
  if (n_reads < 0) return fail(ROPE_ERR_INVALID_ARG, "n_reads < 0");
  if (n_reads == 0) return ROPE_OK;
  if (!emb_f32 || !norms || !out_win || !out_score) return fail(ROPE_ERR_INVALID_ARG, "NULL pointer");
  if (prec_tc(o.precision) && !emb_bf16) return fail(ROPE_ERR_INVALID_ARG, "tensor-core scan needs emb_bf16");
  DeviceCtx* c;
  if ((st = get_ctx(&c)) != ROPE_OK) return st;
  const DevIndex& ix = idx->ix;
  const int64_t jb = o.j_begin > 0 ? o.j_begin : 0;
  const int64_t je = o.j_end > 0 ? (o.j_end < ix.W ? o.j_end : ix.W) : ix.W;
  if (jb > ix.W) return fail(ROPE_ERR_INVALID_ARG, "j_begin beyond the last window");
  if (idx->dense) {
    if (ext) return fail(ROPE_ERR_UNSUPPORTED, "a materialised index takes no caller candidate buffer");
    return dense_scan(idx, emb_bf16, emb_f32, norms, n_reads, o, jb, je, out_win, out_score, nullptr, stream,
                      prof_slot, out_row);
  }

  ScanPlan pl;
  Candidate* cand = nullptr;
  int32_t n_ranges = 1;  // candidate lists per read seen by the merge
  if (je > jb) {
    int32_t variant = 0, nr_req = o.n_ranges;
    if (prec_tc(o.precision) &&
        (st = choose_tc(idx, emb_bf16, emb_f32, norms, n_reads, jb, je, o, c, stream, ext == nullptr, &variant,
                        &nr_req)) != ROPE_OK)
      return st;
    if ((st = plan_scan(idx, o.precision, n_reads, jb, je, nr_req, c->num_sms, &pl, variant)) != ROPE_OK) return st;
    if (pl.tc && !scan_tc_fits(ix, o.cand_depth, variant, pl.a.fp8))
      return fail(ROPE_ERR_UNSUPPORTED, "cand_depth=%d: the tensor-core scan's candidate lists at complex "
                  "dimension %d and stride %d do not fit in shared memory; use a smaller cand_depth",
                  o.cand_depth, ix.D, ix.stride);
    n_ranges = pl.a.n_ranges * pl.a.lists_per_range;
  }
  const size_t cand_bytes = (size_t)n_reads * n_ranges * o.cand_depth * sizeof(Candidate);
  if (ext) {
    if (ext->bytes < cand_bytes)
      return fail(ROPE_ERR_INVALID_ARG, "candidate buffer of %zu bytes, %zu needed", ext->bytes, cand_bytes);
    cand = ext->cand;
  } else if ((st = pool_alloc(c, (void**)&cand, cand_bytes, stream)) != ROPE_OK) {
    return st;
  }
  // the pool block is returned on every exit below; a caller's buffer is not
  auto release = [&]() {
    if (!ext) cudaFreeAsync(cand, stream);
  };
  if (je > jb) {
    pl.a.emb_f32 = emb_f32;
    pl.a.emb_bf16 = emb_bf16;
    pl.a.norms = norms;
    pl.a.cand_depth = o.cand_depth;
    pl.a.sep = o.sep;
    pl.a.cand = cand;
    pl.a.dense = nullptr;
    pl.a.status = c->status;
    cudaError_t e = pl.tc ? launch_scan_tc(ix, pl.a, false, c->num_sms, stream)
                          : launch_scan_fp32(ix, pl.a, false, c->num_sms, stream);
    if (e != cudaSuccess) {
      release();
      return fail(ROPE_ERR_CUDA, "scan launch: %s", cudaGetErrorString(e));
    }
  } else {
    cudaError_t e = cudaMemsetAsync(cand, 0xFF, cand_bytes, stream);  // every slot empty
    if (e != cudaSuccess) {
      release();
      return fail(ROPE_ERR_CUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
    }
  }
  prof_mark(prof_slot, 2, stream);
  MergeArgs m{};
  m.cand = cand;
  m.n_reads = n_reads;
  m.n_ranges = n_ranges;
  m.cand_depth = o.cand_depth;
  m.k = o.k;
  m.sep = o.sep;
  m.rescore = o.rescore;
  m.rescore_depth = o.rescore_depth;
  m.emb_f32 = emb_f32;
  m.norms = norms;
  m.out_win = out_win;
  m.out_score = out_score;
  m.out_row = out_row;
  m.status = c->status;
  cudaError_t e = launch_merge(ix, m, stream);
  prof_mark(prof_slot, 3, stream);
  release();
  if (e != cudaSuccess) return fail(ROPE_ERR_CUDA, "merge launch: %s", cudaGetErrorString(e));
  return ROPE_OK;
}

rope_status rope::topk_cand_bytes(const rope_index* idx, int64_t n_reads, const rope_score_opts* opts,
                                  size_t* bytes) {
  if (!idx || !bytes) return fail(ROPE_ERR_INVALID_ARG, "NULL argument");
  rope_score_opts o;
  rope_status st = check_opts(opts, &o);
  if (st != ROPE_OK) return st;
  DeviceCtx* c;
  if ((st = get_ctx(&c)) != ROPE_OK) return st;
  const DevIndex& ix = idx->ix;
  const int64_t jb = o.j_begin > 0 ? o.j_begin : 0;
  const int64_t je = o.j_end > 0 ? (o.j_end < ix.W ? o.j_end : ix.W) : ix.W;
  int32_t n_ranges = 1;
  if (je > jb && n_reads > 0) {
    int32_t variant = 0, nr_req = o.n_ranges;
    if (prec_tc(o.precision) &&
        (st = choose_tc(idx, nullptr, nullptr, nullptr, n_reads, jb, je, o, c, nullptr, false, &variant, &nr_req)) !=
            ROPE_OK)
      return st;
    ScanPlan pl;
    if ((st = plan_scan(idx, o.precision, n_reads, jb, je, nr_req, c->num_sms, &pl, variant)) != ROPE_OK) return st;
    n_ranges = pl.a.n_ranges * pl.a.lists_per_range;
  }
  *bytes = (size_t)n_reads * n_ranges * o.cand_depth * sizeof(Candidate);
  return ROPE_OK;
}

extern "C" rope_status rope_autotune_enable(int32_t enabled) {
  if (enabled != 0 && enabled != 1) return fail(ROPE_ERR_INVALID_ARG, "enabled must be 0 or 1");
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_autotune = enabled;
  if (!enabled) g_tune.clear();
  return ROPE_OK;
}

extern "C" rope_status rope_autotune_set(const rope_index* idx, int64_t n_reads, const rope_score_opts* opts,
                                         int32_t variant, int32_t items_per_sm) {
  if (!idx || !opts || n_reads < 1) return fail(ROPE_ERR_INVALID_ARG, "bad arguments");
  rope_score_opts o;
  rope_status st = check_opts(opts, &o);
  if (st != ROPE_OK) return st;
  if (!scan_tc_supported(idx->ix.D)) return fail(ROPE_ERR_UNSUPPORTED, "no tensor-core scan at this dimension");
  if (variant < 0 || variant >= scan_tc_variants(idx->ix.D))
    return fail(ROPE_ERR_INVALID_ARG, "variant %d outside [0, %d)", variant, scan_tc_variants(idx->ix.D));
  if (items_per_sm < 1 || items_per_sm > 256) return fail(ROPE_ERR_INVALID_ARG, "items_per_sm outside [1, 256]");
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[tune_key(idx, n_reads, o)] = TuneVal{variant, items_per_sm, 0.f};
  return ROPE_OK;
}

extern "C" rope_status rope_autotune_query(const rope_index* idx, int64_t n_reads, const rope_score_opts* opts,
                                           int32_t* variant, int32_t* items_per_sm, float* sample_ms) {
  if (!idx || !opts || n_reads < 1) return fail(ROPE_ERR_INVALID_ARG, "bad arguments");
  rope_score_opts o;
  rope_status st = check_opts(opts, &o);
  if (st != ROPE_OK) return st;
  if (!scan_tc_supported(idx->ix.D)) return fail(ROPE_ERR_UNSUPPORTED, "no tensor-core scan at this dimension");
  const TuneKey key = tune_key(idx, n_reads, o);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find(key);
  if (it == g_tune.end()) return fail(ROPE_ERR_INVALID_ARG, "no tuned configuration for this shape class yet");
  if (variant) *variant = it->second.variant;
  if (items_per_sm) *items_per_sm = it->second.items_per_sm;
  if (sample_ms) *sample_ms = it->second.sample_ms;
  return ROPE_OK;
}

extern "C" rope_status rope_score_topk(const rope_index* idx, const float* emb_f32, const uint16_t* emb_bf16,
                                       const float* norms, int64_t n_reads, const rope_score_opts* opts,
                                       int64_t* out_win, float* out_score, cudaStream_t stream) {
  const int slot = prof_begin(stream);
  prof_mark(slot, 1, stream);
  const rope_status st = score_topk_impl(idx, emb_f32, emb_bf16, norms, n_reads, opts, out_win, out_score, stream,
                                         slot, nullptr, nullptr);
  if (slot >= 0 && st != ROPE_OK) {
    prof_mark(slot, 2, stream);
    prof_mark(slot, 3, stream);
  }
  return st;
}

extern "C" rope_status rope_score_threshold(const rope_index* idx, const uint16_t* emb_bf16, int64_t n_reads,
                                            const float* thr, int64_t j_begin, int64_t j_end, int64_t cap,
                                            int64_t* out_read, int64_t* out_win, float* out_score,
                                            unsigned long long* out_count, cudaStream_t stream) {
  if (!idx) return fail(ROPE_ERR_INVALID_ARG, "index is NULL");
  if (n_reads < 0 || cap < 0) return fail(ROPE_ERR_INVALID_ARG, "n_reads or cap < 0");
  if (!thr || !out_count || (cap > 0 && (!out_read || !out_win || !out_score)))
    return fail(ROPE_ERR_INVALID_ARG, "NULL pointer");
  const DevIndex& ix = idx->ix;
  const int64_t jb = j_begin > 0 ? j_begin : 0;
  const int64_t je = j_end > 0 ? (j_end < ix.W ? j_end : ix.W) : ix.W;
  if (jb > ix.W) return fail(ROPE_ERR_INVALID_ARG, "j_begin beyond the last window");
  ROPE_CUDA(cudaMemsetAsync(out_count, 0, sizeof(unsigned long long), stream));
  if (n_reads == 0 || je <= jb) return ROPE_OK;
  if (!emb_bf16) return fail(ROPE_ERR_INVALID_ARG, "threshold scan needs emb_bf16");
  if (idx->dense) {
    rope_score_opts o{};
    o.k = 1;
    o.precision = ROPE_PREC_BF16;
    o.cand_depth = 1;
    const ThrOut to{thr, out_count, cap, out_read, out_win, out_score};
    return dense_scan(idx, emb_bf16, nullptr, nullptr, n_reads, o, jb, je, nullptr, nullptr, nullptr, stream, -1,
                      nullptr, &to);
  }
  DeviceCtx* c;
  rope_status st = get_ctx(&c);
  if (st != ROPE_OK) return st;
  ScanPlan pl;
  if ((st = plan_scan(idx, ROPE_PREC_BF16, n_reads, jb, je, 0, c->num_sms, &pl, 0)) != ROPE_OK) return st;
  pl.a.emb_bf16 = emb_bf16;
  pl.a.cand_depth = 1;
  pl.a.status = c->status;
  const ThrOut to{thr, out_count, cap, out_read, out_win, out_score};
  const cudaError_t e = launch_scan_tc_threshold(ix, pl.a, to, c->num_sms, stream);
  if (e != cudaSuccess) return fail(ROPE_ERR_CUDA, "threshold scan launch: %s", cudaGetErrorString(e));
  return ROPE_OK;
}

extern "C" rope_status rope_score_dense(const rope_index* idx, const float* emb_f32, const uint16_t* emb_bf16,
                                        const float* norms, int64_t n_reads, int32_t precision, int64_t j_begin,
                                        int64_t count, float* out, cudaStream_t stream) {
  if (!idx) return fail(ROPE_ERR_INVALID_ARG, "index is NULL");
  if (n_reads < 0 || count < 0 || j_begin < 0 || j_begin + count > idx->ix.W)
    return fail(ROPE_ERR_INVALID_ARG, "bad dense range");
  if (n_reads == 0 || count == 0) return ROPE_OK;
  if (!emb_f32 || !norms || !out) return fail(ROPE_ERR_INVALID_ARG, "NULL pointer");
  if (prec_tc(precision) && !emb_bf16) return fail(ROPE_ERR_INVALID_ARG, "tensor-core scan needs emb_bf16");
  if (idx->dense) {
    rope_score_opts o{};
    o.k = 1;
    o.precision = precision;
    o.cand_depth = 1;
    return dense_scan(idx, emb_bf16, emb_f32, norms, n_reads, o, j_begin, j_begin + count, nullptr, nullptr, out,
                      stream, -1, nullptr);
  }
  DeviceCtx* c;
  rope_status st = get_ctx(&c);
  if (st != ROPE_OK) return st;
  ScanPlan pl;
  if ((st = plan_scan(idx, precision, n_reads, j_begin, j_begin + count, 0, c->num_sms, &pl)) != ROPE_OK) return st;
  pl.a.emb_f32 = emb_f32;
  pl.a.emb_bf16 = emb_bf16;
  pl.a.norms = norms;
  pl.a.cand_depth = 1;
  pl.a.sep = 0;
  pl.a.cand = nullptr;
  pl.a.dense = out;
  pl.a.status = c->status;
  cudaError_t e = pl.tc ? launch_scan_tc(idx->ix, pl.a, true, c->num_sms, stream)
                        : launch_scan_fp32(idx->ix, pl.a, true, c->num_sms, stream);
  if (e != cudaSuccess) return fail(ROPE_ERR_CUDA, "dense scan launch: %s", cudaGetErrorString(e));
  return ROPE_OK;
}

extern "C" rope_status rope_map(const rope_index* idx, const uint8_t* seqs, const int64_t* offsets, int64_t n_reads,
                                const rope_score_opts* opts, int64_t* out_win, float* out_score, cudaStream_t stream) {
  if (!idx) return fail(ROPE_ERR_INVALID_ARG, "index is NULL");
  rope_score_opts o;
  rope_status st = check_opts(opts, &o);
  if (st != ROPE_OK) return st;
  if (n_reads < 0) return fail(ROPE_ERR_INVALID_ARG, "n_reads < 0");
  if (n_reads == 0) return ROPE_OK;
  if (!seqs || !offsets || !out_win || !out_score) return fail(ROPE_ERR_INVALID_ARG, "NULL pointer");
  DeviceCtx* c;
  if ((st = get_ctx(&c)) != ROPE_OK) return st;
  const int D = idx->ix.D, m = idx->ix.m;
  float* emb = nullptr;
  uint16_t* embh = nullptr;
  float* norms = nullptr;
  if ((st = pool_alloc(c, (void**)&emb, (size_t)n_reads * 2 * D * sizeof(float), stream)) != ROPE_OK) return st;
  if ((st = pool_alloc(c, (void**)&embh, (size_t)n_reads * 2 * D * sizeof(uint16_t), stream)) != ROPE_OK) {
    cudaFreeAsync(emb, stream);
    return st;
  }
  if ((st = pool_alloc(c, (void**)&norms, (size_t)n_reads * (1 + m) * sizeof(float), stream)) != ROPE_OK) {
    cudaFreeAsync(emb, stream);
    cudaFreeAsync(embh, stream);
    return st;
  }
  const int slot = prof_begin(stream);
  cudaError_t e = launch_encode_reads(idx->enc, seqs, offsets, n_reads, emb, embh, norms, c->status, stream);
  prof_mark(slot, 1, stream);
  if (e != cudaSuccess) st = fail(ROPE_ERR_CUDA, "encode launch: %s", cudaGetErrorString(e));
  if (st == ROPE_OK) {
    o.j_begin = 0;
    o.j_end = 0;
    st = score_topk_impl(idx, emb, embh, norms, n_reads, &o, out_win, out_score, stream, slot, nullptr, nullptr);
  }
  if (slot >= 0 && st != ROPE_OK) {
    prof_mark(slot, 2, stream);
    prof_mark(slot, 3, stream);
  }
  cudaFreeAsync(emb, stream);
  cudaFreeAsync(embh, stream);
  cudaFreeAsync(norms, stream);
  return st;
}

extern "C" rope_status rope_map_strands(const rope_index* idx, const uint8_t* seqs, const int64_t* offsets,
                                        int64_t n_reads, const rope_score_opts* opts, int64_t* out_win,
                                        float* out_score, int8_t* out_strand, cudaStream_t stream) {
  if (!idx) return fail(ROPE_ERR_INVALID_ARG, "index is NULL");
  rope_score_opts o;
  rope_status st = check_opts(opts, &o);
  if (st != ROPE_OK) return st;
  if (n_reads < 0) return fail(ROPE_ERR_INVALID_ARG, "n_reads < 0");
  if (n_reads == 0) return ROPE_OK;
  if (!seqs || !offsets || !out_win || !out_score || !out_strand) return fail(ROPE_ERR_INVALID_ARG, "NULL pointer");
  DeviceCtx* c;
  if ((st = get_ctx(&c)) != ROPE_OK) return st;
  const int D = idx->ix.D, m = idx->ix.m, k = o.k;
  const size_t n2 = 2 * (size_t)n_reads;
  // one scratch block: emb_f32 | norms | win2 | score2 | emb_bf16 (rows n..2n-1: reverse strand)
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  const size_t b_f32 = al(n2 * 2 * D * sizeof(float)), b_norm = al(n2 * (1 + m) * sizeof(float));
  const size_t b_win = al(n2 * k * sizeof(int64_t)), b_sc = al(n2 * k * sizeof(float));
  const size_t b_bf16 = al(n2 * 2 * D * sizeof(uint16_t));
  uint8_t* scratch = nullptr;
  if ((st = pool_alloc(c, (void**)&scratch, b_f32 + b_norm + b_win + b_sc + b_bf16, stream)) != ROPE_OK) return st;
  float* emb = reinterpret_cast<float*>(scratch);
  float* norms = reinterpret_cast<float*>(scratch + b_f32);
  int64_t* win2 = reinterpret_cast<int64_t*>(scratch + b_f32 + b_norm);
  float* score2 = reinterpret_cast<float*>(scratch + b_f32 + b_norm + b_win);
  uint16_t* embh = reinterpret_cast<uint16_t*>(scratch + b_f32 + b_norm + b_win + b_sc);
  const int slot = prof_begin(stream);
  cudaError_t e = launch_encode_reads(idx->enc, seqs, offsets, n_reads, emb, embh, norms, c->status, stream);
  if (e == cudaSuccess)
    e = launch_encode_reads(idx->enc, seqs, offsets, n_reads, emb + (size_t)n_reads * 2 * D,
                            embh + (size_t)n_reads * 2 * D, norms + (size_t)n_reads * (1 + m), c->status, stream,
                            nullptr, true);
  prof_mark(slot, 1, stream);
  if (e != cudaSuccess) st = fail(ROPE_ERR_CUDA, "encode launch: %s", cudaGetErrorString(e));
  if (st == ROPE_OK) {
    o.j_begin = 0;
    o.j_end = 0;
    st = score_topk_impl(idx, emb, embh, norms, (int64_t)n2, &o, win2, score2, stream, slot, nullptr, nullptr);
  }
  if (st == ROPE_OK) {
    e = launch_strand_merge(win2, score2, n_reads, k, out_win, out_score, out_strand, stream);
    if (e != cudaSuccess) st = fail(ROPE_ERR_CUDA, "strand merge launch: %s", cudaGetErrorString(e));
  }
  if (slot >= 0 && st != ROPE_OK) {
    prof_mark(slot, 2, stream);
    prof_mark(slot, 3, stream);
  }
  cudaFreeAsync(scratch, stream);
  return st;
}

// ---------------------------------------------------------------- allocation-free scan
//
// rope_score_topk_noalloc: the same scan, merge and re-scoring as
// rope_score_topk, for callers that must not have the library allocate device
// memory at call time -- for example a process that hands nearly all device
// memory to its own arena up front, or a latency-critical loop that cannot
// afford the device-wide synchronisation cudaMalloc/cudaFree imply. Its scratch
// (a status word and the per-read candidate lists) is this file-scope array,
// which every GPU that loads the library holds until the process exits.

namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)16 << 20;  // 16 MiB per device
constexpr size_t kNoAllocHeadBytes = 256;                   // status word, padded
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[kNoAllocMaxDevices];  // device address of g_noalloc_scratch
int g_noalloc_sms[kNoAllocMaxDevices];

// Once per device, with that device current: the host-side name of the array
// is only a stand-in, so fetch the array's device address.
rope_status noalloc_setup(int dev, void** addr, int* sms) {
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return fail(ROPE_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    int n = 0;
    e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return fail(ROPE_ERR_CUDA, "cudaDeviceGetAttribute: %s", cudaGetErrorString(e));
    g_noalloc_sms[dev] = n;
    g_noalloc_addr[dev] = p;
  }
  *addr = g_noalloc_addr[dev];
  *sms = g_noalloc_sms[dev];
  return ROPE_OK;
}

}  // namespace

extern "C" rope_status rope_score_topk_noalloc(const rope_index* idx, const float* emb_f32, const uint16_t* emb_bf16,
                                               const float* norms, int64_t n_reads, const rope_score_opts* opts,
                                               int64_t* out_win, float* out_score, cudaStream_t stream) {
  if (!idx) return fail(ROPE_ERR_INVALID_ARG, "index is NULL");
  rope_score_opts o;
  rope_status st = check_opts(opts, &o);
  if (st != ROPE_OK) return st;
  if (n_reads < 0) return fail(ROPE_ERR_INVALID_ARG, "n_reads < 0");
  if (n_reads == 0) return ROPE_OK;
  if (!emb_f32 || !norms || !out_win || !out_score) return fail(ROPE_ERR_INVALID_ARG, "NULL pointer");
  if (prec_tc(o.precision) && !emb_bf16) return fail(ROPE_ERR_INVALID_ARG, "tensor-core scan needs emb_bf16");
  int dev = 0;
  ROPE_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(ROPE_ERR_UNSUPPORTED, "device ordinal %d", dev);
  void* base = nullptr;
  int num_sms = 0;
  if (idx->dense)
    return fail(ROPE_ERR_UNSUPPORTED, "the allocation-free scan takes the on-the-fly index, not a materialised one");
  if ((st = noalloc_setup(dev, &base, &num_sms)) != ROPE_OK) return st;

  const DevIndex& ix = idx->ix;
  const int64_t jb = o.j_begin > 0 ? o.j_begin : 0;
  const int64_t je = o.j_end > 0 ? (o.j_end < ix.W ? o.j_end : ix.W) : ix.W;
  if (jb > ix.W) return fail(ROPE_ERR_INVALID_ARG, "j_begin beyond the last window");
  const size_t cap = kNoAllocScratchBytes - kNoAllocHeadBytes;
  const size_t per_range = (size_t)n_reads * o.cand_depth * sizeof(Candidate);
  if (per_range > cap)
    return fail(ROPE_ERR_INVALID_ARG,
                "n_reads=%lld x cand_depth=%d needs %zu bytes of candidates per window range; the allocation-free "
                "scratch holds %zu bytes (at most %zu reads at this depth)",
                (long long)n_reads, o.cand_depth, per_range, cap, cap / ((size_t)o.cand_depth * sizeof(Candidate)));

  ScanPlan pl;
  int32_t n_ranges = 1;  // candidate lists per read seen by the merge
  if (je > jb) {
    int32_t variant = 0, nr_req = o.n_ranges;
    if (prec_tc(o.precision)) {
      // an earlier tuned choice for this shape class, if any (never tunes here:
      // tuning allocates)
      DeviceCtx tmp{};
      tmp.num_sms = num_sms;
      if ((st = choose_tc(idx, emb_bf16, emb_f32, norms, n_reads, jb, je, o, &tmp, stream, false, &variant,
                          &nr_req)) != ROPE_OK)
        return st;
    }
    if ((st = plan_scan(idx, o.precision, n_reads, jb, je, nr_req, num_sms, &pl, variant)) != ROPE_OK) return st;
    if (pl.tc && !scan_tc_fits(idx->ix, o.cand_depth, variant, pl.a.fp8))
      return fail(ROPE_ERR_UNSUPPORTED, "cand_depth=%d: the tensor-core scan's candidate lists at complex "
                  "dimension %d and stride %d do not fit in shared memory; use a smaller cand_depth",
                  o.cand_depth, idx->ix.D, idx->ix.stride);
    const size_t lpr = (size_t)pl.a.lists_per_range;
    if ((size_t)pl.a.n_ranges * lpr * per_range > cap) {
      if (o.n_ranges > 0)
        return fail(ROPE_ERR_INVALID_ARG, "n_ranges=%d needs %zu bytes of scratch; the allocation-free scratch "
                    "holds %zu", o.n_ranges, (size_t)pl.a.n_ranges * lpr * per_range, cap);
      if (lpr * per_range > cap)
        return fail(ROPE_ERR_INVALID_ARG, "n_reads=%lld needs %zu bytes of candidates; the allocation-free scratch "
                    "holds %zu", (long long)n_reads, lpr * per_range, cap);
      if ((st = plan_scan(idx, o.precision, n_reads, jb, je, (int32_t)(cap / (lpr * per_range)), num_sms, &pl,
                          variant)) != ROPE_OK)
        return st;
    }
    n_ranges = pl.a.n_ranges * pl.a.lists_per_range;
  }
  int* status = static_cast<int*>(base);
  Candidate* cand = reinterpret_cast<Candidate*>(static_cast<unsigned char*>(base) + kNoAllocHeadBytes);
  const size_t cand_bytes = (size_t)n_ranges * per_range;
  // The call's status word starts at zero and every candidate slot empty on
  // every call: a scan block that gives up on a bounded wait leaves its lists
  // unwritten, and those slots must not show the previous call's candidates.
  // The merge also ORs the call's bits into the sticky word (status[1]) that
  // rope_noalloc_sync_status reads and clears.
  ROPE_CUDA(cudaMemsetAsync(status, 0, sizeof(int), stream));
  ROPE_CUDA(cudaMemsetAsync(cand, 0xFF, cand_bytes, stream));
  if (je > jb) {
    pl.a.emb_f32 = emb_f32;
    pl.a.emb_bf16 = emb_bf16;
    pl.a.norms = norms;
    pl.a.cand_depth = o.cand_depth;
    pl.a.sep = o.sep;
    pl.a.cand = cand;
    pl.a.dense = nullptr;
    pl.a.status = status;
    cudaError_t e = pl.tc ? launch_scan_tc(ix, pl.a, false, num_sms, stream)
                          : launch_scan_fp32(ix, pl.a, false, num_sms, stream);
    if (e != cudaSuccess) return fail(ROPE_ERR_CUDA, "scan launch: %s", cudaGetErrorString(e));
  }
  MergeArgs m{};
  m.empty_on_timeout = 1;
  m.sticky_status = status + 1;
  m.cand = cand;
  m.n_reads = n_reads;
  m.n_ranges = n_ranges;
  m.cand_depth = o.cand_depth;
  m.k = o.k;
  m.sep = o.sep;
  m.rescore = o.rescore;
  m.rescore_depth = o.rescore_depth;
  m.emb_f32 = emb_f32;
  m.norms = norms;
  m.out_win = out_win;
  m.out_score = out_score;
  m.status = status;
  cudaError_t e = launch_merge(ix, m, stream);
  if (e != cudaSuccess) return fail(ROPE_ERR_CUDA, "merge launch: %s", cudaGetErrorString(e));
  return ROPE_OK;
}

extern "C" rope_status rope_noalloc_sync_status(cudaStream_t stream) {
  int dev = 0;
  ROPE_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(ROPE_ERR_UNSUPPORTED, "device ordinal %d", dev);
  void* base = nullptr;
  int num_sms = 0;
  rope_status st = noalloc_setup(dev, &base, &num_sms);
  if (st != ROPE_OK) return st;
  ROPE_CUDA(cudaStreamSynchronize(stream));
  int* sticky = static_cast<int*>(base) + 1;
  int v = 0;
  ROPE_CUDA(cudaMemcpy(&v, sticky, sizeof(int), cudaMemcpyDeviceToHost));
  ROPE_CUDA(cudaMemset(sticky, 0, sizeof(int)));
  if (v & kStatusTimeout)
    return fail(ROPE_ERR_TIMEOUT, "a bounded in-kernel wait ran out; the results were set to (-1, -inf)");
  if (v & kStatusBadArg) return fail(ROPE_ERR_INVALID_ARG, "a kernel saw an out-of-range argument");
  return ROPE_OK;
}
