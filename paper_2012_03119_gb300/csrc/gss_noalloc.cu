// gss_noalloc.cu -- gss_test_noalloc: the clause test without any device allocation.
//
// Who needs this: programs that must not allocate GPU memory at the moment they test
// clauses -- for example a solver whose device memory is owned by another runtime's
// pool (a framework that reserved the GPU up front), or a latency-sensitive loop in which
// a cudaMalloc, which may synchronise the whole device, is not acceptable.  They pass
// their own device buffers for the clauses, the value codes and the results; everything
// else the test needs (status words, a copy of the offsets, the head planes and the bit
// planes) lives in one fixed array compiled into the library, sized GSS_NOALLOC_SCRATCH_BYTES.
//
// The array is a file-scope __device__ variable: every GPU that loads the library holds it
// until the process exits, and every call on a device reuses it, so calls that overlap on
// the GPU (two streams, two threads) race on it.  Host code cannot use the array's name as
// a device address; the first call on each device asks the runtime for the address
// (cudaGetSymbolAddress, with that device current) and keeps it together with the identity
// of the device's current context.  A later call in another context of that device (after
// a cudaDeviceReset, say) looks the address up again instead of using the old one.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <mutex>

#include "gss_internal.h"

using namespace gss;

static __device__ __align__(256) unsigned char g_noalloc_scratch[GSS_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mutex;
unsigned char* g_scratch_addr[MAX_DEVICES] = {};
unsigned long long g_scratch_ctx[MAX_DEVICES] = {};  // id of the context the address belongs to

// Identity of the calling thread's current context (driver entry points fetched through the
// runtime, so the library links no driver library); 0 when there is none or it cannot be told.
unsigned long long current_context_id() {
  using GetCurrent = CUresult (*)(CUcontext*);
  using GetId = CUresult (*)(CUcontext, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {  // under g_setup_mutex
    looked_up = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<GetCurrent>(p);
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<GetId>(p);
  }
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

int say(char* buf, size_t len, int code, const char* msg) {
  if (buf && len) {
    strncpy(buf, msg, len - 1);
    buf[len - 1] = '\0';
  }
  return code;
}

uint64_t up256(uint64_t x) { return (x + 255) / 256 * 256; }

// Address of this device's scratch array, looked up with that device current on the first
// call and again whenever the device's current context is not the one it was looked up in.
cudaError_t scratch_for(int dev, unsigned char** out) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  const unsigned long long ctx = current_context_id();
  if (!g_scratch_addr[dev] || ctx == 0 || ctx != g_scratch_ctx[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);  // makes the primary context current
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<unsigned char*>(p);
    g_scratch_ctx[dev] = current_context_id();
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" int gss_test_noalloc(const uint64_t* d_offsets, uint64_t n_clauses, const uint32_t* d_lits, uint32_t n_vars,
                                const uint8_t* d_values, uint64_t pitch, uint32_t n_assign, uint32_t mode,
                                gss_report* d_out, uint64_t cap, unsigned long long* d_count, void* stream,
                                char* errbuf, size_t errbuf_len) {
  if (errbuf && errbuf_len) errbuf[0] = '\0';
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!d_count) return say(errbuf, errbuf_len, GSS_E_INVAL, "d_count is NULL");
  if (n_vars == 0 || n_vars >= (1u << 31)) return say(errbuf, errbuf_len, GSS_E_INVAL, "n_vars out of range");
  if (mode != GSS_MODE_ALLF && mode != GSS_MODE_TRIGGER) return say(errbuf, errbuf_len, GSS_E_INVAL, "unknown mode");
  if (n_assign > GSS_MAX_NARROW_ASSIGNMENTS)
    return say(errbuf, errbuf_len, GSS_E_INVAL, "n_assign > GSS_MAX_NARROW_ASSIGNMENTS");
  if (n_clauses >= (1ull << 32)) return say(errbuf, errbuf_len, GSS_E_INVAL, "more than 2^32 - 1 clauses");
  if (n_clauses && (!d_offsets || !d_lits)) return say(errbuf, errbuf_len, GSS_E_INVAL, "clause arrays are NULL");
  if (n_assign && !d_values) return say(errbuf, errbuf_len, GSS_E_INVAL, "d_values is NULL");
  if (cap && !d_out) return say(errbuf, errbuf_len, GSS_E_INVAL, "d_out is NULL");
  if (n_assign && (pitch < n_vars || pitch % 16 != 0 || reinterpret_cast<uintptr_t>(d_values) % 16 != 0))
    return say(errbuf, errbuf_len, GSS_E_INVAL, "d_values must be 16-byte aligned with pitch >= n_vars, pitch % 16 == 0");

  // scratch layout: status[2] | offsets copy | head0 | head1 | P | aggF | aggU
  uint32_t Wp = 4;
  while (Wp < (n_assign + 31) / 32) Wp <<= 1;
  const uint32_t AWp = Wp <= 32 ? 1 : Wp / 32;
  const uint64_t o_off = up256(2 * sizeof(DevStatus));
  const uint64_t o_h0 = o_off + up256((n_clauses + 1) * sizeof(uint64_t));
  const uint64_t o_h1 = o_h0 + up256(n_clauses * 32);
  const uint64_t o_P = o_h1 + up256(n_clauses * 32);
  const uint64_t o_aF = o_P + up256((2ull * n_vars + 2) * Wp * 4);
  const uint64_t o_aU = o_aF + up256((2ull * n_vars + 2) * AWp * 4);
  const uint64_t total = o_aU + up256((n_vars + 1ull) * AWp * 4);
  if (total > GSS_NOALLOC_SCRATCH_BYTES) {
    char msg[200];
    snprintf(msg, sizeof msg, "problem needs %llu bytes of scratch, more than GSS_NOALLOC_SCRATCH_BYTES (%llu)",
             (unsigned long long)total, (unsigned long long)GSS_NOALLOC_SCRATCH_BYTES);
    return say(errbuf, errbuf_len, GSS_E_INVAL, msg);
  }

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES)
    return say(errbuf, errbuf_len, GSS_E_CUDA, "no usable current device");
  unsigned char* base = nullptr;
  cudaError_t e = scratch_for(dev, &base);
  if (e != cudaSuccess) return say(errbuf, errbuf_len, GSS_E_CUDA, cudaGetErrorString(e));
  DevStatus* st = reinterpret_cast<DevStatus*>(base);
  uint64_t* off = reinterpret_cast<uint64_t*>(base + o_off);
  uint32_t* head0 = reinterpret_cast<uint32_t*>(base + o_h0);
  uint32_t* head1 = reinterpret_cast<uint32_t*>(base + o_h1);
  uint32_t* P = reinterpret_cast<uint32_t*>(base + o_P);
  uint32_t* aggF = reinterpret_cast<uint32_t*>(base + o_aF);
  uint32_t* aggU = reinterpret_cast<uint32_t*>(base + o_aU);

#define NA_CK(call)                                                              \
  do {                                                                           \
    cudaError_t e_ = (call);                                                     \
    if (e_ != cudaSuccess) return say(errbuf, errbuf_len, GSS_E_CUDA, cudaGetErrorString(e_)); \
  } while (0)

  // every call starts from zeroed status words and record count (the array keeps old contents)
  NA_CK(cudaMemsetAsync(st, 0, 2 * sizeof(DevStatus), s));
  NA_CK(cudaMemsetAsync(d_count, 0, sizeof(unsigned long long), s));
  if (n_clauses == 0 || n_assign == 0) {
    NA_CK(cudaStreamSynchronize(s));
    return GSS_OK;
  }
  uint64_t ends[2] = {1, 0};
  NA_CK(cudaMemcpyAsync(&ends[0], d_offsets, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
  NA_CK(cudaMemcpyAsync(&ends[1], d_offsets + n_clauses, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
  NA_CK(cudaStreamSynchronize(s));
  if (ends[0] != 0) return say(errbuf, errbuf_len, GSS_E_INVAL, "offsets[0] must be 0");
  const uint64_t L = ends[1];
  NA_CK(cudaMemsetAsync(off, 0, sizeof(uint64_t), s));
  NA_CK(launch_validate(d_offsets, n_clauses, L, 0, off, d_lits, n_vars, st + 1, s));
  DevStatus h[2];
  NA_CK(cudaMemcpyAsync(h, st, sizeof h, cudaMemcpyDeviceToHost, s));
  NA_CK(cudaStreamSynchronize(s));
  if (h[1].bad_size) return say(errbuf, errbuf_len, GSS_E_INVAL, "empty clause or offsets not increasing");
  if (h[1].bad_lit) return say(errbuf, errbuf_len, GSS_E_INVAL, "literal >= 2 * n_vars");

  NA_CK(launch_build_heads(d_offsets, n_clauses, 0, head0, head1, d_lits, n_vars, s));
  NA_CK(launch_pack(d_values, pitch, n_vars, n_assign, Wp, AWp, nullptr, P, aggF, aggU, st, s));
  int n_sms = 1;
  cudaDeviceGetAttribute(&n_sms, cudaDevAttrMultiProcessorCount, dev);
  const ClauseView db{off, d_lits, head0, head1, 2u * n_vars};
  const PlaneView pv{P, aggF, aggU, Wp, AWp, n_assign, n_vars};
  const int cpw = test_tile_shape(n_clauses, L);
  NA_CK(launch_test((int)mode, db, 0, n_clauses, pv, d_out, cap, st, test_grid_size((int)mode, AWp, n_sms, false, cpw), s,
                    nullptr, 0, ActivityView{}, WideView{}, cpw));
  NA_CK(cudaMemcpyAsync(d_count, &st->n_records, sizeof(unsigned long long), cudaMemcpyDeviceToDevice, s));
  NA_CK(cudaMemcpyAsync(h, st, sizeof h, cudaMemcpyDeviceToHost, s));
  NA_CK(cudaStreamSynchronize(s));
#undef NA_CK
  if (h[0].bad_code) return say(errbuf, errbuf_len, GSS_E_INVAL, "value code outside {0 = U, 1 = T, 2 = F}");
  if (h[0].timeout) return say(errbuf, errbuf_len, GSS_E_TIMEOUT, "a bounded device wait gave up");
  if (h[0].n_records > cap) return say(errbuf, errbuf_len, GSS_E_OVERFLOW, "more records than cap (count written)");
  return GSS_OK;
}
