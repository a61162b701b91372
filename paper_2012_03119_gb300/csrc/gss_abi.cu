// gss_abi.cu -- host implementation of the C ABI declared in include/gss.h.
//
// Owns the context: device buffers (clause database, assignment planes, report
// buffer, status words), the stream, validation and error reporting.  Every step
// of the tested path runs in the kernels of k_ingest.cu, k_pack.cu and k_test.cu;
// this file only sizes buffers, copies host data in and out, and launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <unordered_map>

#include "gss_ctx.h"

using namespace gss;
using namespace gss::host;

namespace gss {
namespace host {

std::atomic<long> g_alloc_counter{0};

int fail(gss_ctx* c, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return code;
}

#define CK(ctx, call)                                                                         \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess) return fail((ctx), GSS_E_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

struct DeviceGuard {
  int prev = -1;
  bool changed = false;
  explicit DeviceGuard(int d) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != d) changed = cudaSetDevice(d) == cudaSuccess;
  }
  ~DeviceGuard() {
    if (changed && prev >= 0) cudaSetDevice(prev);
  }
};

// Host-side fault injection for tests: GSS_FAULT_ALLOC_AT=n fails the n-th device
// allocation of the process (1-based) with GSS_E_NOMEM; no GPU fault is involved.
bool injected_alloc_failure() {
  const char* s = getenv("GSS_FAULT_ALLOC_AT");
  long n = g_alloc_counter.fetch_add(1) + 1;
  return s && *s && atol(s) == n;
}

int dev_alloc(gss_ctx* c, void** p, uint64_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 256;
  if (injected_alloc_failure()) return fail(c, GSS_E_NOMEM, "injected allocation failure (%llu bytes)",
                                            (unsigned long long)bytes);
  if (c->budget && c->bytes + bytes > c->budget)
    return fail(c, GSS_E_NOMEM, "memory budget exceeded: %llu + %llu > %llu bytes", (unsigned long long)c->bytes,
                (unsigned long long)bytes, (unsigned long long)c->budget);
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(c, GSS_E_NOMEM, "cudaMalloc(%llu): %s", (unsigned long long)bytes, cudaGetErrorString(e));
  }
  c->bytes += bytes;
  c->allocs[*p] = bytes;
  return GSS_OK;
}

void dev_free(gss_ctx* c, void* p) {
  if (!p) return;
  auto it = c->allocs.find(p);
  if (it != c->allocs.end()) {
    c->bytes -= it->second;
    c->allocs.erase(it);
  }
  cudaFree(p);
}

// Grow a device array to hold `need` elements, preserving the first `used`.
template <class T>
int grow(gss_ctx* c, T*& ptr, uint64_t& cap, uint64_t used, uint64_t need) {
  if (need <= cap && ptr) return GSS_OK;
  uint64_t ncap = cap + cap / 2;
  if (ncap < need) ncap = need;
  if (ncap < 1024) ncap = 1024;
  void* np = nullptr;
  int rc = dev_alloc(c, &np, ncap * sizeof(T));
  if (rc) return rc;
  if (ptr && used) {
    cudaError_t e = cudaMemcpyAsync(np, ptr, used * sizeof(T), cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
      dev_free(c, np);
      return fail(c, GSS_E_CUDA, "grow copy: %s", cudaGetErrorString(e));
    }
  }
  dev_free(c, ptr);
  ptr = static_cast<T*>(np);
  cap = ncap;
  return GSS_OK;
}

uint32_t words_stride(uint32_t N) {  // plane row stride in 32-bit words: a power of two >= 4
  const uint32_t W = (N + 31) / 32;
  uint32_t p = 4;
  while (p < W) p <<= 1;
  return p;
}

uint32_t agg_stride(uint32_t Wp) { return Wp <= 32 ? 1 : Wp / 32; }  // 1, 2, 4, ... 32 words

// Point the latest-set aliases (P, aggF, ...) at plane set b.
void use_set(gss_ctx* c, uint32_t b) {
  c->cur = b;
  c->P = c->sets[b].P;
  c->aggF = c->sets[b].aggF;
  c->aggU = c->sets[b].aggU;
  c->agg2F = c->sets[b].agg2F;
  c->agg2U = c->sets[b].agg2U;
}

int ensure_planes(gss_ctx* c) {  // allocates what is missing, so a call after a failed one completes the sets
  const uint32_t Wp = words_stride(c->max_N), AWp = agg_stride(Wp);
  int rc;
  void* p;
  for (uint32_t b = 0; b < c->pipeline; ++b) {
    gss_ctx::PlaneSet& q = c->sets[b];
    if (!q.P) {
      if ((rc = dev_alloc(c, &p, (2ull * c->V + 2) * Wp * 4))) return rc;
      q.P = static_cast<uint32_t*>(p);
    }
    if (!q.aggF) {
      if ((rc = dev_alloc(c, &p, (2ull * c->V + 2) * AWp * 4))) return rc;
      q.aggF = static_cast<uint32_t*>(p);
    }
    if (!q.aggU) {
      if ((rc = dev_alloc(c, &p, (c->V + 1ull) * AWp * 4))) return rc;
      q.aggU = static_cast<uint32_t*>(p);
    }
    if (AWp > 4 && !q.agg2F) {
      if ((rc = dev_alloc(c, &p, (2ull * c->V + 2) * 4))) return rc;
      q.agg2F = static_cast<uint32_t*>(p);
    }
    if (AWp > 4 && !q.agg2U) {
      if ((rc = dev_alloc(c, &p, (c->V + 1ull) * 4))) return rc;
      q.agg2U = static_cast<uint32_t*>(p);
    }
  }
  use_set(c, c->cur);
  return GSS_OK;
}

// Read the ingest status and the status of the plane set the last test read (the other
// set's may be in the middle of a packing on pack_stream).
int sync_status(gss_ctx* c) {
  const uint32_t i = set_status_index(c->tested_set);
  CK(c, cudaMemcpyAsync(c->h_st + 1, c->st + 1, sizeof(DevStatus), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaMemcpyAsync(c->h_st + i, c->st + i, sizeof(DevStatus), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  return GSS_OK;
}

int launch_grid(gss_ctx* c, int mode, uint32_t AWp, int cpw) {
  const bool wide = AWp > 4;
  int& g = wide ? c->grid_wide[mode] : c->grid[mode][AWp][cpw == 16 ? 1 : 0];
  if (!g) g = test_grid_size(mode, AWp, c->n_sms, wide, cpw);
  return g;
}

void release(gss_ctx* c) {
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->pack_stream && c->pack_stream != c->stream) cudaStreamSynchronize(c->pack_stream);
  if (c->copy_stream) cudaStreamSynchronize(c->copy_stream);
  while (!c->allocs.empty()) dev_free(c, c->allocs.begin()->first);
  if (c->h_st) cudaFreeHost(c->h_st);
  for (int b = 0; b < 2; ++b) {
    if (c->ev_packed[b]) cudaEventDestroy(c->ev_packed[b]);
    if (c->ev_tested[b]) cudaEventDestroy(c->ev_tested[b]);
    if (c->ev_staged[b]) cudaEventDestroy(c->ev_staged[b]);
  }
  if (c->ev_copied) cudaEventDestroy(c->ev_copied);

  if (c->own_pack_stream && c->pack_stream) cudaStreamDestroy(c->pack_stream);
  if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
}

}  // namespace host
}  // namespace gss

extern "C" {

int gss_config_init(gss_config* cfg) {
  if (!cfg) return GSS_E_INVAL;
  memset(cfg, 0, sizeof *cfg);
  cfg->device = 0;
  cfg->stream = nullptr;
  cfg->report_capacity = 1ull << 22;
  cfg->max_assignments = 1024;
  cfg->mode = GSS_MODE_ALLF;
  cfg->mem_budget_bytes = 0;
  cfg->layout = GSS_LAYOUT_FREQUENCY;
  cfg->pipeline = 1;
  cfg->pack_stream = nullptr;
  cfg->clauses_per_tile = 0;
  return GSS_OK;
}

int gss_create(gss_ctx** out, uint32_t n_vars, const gss_config* cfg_in) {
  if (!out) return GSS_E_INVAL;
  *out = nullptr;
  gss_config cfg;
  if (cfg_in) cfg = *cfg_in; else gss_config_init(&cfg);
  if (n_vars == 0 || n_vars >= (1u << 31)) return GSS_E_INVAL;
  if (cfg.max_assignments == 0 || cfg.max_assignments > GSS_MAX_ASSIGNMENTS) return GSS_E_INVAL;
  if (cfg.mode != GSS_MODE_ALLF && cfg.mode != GSS_MODE_TRIGGER) return GSS_E_INVAL;
  if (cfg.layout != GSS_LAYOUT_IDENTITY && cfg.layout != GSS_LAYOUT_FREQUENCY) return GSS_E_INVAL;
  if (cfg.pipeline != 1 && cfg.pipeline != 2) return GSS_E_INVAL;
  if (cfg.clauses_per_tile != 0 && cfg.clauses_per_tile != 16 && cfg.clauses_per_tile != 32) return GSS_E_INVAL;
  int n_dev = 0;
  if (cudaGetDeviceCount(&n_dev) != cudaSuccess || cfg.device < 0 || cfg.device >= n_dev) {
    cudaGetLastError();
    return GSS_E_CUDA;
  }
  gss_ctx* c = new (std::nothrow) gss_ctx();
  if (!c) return GSS_E_NOMEM;
  DeviceGuard dg(cfg.device);
  c->device = cfg.device;
  c->V = n_vars;
  c->max_N = cfg.max_assignments;
  c->mode = cfg.mode;
  c->layout = cfg.layout;
  c->budget = cfg.mem_budget_bytes;
  c->Vp = (n_vars + 15ull) / 16 * 16;
  int rc = GSS_OK;
  if (cudaDeviceGetAttribute(&c->n_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) c->n_sms = 1;
  if (cfg.stream) {
    c->stream = static_cast<cudaStream_t>(cfg.stream);
  } else if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
    delete c;
    return GSS_E_CUDA;
  } else {
    c->own_stream = true;
  }
  c->pipeline = cfg.pipeline;
  c->tile_clauses = cfg.clauses_per_tile;
  c->pack_stream = c->stream;
  if (c->pipeline == 2) {
    if (cfg.pack_stream) {
      c->pack_stream = static_cast<cudaStream_t>(cfg.pack_stream);
    } else if (cudaStreamCreateWithFlags(&c->pack_stream, cudaStreamNonBlocking) != cudaSuccess) {
      c->pack_stream = nullptr;
      rc = GSS_E_CUDA;
    } else {
      c->own_pack_stream = true;
    }
    if (!rc && cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking) != cudaSuccess) {
      c->copy_stream = nullptr;
      rc = GSS_E_CUDA;
    }
    for (int b = 0; b < 2 && !rc; ++b)
      if (cudaEventCreateWithFlags(&c->ev_packed[b], cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&c->ev_tested[b], cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&c->ev_staged[b], cudaEventDisableTiming) != cudaSuccess)
        rc = GSS_E_CUDA;
  }
  if (!rc && cudaEventCreateWithFlags(&c->ev_copied, cudaEventDisableTiming) != cudaSuccess) rc = GSS_E_CUDA;

  void* p = nullptr;
  if (!rc && cudaMallocHost(&p, 3 * sizeof(DevStatus)) != cudaSuccess) rc = GSS_E_NOMEM;
  c->h_st = static_cast<DevStatus*>(p);
  if (!rc) rc = dev_alloc(c, &p, 3 * sizeof(DevStatus));
  if (!rc) {
    c->st = static_cast<DevStatus*>(p);
    if (cudaMemsetAsync(c->st, 0, 3 * sizeof(DevStatus), c->stream) != cudaSuccess) rc = GSS_E_CUDA;
  }
  if (!rc) {
    c->rec_cap = cfg.report_capacity ? cfg.report_capacity : 1;
    rc = dev_alloc(c, &p, c->rec_cap * sizeof(gss_report));
    c->rec = static_cast<gss_report*>(p);
  }
  if (!rc) {
    rc = grow(c, c->off, c->cap_m, 0, 1025);
    if (!rc && cudaMemsetAsync(c->off, 0, sizeof(uint64_t), c->stream) != cudaSuccess) rc = GSS_E_CUDA;
  }
  if (!rc && cudaStreamSynchronize(c->stream) != cudaSuccess) rc = GSS_E_CUDA;
  if (rc) {
    release(c);
    delete c;
    return rc;
  }
  *out = c;
  return GSS_OK;
}

int gss_destroy(gss_ctx* c) {
  if (!c) return GSS_OK;
  DeviceGuard dg(c->device);
  release(c);
  delete c;
  return GSS_OK;
}

int gss_add_clauses(gss_ctx* c, const uint64_t* offsets, uint64_t n, const uint32_t* lits, uint32_t* first_id) {
  if (!c) return GSS_E_INVAL;
  TraceRange tr("gss_add_clauses");
  c->err.clear();
  if (n == 0) {
    if (first_id) *first_id = (uint32_t)c->next_id;
    return GSS_OK;
  }
  if (!offsets) return fail(c, GSS_E_INVAL, "offsets is NULL");
  if (offsets[0] != 0) return fail(c, GSS_E_INVAL, "offsets[0] must be 0");
  const uint64_t L = offsets[n];
  if (L && !lits) return fail(c, GSS_E_INVAL, "lits is NULL");
  if (c->next_id + n >= (1ull << 32)) return fail(c, GSS_E_INVAL, "more than 2^32 - 1 clauses");
  DeviceGuard dg(c->device);
  int rc;
  if (c->act) {  // activities and bump stamps of the new clauses
    if ((rc = grow(c, c->act, c->cap_act, c->m, c->m + n))) return rc;
    if ((rc = grow(c, c->stamp, c->cap_stamp, c->m, c->m + n))) return rc;
  }
  if (c->ext && (rc = grow(c, c->ext, c->cap_ext, c->m, c->m + n))) return rc;
  // cap_m counts offsets entries (m + 1); head capacities count literals (8 per clause per plane)
  if ((rc = grow(c, c->off, c->cap_m, c->m + 1, c->m + n + 1))) return rc;
  if ((rc = grow(c, c->head0, c->cap_head0, c->m * 8, (c->m + n) * 8))) return rc;
  if ((rc = grow(c, c->head1, c->cap_head1, c->m * 8, (c->m + n) * 8))) return rc;
  if ((rc = grow(c, c->lits, c->cap_L, c->L, c->L + L))) return rc;
  if ((rc = grow(c, c->boff, c->cap_boff, 0, n + 1))) return rc;
  CK(c, cudaMemsetAsync(c->st + 1, 0, sizeof(DevStatus), c->stream));
  CK(c, cudaMemcpyAsync(c->boff, offsets, (n + 1) * sizeof(uint64_t), cudaMemcpyHostToDevice, c->stream));
  if (L) CK(c, cudaMemcpyAsync(c->lits + c->L, lits, L * sizeof(uint32_t), cudaMemcpyHostToDevice, c->stream));
  uint32_t* blits = c->lits + c->L;  // this batch's literals (caller numbering until translated)
  CK(c, launch_validate(c->boff, n, L, c->L, c->off + c->m, blits, c->V, c->st + 1, c->stream));
  if ((rc = sync_status(c))) return rc;
  if (c->h_st[1].bad_size) return fail(c, GSS_E_INVAL, "empty clause or offsets not increasing / past the batch");
  if (c->h_st[1].bad_lit) return fail(c, GSS_E_INVAL, "literal >= 2 * n_vars (%u)", 2 * c->V);
  if (c->layout == GSS_LAYOUT_FREQUENCY && !c->map) {  // the first batch fixes the numbering
    void* pm = nullptr;
    void* ps = nullptr;
    if ((rc = dev_alloc(c, &pm, (uint64_t)c->V * sizeof(uint32_t)))) return rc;
    if ((rc = dev_alloc(c, &ps, rank_scratch_words(c->V) * sizeof(uint32_t)))) {
      dev_free(c, pm);
      return rc;
    }
    cudaError_t e = launch_rank_vars(blits, L, c->V, static_cast<uint32_t*>(ps), static_cast<uint32_t*>(pm), c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    dev_free(c, ps);
    if (e != cudaSuccess) {
      dev_free(c, pm);
      return fail(c, GSS_E_CUDA, "variable ranking: %s", cudaGetErrorString(e));
    }
    c->map = static_cast<uint32_t*>(pm);
    if (c->have_assign && c->N) {  // a set packed before the numbering existed: pack it again in the numbering
      c->pack_set = c->cur;
      if ((rc = pack_staged(c, c->pack_stream))) return rc;
    }
  }
  if (c->map) CK(c, launch_translate(blits, L, c->map, c->stream));
  CK(c, launch_build_heads(c->boff, n, c->L, c->head0 + c->m * 8, c->head1 + c->m * 8, c->lits, c->V, c->stream));
  if (c->act) {  // a new clause starts at the current increment, as if bumped once
    CK(c, launch_fill_f32(c->act + c->m, n, c->inc, c->stream));
    CK(c, launch_fill_u32(c->stamp + c->m, n, 0xFFFFFFFFu, c->stream));
  }
  if (c->ext) CK(c, launch_iota_u32(c->ext + c->m, n, (uint32_t)c->next_id, c->stream));
  if (first_id) *first_id = (uint32_t)c->next_id;
  c->m += n;
  c->L += L;
  c->next_id += n;
  return GSS_OK;
}

}  // extern "C"

namespace gss {
namespace host {
int reserve_db(gss_ctx* c, uint64_t max_clauses, uint64_t max_lits) {
  if (!c) return GSS_E_INVAL;
  if (max_clauses >= (1ull << 32)) return fail(c, GSS_E_INVAL, "more than 2^32 - 1 clauses");
  DeviceGuard dg(c->device);
  int rc;
  if ((rc = grow(c, c->off, c->cap_m, c->m + 1, max_clauses + 1))) return rc;
  if ((rc = grow(c, c->head0, c->cap_head0, c->m * 8, max_clauses * 8))) return rc;
  if ((rc = grow(c, c->head1, c->cap_head1, c->m * 8, max_clauses * 8))) return rc;
  if ((rc = grow(c, c->lits, c->cap_L, c->L, max_lits ? max_lits : 1))) return rc;
  return GSS_OK;
}

int stage_assignments(gss_ctx* c, const uint8_t* src, uint64_t pitch, uint32_t n, bool device_src, bool wait_copy) {
  if (!c) return GSS_E_INVAL;
  c->err.clear();
  if (n > c->max_N) return fail(c, GSS_E_INVAL, "n_assign %u > max_assignments %u", n, c->max_N);
  if (n && !src) return fail(c, GSS_E_INVAL, "values is NULL");
  if (device_src && pitch < c->V) return fail(c, GSS_E_INVAL, "pitch %llu < n_vars %u", (unsigned long long)pitch, c->V);
  DeviceGuard dg(c->device);
  int rc;
  if ((rc = ensure_planes(c))) return rc;
  // pipeline 2: the set the last test did not read; packing waits for the last test that read it
  const uint32_t b = c->pipeline == 2 ? (c->cur ^ 1u) : 0u;
  cudaStream_t ps = c->pack_stream;
  c->have_assign = false;
  if (b == c->tested_set) c->tested = false;  // its status words are reset below: the last test's results go
  if (c->pipeline == 2) CK(c, cudaStreamWaitEvent(ps, c->ev_tested[b], 0));
  CK(c, cudaMemsetAsync(set_status(c, b), 0, sizeof(DevStatus), ps));
  const uint32_t Wp = words_stride(n ? n : 1);
  const uint32_t AWp = agg_stride(Wp);
  const uint8_t* codes = src;
  uint64_t cpitch = pitch;
  // the packing kernel reads codes with 2-D TMA boxes: rows 16-byte aligned
  const bool aligned = device_src && pitch % 16 == 0 && (reinterpret_cast<uintptr_t>(src) % 16) == 0;
  if (n && !aligned) {  // host data, or a device layout the packing kernel cannot read as 32-bit words
    // pipeline 1: one staging buffer, the copy queued on the packing stream behind the packing
    // that still reads it.  pipeline 2: set b's own buffer; host values are copied on
    // copy_stream once the last packing of set b has read it, and the packing waits for the
    // copy.  Device values are copied on pack_stream, where a caller may order the work that
    // writes them.
    gss_ctx::PlaneSet& q = c->sets[b];
    cudaStream_t cs = (c->pipeline == 2 && !device_src) ? c->copy_stream : ps;
    if (q.codes_rows < n) {
      CK(c, cudaStreamSynchronize(ps));  // a packing may still read the old buffer
      if (cs != ps) CK(c, cudaStreamSynchronize(cs));
      dev_free(c, q.codes);
      q.codes = nullptr;
      q.codes_rows = 0;
      void* p;
      if ((rc = dev_alloc(c, &p, (uint64_t)c->max_N * c->Vp))) return rc;
      q.codes = static_cast<uint8_t*>(p);
      q.codes_rows = c->max_N;
      CK(c, cudaMemsetAsync(q.codes, 0, (uint64_t)c->max_N * c->Vp, cs));  // padding columns stay U
    }
    if (cs != ps) CK(c, cudaStreamWaitEvent(cs, c->ev_packed[b], 0));
    const uint64_t spitch = device_src ? pitch : c->V;
    const cudaMemcpyKind kind = device_src ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    // rows contiguous on both sides: one linear copy (a pitched copy of the same rows ran 3 % slower)
    if (spitch == c->V && c->V == c->Vp)
      CK(c, cudaMemcpyAsync(q.codes, src, (uint64_t)n * c->V, kind, cs));
    else
      CK(c, cudaMemcpy2DAsync(q.codes, c->Vp, src, spitch, c->V, n, kind, cs));
    if (cs != ps) {
      CK(c, cudaEventRecord(c->ev_staged[b], cs));
      CK(c, cudaStreamWaitEvent(ps, c->ev_staged[b], 0));
    }
    if (!device_src) {  // the caller may reuse its host buffer once this call (or gss_copy_wait) returns
      CK(c, cudaEventRecord(c->ev_copied, cs));
      if (wait_copy) CK(c, cudaEventSynchronize(c->ev_copied));
    }
    codes = q.codes;
    cpitch = c->Vp;
  }
  c->pack_src = codes;
  c->pack_pitch = cpitch;
  c->pack_set = b;
  c->sets[b].N = n;
  c->N = n;
  c->Wp = Wp;
  c->AWp = AWp;
  use_set(c, b);
  c->have_assign = true;
  return GSS_OK;
}

int pack_staged(gss_ctx* c, cudaStream_t s) {
  const uint32_t b = c->pack_set;
  const gss_ctx::PlaneSet& q = c->sets[b];
  DevStatus* st = set_status(c, b);
  if (c->N) CK(c, launch_pack(c->pack_src, c->pack_pitch, c->V, c->N, c->Wp, c->AWp, c->map, q.P, q.aggF, q.aggU, st,
                              s));
  if (c->N && c->AWp > 4) CK(c, launch_agg2(q.aggF, q.aggU, c->V, c->AWp, q.agg2F, q.agg2U, s));
  if (c->pipeline == 2) CK(c, cudaEventRecord(c->ev_packed[b], s));
  return GSS_OK;
}
}  // namespace host
}  // namespace gss

extern "C" {

static int set_assignments_common(gss_ctx* c, const uint8_t* src, uint64_t pitch, uint32_t n, bool device_src,
                                  bool wait_copy = true) {
  TraceRange tr("gss_set_assignments (pack)");
  int rc = stage_assignments(c, src, pitch, n, device_src, wait_copy);
  if (rc) return rc;
  DeviceGuard dg(c->device);
  return pack_staged(c, c->pack_stream);
}

int gss_set_assignments(gss_ctx* c, const uint8_t* values, uint32_t n_assign) {
  return set_assignments_common(c, values, 0, n_assign, false);
}

int gss_set_assignments_async(gss_ctx* c, const uint8_t* values, uint32_t n_assign) {
  return set_assignments_common(c, values, 0, n_assign, false, false);
}

int gss_copy_wait(gss_ctx* c) {
  if (!c) return GSS_E_INVAL;
  c->err.clear();
  DeviceGuard dg(c->device);
  CK(c, cudaEventSynchronize(c->ev_copied));  // recorded after every host copy, in queue order
  return GSS_OK;
}

int gss_set_assignments_device(gss_ctx* c, const uint8_t* d_values, uint64_t pitch, uint32_t n_assign) {
  return set_assignments_common(c, d_values, pitch, n_assign, true);
}

int gss_test(gss_ctx* c) {
  if (!c) return GSS_E_INVAL;
  TraceRange tr("gss_test");
  c->err.clear();
  if (!c->have_assign) return fail(c, GSS_E_STATE, "gss_test before gss_set_assignments");
  DeviceGuard dg(c->device);
  const uint32_t b = c->cur;
  DevStatus* st = set_status(c, b);
  if (c->pipeline == 2) CK(c, cudaStreamWaitEvent(c->stream, c->ev_packed[b], 0));  // the set's packing
  CK(c, cudaMemsetAsync(&st->n_records, 0, 3 * sizeof(unsigned long long), c->stream));  // records, candidates, super
  if (c->m && c->N) {
    ClauseView db{c->off, c->lits, c->head0, c->head1, 2u * c->V, c->ext};
    PlaneView pv{c->P, c->aggF, c->aggU, c->Wp, c->AWp, c->N, c->V};
    WideView wv;
    if (c->AWp > 4) {  // stage A on the level-2 rows, the level-1 rows in stage B
      pv = PlaneView{c->P, c->agg2F, c->agg2U, c->Wp, 1u, c->N, c->V};
      wv = WideView{c->aggF, c->aggU, c->AWp};
    }
    ActivityView av;
    if (c->act) av = ActivityView{c->act, c->stamp, c->epoch, c->inc};
    const int cpw = c->tile_clauses ? (int)c->tile_clauses : test_tile_shape(c->m, c->L);
    CK(c, launch_test((int)c->mode, db, 0, c->m, pv, c->rec, c->rec_cap, st, launch_grid(c, c->mode, c->AWp, cpw),
                      c->stream, nullptr, 0, av, wv, cpw));
  }
  if (c->pipeline == 2) CK(c, cudaEventRecord(c->ev_tested[b], c->stream));  // set b may be packed again after this
  c->tested_set = b;
  c->tested_N = c->N;
  if (c->act) {  // after the test's bumps: the increment grows by 1 / decay, rescaled past 1e20
    c->epoch = c->epoch + 1 == 0xFFFFFFFFu ? 0 : c->epoch + 1;
    c->inc = c->inc * c->inv_decay;
    if (c->inc > 1e20f) {
      CK(c, launch_scale_f32(c->act, c->m, 1e-20f, c->stream));
      c->inc = c->inc * 1e-20f;
    }
  }
  c->tested = true;
  c->counted = false;
  c->tests_run += 1;
  c->pair_tests += c->m * (uint64_t)c->N;
  return GSS_OK;
}

}  // extern "C"

namespace gss {
namespace host {
int wait_test(gss_ctx* c, uint64_t* n, bool sync) {
  if (!c->tested) return fail(c, GSS_E_STATE, "no gss_test to fetch");
  int rc = sync ? sync_status(c) : GSS_OK;
  if (rc) return rc;
  const DevStatus& h = c->h_st[set_status_index(c->tested_set)];
  if (h.bad_code) {
    *n = 0;
    return fail(c, GSS_E_INVAL, "assignment value code outside {0 = U, 1 = T, 2 = F}");
  }
  if (h.timeout) {
    *n = 0;
    return fail(c, GSS_E_TIMEOUT, "a bounded device wait gave up; the records of this test are incomplete");
  }
  *n = h.n_records;
  if (!c->counted) {
    c->counted = true;
    c->records += *n;
    c->overflows += *n > c->rec_cap ? 1 : 0;
  }
  return GSS_OK;
}
}  // namespace host
}  // namespace gss

extern "C" {

int gss_fetch_reports(gss_ctx* c, gss_report* out, uint64_t cap, uint64_t* n_out) {
  TraceRange tr("gss_fetch_reports");
  if (!c || (cap && !out)) return c ? fail(c, GSS_E_INVAL, "out is NULL") : GSS_E_INVAL;
  c->err.clear();
  DeviceGuard dg(c->device);
  uint64_t n = 0;
  int rc = wait_test(c, &n, true);
  if (n_out) *n_out = n;
  if (rc) return rc;
  uint64_t k = n < cap ? n : cap;
  if (k > c->rec_cap) k = c->rec_cap;
  if (k) {
    CK(c, cudaMemcpyAsync(out, c->rec, k * sizeof(gss_report), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
  }
  if (n > c->rec_cap)
    return fail(c, GSS_E_OVERFLOW, "device report buffer overflowed: %llu records > capacity %llu; "
                "raise it with gss_set_report_capacity and re-run gss_test",
                (unsigned long long)n, (unsigned long long)c->rec_cap);
  if (n > cap)
    return fail(c, GSS_E_OVERFLOW, "%llu records > caller capacity %llu", (unsigned long long)n,
                (unsigned long long)cap);
  return GSS_OK;
}

int gss_fetch_reports_async(gss_ctx* c, gss_report* out, uint64_t cap) {
  TraceRange tr("gss_fetch_reports_async");
  if (!c || (cap && !out)) return c ? fail(c, GSS_E_INVAL, "out is NULL") : GSS_E_INVAL;
  c->err.clear();
  if (!c->tested) return fail(c, GSS_E_STATE, "no gss_test to fetch");
  DeviceGuard dg(c->device);
  gss_report* dst = out;
  if (cap) {  // the copy kernel writes out directly: it must be memory the GPU can write
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, out) != cudaSuccess) {
      cudaGetLastError();
      return fail(c, GSS_E_INVAL, "out: not a pointer the runtime knows");
    }
    if (a.type == cudaMemoryTypeHost) {
      if (!a.devicePointer) return fail(c, GSS_E_INVAL, "out: pinned host memory not mapped for the device");
      dst = static_cast<gss_report*>(a.devicePointer);
    } else if (a.type == cudaMemoryTypeUnregistered) {
      int pageable = 0;
      if (cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, c->device) != cudaSuccess || !pageable)
        return fail(c, GSS_E_INVAL, "out: pageable host memory, which this device cannot write; pin it");
    }
  }
  CK(c, launch_copy_records(c->rec, set_status(c, c->tested_set), c->rec_cap, cap, dst, 2 * c->n_sms, c->stream));
  c->fetch_pending = true;
  c->fetch_cap = cap;
  return GSS_OK;
}

int gss_fetch_wait(gss_ctx* c, uint64_t* n_out) {
  if (!c) return GSS_E_INVAL;
  c->err.clear();
  if (!c->fetch_pending) return fail(c, GSS_E_STATE, "no gss_fetch_reports_async to wait for");
  c->fetch_pending = false;
  DeviceGuard dg(c->device);
  uint64_t n = 0;
  int rc = wait_test(c, &n, true);  // synchronises the stream: the records have landed
  if (n_out) *n_out = n;
  if (rc) return rc;
  if (n > c->rec_cap)
    return fail(c, GSS_E_OVERFLOW, "device report buffer overflowed: %llu records > capacity %llu; "
                "raise it with gss_set_report_capacity and re-run gss_test",
                (unsigned long long)n, (unsigned long long)c->rec_cap);
  if (n > c->fetch_cap)
    return fail(c, GSS_E_OVERFLOW, "%llu records > caller capacity %llu", (unsigned long long)n,
                (unsigned long long)c->fetch_cap);
  return GSS_OK;
}

int gss_report_count(gss_ctx* c, uint64_t* n_out) {
  if (!c || !n_out) return GSS_E_INVAL;
  c->err.clear();
  DeviceGuard dg(c->device);
  int rc = wait_test(c, n_out, true);
  if (rc) return rc;
  if (*n_out > c->rec_cap)
    return fail(c, GSS_E_OVERFLOW, "device report buffer overflowed: %llu records > capacity %llu",
                (unsigned long long)*n_out, (unsigned long long)c->rec_cap);
  return GSS_OK;
}

int gss_reports_device(gss_ctx* c, const gss_report** d_records, uint64_t* capacity) {
  if (!c || !d_records) return GSS_E_INVAL;
  *d_records = c->rec;
  if (capacity) *capacity = c->rec_cap;
  return GSS_OK;
}

int gss_set_report_capacity(gss_ctx* c, uint64_t cap) {
  if (!c || cap == 0) return c ? fail(c, GSS_E_INVAL, "capacity must be > 0") : GSS_E_INVAL;
  c->err.clear();
  DeviceGuard dg(c->device);
  CK(c, cudaStreamSynchronize(c->stream));
  void* p = nullptr;
  int rc = dev_alloc(c, &p, cap * sizeof(gss_report));
  if (rc) return rc;
  dev_free(c, c->rec);
  c->rec = static_cast<gss_report*>(p);
  c->rec_cap = cap;
  c->tested = false;
  return GSS_OK;
}

int gss_set_mode(gss_ctx* c, uint32_t mode) {
  if (!c) return GSS_E_INVAL;
  if (mode != GSS_MODE_ALLF && mode != GSS_MODE_TRIGGER) return fail(c, GSS_E_INVAL, "unknown mode %u", mode);
  c->mode = mode;
  return GSS_OK;
}

int gss_debug_bounds(uint32_t* enabled, uint64_t* errors, int reset) {
#ifdef GSS_DEBUG_BOUNDS
  if (enabled) *enabled = 1;
#else
  if (enabled) *enabled = 0;
#endif
  unsigned long long n = 0;
  if (cudaDeviceSynchronize() != cudaSuccess || debug_bounds_errors(&n, reset != 0) != cudaSuccess) {
    cudaGetLastError();
    return GSS_E_CUDA;
  }
  if (errors) *errors = n;
  return GSS_OK;
}

int gss_get_stats(const gss_ctx* c, gss_stats* o) {
  if (!c || !o) return GSS_E_INVAL;
  o->n_vars = c->V;
  o->n_assign = c->have_assign ? c->N : 0;
  o->n_clauses = c->m;
  o->n_lits = c->L;
  o->device_bytes = c->bytes;
  o->report_capacity = c->rec_cap;
  o->tests_run = c->tests_run;
  o->pair_tests = c->pair_tests;
  const DevStatus& h = c->h_st[set_status_index(c->tested_set)];
  o->candidate_pairs = c->tested ? h.n_candidates : 0;
  o->super_pairs = c->tested ? h.n_super : 0;
  o->clauses_removed = c->removed;
  o->records = c->records;
  o->overflows = c->overflows;
  o->next_clause_id = c->next_id;
  o->group_pairs = c->tested ? c->m * (uint64_t)((c->tested_N + 31) / 32) : 0;
  return GSS_OK;
}

const char* gss_last_error(const gss_ctx* c) {
  if (!c) return "no context";
  return c->err.c_str();
}

const char* gss_strerror(int code) {
  switch (code) {
    case GSS_OK: return "GSS_OK";
    case GSS_E_INVAL: return "GSS_E_INVAL";
    case GSS_E_NOMEM: return "GSS_E_NOMEM";
    case GSS_E_CUDA: return "GSS_E_CUDA";
    case GSS_E_OVERFLOW: return "GSS_E_OVERFLOW";
    case GSS_E_TIMEOUT: return "GSS_E_TIMEOUT";
    case GSS_E_BUSY: return "GSS_E_BUSY";
    case GSS_E_STATE: return "GSS_E_STATE";
    default: return "GSS_E_UNKNOWN";
  }
}

uint32_t gss_version(void) { return (0u << 16) | 1u; }

}  // extern "C"
