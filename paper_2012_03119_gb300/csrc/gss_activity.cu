// gss_activity.cu -- database upkeep on a context: clause activity and activity-based
// deletion (Section 3.6:
// the GPU, like the CPU solvers, has to delete clauses or it would slow down and run out of
// memory; it deletes by activity as MiniSat does, and bumps a clause whenever it triggers).
//
// The bumps happen inside the test kernel (one per clause per test); the increment is kept
// on the host and grows by 1 / decay after every test, with MiniSat's rescale by 1e-20 once
// it passes 1e20 (see gss_test).  gss_reduce_db removes the requested fraction of the
// clauses longer than two literals with the smallest (activity, id) and compacts the
// database in place of the old arrays; ids stay with their clauses and are never reused.
// gss_export_clauses copies the resident database back out in the caller's numbering.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "gss_ctx.h"

using namespace gss;
using namespace gss::host;

namespace {

struct Guard {  // the context's device, restored afterwards
  int prev = -1;
  explicit Guard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~Guard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

#define ACK(call)                                                                          \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) return fail(c, GSS_E_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

template <class T>
int alloc(gss_ctx* c, T*& p, uint64_t n) {
  void* q = nullptr;
  const int rc = dev_alloc(c, &q, (n ? n : 1) * sizeof(T));
  p = static_cast<T*>(q);
  return rc;
}

// Grow p (capacity cap elements, the first `used` kept) to n elements.
template <class T>
int reserve_array(gss_ctx* c, T*& p, uint64_t& cap, uint64_t used, uint64_t n) {
  if (!p || cap >= n) return GSS_OK;
  T* q = nullptr;
  int rc = alloc(c, q, n);
  if (rc) return rc;
  cudaError_t e = used ? cudaMemcpyAsync(q, p, used * sizeof(T), cudaMemcpyDeviceToDevice, c->stream) : cudaSuccess;
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    dev_free(c, q);
    return fail(c, GSS_E_CUDA, "reserve: %s", cudaGetErrorString(e));
  }
  dev_free(c, p);
  p = q;
  cap = n;
  return GSS_OK;
}

}  // namespace

namespace gss {
namespace host {
int reserve_clause_arrays(gss_ctx* c, uint64_t max_clauses) {
  Guard g(c->device);
  int rc;
  if ((rc = reserve_array(c, c->act, c->cap_act, c->m, max_clauses))) return rc;
  if ((rc = reserve_array(c, c->stamp, c->cap_stamp, c->m, max_clauses))) return rc;
  return reserve_array(c, c->ext, c->cap_ext, c->m, max_clauses);
}
}  // namespace host
}  // namespace gss

extern "C" {

int gss_set_activity(gss_ctx* c, float decay) {
  if (!c) return GSS_E_INVAL;
  c->err.clear();
  if (!(decay > 0.0f && decay <= 1.0f)) return fail(c, GSS_E_INVAL, "decay must be in (0, 1]");
  Guard g(c->device);
  if (!c->act) {  // clauses already resident start at the increment, like new ones
    int rc;
    const uint64_t cap = c->m > 1024 ? c->m : 1024;
    if ((rc = alloc(c, c->act, cap))) return rc;
    if ((rc = alloc(c, c->stamp, cap))) {
      dev_free(c, c->act);
      c->act = nullptr;
      return rc;
    }
    c->cap_act = c->cap_stamp = cap;
    c->inc = 1.0f;
    c->epoch = 0;
    ACK(launch_fill_f32(c->act, c->m, c->inc, c->stream));
    ACK(launch_fill_u32(c->stamp, c->m, 0xFFFFFFFFu, c->stream));
  }
  c->decay = decay;
  c->inv_decay = 1.0f / decay;
  return GSS_OK;
}

int gss_get_activity(gss_ctx* c, float* out, uint64_t cap, uint64_t* n_out) {
  if (!c) return GSS_E_INVAL;
  c->err.clear();
  if (!c->act) return fail(c, GSS_E_STATE, "activity is off (gss_set_activity)");
  if (n_out) *n_out = c->m;
  Guard g(c->device);
  const uint64_t k = cap < c->m ? cap : c->m;
  if (k && !out) return fail(c, GSS_E_INVAL, "out is NULL");
  if (k) ACK(cudaMemcpyAsync(out, c->act, k * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
  ACK(cudaStreamSynchronize(c->stream));
  if (cap < c->m) return fail(c, GSS_E_OVERFLOW, "%llu clauses > capacity %llu", (unsigned long long)c->m,
                              (unsigned long long)cap);
  return GSS_OK;
}

int gss_get_clause_ids(gss_ctx* c, uint32_t* out, uint64_t cap, uint64_t* n_out) {
  if (!c) return GSS_E_INVAL;
  c->err.clear();
  if (n_out) *n_out = c->m;
  const uint64_t k = cap < c->m ? cap : c->m;
  if (k && !out) return fail(c, GSS_E_INVAL, "out is NULL");
  Guard g(c->device);
  if (c->ext) {
    if (k) ACK(cudaMemcpyAsync(out, c->ext, k * sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream));
    ACK(cudaStreamSynchronize(c->stream));
  } else {
    for (uint64_t i = 0; i < k; ++i) out[i] = (uint32_t)i;  // nothing removed yet: id = position
  }
  if (cap < c->m) return fail(c, GSS_E_OVERFLOW, "%llu clauses > capacity %llu", (unsigned long long)c->m,
                              (unsigned long long)cap);
  return GSS_OK;
}

int gss_reduce_db(gss_ctx* c, double remove_fraction, uint64_t* n_removed) {
  if (!c) return GSS_E_INVAL;
  TraceRange tr("gss_reduce_db");
  c->err.clear();
  if (n_removed) *n_removed = 0;
  if (!(remove_fraction >= 0.0 && remove_fraction <= 1.0)) return fail(c, GSS_E_INVAL, "fraction outside [0, 1]");
  if (!c->act) return fail(c, GSS_E_STATE, "gss_reduce_db needs activities (gss_set_activity)");
  if (c->m == 0) return GSS_OK;
  Guard g(c->device);
  int rc;
  uint32_t* hist = nullptr;
  if ((rc = alloc(c, hist, 256))) return rc;
  std::vector<uint32_t> h(256);
  auto pass = [&](uint32_t shift, uint64_t prefix) -> int {
    ACK(launch_key_hist(c->off, c->act, c->ext, c->m, shift, prefix, hist, c->stream));
    ACK(cudaMemcpyAsync(h.data(), hist, 256 * sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream));
    ACK(cudaStreamSynchronize(c->stream));
    return GSS_OK;
  };
  // the first pass also counts the candidates: every clause longer than two literals
  if ((rc = pass(56, 0))) {
    dev_free(c, hist);
    return rc;
  }
  uint64_t n_long = 0;
  for (uint32_t b = 0; b < 256; ++b) n_long += h[b];
  const uint64_t n_remove = (uint64_t)std::floor(remove_fraction * (double)n_long);
  if (n_remove == 0) {
    dev_free(c, hist);
    return GSS_OK;
  }
  // radix select of the key of rank n_remove - 1 (ascending), 8 bits per pass
  uint64_t r = n_remove - 1, prefix = 0;
  for (int shift = 56;; shift -= 8) {
    uint64_t below = 0;
    uint32_t b = 0;
    while (b < 255 && below + h[b] <= r) below += h[b++];  // r < the bucket counts' sum
    r -= below;
    prefix = (prefix << 8) | b;
    if (shift == 0) break;
    if ((rc = pass((uint32_t)shift - 8, prefix))) {
      dev_free(c, hist);
      return rc;
    }
  }
  dev_free(c, hist);
  const uint64_t kmax = prefix;  // the largest removed key

  // plan: keep flags and scans, then the kept counts
  void* scratch = nullptr;
  unsigned long long* d_counts = nullptr;
  if ((rc = dev_alloc(c, &scratch, compact_scratch_bytes(c->m)))) return rc;
  if ((rc = alloc(c, d_counts, 2))) {
    dev_free(c, scratch);
    return rc;
  }
  unsigned long long counts[2] = {0, 0};
  cudaError_t e = launch_compact_plan(c->off, c->act, c->ext, c->m, kmax, scratch, d_counts, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(counts, d_counts, sizeof counts, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  dev_free(c, d_counts);
  if (e != cudaSuccess) {
    dev_free(c, scratch);
    return fail(c, GSS_E_CUDA, "compaction plan: %s", cudaGetErrorString(e));
  }
  const uint64_t nm = counts[0], nL = counts[1];
  if (nm + n_remove != c->m) {
    dev_free(c, scratch);
    return fail(c, GSS_E_CUDA, "compaction kept %llu of %llu clauses, %llu to remove", (unsigned long long)nm,
                (unsigned long long)c->m, (unsigned long long)n_remove);
  }

  // new arrays, the kept clauses moved in order, then the old arrays released
  uint64_t* noff = nullptr;
  uint32_t *nlits = nullptr, *nh0 = nullptr, *nh1 = nullptr, *nstamp = nullptr, *next = nullptr;
  float* nact = nullptr;
  const uint64_t cm = nm + 1 > 1025 ? nm + 1 : 1025;
  rc = alloc(c, noff, cm);
  if (!rc) rc = alloc(c, nlits, nL);
  if (!rc) rc = alloc(c, nh0, (cm - 1) * 8);
  if (!rc) rc = alloc(c, nh1, (cm - 1) * 8);
  if (!rc) rc = alloc(c, nact, cm - 1);
  if (!rc) rc = alloc(c, nstamp, cm - 1);
  if (!rc) rc = alloc(c, next, cm - 1);
  if (!rc) {
    e = cudaMemsetAsync(noff, 0, sizeof(uint64_t), c->stream);
    if (e == cudaSuccess)
      e = launch_compact_copy(c->off, c->lits, c->head0, c->head1, c->act, c->stamp, c->ext, c->m, kmax, scratch, noff,
                              nlits, nh0, nh1, nact, nstamp, next, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) rc = fail(c, GSS_E_CUDA, "compaction: %s", cudaGetErrorString(e));
  }
  dev_free(c, scratch);
  if (rc) {  // the database is unchanged
    dev_free(c, noff);
    dev_free(c, nlits);
    dev_free(c, nh0);
    dev_free(c, nh1);
    dev_free(c, nact);
    dev_free(c, nstamp);
    dev_free(c, next);
    return rc;
  }
  dev_free(c, c->off);
  dev_free(c, c->lits);
  dev_free(c, c->head0);
  dev_free(c, c->head1);
  dev_free(c, c->act);
  dev_free(c, c->stamp);
  dev_free(c, c->ext);
  c->off = noff;
  c->lits = nlits;
  c->head0 = nh0;
  c->head1 = nh1;
  c->act = nact;
  c->stamp = nstamp;
  c->ext = next;
  c->cap_m = cm;
  c->cap_L = nL ? nL : 1;
  c->cap_head0 = c->cap_head1 = (cm - 1) * 8;
  c->cap_act = c->cap_stamp = c->cap_ext = cm - 1;
  c->m = nm;
  c->L = nL;
  c->removed += n_remove;
  if (n_removed) *n_removed = n_remove;
  return GSS_OK;
}

int gss_export_clauses(gss_ctx* c, uint64_t* offsets, uint64_t cap_clauses, uint32_t* lits, uint64_t cap_lits,
                       uint32_t* ids, uint64_t* n_clauses, uint64_t* n_lits) {
  if (!c) return GSS_E_INVAL;
  c->err.clear();
  if (n_clauses) *n_clauses = c->m;
  if (n_lits) *n_lits = c->L;
  if (cap_clauses < c->m || cap_lits < c->L)
    return fail(c, GSS_E_OVERFLOW, "%llu clauses, %llu literals to export", (unsigned long long)c->m,
                (unsigned long long)c->L);
  if (!offsets || (c->L && !lits)) return fail(c, GSS_E_INVAL, "offsets / lits is NULL");
  Guard g(c->device);
  ACK(cudaMemcpyAsync(offsets, c->off, (c->m + 1) * sizeof(uint64_t), cudaMemcpyDeviceToHost, c->stream));
  if (c->L) {
    if (c->map) {  // literals back in the caller's variable numbering
      uint32_t *tmp = nullptr, *inv = nullptr;
      int rc;
      if ((rc = alloc(c, tmp, c->L))) return rc;
      if ((rc = alloc(c, inv, c->V))) {
        dev_free(c, tmp);
        return rc;
      }
      cudaError_t e = cudaMemcpyAsync(tmp, c->lits, c->L * sizeof(uint32_t), cudaMemcpyDeviceToDevice, c->stream);
      if (e == cudaSuccess) e = launch_invert_u32(c->map, c->V, inv, c->stream);
      if (e == cudaSuccess) e = launch_translate(tmp, c->L, inv, c->stream);
      if (e == cudaSuccess) e = cudaMemcpyAsync(lits, tmp, c->L * sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
      dev_free(c, tmp);
      dev_free(c, inv);
      if (e != cudaSuccess) return fail(c, GSS_E_CUDA, "export: %s", cudaGetErrorString(e));
    } else {
      ACK(cudaMemcpyAsync(lits, c->lits, c->L * sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream));
    }
  }
  ACK(cudaStreamSynchronize(c->stream));
  if (ids) {
    uint64_t n = 0;
    const int rc = gss_get_clause_ids(c, ids, c->m, &n);
    if (rc) return rc;
  }
  return GSS_OK;
}

}  // extern "C"
