// gss_ctx.h -- the context behind the C ABI, shared by the single-instance (gss_abi.cu)
// and batch (gss_batch.cu) host code.  Not part of the public interface.
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <string>
#include <unordered_map>

#include "gss_internal.h"

using gss::DevStatus;

struct gss_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  uint32_t V = 0, max_N = 0, mode = GSS_MODE_ALLF, layout = GSS_LAYOUT_FREQUENCY;
  uint64_t budget = 0, bytes = 0;
  int n_sms = 1;
  std::unordered_map<void*, uint64_t> allocs;

  // clause database
  uint64_t m = 0, L = 0, cap_m = 0, cap_head0 = 0, cap_head1 = 0, cap_L = 0, cap_boff = 0;
  uint64_t* off = nullptr;
  uint32_t* lits = nullptr;
  uint32_t* head0 = nullptr;
  uint32_t* head1 = nullptr;
  uint64_t* boff = nullptr;
  uint32_t* map = nullptr;  // internal variable ids (frequency layout), fixed by the first batch
  uint64_t next_id = 0;     // id of the next clause added; ids are never reused
  uint32_t* ext = nullptr;  // id of each resident clause, once a reduction has removed some (else: position)
  uint64_t cap_ext = 0, removed = 0;

  // clause activity (Section 3.6), off until gss_set_activity
  float* act = nullptr;
  uint32_t* stamp = nullptr;  // test epoch that last bumped the clause
  uint64_t cap_act = 0, cap_stamp = 0;
  float decay = 1.0f, inv_decay = 1.0f, inc = 1.0f;
  uint32_t epoch = 0;

  // assignment sets.  pipeline 1: one plane set, packed and tested on `stream`.  pipeline 2:
  // two plane sets; gss_set_assignments packs into the set the last test did not read, on
  // pack_stream, so that packing the next set overlaps the test of the last one, and copies
  // host values into that set's own staging buffer on copy_stream, so that the next set's
  // copy need not wait for the last set's packing.
  struct PlaneSet {
    uint32_t* P = nullptr;
    uint32_t* aggF = nullptr;
    uint32_t* aggU = nullptr;
    uint32_t* agg2F = nullptr;  // level-2 rows, held when max_N > GSS_MAX_NARROW_ASSIGNMENTS
    uint32_t* agg2U = nullptr;
    uint32_t N = 0;
    uint8_t* codes = nullptr;   // staging buffer for values the packing cannot read in place
    uint64_t codes_rows = 0;
  };
  uint32_t pipeline = 1;
  uint32_t tile_clauses = 0;  // test tile shape (32 or 16); 0: from the mean clause length
  PlaneSet sets[2];
  uint32_t cur = 0;          // plane set of the latest assignment set (the next test reads it)
  uint32_t tested_set = 0;   // plane set the last test read
  uint32_t tested_N = 0;
  cudaStream_t pack_stream = nullptr;  // == stream for pipeline 1
  bool own_pack_stream = false;
  cudaEvent_t ev_packed[2] = {nullptr, nullptr};  // pipeline 2: packing of set b done
  cudaEvent_t ev_tested[2] = {nullptr, nullptr};  // pipeline 2: the last test that read set b done
  cudaEvent_t ev_copied = nullptr;  // host codes landed in the staging buffer
  cudaStream_t copy_stream = nullptr;             // pipeline 2: copies into the staging buffers
  cudaEvent_t ev_staged[2] = {nullptr, nullptr};  // pipeline 2: the copy into set b's staging buffer done
  uint32_t N = 0, Wp = 4, AWp = 1;  // of the latest assignment set
  bool have_assign = false;
  uint64_t Vp = 0;
  uint32_t* P = nullptr;      // the latest set's planes (aliases of sets[cur])
  uint32_t* aggF = nullptr;
  uint32_t* aggU = nullptr;
  uint32_t* agg2F = nullptr;
  uint32_t* agg2U = nullptr;
  const uint8_t* pack_src = nullptr;  // codes the next packing reads (staging buffer or caller memory)
  uint64_t pack_pitch = 0;
  uint32_t pack_set = 0;               // plane set the staged codes are packed into

  // reports
  gss_report* rec = nullptr;
  uint64_t rec_cap = 0;
  DevStatus* st = nullptr;    // [0]: pack + test of plane set 0, [1]: ingest, [2]: pack + test of plane set 1
  DevStatus* h_st = nullptr;  // pinned mirror
  bool tested = false;
  bool fetch_pending = false;  // a gss_fetch_reports_async not yet waited for
  uint64_t fetch_cap = 0;
  int grid[2][5][2] = {};     // cached persistent grid per (mode, AWp <= 4, tile shape 32 / 16)
  int grid_wide[2] = {0, 0};  // per mode, for sets of more than GSS_MAX_NARROW_ASSIGNMENTS

  uint64_t tests_run = 0, pair_tests = 0;
  uint64_t records = 0, overflows = 0;  // of tests whose status was read
  bool counted = false;                 // the last test's records are in `records`
  std::string err;
};

namespace gss {
namespace host {

// A named NVTX range around an entry point, for timeline tools; free when no tool listens.
struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

int fail(gss_ctx* c, int code, const char* fmt, ...);
int dev_alloc(gss_ctx* c, void** p, uint64_t bytes);
void dev_free(gss_ctx* c, void* p);
int sync_status(gss_ctx* c);
// Status words of plane set b (pack and test), and their index in h_st.
inline uint32_t set_status_index(uint32_t b) { return b ? 2u : 0u; }
inline DevStatus* set_status(gss_ctx* c, uint32_t b) { return c->st + set_status_index(b); }
uint32_t words_stride(uint32_t N);
uint32_t agg_stride(uint32_t Wp);
// Copy / register an assignment set without packing it (the batch packs inside its graph).
// wait_copy: return only once host values have been read (else gss_copy_wait does).
int stage_assignments(gss_ctx* c, const uint8_t* src, uint64_t pitch, uint32_t n, bool device_src,
                      bool wait_copy = true);
// Pack the staged assignment set on stream s.
int pack_staged(gss_ctx* c, cudaStream_t s);
// Reserve database capacity for max_clauses clauses and max_lits literals, so that later
// gss_add_clauses calls within it never move the arrays.
int reserve_db(gss_ctx* c, uint64_t max_clauses, uint64_t max_lits);
// Reserve the per-clause activity, bump-stamp and id arrays (those that exist) likewise.
int reserve_clause_arrays(gss_ctx* c, uint64_t max_clauses);
// Wait for the last test of c and read its record count (status already synchronised when sync = false).
int wait_test(gss_ctx* c, uint64_t* n, bool sync);

}  // namespace host
}  // namespace gss
