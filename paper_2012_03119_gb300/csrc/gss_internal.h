// gss_internal.h -- shared declarations of the CUDA translation units of libgss.
//
// Device data layout (all resident in HBM, owned by the context):
//   off    u64 [m + 1]           CSR offsets of the clause database (global literal index)
//   lits   u32 [L]               literals, l = 2v + s
//   head0  u32 [m][8]            literals 0..7 of each clause, padded with PAD = 2V
//   head1  u32 [m][8]            literals 8..15 of each clause, padded with PAD
//   map    u32 [V]               internal id of each variable (hottest first); stored literals
//                                and plane rows use internal ids
//   P      u32 [2V + 2][Wp]      false planes: P[l][w] bit j set iff assignment 32w + j gives
//                                literal l the value F (P[2v] = isFalse(v), P[2v+1] = isTrue(v));
//                                rows 2V, 2V + 1 are all ones (PAD is neutral under AND)
//   aggF   u32 [2V + 2][AWp]     group aggregate of P: bit g set iff P[l][g] != 0
//                                ("F is in G(l)" for the 32-assignment group g, Section 4.2)
//   aggU   u32 [V + 1][AWp]      bit g set iff some assignment of group g leaves v U (row V = 0)
//   agg2F  u32 [2V + 2]          wide sets only (AWp > 4): bit s set iff aggF[l][s] != 0, i.e. F is
//   agg2U  u32 [V + 1]           in G(l) for the 1024-assignment super-group s; agg2U likewise
// W = ceil(N / 32) words, Wp = row stride (a power of two >= max(4, W)),
// AWp = max(1, Wp / 32) (1, 2, 4, ... 32).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gss.h"

namespace gss {

constexpr uint32_t HEAD_K = GSS_HEAD_WIDTH;  // literals kept per clause outside the CSR (two planes of 8)
static_assert(HEAD_K == 16, "kernels read the head as two planes of 8 literals");

// Device-side status words, reset by the host between phases.
struct DevStatus {
  // the test's counters, first and together: one memset clears them before a test
  unsigned long long n_records;     // records produced by the last test (may exceed capacity)
  unsigned long long n_candidates;  // (clause, group) pairs that passed the aggregate test (stage A)
  unsigned long long n_super;       // wide sets: (clause, super-group) pairs that passed the level-2 test
  unsigned int bad_code;         // packing saw a value code outside {0, 1, 2}: bit (w mod 32) for plane word w
  unsigned int bad_lit;          // ingest saw a literal >= 2V
  unsigned int bad_size;         // ingest saw an empty clause or offsets beyond the batch
  unsigned int timeout;          // a bounded device wait gave up
};

// Planes of one assignment set.
struct PlaneView {
  const uint32_t* P;
  const uint32_t* aggF;
  const uint32_t* aggU;
  uint32_t Wp, AWp, N;
  uint32_t V;  // rows: P and aggF 2V + 2, aggU V + 1
  // Serving: bits of plane word w that hold real assignments (wvalid[w], w < ceil(N / 32));
  // the other rows of a word are U padding and must not report.  nullptr: every row below N.
  const uint32_t* wvalid = nullptr;
};

// Wide assignment sets (more than 4096 assignments; Section 7's aggregate of aggregates): the
// test's stage A then filters on level-2 rows of one word per literal (bit s: some assignment
// of super-group s -- 32 groups, 1024 assignments -- makes the literal F / leaves the variable
// U), and each (clause, super-group) pair left is tested on its level-1 words (one bit per
// 32-assignment group) before the exact test of each group left.
struct WideView {
  const uint32_t* aggF1 = nullptr;  // [2V + 2][AWp1] level-1 rows
  const uint32_t* aggU1 = nullptr;  // [V + 1][AWp1]
  uint32_t AWp1 = 0;
};
// agg2F[r] bit s = (aggF1[r][s] != 0) for r < 2V + 2; agg2U[v] bit s = (aggU1[v][s] != 0) for v <= V.
cudaError_t launch_agg2(const uint32_t* aggF1, const uint32_t* aggU1, uint32_t V, uint32_t AWp1, uint32_t* agg2F,
                        uint32_t* agg2U, cudaStream_t s);

// Bounds-checked build (GSS_DEBUG_BOUNDS): the test kernels check every row they gather from
// and count violations in a device counter, reading the neutral PAD row instead.
cudaError_t debug_bounds_errors(unsigned long long* out, bool reset);  // 0 when not built in

// Clause database (device pointers).
struct ClauseView {
  const uint64_t* off;
  const uint32_t* lits;
  const uint32_t* head0;
  const uint32_t* head1;
  uint32_t pad;  // PAD literal = 2V
  const uint32_t* ext = nullptr;  // caller-visible id of each resident clause (nullptr: its position)
};

// Clause activity (Section 3.6): during a test, each reported clause gets act += inc once;
// stamp[c] == epoch marks a clause already bumped by this test.  act == nullptr: off.
struct ActivityView {
  float* act = nullptr;
  uint32_t* stamp = nullptr;
  uint32_t epoch = 0;
  float inc = 0.0f;
};

// ---------------------------------------------------------------- launchers
// Pack value codes [N][pitch] (device) into P, aggF, aggU, variable v at row map[v] (identity
// when map is null).  pitch % 16 == 0 and the base 16-byte aligned (TMA).  PAD rows too.
cudaError_t launch_pack(const uint8_t* codes, uint64_t pitch, uint32_t V, uint32_t N, uint32_t Wp, uint32_t AWp,
                        const uint32_t* map, uint32_t* P, uint32_t* aggF, uint32_t* aggU, DevStatus* st,
                        cudaStream_t s);

// As launch_pack, but plane word w takes its 32 assignments from code rows
// word_rows[w] .. word_rows[w] + 31 (device array) of a code array of code_rows rows, of
// which only the rows of bits word_valid[w] are real assignments (word_valid nullable: all
// rows below N): the U padding of a word then leaves no trace in aggU.
cudaError_t launch_pack_rows(const uint8_t* codes, uint64_t pitch, uint32_t V, uint32_t N, uint32_t Wp,
                             uint32_t AWp, const uint32_t* map, const uint32_t* word_rows, uint32_t code_rows,
                             uint32_t* P, uint32_t* aggF, uint32_t* aggU, DevStatus* st, cudaStream_t s,
                             const uint32_t* word_valid = nullptr);

// Ingest, in order: validate a batch (offsets -> db offsets at off_db[n0 + 1 ..], literal range);
// on the first batch rank the variables hot-first (map[v] = internal id; scratch holds
// rank_scratch_words(V) words); translate the batch literals through map; build head planes.
uint64_t rank_scratch_words(uint32_t V);
cudaError_t launch_validate(const uint64_t* boff, uint64_t n, uint64_t L, uint64_t L0, uint64_t* off_db_at_n0,
                            const uint32_t* lits_batch, uint32_t V, DevStatus* st, cudaStream_t s);
cudaError_t launch_rank_vars(const uint32_t* lits, uint64_t L, uint32_t V, uint32_t* scratch, uint32_t* map,
                             cudaStream_t s);
cudaError_t launch_translate(uint32_t* lits, uint64_t L, const uint32_t* map, cudaStream_t s);
cudaError_t launch_build_heads(const uint64_t* boff, uint64_t n, uint64_t L0, uint32_t* head0_at_n0,
                               uint32_t* head1_at_n0, const uint32_t* lits_db, uint32_t V, cudaStream_t s);

// Test clauses [c_lo, c_hi) against the planes; append records.  With wm (device, n_wm
// entries, non-decreasing), clause c is tested against plane word w only if c < wm[w].
// cpw: tile shape, 32 clauses per warp tile (one lane each) or 16 (two lanes each: head0 and
// head1 of a clause in parallel); the wide build always takes 32.
cudaError_t launch_test(int mode, const ClauseView& db, uint64_t c_lo, uint64_t c_hi, const PlaneView& pv,
                        gss_report* rec, uint64_t cap, DevStatus* st, int grid, cudaStream_t s,
                        const uint64_t* wm = nullptr, uint32_t n_wm = 0, const ActivityView& av = ActivityView{},
                        const WideView& wide = WideView{}, int cpw = 32);

// Copy min(st->n_records, cap_dev, cap_out) records to out (device memory, or host memory the
// GPU can write), on stream s after the test that made them.
cudaError_t launch_copy_records(const gss_report* rec, const DevStatus* st, uint64_t cap_dev, uint64_t cap_out,
                                gss_report* out, int grid, cudaStream_t s);

// Group a serving launch's records by plane word (request) into out: records of word w at
// [sum of count[0..w), + count[w]), their mask ANDed with nmask[w], records left without a bit
// dropped, word set to 0.  count / cursor: 32 device counters each (zeroed here); out holds
// min(st->n_records, cap) records and may be mapped host memory.
cudaError_t launch_route(const gss_report* rec, const DevStatus* st, uint64_t cap, const uint32_t* nmask, uint32_t k,
                         unsigned long long* count, unsigned long long* cursor, gss_report* out, int grid,
                         cudaStream_t s);

// ---------------------------------------------------------------- clause activity and deletion (k_reduce.cu)
cudaError_t launch_fill_u32(uint32_t* p, uint64_t n, uint32_t value, cudaStream_t s);
cudaError_t launch_fill_f32(float* p, uint64_t n, float value, cudaStream_t s);
cudaError_t launch_iota_u32(uint32_t* p, uint64_t n, uint32_t first, cudaStream_t s);
cudaError_t launch_scale_f32(float* p, uint64_t n, float factor, cudaStream_t s);
// inv[map[i]] = i for i < n (map a permutation of [0, n)).
cudaError_t launch_invert_u32(const uint32_t* map, uint32_t n, uint32_t* inv, cudaStream_t s);
// Histogram of the 8 key bits at `shift` over the clauses longer than two literals whose key
// agrees with `prefix` above shift + 8; key = (bits of act) << 32 | id.  hist: 256 counters (zeroed here).
cudaError_t launch_key_hist(const uint64_t* off, const float* act, const uint32_t* ids, uint64_t m, uint32_t shift,
                            uint64_t prefix, uint32_t* hist, cudaStream_t s);
// Compact the database: clause c is kept iff it has at most two literals or its key > kmax.
// The plan scans keep flags and kept sizes into scratch (compact_scratch_bytes(m)) and writes
// the kept clauses and literals to d_counts[0..1]; the copy then moves the kept clauses, in
// order, into the n* arrays sized for them (noff[0] is left to the caller).
uint64_t compact_scratch_bytes(uint64_t m);
cudaError_t launch_compact_plan(const uint64_t* off, const float* act, const uint32_t* ids, uint64_t m, uint64_t kmax,
                                void* scratch, unsigned long long* d_counts, cudaStream_t s);
cudaError_t launch_compact_copy(const uint64_t* off, const uint32_t* lits, const uint32_t* head0,
                                const uint32_t* head1, const float* act, const uint32_t* stamp, const uint32_t* ids,
                                uint64_t m, uint64_t kmax, const void* scratch, uint64_t* noff, uint32_t* nlits,
                                uint32_t* nhead0, uint32_t* nhead1, float* nact, uint32_t* nstamp, uint32_t* nids,
                                cudaStream_t s);

// Occupancy-derived persistent grid for launch_test on this device.
int test_grid_size(int mode, uint32_t AWp, int n_sms, bool wide = false, int cpw = 32);
// Default tile shape for a database of m clauses and L literals (see k_test.cu).
int test_tile_shape(uint64_t m, uint64_t L);

// One instance of a batch as the batched test kernel sees it.
struct BatchInst {
  ClauseView db;
  PlaneView pv;
  uint64_t m;      // clauses
  uint64_t tile0;  // index of the instance's first tile among all the batch's tiles (of the launch's shape)
  gss_report* rec;
  uint64_t cap;
  DevStatus* st;   // the instance's test status (records, bad codes)
};

// Zero the work counter, the batch status and each instance's test status.
cudaError_t launch_batch_reset(const BatchInst* d_inst, uint32_t n_inst, unsigned long long* work, DevStatus* bst,
                               cudaStream_t s);
// Test every instance (all with the same AWp) in one persistent launch; warps take `grab`
// tiles at a time from the device counter *work (zeroed by launch_batch_reset).
cudaError_t launch_test_batch(int mode, uint32_t AWp, int cpw, const BatchInst* d_inst, uint32_t n_inst,
                              uint64_t n_tiles, unsigned long long* work, uint32_t grab, DevStatus* bst, int grid,
                              cudaStream_t s);
int test_batch_grid_size(int mode, uint32_t AWp, int cpw, int n_sms);

}  // namespace gss
