/*
 * gss.h -- C ABI of the GB300 clause x assignment test library (libgss.so).
 *
 * The library tests a resident database of clauses against a set of
 * three-valued assignments at once and reports every (clause, assignment) pair
 * in which every literal of the clause is F under the assignment -- the pairs
 * where the clause "would have been in conflict" (Section 3.3), i.e. the
 * allFalse output of Listing assignmentTrigger (Section 3.4), evaluated over
 * many clauses in parallel and 32 assignments per machine word (Section 3.5).
 * GSS_MODE_TRIGGER switches the test to Definition "triggers" (Section 3.3):
 * no literal T and at least s - 1 of the s literals F.
 *
 * Notation.  V variables 0..V-1; literal l = 2v + s, s = 1 meaning "not v";
 * value codes 0 = U, 1 = T, 2 = F (Section 3.1: truth values {T, F, U},
 * not T = F, not F = T, not U = U, A(not v) = not A(v)).  N assignments per
 * set; assignment a lives in 32-bit word a / 32, bit a % 32.
 *
 * Conventions.
 *   - Every call returns an int status (GSS_OK or a negative GSS_E_* code);
 *     no C++ exception crosses the ABI.  gss_last_error() gives the message.
 *   - Host pointers stay owned by the caller and may be released as soon as
 *     the call returns.  Device pointers passed in stay owned by the caller
 *     and must stay valid until the work that reads them has completed on the
 *     context's stream.  All device memory the library allocates is owned by
 *     the context and released by gss_destroy().
 *   - Device work is queued on the context's stream (gss_config.stream, or a
 *     stream the context creates).  Calls that return results to the host
 *     (gss_fetch_reports, gss_report_count) synchronise that stream.
 *   - One context must not be used by two host threads at the same time.
 *   - Clause ids are dense and assigned in insertion order starting at 0.
 */
#ifndef GSS_H
#define GSS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ codes */
enum {
  GSS_OK = 0,
  GSS_E_INVAL = -1,     /* bad argument, literal >= 2V, empty clause, value code > 2 */
  GSS_E_NOMEM = -2,     /* device allocation failed or the memory budget is exhausted */
  GSS_E_CUDA = -3,      /* a CUDA runtime call failed (message in gss_last_error) */
  GSS_E_OVERFLOW = -4,  /* more report records than the buffer given (count still returned) */
  GSS_E_TIMEOUT = -5,   /* a bounded wait gave up (device side, or gss_server_wait) */
  GSS_E_BUSY = -6,      /* no free slot (serving admission) */
  GSS_E_STATE = -7      /* call out of order (e.g. gss_test before gss_set_assignments) */
};

enum { GSS_MODE_ALLF = 0, GSS_MODE_TRIGGER = 1 };

/*
 * Internal variable numbering.  GSS_LAYOUT_FREQUENCY (default): the first
 * gss_add_clauses batch fixes an internal numbering, most frequent variables
 * first, so the hottest literals' assignment rows sit together in memory (the
 * locality Section 7 proposes to exploit).  GSS_LAYOUT_IDENTITY keeps the
 * caller's numbering.  Reports are per clause id and identical either way.
 */
enum { GSS_LAYOUT_IDENTITY = 0, GSS_LAYOUT_FREQUENCY = 1 };

/*
 * Largest N per assignment set.  Sets of more than GSS_MAX_NARROW_ASSIGNMENTS are tested
 * with a second aggregate level (Section 7's aggregate of aggregates): one bit per
 * 1024-assignment super-group per literal filters (clause, super-group) pairs before the
 * 32-assignment groups of Section 4.2 do; results are the same.  Batches
 * (gss_batch_*) and gss_test_noalloc take at most GSS_MAX_NARROW_ASSIGNMENTS.
 */
#define GSS_MAX_ASSIGNMENTS 32768u
#define GSS_MAX_NARROW_ASSIGNMENTS 4096u
#define GSS_HEAD_WIDTH 16u        /* literals per clause kept in the head planes */

typedef struct gss_ctx gss_ctx;

/* Context configuration; gss_config_init() fills the defaults. */
typedef struct {
  int device;                /* CUDA device ordinal (default 0) */
  void* stream;              /* cudaStream_t to queue work on; NULL: the context creates one */
  uint64_t report_capacity;  /* report records the device buffer holds (default 1 << 22) */
  uint32_t max_assignments;  /* upper bound on N, <= GSS_MAX_ASSIGNMENTS (default 1024) */
  uint32_t mode;             /* GSS_MODE_ALLF (default) or GSS_MODE_TRIGGER */
  uint64_t mem_budget_bytes; /* cap on device bytes the context may hold; 0 = no cap */
  uint32_t layout;           /* GSS_LAYOUT_FREQUENCY (default) or GSS_LAYOUT_IDENTITY */
  uint32_t pipeline;         /* 1 (default) or 2: see below */
  void* pack_stream;         /* pipeline 2: cudaStream_t the packing runs on; NULL: the context creates one */
  uint32_t clauses_per_tile; /* test tile shape: 32 (a lane per clause), 16 (two lanes per clause: its
                                first 8 and next 8 literals in parallel), or 0 (default: 32, which
                                measured faster on GB300 for short and long clauses alike) */
} gss_config;

/*
 * pipeline = 2 keeps two plane sets.  gss_set_assignments / _device pack the new set on
 * pack_stream into the plane set the last gss_test does not read, while that test may still
 * run on `stream`; gss_test waits (on the device) for its set's packing.  So a caller that
 * issues gss_set_assignments for set k + 1 before it reads the results of set k lets the
 * next set's host copy and packing proceed while the last test runs.  (On GB300 the packing
 * and test kernels each fill the GPU: running them side by side was measured slower than
 * running them in turn, so the gain is in hiding host copies and host round trips.)
 * Host values are copied into a staging buffer of the plane set they go to, on a copy
 * stream of the context's own, so that a set's copy does not wait for the last set's
 * packing: the host link can stay busy from one set to the next.
 * Results are the same as with pipeline = 1.  Ordering: packing is not ordered after work
 * queued on `stream`; device codes written by other work must be complete before the
 * call (or ordered onto pack_stream by the caller).  Twice the plane memory is held, and
 * twice the staging memory once host values have gone to both sets.
 */

/*
 * One report record: clause `clause_id` passes the test on assignment
 * 32 * word + j for every bit j set in `mask` (never 0).  This is the
 * report(i, mask) record of Listing multiTrigger (Section 4.3) with i the
 * 32-assignment word.  Record order is unspecified.
 */
typedef struct {
  uint32_t clause_id;
  uint32_t word;
  uint32_t mask;
} gss_report;

/* Context statistics (host-side counters, no synchronisation). */
typedef struct {
  uint32_t n_vars;
  uint32_t n_assign;        /* N of the current assignment set (0 if none) */
  uint64_t n_clauses;
  uint64_t n_lits;
  uint64_t device_bytes;    /* device memory held by the context */
  uint64_t report_capacity;
  uint64_t tests_run;       /* gss_test calls completed */
  uint64_t pair_tests;      /* sum over gss_test calls of n_clauses * N */
  uint64_t candidate_pairs; /* last test: (clause, 32-assignment group) pairs whose aggregate test
                               (Section 4.2) was positive; valid after gss_report_count / fetch */
  uint64_t group_pairs;     /* last test: n_clauses * ceil(N / 32), all (clause, group) pairs */
  uint64_t clauses_removed; /* by gss_reduce_db, in total */
  uint64_t next_clause_id;  /* id the next added clause gets (ids are never reused) */
  uint64_t records;         /* records produced by the tests whose results were read, in total */
  uint64_t overflows;       /* of those tests, how many produced more records than the capacity */
  uint64_t super_pairs;     /* last test, sets of more than GSS_MAX_NARROW_ASSIGNMENTS only:
                               (clause, 1024-assignment super-group) pairs whose level-2 aggregate
                               test was positive; 0 otherwise */
} gss_stats;

/* ------------------------------------------------------------ lifecycle */

/* Fill *cfg with the defaults listed in gss_config.  Returns GSS_E_INVAL if cfg is NULL. */
int gss_config_init(gss_config* cfg);

/*
 * Create a context for V = n_vars variables (1 <= V < 2^31) on cfg->device:
 * the GPU-side clause store of Section 3.6 (the GPU keeps every clause the
 * solver threads export to it) with room for one assignment set of up to
 * cfg->max_assignments assignments (Section 3.4's bit-packed assignments).
 * cfg may be NULL (defaults).  On success *out owns the device state.
 * Errors: GSS_E_INVAL (bad V, bad config), GSS_E_CUDA (no device / bad
 * stream), GSS_E_NOMEM.
 */
int gss_create(gss_ctx** out, uint32_t n_vars, const gss_config* cfg);

/*
 * Release every device and host resource of ctx (the clause store and
 * assignment planes of Sections 3.4 and 3.6); waits for its queued work.
 * NULL is a no-op.
 */
int gss_destroy(gss_ctx* ctx);

/* ------------------------------------------------------------- clauses */

/*
 * Append n_clauses clauses to the resident database (Section 3.6: every
 * learned clause is exported to the GPU, which keeps all of them).
 *   offsets  host, n_clauses + 1 entries, offsets[0] = 0, strictly
 *            increasing: clause i is lits[offsets[i] .. offsets[i+1]).
 *   lits     host, offsets[n_clauses] literals, each l = 2v + s < 2V.
 *   first_id out (nullable): id of the first new clause; the others follow.
 * All or nothing: on GSS_E_INVAL (empty clause, literal >= 2V, offsets[0]
 * != 0) or GSS_E_NOMEM the database is unchanged.  Synchronises the stream
 * (validation result).  Duplicate literals are allowed; a clause holding
 * l and not l is accepted and is never reported.  With GSS_LAYOUT_FREQUENCY the
 * first batch fixes the internal variable numbering; an assignment set given
 * before it is packed again from the same codes (so device codes passed to
 * gss_set_assignments_device before the first batch must still be valid).
 */
int gss_add_clauses(gss_ctx* ctx, const uint64_t* offsets, uint64_t n_clauses, const uint32_t* lits,
                    uint32_t* first_id);

/* --------------------------------------------------------- assignments */

/*
 * Replace the assignment set by N = n_assign assignments (Section 3.4: each
 * variable's values over the N assignments are packed into bit-words; here
 * one false-plane row per literal, bit a set iff A_a(l) = F, plus one
 * aggregate word per literal and 32-assignment group, Section 4.2).
 *   values host, row-major [n_assign][n_vars] bytes, 0 = U, 1 = T, 2 = F.
 * 0 <= n_assign <= cfg.max_assignments.  Assignments 32g .. 32g+31 form
 * group g; grouping assignments of one solver thread together (Section 4.3)
 * makes the group prefilter effective but never changes results.  Above
 * GSS_MAX_NARROW_ASSIGNMENTS, assignments 1024s .. 1024s+1023 also form
 * super-group s, with one more aggregate word per literal (Section 7); the
 * records are the same.
 * Queued on the stream (the host buffer is copied before return).  A value
 * code above 2 is detected on the device and reported as GSS_E_INVAL by the
 * next gss_fetch_reports / gss_report_count, with no records.
 */
int gss_set_assignments(gss_ctx* ctx, const uint8_t* values, uint32_t n_assign);

/*
 * As gss_set_assignments (the same packing, Section 3.4, and aggregates, Section 4.2, of
 * the same arguments), but returns as soon as the copy is queued: `values` (host memory;
 * pinned memory lets the copy run while the caller goes on) must stay unchanged until
 * gss_copy_wait returns.  With two plane sets (gss_config.pipeline = 2) the copy of set k + 1
 * then queues behind the copy of set k, so that the host link stays busy while the caller
 * tests set k and reads its records.  gss_copy_wait waits until every host copy queued so far
 * has read the caller's memory.  Errors as gss_set_assignments.
 */
int gss_set_assignments_async(gss_ctx* ctx, const uint8_t* values, uint32_t n_assign);
int gss_copy_wait(gss_ctx* ctx);

/*
 * As gss_set_assignments, but `d_values` is a DEVICE pointer on the
 * context's device, rows `pitch` bytes apart (pitch >= n_vars), the buffer
 * spanning n_assign * pitch bytes.  Bytes past n_vars in a row are ignored.
 * When pitch and the pointer are multiples of 16 the codes are packed in
 * place; otherwise they are first copied (device to device) into a context
 * buffer.  The buffer must stay valid until the queued work has run.
 */
int gss_set_assignments_device(gss_ctx* ctx, const uint8_t* d_values, uint64_t pitch, uint32_t n_assign);

/* ---------------------------------------------------------------- test */

/*
 * Test every resident clause against the current assignment set (Section
 * 3.5: clauses in parallel, 32 assignments per word) and write report records
 * to the context's device buffer, replacing those of the previous test.
 * Queued on the stream; returns at once.  Errors: GSS_E_STATE (no assignment
 * set), GSS_E_CUDA.
 */
int gss_test(gss_ctx* ctx);

/*
 * Wait for the last gss_test and copy its records to host buffer `out`: the
 * report(i, mask) calls of Listing multiTrigger (Section 4.3), by which the
 * GPU tells each solver thread which clauses triggered on its assignments
 * (Section 3.6).  `out` has capacity `cap` records (out may be NULL when cap
 * is 0).  *n_out receives
 * the total number of records the test produced.  Returns GSS_E_OVERFLOW if
 * that number exceeds cap (min(cap, n) records written) or the device buffer
 * (the test must then be re-run after gss_set_report_capacity), GSS_E_INVAL
 * if the assignment set held a bad value code, GSS_E_STATE if no test ran.
 */
int gss_fetch_reports(gss_ctx* ctx, gss_report* out, uint64_t cap, uint64_t* n_out);

/*
 * The same copy without waiting: queue, on the context's stream after the last gss_test, a
 * kernel that writes min(records, cap) records straight into `out`, and return at once.
 * `out` must be memory the GPU can write: pinned host memory (cudaMallocHost /
 * cudaHostAlloc / cudaHostRegister), device or managed memory, or pageable host memory on a
 * device that can access it (GSS_E_INVAL otherwise); it must stay valid until
 * gss_fetch_wait returns.  gss_fetch_wait synchronises the stream and returns as
 * gss_fetch_reports would (*n_out: all the test's records; GSS_E_OVERFLOW, GSS_E_INVAL,
 * GSS_E_TIMEOUT likewise).  A caller that sets the next assignment set between the two calls
 * (two plane sets, gss_config.pipeline = 2) moves the records back while the next set's
 * codes come in.  GSS_E_STATE: no test to fetch / nothing to wait for.
 */
int gss_fetch_reports_async(gss_ctx* ctx, gss_report* out, uint64_t cap);
int gss_fetch_wait(gss_ctx* ctx, uint64_t* n_out);

/*
 * As gss_fetch_reports but copies nothing: waits for the last test and
 * returns its record count.  The records stay in device memory, readable
 * through gss_reports_device().
 */
int gss_report_count(gss_ctx* ctx, uint64_t* n_out);

/* Device address of the context's report buffer (valid until the next capacity change or gss_destroy). */
int gss_reports_device(gss_ctx* ctx, const gss_report** d_records, uint64_t* capacity);

/* Resize the device report buffer to `cap` records (discards current records). */
int gss_set_report_capacity(gss_ctx* ctx, uint64_t cap);

/* Select GSS_MODE_ALLF or GSS_MODE_TRIGGER for the following gss_test calls. */
int gss_set_mode(gss_ctx* ctx, uint32_t mode);

/* ------------------------------------------------------------- batches */

/*
 * A batch: many independent clause databases ("instances"), each with its own
 * variables, assignment set and report buffer -- e.g. the databases of several
 * solver portfolios sharing one GPU.  Every instance is tested exactly as a
 * context would test it (same definitions, same records); gss_batch_test runs
 * all of them as one CUDA graph: per-instance packing on parallel branches,
 * then one persistent launch in which warps steal 32-clause tiles of any
 * instance from a device counter.  The graph is captured on the first test
 * and again whenever an instance is added, the mode changes, or an instance's
 * assignment set changes size or source buffer.  The launch shape (tile shape:
 * clauses per warp tile; tiles per steal; grid) is chosen on the first test by
 * timing candidates on the batch.
 * Instances sharing a batch use the batch's device, stream, mode and layout.
 */
typedef struct gss_batch gss_batch;

typedef struct {
  uint32_t n_instances;
  uint32_t n_groups;           /* test launches per run: one per aggregate row width */
  uint32_t tiles_per_steal[3]; /* autotuned, per group */
  uint32_t grid[3];            /* autotuned CTAs, per group */
  uint64_t n_tiles[3];         /* tiles (of the tuned shape) per group */
  uint64_t runs;               /* gss_batch_test calls */
  float tuned_test_us;         /* test-launch time measured by the autotuner (0 when the choices came
                                  from the cache file named by the environment variable
                                  GSS_AUTOTUNE_CACHE, which keeps them across processes) */
  uint32_t clauses_per_tile[3];/* autotuned tile shape, per group: 32 (a lane per clause) or 16 (two
                                  lanes per clause, head0 and head1 tested in parallel) */
} gss_batch_info;

/* Create an empty batch (cfg: device, stream, mode, layout; the rest is per instance). */
int gss_batch_create(gss_batch** out, const gss_config* cfg);

/* Release the batch and every instance. */
int gss_batch_destroy(gss_batch* b);

/*
 * Add an instance of n_vars variables holding the given clauses (as
 * gss_add_clauses), able to take up to max_assignments assignments and to hold
 * report_capacity records (0: the defaults of gss_config_init).  *instance_id
 * receives its index (dense, from 0).  max_assignments <= GSS_MAX_NARROW_ASSIGNMENTS
 * (GSS_E_INVAL otherwise).  Synchronises the stream.
 */
int gss_batch_add_instance(gss_batch* b, uint32_t n_vars, uint32_t max_assignments, uint64_t report_capacity,
                           const uint64_t* offsets, uint64_t n_clauses, const uint32_t* lits,
                           uint32_t* instance_id);

/* Stage an instance's assignment set (host codes, as gss_set_assignments); packed by gss_batch_test. */
int gss_batch_set_assignments(gss_batch* b, uint32_t instance, const uint8_t* values, uint32_t n_assign);

/* As above with device codes (as gss_set_assignments_device); the buffer must stay valid and
 * unchanged in place until the tests that read it have run. */
int gss_batch_set_assignments_device(gss_batch* b, uint32_t instance, const uint8_t* d_values, uint64_t pitch,
                                     uint32_t n_assign);

/* Pack and test every instance (queued on the stream).  Every instance needs an assignment
 * set.  Errors: GSS_E_STATE, GSS_E_CUDA. */
int gss_batch_test(gss_batch* b);

/* Per-instance results of the last gss_batch_test, as gss_report_count / gss_fetch_reports. */
int gss_batch_report_count(gss_batch* b, uint32_t instance, uint64_t* n_out);
int gss_batch_fetch_reports(gss_batch* b, uint32_t instance, gss_report* out, uint64_t cap, uint64_t* n_out);

/* The batch's launch groups and the autotuner's choices (GSS_E_INVAL for NULL arguments). */
int gss_batch_get_info(const gss_batch* b, gss_batch_info* out);
const char* gss_batch_last_error(const gss_batch* b);

/* ------------------------------------------- clause activity and deletion */

/*
 * Section 3.6: the GPU deletes clauses by activity, as MiniSat does on the CPU, and a
 * clause's activity is bumped whenever it triggers.  The paper gives no constants; this
 * library follows MiniSat:
 *   - activities are single-precision floats; a clause starts at the current increment inc
 *     (clauses already resident when activity is switched on start at inc = 1);
 *   - each gss_test bumps every clause it reports (for any assignment) once: act += inc;
 *   - after each gss_test, inc *= (1 / decay); once inc exceeds 1e20 all activities and inc
 *     are multiplied by 1e-20.
 * A test whose assignment set holds an invalid code bumps nothing.
 */

/* Switch activity on (0 < decay <= 1), or change the decay of an active context. */
int gss_set_activity(gss_ctx* ctx, float decay);

/* Activities of the resident clauses in clause order (as gss_get_clause_ids); *n_out = the
 * number of resident clauses.  GSS_E_STATE if activity is off; GSS_E_OVERFLOW if cap is
 * smaller (the first cap are written). */
int gss_get_activity(gss_ctx* ctx, float* out, uint64_t cap, uint64_t* n_out);

/* Ids of the resident clauses, increasing (ids are assigned by gss_add_clauses and never
 * reused).  Errors as gss_get_activity. */
int gss_get_clause_ids(gss_ctx* ctx, uint32_t* out, uint64_t cap, uint64_t* n_out);

/*
 * Remove floor(remove_fraction * n) of the n resident clauses longer than two literals:
 * those with the smallest activity, ties broken by the smaller id (MiniSat removes the half
 * of its learnt clauses with the lowest activity and keeps binary clauses).  Kept clauses keep
 * their ids, activities and order; records of later tests carry the ids.  *n_removed
 * (nullable) receives the count.  Needs activity on (GSS_E_STATE); GSS_E_NOMEM if the
 * compacted copy does not fit (the database is then unchanged).  Records of an earlier test
 * stay valid.
 */
int gss_reduce_db(gss_ctx* ctx, double remove_fraction, uint64_t* n_removed);

/*
 * Copy the resident clauses out, in the caller's variable numbering: offsets[0..n] (CSR,
 * offsets[0] = 0), lits[0..L) and, if ids is not NULL, their ids[0..n), in the order of
 * gss_get_clause_ids.  *n_clauses / *n_lits (nullable) receive n and L; with cap_clauses < n
 * or cap_lits < L nothing is copied and GSS_E_OVERFLOW is returned.  Feeding the export to
 * gss_add_clauses of a new context rebuilds the database (new ids count from 0).
 */
int gss_export_clauses(gss_ctx* ctx, uint64_t* offsets, uint64_t cap_clauses, uint32_t* lits, uint64_t cap_lits,
                       uint32_t* ids, uint64_t* n_clauses, uint64_t* n_lits);

/* ------------------------------------------------- without allocation */

/*
 * Size of the fixed device array gss_test_noalloc works in (32 MiB).  The paper has no
 * counterpart to this entry point; it exists for callers that cannot allocate.
 */
#define GSS_NOALLOC_SCRATCH_BYTES (32ull << 20)

/*
 * The whole test -- validation, clause heads, packing, testing, record compaction --
 * for callers that must not allocate device memory while they run it: a program whose
 * GPU memory belongs to another runtime's pool, or a loop that cannot afford the device
 * synchronisation a cudaMalloc may cause.  The caller provides every input and output
 * in device memory on the current device; the function allocates nothing (no cudaMalloc,
 * no library allocator).  Its working memory is one array of GSS_NOALLOC_SCRATCH_BYTES
 * compiled into the library, which every GPU that loads the library holds until the
 * process exits.
 *   d_offsets, n_clauses, d_lits  the clauses, as gss_add_clauses but in device memory
 *   n_vars                        V (literals 2v + s < 2V)
 *   d_values, pitch, n_assign     value codes as gss_set_assignments_device; here the
 *                                 pointer and pitch must be multiples of 16 and
 *                                 n_assign <= GSS_MAX_NARROW_ASSIGNMENTS
 *   mode                          GSS_MODE_ALLF or GSS_MODE_TRIGGER
 *   d_out, cap                    record buffer (gss_report, record order unspecified)
 *   d_count                       device counter that receives the number of records
 *   stream                        cudaStream_t to work on (NULL: the legacy default stream)
 *   errbuf, errbuf_len            optional host buffer for a message (nullable)
 * Results equal those of gss_add_clauses + gss_set_assignments_device + gss_test on a
 * context (the caller's variable numbering is kept).  The call returns when the results
 * are in d_out / d_count (it synchronises the stream).  Problems whose working memory
 * (about 72 bytes per clause plus 8 (Wp + 1.5 AWp) bytes per variable, Wp = N/32 rounded up to a power of
 * two >= 4) exceeds GSS_NOALLOC_SCRATCH_BYTES are rejected with GSS_E_INVAL and a
 * message; larger problems go through a context.  Errors otherwise as gss_add_clauses,
 * gss_test and gss_fetch_reports (GSS_E_OVERFLOW: *d_count holds the full count).
 * Every call on a device reuses the same array and leaves its contents behind, so calls
 * that may overlap on the GPU (other streams, other host threads) must not be issued:
 * they would race on it.  The first call on a device looks up the array's device address
 * (with that device current); make that first call before any stream capture.  A call in
 * a new context of the device (after cudaDeviceReset) looks the address up again, so make
 * the first call after a reset before any stream capture as well.
 */
int gss_test_noalloc(const uint64_t* d_offsets, uint64_t n_clauses, const uint32_t* d_lits, uint32_t n_vars,
                     const uint8_t* d_values, uint64_t pitch, uint32_t n_assign, uint32_t mode, gss_report* d_out,
                     uint64_t cap, unsigned long long* d_count, void* stream, char* errbuf, size_t errbuf_len);

/* ------------------------------------------------------------- serving */

/*
 * A server keeps one clause database resident on the device while solver threads stream
 * in learned clauses and submit assignment snapshots (Section 3.6: each CPU thread sends
 * the parent assignment of its conflicts and every clause it learns; the GPU tests all of
 * its clauses against the assignments not yet tested and reports the hits to the thread
 * that sent the assignment; assignments are not sent when the GPU is full).
 *
 * A request is a snapshot of 1 to 32 assignments (one plane word).  It is admitted into
 * one of a fixed number of device slots; when none frees up within the caller's wait the
 * submission is refused with GSS_E_BUSY (memory admission).  Admitted requests that are
 * not yet on the GPU join the next launch: a scheduler thread keeps up to `lanes` launches
 * in flight, each testing the clause database against up to 32 requests at once.  A new
 * launch takes every waiting request and starts only while fewer than tests_in_flight
 * test kernels run: the cost of a launch hardly depends on how many requests it carries
 * (it streams the whole database prefix once), so under load requests gather into larger
 * launches instead of splitting the GPU between many small ones; the other lanes overlap
 * a launch's packing with the routing and copies of the one before.
 *
 * Each request tests the clauses with id < its watermark: the number of clauses committed
 * when it was admitted (or a smaller value the caller asks for).  Its records therefore do
 * not depend on the other requests of its launch nor on clauses added later.  Records use
 * the caller's clause ids (in order of gss_server_add_clauses) and word 0; bit b of mask is
 * assignment b of the request.
 *
 * Threads: gss_server_add_clauses, gss_server_submit and gss_server_wait may be called from
 * any number of host threads; the database may grow while launches run.
 */
typedef struct gss_server gss_server;

typedef struct {
  int device;                    /* CUDA device ordinal */
  uint32_t mode;                 /* GSS_MODE_ALLF or GSS_MODE_TRIGGER */
  uint32_t layout;               /* GSS_LAYOUT_*; frequency numbering is fixed by the first clause batch */
  uint64_t max_clauses;          /* clause capacity reserved at creation (the database never moves) */
  uint64_t max_lits;             /* literal capacity reserved at creation */
  uint32_t slots;                /* request slots, 32 * ceil16(n_vars) bytes of device memory each */
  uint32_t lanes;                /* launches in flight at once (1 to 8) */
  uint64_t lane_report_capacity; /* records one launch can hold; more fail the launch's requests */
  uint64_t slot_memory_bytes;    /* non-zero: slots = min(slots, slot_memory_bytes / slot size) */
  uint32_t tests_in_flight;      /* launches whose test kernels may overlap (default 1; 0: lanes) */
  uint32_t pad;
  uint64_t result_ttl_us;        /* kept results not taken by gss_server_wait within this time after
                                    completion are dropped (a client that died; checked about every
                                    10-100 ms); 0: kept forever */
} gss_server_config;

/* Flags of gss_server_submit. */
#define GSS_SUBMIT_KEEP 1u /* keep the records for gss_server_wait (otherwise only counted) */

/* Watermark meaning "every clause committed at admission". */
#define GSS_WATERMARK_ALL 0xFFFFFFFFFFFFFFFFull

typedef struct {
  uint64_t watermark;  /* clauses the request was tested against: ids [0, watermark) */
  uint32_t n_assign;
  uint32_t batch_words; /* requests in the launch that carried it */
  double latency_us;    /* from the start of gss_server_submit to results on the host: */
  double admit_us;      /*   waiting for a slot and copying the request to the device */
  double queue_us;      /*   admitted, waiting for a launch */
  double run_us;        /*   the launch (pack, test, routing) and the hand-over */
} gss_request_info;

typedef struct {
  uint64_t submitted, dropped, completed; /* dropped: refused with GSS_E_BUSY */
  uint64_t launches, words_launched;      /* launches and the requests they carried */
  uint64_t pair_tests;                    /* sum over completed requests of watermark * n_assign */
  uint64_t reports;                       /* records delivered (after dropping padded assignments) */
  uint64_t committed_clauses;
  uint64_t expired;                       /* kept results dropped after result_ttl_us */
  uint32_t slots, pad;
  double p50_us, p99_us, max_us, mean_us; /* latency of completed requests */
  uint64_t next_clause_id;                /* requests admitted now test the resident clauses with
                                             smaller ids (committed_clauses counts the resident ones) */
  uint64_t reductions, clauses_removed;   /* gss_server_reduce calls and the clauses they removed */
} gss_server_stats;

/* Fill *cfg with the defaults: device 0, all-F, frequency layout, 1M clauses and 16M literals
 * reserved, 64 slots, 3 lanes, one test in flight, 1M records per lane, results kept forever. */
int gss_server_config_init(gss_server_config* cfg);

/* Create a server for n_vars variables; reserves the database and request slots and starts
 * the scheduler thread.  GSS_E_NOMEM if the reservation does not fit. */
int gss_server_create(gss_server** out, uint32_t n_vars, const gss_server_config* cfg);

/* Stop the scheduler (launches in flight finish first) and free everything. */
int gss_server_destroy(gss_server* srv);

/* Append clauses as gss_add_clauses (host CSR).  They are visible to requests admitted
 * after the call returns.  GSS_E_NOMEM when the reserved capacity would be exceeded. */
int gss_server_add_clauses(gss_server* srv, const uint64_t* offsets, uint64_t n_clauses, const uint32_t* lits,
                           uint32_t* first_id);

/*
 * Submit a request: values holds n_assign (1..32) rows of n_vars codes (0 = U, 1 = T,
 * 2 = F), row-major, in host memory; it may be reused when the call returns.  watermark
 * caps the clauses tested (GSS_WATERMARK_ALL: all committed ones).  wait_us: how long to
 * wait for a free slot (0: refuse at once with GSS_E_BUSY).  *request_id identifies the
 * request for gss_server_wait when flags has GSS_SUBMIT_KEEP.
 */
int gss_server_submit(gss_server* srv, const uint8_t* values, uint32_t n_assign, uint64_t watermark, int64_t wait_us,
                      uint32_t flags, uint64_t* request_id);

/*
 * Wait up to wait_us (negative: without limit) for a kept request and take its records
 * into out (*n_out = their number; records in no particular order).  With more than cap
 * records nothing is copied, *n_out holds the count, GSS_E_OVERFLOW is returned and the
 * request is kept: call again with a larger buffer.  Otherwise the request is forgotten
 * afterwards unless the result is GSS_E_TIMEOUT (not finished yet).  GSS_E_OVERFLOW with
 * records copied: the launch's record buffer overflowed and the records are incomplete.
 * GSS_E_INVAL: a code outside {0, 1, 2} was in the request's launch.  One waiter per
 * request.  info (nullable) receives the watermark, batch size and latency.
 */
int gss_server_wait(gss_server* srv, uint64_t request_id, int64_t wait_us, gss_report* out, uint64_t cap,
                    uint64_t* n_out, gss_request_info* info);

/*
 * Clause activity and deletion on the server's resident database (Section 3.6: the GPU
 * deletes clauses by activity as MiniSat does, bumping a clause whenever it triggers).
 * gss_server_set_activity switches activities on (decay as gss_set_activity) and reserves
 * the activity arrays for max_clauses; it needs tests_in_flight = 1, so that one test bumps
 * at a time (GSS_E_STATE otherwise).  Each launch then counts as one test of gss_set_activity's
 * rules: every clause reported by the launch (for any of its requests) is bumped once by the
 * increment, which grows by 1 / decay after each launch; a clause added starts at the
 * current increment.
 *
 * gss_server_reduce removes floor(f * n) of the n resident clauses longer than two literals,
 * those with the smallest (activity, id), exactly as gss_reduce_db.  It waits until no launch
 * runs, holds new launches (requests are still admitted) and ingest meanwhile, compacts the
 * database into new arrays, reserves capacity again and publishes it; launches started
 * afterwards read the compacted database.  Watermarks are clause-id bounds: a request tests
 * the clauses resident at its launch whose id is below its watermark, so a request admitted
 * before a reduction but launched after it skips the removed clauses.  Ids never change and
 * are never reused.  Needs room for a second copy of the database while it runs; on
 * GSS_E_NOMEM the database is unchanged.  *n_removed (nullable) receives the count.
 *
 * gss_server_get_activity / gss_server_get_clause_ids copy the activities / ids of the
 * resident clauses in position order (as gss_get_activity / gss_get_clause_ids); values read
 * while launches run may be mid-update.
 */
int gss_server_set_activity(gss_server* srv, float decay);
int gss_server_reduce(gss_server* srv, double remove_fraction, uint64_t* n_removed);
int gss_server_get_activity(gss_server* srv, float* out, uint64_t cap, uint64_t* n_out);
int gss_server_get_clause_ids(gss_server* srv, uint32_t* out, uint64_t cap, uint64_t* n_out);

/* Counters since creation and the latency percentiles of every completed request. */
int gss_server_get_stats(gss_server* srv, gss_server_stats* out);
/* Message of the calling thread's last failed call on a server (each thread keeps its own). */
const char* gss_server_last_error(const gss_server* srv);

/* ---------------------------------------------------------- diagnostics */

/*
 * The bounds-checked build (compiled with GSS_DEBUG_BOUNDS; the Python binding loads it when
 * the environment variable GSS_DEBUG_BOUNDS=1 is set) checks, in the test kernels, every
 * plane row index before gathering with it; an index out of range is counted on the device
 * and replaced by the neutral PAD row.  *enabled = 1 in that build (0 otherwise, *errors = 0);
 * *errors = violations counted on the current device since the last reset (reset != 0
 * zeroes the counter).  Synchronises the device.
 */
int gss_debug_bounds(uint32_t* enabled, uint64_t* errors, int reset);

/* Sizes, counters and the last test's aggregate-test counts (see gss_stats). */
int gss_get_stats(const gss_ctx* ctx, gss_stats* out);

/* Message of the last failed call on ctx ("" if none); a static string for NULL ctx. */
const char* gss_last_error(const gss_ctx* ctx);

/* Name of a status code. */
const char* gss_strerror(int code);

/* Library version, (major << 16) | minor. */
uint32_t gss_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GSS_H */
