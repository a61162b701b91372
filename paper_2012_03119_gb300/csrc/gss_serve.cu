// gss_serve.cu -- serving: continuous batching of assignment snapshots against a growing,
// resident clause database (Section 3.6: solver threads send the parent assignment of
// each conflict and every learned clause to the GPU; the GPU tests all of its clauses
// against the assignments it has not tested yet and reports back to each thread).
//
// Requests.  A request is one snapshot of up to 32 assignments (one plane word).
// gss_server_submit copies it into a free device slot; when no slot frees up within the
// caller's wait the request is refused with GSS_E_BUSY -- the paper's "not sent to the GPU
// when it is full".  Slots are the unit of memory admission.  A request tests the clauses
// present when it was admitted (its watermark): clause c is tested against the request iff
// c < watermark, so its result depends neither on the other requests of its launch nor on
// clauses arriving later.
//
// Scheduling.  A scheduler thread keeps up to `lanes` launches in flight, each on its own
// stream with its own planes and record buffer.  Whenever a lane is free it takes the
// admitted requests not yet launched (up to 32, oldest first), orders them by watermark,
// packs their slots into one plane set (plane word w = request w, read from its slot
// through a row table) and tests clauses [0, largest watermark) with per-word watermarks.
// Requests that arrive while launches run are admitted into free slots and join the next
// launch; the launches of different lanes overlap on the device.  After the test, a routing
// kernel groups the launch's records by request straight into mapped host memory, and a
// host function on the lane's stream wakes the scheduler, which hands each request its run
// of records.
//
// Clause ingest.  gss_server_add_clauses appends learned clauses (gss_add_clauses on the
// server's own context and stream) into capacity reserved at creation, so the arrays that
// running launches read never move and only rows past every watermark are written; new
// clauses become visible to requests admitted after the call returns.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "gss_ctx.h"

using namespace gss;
using namespace gss::host;
using Clock = std::chrono::steady_clock;

namespace {

constexpr uint32_t MAX_LANES = 8;

struct Request {
  uint32_t slot = 0, n = 0;
  uint64_t wm = 0;      // watermark: clause ids below it
  uint64_t wm_pos = 0;  // the same bound in positions of the database the launch read
  bool keep = false, done = false, overflow = false, bad = false;
  uint32_t waiters = 0;  // clients inside gss_server_wait on it: never dropped meanwhile
  uint32_t batch_words = 0;
  Clock::time_point t_submit, t_admit, t_launch, t_done;
  std::vector<gss_report> recs;
};

// Per-launch inputs (one host-to-device copy) and outputs (one device-to-host copy).
struct LaunchIn {
  uint64_t wm[32];     // watermark of each plane word, non-decreasing
  uint32_t rows[32];   // first code row of each word's slot
  uint32_t nmask[32];  // bits of each word that are real assignments
};
struct LaunchOut {
  DevStatus st;       // test and routing
  DevStatus pack_st;  // packing: invalid codes per word (kept apart so the test still runs for the others)
  unsigned long long count[32];  // routed records per word
  unsigned long long cursor[32];
};

struct Lane {
  gss_server* srv = nullptr;
  cudaStream_t s = nullptr;
  uint32_t *P = nullptr, *aggF = nullptr, *aggU = nullptr;
  gss_report* rec = nullptr;    // device: the test's records
  gss_report* h_rec = nullptr;  // mapped host: routed records
  uint64_t cap = 0;
  LaunchIn *d_in = nullptr, *h_in = nullptr;
  LaunchOut *d_out = nullptr, *h_out = nullptr;
  cudaEvent_t ev = nullptr;
  std::vector<uint64_t> ids;
  bool busy = false, testing = false;  // testing: the launch's test kernel may still run
  std::atomic<int> signalled{0}, tested{0};
};

}  // namespace

struct gss_server {
  int device = 0;
  uint32_t V = 0, Vp = 0, mode = GSS_MODE_ALLF;
  gss_ctx* ctx = nullptr;
  ClauseView db{};                            // reserved arrays: fixed after creation
  std::atomic<const uint32_t*> map{nullptr};  // variable numbering, fixed by the first batch
  uint32_t n_slots = 0;
  uint8_t* d_slots = nullptr;  // [n_slots * 32][Vp] value codes
  std::vector<cudaEvent_t> slot_ev;
  cudaStream_t copy_stream = nullptr;
  std::vector<Lane> lanes;  // sized once at creation (lanes are not movable)
  int grid = 0, route_grid = 0;
  uint32_t tests_in_flight = 1;  // launches whose test may overlap
  uint64_t ttl_us = 0;           // kept results older than this are dropped (0: never)
  Clock::time_point last_sweep;

  std::mutex mu, ingest_mu;
  std::condition_variable cv_slot, cv_done;
  std::deque<uint32_t> free_slots;
  std::deque<uint64_t> ready;
  std::unordered_map<uint64_t, Request> reqs;
  uint64_t next_id = 1;
  std::atomic<uint64_t> committed{0};  // clause ids below this are committed (visible to new requests)
  std::atomic<uint64_t> resident{0};   // clauses held (fewer than committed once a reduction removed some)
  uint64_t max_clauses = 0, max_lits = 0;
  // clause activity (Section 3.6): each launch is one test for the bumps; off until enabled
  bool activity = false;
  float act_inc = 1.0f, act_inv_decay = 1.0f;
  uint32_t act_epoch = 0;
  // after a reduction, the ids of the resident clauses in position order (host copy), to turn
  // a request's watermark (a clause id bound) into a position bound at launch time
  bool reduced = false, reducing = false;
  std::vector<uint32_t> h_ids;
  uint64_t reductions = 0, removed = 0;
  std::thread sched;
  bool stop = false, closed = false;  // closed: the scheduler has exited
  int sched_err = GSS_OK;
  std::string sched_msg;

  std::mutex wake_mu;  // wakes the scheduler: submissions, finished launches, destroy
  std::condition_variable cv_wake;
  bool wake = false;

  uint64_t submitted = 0, dropped = 0, completed = 0, launches = 0, words = 0, pair_tests = 0, reports = 0;
  uint64_t expired = 0;
  std::vector<double> lat_us;
};

namespace {

// The message of the calling thread's last failed server call: several threads use one
// server at once, so each keeps its own.
thread_local std::string t_err;

int sfail(gss_server* v, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (v) {
    t_err = buf;
  }
  return code;
}

void wake_scheduler(gss_server* v) {
  {
    std::lock_guard<std::mutex> g(v->wake_mu);
    v->wake = true;
  }
  v->cv_wake.notify_one();
}

// Host functions after a launch's test and at its end (a driver thread; no CUDA calls here).
void CUDART_CB lane_tested(void* p) {
  Lane* L = static_cast<Lane*>(p);
  L->tested.store(1);
  wake_scheduler(L->srv);
}

void CUDART_CB lane_done(void* p) {
  Lane* L = static_cast<Lane*>(p);
  L->signalled.store(1);
  wake_scheduler(L->srv);
}

// Position bound of a watermark (a clause id bound): the number of resident clauses whose
// id is below it (v->mu held).  Ids grow with position, so this is a lower bound search.
uint64_t position_bound(const gss_server* v, uint64_t wm) {
  if (!v->reduced) return wm;  // ids are positions until the first reduction
  return (uint64_t)(std::lower_bound(v->h_ids.begin(), v->h_ids.end(), wm) - v->h_ids.begin());
}

// Start a launch on lane L with the oldest admitted requests (v->mu held).
cudaError_t start_launch(gss_server* v, Lane& L) {
  TraceRange tr("gss_server launch");
  const uint32_t k = (uint32_t)std::min<size_t>(32, v->ready.size());
  L.ids.assign(v->ready.begin(), v->ready.begin() + k);
  v->ready.erase(v->ready.begin(), v->ready.begin() + k);
  // watermarks must be non-decreasing over plane words
  std::stable_sort(L.ids.begin(), L.ids.end(), [&](uint64_t a, uint64_t b) { return v->reqs[a].wm < v->reqs[b].wm; });
  uint64_t max_wm = 0;
  for (uint32_t w = 0; w < k; ++w) {
    Request& r = v->reqs[L.ids[w]];
    r.batch_words = k;
    r.t_launch = Clock::now();
    L.h_in->rows[w] = r.slot * 32u;
    L.h_in->wm[w] = r.wm_pos = position_bound(v, r.wm);  // clause positions < this have ids < the watermark
    L.h_in->nmask[w] = r.n >= 32 ? 0xFFFFFFFFu : ((1u << r.n) - 1u);
    max_wm = std::max(max_wm, L.h_in->wm[w]);
  }
  const uint32_t N = 32u * k;
  const uint32_t Wp = words_stride(N), AWp = agg_stride(Wp);
  L.busy = L.testing = true;
  L.signalled.store(0);
  L.tested.store(0);
  v->launches += 1;
  v->words += k;
  cudaError_t e = cudaSuccess;
  for (uint32_t w = 0; w < k && e == cudaSuccess; ++w)  // the slot copies must have landed
    e = cudaStreamWaitEvent(L.s, v->slot_ev[L.h_in->rows[w] / 32u], 0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(L.d_in, L.h_in, sizeof(LaunchIn), cudaMemcpyHostToDevice, L.s);
  if (e == cudaSuccess) e = cudaMemsetAsync(&L.d_out->st, 0, 2 * sizeof(DevStatus), L.s);
  if (e == cudaSuccess)
    e = launch_pack_rows(v->d_slots, v->Vp, v->V, N, Wp, AWp, v->map.load(), L.d_in->rows, v->n_slots * 32u, L.P,
                         L.aggF, L.aggU, &L.d_out->pack_st, L.s, L.d_in->nmask);
  if (e == cudaSuccess && max_wm) {
    // the U rows that pad a request of fewer than 32 assignments make no record (in trigger
    // mode a unit clause triggers on them), so they never count against the launch's capacity
    PlaneView pv{L.P, L.aggF, L.aggU, Wp, AWp, N, v->V};
    pv.wvalid = L.d_in->nmask;
    ActivityView av;
    if (v->activity) av = ActivityView{v->ctx->act, v->ctx->stamp, v->act_epoch, v->act_inc};
    e = launch_test((int)v->mode, v->db, 0, max_wm, pv, L.rec, L.cap, &L.d_out->st, v->grid, L.s, L.d_in->wm, k, av);
  }
  if (v->activity) {  // the launch was one test: the increment grows, rescaled past 1e20 after its bumps
    v->act_epoch = v->act_epoch + 1 == 0xFFFFFFFFu ? 0 : v->act_epoch + 1;
    v->act_inc = v->act_inc * v->act_inv_decay;
    if (e == cudaSuccess && v->act_inc > 1e20f) {
      e = launch_scale_f32(v->ctx->act, v->resident.load(), 1e-20f, L.s);  // before the next launch's test
      v->act_inc = v->act_inc * 1e-20f;
    }
  }
  if (e == cudaSuccess) e = cudaLaunchHostFunc(L.s, lane_tested, &L);
  if (e == cudaSuccess)
    e = launch_route(L.rec, &L.d_out->st, L.cap, L.d_in->nmask, k, L.d_out->count, L.d_out->cursor, L.h_rec,
                     v->route_grid, L.s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(L.h_out, L.d_out, sizeof(LaunchOut), cudaMemcpyDeviceToHost, L.s);
  if (e == cudaSuccess) e = cudaEventRecord(L.ev, L.s);
  if (e == cudaSuccess) e = cudaLaunchHostFunc(L.s, lane_done, &L);
  return e;
}

// L's launch has finished (v->mu held): hand each request its run of records.
void finish_launch(gss_server* v, Lane& L) {
  const DevStatus& st = L.h_out->st;
  const DevStatus& pst = L.h_out->pack_st;
  const bool overflow = st.n_records > L.cap;
  const Clock::time_point now = Clock::now();
  uint64_t at = 0;
  for (size_t w = 0; w < L.ids.size(); ++w) {
    const uint64_t cnt = L.h_out->count[w];
    Request& q = v->reqs[L.ids[w]];
    if (q.keep && cnt) q.recs.assign(L.h_rec + at, L.h_rec + at + cnt);
    at += cnt;
    v->reports += cnt;
    q.done = true;
    q.overflow = overflow;
    // an invalid code spoils only its own request; a timeout or an overflow spoils the whole launch
    q.bad = ((pst.bad_code >> w) & 1u) != 0u || st.timeout != 0u || pst.timeout != 0u;
    q.t_done = now;
    v->lat_us.push_back(std::chrono::duration<double, std::micro>(q.t_done - q.t_submit).count());
    v->pair_tests += q.wm_pos * (uint64_t)q.n;
    v->completed += 1;
    v->free_slots.push_back(q.slot);
    if (!q.keep) v->reqs.erase(L.ids[w]);
  }
  L.ids.clear();
  L.busy = L.testing = false;
  v->cv_slot.notify_all();
  v->cv_done.notify_all();
}

void scheduler(gss_server* v) {
  cudaSetDevice(v->device);
  for (;;) {
    {
      std::unique_lock<std::mutex> wl(v->wake_mu);
      // the timeout is a backstop that notices a launch whose stream failed
      v->cv_wake.wait_for(wl, std::chrono::milliseconds(100), [&] { return v->wake; });
      v->wake = false;
    }
    std::lock_guard<std::mutex> g(v->mu);
    uint32_t testing = 0;
    for (Lane& L : v->lanes) {
      if (!L.busy) continue;
      if (L.testing && L.tested.exchange(0)) L.testing = false;
      if (L.signalled.exchange(0)) {
        finish_launch(v, L);
        continue;
      }
      const cudaError_t q = cudaEventQuery(L.ev);
      if (q != cudaSuccess && q != cudaErrorNotReady && v->sched_err == GSS_OK) {
        v->sched_err = GSS_E_CUDA;
        v->sched_msg = cudaGetErrorString(q);
        v->stop = true;
      }
    }
    for (Lane& L : v->lanes) testing += L.testing ? 1u : 0u;
    // a new launch takes every waiting request; it starts only while fewer than
    // tests_in_flight tests run, so that requests gather into larger launches under load
    for (Lane& L : v->lanes) {
      if (v->stop || v->reducing || v->ready.empty() || L.busy || testing >= v->tests_in_flight) continue;
      ++testing;
      const cudaError_t e = start_launch(v, L);
      if (e != cudaSuccess && v->sched_err == GSS_OK) {
        v->sched_err = GSS_E_CUDA;
        v->sched_msg = cudaGetErrorString(e);
        v->stop = true;
      }
    }
    if (v->ttl_us) {  // drop kept results whose client has not taken them in time (a dead solver thread)
      const Clock::time_point now = Clock::now();
      if (now - v->last_sweep > std::chrono::milliseconds(10)) {
        v->last_sweep = now;
        for (auto it = v->reqs.begin(); it != v->reqs.end();) {
          const Request& q = it->second;
          if (q.done && q.waiters == 0 && now - q.t_done > std::chrono::microseconds(v->ttl_us)) {
            it = v->reqs.erase(it);
            v->expired += 1;
          } else {
            ++it;
          }
        }
      }
    }
    if (v->stop) {  // on destroy, let launches in flight finish; on an error, leave now
      bool in_flight = false;
      for (Lane& L : v->lanes) in_flight |= L.busy;
      if (!in_flight || v->sched_err != GSS_OK) break;
    }
  }
  {
    std::lock_guard<std::mutex> g(v->mu);
    v->closed = true;
  }
  v->cv_done.notify_all();
  v->cv_slot.notify_all();
}

void release(gss_server* v) {
  if (v->sched.joinable()) {
    {
      std::lock_guard<std::mutex> g(v->mu);
      v->stop = true;
    }
    wake_scheduler(v);
    v->sched.join();
  }
  cudaSetDevice(v->device);
  for (Lane& L : v->lanes) {
    if (L.s) cudaStreamSynchronize(L.s);
    cudaFree(L.P);
    cudaFree(L.aggF);
    cudaFree(L.aggU);
    cudaFree(L.rec);
    cudaFree(L.d_in);
    cudaFree(L.d_out);
    cudaFreeHost(L.h_rec);
    cudaFreeHost(L.h_in);
    cudaFreeHost(L.h_out);
    if (L.ev) cudaEventDestroy(L.ev);
    if (L.s) cudaStreamDestroy(L.s);
  }
  if (v->copy_stream) {
    cudaStreamSynchronize(v->copy_stream);
    cudaStreamDestroy(v->copy_stream);
  }
  for (cudaEvent_t e : v->slot_ev) cudaEventDestroy(e);
  cudaFree(v->d_slots);
  if (v->ctx) gss_destroy(v->ctx);
  cudaGetLastError();
}

}  // namespace

extern "C" {

int gss_server_config_init(gss_server_config* c) {
  if (!c) return GSS_E_INVAL;
  memset(c, 0, sizeof *c);
  c->device = 0;
  c->mode = GSS_MODE_ALLF;
  c->layout = GSS_LAYOUT_FREQUENCY;
  c->max_clauses = 1u << 20;
  c->max_lits = 1u << 24;
  c->slots = 64;
  c->lanes = 3;
  c->lane_report_capacity = 1u << 20;
  c->slot_memory_bytes = 0;
  c->tests_in_flight = 1;
  return GSS_OK;
}

int gss_server_create(gss_server** out, uint32_t n_vars, const gss_server_config* cfg_in) {
  if (!out) return GSS_E_INVAL;
  *out = nullptr;
  gss_server_config cfg;
  if (cfg_in) cfg = *cfg_in;
  else gss_server_config_init(&cfg);
  if (n_vars == 0 || n_vars >= (1u << 31) || cfg.slots == 0 || cfg.lanes == 0 || cfg.lanes > MAX_LANES ||
      cfg.lane_report_capacity == 0 || cfg.max_clauses == 0 || cfg.max_clauses >= (1ull << 32) ||
      (cfg.mode != GSS_MODE_ALLF && cfg.mode != GSS_MODE_TRIGGER))
    return GSS_E_INVAL;
  gss_server* v = new (std::nothrow) gss_server();
  if (!v) return GSS_E_NOMEM;
  v->device = cfg.device;
  v->V = n_vars;
  v->Vp = (n_vars + 15u) / 16u * 16u;  // slot rows 16-byte aligned for the tensor map
  v->mode = cfg.mode;
  const uint64_t slot_bytes = 32ull * v->Vp;
  v->n_slots = cfg.slots;
  if (cfg.slot_memory_bytes) {  // memory admission: as many slots as the budget holds
    const uint64_t fit = cfg.slot_memory_bytes / slot_bytes;
    if (fit == 0) {
      delete v;
      return GSS_E_NOMEM;
    }
    if (fit < v->n_slots) v->n_slots = (uint32_t)fit;
  }
  gss_config cc;
  gss_config_init(&cc);
  cc.device = cfg.device;
  cc.mode = cfg.mode;
  cc.layout = cfg.layout;
  cc.max_assignments = 32;
  cc.report_capacity = 1;
  int rc = gss_create(&v->ctx, n_vars, &cc);
  if (rc) {
    delete v;
    return rc;
  }
  rc = reserve_db(v->ctx, cfg.max_clauses, cfg.max_lits);
  v->max_clauses = cfg.max_clauses;
  v->max_lits = cfg.max_lits;
  bool ok = rc == GSS_OK && cudaSetDevice(cfg.device) == cudaSuccess;
  if (ok) v->db = ClauseView{v->ctx->off, v->ctx->lits, v->ctx->head0, v->ctx->head1, 2u * n_vars};
  ok = ok && cudaStreamCreateWithFlags(&v->copy_stream, cudaStreamNonBlocking) == cudaSuccess;
  ok = ok && cudaMalloc(&v->d_slots, v->n_slots * slot_bytes) == cudaSuccess;
  ok = ok && cudaMemset(v->d_slots, 0, v->n_slots * slot_bytes) == cudaSuccess;
  for (uint32_t i = 0; ok && i < v->n_slots; ++i) {
    cudaEvent_t e;
    ok = cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
    if (ok) v->slot_ev.push_back(e);
    v->free_slots.push_back(i);
  }
  const uint32_t Wp = 32, AWp = 1;  // planes for up to 32 requests
  std::vector<Lane> lanes(cfg.lanes);
  v->lanes.swap(lanes);
  for (Lane& L : v->lanes) {
    L.srv = v;
    L.cap = cfg.lane_report_capacity;
    ok = ok && cudaStreamCreateWithFlags(&L.s, cudaStreamNonBlocking) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&L.ev, cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaMalloc(&L.P, (2ull * n_vars + 2) * Wp * 4) == cudaSuccess;
    ok = ok && cudaMalloc(&L.aggF, (2ull * n_vars + 2) * AWp * 4) == cudaSuccess;
    ok = ok && cudaMalloc(&L.aggU, (n_vars + 1ull) * AWp * 4) == cudaSuccess;
    ok = ok && cudaMalloc(&L.rec, L.cap * sizeof(gss_report)) == cudaSuccess;
    ok = ok && cudaMalloc(&L.d_in, sizeof(LaunchIn)) == cudaSuccess;
    ok = ok && cudaMalloc(&L.d_out, sizeof(LaunchOut)) == cudaSuccess;
    ok = ok && cudaHostAlloc(&L.h_rec, L.cap * sizeof(gss_report), cudaHostAllocMapped) == cudaSuccess;
    ok = ok && cudaMallocHost(&L.h_in, sizeof(LaunchIn)) == cudaSuccess;
    ok = ok && cudaMallocHost(&L.h_out, sizeof(LaunchOut)) == cudaSuccess;
  }
  if (!ok) {
    release(v);
    delete v;
    return rc ? rc : GSS_E_NOMEM;
  }
  v->grid = test_grid_size((int)cfg.mode, 1, v->ctx->n_sms);
  v->route_grid = 2 * v->ctx->n_sms;
  v->tests_in_flight = cfg.tests_in_flight ? cfg.tests_in_flight : cfg.lanes;
  v->ttl_us = cfg.result_ttl_us;
  v->last_sweep = Clock::now();
  v->sched = std::thread(scheduler, v);
  *out = v;
  return GSS_OK;
}

int gss_server_destroy(gss_server* v) {
  if (!v) return GSS_OK;
  release(v);
  delete v;
  return GSS_OK;
}

int gss_server_add_clauses(gss_server* v, const uint64_t* offsets, uint64_t n, const uint32_t* lits,
                           uint32_t* first_id) {
  if (!v) return GSS_E_INVAL;
  std::lock_guard<std::mutex> g(v->ingest_mu);
  gss_ctx* c = v->ctx;
  if (n && !offsets) return sfail(v, GSS_E_INVAL, "offsets is NULL");
  const uint64_t L = n ? offsets[n] : 0;
  if (c->m + n + 1 > c->cap_m || (c->m + n) * 8 > c->cap_head0 || c->L + L > c->cap_L ||
      (c->act && c->m + n > c->cap_act) || (c->ext && c->m + n > c->cap_ext))
    return sfail(v, GSS_E_NOMEM, "reserved database capacity exceeded (%llu clauses, %llu literals reserved)",
                 (unsigned long long)(c->cap_m - 1), (unsigned long long)c->cap_L);
  {
    std::lock_guard<std::mutex> g(v->mu);
    c->inc = v->act_inc;  // a new clause starts at the current increment
  }
  uint32_t first = 0;
  int rc = gss_add_clauses(c, offsets, n, lits, &first);
  if (rc) return sfail(v, rc, "%s", gss_last_error(c));
  if (first_id) *first_id = first;
  cudaError_t e = cudaStreamSynchronize(c->stream);  // rows complete before any request may see them
  if (e != cudaSuccess) return sfail(v, GSS_E_CUDA, "ingest: %s", cudaGetErrorString(e));
  v->map.store(c->map);
  if (v->reduced) {
    std::lock_guard<std::mutex> g(v->mu);
    for (uint64_t i = 0; i < n; ++i) v->h_ids.push_back(first + (uint32_t)i);
  }
  v->resident.store(c->m);
  v->committed.store(c->next_id);
  return GSS_OK;
}

// Wait until no launch runs and none starts (ingest_mu held): the database may then change.
static int drain_launches(gss_server* v) {
  std::unique_lock<std::mutex> lk(v->mu);
  v->reducing = true;
  v->cv_done.wait(lk, [&] {
    bool busy = false;
    for (const Lane& L : v->lanes) busy |= L.busy;
    return !busy || v->sched_err != GSS_OK || v->closed;
  });
  if (v->sched_err != GSS_OK) {
    v->reducing = false;
    return sfail(v, v->sched_err, "scheduler stopped: %s", v->sched_msg.c_str());
  }
  return GSS_OK;
}

static void resume_launches(gss_server* v) {
  {
    std::lock_guard<std::mutex> g(v->mu);
    v->reducing = false;
  }
  wake_scheduler(v);
}

int gss_server_set_activity(gss_server* v, float decay) {
  if (!v) return GSS_E_INVAL;
  if (!(decay > 0.0f && decay <= 1.0f)) return sfail(v, GSS_E_INVAL, "decay must be in (0, 1]");
  if (v->tests_in_flight != 1)
    return sfail(v, GSS_E_STATE, "activity needs tests_in_flight = 1 (one test bumps at a time)");
  std::lock_guard<std::mutex> g(v->ingest_mu);
  int rc = drain_launches(v);
  if (rc) return rc;
  gss_ctx* c = v->ctx;
  const bool first = c->act == nullptr;
  rc = gss_set_activity(c, decay);
  if (!rc) rc = reserve_clause_arrays(c, v->max_clauses);  // the arrays never move under a launch
  if (rc) {
    resume_launches(v);
    return sfail(v, rc, "%s", gss_last_error(c));
  }
  {
    std::lock_guard<std::mutex> lk(v->mu);
    if (first) {
      v->act_inc = 1.0f;
      v->act_epoch = 0;
    }
    v->act_inv_decay = c->inv_decay;
    v->activity = true;
  }
  resume_launches(v);
  return GSS_OK;
}

int gss_server_reduce(gss_server* v, double remove_fraction, uint64_t* n_removed) {
  if (!v) return GSS_E_INVAL;
  if (n_removed) *n_removed = 0;
  TraceRange tr("gss_server_reduce");
  std::lock_guard<std::mutex> g(v->ingest_mu);
  if (!v->activity) return sfail(v, GSS_E_STATE, "gss_server_reduce needs activities (gss_server_set_activity)");
  int rc = drain_launches(v);
  if (rc) return rc;
  gss_ctx* c = v->ctx;
  uint64_t n = 0;
  rc = gss_reduce_db(c, remove_fraction, &n);
  // the compacted arrays are sized to the kept clauses: reserve them again, so that later
  // ingest never moves them under a running launch
  if (!rc) rc = reserve_db(c, v->max_clauses, v->max_lits);
  if (!rc) rc = reserve_clause_arrays(c, v->max_clauses);
  std::vector<uint32_t> ids(c->m);
  if (!rc && c->m) {
    const cudaError_t e = c->ext ? cudaMemcpy(ids.data(), c->ext, c->m * sizeof(uint32_t), cudaMemcpyDeviceToHost)
                                 : cudaErrorInvalidValue;
    if (e != cudaSuccess) rc = fail(c, GSS_E_CUDA, "clause ids: %s", cudaGetErrorString(e));
  }
  if (rc) {  // gss_reduce_db leaves the database unchanged on failure; a failed reservation leaves it valid
    resume_launches(v);
    return sfail(v, rc, "%s", gss_last_error(c));
  }
  {
    std::lock_guard<std::mutex> lk(v->mu);
    v->db = ClauseView{c->off, c->lits, c->head0, c->head1, 2u * c->V, c->ext};
    v->h_ids.swap(ids);
    v->reduced = true;
    v->reductions += 1;
    v->removed += n;
  }
  v->resident.store(c->m);
  resume_launches(v);
  if (n_removed) *n_removed = n;
  return GSS_OK;
}

// Copies of the server context's per-clause arrays (activities, ids), in position order.
int gss_server_get_activity(gss_server* v, float* out, uint64_t cap, uint64_t* n_out) {
  if (!v) return GSS_E_INVAL;
  std::lock_guard<std::mutex> g(v->ingest_mu);
  const int rc = gss_get_activity(v->ctx, out, cap, n_out);
  return rc ? sfail(v, rc, "%s", gss_last_error(v->ctx)) : GSS_OK;
}

int gss_server_get_clause_ids(gss_server* v, uint32_t* out, uint64_t cap, uint64_t* n_out) {
  if (!v) return GSS_E_INVAL;
  std::lock_guard<std::mutex> g(v->ingest_mu);
  const int rc = gss_get_clause_ids(v->ctx, out, cap, n_out);
  return rc ? sfail(v, rc, "%s", gss_last_error(v->ctx)) : GSS_OK;
}

int gss_server_submit(gss_server* v, const uint8_t* values, uint32_t n_assign, uint64_t watermark, int64_t wait_us,
                      uint32_t flags, uint64_t* request_id) {
  if (!v || !values || !request_id) return GSS_E_INVAL;
  if (n_assign == 0 || n_assign > 32) return sfail(v, GSS_E_INVAL, "a request holds 1 to 32 assignments");
  const Clock::time_point t0 = Clock::now();
  uint32_t slot;
  {
    std::unique_lock<std::mutex> lk(v->mu);
    if (v->sched_err) return sfail(v, v->sched_err, "scheduler stopped: %s", v->sched_msg.c_str());
    v->submitted += 1;
    if (v->free_slots.empty() && wait_us > 0)
      v->cv_slot.wait_for(lk, std::chrono::microseconds(wait_us), [&] { return !v->free_slots.empty() || v->stop; });
    if (v->free_slots.empty()) {
      v->dropped += 1;
      return sfail(v, GSS_E_BUSY, "no free request slot");
    }
    slot = v->free_slots.front();
    v->free_slots.pop_front();
  }
  cudaSetDevice(v->device);
  uint8_t* dst = v->d_slots + (uint64_t)slot * 32u * v->Vp;
  // rows contiguous on both sides (n_vars a multiple of 16): one linear copy, faster than a pitched one
  cudaError_t e = v->V == v->Vp
                      ? cudaMemcpyAsync(dst, values, (uint64_t)n_assign * v->V, cudaMemcpyHostToDevice, v->copy_stream)
                      : cudaMemcpy2DAsync(dst, v->Vp, values, v->V, v->V, n_assign, cudaMemcpyHostToDevice,
                                          v->copy_stream);
  if (e == cudaSuccess && n_assign < 32)  // rows past the request are U
    e = cudaMemsetAsync(dst + (uint64_t)n_assign * v->Vp, 0, (uint64_t)(32 - n_assign) * v->Vp, v->copy_stream);
  if (e == cudaSuccess) e = cudaEventRecord(v->slot_ev[slot], v->copy_stream);
  if (e == cudaSuccess) e = cudaEventSynchronize(v->slot_ev[slot]);  // the caller may reuse values
  std::lock_guard<std::mutex> g(v->mu);
  if (e != cudaSuccess) {
    v->free_slots.push_back(slot);
    return sfail(v, GSS_E_CUDA, "request copy: %s", cudaGetErrorString(e));
  }
  const uint64_t now_m = v->committed.load();
  const uint64_t id = v->next_id++;
  Request& r = v->reqs[id];
  r.slot = slot;
  r.n = n_assign;
  r.wm = watermark < now_m ? watermark : now_m;
  r.keep = (flags & GSS_SUBMIT_KEEP) != 0;
  r.t_submit = t0;
  r.t_admit = Clock::now();
  v->ready.push_back(id);
  *request_id = id;
  wake_scheduler(v);
  return GSS_OK;
}

int gss_server_wait(gss_server* v, uint64_t id, int64_t wait_us, gss_report* out, uint64_t cap, uint64_t* n_out,
                    gss_request_info* info) {
  if (!v) return GSS_E_INVAL;
  std::unique_lock<std::mutex> lk(v->mu);
  auto it = v->reqs.find(id);
  if (it == v->reqs.end() || !it->second.keep) return sfail(v, GSS_E_INVAL, "unknown request or results not kept");
  Request* rp = &it->second;  // element references survive rehashing by other submits; iterators do not
  auto finished = [&] { return rp->done || v->sched_err != GSS_OK || v->closed; };
  if (!finished()) {
    rp->waiters += 1;
    if (wait_us < 0) v->cv_done.wait(lk, finished);
    else v->cv_done.wait_for(lk, std::chrono::microseconds(wait_us), finished);
    rp->waiters -= 1;
  }
  if (!rp->done) {
    if (v->sched_err) return sfail(v, v->sched_err, "scheduler stopped: %s", v->sched_msg.c_str());
    if (v->closed) return sfail(v, GSS_E_STATE, "server stopped before request %llu ran", (unsigned long long)id);
    return sfail(v, GSS_E_TIMEOUT, "request %llu not finished", (unsigned long long)id);
  }
  const uint64_t n = rp->recs.size();
  if (n_out) *n_out = n;
  if (info) {
    info->watermark = rp->wm;
    info->n_assign = rp->n;
    info->batch_words = rp->batch_words;
    auto us = [](Clock::time_point a, Clock::time_point b) { return std::chrono::duration<double, std::micro>(b - a).count(); };
    info->latency_us = us(rp->t_submit, rp->t_done);
    info->admit_us = us(rp->t_submit, rp->t_admit);
    info->queue_us = us(rp->t_admit, rp->t_launch);
    info->run_us = us(rp->t_launch, rp->t_done);
  }
  if (n > cap && !rp->bad)  // kept: the caller asks again with a larger buffer
    return sfail(v, GSS_E_OVERFLOW, "%llu records > capacity %llu", (unsigned long long)n, (unsigned long long)cap);
  Request r = std::move(*rp);
  v->reqs.erase(id);
  lk.unlock();
  if (r.bad) return sfail(v, GSS_E_INVAL, "a value code outside {0, 1, 2} in this request, or a device wait gave up");
  if (n && out) memcpy(out, r.recs.data(), n * sizeof(gss_report));
  if (r.overflow) return sfail(v, GSS_E_OVERFLOW, "the launch's record buffer overflowed; records are incomplete");
  return GSS_OK;
}

int gss_server_get_stats(gss_server* v, gss_server_stats* o) {
  if (!v || !o) return GSS_E_INVAL;
  std::vector<double> l;
  {
    std::lock_guard<std::mutex> g(v->mu);
    memset(o, 0, sizeof *o);
    o->submitted = v->submitted;
    o->dropped = v->dropped;
    o->completed = v->completed;
    o->launches = v->launches;
    o->words_launched = v->words;
    o->pair_tests = v->pair_tests;
    o->reports = v->reports;
    o->committed_clauses = v->resident.load();
    o->next_clause_id = v->committed.load();
    o->reductions = v->reductions;
    o->clauses_removed = v->removed;
    o->expired = v->expired;
    o->slots = v->n_slots;
    l = v->lat_us;
  }
  if (!l.empty()) {
    std::sort(l.begin(), l.end());
    auto pct = [&](double p) { return l[std::min(l.size() - 1, (size_t)(p * (double)(l.size() - 1) + 0.5))]; };
    o->p50_us = pct(0.50);
    o->p99_us = pct(0.99);
    o->max_us = l.back();
    double sum = 0;
    for (double x : l) sum += x;
    o->mean_us = sum / (double)l.size();
  }
  return GSS_OK;
}

const char* gss_server_last_error(const gss_server* v) { return v ? t_err.c_str() : "no server"; }

}  // extern "C"
