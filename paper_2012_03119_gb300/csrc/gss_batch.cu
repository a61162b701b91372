// gss_batch.cu -- host side of the batch ABI (include/gss.h, "batches").
//
// A batch holds many independent clause databases ("instances"), each with its own
// assignment set and report buffer -- the independent problems of a multi-solver
// deployment.  One gss_batch_test runs a CUDA graph captured once per batch layout:
//   1. reset the work counters and every instance's test status;
//   2. pack every instance's assignment set (one packing kernel per instance, on parallel
//      branches of the graph so small instances run side by side);
//   3. test every clause of every instance in ONE persistent launch per row width (AWp)
//      in which warps steal clause tiles from a device counter (k_test_batch).
// The launch shape of step 3 (tile shape -- 32 clauses per warp tile with a lane each, or 16
// with two lanes each --, tiles per steal, grid size) is chosen by timing candidates on the
// batch itself the first time it runs (gss_batch_get_info reports the choice).
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <new>
#include <sstream>
#include <string>
#include <vector>

#include "gss_ctx.h"

using namespace gss;
using namespace gss::host;

namespace {

constexpr int SIDE_STREAMS = 8;

constexpr int SHAPES = 2;  // tile shapes: index 0 = 32 clauses per tile, 1 = 16 (two lanes per clause)
inline int shape_cpw(int k) { return k ? 16 : 32; }

struct Group {  // instances sharing one aggregate row width
  uint32_t awp = 1;
  std::vector<uint32_t> members;
  uint64_t n_tiles[SHAPES] = {0, 0};     // tiles of each shape
  BatchInst* d_inst[SHAPES] = {nullptr, nullptr};  // descriptors, tile0 counted in tiles of each shape
  int full_grid[SHAPES] = {0, 0};        // occupancy-derived persistent grid of each shape
  unsigned long long* work = nullptr;
  uint32_t grab = 4;
  int grid = 0;
  int shape = 0;  // tuned shape
};

struct Captured {  // what the graph baked in for one instance
  const uint8_t* src;
  uint64_t pitch;
  uint32_t N, Wp;
};

}  // namespace

struct gss_batch {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  uint32_t mode = GSS_MODE_ALLF, layout = GSS_LAYOUT_FREQUENCY;
  int n_sms = 1;
  std::vector<gss_ctx*> inst;
  std::vector<Captured> captured;
  std::vector<Group> groups;
  DevStatus* bst = nullptr;
  DevStatus* h_bst = nullptr;
  cudaStream_t side[SIDE_STREAMS] = {};
  cudaEvent_t fork = nullptr, join[SIDE_STREAMS] = {};
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool dirty = true, tuned = false;
  float tuned_us = 0.f;
  uint64_t runs = 0;
  std::string err;
};

namespace {

int bfail(gss_batch* b, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (b) b->err = buf;
  return code;
}

#define BCK(b, call)                                                                              \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess) return bfail((b), GSS_E_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

struct Guard {
  int prev = -1;
  bool changed = false;
  explicit Guard(int d) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != d) changed = cudaSetDevice(d) == cudaSuccess;
  }
  ~Guard() {
    if (changed && prev >= 0) cudaSetDevice(prev);
  }
};

void drop_graph(gss_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

void drop_groups(gss_batch* b) {
  for (Group& g : b->groups) {
    for (int k = 0; k < SHAPES; ++k)
      if (g.d_inst[k]) cudaFree(g.d_inst[k]);
    if (g.work) cudaFree(g.work);
  }
  b->groups.clear();
}

int child_fail(gss_batch* b, gss_ctx* c, int rc) { return bfail(b, rc, "%s", gss_last_error(c)); }

// Descriptor tables, one group per aggregate row width.
int build_groups(gss_batch* b) {
  drop_groups(b);
  for (uint32_t i = 0; i < b->inst.size(); ++i) {
    gss_ctx* c = b->inst[i];
    if (!c->have_assign) return bfail(b, GSS_E_STATE, "instance %u has no assignment set", i);
    Group* g = nullptr;
    for (Group& x : b->groups)
      if (x.awp == c->AWp) g = &x;
    if (!g) {
      b->groups.emplace_back();
      g = &b->groups.back();
      g->awp = c->AWp;
    }
    g->members.push_back(i);
  }
  for (Group& g : b->groups) {
    for (int k = 0; k < SHAPES; ++k) {
      const uint64_t cpw = (uint64_t)shape_cpw(k);
      std::vector<BatchInst> h;
      uint64_t tiles = 0;
      for (uint32_t i : g.members) {
        gss_ctx* c = b->inst[i];
        BatchInst d{};
        d.db = ClauseView{c->off, c->lits, c->head0, c->head1, 2u * c->V};
        d.pv = PlaneView{c->P, c->aggF, c->aggU, c->Wp, c->AWp, c->N, c->V};
        d.m = c->N ? c->m : 0;  // an empty assignment set has nothing to test
        d.tile0 = tiles;
        d.rec = c->rec;
        d.cap = c->rec_cap;
        d.st = c->st;
        tiles += (d.m + cpw - 1) / cpw;
        h.push_back(d);
      }
      g.n_tiles[k] = tiles;
      BCK(b, cudaMalloc(&g.d_inst[k], h.size() * sizeof(BatchInst)));
      BCK(b, cudaMemcpyAsync(g.d_inst[k], h.data(), h.size() * sizeof(BatchInst), cudaMemcpyHostToDevice, b->stream));
      g.full_grid[k] = test_batch_grid_size((int)b->mode, g.awp, (int)cpw, b->n_sms);
    }
    BCK(b, cudaMalloc(&g.work, sizeof(unsigned long long)));
    g.shape = 0;
    g.grid = g.full_grid[0];
  }
  BCK(b, cudaStreamSynchronize(b->stream));
  return GSS_OK;
}

int enqueue_resets(gss_batch* b, cudaStream_t s) {
  for (Group& g : b->groups)
    BCK(b, launch_batch_reset(g.d_inst[0], (uint32_t)g.members.size(), g.work, b->bst, s));
  return GSS_OK;
}

int enqueue_tests(gss_batch* b, cudaStream_t s) {
  for (Group& g : b->groups)
    BCK(b, launch_test_batch((int)b->mode, g.awp, shape_cpw(g.shape), g.d_inst[g.shape], (uint32_t)g.members.size(),
                             g.n_tiles[g.shape], g.work, g.grab, b->bst, g.grid, s));
  return GSS_OK;
}

int enqueue_packs(gss_batch* b) {  // on the side streams, forked from and joined into b->stream
  BCK(b, cudaEventRecord(b->fork, b->stream));
  for (int k = 0; k < SIDE_STREAMS; ++k) BCK(b, cudaStreamWaitEvent(b->side[k], b->fork, 0));
  for (uint32_t i = 0; i < b->inst.size(); ++i) {
    int rc = pack_staged(b->inst[i], b->side[i % SIDE_STREAMS]);
    if (rc) return child_fail(b, b->inst[i], rc);
  }
  for (int k = 0; k < SIDE_STREAMS; ++k) {
    BCK(b, cudaEventRecord(b->join[k], b->side[k]));
    BCK(b, cudaStreamWaitEvent(b->stream, b->join[k], 0));
  }
  return GSS_OK;
}

// Tuned choices can persist across processes: with GSS_AUTOTUNE_CACHE naming a file, each
// group's (tiles per steal, grid, clauses per tile) is stored under a key of the device, the
// mode, the row width and the octave of the group's tile count, and reused by later runs.
std::mutex g_cache_mutex;

std::string cache_key(const gss_batch* b, const Group& g) {
  cudaDeviceProp p{};
  cudaGetDeviceProperties(&p, b->device);
  uint32_t oct = 0;
  while ((g.n_tiles[0] >> oct) > 1) ++oct;
  std::ostringstream k;
  for (const char* c = p.name; *c; ++c) k << (*c == ' ' ? '_' : *c);
  k << "/sm" << b->n_sms << "/mode" << b->mode << "/awp" << g.awp << "/oct" << oct;
  return k.str();
}

struct Choice {
  uint32_t grab;
  int grid;
  int cpw;
};

std::map<std::string, Choice> read_cache(const char* path) {
  std::map<std::string, Choice> m;
  std::ifstream f(path);
  std::string key;
  uint32_t grab;
  int grid, cpw;
  while (f >> key >> grab >> grid >> cpw)
    if (grab >= 1 && grab <= 64 && grid >= 1 && (cpw == 16 || cpw == 32)) m[key] = Choice{grab, grid, cpw};
  return m;
}

// CUDA events that are destroyed on every way out of the autotuner.
struct EventPair {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ~EventPair() {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  }
};

// Time (tile shape, tiles per steal, grid) candidates for each group's test launch; keep the fastest.
int autotune(gss_batch* b) {
  int rc;
  const char* cache_path = getenv("GSS_AUTOTUNE_CACHE");
  std::map<std::string, Choice> cache;
  if (cache_path && *cache_path) {
    std::lock_guard<std::mutex> lk(g_cache_mutex);
    cache = read_cache(cache_path);
  }
  bool all_cached = !cache.empty();
  for (const Group& g : b->groups) all_cached = all_cached && cache.count(cache_key(b, g)) > 0;
  if (all_cached) {  // earlier runs tuned every group of this shape
    for (Group& g : b->groups) {
      const Choice& v = cache[cache_key(b, g)];
      g.shape = v.cpw == 16 ? 1 : 0;
      g.grab = v.grab;
      g.grid = v.grid < g.full_grid[g.shape] ? v.grid : g.full_grid[g.shape];
    }
    b->tuned_us = 0.f;
    b->tuned = true;
    return GSS_OK;
  }
  if ((rc = enqueue_resets(b, b->stream)) || (rc = enqueue_packs(b))) return rc;
  EventPair ev;
  BCK(b, cudaEventCreate(&ev.e0));
  BCK(b, cudaEventCreate(&ev.e1));
  float total = 0.f;
  for (Group& g : b->groups) {
    float best = 1e30f;
    uint32_t best_grab = 4;
    int best_grid = g.full_grid[0], best_shape = 0;
    for (int k = 0; k < SHAPES; ++k) {
      const int full = g.full_grid[k];
      const uint32_t grabs[] = {1, 2, 4, 8, 16};
      const int grids[] = {full, full / 2 > 0 ? full / 2 : 1};
      for (int gd : grids)
        for (uint32_t gr : grabs) {
          float ms_min = 1e30f;
          for (int rep = 0; rep < 3; ++rep) {
            BCK(b, launch_batch_reset(g.d_inst[k], (uint32_t)g.members.size(), g.work, b->bst, b->stream));
            BCK(b, cudaEventRecord(ev.e0, b->stream));
            BCK(b, launch_test_batch((int)b->mode, g.awp, shape_cpw(k), g.d_inst[k], (uint32_t)g.members.size(),
                                     g.n_tiles[k], g.work, gr, b->bst, gd, b->stream));
            BCK(b, cudaEventRecord(ev.e1, b->stream));
            BCK(b, cudaEventSynchronize(ev.e1));
            float ms = 0.f;
            BCK(b, cudaEventElapsedTime(&ms, ev.e0, ev.e1));
            if (ms < ms_min) ms_min = ms;
          }
          if (ms_min < best) {
            best = ms_min;
            best_grab = gr;
            best_grid = gd;
            best_shape = k;
          }
        }
    }
    g.shape = best_shape;
    g.grab = best_grab;
    g.grid = best_grid;
    total += best;
  }
  b->tuned_us = total * 1e3f;
  b->tuned = true;
  if (cache_path && *cache_path) {  // append this batch's choices (a later line wins on reading)
    std::lock_guard<std::mutex> lk(g_cache_mutex);
    std::ofstream f(cache_path, std::ios::app);
    for (const Group& g : b->groups)
      f << cache_key(b, g) << ' ' << g.grab << ' ' << g.grid << ' ' << shape_cpw(g.shape) << '\n';
  }
  return GSS_OK;
}

int capture(gss_batch* b) {
  drop_graph(b);
  BCK(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
  int rc = enqueue_resets(b, b->stream);
  if (!rc) rc = enqueue_packs(b);
  if (!rc) rc = enqueue_tests(b, b->stream);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(b->stream, &g);
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return bfail(b, GSS_E_CUDA, "graph capture: %s", cudaGetErrorString(e));
  b->graph = g;
  BCK(b, cudaGraphInstantiate(&b->exec, b->graph, 0));
  b->captured.clear();
  for (gss_ctx* c : b->inst) b->captured.push_back(Captured{c->pack_src, c->pack_pitch, c->N, c->Wp});
  b->dirty = false;
  return GSS_OK;
}

bool still_captured(gss_batch* b, uint32_t i) {
  if (b->dirty || i >= b->captured.size()) return false;
  const gss_ctx* c = b->inst[i];
  const Captured& k = b->captured[i];
  return k.src == c->pack_src && k.pitch == c->pack_pitch && k.N == c->N && k.Wp == c->Wp;
}

gss_ctx* instance(gss_batch* b, uint32_t i) { return i < b->inst.size() ? b->inst[i] : nullptr; }

}  // namespace

extern "C" {

int gss_batch_create(gss_batch** out, const gss_config* cfg_in) {
  if (!out) return GSS_E_INVAL;
  *out = nullptr;
  gss_config cfg;
  if (cfg_in) cfg = *cfg_in; else gss_config_init(&cfg);
  if (cfg.mode != GSS_MODE_ALLF && cfg.mode != GSS_MODE_TRIGGER) return GSS_E_INVAL;
  if (cfg.layout != GSS_LAYOUT_IDENTITY && cfg.layout != GSS_LAYOUT_FREQUENCY) return GSS_E_INVAL;
  int n_dev = 0;
  if (cudaGetDeviceCount(&n_dev) != cudaSuccess || cfg.device < 0 || cfg.device >= n_dev) {
    cudaGetLastError();
    return GSS_E_CUDA;
  }
  gss_batch* b = new (std::nothrow) gss_batch();
  if (!b) return GSS_E_NOMEM;
  Guard gd(cfg.device);
  b->device = cfg.device;
  b->mode = cfg.mode;
  b->layout = cfg.layout;
  if (cudaDeviceGetAttribute(&b->n_sms, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess) b->n_sms = 1;
  bool ok = true;
  if (cfg.stream) {
    b->stream = static_cast<cudaStream_t>(cfg.stream);
  } else {
    ok = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) == cudaSuccess;
    b->own_stream = ok;
  }
  for (int k = 0; ok && k < SIDE_STREAMS; ++k) {
    ok = cudaStreamCreateWithFlags(&b->side[k], cudaStreamNonBlocking) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&b->join[k], cudaEventDisableTiming) == cudaSuccess;
  }
  ok = ok && cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess;
  ok = ok && cudaMalloc(&b->bst, sizeof(DevStatus)) == cudaSuccess;
  ok = ok && cudaMallocHost(&b->h_bst, sizeof(DevStatus)) == cudaSuccess;
  ok = ok && cudaMemset(b->bst, 0, sizeof(DevStatus)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    gss_batch_destroy(b);
    return GSS_E_CUDA;
  }
  *out = b;
  return GSS_OK;
}

int gss_batch_destroy(gss_batch* b) {
  if (!b) return GSS_OK;
  Guard gd(b->device);
  if (b->stream) cudaStreamSynchronize(b->stream);
  drop_graph(b);
  drop_groups(b);
  for (gss_ctx* c : b->inst) gss_destroy(c);
  for (int k = 0; k < SIDE_STREAMS; ++k) {
    if (b->side[k]) cudaStreamDestroy(b->side[k]);
    if (b->join[k]) cudaEventDestroy(b->join[k]);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->bst) cudaFree(b->bst);
  if (b->h_bst) cudaFreeHost(b->h_bst);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
  return GSS_OK;
}

int gss_batch_add_instance(gss_batch* b, uint32_t n_vars, uint32_t max_assignments, uint64_t report_capacity,
                           const uint64_t* offsets, uint64_t n_clauses, const uint32_t* lits, uint32_t* instance_id) {
  if (!b) return GSS_E_INVAL;
  b->err.clear();
  gss_config cfg;
  gss_config_init(&cfg);
  cfg.device = b->device;
  cfg.stream = b->stream;
  cfg.mode = b->mode;
  cfg.layout = b->layout;
  if (max_assignments) cfg.max_assignments = max_assignments;
  if (cfg.max_assignments > GSS_MAX_NARROW_ASSIGNMENTS)  // the batched kernel has no second aggregate level
    return bfail(b, GSS_E_INVAL, "max_assignments %u > %u for a batch instance", max_assignments,
                 GSS_MAX_NARROW_ASSIGNMENTS);
  if (report_capacity) cfg.report_capacity = report_capacity;
  gss_ctx* c = nullptr;
  int rc = gss_create(&c, n_vars, &cfg);
  if (rc) return bfail(b, rc, "instance creation failed (n_vars %u, max_assignments %u)", n_vars, max_assignments);
  rc = gss_add_clauses(c, offsets, n_clauses, lits, nullptr);
  if (rc) {
    bfail(b, rc, "%s", gss_last_error(c));
    gss_destroy(c);
    return rc;
  }
  if (instance_id) *instance_id = (uint32_t)b->inst.size();
  b->inst.push_back(c);
  b->dirty = true;
  return GSS_OK;
}

int gss_batch_set_assignments(gss_batch* b, uint32_t i, const uint8_t* values, uint32_t n_assign) {
  if (!b) return GSS_E_INVAL;
  gss_ctx* c = instance(b, i);
  if (!c) return bfail(b, GSS_E_INVAL, "no instance %u", i);
  Guard gd(b->device);
  int rc = stage_assignments(c, values, 0, n_assign, false);
  if (rc) return child_fail(b, c, rc);
  if (!still_captured(b, i)) b->dirty = true;
  return GSS_OK;
}

int gss_batch_set_assignments_device(gss_batch* b, uint32_t i, const uint8_t* d_values, uint64_t pitch,
                                     uint32_t n_assign) {
  if (!b) return GSS_E_INVAL;
  gss_ctx* c = instance(b, i);
  if (!c) return bfail(b, GSS_E_INVAL, "no instance %u", i);
  Guard gd(b->device);
  int rc = stage_assignments(c, d_values, pitch, n_assign, true);
  if (rc) return child_fail(b, c, rc);
  if (!still_captured(b, i)) b->dirty = true;
  return GSS_OK;
}

int gss_batch_test(gss_batch* b) {
  TraceRange tr("gss_batch_test");
  if (!b) return GSS_E_INVAL;
  b->err.clear();
  if (b->inst.empty()) return bfail(b, GSS_E_STATE, "the batch has no instances");
  Guard gd(b->device);
  int rc;
  if (b->dirty) {
    if ((rc = build_groups(b))) return rc;
    if (!b->tuned && (rc = autotune(b))) return rc;
    if ((rc = capture(b))) return rc;
  }
  BCK(b, cudaGraphLaunch(b->exec, b->stream));
  for (gss_ctx* c : b->inst) {
    c->tested = true;
    c->tests_run += 1;
    c->pair_tests += c->m * (uint64_t)c->N;
  }
  b->runs += 1;
  return GSS_OK;
}

int gss_batch_report_count(gss_batch* b, uint32_t i, uint64_t* n_out) {
  if (!b || !n_out) return GSS_E_INVAL;
  gss_ctx* c = instance(b, i);
  if (!c) return bfail(b, GSS_E_INVAL, "no instance %u", i);
  Guard gd(b->device);
  BCK(b, cudaMemcpyAsync(b->h_bst, b->bst, sizeof(DevStatus), cudaMemcpyDeviceToHost, b->stream));
  BCK(b, cudaStreamSynchronize(b->stream));
  if (b->h_bst->timeout) return bfail(b, GSS_E_TIMEOUT, "a bounded device wait gave up during the batched test");
  int rc = gss_report_count(c, n_out);
  return rc ? child_fail(b, c, rc) : GSS_OK;
}

int gss_batch_fetch_reports(gss_batch* b, uint32_t i, gss_report* out, uint64_t cap, uint64_t* n_out) {
  if (!b) return GSS_E_INVAL;
  gss_ctx* c = instance(b, i);
  if (!c) return bfail(b, GSS_E_INVAL, "no instance %u", i);
  Guard gd(b->device);
  BCK(b, cudaMemcpyAsync(b->h_bst, b->bst, sizeof(DevStatus), cudaMemcpyDeviceToHost, b->stream));
  BCK(b, cudaStreamSynchronize(b->stream));
  if (b->h_bst->timeout) return bfail(b, GSS_E_TIMEOUT, "a bounded device wait gave up during the batched test");
  int rc = gss_fetch_reports(c, out, cap, n_out);
  return rc ? child_fail(b, c, rc) : GSS_OK;
}

int gss_batch_get_info(const gss_batch* b, gss_batch_info* out) {
  if (!b || !out) return GSS_E_INVAL;
  memset(out, 0, sizeof *out);
  out->n_instances = (uint32_t)b->inst.size();
  out->runs = b->runs;
  out->tuned_test_us = b->tuned_us;
  uint32_t k = 0;
  for (const Group& g : b->groups) {
    if (k >= 3) break;
    out->tiles_per_steal[k] = g.grab;
    out->grid[k] = (uint32_t)g.grid;
    out->clauses_per_tile[k] = (uint32_t)shape_cpw(g.shape);
    out->n_tiles[k] = g.n_tiles[g.shape];
    ++k;
  }
  out->n_groups = k;
  return GSS_OK;
}

const char* gss_batch_last_error(const gss_batch* b) { return b ? b->err.c_str() : "no batch"; }

}  // extern "C"
