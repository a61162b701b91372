/*
 * gss_synth.c -- seeded synthetic inputs for the clause x assignment test.
 *
 * This file draws random clause databases and three-valued assignments.  It
 * holds none of the tested method's arithmetic: it never evaluates a literal
 * against an assignment except in synth_plant(), which FORCES chosen literals
 * to F (writes codes) so that known hits exist.  Both the CUDA path and the
 * oracle consume its output arrays; neither is linked against the other.
 *
 * Workload shapes (clause sizes, variable popularity, trail-correlated
 * assignments) follow the statistics the paper reports: learned clauses are
 * often 20+ literals long (Section 5), up to 1024 assignments arrive in groups
 * of 32 from one solver thread (Section 4.3), and successive assignments of a
 * thread share most of their values (Section 4.1, commonality table).
 *
 * Determinism: every random stream is seeded from (seed, index) with
 * splitmix64, so the output does not depend on the thread count.  The only
 * transcendental functions used (log, exp) are computed here from IEEE basic
 * operations (build with -ffp-contract=off), so x86_64 and aarch64 hosts
 * produce identical bytes.
 *
 * Value codes: 0 = U, 1 = T, 2 = F.  Literal encoding: l = 2v + s, s = 1 is
 * the negated literal.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define CODE_U 0
#define CODE_T 1
#define CODE_F 2

/* ------------------------------------------------------------------ RNG */
static inline uint64_t mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

typedef struct { uint64_t s[4]; } xo256;

static void xo_seed(xo256* r, uint64_t seed) {
  uint64_t t = seed;
  for (int i = 0; i < 4; ++i) { t = mix64(t); r->s[i] = t; }
}
static inline uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }
static inline uint64_t xo_next(xo256* r) {  /* xoshiro256** (Blackman & Vigna) */
  uint64_t* s = r->s;
  uint64_t out = rotl64(s[1] * 5, 7) * 9;
  uint64_t t = s[1] << 17;
  s[2] ^= s[0]; s[3] ^= s[1]; s[1] ^= s[2]; s[0] ^= s[3];
  s[2] ^= t; s[3] = rotl64(s[3], 45);
  return out;
}
static inline double xo_unif(xo256* r) { return (double)(xo_next(r) >> 11) * (1.0 / 9007199254740992.0); }
/* uniform integer in [0, n) without bias (Lemire's multiply-shift with rejection) */
static inline uint64_t xo_below(xo256* r, uint64_t n) {
  uint64_t x = xo_next(r);
  __uint128_t m = (__uint128_t)x * n;
  uint64_t lo = (uint64_t)m;
  if (lo < n) {
    uint64_t t = (0 - n) % n;
    while (lo < t) { x = xo_next(r); m = (__uint128_t)x * n; lo = (uint64_t)m; }
  }
  return (uint64_t)(m >> 64);
}
static inline uint64_t stream_seed(uint64_t seed, uint64_t tag, uint64_t idx) {
  return mix64(mix64(seed ^ (tag * 0xD1B54A32D192ED03ULL)) + idx);
}

/* ---------------------------------------- deterministic log / exp (IEEE ops only) */
static const double LN2 = 0.69314718055994530942;
static double det_log(double x) {  /* x > 0, finite */
  int e = 0;
  /* scale into [sqrt(1/2), sqrt(2)) by exact powers of two */
  while (x >= 1.4142135623730951) { x *= 0.5; ++e; }
  while (x < 0.7071067811865476) { x *= 2.0; --e; }
  double t = (x - 1.0) / (x + 1.0), t2 = t * t, term = t, sum = 0.0;
  for (int k = 1; k <= 41; k += 2) { sum += term / (double)k; term *= t2; }
  return 2.0 * sum + (double)e * LN2;
}
static double det_exp(double x) {
  double kd = x / LN2;
  long k = (long)(kd >= 0 ? kd + 0.5 : kd - 0.5);
  double r = x - (double)k * LN2, term = 1.0, sum = 1.0;
  for (int i = 1; i <= 24; ++i) { term *= r / (double)i; sum += term; }
  while (k > 0) { sum *= 2.0; --k; }
  while (k < 0) { sum *= 0.5; ++k; }
  return sum;
}
static double det_sqrt(double x) {  /* Newton on IEEE ops; x >= 0 */
  if (x <= 0) return 0.0;
  double y = x > 1 ? x : 1.0;
  for (int i = 0; i < 200; ++i) {
    double ny = 0.5 * (y + x / y);
    if (ny >= y) break;
    y = ny;
  }
  return y;
}
static double xo_normal(xo256* r) {  /* Marsaglia polar method */
  for (;;) {
    double u = 2.0 * xo_unif(r) - 1.0, v = 2.0 * xo_unif(r) - 1.0, s = u * u + v * v;
    if (s > 0.0 && s < 1.0) return u * det_sqrt(-2.0 * det_log(s) / s);
  }
}

/* ------------------------------------------------------------ thread pool */
typedef void (*range_fn)(void* ctx, uint64_t lo, uint64_t hi);
typedef struct { range_fn fn; void* ctx; uint64_t lo, hi; } range_job;
static void* range_trampoline(void* p) { range_job* j = (range_job*)p; j->fn(j->ctx, j->lo, j->hi); return 0; }
static void parallel_for(uint64_t n, int threads, range_fn fn, void* ctx) {
  if (threads < 1) threads = 1;
  if ((uint64_t)threads > n) threads = n ? (int)n : 1;
  if (threads == 1) { fn(ctx, 0, n); return; }
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * threads);
  range_job* jobs = (range_job*)malloc(sizeof(range_job) * threads);
  for (int t = 0; t < threads; ++t) {
    jobs[t].fn = fn; jobs[t].ctx = ctx;
    jobs[t].lo = n * (uint64_t)t / threads; jobs[t].hi = n * (uint64_t)(t + 1) / threads;
    pthread_create(&th[t], 0, range_trampoline, &jobs[t]);
  }
  for (int t = 0; t < threads; ++t) pthread_join(th[t], 0);
  free(th); free(jobs);
}

/* ------------------------------------------------------------ clause sizes */
typedef struct { int law; double p1, p2; uint32_t cap, max_distinct; uint64_t seed; uint32_t* sizes; } sizes_ctx;
static void sizes_range(void* p, uint64_t lo, uint64_t hi) {
  sizes_ctx* c = (sizes_ctx*)p;
  double mu = c->law == 1 ? det_log(c->p1) : 0.0;
  /* geometric success threshold: success iff 64-bit draw < p * 2^64 */
  uint64_t thresh = (uint64_t)(c->p1 * 18446744073709551616.0 >= 18446744073709551615.0 ? 18446744073709551615.0
                                                                                       : c->p1 * 18446744073709551616.0);
  for (uint64_t i = lo; i < hi; ++i) {
    xo256 r; xo_seed(&r, stream_seed(c->seed, 1, i));
    uint32_t s;
    if (c->law == 0) {           /* 2 + Geom(p), redrawn while above cap */
      for (;;) {
        uint32_t g = 0;
        while (xo_next(&r) >= thresh && g < 100000) ++g;
        s = 2 + g;
        if (s <= c->cap) break;
      }
    } else {                     /* clamp(round(exp(mu + sigma Z)), 2, cap) */
      double x = det_exp(mu + c->p2 * xo_normal(&r));
      double rx = x + 0.5;
      s = rx >= (double)c->cap ? c->cap : (uint32_t)rx;
      if (s < 2) s = 2;
      if (s > c->cap) s = c->cap;
    }
    if (s > c->max_distinct) s = c->max_distinct;
    c->sizes[i] = s;
  }
}
/* law 0: geometric(p1), law 1: lognormal(median p1, sigma p2).  Returns 0. */
int synth_sizes(uint64_t m, int law, double p1, double p2, uint32_t cap, uint32_t max_distinct,
                uint64_t seed, int threads, uint32_t* sizes) {
  sizes_ctx c = {law, p1, p2, cap, max_distinct, seed, sizes};
  parallel_for(m, threads, sizes_range, &c);
  return 0;
}

/* ------------------------------------------------------------ Zipf sampler */
typedef struct {
  uint32_t n;        /* ranks 0..n-1 (rank r has weight (r+1)^-s) */
  double* cdf;       /* inclusive prefix sums */
  uint32_t* perm;    /* rank -> id */
  uint32_t* guide;   /* guide[k] = first rank whose cdf exceeds k*total/G */
  uint32_t gn;
  double total;
} zipf_t;

static void zipf_init(zipf_t* z, uint32_t n, double s, uint64_t seed, int permute) {
  z->n = n;
  z->cdf = (double*)malloc(sizeof(double) * (n ? n : 1));
  double acc = 0.0;
  for (uint32_t r = 0; r < n; ++r) { acc += det_exp(-s * det_log((double)r + 1.0)); z->cdf[r] = acc; }
  z->total = acc;
  z->perm = (uint32_t*)malloc(sizeof(uint32_t) * (n ? n : 1));
  for (uint32_t r = 0; r < n; ++r) z->perm[r] = r;
  if (permute) {
    xo256 rg; xo_seed(&rg, stream_seed(seed, 2, 0));
    for (uint32_t i = n; i > 1; --i) {
      uint32_t j = (uint32_t)xo_below(&rg, i);
      uint32_t t = z->perm[i - 1]; z->perm[i - 1] = z->perm[j]; z->perm[j] = t;
    }
  }
  z->gn = n < 65536 ? (n ? n : 1) : 65536;
  z->guide = (uint32_t*)malloc(sizeof(uint32_t) * (z->gn + 1));
  uint32_t r = 0;
  for (uint32_t k = 0; k <= z->gn; ++k) {
    double thr = z->total * (double)k / (double)z->gn;
    while (r + 1 < n && z->cdf[r] <= thr) ++r;
    z->guide[k] = r;
  }
}
static void zipf_free(zipf_t* z) { free(z->cdf); free(z->perm); free(z->guide); }
static inline uint32_t zipf_draw(const zipf_t* z, xo256* r) {
  double u = xo_unif(r) * z->total;
  uint32_t k = (uint32_t)(u / z->total * (double)z->gn);
  if (k >= z->gn) k = z->gn - 1;
  /* the answer lies in [guide[k], guide[k+1]]; widen if rounding put u just outside */
  uint32_t lo = z->guide[k], hi = z->guide[k + 1];
  if (lo > 0 && z->cdf[lo - 1] > u) lo = 0;
  if (z->cdf[hi] <= u) hi = z->n - 1;
  /* smallest rank with cdf > u in [lo, hi] (hi if none) */
  while (lo < hi) {
    uint32_t mid = lo + (hi - lo) / 2;
    if (z->cdf[mid] > u) hi = mid; else lo = mid + 1;
  }
  return z->perm[lo];
}

/* --------------------------------------------------------- clause literals */
typedef struct {
  const uint64_t* off; uint32_t V; uint64_t seed;
  const zipf_t* zv;              /* global variable popularity */
  uint32_t n_comm, comm_size;    /* communities: community k = vars [k*size, (k+1)*size) */
  const zipf_t* zc;              /* community popularity (home draw) */
  double p_home;
  uint32_t table_bits;
  uint32_t* lits;
} lits_ctx;

static void lits_range(void* p, uint64_t lo, uint64_t hi) {
  lits_ctx* c = (lits_ctx*)p;
  uint32_t tsize = 1u << c->table_bits, tmask = tsize - 1;
  uint32_t* key = (uint32_t*)malloc(sizeof(uint32_t) * tsize);
  uint32_t* stamp = (uint32_t*)calloc(tsize, sizeof(uint32_t));
  uint32_t cur = 0;
  uint64_t p_home_thr = (uint64_t)(c->p_home * 9007199254740992.0);
  for (uint64_t i = lo; i < hi; ++i) {
    xo256 r; xo_seed(&r, stream_seed(c->seed, 3, i));
    if (++cur == 0) { memset(stamp, 0, sizeof(uint32_t) * tsize); cur = 1; }
    uint64_t b = c->off[i], e = c->off[i + 1];
    uint32_t home = c->n_comm ? zipf_draw(c->zc, &r) : 0;
    for (uint64_t k = b; k < e; ++k) {
      for (;;) {  /* draw until the literal is new to this clause (exact duplicates redrawn) */
        uint32_t v;
        if (c->n_comm && (xo_next(&r) >> 11) < p_home_thr) v = home * c->comm_size + (uint32_t)xo_below(&r, c->comm_size);
        else v = zipf_draw(c->zv, &r);
        uint32_t l = 2u * v + (uint32_t)(xo_next(&r) >> 63);
        uint32_t h = (uint32_t)(mix64(l) & tmask);
        int dup = 0;
        while (stamp[h] == cur) { if (key[h] == l) { dup = 1; break; } h = (h + 1) & tmask; }
        if (dup) continue;
        stamp[h] = cur; key[h] = l;
        c->lits[k] = l;
        break;
      }
    }
  }
  free(key); free(stamp);
}

/*
 * Fill lits[off[i]..off[i+1]) for every clause i.  Variables follow Zipf(zipf_s)
 * over [0, V) through a seeded rank->id permutation; with n_comm > 0 each
 * clause draws a home community by Zipf(zipf_s) over communities and takes each
 * literal from it (uniformly) with probability p_home.  Signs are fair coins.
 * Caller guarantees off[i+1]-off[i] <= 2V (and <= the community's 2*size when
 * p_home == 1).
 */
int synth_lits(uint64_t m, const uint64_t* off, uint32_t V, double zipf_s, uint32_t n_comm, uint32_t comm_size,
               double p_home, uint32_t max_size, uint64_t seed, int threads, uint32_t* lits) {
  zipf_t zv, zc;
  zipf_init(&zv, V, zipf_s, stream_seed(seed, 4, 0), 1);
  if (n_comm) zipf_init(&zc, n_comm, zipf_s, stream_seed(seed, 5, 0), 1);
  uint32_t bits = 4;
  while ((1u << bits) < 4u * (max_size ? max_size : 1)) ++bits;
  lits_ctx c = {off, V, seed, &zv, n_comm, comm_size, n_comm ? &zc : 0, p_home, bits, lits};
  parallel_for(m, threads, lits_range, &c);
  zipf_free(&zv);
  if (n_comm) zipf_free(&zc);
  return 0;
}

/* ----------------------------------------------- independent assignments */
typedef struct { uint32_t V; double p_set; uint64_t seed; uint8_t* codes; } indep_ctx;
static void indep_range(void* p, uint64_t lo, uint64_t hi) {
  indep_ctx* c = (indep_ctx*)p;
  uint64_t thr = (uint64_t)(c->p_set * 9007199254740992.0);
  for (uint64_t a = lo; a < hi; ++a) {
    xo256 r; xo_seed(&r, stream_seed(c->seed, 6, a));
    uint8_t* row = c->codes + a * (uint64_t)c->V;
    for (uint32_t v = 0; v < c->V; ++v) {
      uint64_t x = xo_next(&r);
      row[v] = (x >> 11) < thr ? (uint8_t)((x & 1) ? CODE_T : CODE_F) : (uint8_t)CODE_U;
    }
  }
}
/* Each variable of each assignment is set with probability p_set, then T or F with 1/2 each. */
int synth_assign_indep(uint32_t V, uint32_t N, double p_set, uint64_t seed, int threads, uint8_t* codes) {
  indep_ctx c = {V, p_set, seed, codes};
  parallel_for(N, threads, indep_range, &c);
  return 0;
}

/* ------------------------------------------- trail-prefix correlated assignments */
typedef struct { uint32_t V, N, group; double lo, hi, flip_frac; uint64_t seed; uint8_t* codes; } trail_ctx;
static void trail_range(void* p, uint64_t glo, uint64_t ghi) {
  trail_ctx* c = (trail_ctx*)p;
  uint32_t V = c->V;
  uint32_t* perm = (uint32_t*)malloc(sizeof(uint32_t) * (V ? V : 1));
  uint32_t* pos = (uint32_t*)malloc(sizeof(uint32_t) * (V ? V : 1));
  for (uint64_t g = glo; g < ghi; ++g) {
    xo256 r; xo_seed(&r, stream_seed(c->seed, 7, g));
    for (uint32_t v = 0; v < V; ++v) perm[v] = v;
    for (uint32_t i = V; i > 1; --i) {
      uint32_t j = (uint32_t)xo_below(&r, i);
      uint32_t t = perm[i - 1]; perm[i - 1] = perm[j]; perm[j] = t;
    }
    for (uint32_t i = 0; i < V; ++i) pos[perm[i]] = i;   /* trail position of each variable */
    uint64_t pol_seed = stream_seed(c->seed, 8, g);
    uint64_t a_end = (g + 1) * (uint64_t)c->group;
    if (a_end > c->N) a_end = c->N;
    for (uint64_t a = g * (uint64_t)c->group; a < a_end; ++a) {
      xo256 ra; xo_seed(&ra, stream_seed(c->seed, 9, a));
      double f = c->lo + (c->hi - c->lo) * xo_unif(&ra);
      uint32_t k = (uint32_t)(f * (double)V);
      if (k > V) k = V;
      uint32_t k_flip = (uint32_t)((1.0 - c->flip_frac) * (double)k);
      uint64_t flip_seed = stream_seed(c->seed, 10, a);
      uint8_t* row = c->codes + a * (uint64_t)V;
      for (uint32_t v = 0; v < V; ++v) {
        uint32_t q = pos[v];
        if (q >= k) { row[v] = CODE_U; continue; }
        uint32_t phi = (uint32_t)(mix64(pol_seed + v) & 1);          /* group polarity */
        if (q >= k_flip) phi ^= (uint32_t)(mix64(flip_seed + v) & 1); /* re-decided after a backjump */
        row[v] = phi ? CODE_T : CODE_F;
      }
    }
  }
  free(perm); free(pos);
}
/*
 * Assignments 0..N-1 in groups of `group` (one simulated solver thread per
 * group).  Group g owns a random trail (variable order) and polarity; its
 * assignment j assigns the first floor(f_j V) trail variables, f_j ~ U[lo, hi),
 * with the group's polarity, each variable in the last flip_frac of that prefix
 * flipping with probability 1/2.  All other variables are U.
 */
int synth_assign_trail(uint32_t V, uint32_t N, uint32_t group, double lo, double hi, double flip_frac,
                       uint64_t seed, int threads, uint8_t* codes) {
  if (group == 0) return -1;
  trail_ctx c = {V, N, group, lo, hi, flip_frac, seed, codes};
  uint64_t groups = (N + (uint64_t)group - 1) / group;
  parallel_for(groups, threads, trail_range, &c);
  return 0;
}

/* ------------------------------------------------------------- planting */
typedef struct { uint64_t* k; uint8_t* v; uint8_t* used; uint64_t cap, n; } u64map;
static void map_init(u64map* m, uint64_t cap) {
  uint64_t c = 1024; while (c < cap) c <<= 1;
  m->cap = c; m->n = 0;
  m->k = (uint64_t*)malloc(sizeof(uint64_t) * c); m->v = (uint8_t*)malloc(c); m->used = (uint8_t*)calloc(c, 1);
}
static void map_free(u64map* m) { free(m->k); free(m->v); free(m->used); }
static int map_get(const u64map* m, uint64_t key, uint8_t* out) {
  uint64_t h = mix64(key) & (m->cap - 1);
  while (m->used[h]) { if (m->k[h] == key) { if (out) *out = m->v[h]; return 1; } h = (h + 1) & (m->cap - 1); }
  return 0;
}
static void map_put(u64map* m, uint64_t key, uint8_t val);
static void map_grow(u64map* m) {
  u64map n; map_init(&n, m->cap * 2);
  for (uint64_t i = 0; i < m->cap; ++i) if (m->used[i]) map_put(&n, m->k[i], m->v[i]);
  map_free(m); *m = n;
}
static void map_put(u64map* m, uint64_t key, uint8_t val) {
  if (2 * (m->n + 1) > m->cap) map_grow(m);
  uint64_t h = mix64(key) & (m->cap - 1);
  while (m->used[h]) { if (m->k[h] == key) { m->v[h] = val; return; } h = (h + 1) & (m->cap - 1); }
  m->used[h] = 1; m->k[h] = key; m->v[h] = val; m->n++;
}

static int clause_is_tautology(const uint32_t* lits, uint64_t b, uint64_t e, u64map* scratch) {
  scratch->n = 0; memset(scratch->used, 0, scratch->cap);
  for (uint64_t k = b; k < e; ++k) {
    if (map_get(scratch, lits[k] ^ 1u, 0)) return 1;
    map_put(scratch, lits[k], 1);
  }
  return 0;
}

/*
 * Plant K distinct (clause, assignment) pairs: draw uniformly, skip
 * tautologies, assignments with exclude[a] != 0 and draws whose forcing would
 * contradict a variable already forced for the same assignment; then set every
 * variable of the clause so that each of its literals is F (v = F for l = v,
 * v = T for l = not v).  Returns the number planted (< K only if draws ran out).
 */
int64_t synth_plant(uint64_t m, const uint64_t* off, const uint32_t* lits, uint32_t V, uint32_t N, uint8_t* codes,
                    const uint8_t* exclude, uint64_t K, uint64_t seed, uint32_t* out_c, uint32_t* out_a) {
  if (m == 0 || N == 0) return 0;
  xo256 r; xo_seed(&r, stream_seed(seed, 11, 0));
  u64map forced, pairs, scratch;
  map_init(&forced, 4 * K * 16 + 1024); map_init(&pairs, 4 * K + 1024); map_init(&scratch, 4096);
  uint64_t got = 0, attempts = 0, max_attempts = 1000 * K + 100000;
  while (got < K && attempts < max_attempts) {
    ++attempts;
    uint64_t c = xo_below(&r, m), a = xo_below(&r, N);
    if (exclude && exclude[a]) continue;
    uint64_t pk = (c << 32) | a;
    if (map_get(&pairs, pk, 0)) continue;
    uint64_t b = off[c], e = off[c + 1];
    if (e == b) continue;
    if (e - b > scratch.cap / 4) { map_free(&scratch); map_init(&scratch, 4 * (e - b)); }
    if (clause_is_tautology(lits, b, e, &scratch)) continue;
    int ok = 1;
    for (uint64_t k = b; k < e && ok; ++k) {
      uint32_t v = lits[k] >> 1;
      uint8_t need = (lits[k] & 1u) ? CODE_T : CODE_F, have;
      if (map_get(&forced, (a << 32) | v, &have) && have != need) ok = 0;
    }
    if (!ok) continue;
    for (uint64_t k = b; k < e; ++k) {
      uint32_t v = lits[k] >> 1;
      uint8_t need = (lits[k] & 1u) ? CODE_T : CODE_F;
      codes[a * (uint64_t)V + v] = need;
      map_put(&forced, (a << 32) | v, need);
    }
    map_put(&pairs, pk, 1);
    out_c[got] = (uint32_t)c; out_a[got] = (uint32_t)a;
    ++got;
  }
  map_free(&forced); map_free(&pairs); map_free(&scratch);
  return (int64_t)got;
}

/*
 * Turn `count` distinct, non-tautological clauses of size >= 2 into explicit
 * tautologies by overwriting their last literal with the negation of their
 * first.  Returns the number made; their ids go to out_ids.
 */
int64_t synth_tautologies(uint64_t m, const uint64_t* off, uint32_t* lits, uint64_t count, uint64_t seed,
                          uint32_t* out_ids) {
  xo256 r; xo_seed(&r, stream_seed(seed, 12, 0));
  u64map chosen, scratch;
  map_init(&chosen, 4 * count + 1024); map_init(&scratch, 4096);
  uint64_t got = 0, attempts = 0;
  while (got < count && attempts < 1000 * count + 1000 && m) {
    ++attempts;
    uint64_t c = xo_below(&r, m), b = off[c], e = off[c + 1];
    if (e - b < 2 || map_get(&chosen, c, 0)) continue;
    if (e - b > scratch.cap / 4) { map_free(&scratch); map_init(&scratch, 4 * (e - b)); }
    if (clause_is_tautology(lits, b, e, &scratch)) continue;
    int clash = 0;  /* the negated first literal must not already sit elsewhere (it would then be a duplicate) */
    for (uint64_t k = b + 1; k + 1 < e; ++k) if (lits[k] == (lits[b] ^ 1u)) clash = 1;
    if (clash) continue;
    lits[e - 1] = lits[b] ^ 1u;
    map_put(&chosen, c, 1);
    out_ids[got++] = (uint32_t)c;
  }
  map_free(&chosen); map_free(&scratch);
  return (int64_t)got;
}

/* 64-bit content hash of a byte buffer (blocks hashed in parallel, combined in order). */
typedef struct { const uint8_t* p; uint64_t n, block; uint64_t* out; } hash_ctx;
static void hash_range(void* vp, uint64_t lo, uint64_t hi) {
  hash_ctx* c = (hash_ctx*)vp;
  for (uint64_t b = lo; b < hi; ++b) {
    uint64_t s = b * 0x9E3779B97F4A7C15ULL, e = (b + 1) * c->block;
    if (e > c->n) e = c->n;
    uint64_t i = b * c->block;
    for (; i + 8 <= e; i += 8) { uint64_t w; memcpy(&w, c->p + i, 8); s = mix64(s ^ w); }
    for (; i < e; ++i) s = mix64(s ^ c->p[i]);
    c->out[b] = s;
  }
}
uint64_t synth_hash(const uint8_t* p, uint64_t n, int threads) {
  uint64_t block = 1u << 22, nb = (n + block - 1) / block;
  uint64_t* hs = (uint64_t*)malloc(sizeof(uint64_t) * (nb ? nb : 1));
  hash_ctx c = {p, n, block, hs};
  parallel_for(nb, threads, hash_range, &c);
  uint64_t s = mix64(n);
  for (uint64_t b = 0; b < nb; ++b) s = mix64(s ^ hs[b]);
  free(hs);
  return s;
}
