/*
 * gss_oracle.c -- TEST INFRASTRUCTURE ONLY (the oracle).
 *
 * A plain, slow, obviously correct CPU statement of what the clause tests
 * compute, written from the paper's definitions.  Only the tests, the smoke
 * check and the benchmark's CPU-baseline leg may load this library; the
 * product path never does.  It shares no code, header or helper with the CUDA
 * library: it reads the generator's arrays (offsets, literals, value codes)
 * and nothing else.
 *
 * Definitions followed (Section 3.1, Preliminaries):
 *   truth values {T, F, U}; negation: not T = F, not F = T, not U = U;
 *   A(l) = A(v) if l = v, and A(l) = not A(v) if l = not v.
 * Encodings: value codes 0 = U, 1 = T, 2 = F, row-major codes[a * V + v];
 * literal l = 2v + s, s = 1 meaning "not v".
 *
 * Tests (one clause C of size s, one assignment A):
 *   ALLF    every literal of C is F under A: C "would have been in conflict"
 *           (Section 3.3), the allFalse output of Listing assignmentTrigger.
 *   TRIGGER Definition "triggers" (Section 3.3): no literal is T and at least
 *           s - 1 literals are F.
 * Aggregates (Section 4.2): for a group of assignments, G(v) is the set of
 * values the group gives v, and G(l) = G(v) or not G(v).  Aggregate all-F:
 * F is in G(l) for every literal; aggregate trigger (Definition in Section
 * 4.2): F or U is in G(l) for every literal, and F is in G(l) for at least
 * s - 1 literals.
 *
 * Parity pinning: every entry point is pinned by the CPU tests (worked
 * examples of Sections 3.3 and 4.2, brute force over all 3^V assignments with
 * closed-form counts, the aggregate tests of both modes against their set
 * definitions over every small group of assignments, invariants, a recount in
 * another loop order, and the Theorem of Section 4.2 as a property).  ORACLE_MUTANT builds deliberately
 * wrong variants that those pins must reject.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

enum { VAL_U = 0, VAL_T = 1, VAL_F = 2 };
enum { MODE_ALLF = 0, MODE_TRIGGER = 1 };

#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif

/* Section 3.1: negation of a truth value. */
static uint8_t negate(uint8_t w) {
  if (w == VAL_T) return VAL_F;
  if (w == VAL_F) return VAL_T;
  return VAL_U;
}

/* Section 3.1: A(l) for l = 2v + s. */
static uint8_t literal_value(const uint8_t* A, uint32_t l) {
  uint32_t v = l >> 1, negated = l & 1u;
#if ORACLE_MUTANT == 1 /* wrong sign convention */
  negated = !negated;
#endif
  return negated ? negate(A[v]) : A[v];
}

/* Section 3.3: a clause every literal of which is F under A would have been the conflicting clause. */
static int clause_all_false(const uint32_t* lits, uint64_t b, uint64_t e, const uint8_t* A) {
#if ORACLE_MUTANT == 2 /* drops the last literal */
  if (e > b) --e;
#endif
#if ORACLE_MUTANT == 4 /* skips the first literal */
  ++b;
#endif
#if ORACLE_MUTANT == 5 /* exists instead of for-all */
  for (uint64_t k = b; k < e; ++k) if (literal_value(A, lits[k]) == VAL_F) return 1;
  return 0;
#endif
  for (uint64_t k = b; k < e; ++k) {
#if ORACLE_MUTANT == 3 /* treats U as F */
    if (literal_value(A, lits[k]) == VAL_T) return 0;
#else
    if (literal_value(A, lits[k]) != VAL_F) return 0;
#endif
  }
  return 1;
}

/* Definition "triggers" (Section 3.3): each literal != T, and at least s - 1 literals == F. */
static int clause_triggers(const uint32_t* lits, uint64_t b, uint64_t e, const uint8_t* A) {
  uint64_t s = e - b, n_false = 0;
  for (uint64_t k = b; k < e; ++k) {
    uint8_t x = literal_value(A, lits[k]);
    if (x == VAL_T) return 0;
    if (x == VAL_F) ++n_false;
  }
#if ORACLE_MUTANT == 6 /* off-by-one threshold */
  return n_false + 2 >= s;
#endif
  return n_false + 1 >= s;
}

static int pair_test(int mode, const uint32_t* lits, uint64_t b, uint64_t e, const uint8_t* A) {
  return mode == MODE_TRIGGER ? clause_triggers(lits, b, e, A) : clause_all_false(lits, b, e, A);
}

/* One pair: 1 if clause c passes the test under assignment row A (V codes), else 0. */
int gss_oracle_pair(int mode, const uint64_t* off, const uint32_t* lits, uint64_t c, const uint8_t* A) {
  return pair_test(mode, lits, off[c], off[c + 1], A);
}

/* ------------------------------------------------------------ all pairs */
typedef struct {
  int mode; uint64_t m; const uint64_t* off; const uint32_t* lits; uint32_t V; const uint8_t* codes;
  uint64_t a_lo, a_hi;
  uint32_t *pc, *pa; uint64_t n, cap;   /* this worker's hits, (a, c) order */
} worker;

static void push(worker* w, uint32_t c, uint32_t a) {
  if (w->n == w->cap) {
    w->cap = w->cap ? 2 * w->cap : 1024;
    w->pc = (uint32_t*)realloc(w->pc, sizeof(uint32_t) * w->cap);
    w->pa = (uint32_t*)realloc(w->pa, sizeof(uint32_t) * w->cap);
  }
  w->pc[w->n] = c; w->pa[w->n] = a; ++w->n;
}

/* The definition, written out: for every assignment a, for every clause c, test the pair. */
static void* worker_main(void* p) {
  worker* w = (worker*)p;
  for (uint64_t a = w->a_lo; a < w->a_hi; ++a) {
    const uint8_t* A = w->codes + a * (uint64_t)w->V;
    for (uint64_t c = 0; c < w->m; ++c)
      if (pair_test(w->mode, w->lits, w->off[c], w->off[c + 1], A)) push(w, (uint32_t)c, (uint32_t)a);
  }
  return 0;
}

/*
 * Every (clause, assignment) pair with a_lo <= a < a_hi that passes `mode`.
 * Results are malloc'd into *out_c / *out_a (release with gss_oracle_free),
 * ordered by assignment, then clause.  Returns the number of pairs, or -1.
 */
int64_t gss_oracle_pairs(int mode, uint64_t m, const uint64_t* off, const uint32_t* lits, uint32_t V,
                         const uint8_t* codes, uint64_t a_lo, uint64_t a_hi, int threads,
                         uint32_t** out_c, uint32_t** out_a) {
  if (a_hi < a_lo) return -1;
  uint64_t n_a = a_hi - a_lo;
  if (threads < 1) threads = 1;
  if ((uint64_t)threads > n_a) threads = n_a ? (int)n_a : 1;
  worker* ws = (worker*)calloc(threads, sizeof(worker));
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * threads);
  for (int t = 0; t < threads; ++t) {
    worker* w = &ws[t];
    w->mode = mode; w->m = m; w->off = off; w->lits = lits; w->V = V; w->codes = codes;
    w->a_lo = a_lo + n_a * (uint64_t)t / threads; w->a_hi = a_lo + n_a * (uint64_t)(t + 1) / threads;
    pthread_create(&th[t], 0, worker_main, w);
  }
  uint64_t total = 0;
  for (int t = 0; t < threads; ++t) { pthread_join(th[t], 0); total += ws[t].n; }
  uint32_t* rc = (uint32_t*)malloc(sizeof(uint32_t) * (total ? total : 1));
  uint32_t* ra = (uint32_t*)malloc(sizeof(uint32_t) * (total ? total : 1));
  uint64_t k = 0;
  for (int t = 0; t < threads; ++t) {
    if (ws[t].n) {
      memcpy(rc + k, ws[t].pc, sizeof(uint32_t) * ws[t].n);
      memcpy(ra + k, ws[t].pa, sizeof(uint32_t) * ws[t].n);
    }
    k += ws[t].n;
    free(ws[t].pc); free(ws[t].pa);
  }
  free(ws); free(th);
  *out_c = rc; *out_a = ra;
  return (int64_t)total;
}

void gss_oracle_free(void* p) { free(p); }

/* ------------------------------------------------------------ aggregates */
/*
 * Section 4.2: the aggregate of assignments a in [g*group, min((g+1)*group, N))
 * maps v to the set {A_a(v)}, stored as three booleans (T in set, F in set,
 * U in set) packed as bits 1, 2, 4.  agg[g * V + v] receives that byte.
 */
void gss_oracle_aggregate(uint32_t V, uint32_t N, const uint8_t* codes, uint32_t group, uint8_t* agg) {
  uint32_t G = (N + group - 1) / group;
  for (uint32_t g = 0; g < G; ++g)
    for (uint32_t v = 0; v < V; ++v) {
      uint8_t set = 0;
      for (uint32_t a = g * group; a < N && a < (g + 1) * group; ++a) {
        uint8_t x = codes[(uint64_t)a * V + v];
        set |= (uint8_t)(x == VAL_T ? 1 : x == VAL_F ? 2 : 4);
      }
      agg[(uint64_t)g * V + v] = set;
    }
}

/* Section 4.2: G(l) = G(v) for l = v, and not G(v) = {not w : w in G(v)} for l = not v. */
static uint8_t aggregate_literal(const uint8_t* Gv, uint32_t l) {
  uint8_t set = Gv[l >> 1];
  if (!(l & 1u)) return set;
  uint8_t out = 0;
  if (set & 1) out |= 2;  /* T -> F */
  if (set & 2) out |= 1;  /* F -> T */
  if (set & 4) out |= 4;  /* U -> U */
  return out;
}

/*
 * Aggregate test of clause c against one aggregate assignment Gv (V bytes as
 * above).  ALLF: F in G(l) for every literal.  TRIGGER (Definition in Section
 * 4.2): F or U in G(l) for every literal, and F in G(l) for at least s - 1.
 */
int gss_oracle_aggregate_test(int mode, const uint64_t* off, const uint32_t* lits, uint64_t c, const uint8_t* Gv) {
  uint64_t b = off[c], e = off[c + 1], s = e - b, n_f = 0;
  for (uint64_t k = b; k < e; ++k) {
    uint8_t g = aggregate_literal(Gv, lits[k]);
    if (mode == MODE_ALLF) {
#if ORACLE_MUTANT == 7 /* F or U in G(l) taken for F in G(l) */
      if (!(g & 6)) return 0;
#else
      if (!(g & 2)) return 0;
#endif
    } else {
      if (!(g & 6)) return 0;
      if (g & 2) ++n_f;
    }
  }
#if ORACLE_MUTANT == 8 /* aggregate trigger threshold off by one */
  return mode == MODE_ALLF ? 1 : (n_f + 2 >= s);
#endif
  return mode == MODE_ALLF ? 1 : (n_f + 1 >= s);
}
