// k_test.cu -- test every clause against every assignment of the current set.
//
// What is computed (per clause c, per assignment a):
//   GSS_MODE_ALLF     every literal of c is F under a: c "would have been in conflict"
//                     (Section 3.3); the allFalse recurrence of Listing assignmentTrigger
//                     (Section 3.4), allFalse &= isFalse(l), 32 assignments per word.
//   GSS_MODE_TRIGGER  Definition "triggers" (Section 3.3): the full recurrence of Listing
//                     assignmentTrigger, oneUndef = (allFalse & U(l)) | (oneUndef & F(l)),
//                     allFalse &= F(l), result allFalse | oneUndef.
//
// How (Sections 3.5 and 4.3, re-planned for GB300):
//   * one lane per clause, 32 clauses per warp, persistent grid-stride over 32-clause tiles;
//   * the tile's head0 (literals 0..7 of its 32 clauses, 1 KiB) is brought into shared
//     memory by a TMA bulk copy (cp.async.bulk + mbarrier), double-buffered: the copy of
//     the warp's next tile is in flight while the current one is tested;
//   * stage A is Listing multiTrigger's group test: per 32-assignment group one aggregate
//     bit per literal (Section 4.2), ANDed (all-F) or run through the aggregateTrigger
//     recurrence (trigger).  All gathers of a batch of literals are issued before they are
//     combined, so a batch costs one L2 round trip.  Literals 8..15 come from head1 (one
//     sector per clause, no offset lookup, fetched while the first batch is tested) and
//     later ones from the CSR, only while some group is alive.  By the Theorem of Section 4.2 a group whose aggregate test fails
//     holds no hit;
//   * stage B is multiTrigger's inner assignmentTrigger call: the warp's surviving
//     (clause, group) pairs are compacted into shared memory and each lane runs the exact
//     word recurrence of one pair, again with a batch's gathers in flight together;
//   * each non-zero word becomes one record {clause, word, mask} (report(i, mask) of
//     Listing multiTrigger), placed with a ballot and a population count into the warp's
//     outbox in shared memory; a full outbox reserves its space in the output with one
//     atomicAdd and is written out as whole words.  Records past the capacity are counted
//     but not written.
//
// Wide sets (more than 4096 assignments, the aggregate of aggregates that Section 7 proposes):
// stage A runs on level-2 rows (one bit per 1024-assignment super-group), and each surviving
// (clause, super-group) pair first runs the group recurrence on its level-1 word (one bit per
// 32-assignment group of the super-group) before the exact test of each group left.  Both
// aggregate levels are ORs of the level below, so the Theorem of Section 4.2 applies to each.
//
// The PAD literal 2V is neutral in both modes: its P and aggF rows are all ones and its
// aggU row is zero, so padded head slots need no branch.
//
// The internal variable numbering puts the hottest variables first (see k_ingest.cu), so
// the aggregate rows gathered most often share a few cache lines and stay in L1.  (A copy
// of those rows in shared memory was measured: 182 us against 171 us without it on the
// 4M-clause workload, so the L1 serves them better.)
#include <type_traits>

#include "gss_internal.h"
#include "gss_ptx.h"

namespace gss {
namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr int TEST_THREADS = 256;
constexpr int TEST_WARPS = TEST_THREADS / 32;
constexpr uint32_t PAIR_CAP = 64;        // candidate pairs staged per warp per round
constexpr uint32_t OUT_CAP = 64;         // records staged per warp before one reservation

struct __align__(128) WarpSmem {
  uint32_t ring[2][32 * 8];  // head0 of the current and the next tile
  uint32_t pairs[PAIR_CAP];  // owner lane | group << 5
  uint32_t out[3 * OUT_CAP]; // staged records {clause, word, mask}
  unsigned long long bar[2];
};
// Wide sets: pairs holds (clause, super-group) pairs, pairs2 the (clause, group) pairs of a round.
struct __align__(128) WarpSmemWide : WarpSmem {
  uint32_t pairs2[PAIR_CAP];
};

// ------------------------------------------------------------------ math helpers
__device__ __forceinline__ uint32_t valid_bits(uint32_t N, uint32_t w) {
  const uint32_t lo = w * 32u;
  if (lo >= N) return 0u;
  const uint32_t rem = N - lo;
  return rem >= 32u ? FULL : ((1u << rem) - 1u);
}

#ifdef GSS_DEBUG_BOUNDS
__device__ unsigned long long g_bounds_errors;  // rows out of range met by the test kernels
// row if row < rows, else the PAD row (rows - 2 for literal rows, rows - 1 for variable rows) and a count
__device__ __forceinline__ uint32_t checked_row(uint32_t row, uint32_t rows, uint32_t pad_row) {
  if (row < rows) return row;
  atomicAdd(&g_bounds_errors, 1ull);
  return pad_row;
}
#define GSS_ROW(row, rows, pad_row) checked_row((row), (rows), (pad_row))
#else
#define GSS_ROW(row, rows, pad_row) (row)
#endif

template <int AW>
__device__ __forceinline__ void load_agg(const uint32_t* __restrict__ base, uint32_t row, uint32_t (&r)[AW]) {
  if constexpr (AW == 1) {
    r[0] = __ldg(base + row);
  } else if constexpr (AW == 2) {
    const uint2 t = __ldg(reinterpret_cast<const uint2*>(base) + row);
    r[0] = t.x; r[1] = t.y;
  } else {
    const uint4 t = __ldg(reinterpret_cast<const uint4*>(base) + row);
    r[0] = t.x; r[1] = t.y; r[2] = t.z; r[3] = t.w;
  }
}

template <int AW>
__device__ __forceinline__ bool any2(const uint32_t (&a)[AW], const uint32_t (&b)[AW]) {
  uint32_t o = 0;
#pragma unroll
  for (int i = 0; i < AW; ++i) o |= a[i] | b[i];
  return o != 0u;
}

// Stage A on 8 literals: gathers first, then the recurrence in order.

template <int MODE, int AW>
__device__ __forceinline__ void group_batch8(const PlaneView& pv, const uint32_t (&l)[8],
                                             uint32_t (&af)[AW], uint32_t (&ou)[AW]) {
  constexpr int B = (AW == 4) ? 4 : 8;  // literals per sub-batch (bounds registers for wide rows)
#pragma unroll
  for (int j0 = 0; j0 < 8; j0 += B) {
    uint32_t cf[B][AW];
#pragma unroll
    for (int j = 0; j < B; ++j) load_agg<AW>(pv.aggF, GSS_ROW(l[j0 + j], 2u * pv.V + 2u, 2u * pv.V), cf[j]);
    if constexpr (MODE == GSS_MODE_ALLF) {
#pragma unroll
      for (int j = 0; j < B; ++j)
#pragma unroll
        for (int i = 0; i < AW; ++i) af[i] &= cf[j][i];
    } else {
      uint32_t cu[B][AW];
#pragma unroll
      for (int j = 0; j < B; ++j) load_agg<AW>(pv.aggU, GSS_ROW(l[j0 + j] >> 1, pv.V + 1u, pv.V), cu[j]);
#pragma unroll
      for (int j = 0; j < B; ++j)
#pragma unroll
        for (int i = 0; i < AW; ++i) {
          ou[i] = (af[i] & cu[j][i]) | (ou[i] & cf[j][i]);
          af[i] &= cf[j][i];
        }
    }
  }
}

// Stage B on 8 literals of one (clause, word g) pair.
template <int MODE>
__device__ __forceinline__ void word_batch8(const PlaneView& pv, const uint32_t (&l)[8], uint32_t g, uint32_t valid,
                                            uint32_t& af, uint32_t& ou) {
  g = GSS_ROW(g, pv.Wp, 0u);  // plane word (checked in the bounds build)
  uint32_t F[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) F[j] = __ldg(pv.P + (uint64_t)GSS_ROW(l[j], 2u * pv.V + 2u, 2u * pv.V) * pv.Wp + g);
  if constexpr (MODE == GSS_MODE_ALLF) {
#pragma unroll
    for (int j = 0; j < 8; ++j) af &= F[j];
  } else {
    uint32_t T[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) T[j] = __ldg(pv.P + (uint64_t)GSS_ROW(l[j] ^ 1u, 2u * pv.V + 2u, 2u * pv.V) * pv.Wp + g);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const uint32_t U = ~(F[j] | T[j]) & valid;
      ou = (af & U) | (ou & F[j]);
      af &= F[j];
    }
  }
}

__device__ __forceinline__ void load8_global(const uint32_t* p, uint32_t (&l)[8]) {
  const uint4 a = __ldg(reinterpret_cast<const uint4*>(p)), b = __ldg(reinterpret_cast<const uint4*>(p) + 1);
  l[0] = a.x; l[1] = a.y; l[2] = a.z; l[3] = a.w;
  l[4] = b.x; l[5] = b.y; l[6] = b.z; l[7] = b.w;
}

// Literals [b, e) of the CSR as 8-literal chunks, PAD past e.
__device__ __forceinline__ void load8_csr(const uint32_t* __restrict__ lits, uint64_t k0, uint64_t e, uint32_t pad,
                                          uint32_t (&l)[8]) {
#pragma unroll
  for (int j = 0; j < 8; ++j) l[j] = (k0 + j < e) ? __ldg(lits + k0 + j) : pad;
}

__device__ __forceinline__ void load8_smem(const uint32_t* p, uint32_t (&l)[8]) {
  const uint4 a = reinterpret_cast<const uint4*>(p)[0], b = reinterpret_cast<const uint4*>(p)[1];
  l[0] = a.x; l[1] = a.y; l[2] = a.z; l[3] = a.w;
  l[4] = b.x; l[5] = b.y; l[6] = b.z; l[7] = b.w;
}

// The exact recurrence of a (clause, word) pair past its first 8 literals (head0, already
// applied): literals 8..15 from head1 (h1s: the clause's head1 in shared memory, or nullptr
// to read it from global memory), then the CSR, while the word is alive.
template <int MODE>
__device__ __forceinline__ void exact_tail(const ClauseView& db, const PlaneView& pv, uint64_t c, const uint32_t* h1s,
                                           uint32_t g, uint32_t valid, uint32_t last_head0, uint32_t& af,
                                           uint32_t& ou) {
  uint32_t l[8];
  if ((af | ou) != 0u && last_head0 != db.pad) {
    if (h1s) load8_smem(h1s, l);
    else load8_global(db.head1 + c * 8u, l);
    word_batch8<MODE>(pv, l, g, valid, af, ou);
    if ((af | ou) != 0u && l[7] != db.pad) {
      const uint64_t e = db.off[c + 1];
      for (uint64_t k0 = db.off[c] + HEAD_K; k0 < e && (af | ou) != 0u; k0 += 8) {
        load8_csr(db.lits, k0, e, db.pad, l);
        word_batch8<MODE>(pv, l, g, valid, af, ou);
      }
    }
  }
}

// Wide sets: the group recurrence of 8 literals on the level-1 word of super-group sg (bit b:
// group 32 sg + b), gathers first.
template <int MODE>
__device__ __forceinline__ void group1_batch8(const WideView& wv, uint32_t V, const uint32_t (&l)[8], uint32_t sg,
                                              uint32_t& af, uint32_t& ou) {
  sg = GSS_ROW(sg, wv.AWp1, 0u);  // word of the level-1 rows (checked in the bounds build)
  uint32_t cf[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) cf[j] = __ldg(wv.aggF1 + (uint64_t)GSS_ROW(l[j], 2u * V + 2u, 2u * V) * wv.AWp1 + sg);
  if constexpr (MODE == GSS_MODE_ALLF) {
#pragma unroll
    for (int j = 0; j < 8; ++j) af &= cf[j];
  } else {
    uint32_t cu[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) cu[j] = __ldg(wv.aggU1 + (uint64_t)GSS_ROW(l[j] >> 1, V + 1u, V) * wv.AWp1 + sg);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      ou = (af & cu[j]) | (ou & cf[j]);
      af &= cf[j];
    }
  }
}

// Groups of super-group sg whose level-1 aggregate test is positive for clause c (head0 in l0):
// literals 8..15 from head1, then the CSR, while some group is alive.
template <int MODE>
__device__ __forceinline__ uint32_t group1_mask(const ClauseView& db, const PlaneView& pv, const WideView& wv,
                                                const uint32_t (&l0)[8], uint64_t c, uint32_t sg) {
  uint32_t af = FULL, ou = 0u;
  group1_batch8<MODE>(wv, pv.V, l0, sg, af, ou);
  if ((af | ou) != 0u && l0[7] != db.pad) {
    uint32_t l[8];
    load8_global(db.head1 + c * 8u, l);
    group1_batch8<MODE>(wv, pv.V, l, sg, af, ou);
    if ((af | ou) != 0u && l[7] != db.pad) {
      const uint64_t e = db.off[c + 1];
      for (uint64_t k0 = db.off[c] + HEAD_K; k0 < e && (af | ou) != 0u; k0 += 8) {
        load8_csr(db.lits, k0, e, db.pad, l);
        group1_batch8<MODE>(wv, pv.V, l, sg, af, ou);
      }
    }
  }
  return af | ou;
}

// Head0 of a staged pair: its owner lane's 8 literals in the warp's ring (PAD for no pair).
__device__ __forceinline__ void pair_head(const uint32_t* __restrict__ h0, bool has, uint32_t pad, uint32_t (&l)[8]) {
  if (has) {
    const uint4 a = reinterpret_cast<const uint4*>(h0)[0], b = reinterpret_cast<const uint4*>(h0)[1];
    l[0] = a.x; l[1] = a.y; l[2] = a.z; l[3] = a.w;
    l[4] = b.x; l[5] = b.y; l[6] = b.z; l[7] = b.w;
  } else {
#pragma unroll
    for (int j = 0; j < 8; ++j) l[j] = pad;
  }
}

// Records of a warp are staged in shared memory and reserved in the output with one
// atomicAdd per OUT_CAP records: a single counter shared by every warp of the grid is the
// contended resource otherwise.  Records past the capacity are counted but not written.
struct Outbox {
  gss_report* rec;
  uint64_t cap;
  unsigned long long* cnt;
  unsigned long long* cand_cnt;  // candidate-pair counter of the same test
  uint32_t n;                    // staged records (warp-uniform)
  uint32_t cand;                 // candidate pairs counted by this lane, not yet added
  unsigned long long* cand2_cnt = nullptr;  // wide sets: (clause, super-group) pairs past stage A
  uint32_t cand2 = 0u;
};
static_assert(sizeof(gss_report) == 12, "gss_report is three 32-bit words");

template <typename Smem>
__device__ __forceinline__ void out_flush(Smem& S, Outbox& o, uint32_t lane) {
  __syncwarp();
  if (o.n == 0u) return;
  unsigned long long base = 0;
  if (lane == 0) base = atomicAdd(o.cnt, (unsigned long long)o.n);
  base = __shfl_sync(FULL, base, 0);
  const uint64_t fit = o.cap > base ? 3ull * (o.cap - base) : 0ull;  // words that fit below the capacity
  uint32_t* dst = reinterpret_cast<uint32_t*>(o.rec) + 3ull * base;
  for (uint32_t i = lane; i < 3u * o.n; i += 32u)
    if (i < fit) dst[i] = S.out[i];
  o.n = 0u;
  __syncwarp();
}

// Flush and add the warp's candidate count: at the end, or before the outbox changes target.
template <typename Smem>
__device__ __forceinline__ void out_close(Smem& S, Outbox& o, uint32_t lane) {
  out_flush(S, o, lane);
  const uint32_t c = __reduce_add_sync(FULL, o.cand);
  if (lane == 0 && c) atomicAdd(o.cand_cnt, (unsigned long long)c);
  o.cand = 0u;
  if (o.cand2_cnt) {  // warp-uniform
    const uint32_t c2 = __reduce_add_sync(FULL, o.cand2);
    if (lane == 0 && c2) atomicAdd(o.cand2_cnt, (unsigned long long)c2);
    o.cand2 = 0u;
  }
}

template <typename Smem>
__device__ __forceinline__ void out_append(Smem& S, Outbox& o, bool has, uint32_t c, uint32_t g, uint32_t mask,
                                           uint32_t lane) {
  const uint32_t ball = __ballot_sync(FULL, has);
  if (ball == 0u) return;
  const uint32_t k = __popc(ball);
  if (o.n + k > OUT_CAP) out_flush(S, o, lane);
  if (has) {
    const uint32_t j = 3u * (o.n + __popc(ball & ((1u << lane) - 1u)));
    S.out[j] = c;
    S.out[j + 1] = g;
    S.out[j + 2] = mask;
  }
  o.n += k;
}

// Stage B proper: the exact recurrence of np staged pairs buf[0 .. np) (owner | group << 5, the
// owner being the clause's index in the tile, its head0 at ring + 8 owner and, when ring1 is
// not null, its head1 at ring1 + 8 owner), one pair per lane, records into the outbox.
template <int MODE, bool EXTRA, typename Smem>
__device__ __forceinline__ void exact_pairs(const ClauseView& db, const PlaneView& pv, Smem& S, const uint32_t* ring,
                                            const uint32_t* ring1, const uint32_t* buf, uint32_t np, uint64_t c0,
                                            uint32_t lane, Outbox& out, const ActivityView& av) {
  for (uint32_t p0 = 0; p0 < np; p0 += 32u) {
    const uint32_t pa = p0 + lane;
    const bool ha = pa < np;
    const uint32_t ea = ha ? buf[pa] : 0u;
    const uint32_t oa = ea & 31u, ga = ea >> 5;
    uint32_t la[8];
    pair_head(ring + oa * 8u, ha, db.pad, la);
    const uint32_t va = valid_bits(pv.N, ga) & ((pv.wvalid && ha) ? __ldg(pv.wvalid + ga) : FULL);  // real rows only
    uint32_t afa = ha ? ((MODE == GSS_MODE_ALLF) ? FULL : va) : 0u, oua = 0u;
    word_batch8<MODE>(pv, la, ga, va, afa, oua);
    exact_tail<MODE>(db, pv, c0 + oa, ring1 ? ring1 + oa * 8u : nullptr, ga, va, la[7], afa, oua);
    const uint32_t ra = afa | oua;
    const uint64_t cp = c0 + oa;  // position of the pair's clause
    uint32_t id = (uint32_t)cp;
    if constexpr (EXTRA) {
      if (ra != 0u && av.act && atomicExch(av.stamp + cp, av.epoch) != av.epoch)
        av.act[cp] += av.inc;  // bumped once per test, by the first of its reported pairs
      if (db.ext) id = __ldg(db.ext + cp);
    }
    out_append(S, out, ra != 0u, id, ga, ra, lane);
  }
}

// Exclusive prefix sum of x over the warp.
__device__ __forceinline__ uint32_t warp_excl_scan(uint32_t x, uint32_t lane) {
  uint32_t incl = x;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(FULL, incl, d);
    if (lane >= (uint32_t)d) incl += y;
  }
  return incl - x;
}

// Live plane words of clause c under per-word watermarks wm[0 .. n_wm) (non-decreasing, in
// shared memory): word w is tested iff c < wm[w]; without watermarks every word is live.
template <int AW>
__device__ __forceinline__ void live_words(const uint64_t* wm, uint32_t n_wm, uint64_t c, uint32_t (&af)[AW]) {
  if (!wm) {
#pragma unroll
    for (int i = 0; i < AW; ++i) af[i] = FULL;
    return;
  }
  uint32_t lo = 0, hi = n_wm;  // k = number of words whose watermark is <= c
  while (lo < hi) {
    const uint32_t mid = (lo + hi) / 2;
    if (wm[mid] <= c) lo = mid + 1;
    else hi = mid;
  }
#pragma unroll
  for (int i = 0; i < AW; ++i) {
    const uint32_t b = 32u * i;
    af[i] = lo <= b ? FULL : (lo >= b + 32u ? 0u : (FULL << (lo - b)));
  }
}

// Stage A and stage B for the tile of clauses [c0, min(c0 + 32, c_hi)), whose head0 is in
// S.ring[s]; records are staged in the warp's outbox.  EXTRA: the database has clause ids
// apart from positions and/or activities to bump (a separate build of the kernel, so that
// databases without them pay nothing).  WIDE (with AW == 1): pv's aggregate rows are the
// level-2 rows and stage A's bits are super-groups; wv holds the level-1 rows.
// Stage A with two lanes per clause (16 clauses per tile): lane 2i + h starts on head h of
// clause i.  Each lane runs the recurrence over its own 8 literals, the even lane from the
// clause's live words, the odd one from the identity (all ones, nothing U-implied); the two
// segment results compose -- the recurrence is linear over the bits, so (A0, O0) then
// (A1, O1) give (A0 A1, O0 A1 | A0 O1) -- and both lanes continue with the composed state
// over 16 CSR literals per round, 8 each.  mask: the two lanes of the pair.
template <int MODE, int AW>
__device__ __forceinline__ void compose_pair(uint32_t (&af)[AW], uint32_t (&ou)[AW], uint32_t half, uint32_t mask) {
#pragma unroll
  for (int i = 0; i < AW; ++i) {
    const uint32_t pa = __shfl_xor_sync(mask, af[i], 1), po = __shfl_xor_sync(mask, ou[i], 1);
    if constexpr (MODE == GSS_MODE_ALLF) {
      af[i] &= pa;
    } else {
      const uint32_t a0 = half ? pa : af[i], o0 = half ? po : ou[i];  // even lane's segment first
      const uint32_t a1 = half ? af[i] : pa, o1 = half ? ou[i] : po;
      af[i] = a0 & a1;
      ou[i] = (o0 & a1) | (a0 & o1);
    }
  }
}

template <int MODE, int AW>
__device__ __forceinline__ void stage_a_paired(const ClauseView& db, const PlaneView& pv, const uint32_t* ring,
                                               uint64_t c0, uint64_t c_hi, uint32_t lane, const uint64_t* wm,
                                               uint32_t n_wm, uint32_t (&af)[AW], uint32_t (&ou)[AW]) {
  const uint32_t PAD = db.pad;
  const uint32_t ci = lane >> 1, half = lane & 1u;
  const uint64_t c = c0 + ci;
  const bool act = c < c_hi;
  live_words<AW>(wm, n_wm, c, af);
#pragma unroll
  for (int i = 0; i < AW; ++i) { af[i] = act ? (half ? FULL : af[i]) : 0u; ou[i] = 0u; }
  uint32_t l[8];
  if (act) load8_smem(ring + half * 128u + ci * 8u, l);
  else {
#pragma unroll
    for (int j = 0; j < 8; ++j) l[j] = PAD;
  }
  // more than 16 literals: the odd lane's head1 is full; the rest is in the CSR
  const bool tail = __shfl_sync(FULL, l[7], lane | 1u) != PAD && act;
  uint64_t b = 0, e = 0;
  if (tail) {  // in flight during the head batch
    b = __ldg(db.off + c);
    e = __ldg(db.off + c + 1);
  }
  if (act) group_batch8<MODE, AW>(pv, l, af, ou);
  compose_pair<MODE, AW>(af, ou, half, FULL);
  if (tail && any2<AW>(af, ou)) {
    const uint32_t mask = 3u << (lane & ~1u);  // both lanes of the pair take the same iterations
    for (uint64_t k0 = b + HEAD_K; k0 < e && any2<AW>(af, ou); k0 += 16) {
      load8_csr(db.lits, k0 + 8u * half, e, PAD, l);
      if (half) {  // the odd lane's chunk starts from the identity
#pragma unroll
        for (int i = 0; i < AW; ++i) { af[i] = FULL; ou[i] = 0u; }
      }
      group_batch8<MODE, AW>(pv, l, af, ou);
      compose_pair<MODE, AW>(af, ou, half, mask);
    }
  }
}

// Stage A and stage B for the tile of clauses [c0, min(c0 + CPW, c_hi)), whose heads are in
// S.ring[s] (CPW = 32: head0 of each lane's clause; CPW = 16: head0 of the 16 clauses, then
// their head1); records are staged in the warp's outbox.  EXTRA: the database has clause ids
// apart from positions and/or activities to bump (a separate build of the kernel, so that
// databases without them pay nothing).  WIDE (with AW == 1, CPW == 32): pv's aggregate rows
// are the level-2 rows and stage A's bits are super-groups; wv holds the level-1 rows.
template <int MODE, int AW, bool EXTRA = false, bool WIDE = false, int CPW = 32, typename Smem>
__device__ __forceinline__ void test_tile(const ClauseView& db, const PlaneView& pv, Smem& S,
                                          int s, uint64_t c0, uint64_t c_hi, uint32_t lane, Outbox& out,
                                          const uint64_t* wm = nullptr, uint32_t n_wm = 0,
                                          const ActivityView& av = ActivityView{}, const WideView& wv = WideView{}) {
  static_assert(!WIDE || AW == 1, "wide sets have one level-2 word per row");
  static_assert(CPW == 32 || (CPW == 16 && !WIDE), "tile shapes: 32 clauses, or 16 with two lanes each");
  const uint32_t PAD = db.pad;
  uint32_t af[AW], ou[AW];
  if constexpr (CPW == 16) {
    // ---------------- stage A: group test, two lanes per clause
    stage_a_paired<MODE, AW>(db, pv, S.ring[s], c0, c_hi, lane, wm, n_wm, af, ou);
    if (lane & 1u) {  // the even lane of a pair owns its candidates
#pragma unroll
      for (int i = 0; i < AW; ++i) { af[i] = 0u; ou[i] = 0u; }
    }
  } else {
  const uint64_t c = c0 + lane;
  const bool act = c < c_hi;
  const uint32_t* h0 = &S.ring[s][lane * 8u];

  // ---------------- stage A: group (aggregate) test of this lane's clause
  live_words<AW>(wm, n_wm, c, af);
#pragma unroll
  for (int i = 0; i < AW; ++i) { af[i] = act ? af[i] : 0u; ou[i] = 0u; }
  if (act) {
    uint32_t l[8], l1[8];
    load8_smem(h0, l);
    const bool long_clause = l[7] != PAD;
    if (long_clause) load8_global(db.head1 + c * 8u, l1);  // in flight during the first batch
    group_batch8<MODE, AW>(pv, l, af, ou);
    if (long_clause && any2<AW>(af, ou)) {
      const bool tail = l1[7] != PAD;
      uint64_t b = 0, e = 0;
      if (tail) { b = __ldg(db.off + c); e = __ldg(db.off + c + 1); }  // in flight during the second batch
      group_batch8<MODE, AW>(pv, l1, af, ou);
      if (tail && any2<AW>(af, ou)) {
        for (uint64_t k0 = b + HEAD_K; k0 < e && any2<AW>(af, ou); k0 += 8) {
          load8_csr(db.lits, k0, e, PAD, l);
          group_batch8<MODE, AW>(pv, l, af, ou);
        }
      }
    }
  }
  }
  uint32_t cand[AW];
#pragma unroll
  for (int i = 0; i < AW; ++i) {
    cand[i] = af[i] | ou[i];
    if constexpr (WIDE) out.cand2 += __popc(cand[i]);  // (clause, super-group) pairs left by the level-2 test
    else out.cand += __popc(cand[i]);                  // pairs the aggregate test let through
  }

  // ---------------- stage B: exact test of the warp's candidate (clause, group) pairs (wide
  // sets: (clause, super-group) pairs, each first narrowed to its groups by the level-1 test)
  for (;;) {
    uint32_t cnt = 0;
#pragma unroll
    for (int i = 0; i < AW; ++i) cnt += __popc(cand[i]);
    const uint32_t total = __reduce_add_sync(FULL, cnt);
    if (total == 0u) break;
    uint32_t pos = warp_excl_scan(cnt, lane);
#pragma unroll
    for (int i = 0; i < AW; ++i) {
      while (cand[i] != 0u && pos < PAIR_CAP) {
        const uint32_t bit = (uint32_t)(__ffs(cand[i]) - 1);
        cand[i] &= cand[i] - 1u;
        S.pairs[pos++] = (CPW == 16 ? lane >> 1 : lane) | ((32u * i + bit) << 5);
      }
    }
    __syncwarp();
    const uint32_t np = total < PAIR_CAP ? total : PAIR_CAP;
    if constexpr (WIDE) {
      for (uint32_t p0 = 0; p0 < np; p0 += 32u) {
        const uint32_t pa = p0 + lane;
        const bool ha = pa < np;
        const uint32_t ea = ha ? S.pairs[pa] : 0u;
        const uint32_t oa = ea & 31u, sg = ea >> 5;
        uint32_t gm = 0u;  // groups of super-group sg left by the level-1 test
        if (ha) {
          uint32_t la[8];
          pair_head(&S.ring[s][oa * 8u], true, PAD, la);
          gm = group1_mask<MODE>(db, pv, wv, la, c0 + oa, sg);
        }
        out.cand += __popc(gm);
        for (;;) {  // compact the (clause, group) pairs over the warp, PAIR_CAP per round
          const uint32_t n1 = __popc(gm);
          const uint32_t t1 = __reduce_add_sync(FULL, n1);
          if (t1 == 0u) break;
          uint32_t q = warp_excl_scan(n1, lane);
          while (gm != 0u && q < PAIR_CAP) {
            const uint32_t b = (uint32_t)(__ffs(gm) - 1);
            gm &= gm - 1u;
            S.pairs2[q++] = oa | ((32u * sg + b) << 5);
          }
          __syncwarp();
          exact_pairs<MODE, EXTRA>(db, pv, S, S.ring[s], nullptr, S.pairs2, t1 < PAIR_CAP ? t1 : PAIR_CAP, c0, lane,
                                   out, av);
          __syncwarp();
        }
      }
    } else {
      exact_pairs<MODE, EXTRA>(db, pv, S, S.ring[s], CPW == 16 ? &S.ring[s][128] : nullptr, S.pairs, np, c0, lane,
                               out, av);
    }
    __syncwarp();
  }
}

// Lane 0: bulk-copy the heads of the n clauses from c0 into ring stage `stage`: head0 (CPW =
// 32), or head0 then head1 of the 16 clauses of a paired-lane tile (CPW = 16).
template <int CPW, typename Smem>
__device__ __forceinline__ void issue_heads(Smem& S, int stage, const ClauseView& db, uint64_t c0, uint32_t n) {
  ptx::fence_proxy_async();
  ptx::mbar_expect_tx(&S.bar[stage], (CPW == 16 ? 2u : 1u) * n * 32u);
  ptx::bulk_g2s(S.ring[stage], db.head0 + c0 * 8u, n * 32u, &S.bar[stage]);
  if constexpr (CPW == 16) ptx::bulk_g2s(&S.ring[stage][128], db.head1 + c0 * 8u, n * 32u, &S.bar[stage]);
}

template <int MODE, int AW, bool EXTRA, bool WIDE = false, int CPW = 32>
__global__ void __launch_bounds__(TEST_THREADS) k_test(ClauseView db, uint64_t c_lo, uint64_t c_hi, PlaneView pv,
                                                       gss_report* __restrict__ rec, uint64_t cap, DevStatus* st,
                                                       const uint64_t* __restrict__ wm, uint32_t n_wm,
                                                       ActivityView av, WideView wv) {
  using Smem = std::conditional_t<WIDE, WarpSmemWide, WarpSmem>;
  __shared__ Smem smem[TEST_WARPS];
  __shared__ uint64_t s_wm[32 * AW];  // per-word clause watermarks (serving launches)
  if (st->bad_code) return;  // the assignment set held an invalid value code: no records
  if (n_wm > 32u * AW) n_wm = 32u * AW;
  for (uint32_t i = threadIdx.x; wm && i < n_wm; i += TEST_THREADS) s_wm[i] = wm[i];
  __syncthreads();
  const uint64_t* wms = wm ? s_wm : nullptr;
  const uint32_t lane = threadIdx.x & 31u, wib = threadIdx.x >> 5;
  Smem& S = smem[wib];
  const uint64_t warp_id = (uint64_t)blockIdx.x * TEST_WARPS + wib;
  const uint64_t n_warps = (uint64_t)gridDim.x * TEST_WARPS;
  const uint64_t n_tiles = (c_hi - c_lo + CPW - 1) / CPW;
  if (warp_id >= n_tiles) return;

  if (lane == 0) {
    ptx::mbar_init(&S.bar[0], 1);
    ptx::mbar_init(&S.bar[1], 1);
    ptx::fence_mbar_init();
  }
  __syncwarp();
  auto issue = [&](uint64_t tile, int stage) {  // lane 0: bulk-copy the tile's heads into ring[stage]
    const uint64_t c0 = c_lo + tile * CPW;
    const uint64_t left = c_hi - c0;
    issue_heads<CPW>(S, stage, db, c0, left < (uint64_t)CPW ? (uint32_t)left : (uint32_t)CPW);
  };
  if (lane == 0) issue(warp_id, 0);

  Outbox out{rec, cap, &st->n_records, &st->n_candidates, 0u, 0u, WIDE ? &st->n_super : nullptr, 0u};
  uint32_t it = 0;
  for (uint64_t t = warp_id; t < n_tiles; t += n_warps, ++it) {
    const int s = it & 1;
    const bool has_next = t + n_warps < n_tiles;
    if (lane == 0 && has_next) issue(t + n_warps, s ^ 1);
    const bool ok = ptx::mbar_wait(&S.bar[s], (it >> 1) & 1u);
    if (!__all_sync(FULL, ok)) {  // bounded wait gave up: flag it, drain our copies (bounded), leave
      if (lane == 0) {
        atomicOr(&st->timeout, 1u);
        ptx::mbar_wait(&S.bar[s], (it >> 1) & 1u);
        if (has_next) ptx::mbar_wait(&S.bar[s ^ 1], ((it + 1) >> 1) & 1u);
      }
      out_close(S, out, lane);
      return;
    }
    test_tile<MODE, AW, EXTRA, WIDE, CPW>(db, pv, S, s, c_lo + t * CPW, c_hi, lane, out, wms, n_wm, av, wv);
    __syncwarp();
  }
  out_close(S, out, lane);
}

// Last instance whose first tile is <= t (instances without clauses are skipped because a
// later instance starts at the same tile).
__device__ __forceinline__ uint32_t find_inst(const BatchInst* __restrict__ inst, uint32_t n, uint64_t t) {
  uint32_t lo = 0, hi = n - 1;
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) / 2;
    if (__ldg(&inst[mid].tile0) <= t) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// One persistent launch over the 32-clause tiles of every instance of a batch.  Warps take
// `grab` consecutive tiles at a time from a device counter (work stealing), so instances of
// very different sizes share the GPU without a launch each; the head0 copy of a warp's next
// tile is in flight while the current one is tested, as in k_test.
template <int MODE, int AW, int CPW = 32>
__global__ void __launch_bounds__(TEST_THREADS) k_test_batch(const BatchInst* __restrict__ inst, uint32_t n_inst,
                                                             uint64_t n_tiles, unsigned long long* __restrict__ work,
                                                             uint32_t grab, DevStatus* bst) {
  __shared__ WarpSmem smem[TEST_WARPS];
  const uint32_t lane = threadIdx.x & 31u, wib = threadIdx.x >> 5;
  WarpSmem& S = smem[wib];
  unsigned long long cb = 0;
  if (lane == 0) cb = atomicAdd(work, (unsigned long long)grab);
  cb = __shfl_sync(FULL, cb, 0);
  if (cb >= n_tiles) return;
  uint64_t ce = min((uint64_t)cb + grab, n_tiles);
  if (lane == 0) {
    ptx::mbar_init(&S.bar[0], 1);
    ptx::mbar_init(&S.bar[1], 1);
    ptx::fence_mbar_init();
  }
  __syncwarp();
  auto issue = [&](uint64_t t, int stage) {  // lane 0: bulk-copy tile t's heads into ring[stage]
    const BatchInst& d = inst[find_inst(inst, n_inst, t)];
    const uint64_t c0 = (t - d.tile0) * CPW;
    const uint64_t left = d.m - c0;
    issue_heads<CPW>(S, stage, d.db, c0, left < (uint64_t)CPW ? (uint32_t)left : (uint32_t)CPW);
  };
  uint64_t t = cb;
  if (lane == 0) issue(t, 0);
  Outbox out{nullptr, 0, nullptr, nullptr, 0u, 0u};
  uint32_t cur = 0xFFFFFFFFu;  // instance whose records the outbox holds
  for (uint32_t it = 0;; ++it) {
    uint64_t tn = t + 1;
    if (tn >= ce) {  // take the next chunk of tiles
      unsigned long long nb = 0;
      if (lane == 0) nb = atomicAdd(work, (unsigned long long)grab);
      tn = __shfl_sync(FULL, nb, 0);
      ce = min(tn + grab, n_tiles);
    }
    const bool has_next = tn < n_tiles;
    const int s = it & 1;
    if (lane == 0 && has_next) issue(tn, s ^ 1);
    const bool ok = ptx::mbar_wait(&S.bar[s], (it >> 1) & 1u);
    if (!__all_sync(FULL, ok)) {  // bounded wait gave up: flag it, drain our copies (bounded), leave
      if (lane == 0) {
        atomicOr(&bst->timeout, 1u);
        ptx::mbar_wait(&S.bar[s], (it >> 1) & 1u);
        if (has_next) ptx::mbar_wait(&S.bar[s ^ 1], ((it + 1) >> 1) & 1u);
      }
      out_close(S, out, lane);
      return;
    }
    const uint32_t i = find_inst(inst, n_inst, t);
    const ClauseView db = inst[i].db;
    const PlaneView pv = inst[i].pv;
    DevStatus* st = inst[i].st;
    if (i != cur) {  // records go to another instance from here on
      out_close(S, out, lane);
      out = Outbox{inst[i].rec, inst[i].cap, &st->n_records, &st->n_candidates, 0u, 0u};
      cur = i;
    }
    if (!st->bad_code)
      test_tile<MODE, AW, false, false, CPW>(db, pv, S, s, (t - inst[i].tile0) * CPW, inst[i].m, lane, out);
    __syncwarp();  // every lane is done with ring[s] before it is refilled
    if (!has_next) break;
    t = tn;
  }
  out_close(S, out, lane);
}

// Zero the work counter, the batch status and every instance's test status (records, bad
// codes, timeouts) before a batched run.
__global__ void k_batch_reset(const BatchInst* __restrict__ inst, uint32_t n_inst, unsigned long long* work,
                              DevStatus* bst) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    *work = 0ull;
    *bst = DevStatus{};
  }
  if (i < n_inst) *inst[i].st = DevStatus{};
}

template <int MODE, int AW, bool WIDE = false, int CPW = 32>
void launch_one(const ClauseView& db, uint64_t c_lo, uint64_t c_hi, const PlaneView& pv, gss_report* rec,
                uint64_t cap, DevStatus* st, int grid, cudaStream_t s, const uint64_t* wm, uint32_t n_wm,
                const ActivityView& av, const WideView& wv) {
  if (db.ext || av.act)
    k_test<MODE, AW, true, WIDE, CPW><<<grid, TEST_THREADS, 0, s>>>(db, c_lo, c_hi, pv, rec, cap, st, wm, n_wm, av, wv);
  else
    k_test<MODE, AW, false, WIDE, CPW><<<grid, TEST_THREADS, 0, s>>>(db, c_lo, c_hi, pv, rec, cap, st, wm, n_wm, av,
                                                                     wv);
}

template <int MODE, int AW>
void launch_cpw(int cpw, const ClauseView& db, uint64_t c_lo, uint64_t c_hi, const PlaneView& pv, gss_report* rec,
                uint64_t cap, DevStatus* st, int grid, cudaStream_t s, const uint64_t* wm, uint32_t n_wm,
                const ActivityView& av, const WideView& wv) {
  if (cpw == 16) launch_one<MODE, AW, false, 16>(db, c_lo, c_hi, pv, rec, cap, st, grid, s, wm, n_wm, av, wv);
  else launch_one<MODE, AW, false, 32>(db, c_lo, c_hi, pv, rec, cap, st, grid, s, wm, n_wm, av, wv);
}

template <int MODE, int AW, bool WIDE = false, int CPW = 32>
int grid_for(int n_sms) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_test<MODE, AW, false, WIDE, CPW>, TEST_THREADS, 0) !=
          cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  return per_sm * n_sms;
}

// agg2F / agg2U: one thread per level-2 row; bit s set iff level-1 word s of the row is non-zero.
__global__ void k_agg2(const uint32_t* __restrict__ aggF1, const uint32_t* __restrict__ aggU1, uint32_t V,
                       uint32_t AWp1, uint32_t* __restrict__ agg2F, uint32_t* __restrict__ agg2U) {
  const uint64_t nF = 2ull * V + 2ull, n = nF + V + 1ull;
  for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (uint64_t)gridDim.x * blockDim.x) {
    const bool f = r < nF;
    const uint32_t* src = f ? aggF1 + r * AWp1 : aggU1 + (r - nF) * AWp1;
    uint32_t b = 0u;
    for (uint32_t i = 0; i < AWp1; i += 4) {  // AWp1 is 8, 16 or 32: 16-byte rows
      const uint4 x = __ldg(reinterpret_cast<const uint4*>(src + i));
      b |= (x.x != 0u ? 1u : 0u) << i;
      b |= (x.y != 0u ? 1u : 0u) << (i + 1);
      b |= (x.z != 0u ? 1u : 0u) << (i + 2);
      b |= (x.w != 0u ? 1u : 0u) << (i + 3);
    }
    if (f) agg2F[r] = b;
    else agg2U[r - nF] = b;
  }
}

template <int MODE, int AW, int CPW>
int batch_grid_for(int n_sms) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_test_batch<MODE, AW, CPW>, TEST_THREADS, 0) !=
          cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  return per_sm * n_sms;
}

}  // namespace

cudaError_t launch_batch_reset(const BatchInst* d_inst, uint32_t n_inst, unsigned long long* work, DevStatus* bst,
                               cudaStream_t s) {
  k_batch_reset<<<(n_inst + 255) / 256 + 1, 256, 0, s>>>(d_inst, n_inst, work, bst);
  return cudaGetLastError();
}

cudaError_t launch_test_batch(int mode, uint32_t AWp, int cpw, const BatchInst* d_inst, uint32_t n_inst,
                              uint64_t n_tiles, unsigned long long* work, uint32_t grab, DevStatus* bst, int grid,
                              cudaStream_t s) {
  if (n_inst == 0 || n_tiles == 0) return cudaSuccess;
  if (grid < 1) grid = 1;
  if (grab < 1) grab = 1;
#define GSS_BATCH_LAUNCH(M, A)                                                                                   \
  do {                                                                                                           \
    if (cpw == 16) k_test_batch<M, A, 16><<<grid, TEST_THREADS, 0, s>>>(d_inst, n_inst, n_tiles, work, grab, bst); \
    else k_test_batch<M, A, 32><<<grid, TEST_THREADS, 0, s>>>(d_inst, n_inst, n_tiles, work, grab, bst);          \
  } while (0)
  if (mode == GSS_MODE_ALLF) {
    if (AWp == 1) GSS_BATCH_LAUNCH(GSS_MODE_ALLF, 1);
    else if (AWp == 2) GSS_BATCH_LAUNCH(GSS_MODE_ALLF, 2);
    else GSS_BATCH_LAUNCH(GSS_MODE_ALLF, 4);
  } else {
    if (AWp == 1) GSS_BATCH_LAUNCH(GSS_MODE_TRIGGER, 1);
    else if (AWp == 2) GSS_BATCH_LAUNCH(GSS_MODE_TRIGGER, 2);
    else GSS_BATCH_LAUNCH(GSS_MODE_TRIGGER, 4);
  }
#undef GSS_BATCH_LAUNCH
  return cudaGetLastError();
}

int test_batch_grid_size(int mode, uint32_t AWp, int cpw, int n_sms) {
#define GSS_BGRID(M, A) (cpw == 16 ? batch_grid_for<M, A, 16>(n_sms) : batch_grid_for<M, A, 32>(n_sms))
  if (mode == GSS_MODE_ALLF) {
    if (AWp == 1) return GSS_BGRID(GSS_MODE_ALLF, 1);
    if (AWp == 2) return GSS_BGRID(GSS_MODE_ALLF, 2);
    return GSS_BGRID(GSS_MODE_ALLF, 4);
  }
  if (AWp == 1) return GSS_BGRID(GSS_MODE_TRIGGER, 1);
  if (AWp == 2) return GSS_BGRID(GSS_MODE_TRIGGER, 2);
  return GSS_BGRID(GSS_MODE_TRIGGER, 4);
#undef GSS_BGRID
}

cudaError_t launch_agg2(const uint32_t* aggF1, const uint32_t* aggU1, uint32_t V, uint32_t AWp1, uint32_t* agg2F,
                        uint32_t* agg2U, cudaStream_t s) {
  if (AWp1 < 8 || AWp1 > 32 || (AWp1 & (AWp1 - 1)) != 0) return cudaErrorInvalidValue;
  const uint64_t n = 3ull * V + 3ull;
  const uint64_t blocks = (n + 255) / 256;
  k_agg2<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(aggF1, aggU1, V, AWp1, agg2F, agg2U);
  return cudaGetLastError();
}

cudaError_t launch_test(int mode, const ClauseView& db, uint64_t c_lo, uint64_t c_hi, const PlaneView& pv,
                        gss_report* rec, uint64_t cap, DevStatus* st, int grid, cudaStream_t s, const uint64_t* wm,
                        uint32_t n_wm, const ActivityView& av, const WideView& wv, int cpw) {
  if (c_hi <= c_lo) return cudaSuccess;
  if (wv.aggF1) cpw = 32;  // the wide build has one tile shape
  cpw = cpw == 16 ? 16 : 32;
  const uint64_t tiles = (c_hi - c_lo + cpw - 1) / cpw;
  const uint64_t max_blocks = (tiles + TEST_WARPS - 1) / TEST_WARPS;
  if ((uint64_t)grid > max_blocks) grid = (int)max_blocks;
  if (grid < 1) grid = 1;
  if (wv.aggF1) {  // wide set: pv holds the level-2 rows (one word each)
    if (pv.AWp != 1 || wm) return cudaErrorInvalidValue;
    if (mode == GSS_MODE_ALLF) launch_one<GSS_MODE_ALLF, 1, true>(db, c_lo, c_hi, pv, rec, cap, st, grid, s, nullptr, 0, av, wv);
    else launch_one<GSS_MODE_TRIGGER, 1, true>(db, c_lo, c_hi, pv, rec, cap, st, grid, s, nullptr, 0, av, wv);
    return cudaGetLastError();
  }
  if (mode == GSS_MODE_ALLF) {
    if (pv.AWp == 1) launch_cpw<GSS_MODE_ALLF, 1>(cpw, db, c_lo, c_hi, pv, rec, cap, st, grid, s, wm, n_wm, av, wv);
    else if (pv.AWp == 2) launch_cpw<GSS_MODE_ALLF, 2>(cpw, db, c_lo, c_hi, pv, rec, cap, st, grid, s, wm, n_wm, av, wv);
    else launch_cpw<GSS_MODE_ALLF, 4>(cpw, db, c_lo, c_hi, pv, rec, cap, st, grid, s, wm, n_wm, av, wv);
  } else {
    if (pv.AWp == 1) launch_cpw<GSS_MODE_TRIGGER, 1>(cpw, db, c_lo, c_hi, pv, rec, cap, st, grid, s, wm, n_wm, av, wv);
    else if (pv.AWp == 2) launch_cpw<GSS_MODE_TRIGGER, 2>(cpw, db, c_lo, c_hi, pv, rec, cap, st, grid, s, wm, n_wm, av, wv);
    else launch_cpw<GSS_MODE_TRIGGER, 4>(cpw, db, c_lo, c_hi, pv, rec, cap, st, grid, s, wm, n_wm, av, wv);
  }
  return cudaGetLastError();
}

int test_tile_shape(uint64_t m, uint64_t L) {
  // 32 clauses per tile.  Pairing lanes on long clauses halves a clause's chain of dependent
  // gathers but also the clauses a warp has in flight; measured on GB300 it was slower on
  // every workload, long clauses included (4M clauses of median 20 literals: 217 us against
  // 168 us; 10M of median 40: 662 us against 445 us).  The batch autotuner still times both.
  (void)m;
  (void)L;
  return 32;
}

int test_grid_size(int mode, uint32_t AWp, int n_sms, bool wide, int cpw) {
  if (wide) return mode == GSS_MODE_ALLF ? grid_for<GSS_MODE_ALLF, 1, true>(n_sms) : grid_for<GSS_MODE_TRIGGER, 1, true>(n_sms);
#define GSS_GRID(M, A) (cpw == 16 ? grid_for<M, A, false, 16>(n_sms) : grid_for<M, A, false, 32>(n_sms))
  if (mode == GSS_MODE_ALLF) {
    if (AWp == 1) return GSS_GRID(GSS_MODE_ALLF, 1);
    if (AWp == 2) return GSS_GRID(GSS_MODE_ALLF, 2);
    return GSS_GRID(GSS_MODE_ALLF, 4);
  }
  if (AWp == 1) return GSS_GRID(GSS_MODE_TRIGGER, 1);
  if (AWp == 2) return GSS_GRID(GSS_MODE_TRIGGER, 2);
  return GSS_GRID(GSS_MODE_TRIGGER, 4);
#undef GSS_GRID
}

cudaError_t debug_bounds_errors(unsigned long long* out, bool reset) {
#ifdef GSS_DEBUG_BOUNDS
  cudaError_t e = cudaMemcpyFromSymbol(out, g_bounds_errors, sizeof(unsigned long long));
  if (e == cudaSuccess && reset) {
    const unsigned long long zero = 0;
    e = cudaMemcpyToSymbol(g_bounds_errors, &zero, sizeof zero);
  }
  return e;
#else
  (void)reset;
  *out = 0;
  return cudaSuccess;
#endif
}

}  // namespace gss
