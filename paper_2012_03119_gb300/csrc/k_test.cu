// k_test.cu -- test every clause against every assignment of the current set.
//
// What is computed (per clause c, per assignment a):
//   GSS_MODE_ALLF     every literal of c is F under a: c "would have been in conflict"
//                     (Section 3.3); the allFalse recurrence of Listing assignmentTrigger
//                     (Section 3.4), allFalse &= isFalse(l), over 32 assignments per word.
//   GSS_MODE_TRIGGER  Definition "triggers" (Section 3.3): the full recurrence of Listing
//                     assignmentTrigger, oneUndef = (allFalse & U(l)) | (oneUndef & F(l)),
//                     allFalse &= F(l), result allFalse | oneUndef.
//
// How (Sections 3.5 and 4.3, re-planned for GB300):
//   * one lane per clause, 32 clauses per warp, persistent grid-stride over 32-clause tiles;
//   * the clause's first 8 literals come from the head array: two 16-byte streaming loads
//     per lane, 1 KiB contiguous per warp;
//   * stage A is Listing multiTrigger's group test: the aggregate words (one bit per
//     32-assignment group, Section 4.2) are ANDed (all-F) or run through the
//     aggregateTrigger recurrence (trigger).  The aggregate rows are 4-16 bytes per literal
//     and small enough (8 MiB at V = 1M) to stay in L2, the hottest ones in L1.  By the
//     Theorem of Section 4.2 a group whose aggregate test is negative holds no hit;
//   * literals past the head are read from the CSR only while some group is alive;
//   * stage B runs the exact word recurrence on each surviving group (Listing
//     multiTrigger's inner assignmentTrigger call) and appends one record per non-zero
//     word with a warp ballot, a population count and one atomicAdd per warp
//     (report(i, mask) of Listing multiTrigger).
// Records past the buffer capacity are counted but not written.
#include "gss_internal.h"

namespace gss {
namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr int TEST_THREADS = 256;

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
__device__ __forceinline__ bool any_bit(const uint32_t (&a)[AW]) {
  uint32_t o = 0;
#pragma unroll
  for (int i = 0; i < AW; ++i) o |= a[i];
  return o != 0u;
}

__device__ __forceinline__ uint32_t valid_bits(uint32_t N, uint32_t w) {
  const uint32_t lo = w * 32u;
  if (lo >= N) return 0u;
  const uint32_t rem = N - lo;
  return rem >= 32u ? FULL : ((1u << rem) - 1u);
}

// One step of the group test for literal l.
template <int MODE, int AW>
__device__ __forceinline__ void group_step(const PlaneView& pv, uint32_t l, uint32_t (&af)[AW], uint32_t (&ou)[AW]) {
  uint32_t cf[AW];
  load_agg<AW>(pv.aggF, l, cf);
  if constexpr (MODE == GSS_MODE_ALLF) {
#pragma unroll
    for (int i = 0; i < AW; ++i) af[i] &= cf[i];
  } else {
    uint32_t cu[AW];
    load_agg<AW>(pv.aggU, l >> 1, cu);
#pragma unroll
    for (int i = 0; i < AW; ++i) {
      ou[i] = (af[i] & cu[i]) | (ou[i] & cf[i]);
      af[i] &= cf[i];
    }
  }
}

// Exact recurrence for one literal on plane word g.
template <int MODE>
__device__ __forceinline__ void word_step(const PlaneView& pv, uint32_t l, uint32_t g, uint32_t valid, uint32_t& af,
                                          uint32_t& ou) {
  const uint32_t F = __ldg(pv.P + (uint64_t)l * pv.Wp + g);
  if constexpr (MODE == GSS_MODE_ALLF) {
    af &= F;
  } else {
    const uint32_t T = __ldg(pv.P + (uint64_t)(l ^ 1u) * pv.Wp + g);
    const uint32_t U = ~(F | T) & valid;
    ou = (af & U) | (ou & F);
    af &= F;
  }
}

template <int MODE>
__device__ __forceinline__ uint32_t exact_word(const ClauseView& db, const PlaneView& pv, uint64_t c,
                                               const uint32_t (&l)[HEAD_K], bool has_tail, uint32_t g) {
  const uint32_t valid = valid_bits(pv.N, g);
  uint32_t af = valid, ou = 0u;
#pragma unroll
  for (uint32_t k = 0; k < HEAD_K; ++k)
    if (l[k] != db.pad && (af | ou) != 0u) word_step<MODE>(pv, l[k], g, valid, af, ou);
  if (has_tail && (af | ou) != 0u) {
    const uint64_t b = db.off[c] + HEAD_K, e = db.off[c + 1];
    for (uint64_t k = b; k < e && (af | ou) != 0u; ++k) word_step<MODE>(pv, __ldg(db.lits + k), g, valid, af, ou);
  }
  return af | ou;
}

__device__ __forceinline__ void warp_append(bool has, uint32_t c, uint32_t g, uint32_t mask, uint32_t lane,
                                            gss_report* __restrict__ rec, uint64_t cap,
                                            unsigned long long* cnt) {
  const uint32_t ball = __ballot_sync(FULL, has);
  if (ball == 0u) return;
  const int leader = __ffs(ball) - 1;
  unsigned long long base = 0;
  if ((int)lane == leader) base = atomicAdd(cnt, (unsigned long long)__popc(ball));
  base = __shfl_sync(FULL, base, leader);
  if (has) {
    const unsigned long long idx = base + (unsigned long long)__popc(ball & ((1u << lane) - 1u));
    if (idx < cap) {
      gss_report r;
      r.clause_id = c; r.word = g; r.mask = mask;
      rec[idx] = r;
    }
  }
}

template <int MODE, int AW>
__global__ void __launch_bounds__(TEST_THREADS) k_test(ClauseView db, uint64_t c_lo, uint64_t c_hi, PlaneView pv,
                                                       gss_report* __restrict__ rec, uint64_t cap, DevStatus* st) {
  if (st->bad_code) return;  // the assignment set held an invalid value code: no records
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t warp_id = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const uint64_t n_warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  const uint32_t PAD = db.pad;

  for (uint64_t tile = c_lo + warp_id * 32u; tile < c_hi; tile += n_warps * 32u) {
    const uint64_t c = tile + lane;
    const bool act = c < c_hi;
    uint32_t l[HEAD_K];
    if (act) {
      const uint4* hp = reinterpret_cast<const uint4*>(db.head + c * HEAD_K);
      const uint4 h0 = __ldcs(hp), h1 = __ldcs(hp + 1);
      l[0] = h0.x; l[1] = h0.y; l[2] = h0.z; l[3] = h0.w;
      l[4] = h1.x; l[5] = h1.y; l[6] = h1.z; l[7] = h1.w;
    } else {
#pragma unroll
      for (uint32_t k = 0; k < HEAD_K; ++k) l[k] = PAD;
    }
    const bool has_tail = act && l[HEAD_K - 1] != PAD;

    // ---- stage A: group (aggregate) test
    uint32_t af[AW], ou[AW];
#pragma unroll
    for (int i = 0; i < AW; ++i) { af[i] = act ? FULL : 0u; ou[i] = 0u; }
    if constexpr (MODE == GSS_MODE_ALLF) {
      // PAD rows are all ones, so the head is ANDed branch-free in two batches of four
      // (four gathers in flight, then a second round only if some group is still alive).
#pragma unroll
      for (uint32_t k = 0; k < 4; ++k) group_step<MODE, AW>(pv, l[k], af, ou);
      if (any_bit<AW>(af)) {
#pragma unroll
        for (uint32_t k = 4; k < HEAD_K; ++k) group_step<MODE, AW>(pv, l[k], af, ou);
      }
    } else {
#pragma unroll
      for (uint32_t k = 0; k < HEAD_K; ++k) {
        uint32_t alive[AW];
#pragma unroll
        for (int i = 0; i < AW; ++i) alive[i] = af[i] | ou[i];
        if (l[k] != PAD && any_bit<AW>(alive)) group_step<MODE, AW>(pv, l[k], af, ou);
      }
    }
    uint32_t cand[AW];
#pragma unroll
    for (int i = 0; i < AW; ++i) cand[i] = af[i] | ou[i];
    if (has_tail && any_bit<AW>(cand)) {
      const uint64_t b = db.off[c] + HEAD_K, e = db.off[c + 1];
      for (uint64_t k = b; k < e; ++k) {
        group_step<MODE, AW>(pv, __ldg(db.lits + k), af, ou);
#pragma unroll
        for (int i = 0; i < AW; ++i) cand[i] = af[i] | ou[i];
        if (!any_bit<AW>(cand)) break;
      }
    }

    // ---- stage B: exact test of each surviving group, warp-aggregated append
    while (__any_sync(FULL, any_bit<AW>(cand))) {
      uint32_t g = 0u, res = 0u;
      if (any_bit<AW>(cand)) {
        bool found = false;
#pragma unroll
        for (int i = 0; i < AW; ++i) {
          if (!found && cand[i] != 0u) {
            g = 32u * i + (uint32_t)(__ffs(cand[i]) - 1);
            cand[i] &= cand[i] - 1u;
            found = true;
          }
        }
        res = exact_word<MODE>(db, pv, c, l, has_tail, g);
      }
      warp_append(res != 0u, (uint32_t)c, g, res, lane, rec, cap, &st->n_records);
    }
  }
}

template <int MODE, int AW>
void launch_one(const ClauseView& db, uint64_t c_lo, uint64_t c_hi, const PlaneView& pv, gss_report* rec,
                uint64_t cap, DevStatus* st, int grid, cudaStream_t s) {
  k_test<MODE, AW><<<grid, TEST_THREADS, 0, s>>>(db, c_lo, c_hi, pv, rec, cap, st);
}

template <int MODE, int AW>
int grid_for(int n_sms) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_test<MODE, AW>, TEST_THREADS, 0) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  return per_sm * n_sms;
}

}  // namespace

cudaError_t launch_test(int mode, const ClauseView& db, uint64_t c_lo, uint64_t c_hi, const PlaneView& pv,
                        gss_report* rec, uint64_t cap, DevStatus* st, int grid, cudaStream_t s) {
  if (c_hi <= c_lo) return cudaSuccess;
  const uint64_t tiles = (c_hi - c_lo + 31) / 32;
  const uint64_t max_blocks = (tiles + (TEST_THREADS / 32) - 1) / (TEST_THREADS / 32);
  if ((uint64_t)grid > max_blocks) grid = (int)max_blocks;
  if (grid < 1) grid = 1;
  if (mode == GSS_MODE_ALLF) {
    if (pv.AWp == 1) launch_one<GSS_MODE_ALLF, 1>(db, c_lo, c_hi, pv, rec, cap, st, grid, s);
    else if (pv.AWp == 2) launch_one<GSS_MODE_ALLF, 2>(db, c_lo, c_hi, pv, rec, cap, st, grid, s);
    else launch_one<GSS_MODE_ALLF, 4>(db, c_lo, c_hi, pv, rec, cap, st, grid, s);
  } else {
    if (pv.AWp == 1) launch_one<GSS_MODE_TRIGGER, 1>(db, c_lo, c_hi, pv, rec, cap, st, grid, s);
    else if (pv.AWp == 2) launch_one<GSS_MODE_TRIGGER, 2>(db, c_lo, c_hi, pv, rec, cap, st, grid, s);
    else launch_one<GSS_MODE_TRIGGER, 4>(db, c_lo, c_hi, pv, rec, cap, st, grid, s);
  }
  return cudaGetLastError();
}

int test_grid_size(int mode, uint32_t AWp, int n_sms) {
  if (mode == GSS_MODE_ALLF) {
    if (AWp == 1) return grid_for<GSS_MODE_ALLF, 1>(n_sms);
    if (AWp == 2) return grid_for<GSS_MODE_ALLF, 2>(n_sms);
    return grid_for<GSS_MODE_ALLF, 4>(n_sms);
  }
  if (AWp == 1) return grid_for<GSS_MODE_TRIGGER, 1>(n_sms);
  if (AWp == 2) return grid_for<GSS_MODE_TRIGGER, 2>(n_sms);
  return grid_for<GSS_MODE_TRIGGER, 4>(n_sms);
}

}  // namespace gss
