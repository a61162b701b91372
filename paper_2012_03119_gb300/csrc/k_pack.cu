// k_pack.cu -- pack three-valued assignments into literal-indexed bit planes.
//
// Section 3.4 represents the values A_i(v) of N assignments by N-bit words per
// variable (isTrue, isSet), 32 assignments per machine word.  The test only ever
// asks "is literal l F under assignment i", so this kernel stores that question's
// answer directly, one row per LITERAL:
//   P[2v][w]   bit j = (A_{32w+j}(v) == F)   -- literal v is F
//   P[2v+1][w] bit j = (A_{32w+j}(v) == T)   -- literal not v is F
// U sets neither bit (Section 3.4 leaves isTrue free for U; here it is 0, and not-v
// is read from isTrue masked by isSet rather than from ~isTrue).
// Section 4.2's aggregate of a 32-assignment group g is derived in the same pass:
//   aggF[l] bit g = (P[l][g] != 0)      -- F is in G(l)
//   aggU[v] bit g = some assignment of group g leaves v U   -- U is in G(v)
//
// Structure: four persistent CTAs per SM walk (variable tile, pass) units, a pass being 32
// plane words of the tile's 128 variables.  A producer warp streams the value codes
// [N][pitch] as 2-D TMA boxes of 32 assignment rows x 128 variables (4 KiB: one plane word
// of 128 variables) into shared memory; rows past N and variables past V arrive as zeros
// (U).  Word w belongs to consumer warp w % C, which owns D stages of the ring and uses them
// in its own program order, so each full / empty mbarrier is waited on at most one phase
// ahead (a parity wait cannot be fooled by a stage two uses behind).  The C consumer warps
// transpose boxes: a lane takes 4 codes of each of the 32 rows; the F bit (bit 1 of a code
// byte) and the T bit (bit 0) move to bit r % 8 of their byte with one shift and one fused
// and-or each, and byte permutes turn four 8-row accumulators into per-variable words.
// Words are staged in shared memory under an XOR swizzle, so the by-lane write and the
// coalesced 16-byte read-out are both bank-conflict free; each lane ORs its words' aggregate
// bits in registers and merges them once per pass.  The producer keeps loading the next
// unit while consumers write out.
#include <atomic>

#include <cudaTypedefs.h>

#include "gss_internal.h"
#include "gss_ptx.h"

namespace gss {
namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr int PK_VT = 128;                         // variables per box (bytes per box row)
constexpr int PK_ROWS = 32;                        // assignment rows per box: one plane word
// The shape of a CTA: C consumer warps, each owning D ring stages (the ring holds C * D
// boxes), MINB CTAs per SM.  Measured on the 1M-variable x 1024-assignment packing: the
// write-out after each pass is the costly phase, and small CTAs (4 consumers, one stage
// each, 4 CTAs per SM: 279 us) overlap it across CTAs better than large ones (8 consumers,
// 2 stages, 2 CTAs: 366 us; deeper rings with 1 CTA per SM: 430-530 us).
constexpr int PK_CONSUMERS = 4;
constexpr int PK_DEPTH = 1;
constexpr int PK_MINB = 4;
constexpr int PK_PASS = 32;  // plane words staged per pass (a variable's row is written in pieces of this width)
constexpr int PK_BOX = PK_VT * PK_ROWS;            // 4 KiB
// Staged words of a pass: row r = 2 vl + s (variable vl of the tile, literal sign s) holds
// its 32 plane words, word wl at r * 32 + (wl ^ stage_swizzle(r)).  The swizzle makes both
// the transposition's stores (32 lanes: rows 8 lane + c, one word) and the write-out's loads
// (4 consecutive rows x 8 word quads) free of bank conflicts.
constexpr uint32_t BAR_CONSUMERS = 1;              // named barrier of the consumer warps

template <int C, int D, int PW>
struct PackSmem {
  uint8_t ring[C * D][PK_BOX];
  uint32_t stage[2 * PK_VT * PW];
  uint32_t rowid[PK_VT];  // internal id of each variable of the current tile
  uint32_t aggw[3 * PK_VT];  // aggregate bits of the pass: aggF rows (2 vl, 2 vl + 1), then aggU (vl)
  unsigned long long full[C * D], empty[C * D];
  volatile int err;
};

__device__ __forceinline__ uint32_t stage_swizzle(uint32_t r) { return ((r >> 3) + (r & 3u)) & 31u; }

__device__ __forceinline__ uint32_t valid_bits(uint32_t N, uint32_t w) {
  const uint32_t lo = w * 32u;
  if (lo >= N) return 0u;
  const uint32_t rem = N - lo;
  return rem >= 32u ? FULL : ((1u << rem) - 1u);
}

// Units of work: (variable tile t, pass p) for u = t * n_pass + p, walked grid-stride by
// every CTA (u = blockIdx.x, blockIdx.x + gridDim.x, ...).  A pass is PW plane words of the
// tile's 128 variables, so wide assignment sets split into many units and the last round of
// CTAs is short; with one pass per tile a unit is a whole tile.  (Tile-major order keeps the
// CTAs that run at the same time on fewer tiles; pass-major order measured 3-4 % slower.)
__device__ __forceinline__ uint32_t unit_tile(uint32_t u, uint32_t n_pass) { return u / n_pass; }
__device__ __forceinline__ uint32_t unit_pass(uint32_t u, uint32_t n_pass) { return u % n_pass; }

template <int C, int D, int MINB, int PW>
__global__ void __launch_bounds__(32 * (C + 1), MINB) k_pack(const __grid_constant__ CUtensorMap tmap, uint32_t V,
                                                        uint32_t N, uint32_t Wp, uint32_t AWp,
                                                        const uint32_t* __restrict__ map,
                                                        const uint32_t* __restrict__ word_rows,
                                                        const uint32_t* __restrict__ word_valid,
                                                        uint32_t* __restrict__ P, uint32_t* __restrict__ aggF,
                                                        uint32_t* __restrict__ aggU, DevStatus* st) {
  // the consumer threads load the row ids of a whole tile: one thread per variable
  static_assert(32 * C >= PK_VT, "k_pack needs at least PK_VT / 32 consumer warps");
  static_assert(PW >= 4 && PW <= 32 && (PW & (PW - 1)) == 0 && PW % C == 0, "pass width");
  extern __shared__ uint8_t smem_raw[];
  PackSmem<C, D, PW>& S = *reinterpret_cast<PackSmem<C, D, PW>*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  const uint32_t n_vt = (V + PK_VT - 1) / PK_VT;
  const uint32_t Wd = (N + 31) / 32;  // plane words that hold assignments
  const uint32_t n_pass = (Wp + PW - 1) / PW;
  const uint32_t n_units = n_vt * n_pass;  // V < 2^32 and Wp <= 1024: below 2^30
  if (threadIdx.x == 0) {
    for (int s = 0; s < C * D; ++s) {
      ptx::mbar_init(&S.full[s], 1);
      ptx::mbar_init(&S.empty[s], 1);
    }
    S.err = 0;
    ptx::fence_mbar_init();
  }
  for (uint32_t i = threadIdx.x; i < 3u * PK_VT; i += blockDim.x) S.aggw[i] = 0u;
  if (blockIdx.x == 0) {  // PAD literal rows 2V, 2V + 1: all ones in P and aggF (neutral under AND); aggU row V: zero
    for (uint32_t i = threadIdx.x; i < 2u * Wp; i += blockDim.x) P[2ull * V * Wp + i] = FULL;
    for (uint32_t i = threadIdx.x; i < 2u * AWp; i += blockDim.x) aggF[2ull * V * AWp + i] = FULL;
    for (uint32_t i = threadIdx.x; i < AWp; i += blockDim.x) aggU[(uint64_t)V * AWp + i] = 0u;
  }
  __syncthreads();

  if (warp == C) {  // ---------------- producer
    if (lane == 0) {
      ptx::prefetch_tensormap(&tmap);
      uint32_t uses[C * D];  // loads issued into each stage so far
      uint32_t cnt[C];       // boxes issued to each consumer warp so far
      for (int s = 0; s < C * D; ++s) uses[s] = 0u;
      for (int q = 0; q < C; ++q) cnt[q] = 0u;
      bool ok = true;
      for (uint32_t u = blockIdx.x; u < n_units && ok; u += gridDim.x) {
        const uint32_t t = unit_tile(u, n_pass), wc = unit_pass(u, n_pass) * PW;
        const uint32_t we = min(wc + (uint32_t)PW, Wd);
        for (uint32_t w = wc; w < we; ++w) {
          // word w goes to consumer q = w % C; its m-th box of this CTA uses stage q + C (m % D)
          const uint32_t q = w % C;
          uint32_t s = q;
          if constexpr (D > 1) s += C * (cnt[q] % D);
          if (uses[s] > 0u) ok = ptx::mbar_wait(&S.empty[s], (uses[s] - 1u) & 1u);  // previous use consumed
          if (!ok || S.err) { ok = false; break; }
          ptx::mbar_expect_tx(&S.full[s], PK_BOX);
          const uint32_t row0 = word_rows ? __ldg(word_rows + w) : w * PK_ROWS;  // first code row of word w
          ptx::tma_load_2d(S.ring[s], &tmap, (int32_t)(t * PK_VT), (int32_t)row0, &S.full[s]);
          ++uses[s];
          if constexpr (D > 1) ++cnt[q];
        }
      }
      if (!ok) {
        S.err = 1;
        atomicOr(&st->timeout, 1u);
      }
      // every issued box must have landed before the CTA may exit (bounded)
      for (int s = 0; s < C * D; ++s)
        if (uses[s] > 0u) ptx::mbar_wait(&S.full[s], (uses[s] - 1u) & 1u);
    }
    return;
  }

  // ---------------- consumers
  uint32_t bad = 0;
  // internal row ids of the next unit's variables, loaded one unit ahead (threads < PK_VT)
  auto row_of = [&](uint32_t u) -> uint32_t {
    const uint32_t v = unit_tile(u, n_pass) * PK_VT + threadIdx.x;
    return v < V ? (map ? __ldg(map + v) : v) : 0u;
  };
  uint32_t next_row = (threadIdx.x < PK_VT && blockIdx.x < n_units) ? row_of(blockIdx.x) : 0u;
  uint32_t m = 0;  // boxes this consumer warp has taken so far (its m-th sits in stage warp + C (m % D))
  uint32_t cur_t = 0xFFFFFFFFu;
  for (uint32_t u = blockIdx.x; u < n_units; u += gridDim.x) {
    const uint32_t t = unit_tile(u, n_pass);
    const uint32_t v0 = t * PK_VT;
    const uint32_t nv = min((uint32_t)PK_VT, V - v0);
    {
      const uint32_t wc = unit_pass(u, n_pass) * PW;
      const uint32_t nw = min((uint32_t)PW, Wp - wc);  // 4 .. PW words in this pass
      const uint32_t lg_nw = 31u - __clz(nw);
      if (threadIdx.x < PK_VT) {  // row ids of this unit's tile, read by the write-out after the next barrier
        if (t != cur_t) S.rowid[threadIdx.x] = next_row;
        if (u + gridDim.x < n_units) next_row = row_of(u + gridDim.x);
      }
      cur_t = t;
      // aggregate bits of this lane's 4 variables over the pass's words it transposes
      uint32_t aF[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u}, aU[4] = {0u, 0u, 0u, 0u};
      for (uint32_t wl = warp; wl < nw; wl += C) {
        const uint32_t w = wc + wl;
        uint32_t f[4] = {0u, 0u, 0u, 0u}, tt[4] = {0u, 0u, 0u, 0u};
        if (w < Wd) {
          const uint32_t s = warp + C * (m % D);
          bool ok = !S.err && ptx::mbar_wait(&S.full[s], (m / D) & 1u);
          ++m;
          if (!__all_sync(FULL, ok)) {
            if (lane == 0 && !S.err) {
              S.err = 1;
              atomicOr(&st->timeout, 1u);
            }
          } else {
            const uint8_t* box = S.ring[s] + 4u * lane;
            uint32_t any = 0u;
#pragma unroll
            for (int r = 0; r < 32; ++r) {
              const uint32_t x = *reinterpret_cast<const uint32_t*>(box + r * PK_VT);
              const int sh = r & 7;
              any |= x;
              if (sh == 0) f[r >> 3] |= (x >> 1) & 0x01010101u;
              else f[r >> 3] |= (x << (sh - 1)) & (0x01010101u << sh);
              tt[r >> 3] |= (x << sh) & (0x01010101u << sh);
            }
            // invalid codes: a bit above bit 1 of a byte, or code 3 (F and T bits both set);
            // flagged per plane word (mod 32) so that a caller can tell which word held them
            if ((any & 0xFCFCFCFCu) | (f[0] & tt[0]) | (f[1] & tt[1]) | (f[2] & tt[2]) | (f[3] & tt[3]))
              bad |= 1u << (w & 31u);
          }
          __syncwarp();
          if (lane == 0) ptx::mbar_arrive(&S.empty[s]);  // the box may be overwritten now
        }
        // byte k of f[j] holds rows 8j..8j+7 of variable v0 + 4 lane + k
        const uint32_t fa = __byte_perm(f[0], f[1], 0x5140), fb = __byte_perm(f[2], f[3], 0x5140);
        const uint32_t fc = __byte_perm(f[0], f[1], 0x7362), fd = __byte_perm(f[2], f[3], 0x7362);
        const uint32_t ta = __byte_perm(tt[0], tt[1], 0x5140), tb = __byte_perm(tt[2], tt[3], 0x5140);
        const uint32_t tc = __byte_perm(tt[0], tt[1], 0x7362), td = __byte_perm(tt[2], tt[3], 0x7362);
        // word (variable 4 lane + k, literal sign s) sits at index 2 k + s; staged at (2 k + s) * 32 + lane
        uint32_t x[8];
        x[0] = __byte_perm(fa, fb, 0x5410);
        x[1] = __byte_perm(ta, tb, 0x5410);
        x[2] = __byte_perm(fa, fb, 0x7632);
        x[3] = __byte_perm(ta, tb, 0x7632);
        x[4] = __byte_perm(fc, fd, 0x5410);
        x[5] = __byte_perm(tc, td, 0x5410);
        x[6] = __byte_perm(fc, fd, 0x7632);
        x[7] = __byte_perm(tc, td, 0x7632);
        // bit of the word in its aggregate word; rows of the word that are real assignments
        const uint32_t bit = 1u << (w & 31u);
        const uint32_t vw = valid_bits(N, w) & ((word_valid && w < Wd) ? __ldg(word_valid + w) : FULL);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const uint32_t r = 8u * lane + (uint32_t)j;  // row of (variable 4 lane + j / 2, sign j % 2)
          S.stage[r * PW + (wl ^ (stage_swizzle(r) & (PW - 1u)))] = x[j];
          aF[j] |= x[j] != 0u ? bit : 0u;  // F is in G(l)
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) aU[k] |= (~(x[2 * k] | x[2 * k + 1]) & vw) != 0u ? bit : 0u;  // U is in G(v)
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {  // merge the consumers' bits
        const uint32_t vl = 4u * lane + (uint32_t)k;
        if (aF[2 * k]) atomicOr(&S.aggw[2u * vl], aF[2 * k]);
        if (aF[2 * k + 1]) atomicOr(&S.aggw[2u * vl + 1u], aF[2 * k + 1]);
        if (aU[k]) atomicOr(&S.aggw[2u * PK_VT + vl], aU[k]);
      }
      ptx::named_bar_sync(BAR_CONSUMERS, 32 * C);
      // coalesced write-out: one 16-byte store per 4 words of a row, quads fastest
      const uint32_t lg_nq = lg_nw - 2u;  // nw >= 4
      const uint32_t total = 2u * PK_VT << lg_nq;
      for (uint32_t i = threadIdx.x; i < total; i += 32 * C) {
        const uint32_t r = i >> lg_nq, q = i & ((1u << lg_nq) - 1u);
        const uint32_t vl = r >> 1, sw = stage_swizzle(r) & (PW - 1u);
        const uint32_t* row = S.stage + r * PW;
        uint4 x4;
        x4.x = row[(4u * q) ^ sw];
        x4.y = row[(4u * q + 1u) ^ sw];
        x4.z = row[(4u * q + 2u) ^ sw];
        x4.w = row[(4u * q + 3u) ^ sw];
        if (vl < nv) {
          const uint64_t v = S.rowid[vl];  // internal row of variable v0 + vl
          *reinterpret_cast<uint4*>(P + (2u * v + (r & 1u)) * Wp + wc + 4u * q) = x4;
        }
      }
      const bool agg_done = ((wc + nw) & 31u) == 0u || wc + nw >= Wp;  // the pass ends an aggregate word
      if (agg_done && threadIdx.x < PK_VT) {  // one aggregate word per row; cleared for the next one
        const uint32_t vl = threadIdx.x;
        const uint32_t gF = S.aggw[2u * vl], gT = S.aggw[2u * vl + 1u], gU = S.aggw[2u * PK_VT + vl];
        S.aggw[2u * vl] = 0u;
        S.aggw[2u * vl + 1u] = 0u;
        S.aggw[2u * PK_VT + vl] = 0u;
        if (vl < nv) {
          const uint64_t v = S.rowid[vl];
          const uint32_t u = wc >> 5;
          aggF[(2u * v) * AWp + u] = gF;
          aggF[(2u * v + 1u) * AWp + u] = gT;
          aggU[v * AWp + u] = gU;
        }
      }
      ptx::named_bar_sync(BAR_CONSUMERS, 32 * C);
    }
  }
  if (bad) atomicOr(&st->bad_code, bad);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// Launch k_pack<C, D, MINB> over every variable tile: MINB persistent CTAs per SM.
template <int C, int D, int MINB, int PW = PK_PASS>
cudaError_t launch_pack_cfg(const CUtensorMap& tmap, uint32_t V, uint32_t N, uint32_t Wp, uint32_t AWp,
                            const uint32_t* map, const uint32_t* word_rows, const uint32_t* word_valid, uint32_t* P,
                            uint32_t* aggF, uint32_t* aggU, DevStatus* st, cudaStream_t s) {
  const size_t smem = sizeof(PackSmem<C, D, PW>) + 128;
  int dev = 0, n_sms = 1;
  cudaGetDevice(&dev);
  static std::atomic<bool> smem_set[64];  // once per device, before any graph capture that packs
  if (dev < 0 || dev >= 64 || !smem_set[dev].load(std::memory_order_acquire)) {
    const cudaError_t e =
        cudaFuncSetAttribute(k_pack<C, D, MINB, PW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) smem_set[dev].store(true, std::memory_order_release);
  }
  cudaDeviceGetAttribute(&n_sms, cudaDevAttrMultiProcessorCount, dev);
  const uint32_t n_units = ((V + PK_VT - 1) / PK_VT) * ((Wp + PW - 1) / PW);
  const uint32_t slots = (uint32_t)MINB * (uint32_t)n_sms;
  const uint32_t grid = n_units < slots ? n_units : slots;
  k_pack<C, D, MINB, PW><<<grid, 32 * (C + 1), smem, s>>>(tmap, V, N, Wp, AWp, map, word_rows, word_valid, P, aggF,
                                                          aggU, st);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_pack_rows(const uint8_t* codes, uint64_t pitch, uint32_t V, uint32_t N, uint32_t Wp,
                             uint32_t AWp, const uint32_t* map, const uint32_t* word_rows, uint32_t code_rows,
                             uint32_t* P, uint32_t* aggF, uint32_t* aggU, DevStatus* st, cudaStream_t s,
                             const uint32_t* word_valid) {
  if (V == 0 || N == 0) {  // no kernel: the PAD literal rows still have to be set (the kernel writes them otherwise)
    cudaError_t e = cudaMemsetAsync(P + 2ull * V * Wp, 0xFF, 2ull * Wp * sizeof(uint32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(aggF + 2ull * V * AWp, 0xFF, 2ull * AWp * sizeof(uint32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(aggU + (uint64_t)V * AWp, 0, AWp * sizeof(uint32_t), s);
    return e;
  }
  if (pitch % 16 != 0 || reinterpret_cast<uintptr_t>(codes) % 16 != 0) return cudaErrorInvalidValue;
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  CUtensorMap tmap;
  const cuuint64_t dims[2] = {V, word_rows ? code_rows : N};
  const cuuint64_t strides[1] = {pitch};
  const cuuint32_t box[2] = {PK_VT, PK_ROWS};
  const cuuint32_t estr[2] = {1, 1};
  if (enc(&tmap, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<uint8_t*>(codes), dims, strides, box, estr,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  return launch_pack_cfg<PK_CONSUMERS, PK_DEPTH, PK_MINB>(tmap, V, N, Wp, AWp, map, word_rows, word_valid, P, aggF,
                                                         aggU, st, s);
}

cudaError_t launch_pack(const uint8_t* codes, uint64_t pitch, uint32_t V, uint32_t N, uint32_t Wp, uint32_t AWp,
                        const uint32_t* map, uint32_t* P, uint32_t* aggF, uint32_t* aggU, DevStatus* st,
                        cudaStream_t s) {
  return launch_pack_rows(codes, pitch, V, N, Wp, AWp, map, nullptr, 0, P, aggF, aggU, st, s);
}

}  // namespace gss
