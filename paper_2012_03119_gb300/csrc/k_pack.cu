// k_pack.cu -- pack three-valued assignments into literal-indexed bit planes.
//
// Section 3.4 represents the values A_i(v) of N assignments by N-bit words per
// variable (isTrue, isSet), 32 assignments per machine word.  The test only ever
// asks "is literal l F under assignment i", so this kernel stores that question's
// answer directly, one row per LITERAL:
//   P[2v][w]   bit j = (A_{32w+j}(v) == F)   -- literal v is F
//   P[2v+1][w] bit j = (A_{32w+j}(v) == T)   -- literal not v is F
// U sets neither bit (the paper's "isTrue might be set or not for U" is resolved
// to 0, and not-v is read from isTrue masked by isSet rather than ~isTrue).
// Section 4.2's aggregate of a 32-assignment group g is derived in the same pass:
//   aggF[l] bit g = (P[l][g] != 0)      -- F is in G(l)
//   aggU[v] bit g = some assignment of group g leaves v U   -- U is in G(v)
//
// Input: value codes [N][pitch] bytes (0 = U, 1 = T, 2 = F).  One CTA owns 128
// variables and every assignment word.  Each lane reads 4 codes (one 32-bit word)
// of a row, so a warp reads one 128-byte line per assignment row.  Bits are
// gathered with shifts into four 8-row accumulators and transposed with byte
// permutes; results are staged in shared memory in a layout that is bank-conflict
// free on both the write (by lane) and the coalesced read-out (by plane word).
#include "gss_internal.h"

namespace gss {
namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr int PK_VT = 128;                // variables per CTA (4 per lane)
constexpr int PK_THREADS = 256;           // 8 warps
constexpr int PK_WARPS = PK_THREADS / 32;
constexpr int PK_STRIDE = 2 * PK_VT + 1;  // staged words per plane word (odd => conflict-free read-out)

__device__ __forceinline__ uint32_t valid_bits(uint32_t N, uint32_t w) {
  const uint32_t lo = w * 32u;
  if (lo >= N) return 0u;
  const uint32_t rem = N - lo;
  return rem >= 32u ? FULL : ((1u << rem) - 1u);
}

__global__ void __launch_bounds__(PK_THREADS) k_pack(const uint8_t* __restrict__ codes, uint64_t pitch, uint32_t V,
                                                     uint32_t N, uint32_t Wp, uint32_t AWp, uint32_t* __restrict__ P,
                                                     uint32_t* __restrict__ aggF, uint32_t* __restrict__ aggU,
                                                     DevStatus* st) {
  __shared__ uint32_t stage[32 * PK_STRIDE];
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const uint32_t v0 = blockIdx.x * PK_VT;
  const uint32_t vlane = v0 + 4u * lane;  // first of this lane's 4 variables
  uint32_t bmask = 0;                     // bytes of the lane's word that are real variables
  if (vlane < V) bmask = (V - vlane >= 4u) ? FULL : ((1u << (8u * (V - vlane))) - 1u);
  const uint32_t nv = min((uint32_t)PK_VT, V - v0);
  uint32_t bad = 0;

  for (uint32_t wc = 0; wc < Wp; wc += 32u) {
    const uint32_t nw = min(32u, Wp - wc);  // 4, 8, 16 or 32
    // Phase 1: warp `warp` builds plane words wc + wl for its 128 variables.
    for (uint32_t wl = warp; wl < nw; wl += PK_WARPS) {
      const uint32_t w = wc + wl;
      uint32_t f[4] = {0u, 0u, 0u, 0u}, t[4] = {0u, 0u, 0u, 0u};
      if (bmask != 0u && w * 32u < N) {
        const uint8_t* base = codes + (uint64_t)w * 32u * pitch + vlane;
#pragma unroll
        for (int r = 0; r < 32; ++r) {
          uint32_t x = 0u;
          if (w * 32u + (uint32_t)r < N)
            x = __ldcs(reinterpret_cast<const unsigned int*>(base + (uint64_t)r * pitch)) & bmask;
          bad |= (x & 0xFCFCFCFCu) | (x & (x >> 1) & 0x01010101u);  // code 3 or above
          f[r >> 3] |= ((x >> 1) & 0x01010101u) << (r & 7);         // code 2 = F
          t[r >> 3] |= (x & 0x01010101u) << (r & 7);                // code 1 = T
        }
      }
      // byte k of f[j] holds rows 8j..8j+7 of variable vlane+k; gather the four bytes of each variable
      const uint32_t fa = __byte_perm(f[0], f[1], 0x5140), fb = __byte_perm(f[2], f[3], 0x5140);
      const uint32_t fc = __byte_perm(f[0], f[1], 0x7362), fd = __byte_perm(f[2], f[3], 0x7362);
      const uint32_t ta = __byte_perm(t[0], t[1], 0x5140), tb = __byte_perm(t[2], t[3], 0x5140);
      const uint32_t tc = __byte_perm(t[0], t[1], 0x7362), td = __byte_perm(t[2], t[3], 0x7362);
      uint32_t* sw = stage + wl * PK_STRIDE + lane;
      sw[0 * 32] = __byte_perm(fa, fb, 0x5410);  // variable vlane+0: F word
      sw[1 * 32] = __byte_perm(ta, tb, 0x5410);  //                  T word
      sw[2 * 32] = __byte_perm(fa, fb, 0x7632);  // variable vlane+1
      sw[3 * 32] = __byte_perm(ta, tb, 0x7632);
      sw[4 * 32] = __byte_perm(fc, fd, 0x5410);  // variable vlane+2
      sw[5 * 32] = __byte_perm(tc, td, 0x5410);
      sw[6 * 32] = __byte_perm(fc, fd, 0x7632);  // variable vlane+3
      sw[7 * 32] = __byte_perm(tc, td, 0x7632);
    }
    __syncthreads();
    // Phase 2: coalesced write-out, (variable, word) pairs with the word index fastest.
    const uint32_t total = PK_VT * nw;  // a multiple of 32: every lane runs the same trip count
    for (uint32_t i = threadIdx.x; i < total; i += PK_THREADS) {
      const uint32_t vl = i / nw, wl = i - vl * nw;
      const uint32_t k = vl & 3u, ln = vl >> 2;
      const uint32_t Fw = stage[wl * PK_STRIDE + (2u * k) * 32u + ln];
      const uint32_t Tw = stage[wl * PK_STRIDE + (2u * k + 1u) * 32u + ln];
      const uint32_t w = wc + wl;
      const uint32_t Uw = ~(Fw | Tw) & valid_bits(N, w);
      const uint32_t bF = __ballot_sync(FULL, Fw != 0u);
      const uint32_t bT = __ballot_sync(FULL, Tw != 0u);
      const uint32_t bU = __ballot_sync(FULL, Uw != 0u);
      if (vl < nv) {
        const uint64_t v = v0 + vl;
        P[(2u * v) * Wp + w] = Fw;
        P[(2u * v + 1u) * Wp + w] = Tw;
        if (wl == 0u) {  // this variable's nw words sit in lanes [lane, lane + nw)
          const uint32_t m = nw == 32u ? FULL : ((1u << nw) - 1u);
          const uint32_t u = wc >> 5;
          aggF[(2u * v) * AWp + u] = (bF >> lane) & m;
          aggF[(2u * v + 1u) * AWp + u] = (bT >> lane) & m;
          aggU[v * AWp + u] = (bU >> lane) & m;
        }
      }
    }
    __syncthreads();
  }
  if (bad) atomicOr(&st->bad_code, 1u);
}

}  // namespace

cudaError_t launch_pack(const uint8_t* codes, uint64_t pitch, uint32_t V, uint32_t N, uint32_t Wp, uint32_t AWp,
                        uint32_t* P, uint32_t* aggF, uint32_t* aggU, DevStatus* st, cudaStream_t s) {
  // PAD literal rows 2V, 2V+1: all ones in P and aggF (neutral under AND); aggU row V: zero.
  cudaError_t e = cudaMemsetAsync(P + 2ull * V * Wp, 0xFF, 2ull * Wp * sizeof(uint32_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(aggF + 2ull * V * AWp, 0xFF, 2ull * AWp * sizeof(uint32_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(aggU + (uint64_t)V * AWp, 0, AWp * sizeof(uint32_t), s);
  if (e != cudaSuccess || V == 0) return e;
  const uint32_t grid = (V + PK_VT - 1) / PK_VT;
  k_pack<<<grid, PK_THREADS, 0, s>>>(codes, pitch, V, N, Wp, AWp, P, aggF, aggU, st);
  return cudaGetLastError();
}

}  // namespace gss
