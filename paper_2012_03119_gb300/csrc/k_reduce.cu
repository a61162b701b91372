// k_reduce.cu -- clause activity upkeep and activity-based deletion (Section 3.6: the GPU
// deletes clauses by activity, as MiniSat does on the CPU, and a clause's activity is bumped
// whenever it triggers; the bump itself happens inside the test kernel).
//
// Deletion keeps every clause of one or two literals and removes the requested number of the
// others with the smallest keys, key = (IEEE bits of the activity) << 32 | clause id: bit
// patterns of non-negative floats order like the floats, and ids make keys unique, so the
// cut is exact.  The key of the last removed clause is found by a radix select, 8 bits per
// pass from the top (launch_key_hist gives one pass's histogram; the host picks the bucket);
// then launch_compact_plan marks the survivors and scans their counts and sizes, and
// launch_compact_copy moves them, in order, into new arrays.
#include "gss_internal.h"

namespace gss {
namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr int SCAN_THREADS = 1024;

unsigned grid_of(uint64_t n, unsigned threads, unsigned cap = 8192) {
  const uint64_t b = (n + threads - 1) / threads;
  return (unsigned)(b < 1 ? 1 : (b < cap ? b : cap));
}

__global__ void k_fill_u32(uint32_t* p, uint64_t n, uint32_t v) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    p[i] = v;
}
__global__ void k_fill_f32(float* p, uint64_t n, float v) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    p[i] = v;
}
__global__ void k_iota_u32(uint32_t* p, uint64_t n, uint32_t first) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    p[i] = first + (uint32_t)i;
}
__global__ void k_invert_u32(const uint32_t* __restrict__ map, uint32_t n, uint32_t* __restrict__ inv) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    inv[map[i]] = (uint32_t)i;
}
__global__ void k_scale_f32(float* p, uint64_t n, float f) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    p[i] = p[i] * f;
}

__device__ __forceinline__ uint64_t key_of(const float* act, const uint32_t* ids, uint64_t c) {
  return ((uint64_t)__float_as_uint(act[c]) << 32) | (uint64_t)(ids ? ids[c] : (uint32_t)c);
}

__global__ void k_key_hist(const uint64_t* __restrict__ off, const float* __restrict__ act,
                           const uint32_t* __restrict__ ids, uint64_t m, uint32_t shift, uint64_t prefix,
                           uint32_t* __restrict__ hist) {
  __shared__ uint32_t h[256];
  for (uint32_t i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0u;
  __syncthreads();
  const uint32_t hi = shift + 8u;  // bits above the pass's byte must equal prefix
  for (uint64_t c = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; c < m; c += (uint64_t)gridDim.x * blockDim.x) {
    if (off[c + 1] - off[c] <= 2) continue;  // short clauses are never removed
    const uint64_t k = key_of(act, ids, c);
    if (hi < 64u && (k >> hi) != prefix) continue;
    atomicAdd(&h[(k >> shift) & 255u], 1u);
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < 256; i += blockDim.x)
    if (h[i]) atomicAdd(&hist[i], h[i]);
}

// Inclusive scan of (count, literals) pairs over a block of SCAN_THREADS threads.
__device__ __forceinline__ void block_scan2(unsigned long long& a, unsigned long long& b,
                                            unsigned long long* sa, unsigned long long* sb) {
  const uint32_t lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const unsigned long long ya = __shfl_up_sync(FULL, a, d), yb = __shfl_up_sync(FULL, b, d);
    if (lane >= (uint32_t)d) {
      a += ya;
      b += yb;
    }
  }
  if (lane == 31) {
    sa[w] = a;
    sb[w] = b;
  }
  __syncthreads();
  if (w == 0) {
    unsigned long long xa = sa[lane], xb = sb[lane];  // 32 warps per block
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const unsigned long long ya = __shfl_up_sync(FULL, xa, d), yb = __shfl_up_sync(FULL, xb, d);
      if (lane >= (uint32_t)d) {
        xa += ya;
        xb += yb;
      }
    }
    sa[lane] = xa;
    sb[lane] = xb;
  }
  __syncthreads();
  if (w > 0) {
    a += sa[w - 1];
    b += sb[w - 1];
  }
}

// Phase 1: per clause, keep flag and kept size; block-local exclusive prefixes; block totals.
__global__ void __launch_bounds__(SCAN_THREADS) k_plan_blocks(const uint64_t* __restrict__ off,
                                                              const float* __restrict__ act,
                                                              const uint32_t* __restrict__ ids, uint64_t m,
                                                              uint64_t kmax, unsigned long long* __restrict__ pos,
                                                              unsigned long long* __restrict__ loff,
                                                              unsigned long long* __restrict__ bsum) {
  __shared__ unsigned long long sa[32], sb[32];
  const uint64_t c = blockIdx.x * (uint64_t)SCAN_THREADS + threadIdx.x;
  unsigned long long keep = 0, size = 0;
  if (c < m) {
    size = off[c + 1] - off[c];
    keep = (size <= 2 || key_of(act, ids, c) > kmax) ? 1ull : 0ull;
    size = keep ? size : 0ull;
  }
  unsigned long long a = keep, b = size;
  block_scan2(a, b, sa, sb);
  if (c < m) {
    pos[c] = a - keep;  // exclusive prefixes within the block
    loff[c] = b - size;
  }
  if (threadIdx.x == SCAN_THREADS - 1) {
    bsum[2 * blockIdx.x] = a;
    bsum[2 * blockIdx.x + 1] = b;
  }
}

// Phase 2 (one block): exclusive scan of the block totals, in place; grand totals to counts.
__global__ void __launch_bounds__(SCAN_THREADS) k_plan_sums(unsigned long long* __restrict__ bsum, uint32_t nb,
                                                            unsigned long long* __restrict__ counts) {
  __shared__ unsigned long long sa[32], sb[32];
  __shared__ unsigned long long carry[2];
  if (threadIdx.x == 0) carry[0] = carry[1] = 0ull;
  __syncthreads();
  for (uint32_t base = 0; base < nb; base += SCAN_THREADS) {
    const uint32_t i = base + threadIdx.x;
    const unsigned long long va = i < nb ? bsum[2 * i] : 0ull, vb = i < nb ? bsum[2 * i + 1] : 0ull;
    unsigned long long a = va, b = vb;
    block_scan2(a, b, sa, sb);
    const unsigned long long ca = carry[0], cb = carry[1];
    if (i < nb) {
      bsum[2 * i] = ca + a - va;
      bsum[2 * i + 1] = cb + b - vb;
    }
    __syncthreads();
    if (threadIdx.x == SCAN_THREADS - 1) {
      carry[0] = ca + a;
      carry[1] = cb + b;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    counts[0] = carry[0];
    counts[1] = carry[1];
  }
}

// Phase 3: move each kept clause to its new place.
__global__ void k_compact_copy(const uint64_t* __restrict__ off, const uint32_t* __restrict__ lits,
                               const uint32_t* __restrict__ head0, const uint32_t* __restrict__ head1,
                               const float* __restrict__ act, const uint32_t* __restrict__ stamp,
                               const uint32_t* __restrict__ ids, uint64_t m, uint64_t kmax,
                               const unsigned long long* __restrict__ pos, const unsigned long long* __restrict__ loff,
                               const unsigned long long* __restrict__ bsum, uint64_t* __restrict__ noff,
                               uint32_t* __restrict__ nlits, uint32_t* __restrict__ nhead0,
                               uint32_t* __restrict__ nhead1, float* __restrict__ nact, uint32_t* __restrict__ nstamp,
                               uint32_t* __restrict__ nids) {
  for (uint64_t c = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; c < m; c += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t b = off[c], size = off[c + 1] - b;
    if (!(size <= 2 || key_of(act, ids, c) > kmax)) continue;
    const uint64_t blk = c / SCAN_THREADS;
    const uint64_t p = bsum[2 * blk] + pos[c], o = bsum[2 * blk + 1] + loff[c];
    noff[p + 1] = o + size;
    for (uint64_t k = 0; k < size; ++k) nlits[o + k] = lits[b + k];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      nhead0[p * 8 + j] = head0[c * 8 + j];
      nhead1[p * 8 + j] = head1[c * 8 + j];
    }
    nact[p] = act[c];
    nstamp[p] = stamp[c];
    nids[p] = ids ? ids[c] : (uint32_t)c;
  }
}

}  // namespace

cudaError_t launch_fill_u32(uint32_t* p, uint64_t n, uint32_t v, cudaStream_t s) {
  if (n) k_fill_u32<<<grid_of(n, 256), 256, 0, s>>>(p, n, v);
  return cudaGetLastError();
}
cudaError_t launch_fill_f32(float* p, uint64_t n, float v, cudaStream_t s) {
  if (n) k_fill_f32<<<grid_of(n, 256), 256, 0, s>>>(p, n, v);
  return cudaGetLastError();
}
cudaError_t launch_iota_u32(uint32_t* p, uint64_t n, uint32_t first, cudaStream_t s) {
  if (n) k_iota_u32<<<grid_of(n, 256), 256, 0, s>>>(p, n, first);
  return cudaGetLastError();
}
cudaError_t launch_invert_u32(const uint32_t* map, uint32_t n, uint32_t* inv, cudaStream_t s) {
  if (n) k_invert_u32<<<grid_of(n, 256), 256, 0, s>>>(map, n, inv);
  return cudaGetLastError();
}
cudaError_t launch_scale_f32(float* p, uint64_t n, float f, cudaStream_t s) {
  if (n) k_scale_f32<<<grid_of(n, 256), 256, 0, s>>>(p, n, f);
  return cudaGetLastError();
}

cudaError_t launch_key_hist(const uint64_t* off, const float* act, const uint32_t* ids, uint64_t m, uint32_t shift,
                            uint64_t prefix, uint32_t* hist, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(hist, 0, 256 * sizeof(uint32_t), s);
  if (e != cudaSuccess) return e;
  if (m) k_key_hist<<<grid_of(m, 256, 2048), 256, 0, s>>>(off, act, ids, m, shift, prefix, hist);
  return cudaGetLastError();
}

uint64_t compact_scratch_bytes(uint64_t m) {
  const uint64_t nb = (m + SCAN_THREADS - 1) / SCAN_THREADS;
  return (2 * m + 2 * (nb ? nb : 1)) * sizeof(unsigned long long);
}

cudaError_t launch_compact_plan(const uint64_t* off, const float* act, const uint32_t* ids, uint64_t m, uint64_t kmax,
                                void* scratch, unsigned long long* d_counts, cudaStream_t s) {
  unsigned long long* pos = static_cast<unsigned long long*>(scratch);
  unsigned long long* loff = pos + m;
  unsigned long long* bsum = loff + m;
  const uint64_t nb = (m + SCAN_THREADS - 1) / SCAN_THREADS;
  if (nb >= (1ull << 32)) return cudaErrorInvalidValue;
  if (m) k_plan_blocks<<<(unsigned)nb, SCAN_THREADS, 0, s>>>(off, act, ids, m, kmax, pos, loff, bsum);
  k_plan_sums<<<1, SCAN_THREADS, 0, s>>>(bsum, (uint32_t)nb, d_counts);
  return cudaGetLastError();
}

cudaError_t launch_compact_copy(const uint64_t* off, const uint32_t* lits, const uint32_t* head0,
                                const uint32_t* head1, const float* act, const uint32_t* stamp, const uint32_t* ids,
                                uint64_t m, uint64_t kmax, const void* scratch, uint64_t* noff, uint32_t* nlits,
                                uint32_t* nhead0, uint32_t* nhead1, float* nact, uint32_t* nstamp, uint32_t* nids,
                                cudaStream_t s) {
  const unsigned long long* pos = static_cast<const unsigned long long*>(scratch);
  const unsigned long long* loff = pos + m;
  const unsigned long long* bsum = loff + m;
  if (m)
    k_compact_copy<<<grid_of(m, 256), 256, 0, s>>>(off, lits, head0, head1, act, stamp, ids, m, kmax, pos, loff, bsum,
                                                    noff, nlits, nhead0, nhead1, nact, nstamp, nids);
  return cudaGetLastError();
}

}  // namespace gss
