// k_route.cu -- routing the records of one serving launch back to its requests.
//
// A serving launch tests up to 32 requests at once, one plane word each, and its test
// kernel appends (clause, word, mask) records in no order.  Routing groups them by word,
// so that each request's records form one contiguous run, clears the bits of padded
// assignments (rows past a request's own assignments are U), drops records left without
// a bit and writes word 0 (the request's own word).  Two grid-stride passes: a per-word
// count, then a scatter behind per-word cursors; the destination may be mapped host memory,
// so results reach the host without a second copy.  k_copy_records moves a context's records
// the same way (gss_fetch_reports_async).
#include "gss_internal.h"

namespace gss {
namespace {

constexpr int RT_THREADS = 256;

__global__ void __launch_bounds__(RT_THREADS) k_route_count(const gss_report* __restrict__ rec,
                                                            const DevStatus* __restrict__ st, uint64_t cap,
                                                            const uint32_t* __restrict__ nmask, uint32_t k,
                                                            unsigned long long* __restrict__ count) {
  __shared__ unsigned int h[32];
  if (threadIdx.x < 32) h[threadIdx.x] = 0u;
  __syncthreads();
  const uint64_t n = st->n_records < cap ? st->n_records : cap;
  const uint64_t stride = (uint64_t)gridDim.x * RT_THREADS;
  // trip count uniform over the warp so that every lane takes part in the match
  for (uint64_t base = (uint64_t)blockIdx.x * RT_THREADS; base < n; base += stride) {
    const uint64_t i = base + threadIdx.x;
    uint32_t w = 0xFFFFFFFFu;
    if (i < n) {
      const gss_report r = rec[i];
      if (r.word < k && (r.mask & nmask[r.word]) != 0u) w = r.word;
    }
    const uint32_t peers = __match_any_sync(0xFFFFFFFFu, w);
    if (w != 0xFFFFFFFFu && (threadIdx.x & 31u) == (uint32_t)(__ffs(peers) - 1))
      atomicAdd(&h[w], (unsigned int)__popc(peers));
  }
  __syncthreads();
  if (threadIdx.x < k && h[threadIdx.x]) atomicAdd(&count[threadIdx.x], (unsigned long long)h[threadIdx.x]);
}

__global__ void __launch_bounds__(RT_THREADS) k_route_scatter(const gss_report* __restrict__ rec,
                                                              const DevStatus* __restrict__ st, uint64_t cap,
                                                              const uint32_t* __restrict__ nmask, uint32_t k,
                                                              const unsigned long long* __restrict__ count,
                                                              unsigned long long* __restrict__ cursor,
                                                              gss_report* __restrict__ out) {
  __shared__ unsigned long long first[32];
  if (threadIdx.x == 0) {
    unsigned long long s = 0;
    for (uint32_t w = 0; w < 32; ++w) {
      first[w] = s;
      if (w < k) s += count[w];
    }
  }
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t n = st->n_records < cap ? st->n_records : cap;
  const uint64_t stride = (uint64_t)gridDim.x * RT_THREADS;
  for (uint64_t base = (uint64_t)blockIdx.x * RT_THREADS; base < n; base += stride) {
    const uint64_t i = base + threadIdx.x;
    uint32_t w = 0xFFFFFFFFu, mask = 0u, c = 0u;
    if (i < n) {
      const gss_report r = rec[i];
      if (r.word < k) {
        mask = r.mask & nmask[r.word];
        if (mask) {
          w = r.word;
          c = r.clause_id;
        }
      }
    }
    const uint32_t peers = __match_any_sync(0xFFFFFFFFu, w);
    const int leader = __ffs(peers) - 1;
    unsigned long long at = 0;
    if (w != 0xFFFFFFFFu && (int)lane == leader) at = atomicAdd(&cursor[w], (unsigned long long)__popc(peers));
    at = __shfl_sync(0xFFFFFFFFu, at, leader);
    if (w != 0xFFFFFFFFu) {
      gss_report r;
      r.clause_id = c;
      r.word = 0u;
      r.mask = mask;
      out[first[w] + at + (unsigned long long)__popc(peers & ((1u << lane) - 1u))] = r;
    }
  }
}

// Copy min(records of the test, cap_dev, cap_out) records into out, which may be host memory
// the GPU can write (pinned or mapped): the records travel as the copy runs, on the test's
// stream, with no device-to-host copy call that would need the count first.
__global__ void __launch_bounds__(RT_THREADS) k_copy_records(const uint32_t* __restrict__ rec,
                                                             const DevStatus* __restrict__ st, uint64_t cap_dev,
                                                             uint64_t cap_out, uint32_t* __restrict__ out) {
  uint64_t n = st->n_records;
  if (n > cap_dev) n = cap_dev;
  if (n > cap_out) n = cap_out;
  const uint64_t words = 3ull * n;
  for (uint64_t i = (uint64_t)blockIdx.x * RT_THREADS + threadIdx.x; i < words; i += (uint64_t)gridDim.x * RT_THREADS)
    out[i] = __ldg(rec + i);
}

}  // namespace

cudaError_t launch_copy_records(const gss_report* rec, const DevStatus* st, uint64_t cap_dev, uint64_t cap_out,
                                gss_report* out, int grid, cudaStream_t s) {
  if (cap_out == 0) return cudaSuccess;
  k_copy_records<<<grid, RT_THREADS, 0, s>>>(reinterpret_cast<const uint32_t*>(rec), st, cap_dev, cap_out,
                                             reinterpret_cast<uint32_t*>(out));
  return cudaGetLastError();
}

cudaError_t launch_route(const gss_report* rec, const DevStatus* st, uint64_t cap, const uint32_t* nmask, uint32_t k,
                         unsigned long long* count, unsigned long long* cursor, gss_report* out, int grid,
                         cudaStream_t s) {
  if (k == 0 || k > 32) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(count, 0, 32 * sizeof(unsigned long long), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(cursor, 0, 32 * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  k_route_count<<<grid, RT_THREADS, 0, s>>>(rec, st, cap, nmask, k, count);
  k_route_scatter<<<grid, RT_THREADS, 0, s>>>(rec, st, cap, nmask, k, count, cursor, out);
  return cudaGetLastError();
}

}  // namespace gss
