// k_ingest.cu -- append a batch of clauses to the resident database.
//
// Section 3.6: every learned clause is exported to the GPU, which keeps all of
// them; Section 3.5 reorders the clause representation in memory so that reads
// coalesce.  Here the CSR (offsets + literals) is kept, and the first HEAD_K
// literals of every clause are copied into a dense, fixed-width head array
// (padded with the neutral PAD literal 2V), as two planes of 8 literals: head0
// (literals 0..7) and head1 (8..15), 32 bytes (one sector) per clause each.  The
// test kernel streams head0 by bulk copies, reads head1 only for clauses still
// alive after 8 literals, and touches the CSR only past 16.
//
// Variable numbering.  Section 7 observes that reads of assignment values would be
// cheaper if the values of variables shared by the clauses tested together were kept
// in shared memory.  The first batch fixes an internal numbering: variables are ranked
// by decreasing occurrence count in a sample of about 4M of the batch's literals (one
// 32-literal chunk in every `stride`; counts bucketed on a log scale with 8 steps per
// octave; ties in variable order), the HOT_VARS top-ranked variables take internal ids
// 0 .. HOT_VARS - 1 in rank order, the variables they displace take the vacated ids, and
// every other variable keeps its id (so the packing kernel's writes stay sequential).
// Literals are stored as 2 id + s and plane rows are written at internal ids, so the
// hottest literals' aggregate rows are contiguous and the test kernel keeps them in
// shared memory.  Results are per clause id and do not depend on the numbering.
#include "gss_internal.h"

namespace gss {
namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr uint32_t RANK_BLOCK = 1024;  // variables per block in the ranking kernels
constexpr uint32_t N_BUCKETS = 256;
constexpr uint32_t HOT_VARS = 1024;   // variables moved to the front of the numbering

__global__ void k_validate(const uint64_t* __restrict__ boff, uint64_t n, uint64_t L, uint64_t L0,
                           uint64_t* __restrict__ off_db, const uint32_t* __restrict__ lits_batch, uint32_t two_v,
                           DevStatus* st) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  uint32_t bad_size = 0, bad_lit = 0;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint64_t b = boff[i], e = boff[i + 1];
    if (!(e > b && e <= L)) bad_size = 1;  // empty clause, decreasing offsets or offsets past the batch
    else off_db[i + 1] = L0 + e;
  }
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < L; i += stride)
    bad_lit |= lits_batch[i] >= two_v ? 1u : 0u;
  if (bad_size) atomicOr(&st->bad_size, 1u);
  if (bad_lit) atomicOr(&st->bad_lit, 1u);
}

// Occurrence count of every variable in the chunks 0, stride, 2 stride, ... of 32
// consecutive literals; lanes holding the same variable add once per warp.  Sampling
// bounds the atomics on the hottest counters: under Zipf(1.1) one variable can hold an
// eighth of all literals.
constexpr uint64_t COUNT_SAMPLE = 4ull << 20;  // literals counted (about)
__global__ void k_count_vars(const uint32_t* __restrict__ lits, uint64_t L, uint64_t stride,
                             uint32_t* __restrict__ cnt) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const uint64_t n_warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  const uint64_t n_chunks = (L + 31) / 32;
  for (uint64_t ch = warp * stride; ch < n_chunks; ch += n_warps * stride) {
    const uint64_t i = ch * 32u + lane;
    const uint32_t v = i < L ? (lits[i] >> 1) : 0xFFFFFFFFu;
    const uint32_t same = __match_any_sync(FULL, v);
    if (v != 0xFFFFFFFFu && lane == (uint32_t)(__ffs(same) - 1)) atomicAdd(&cnt[v], (uint32_t)__popc(same));
  }
}

// Bucket of a count, hottest first: 255 - (8 log2(c + 1) rounded down to eighths of an octave).
__device__ __forceinline__ uint32_t bucket_of(uint32_t c) {
  const uint32_t x = c + 1u;
  const uint32_t lg = 31u - __clz(x);
  const uint32_t frac = lg >= 3u ? (x >> (lg - 3u)) & 7u : (x << (3u - lg)) & 7u;
  const uint32_t key = lg * 8u + frac;
  return 255u - (key > 255u ? 255u : key);
}

__global__ void k_bucket_counts(const uint32_t* __restrict__ cnt, uint32_t V, uint32_t* __restrict__ blockcnt) {
  __shared__ uint32_t h[N_BUCKETS];
  for (uint32_t i = threadIdx.x; i < N_BUCKETS; i += blockDim.x) h[i] = 0u;
  __syncthreads();
  const uint32_t v0 = blockIdx.x * RANK_BLOCK;
  for (uint32_t i = threadIdx.x; i < RANK_BLOCK; i += blockDim.x)
    if (v0 + i < V) atomicAdd(&h[bucket_of(cnt[v0 + i])], 1u);
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < N_BUCKETS; i += blockDim.x) blockcnt[(uint64_t)blockIdx.x * N_BUCKETS + i] = h[i];
}

// One block of N_BUCKETS threads: per bucket, exclusive scan over blocks (in place), then the
// bucket bases (exclusive scan over buckets, hottest first).
__global__ void k_bucket_scan(uint32_t* __restrict__ blockcnt, uint32_t nb, uint32_t* __restrict__ base) {
  __shared__ uint32_t tot[N_BUCKETS];
  const uint32_t b = threadIdx.x;
  uint32_t run = 0;
  for (uint32_t k = 0; k < nb; ++k) {
    const uint32_t x = blockcnt[(uint64_t)k * N_BUCKETS + b];
    blockcnt[(uint64_t)k * N_BUCKETS + b] = run;
    run += x;
  }
  tot[b] = run;
  __syncthreads();
  if (b == 0) {
    uint32_t acc = 0;
    for (uint32_t i = 0; i < N_BUCKETS; ++i) {
      const uint32_t x = tot[i];
      tot[i] = acc;
      acc += x;
    }
  }
  __syncthreads();
  base[b] = tot[b];
}

// One warp per block of RANK_BLOCK variables, chunks of 32 in variable order: the rank of
// variable v is base[bucket] + (earlier blocks' count in the bucket) + (earlier chunks) + (lower lanes).
__global__ void k_assign_ranks(const uint32_t* __restrict__ cnt, uint32_t V, const uint32_t* __restrict__ blockcnt,
                               const uint32_t* __restrict__ base, uint32_t* __restrict__ rank) {
  __shared__ uint32_t ctr[N_BUCKETS + 1];
  const uint32_t lane = threadIdx.x;
  for (uint32_t i = lane; i <= N_BUCKETS; i += 32) ctr[i] = 0u;
  __syncwarp();
  const uint32_t v0 = blockIdx.x * RANK_BLOCK;
  for (uint32_t chunk = 0; chunk < RANK_BLOCK / 32; ++chunk) {
    const uint32_t v = v0 + chunk * 32u + lane;
    const bool ok = v < V;
    const uint32_t b = ok ? bucket_of(cnt[v]) : N_BUCKETS;
    const uint32_t same = __match_any_sync(FULL, b);
    const uint32_t r = __popc(same & ((1u << lane) - 1u));
    const uint32_t before = ctr[b];
    if (ok) rank[v] = base[b] + blockcnt[(uint64_t)blockIdx.x * N_BUCKETS + b] + before + r;
    __syncwarp();
    if (lane == (uint32_t)(__ffs(same) - 1)) ctr[b] = before + (uint32_t)__popc(same);
    __syncwarp();
  }
}

// map[v] = rank[v] for the HOT_VARS top-ranked variables, v otherwise; hot_ids[rank] = v.
__global__ void k_hot_map(const uint32_t* __restrict__ rank, uint32_t V, uint32_t* __restrict__ map,
                          uint32_t* __restrict__ hot_ids) {
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < V; v += gridDim.x * blockDim.x) {
    const uint32_t r = rank[v];
    map[v] = r < HOT_VARS ? r : v;
    if (r < HOT_VARS) hot_ids[r] = v;
  }
}

// One block of HOT_VARS threads: the j-th displaced variable (id < HOT_VARS, not hot, in id
// order) takes the id of the j-th mover (hot variable with id >= HOT_VARS, in rank order).
__global__ void k_fix_displaced(const uint32_t* __restrict__ rank, uint32_t V, const uint32_t* __restrict__ hot_ids,
                                uint32_t* __restrict__ map) {
  __shared__ uint32_t movers[HOT_VARS];
  __shared__ uint32_t sd[HOT_VARS], sm[HOT_VARS];
  const uint32_t t = threadIdx.x, nh = V < HOT_VARS ? V : HOT_VARS;
  const uint32_t fd = (t < nh && rank[t] >= HOT_VARS) ? 1u : 0u;  // displaced
  const uint32_t h = t < nh ? hot_ids[t] : 0u;
  const uint32_t fm = (t < nh && h >= HOT_VARS) ? 1u : 0u;       // mover
  sd[t] = fd;
  sm[t] = fm;
  __syncthreads();
  for (uint32_t d = 1; d < HOT_VARS; d <<= 1) {  // inclusive scans
    const uint32_t a = t >= d ? sd[t - d] : 0u, b = t >= d ? sm[t - d] : 0u;
    __syncthreads();
    sd[t] += a;
    sm[t] += b;
    __syncthreads();
  }
  if (fm) movers[sm[t] - 1u] = h;
  __syncthreads();
  if (fd) map[t] = movers[sd[t] - 1u];
}

__global__ void k_translate(uint32_t* __restrict__ lits, uint64_t L, const uint32_t* __restrict__ map) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < L; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t l = lits[i];
    lits[i] = 2u * __ldg(map + (l >> 1)) + (l & 1u);
  }
}

__global__ void k_build_heads(const uint64_t* __restrict__ boff, uint64_t n, uint64_t L0,
                              uint32_t* __restrict__ head0, uint32_t* __restrict__ head1,
                              const uint32_t* __restrict__ lits_db, uint32_t V) {
  const uint32_t PAD = 2u * V;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t b = boff[i], e = boff[i + 1];
    uint32_t h[HEAD_K];
#pragma unroll
    for (uint32_t k = 0; k < HEAD_K; ++k) h[k] = (b + k < e) ? lits_db[L0 + b + k] : PAD;
    uint4* h0 = reinterpret_cast<uint4*>(head0 + i * 8);
    uint4* h1 = reinterpret_cast<uint4*>(head1 + i * 8);
    h0[0] = make_uint4(h[0], h[1], h[2], h[3]);
    h0[1] = make_uint4(h[4], h[5], h[6], h[7]);
    h1[0] = make_uint4(h[8], h[9], h[10], h[11]);
    h1[1] = make_uint4(h[12], h[13], h[14], h[15]);
  }
}

unsigned grid_for(uint64_t work, unsigned cap = 8192) {
  const uint64_t b = (work + 255) / 256;
  return (unsigned)(b < 1 ? 1 : (b < cap ? b : cap));
}

}  // namespace

uint64_t rank_scratch_words(uint32_t V) {
  const uint64_t nb = (V + RANK_BLOCK - 1) / RANK_BLOCK;
  return 2ull * V + nb * N_BUCKETS + N_BUCKETS + HOT_VARS;
}

cudaError_t launch_validate(const uint64_t* boff, uint64_t n, uint64_t L, uint64_t L0, uint64_t* off_db_at_n0,
                            const uint32_t* lits_batch, uint32_t V, DevStatus* st, cudaStream_t s) {
  if (n || L) k_validate<<<grid_for(n > L ? n : L), 256, 0, s>>>(boff, n, L, L0, off_db_at_n0, lits_batch, 2u * V, st);
  return cudaGetLastError();
}

cudaError_t launch_rank_vars(const uint32_t* lits, uint64_t L, uint32_t V, uint32_t* scratch, uint32_t* map,
                             cudaStream_t s) {
  const uint32_t nb = (V + RANK_BLOCK - 1) / RANK_BLOCK;
  uint32_t* cnt = scratch;
  uint32_t* rank = scratch + V;
  uint32_t* blockcnt = rank + V;
  uint32_t* base = blockcnt + (uint64_t)nb * N_BUCKETS;
  uint32_t* hot_ids = base + N_BUCKETS;
  cudaError_t e = cudaMemsetAsync(cnt, 0, (uint64_t)V * sizeof(uint32_t), s);
  if (e != cudaSuccess) return e;
  if (L) {
    const uint64_t n_chunks = (L + 31) / 32, want = COUNT_SAMPLE / 32;
    const uint64_t stride = n_chunks > want ? n_chunks / want : 1;
    k_count_vars<<<grid_for((n_chunks + stride - 1) / stride * 32), 256, 0, s>>>(lits, L, stride, cnt);
  }
  k_bucket_counts<<<nb, 256, 0, s>>>(cnt, V, blockcnt);
  k_bucket_scan<<<1, N_BUCKETS, 0, s>>>(blockcnt, nb, base);
  k_assign_ranks<<<nb, 32, 0, s>>>(cnt, V, blockcnt, base, rank);
  k_hot_map<<<grid_for(V), 256, 0, s>>>(rank, V, map, hot_ids);
  k_fix_displaced<<<1, HOT_VARS, 0, s>>>(rank, V, hot_ids, map);
  return cudaGetLastError();
}

cudaError_t launch_translate(uint32_t* lits, uint64_t L, const uint32_t* map, cudaStream_t s) {
  if (L) k_translate<<<grid_for(L), 256, 0, s>>>(lits, L, map);
  return cudaGetLastError();
}

cudaError_t launch_build_heads(const uint64_t* boff, uint64_t n, uint64_t L0, uint32_t* head0_at_n0,
                               uint32_t* head1_at_n0, const uint32_t* lits_db, uint32_t V, cudaStream_t s) {
  if (n) k_build_heads<<<grid_for(n), 256, 0, s>>>(boff, n, L0, head0_at_n0, head1_at_n0, lits_db, V);
  return cudaGetLastError();
}

}  // namespace gss
