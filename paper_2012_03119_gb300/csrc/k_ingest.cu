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
#include "gss_internal.h"

namespace gss {
namespace {

__global__ void k_ingest(const uint64_t* __restrict__ boff, uint64_t n, uint64_t L, uint64_t L0,
                         uint64_t* __restrict__ off_db, uint32_t* __restrict__ head0,
                         uint32_t* __restrict__ head1,
                         const uint32_t* __restrict__ lits_db, uint32_t V, DevStatus* st) {
  const uint32_t PAD = 2u * V;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t b = boff[i], e = boff[i + 1];
    if (!(e > b && e <= L)) {  // empty clause, decreasing offsets or offsets past the batch
      atomicOr(&st->bad_size, 1u);
      continue;
    }
    off_db[i + 1] = L0 + e;
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

__global__ void k_check_lits(const uint32_t* __restrict__ lits, uint64_t n, uint32_t two_v, DevStatus* st) {
  uint32_t bad = 0;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    bad |= (lits[i] >= two_v) ? 1u : 0u;
  if (bad) atomicOr(&st->bad_lit, 1u);
}

}  // namespace

cudaError_t launch_ingest(const uint64_t* boff, uint64_t n, uint64_t L, uint64_t L0, uint64_t* off_db_at_n0,
                          uint32_t* head0_at_n0, uint32_t* head1_at_n0, const uint32_t* lits_db, uint32_t V,
                          DevStatus* st, cudaStream_t s) {
  if (L) {
    const uint64_t blocks = (L + 255) / 256;
    k_check_lits<<<(unsigned)(blocks < 8192 ? blocks : 8192), 256, 0, s>>>(lits_db + L0, L, 2u * V, st);
  }
  if (n) {
    const uint64_t blocks = (n + 255) / 256;
    k_ingest<<<(unsigned)(blocks < 8192 ? blocks : 8192), 256, 0, s>>>(boff, n, L, L0, off_db_at_n0, head0_at_n0,
                                                                       head1_at_n0, lits_db, V, st);
  }
  return cudaGetLastError();
}

}  // namespace gss
