// edges.cuh -- edge numbering from the scalar (P1) pattern, shared by the P2 and P3 builds.
//
// The edges of a triangle mesh are the entries above the diagonal of the structural P1 pattern
// (every pair of vertices sharing a triangle is stored): edge (a, c), a < c, is numbered by its
// rank among them in CSR order, i.e. in ascending order of (smaller id, larger id). Per row: the
// number of entries right of the diagonal (k_edge_upper), a scan of those counts (the row's first
// edge id), and a binary search of c in row a (edge_rank).
#pragma once

#include "internal.cuh"

namespace {

// Entries right of the diagonal in each scalar row (0 for an empty row), and the diagonal's place.
__global__ void k_edge_upper(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx, int32_t nq,
                           int32_t* __restrict__ ucnt, int32_t* __restrict__ dpos) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nq; r += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = (int32_t)r, b = row_ptr[i], n = row_ptr[i + 1] - b;
        int lo = 0, hi = n;                                   // first column >= i
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (col_idx[b + mid] < i) lo = mid + 1;
            else hi = mid;
        }
        dpos[i] = lo;
        ucnt[i] = n > 0 ? n - lo - 1 : 0;
    }
}

__device__ __forceinline__ int32_t edge_rank(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx,
                                           const int32_t* __restrict__ eoff, const int32_t* __restrict__ dpos,
                                           int32_t u, int32_t v) {
    const int32_t a = min(u, v), c = max(u, v);
    const int32_t b = row_ptr[a];
    int lo = dpos[a] + 1, hi = row_ptr[a + 1] - b - 1;        // c lies right of the diagonal
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (col_idx[b + mid] < c) lo = mid + 1;
        else hi = mid;
    }
    return eoff[a] + (lo - dpos[a] - 1);
}

}  // namespace
