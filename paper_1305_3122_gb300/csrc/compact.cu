// compact.cu -- value-dependent zero dropping of a CSR matrix (fe_csr_drop_zeros).
//
// Matlab's sparse() stores no zero (Section 5 of the paper): an entry of K that is zero adds
// nothing, and a position whose sum is zero is not stored. The assembly calls keep the structural
// pattern; this pass removes the entries equal to 0.0 afterwards, which gives the same stored set.
//
// Two passes over the values, each handled by warps that own 32 consecutive rows (their entries
// are one contiguous range, read with coalesced loads):
//   k_row_nonzeros: the kept count of each row. Each 32-entry chunk of the warp's range is
//     tested once (a ballot); every lane then counts the bits of the chunk that fall in its row.
//     The loads of four chunks are issued before their ballots.
//   (exclusive scan of the counts -> row_ptr_out)
//   k_compact_rows: the warp walks its range again and writes the kept entries at
//     row_ptr_out[first row] + (kept entries before them in the range): ballot and popc, so the
//     writes of a chunk are consecutive.
#include "internal.cuh"

namespace {

constexpr int CZ_BLOCK = 256;
constexpr int CZ_UNROLL = 4;   // 32-entry chunks whose loads are issued together

__device__ __forceinline__ unsigned bits_between(int lo, int hi) {
    // bits lo .. hi-1 of a 32-bit mask (0 <= lo <= hi <= 32)
    unsigned up = hi >= 32 ? 0xffffffffu : ((1u << hi) - 1u);
    unsigned dn = lo >= 32 ? 0xffffffffu : ((1u << lo) - 1u);
    return up & ~dn;
}

// Non-zero test on the bits: the value without its sign bit is zero only for +0 and -0 (NaN and
// subnormals are kept). Integer instructions, so the FP64 pipe stays out of the loop.
__device__ __forceinline__ bool nonzero(double v) { return (__double_as_longlong(v) << 1) != 0; }

__global__ void __launch_bounds__(CZ_BLOCK) k_row_nonzeros(const int32_t* __restrict__ row_ptr,
                                                           const double* __restrict__ values, int32_t n_rows,
                                                           int32_t* __restrict__ cnt) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (CZ_BLOCK / 32);
    for (int64_t w = (int64_t)blockIdx.x * (CZ_BLOCK / 32) + (threadIdx.x >> 5); w * 32 < n_rows; w += nwarps) {
        const int64_t r = w * 32 + lane;
        const int64_t r1 = min((int64_t)n_rows, w * 32 + 32);
        const int32_t beg = row_ptr[w * 32], end = row_ptr[r1];
        const int32_t rs = r < n_rows ? row_ptr[r] : end;            // this lane's row [rs, re)
        const int32_t re = r < n_rows ? row_ptr[r + 1] : end;
        int32_t c = 0;
        for (int32_t base0 = beg; base0 < end; base0 += 32 * CZ_UNROLL) {
            double v[CZ_UNROLL];
#pragma unroll
            for (int u = 0; u < CZ_UNROLL; u++) {                  // all loads of the group first
                const int32_t s = base0 + 32 * u + lane;
                v[u] = s < end ? values[s] : 0.0;
            }
#pragma unroll
            for (int u = 0; u < CZ_UNROLL; u++) {
                const int32_t base = base0 + 32 * u;
                const unsigned m = __ballot_sync(0xffffffffu, nonzero(v[u]));
                const int lo = (int)max(0, min(32, rs - base)), hi = (int)max(0, min(32, re - base));
                c += __popc(m & bits_between(lo, hi));
            }
        }
        if (r < n_rows) cnt[r] = c;
    }
}

__global__ void __launch_bounds__(CZ_BLOCK) k_compact_rows(const int32_t* __restrict__ row_ptr,
                                                           const int32_t* __restrict__ col_idx,
                                                           const double* __restrict__ values, int32_t n_rows,
                                                           const int32_t* __restrict__ out_ptr,
                                                           int32_t* __restrict__ col_out, double* __restrict__ val_out) {
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    const int64_t nwarps = (int64_t)gridDim.x * (CZ_BLOCK / 32);
    for (int64_t w = (int64_t)blockIdx.x * (CZ_BLOCK / 32) + (threadIdx.x >> 5); w * 32 < n_rows; w += nwarps) {
        const int64_t r1 = min((int64_t)n_rows, w * 32 + 32);
        const int32_t beg = row_ptr[w * 32], end = row_ptr[r1];
        int32_t out = out_ptr[w * 32];
        for (int32_t base0 = beg; base0 < end; base0 += 32 * CZ_UNROLL) {
            double v[CZ_UNROLL];
            int32_t c[CZ_UNROLL];
#pragma unroll
            for (int u = 0; u < CZ_UNROLL; u++) {                  // all loads of the group first
                const int32_t s = base0 + 32 * u + lane;
                v[u] = s < end ? values[s] : 0.0;
                c[u] = s < end ? col_idx[s] : 0;
            }
#pragma unroll
            for (int u = 0; u < CZ_UNROLL; u++) {
                const bool keep = nonzero(v[u]);                  // 0.0 beyond the range: never kept
                const unsigned m = __ballot_sync(0xffffffffu, keep);
                if (keep) {
                    const int32_t p = out + __popc(m & below);
                    col_out[p] = c[u];
                    val_out[p] = v[u];
                }
                out += __popc(m);
            }
        }
    }
}

}  // namespace

extern "C" fe_status fe_csr_drop_zeros(int64_t n_rows, const int32_t* row_ptr, const int32_t* col_idx,
                                       const double* values, int32_t* row_ptr_out, int32_t* col_idx_out,
                                       double* values_out, int64_t cap, int64_t* nnz_out, fe_stream stream) {
    FE_RANGE(__func__);
    if (!nnz_out) return fe_fail(FE_ERR_INVALID_ARG, "nnz_out is null");
    *nnz_out = 0;
    if (n_rows < 0 || n_rows >= INT32_MAX) return fe_fail(FE_ERR_INVALID_ARG, "n_rows must be in [0, 2^31 - 1)");
    if (!row_ptr || !row_ptr_out) return fe_fail(FE_ERR_INVALID_ARG, "row_ptr or row_ptr_out is null");
    if (cap < 0) return fe_fail(FE_ERR_INVALID_ARG, "cap must be >= 0");
    if ((const void*)row_ptr_out == (const void*)row_ptr || (const void*)col_idx_out == (const void*)col_idx ||
        (const void*)values_out == (const void*)values)
        return fe_fail(FE_ERR_INVALID_ARG, "the outputs must not overlap the inputs");
    cudaStream_t s = (cudaStream_t)stream;
    FeStreamScope scope(s);
    const int32_t n = (int32_t)n_rows;
    int32_t* cnt = nullptr;
    fe_status st = fe_alloc_n(&cnt, (size_t)n + 1, "row counts");
    if (st) return st;
    const unsigned grid = fe_grid(((int64_t)n + 31) / 32, CZ_BLOCK / 32, 16);
    if (n > 0) {
        if (!values) { fe_free(cnt); return fe_fail(FE_ERR_INVALID_ARG, "values is null"); }
        { FE_PROF("k_row_nonzeros", s); k_row_nonzeros<<<grid, CZ_BLOCK, 0, s>>>(row_ptr, values, n, cnt); }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) { fe_free(cnt); return fe_cuda_fail(e, "k_row_nonzeros"); }
    }
    int64_t kept = 0;
    st = fe_exclusive_scan(cnt, row_ptr_out, n, s, &kept);
    if (st) { fe_free(cnt); return st; }
    *nnz_out = kept;
    if (kept > cap) {
        fe_free(cnt);
        return fe_fail(FE_ERR_BUFFER_TOO_SMALL, "cap " + std::to_string(cap) + " is below the " +
                                                    std::to_string(kept) + " non-zero entries");
    }
    if (n > 0 && kept > 0) {
        if (!col_idx || !col_idx_out || !values_out) {
            fe_free(cnt);
            return fe_fail(FE_ERR_INVALID_ARG, "col_idx, col_idx_out or values_out is null");
        }
        { FE_PROF("k_compact_rows", s); k_compact_rows<<<grid, CZ_BLOCK, 0, s>>>(row_ptr, col_idx, values, n, row_ptr_out, col_idx_out, values_out); }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) { fe_free(cnt); return fe_cuda_fail(e, "k_compact_rows"); }
    }
    fe_free(cnt);
    return FE_OK;
}
