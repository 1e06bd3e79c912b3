// tetelas.cu -- 3-D linear elasticity on tetrahedra: the plane elasticity of Section 7 carried to
// three dimensions (the paper announces the 3-D extension without formulas).
//
// Small strains, an isotropic material with constant Lame parameters lambda, mu. Local dof 3a + s
// is component s of vertex a. With the Voigt strain vector (e_xx, e_yy, e_zz, 2e_xy, 2e_yz, 2e_zx),
// the material matrix C = lambda (1,1,1,0,0,0)^T (1,1,1,0,0,0) + mu diag(2,2,2,1,1,1) and the strain
// matrix B built from g_a = grad(phi_a), K^e = |K| B^T C B has the entries
//   K^e[3a+s][3b+t] = |K| (lambda g_a,s g_b,t + mu g_a,t g_b,s + mu [s = t] g_a . g_b).
// In the unnormalised gradients gt_a = det g_a (det = 6|K|, the cross products of tet.cu) this is
//   K^e[3a+s][3b+t] = L gt_a,s gt_b,t + U (gt_a,t gt_b,s + [s = t] gt_a . gt_b),
// with L = lambda / (6 det) and U = mu / (6 det) formed once per tetrahedron (and L gt, U gt once
// per vertex). The arithmetic is FP64 throughout.
//
// Structure: the scalar entry (i, j) becomes the 3 x 3 block of rows 3i + s and columns 3j + t.
// Row 3i + s starts at 9 row_ptr[i] + 3 s len_i and holds, for each scalar column j in order,
// 3j, 3j + 1, 3j + 2; so entry (3i + s, 3j + t) sits at 9 row_ptr[i] + 3 s len_i + 3 o + t, where o
// is j's place in scalar row i (the scalar map gives row_ptr[i] + o).
//
// Two assemblies:
//   atomic  one thread per tetrahedron adds its 144 entries with FP64 atomics; each of the ten
//           vertex-pair blocks (a <= b) is computed once and added at both of its places;
//   ordered one thread per tetrahedron stages its 12 x 12 matrix (row-major, 1152 bytes, through
//           shared memory so that each block writes one contiguous range), then one thread per
//           row 3i + s walks row i's incidences in ascending element order (the scalar gather
//           lists) and adds row 3a + s of each staged matrix (96 contiguous bytes) to its
//           accumulators at the in-row positions of the four columns; rows of more than 32
//           scalar columns are summed by one warp each. Every value is then a fixed-order sum.
#include "internal.cuh"

namespace {

constexpr int TE_BLOCK = 128;      // atomic kernel and expansion
constexpr int ST_BLOCK = 64;       // stage kernel: 64 matrices of 144 doubles in shared memory
constexpr int ST_STRIDE = 145;     // a matrix's stride in shared memory (odd: no bank conflicts)
constexpr int RS3_BLOCK = 128;     // row sums: one row 3i + s per thread
// The scalar pattern's long-row list and flag decide the row kernels (the same as for the scalar
// row sums): rows of more than FE_TET_RS_MAX scalar columns go to the warp kernel, and the
// accumulators shrink to FE_TET_RS_SHORT scalar columns when no row is longer.
constexpr int RS3_MAX = FE_TET_RS_MAX;
constexpr int RS3_SHORT = FE_TET_RS_SHORT;

__global__ void __launch_bounds__(TE_BLOCK) k_tet_expand3(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx,
                                                          int32_t nq, int32_t* __restrict__ row_ptr3,
                                                          int32_t* __restrict__ col_idx3, int64_t nnz3) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nq; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t rb = row_ptr[i], len = row_ptr[i + 1] - rb;
        for (int s = 0; s < 3; s++) {
            const int32_t o = 9 * rb + 3 * s * len;
            row_ptr3[3 * i + s] = o;
            for (int32_t c = 0; c < len; c++) {
                const int32_t j3 = 3 * col_idx[rb + c];
                col_idx3[FE_IDX(o + 3 * c, nnz3)] = j3;
                col_idx3[FE_IDX(o + 3 * c + 1, nnz3)] = j3 + 1;
                col_idx3[FE_IDX(o + 3 * c + 2, nnz3)] = j3 + 2;
            }
        }
        if (i == nq - 1) row_ptr3[3 * i + 3] = 9 * row_ptr[nq];
    }
}

// Unnormalised gradients of one tetrahedron, and the same scaled by the two parameters.
struct ElasElem {
    double g[4][3];    // gt_a = det grad(phi_a)
    double Lg[4][3];   // L gt_a, L = lambda / (6 det)
    double Ug[4][3];   // U gt_a, U = mu / (6 det)
};

__device__ __forceinline__ void elas_elem(const double4_32a p[4], double lam, double mu, ElasElem& e) {
    const double ax = p[1].x - p[0].x, ay = p[1].y - p[0].y, az = p[1].z - p[0].z;
    const double bx = p[2].x - p[0].x, by = p[2].y - p[0].y, bz = p[2].z - p[0].z;
    const double cx = p[3].x - p[0].x, cy = p[3].y - p[0].y, cz = p[3].z - p[0].z;
    e.g[1][0] = by * cz - bz * cy; e.g[1][1] = bz * cx - bx * cz; e.g[1][2] = bx * cy - by * cx;   // b x c
    e.g[2][0] = cy * az - cz * ay; e.g[2][1] = cz * ax - cx * az; e.g[2][2] = cx * ay - cy * ax;   // c x a
    e.g[3][0] = ay * bz - az * by; e.g[3][1] = az * bx - ax * bz; e.g[3][2] = ax * by - ay * bx;   // a x b
#pragma unroll
    for (int t = 0; t < 3; t++) e.g[0][t] = -(e.g[1][t] + e.g[2][t] + e.g[3][t]);
    const double det = ax * e.g[1][0] + ay * e.g[1][1] + az * e.g[1][2];
    const double inv = 1.0 / (6.0 * det);
    const double L = lam * inv, U = mu * inv;
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
        for (int t = 0; t < 3; t++) {
            e.Lg[a][t] = L * e.g[a][t];
            e.Ug[a][t] = U * e.g[a][t];
        }
}

// The 3 x 3 block of vertices (a, b): B[s][t] = K^e[3a+s][3b+t] = (L gt_a,s) gt_b,t +
// (U gt_a,t) gt_b,s, plus (U gt_a) . gt_b on the diagonal: 24 FP64 operations a block (GB300's
// FP64 rate bounds the element stage).
__device__ __forceinline__ void elas_block(const ElasElem& e, int a, int b, double B[3][3]) {
    const double UG = fma(e.Ug[a][0], e.g[b][0], fma(e.Ug[a][1], e.g[b][1], e.Ug[a][2] * e.g[b][2]));
#pragma unroll
    for (int s = 0; s < 3; s++)
#pragma unroll
        for (int t = 0; t < 3; t++) B[s][t] = fma(e.Lg[a][s], e.g[b][t], e.Ug[a][t] * e.g[b][s]);
#pragma unroll
    for (int s = 0; s < 3; s++) B[s][s] += UG;
}

__device__ __forceinline__ void elas_load(const int32_t* __restrict__ me, int32_t nme, int64_t k, const double4_32a* __restrict__ q,
                                          int32_t nq, int32_t v[4], double4_32a p[4]) {
#pragma unroll
    for (int a = 0; a < 4; a++) {
        v[a] = FE_IDX(me[a * (int64_t)nme + k], nq);
        p[a] = q[v[a]];
    }
}

__global__ void __launch_bounds__(TE_BLOCK) k_tet_elas_atomic(const int32_t* __restrict__ me, int32_t nme, const double4_32a* __restrict__ q,
                                                              int32_t nq, const int32_t* __restrict__ row_ptr,
                                                              const int32_t* __restrict__ map, double lam, double mu,
                                                              double* __restrict__ val, int64_t nnz3) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nme; k += (int64_t)gridDim.x * blockDim.x) {
        int32_t v[4];
        double4_32a p[4];
        elas_load(me, nme, k, q, nq, v, p);
        ElasElem e;
        elas_elem(p, lam, mu, e);
        int32_t rb[4], len[4], o[4][4];
        const int4* m4 = reinterpret_cast<const int4*>(map + 16 * k);
#pragma unroll
        for (int a = 0; a < 4; a++) {
            rb[a] = row_ptr[v[a]];
            len[a] = row_ptr[v[a] + 1] - rb[a];
            const int4 m = m4[a];                                 // scalar positions of (a, 0..3)
            o[a][0] = m.x - rb[a]; o[a][1] = m.y - rb[a]; o[a][2] = m.z - rb[a]; o[a][3] = m.w - rb[a];
        }
#pragma unroll
        for (int a = 0; a < 4; a++)
#pragma unroll
            for (int b = a; b < 4; b++) {
                double B[3][3];
                elas_block(e, a, b, B);
#pragma unroll
                for (int s = 0; s < 3; s++)
#pragma unroll
                    for (int t = 0; t < 3; t++) {
                        const int64_t at = 9 * (int64_t)rb[a] + 3 * s * len[a] + 3 * o[a][b] + t;
                        atomicAdd(&val[FE_IDX(at, nnz3)], B[s][t]);
                        if (b != a) {                              // the transposed block (b, a)
                            const int64_t bt = 9 * (int64_t)rb[b] + 3 * t * len[b] + 3 * o[b][a] + s;
                            atomicAdd(&val[FE_IDX(bt, nnz3)], B[s][t]);
                        }
                    }
            }
    }
}

// Staged element matrices: kg3[144k + 12 (3a + s) + 3b + t] = K^e[3a+s][3b+t]. Each thread fills
// its matrix in shared memory; the block then writes its 64 matrices as one contiguous range.
__global__ void __launch_bounds__(ST_BLOCK) k_tet_elas_stage(const int32_t* __restrict__ me, int32_t nme, const double4_32a* __restrict__ q,
                                                             int32_t nq, double lam, double mu, double* __restrict__ kg3) {
    extern __shared__ double sm[];                                // [ST_BLOCK][ST_STRIDE]
    for (int64_t k0 = blockIdx.x * (int64_t)ST_BLOCK; k0 < nme; k0 += (int64_t)gridDim.x * ST_BLOCK) {
        const int64_t k = k0 + threadIdx.x;
        double* my = sm + threadIdx.x * ST_STRIDE;
        if (k < nme) {
            int32_t v[4];
            double4_32a p[4];
            elas_load(me, nme, k, q, nq, v, p);
            ElasElem e;
            elas_elem(p, lam, mu, e);
#pragma unroll
            for (int a = 0; a < 4; a++)
#pragma unroll
                for (int b = a; b < 4; b++) {
                    double B[3][3];
                    elas_block(e, a, b, B);
#pragma unroll
                    for (int s = 0; s < 3; s++)
#pragma unroll
                        for (int t = 0; t < 3; t++) {
                            my[12 * (3 * a + s) + 3 * b + t] = B[s][t];
                            my[12 * (3 * b + t) + 3 * a + s] = B[s][t];
                        }
                }
        }
        __syncthreads();
        const int64_t nk = min((int64_t)ST_BLOCK, (int64_t)nme - k0);
        const int n = (int)(144 * nk);
        double* dst = kg3 + 144 * k0;
        for (int x = threadIdx.x; x < n; x += ST_BLOCK) {
            const int r = x / 144;
            dst[x] = sm[r * ST_STRIDE + (x - 144 * r)];
        }
        __syncthreads();
    }
}

// Ordered row sums: thread r3 owns row 3i + s. Each incidence (element k, local vertex a of i),
// in ascending element order, adds row 3a + s of the staged matrix (12 values: columns 3b + t of
// the element) to the accumulators 3 slot_b + t, where slot_b is column me[b][k]'s place in scalar
// row i. The twelve accumulators of an incidence are distinct, so all are read before any is
// written back. Accumulators start at -0.0, so each sum equals its first contribution followed by
// the others in ascending element order. Rows of more than RMAX scalar columns are left to
// k_tet_elas_rowsum_long.
template <int RMAX>
__global__ void __launch_bounds__(RS3_BLOCK) k_tet_elas_rowsum(const int32_t* __restrict__ vptr, const int32_t* __restrict__ row_ptr,
                                                               int32_t nq, const int32_t* __restrict__ inc,
                                                               const uint2* __restrict__ islot, const double* __restrict__ kg3,
                                                               double* __restrict__ val, int64_t n4, int64_t nnz3) {
    extern __shared__ double acc3[];                              // [3 RMAX][RS3_BLOCK]
    double* acc = acc3 + threadIdx.x;                             // accumulator c at acc[c * RS3_BLOCK]
    for (int64_t r3 = blockIdx.x * (int64_t)RS3_BLOCK + threadIdx.x; r3 < 3 * (int64_t)nq; r3 += (int64_t)gridDim.x * RS3_BLOCK) {
        const int32_t i = (int32_t)(r3 / 3);
        const int s = (int)(r3 - 3 * (int64_t)i);
        const int32_t rb = row_ptr[i], u = row_ptr[i + 1] - rb;
        if (u > RMAX) continue;
        const int32_t b0 = vptr[i], d = vptr[i + 1] - b0;
        const int n3 = 3 * u;
        for (int c = 0; c < n3; c++) acc[c * RS3_BLOCK] = -0.0;
        for (int32_t t = 0; t < d; t++) {
            const int32_t key = FE_IDX(inc[b0 + t], n4);
            const uint2 sl = islot[b0 + t];
            const double2* e = reinterpret_cast<const double2*>(kg3 + 144 * (int64_t)(key >> 2) + 12 * (3 * (key & 3) + s));
            double2 x[6];
#pragma unroll
            for (int j = 0; j < 6; j++) x[j] = e[j];
            const double v[12] = {x[0].x, x[0].y, x[1].x, x[1].y, x[2].x, x[2].y,
                                  x[3].x, x[3].y, x[4].x, x[4].y, x[5].x, x[5].y};
            const unsigned c4[4] = {sl.x & 0xFFFFu, sl.x >> 16, sl.y & 0xFFFFu, sl.y >> 16};
            double* pc[12];
            double y[12];
#pragma unroll
            for (int b = 0; b < 4; b++)
#pragma unroll
                for (int tt = 0; tt < 3; tt++) {
                    pc[3 * b + tt] = acc + FE_IDX(3 * (int)c4[b] + tt, n3) * RS3_BLOCK;
                    y[3 * b + tt] = *pc[3 * b + tt];
                }
#pragma unroll
            for (int j = 0; j < 12; j++) *pc[j] = y[j] + v[j];
        }
        const int64_t o = 9 * (int64_t)rb + 3 * s * u;
        for (int c = 0; c < n3; c++) val[FE_IDX(o + c, nnz3)] = acc[c * RS3_BLOCK];
    }
}

// Rows of scalar rows with more than RS3_MAX columns, one warp per row 3i + s: lane l owns the
// accumulators c = l (mod 32) and adds their contributions in ascending element order
// (3 (3 FE_TET_MAX_VALENCE + 1) doubles of dynamic shared memory at most).
__global__ void __launch_bounds__(32) k_tet_elas_rowsum_long(const int32_t* __restrict__ long_rows, const int32_t* __restrict__ n_long,
                                                             const int32_t* __restrict__ vptr, const int32_t* __restrict__ row_ptr,
                                                             const int32_t* __restrict__ inc, const uint2* __restrict__ islot,
                                                             const double* __restrict__ kg3, double* __restrict__ val, int64_t nnz3) {
    extern __shared__ double accl[];
    const int lane = threadIdx.x;
    const int32_t n = 3 * *n_long;
    for (int32_t b = blockIdx.x; b < n; b += gridDim.x) {
        const int32_t i = long_rows[b / 3];
        const int s = b % 3;
        const int32_t rb = row_ptr[i], u = row_ptr[i + 1] - rb;
        const int32_t b0 = vptr[i], d = vptr[i + 1] - b0;
        const int n3 = 3 * u;
        for (int c = lane; c < n3; c += 32) accl[c] = -0.0;
        __syncwarp();
        for (int32_t t = 0; t < d; t++) {
            const int32_t key = inc[b0 + t];
            const uint2 sl = islot[b0 + t];
            const double* e = kg3 + 144 * (int64_t)(key >> 2) + 12 * (3 * (key & 3) + s);
            const unsigned c4[4] = {sl.x & 0xFFFFu, sl.x >> 16, sl.y & 0xFFFFu, sl.y >> 16};
#pragma unroll
            for (int bb = 0; bb < 4; bb++)
#pragma unroll
                for (int tt = 0; tt < 3; tt++) {
                    const int c = 3 * (int)c4[bb] + tt;
                    if ((c & 31) == lane) accl[c] += e[3 * bb + tt];
                }
        }
        __syncwarp();
        const int64_t o = 9 * (int64_t)rb + 3 * s * u;
        for (int c = lane; c < n3; c += 32) val[FE_IDX(o + c, nnz3)] = accl[c];
        __syncwarp();
    }
}

}  // namespace

fe_status fe_tet_elas_structure(fe_tet_pattern p, cudaStream_t s) {
    const int64_t nnz3 = 9 * p->nnz;
    if (nnz3 >= INT32_MAX) return fe_fail(FE_ERR_LIMIT, "the 3-D elasticity structure needs 9 nnz < 2^31");
    const int32_t nq = p->nq;
    fe_status st;
    if ((st = fe_alloc_n(&p->row_ptr3, 3 * (size_t)nq + 1, "row_ptr (3-D elasticity)"))) return st;
    if ((st = fe_alloc_n(&p->col_idx3, (size_t)nnz3, "col_idx (3-D elasticity)"))) return st;
    if (nq > 0) {
        { FE_PROF("k_tet_expand3", s); k_tet_expand3<<<fe_grid(nq, TE_BLOCK), TE_BLOCK, 0, s>>>(p->row_ptr, p->col_idx, nq, p->row_ptr3, p->col_idx3, nnz3); }
        FE_LAUNCHED("k_tet_expand3");
    } else {
        FE_CUDA(cudaMemsetAsync(p->row_ptr3, 0, sizeof(int32_t), s));
    }
    return FE_OK;
}

extern "C" fe_status fe_tet_pattern_elas_info(fe_tet_pattern p, int64_t* n_rows, int64_t* nnz, const int32_t** row_ptr,
                                              const int32_t** col_idx) {
    if (!p) return fe_fail(FE_ERR_INVALID_ARG, "null pattern");
    if (!(p->flags & FE_TET_PATTERN_ELAS)) return fe_fail(FE_ERR_INVALID_ARG, "the pattern was built without FE_TET_PATTERN_ELAS");
    if (n_rows) *n_rows = 3 * (int64_t)p->nq;
    if (nnz) *nnz = 9 * p->nnz;
    if (row_ptr) *row_ptr = p->row_ptr3;
    if (col_idx) *col_idx = p->col_idx3;
    return FE_OK;
}

extern "C" fe_status fe_tet_assemble_elas(fe_tet_mesh m, fe_tet_pattern p, double lam, double mu, int variant,
                                          double* values, int64_t cap, fe_stream stream) {
    FE_RANGE(__func__);
    if (!m || !p) return fe_fail(FE_ERR_INVALID_ARG, "null mesh or pattern");
    if (m->topology_id != p->topology_id) return fe_fail(FE_ERR_INVALID_ARG, "the pattern was built for another mesh");
    if (!(p->flags & FE_TET_PATTERN_ELAS)) return fe_fail(FE_ERR_INVALID_ARG, "the pattern was built without FE_TET_PATTERN_ELAS");
    if (!(mu > 0.0) || !(3.0 * lam + 2.0 * mu > 0.0) || !(lam - lam == 0.0) || !(mu - mu == 0.0))
        return fe_fail(FE_ERR_INVALID_ARG, "need finite lambda and mu with mu > 0 and 3 lambda + 2 mu > 0");
    if (variant != FE_VARIANT_ATOMIC && variant != FE_VARIANT_GATHER)
        return fe_fail(FE_ERR_INVALID_ARG, "3-D elasticity takes FE_VARIANT_ATOMIC or FE_VARIANT_GATHER");
    if (variant == FE_VARIANT_GATHER && !(p->flags & FE_PATTERN_GATHER))
        return fe_fail(FE_ERR_INVALID_ARG, "FE_VARIANT_GATHER needs a pattern built with FE_PATTERN_GATHER");
    const int64_t nnz3 = 9 * p->nnz;
    if (cap < nnz3) return fe_fail(FE_ERR_BUFFER_TOO_SMALL, "cap is below nnz");
    if (!values && nnz3 > 0) return fe_fail(FE_ERR_INVALID_ARG, "values is null");
    cudaStream_t s = (cudaStream_t)stream;
    FeStreamScope scope(s);
    m->last_stream = s;
    p->last_stream = s;
    const int32_t nme = m->nme, nq = m->nq;
    if (nnz3 == 0) return FE_OK;
    if (variant == FE_VARIANT_ATOMIC) {
        FE_CUDA(cudaMemsetAsync(values, 0, sizeof(double) * (size_t)nnz3, s));
        if (nme > 0) {
            { FE_PROF("k_tet_elas_atomic", s); k_tet_elas_atomic<<<fe_grid(nme, TE_BLOCK, 8), TE_BLOCK, 0, s>>>(m->me, nme, m->q, nq, p->row_ptr, p->map, lam, mu, values, nnz3); }
            FE_LAUNCHED("k_tet_elas_atomic");
        }
        return FE_OK;
    }
    double* kg3 = nullptr;
    fe_status st;
    if ((st = fe_alloc_n(&kg3, 144 * (size_t)nme, "3-D elasticity element staging"))) return st;
    struct Release {
        double* p;
        ~Release() { fe_free(p); }
    } release{kg3};
    const size_t st_smem = (size_t)ST_BLOCK * ST_STRIDE * sizeof(double);
    FE_CUDA(cudaFuncSetAttribute(k_tet_elas_stage, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)st_smem));
    { FE_PROF("k_tet_elas_stage", s); k_tet_elas_stage<<<fe_grid(nme, ST_BLOCK, 8), ST_BLOCK, st_smem, s>>>(m->me, nme, m->q, nq, lam, mu, kg3); }
    FE_LAUNCHED("k_tet_elas_stage");
    {
        FE_PROF("k_tet_elas_rowsum", s);
        if (!p->n_long_host[1]) {
            const size_t sm = 3 * (size_t)RS3_SHORT * RS3_BLOCK * sizeof(double);
            FE_CUDA(cudaFuncSetAttribute(k_tet_elas_rowsum<RS3_SHORT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
            k_tet_elas_rowsum<RS3_SHORT><<<fe_grid(3 * (int64_t)nq, RS3_BLOCK, 8), RS3_BLOCK, sm, s>>>(
                p->vptr, p->row_ptr, nq, p->inc, p->islot, kg3, values, 4 * (int64_t)nme, nnz3);
        } else {
            const size_t sm = 3 * (size_t)RS3_MAX * RS3_BLOCK * sizeof(double);
            FE_CUDA(cudaFuncSetAttribute(k_tet_elas_rowsum<RS3_MAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
            k_tet_elas_rowsum<RS3_MAX><<<fe_grid(3 * (int64_t)nq, RS3_BLOCK, 4), RS3_BLOCK, sm, s>>>(
                p->vptr, p->row_ptr, nq, p->inc, p->islot, kg3, values, 4 * (int64_t)nme, nnz3);
        }
    }
    FE_LAUNCHED("k_tet_elas_rowsum");
    if (p->n_long_host[0] > 0) {
        const size_t sm = 3 * (3 * (size_t)FE_TET_MAX_VALENCE + 1) * sizeof(double);
        FE_CUDA(cudaFuncSetAttribute(k_tet_elas_rowsum_long, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        { FE_PROF("k_tet_elas_rowsum_long", s); k_tet_elas_rowsum_long<<<fe_sm_count() * 8, 32, sm, s>>>(p->long_rows, p->n_long, p->vptr, p->row_ptr, p->inc, p->islot, kg3, values, nnz3); }
        FE_LAUNCHED("k_tet_elas_rowsum_long");
    }
    return FE_OK;
}
