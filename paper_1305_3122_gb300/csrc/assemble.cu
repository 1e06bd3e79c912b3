// assemble.cu -- the numeric half of sparse(Ig, Jg, Kg): element matrices and their sums.
//
// Element stage (Sections 2 and 5): for triangle k with vertices p0, p1, p2 the edge vectors
// are e0 = p1 - p2, e1 = p2 - p0, e2 = p0 - p1 (the paper's u, v, w) and D = e1 x e2 = 2|T|.
//   mass         Eq. (1):  M_ab  = |T|/12 (1 + delta_ab)
//   weighted     Eq. (2):  Mw_ab = |T|/30 (w_a + w_b + w_c/2)  for a != b (c the third vertex),
//                          Mw_aa = |T|/30 (3 w_a + w_b + w_c)
//   stiffness    Eq. (3):  S_ab  = (e_a . e_b) / (4|T|)
//   elasticity   Sec. 7:   K = |T| B^T C B with grad(phi_a) = (e_a,y, -e_a,x) / (2|T|)
// Scatter stage (Section 5, sparse() sums duplicates): element k's entry (il, jl) is
// contribution c = n*n*k + n*jl + il and lands on non-zero map[...].
//   FE_VARIANT_ATOMIC: one thread per triangle adds its entries with FP64 atomicAdd.
//   FE_VARIANT_GATHER: one thread per triangle writes Kg[c] (staged through shared memory so the
//   stores are contiguous), then one thread per non-zero sums Kg over its contribution list in
//   ascending c -- the summation order of the paper's sparse() -- so the result is bit-identical
//   from run to run.
#include "internal.cuh"

enum Kind { K_MASS = 0, K_WMASS = 1, K_STIFF = 2, K_STIFF_WMASS = 3 };

struct Geo {
    double ex[3], ey[3];
    double D;   // 2|T|
};

__device__ __forceinline__ Geo geometry(const double2* __restrict__ q, int32_t v0, int32_t v1, int32_t v2) {
    double2 p0 = q[v0], p1 = q[v1], p2 = q[v2];
    Geo g;
    g.ex[0] = p1.x - p2.x; g.ey[0] = p1.y - p2.y;
    g.ex[1] = p2.x - p0.x; g.ey[1] = p2.y - p0.y;
    g.ex[2] = p0.x - p1.x; g.ey[2] = p0.y - p1.y;
    g.D = g.ex[1] * g.ey[2] - g.ex[2] * g.ey[1];
    return g;
}

// Element matrices, row-major E[3a + b].
__device__ __forceinline__ void elem_mass(double D, double E[9]) {
    double off = D / 24.0, dia = D / 12.0;
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = 0; b < 3; b++) E[3 * a + b] = a == b ? dia : off;
}

__device__ __forceinline__ void elem_wmass(double D, double w0, double w1, double w2, double E[9]) {
    double c = D / 60.0;   // |T| / 30
    double W[3] = {c * w0, c * w1, c * w2};
    double s = W[0] + W[1] + W[2];
#pragma unroll
    for (int a = 0; a < 3; a++) E[4 * a] = s + 2.0 * W[a];
    E[1] = E[3] = s - 0.5 * W[2];
    E[2] = E[6] = s - 0.5 * W[1];
    E[5] = E[7] = s - 0.5 * W[0];
}

__device__ __forceinline__ void elem_stiff(const Geo& g, double E[9]) {
    double inv = 1.0 / (2.0 * g.D);   // 1 / (4|T|)
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = a; b < 3; b++) {
            double v = (g.ex[a] * g.ex[b] + g.ey[a] * g.ey[b]) * inv;
            E[3 * a + b] = v;
            E[3 * b + a] = v;
        }
}

// 6x6 row-major, local dof 2a + alpha. With r = 1/(2D) = |T| / D^2 and grad(phi_a) = (e_a,y, -e_a,x)/D:
//   K[2a][2b]     = r ((l+2m) ey_a ey_b + m ex_a ex_b)
//   K[2a][2b+1]   = -r (l ey_a ex_b + m ex_a ey_b)
//   K[2a+1][2b]   = -r (l ex_a ey_b + m ey_a ex_b)
//   K[2a+1][2b+1] = r ((l+2m) ex_a ex_b + m ey_a ey_b)
__device__ __forceinline__ void elem_elas(const Geo& g, double lam, double mu, double K[36]) {
    double r = 1.0 / (2.0 * g.D);
    double l2m = lam + 2.0 * mu;
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = 0; b < 3; b++) {
            K[6 * (2 * a) + 2 * b] = r * (l2m * g.ey[a] * g.ey[b] + mu * g.ex[a] * g.ex[b]);
            K[6 * (2 * a) + 2 * b + 1] = -r * (lam * g.ey[a] * g.ex[b] + mu * g.ex[a] * g.ey[b]);
            K[6 * (2 * a + 1) + 2 * b] = -r * (lam * g.ex[a] * g.ey[b] + mu * g.ey[a] * g.ex[b]);
            K[6 * (2 * a + 1) + 2 * b + 1] = r * (l2m * g.ex[a] * g.ex[b] + mu * g.ey[a] * g.ey[b]);
        }
}

__device__ __forceinline__ void flag_orientation(double D, int* err) {
    if (!(D > 0.0)) atomicOr(err, 1);
}

// ---------------------------------------------------------------- scalar, atomic

template <int KIND>
__global__ void k_scalar_atomic(const double2* __restrict__ q, const int32_t* __restrict__ me, int32_t nme,
                                const int32_t* __restrict__ map, const double* __restrict__ w,
                                double* __restrict__ out0, double* __restrict__ out1, int* __restrict__ err,
                                int64_t nnz) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nme; k += (int64_t)gridDim.x * blockDim.x) {
        int32_t v0 = me[k], v1 = me[nme + k], v2 = me[2 * (int64_t)nme + k];
        Geo g = geometry(q, v0, v1, v2);
        flag_orientation(g.D, err);
        double E[9], F[9];
        if (KIND == K_MASS) elem_mass(g.D, E);
        if (KIND == K_WMASS) elem_wmass(g.D, w[v0], w[v1], w[v2], E);
        if (KIND == K_STIFF || KIND == K_STIFF_WMASS) elem_stiff(g, E);
        if (KIND == K_STIFF_WMASS) elem_wmass(g.D, w[v0], w[v1], w[v2], F);
        const int32_t* mk = map + 9 * k;
#pragma unroll
        for (int b = 0; b < 3; b++)
#pragma unroll
            for (int a = 0; a < 3; a++) {
                int32_t p = FE_IDX(mk[3 * b + a], nnz);
                atomicAdd(&out0[p], E[3 * a + b]);
                if (KIND == K_STIFF_WMASS) atomicAdd(&out1[p], F[3 * a + b]);
            }
    }
}

// ---------------------------------------------------------------- scalar, staged + gather

static constexpr int STAGE_BLOCK = 128;

template <int KIND>
__global__ void k_scalar_stage(const double2* __restrict__ q, const int32_t* __restrict__ me, int32_t nme,
                               const double* __restrict__ w, double* __restrict__ kg0, double* __restrict__ kg1,
                               int* __restrict__ err) {
    __shared__ double t0[9 * STAGE_BLOCK];
    __shared__ double t1[KIND == K_STIFF_WMASS ? 9 * STAGE_BLOCK : 1];
    for (int64_t k0 = (int64_t)blockIdx.x * STAGE_BLOCK; k0 < nme; k0 += (int64_t)gridDim.x * STAGE_BLOCK) {
        int64_t k = k0 + threadIdx.x;
        if (k < nme) {
            int32_t v0 = me[k], v1 = me[nme + k], v2 = me[2 * (int64_t)nme + k];
            Geo g = geometry(q, v0, v1, v2);
            flag_orientation(g.D, err);
            double E[9], F[9];
            if (KIND == K_MASS) elem_mass(g.D, E);
            if (KIND == K_WMASS) elem_wmass(g.D, w[v0], w[v1], w[v2], E);
            if (KIND == K_STIFF || KIND == K_STIFF_WMASS) elem_stiff(g, E);
            if (KIND == K_STIFF_WMASS) elem_wmass(g.D, w[v0], w[v1], w[v2], F);
#pragma unroll
            for (int b = 0; b < 3; b++)
#pragma unroll
                for (int a = 0; a < 3; a++) {
                    t0[9 * threadIdx.x + 3 * b + a] = E[3 * a + b];
                    if (KIND == K_STIFF_WMASS) t1[9 * threadIdx.x + 3 * b + a] = F[3 * a + b];
                }
        }
        __syncthreads();
        int64_t n = nme - k0 < STAGE_BLOCK ? nme - k0 : STAGE_BLOCK;
        for (int t = threadIdx.x; t < 9 * n; t += STAGE_BLOCK) {
            kg0[9 * k0 + t] = t0[t];
            if (KIND == K_STIFF_WMASS) kg1[9 * k0 + t] = t1[t];
        }
        __syncthreads();
    }
}

// values[p] = sum over s in [seg_ptr[p], seg_ptr[p+1]) of kg[perm[s]], left to right.
template <bool TWO>
__global__ void k_seg_gather(const int32_t* __restrict__ seg_ptr, const int32_t* __restrict__ perm, int64_t nnz,
                             const double* __restrict__ kg0, const double* __restrict__ kg1,
                             double* __restrict__ out0, double* __restrict__ out1, int64_t nkg) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t s0 = seg_ptr[p], s1 = seg_ptr[p + 1];
        double a0 = 0.0, a1 = 0.0;
        // four contributions per step: their ids, then their values, are loaded together (more
        // loads in flight); they are still added one by one in ascending order, the first one
        // taken as the start of the sum, so the result is that of the plain loop
        for (int32_t b = s0; b < s1; b += 4) {
            int32_t c[4];
            double v0[4], v1[4];
#pragma unroll
            for (int u = 0; u < 4; u++) c[u] = b + u < s1 ? FE_IDX(perm[FE_IDX(b + u, nkg)], nkg) : 0;
#pragma unroll
            for (int u = 0; u < 4; u++) {
                v0[u] = b + u < s1 ? kg0[c[u]] : 0.0;
                v1[u] = TWO && b + u < s1 ? kg1[c[u]] : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 4; u++) {
                if (b + u < s1) {
                    a0 = b + u == s0 ? v0[u] : a0 + v0[u];
                    if (TWO) a1 = b + u == s0 ? v1[u] : a1 + v1[u];
                }
            }
        }
        out0[p] = a0;
        if (TWO) out1[p] = a1;
    }
}

// ---------------------------------------------------------------- elasticity

// Position of K entry (2 i_a + alpha, 2 i_b + beta) from the scalar position p of (i_a, i_b),
// the start rb and degree g of scalar row i_a.
__device__ __forceinline__ int32_t pos2(int32_t p, int32_t rb, int32_t g, int alpha, int beta) {
    return 4 * rb + 2 * alpha * g + 2 * (p - rb) + beta;
}

// A part's weights, given by global vertex id, in its local numbering: wl[i] = w[l2g[i]].
__global__ void k_part_weights(const double* __restrict__ w, const int32_t* __restrict__ l2g, int32_t n,
                               double* __restrict__ wl) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        wl[i] = w[l2g[i]];
}

__global__ void k_elas_atomic(const double2* __restrict__ q, const int32_t* __restrict__ me, int32_t nme,
                              const int32_t* __restrict__ map, const int32_t* __restrict__ row_ptr,
                              double lam, double mu, double* __restrict__ out, int* __restrict__ err, int64_t nnz4) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nme; k += (int64_t)gridDim.x * blockDim.x) {
        int32_t v[3] = {me[k], me[nme + k], me[2 * (int64_t)nme + k]};
        Geo g = geometry(q, v[0], v[1], v[2]);
        flag_orientation(g.D, err);
        double K[36];
        elem_elas(g, lam, mu, K);
        int32_t rb[3], dg[3];
#pragma unroll
        for (int a = 0; a < 3; a++) { rb[a] = row_ptr[v[a]]; dg[a] = row_ptr[v[a] + 1] - rb[a]; }
        const int32_t* mk = map + 9 * k;
#pragma unroll
        for (int a = 0; a < 3; a++)
#pragma unroll
            for (int b = 0; b < 3; b++) {
                int32_t p = mk[3 * b + a];
#pragma unroll
                for (int al = 0; al < 2; al++)
#pragma unroll
                    for (int be = 0; be < 2; be++)
                        atomicAdd(&out[FE_IDX(pos2(p, rb[a], dg[a], al, be), nnz4)], K[6 * (2 * a + al) + 2 * b + be]);
            }
    }
}

static constexpr int ELAS_STAGE_BLOCK = 64;

// kg[36k + 6 jl + il] = K^e[il][jl]
__global__ void k_elas_stage(const double2* __restrict__ q, const int32_t* __restrict__ me, int32_t nme,
                             double lam, double mu, double* __restrict__ kg, int* __restrict__ err) {
    __shared__ double t[36 * ELAS_STAGE_BLOCK];
    for (int64_t k0 = (int64_t)blockIdx.x * ELAS_STAGE_BLOCK; k0 < nme; k0 += (int64_t)gridDim.x * ELAS_STAGE_BLOCK) {
        int64_t k = k0 + threadIdx.x;
        if (k < nme) {
            Geo g = geometry(q, me[k], me[nme + k], me[2 * (int64_t)nme + k]);
            flag_orientation(g.D, err);
            double K[36];
            elem_elas(g, lam, mu, K);
#pragma unroll
            for (int jl = 0; jl < 6; jl++)
#pragma unroll
                for (int il = 0; il < 6; il++) t[36 * threadIdx.x + 6 * jl + il] = K[6 * il + jl];
        }
        __syncthreads();
        int64_t n = nme - k0 < ELAS_STAGE_BLOCK ? nme - k0 : ELAS_STAGE_BLOCK;
        for (int s = threadIdx.x; s < 36 * n; s += ELAS_STAGE_BLOCK) kg[36 * k0 + s] = t[s];
        __syncthreads();
    }
}

// One thread per scalar row i: for each scalar non-zero (i, j) and each of its contributions
// c = 9k + 3b + a (ascending), add the 2x2 block K^e[2a+alpha][2b+beta] of triangle k.
__global__ void k_elas_gather(const int32_t* __restrict__ row_ptr, int32_t nq, const int32_t* __restrict__ seg_ptr,
                              const int32_t* __restrict__ perm, const double* __restrict__ kg, double* __restrict__ out,
                              int64_t ncontrib) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nq; r += (int64_t)gridDim.x * blockDim.x) {
        int32_t rb = row_ptr[r], g = row_ptr[r + 1] - rb;
        for (int32_t t = 0; t < g; t++) {
            int32_t p = rb + t;
            double acc[2][2];
            for (int32_t s = seg_ptr[p]; s < seg_ptr[p + 1]; s++) {
                int32_t c = FE_IDX(perm[FE_IDX(s, ncontrib)], ncontrib);
                int32_t k = c / 9;
                int32_t rr = c - 9 * k;
                int b = rr / 3, a = rr - 3 * b;
                const double* ke = kg + 36 * (int64_t)k;
#pragma unroll
                for (int al = 0; al < 2; al++)
#pragma unroll
                    for (int be = 0; be < 2; be++) {
                        double v = ke[6 * (2 * b + be) + 2 * a + al];
                        acc[al][be] = (s == seg_ptr[p]) ? v : acc[al][be] + v;
                    }
            }
#pragma unroll
            for (int al = 0; al < 2; al++)
#pragma unroll
                for (int be = 0; be < 2; be++) out[pos2(p, rb, g, al, be)] = acc[al][be];
        }
    }
}

// ---------------------------------------------------------------- entry points

static fe_status check_out(fe_pattern p, const double* values, int64_t cap) {
    if (!values && p->nnz > 0) return fe_fail(FE_ERR_INVALID_ARG, "values is null");
    if (cap < p->nnz)
        return fe_fail(FE_ERR_BUFFER_TOO_SMALL, "values capacity " + std::to_string(cap) + " < nnz " + std::to_string(p->nnz));
    return FE_OK;
}

static fe_status check_variant(fe_pattern p, int variant) {
    if (variant != FE_VARIANT_ATOMIC && variant != FE_VARIANT_GATHER && variant != FE_VARIANT_ROW)
        return fe_fail(FE_ERR_INVALID_ARG, "unknown variant");
    if (p->row1 >= 0 && variant != FE_VARIANT_ROW)
        return fe_fail(FE_ERR_INVALID_ARG, "a row-window pattern (fe_pattern_build_part) assembles with FE_VARIANT_ROW only");
    if (variant == FE_VARIANT_GATHER && !(p->flags & FE_PATTERN_GATHER))
        return fe_fail(FE_ERR_INVALID_ARG, "FE_VARIANT_GATHER needs a pattern built with FE_PATTERN_GATHER");
    if (variant == FE_VARIANT_ATOMIC && !p->map)
        return fe_fail(FE_ERR_INVALID_ARG, "FE_VARIANT_ATOMIC needs a pattern built with FE_PATTERN_MAP");
    return FE_OK;
}

static fe_status scalar(int kind, fe_mesh m, fe_pattern p, const double* w, int variant, double* out0,
                        double* out1, int64_t cap, cudaStream_t s) {
    fe_status st;
    if ((st = fe_check_pair(m, p, 1))) return st;
    if ((st = check_variant(p, variant))) return st;
    if ((st = check_out(p, out0, cap))) return st;
    if (kind == K_STIFF_WMASS && (st = check_out(p, out1, cap))) return st;
    if ((kind == K_WMASS || kind == K_STIFF_WMASS) && !w && m->nq > 0) return fe_fail(FE_ERR_INVALID_ARG, "w is null");
    const int32_t nme = m->nme;
    m->last_stream = p->last_stream = s;
    if (variant == FE_VARIANT_ROW) {
        static const int bits[4] = {4, 2, 1, 3};   // K_MASS, K_WMASS, K_STIFF, K_STIFF_WMASS
        if (m->part1 < 0 || !(kind == K_WMASS || kind == K_STIFF_WMASS) || m->nq == 0)
            return fe_row_scalar(bits[kind], m, p, w, out0, out1, s);
        FeStreamScope scope(s);
        double* wl = nullptr;
        if ((st = fe_alloc_n(&wl, (size_t)m->nq, "part weights"))) return st;
        { FE_PROF("k_part_weights", s); k_part_weights<<<fe_grid(m->nq, 256), 256, 0, s>>>(w, m->l2g, m->nq, wl); }
        cudaError_t e = cudaGetLastError();
        st = e != cudaSuccess ? fe_cuda_fail(e, "k_part_weights") : fe_row_scalar(bits[kind], m, p, wl, out0, out1, s);
        fe_free(wl);
        return st;
    }
    if (variant == FE_VARIANT_ATOMIC) {
        if (p->nnz > 0) FE_CUDA(cudaMemsetAsync(out0, 0, sizeof(double) * p->nnz, s));
        if (kind == K_STIFF_WMASS && p->nnz > 0) FE_CUDA(cudaMemsetAsync(out1, 0, sizeof(double) * p->nnz, s));
        if (nme == 0) return FE_OK;
        unsigned grid = fe_grid(nme, 256);
        switch (kind) {
            case K_MASS: { FE_PROF("k_scalar_atomic", s); k_scalar_atomic<K_MASS><<<grid, 256, 0, s>>>(m->q, m->me, nme, p->map, w, out0, out1, m->err, p->nnz); } break;
            case K_WMASS: { FE_PROF("k_scalar_atomic", s); k_scalar_atomic<K_WMASS><<<grid, 256, 0, s>>>(m->q, m->me, nme, p->map, w, out0, out1, m->err, p->nnz); } break;
            case K_STIFF: { FE_PROF("k_scalar_atomic", s); k_scalar_atomic<K_STIFF><<<grid, 256, 0, s>>>(m->q, m->me, nme, p->map, w, out0, out1, m->err, p->nnz); } break;
            default: { FE_PROF("k_scalar_atomic", s); k_scalar_atomic<K_STIFF_WMASS><<<grid, 256, 0, s>>>(m->q, m->me, nme, p->map, w, out0, out1, m->err, p->nnz); } break;
        }
        FE_LAUNCHED("k_scalar_atomic");
        return FE_OK;
    }
    if (nme == 0) return FE_OK;   // nnz == 0 too
    double* kg0 = p->kg;
    double* kg1 = p->kg + 9 * (size_t)nme;
    unsigned grid = fe_grid(nme, STAGE_BLOCK);
    switch (kind) {
        case K_MASS: { FE_PROF("k_scalar_stage", s); k_scalar_stage<K_MASS><<<grid, STAGE_BLOCK, 0, s>>>(m->q, m->me, nme, w, kg0, kg1, m->err); } break;
        case K_WMASS: { FE_PROF("k_scalar_stage", s); k_scalar_stage<K_WMASS><<<grid, STAGE_BLOCK, 0, s>>>(m->q, m->me, nme, w, kg0, kg1, m->err); } break;
        case K_STIFF: { FE_PROF("k_scalar_stage", s); k_scalar_stage<K_STIFF><<<grid, STAGE_BLOCK, 0, s>>>(m->q, m->me, nme, w, kg0, kg1, m->err); } break;
        default: { FE_PROF("k_scalar_stage", s); k_scalar_stage<K_STIFF_WMASS><<<grid, STAGE_BLOCK, 0, s>>>(m->q, m->me, nme, w, kg0, kg1, m->err); } break;
    }
    FE_LAUNCHED("k_scalar_stage");
    if (kind == K_STIFF_WMASS)
        { FE_PROF("k_seg_gather", s); k_seg_gather<true><<<fe_grid(p->nnz, 256), 256, 0, s>>>(p->seg_ptr, p->perm, p->nnz, kg0, kg1, out0, out1, 9 * (int64_t)nme); }
    else
        { FE_PROF("k_seg_gather", s); k_seg_gather<false><<<fe_grid(p->nnz, 256), 256, 0, s>>>(p->seg_ptr, p->perm, p->nnz, kg0, nullptr, out0, nullptr, 9 * (int64_t)nme); }
    FE_LAUNCHED("k_seg_gather");
    return FE_OK;
}

extern "C" fe_status fe_assemble_mass(fe_mesh m, fe_pattern p, int variant, double* values, int64_t cap, fe_stream s) {
    FE_RANGE(__func__);
    return scalar(K_MASS, m, p, nullptr, variant, values, nullptr, cap, (cudaStream_t)s);
}

extern "C" fe_status fe_assemble_wmass(fe_mesh m, fe_pattern p, const double* w, int variant, double* values,
                                       int64_t cap, fe_stream s) {
    FE_RANGE(__func__);
    return scalar(K_WMASS, m, p, w, variant, values, nullptr, cap, (cudaStream_t)s);
}

extern "C" fe_status fe_assemble_stiff(fe_mesh m, fe_pattern p, int variant, double* values, int64_t cap, fe_stream s) {
    FE_RANGE(__func__);
    return scalar(K_STIFF, m, p, nullptr, variant, values, nullptr, cap, (cudaStream_t)s);
}

extern "C" fe_status fe_assemble_stiff_wmass(fe_mesh m, fe_pattern p, const double* w, int variant, double* S,
                                             double* Mw, int64_t cap, fe_stream s) {
    FE_RANGE(__func__);
    return scalar(K_STIFF_WMASS, m, p, w, variant, S, Mw, cap, (cudaStream_t)s);
}

extern "C" fe_status fe_assemble_elas(fe_mesh m, fe_pattern p, double lam, double mu, int variant, double* values,
                                      int64_t cap, fe_stream stream) {
    FE_RANGE(__func__);
    fe_status st;
    if ((st = fe_check_pair(m, p, 2))) return st;
    if ((st = check_variant(p, variant))) return st;
    if ((st = check_out(p, values, cap))) return st;
    if (!(lam + mu > 0.0)) return fe_fail(FE_ERR_INVALID_ARG, "Lame parameters need lambda + mu > 0");
    cudaStream_t s = (cudaStream_t)stream;
    const int32_t nme = m->nme;
    m->last_stream = p->last_stream = s;
    if (variant == FE_VARIANT_ROW) return fe_row_elas(m, p, lam, mu, values, s);
    if (variant == FE_VARIANT_ATOMIC) {
        if (p->nnz > 0) FE_CUDA(cudaMemsetAsync(values, 0, sizeof(double) * p->nnz, s));
        if (nme == 0) return FE_OK;
        { FE_PROF("k_elas_atomic", s); k_elas_atomic<<<fe_grid(nme, 256), 256, 0, s>>>(m->q, m->me, nme, p->map, p->row_ptr, lam, mu, values, m->err, p->nnz); }
        FE_LAUNCHED("k_elas_atomic");
        return FE_OK;
    }
    if (nme == 0) return FE_OK;
    { FE_PROF("k_elas_stage", s); k_elas_stage<<<fe_grid(nme, ELAS_STAGE_BLOCK), ELAS_STAGE_BLOCK, 0, s>>>(m->q, m->me, nme, lam, mu, p->kg, m->err); }
    FE_LAUNCHED("k_elas_stage");
    { FE_PROF("k_elas_gather", s); k_elas_gather<<<fe_grid(m->nq, 128), 128, 0, s>>>(p->row_ptr, m->nq, p->seg_ptr, p->perm, p->kg, values, 9 * (int64_t)nme); }
    FE_LAUNCHED("k_elas_gather");
    return FE_OK;
}

// ---------------------------------------------------------------- allocation-free entry point
//
// fe_assemble_stiff_wmass_noalloc runs the staged-gather assembly of S and M^w with its staging
// buffer in a fixed, file-scope device array instead of memory from an allocator. It serves
// callers that must not allocate device memory during the call: a host framework that owns all
// device memory through its own pool and forbids hidden allocations (a second allocator would
// fragment or overcommit its budget), a solver plug-in loaded into such a host, or a loop with
// a hard latency budget where an allocation could stall. The array is
// FE_NOALLOC_MAX_TRIANGLES * 18 doubles (18 MiB) and stays resident on every GPU that loads the
// library until the process exits.

#include <mutex>

static __device__ __align__(256) double g_noalloc_scratch[(size_t)FE_NOALLOC_MAX_TRIANGLES * 18];

static std::mutex g_noalloc_mu;
static double* g_noalloc_addr[64];   // device address of the array, per device

// The host-side name of g_noalloc_scratch is a stand-in, not a device address; the address is
// looked up once per device, with that device current.
static fe_status noalloc_scratch(double** out) {
    int dev = 0;
    FE_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fe_fail(FE_ERR_CUDA, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return fe_cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_noalloc_addr[dev] = static_cast<double*>(p);
    }
    *out = g_noalloc_addr[dev];
    return FE_OK;
}

extern "C" fe_status fe_assemble_stiff_wmass_noalloc(fe_mesh m, fe_pattern p, const double* w, double* S, double* Mw,
                                                     int64_t cap, fe_stream stream) {
    FE_RANGE(__func__);
    fe_status st;
    if ((st = fe_check_pair(m, p, 1))) return st;
    if (!(p->flags & FE_PATTERN_GATHER))
        return fe_fail(FE_ERR_INVALID_ARG, "fe_assemble_stiff_wmass_noalloc needs a pattern built with FE_PATTERN_GATHER");
    if ((st = check_out(p, S, cap))) return st;
    if ((st = check_out(p, Mw, cap))) return st;
    if (!w && m->nq > 0) return fe_fail(FE_ERR_INVALID_ARG, "w is null");
    if (m->nme > FE_NOALLOC_MAX_TRIANGLES)
        return fe_fail(FE_ERR_LIMIT, "fe_assemble_stiff_wmass_noalloc takes at most FE_NOALLOC_MAX_TRIANGLES=" +
                                         std::to_string(FE_NOALLOC_MAX_TRIANGLES) + " triangles; this mesh has " +
                                         std::to_string(m->nme));
    double* scratch = nullptr;
    if ((st = noalloc_scratch(&scratch))) return st;
    const int32_t nme = m->nme;
    if (nme == 0) return FE_OK;   // then nnz == 0 as well
    cudaStream_t s = (cudaStream_t)stream;
    // the handles' device memory is freed in order on the last stream that used them
    m->last_stream = p->last_stream = s;
    // every staged entry is written before it is read, so nothing needs zeroing between calls
    double* kg0 = scratch;
    double* kg1 = scratch + 9 * (size_t)nme;
    { FE_PROF("k_scalar_stage", s); k_scalar_stage<K_STIFF_WMASS><<<fe_grid(nme, STAGE_BLOCK), STAGE_BLOCK, 0, s>>>(m->q, m->me, nme, w, kg0, kg1, m->err); }
    FE_LAUNCHED("k_scalar_stage (no-alloc)");
    { FE_PROF("k_seg_gather", s); k_seg_gather<true><<<fe_grid(p->nnz, 256), 256, 0, s>>>(p->seg_ptr, p->perm, p->nnz, kg0, kg1, S, Mw, 9 * (int64_t)nme); }
    FE_LAUNCHED("k_seg_gather (no-alloc)");
    return FE_OK;
}
