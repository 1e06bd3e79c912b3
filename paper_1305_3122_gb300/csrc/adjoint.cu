// adjoint.cu -- gradient of L = sum(gS * S.values) + sum(gM * Mw.values) w.r.t. q and w.
//
// Not in the paper: the derivative of the element formulas of Eqs. (2)-(3) with the area taken
// from the coordinates. Per triangle, with A = |T| = D/2, g_ab the upstream gradient at the
// non-zero of (me[a], me[b]) and e0 = p1 - p2, e1 = p2 - p0, e2 = p0 - p1:
//   stiffness:  dL/de_a = sum_b (gS_ab + gS_ba) e_b / (4A),   dL/dA += -sum_ab gS_ab S_ab / A
//   weighted:   dL/dA += sum_ab gM_ab Mw_ab / A,
//               dL/dw_c = A/30 (2 gM_cc + sum_a gM_aa + R_c + (O - R_c)/2)
//               with R_c = sum_{b != c} (gM_cb + gM_bc) and O = sum_{a != b} gM_ab
//   chain rule: dL/dp0 = dL/de2 - dL/de1, dL/dp1 = dL/de0 - dL/de2, dL/dp2 = dL/de1 - dL/de0,
//               plus dL/dA * dA/dp_a with dA/dp_a = (e_a,y, -e_a,x) / 2.
// Per-vertex sums: FE_VARIANT_ATOMIC adds with atomics; FE_VARIANT_GATHER stages the 9 terms of
// each triangle and lets one thread per vertex add its triangles in ascending triangle order.
#include "internal.cuh"

__device__ __forceinline__ void elem_adjoint(const double2* __restrict__ q, const int32_t* __restrict__ mk,
                                             int32_t v0, int32_t v1, int32_t v2, const double* __restrict__ w,
                                             const double* __restrict__ gS, const double* __restrict__ gM,
                                             double dpx[3], double dpy[3], double dw[3], int* err) {
    double2 p0 = q[v0], p1 = q[v1], p2 = q[v2];
    double ex[3] = {p1.x - p2.x, p2.x - p0.x, p0.x - p1.x};
    double ey[3] = {p1.y - p2.y, p2.y - p0.y, p0.y - p1.y};
    double D = ex[1] * ey[2] - ex[2] * ey[1];
    if (!(D > 0.0)) atomicOr(err, 1);
    double A = 0.5 * D;
    double dex[3] = {0, 0, 0}, dey[3] = {0, 0, 0};
    double dA = 0.0;
    if (gS) {
        double g[9];
#pragma unroll
        for (int t = 0; t < 9; t++) g[t] = gS[mk[t]];   // g[3b + a] = gS at (a, b)
        double inv = 1.0 / (2.0 * D);                   // 1 / (4A)
        double sumgS = 0.0;
#pragma unroll
        for (int a = 0; a < 3; a++)
#pragma unroll
            for (int b = 0; b < 3; b++) {
                double gab = g[3 * b + a];
                double gs = (gab + g[3 * a + b]) * inv;
                dex[a] += gs * ex[b];
                dey[a] += gs * ey[b];
                sumgS += gab * (ex[a] * ex[b] + ey[a] * ey[b]);
            }
        dA -= sumgS * inv / A;
    }
    dw[0] = dw[1] = dw[2] = 0.0;
    if (gM) {
        double g[9];
#pragma unroll
        for (int t = 0; t < 9; t++) g[t] = gM[mk[t]];
        double c = A / 30.0;
        double W[3] = {c * w[v0], c * w[v1], c * w[v2]};
        double s = W[0] + W[1] + W[2];
        double diag = g[0] + g[4] + g[8];
        double off = g[1] + g[2] + g[3] + g[5] + g[6] + g[7];
        // sum_ab g_ab Mw_ab with Mw_aa = s + 2 W_a, Mw_ab = s - W_c / 2 (c the third vertex)
        double Lm = s * (diag + off) + 2.0 * (g[0] * W[0] + g[4] * W[1] + g[8] * W[2])
                    - 0.5 * ((g[1] + g[3]) * W[2] + (g[2] + g[6]) * W[1] + (g[5] + g[7]) * W[0]);
        dA += Lm / A;
        double R[3] = {g[1] + g[3] + g[2] + g[6], g[1] + g[3] + g[5] + g[7], g[2] + g[6] + g[5] + g[7]};
        double gd[3] = {g[0], g[4], g[8]};
#pragma unroll
        for (int t = 0; t < 3; t++) dw[t] = c * (2.0 * gd[t] + diag + R[t] + 0.5 * (off - R[t]));
    }
    dpx[0] = dex[2] - dex[1]; dpy[0] = dey[2] - dey[1];
    dpx[1] = dex[0] - dex[2]; dpy[1] = dey[0] - dey[2];
    dpx[2] = dex[1] - dex[0]; dpy[2] = dey[1] - dey[0];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        dpx[a] += dA * 0.5 * ey[a];
        dpy[a] -= dA * 0.5 * ex[a];
    }
}

__global__ void k_adjoint_atomic(const double2* __restrict__ q, const int32_t* __restrict__ me, int32_t nme, int32_t nq,
                                 const int32_t* __restrict__ map, const double* __restrict__ w,
                                 const double* __restrict__ gS, const double* __restrict__ gM,
                                 double* __restrict__ dq, double* __restrict__ dw, int* __restrict__ err) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nme; k += (int64_t)gridDim.x * blockDim.x) {
        int32_t v[3] = {me[k], me[nme + k], me[2 * (int64_t)nme + k]};
        double dpx[3], dpy[3], dwl[3];
        elem_adjoint(q, map + 9 * k, v[0], v[1], v[2], w, gS, gM, dpx, dpy, dwl, err);
#pragma unroll
        for (int a = 0; a < 3; a++) {
            atomicAdd(&dq[v[a]], dpx[a]);
            atomicAdd(&dq[nq + v[a]], dpy[a]);
            if (gM) atomicAdd(&dw[v[a]], dwl[a]);
        }
    }
}

// stage[9k + 3 comp + a]: comp 0 = d/dx, 1 = d/dy, 2 = d/dw of local vertex a.
__global__ void k_adjoint_stage(const double2* __restrict__ q, const int32_t* __restrict__ me, int32_t nme,
                                const int32_t* __restrict__ map, const double* __restrict__ w,
                                const double* __restrict__ gS, const double* __restrict__ gM,
                                double* __restrict__ stage, int* __restrict__ err) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nme; k += (int64_t)gridDim.x * blockDim.x) {
        double dpx[3], dpy[3], dwl[3];
        elem_adjoint(q, map + 9 * k, me[k], me[nme + k], me[2 * (int64_t)nme + k], w, gS, gM, dpx, dpy, dwl, err);
        double* o = stage + 9 * k;
#pragma unroll
        for (int a = 0; a < 3; a++) { o[a] = dpx[a]; o[3 + a] = dpy[a]; o[6 + a] = dwl[a]; }
    }
}

__global__ void k_adjoint_gather(const int32_t* __restrict__ vptr, const int32_t* __restrict__ vel, int32_t nq,
                                 const double* __restrict__ stage, bool want_w, double* __restrict__ dq,
                                 double* __restrict__ dw) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nq; i += (int64_t)gridDim.x * blockDim.x) {
        double sx = 0.0, sy = 0.0, sw = 0.0;
        for (int32_t s = vptr[i]; s < vptr[i + 1]; s++) {
            int32_t e = vel[s];
            int32_t k = e / 3, a = e - 3 * k;
            const double* o = stage + 9 * (int64_t)k;
            sx += o[a];
            sy += o[3 + a];
            sw += o[6 + a];
        }
        dq[i] = sx;
        dq[nq + i] = sy;
        if (want_w) dw[i] = sw;
    }
}

extern "C" fe_status fe_adjoint_stiff_wmass(fe_mesh m, fe_pattern p, const double* w, const double* gS,
                                            const double* gM, int variant, double* dq, double* dw, fe_stream stream) {
    fe_status st;
    if ((st = fe_check_pair(m, p, 1))) return st;
    if (variant != FE_VARIANT_ATOMIC && variant != FE_VARIANT_GATHER) return fe_fail(FE_ERR_INVALID_ARG, "unknown variant");
    if (variant == FE_VARIANT_GATHER && !(p->flags & FE_PATTERN_GATHER))
        return fe_fail(FE_ERR_INVALID_ARG, "FE_VARIANT_GATHER needs a pattern built with FE_PATTERN_GATHER");
    if (!p->map) return fe_fail(FE_ERR_INVALID_ARG, "the adjoint needs a pattern built with FE_PATTERN_MAP");
    if (m->nq > 0 && (!dq || !dw)) return fe_fail(FE_ERR_INVALID_ARG, "dq or dw is null");
    if (gM && !w && m->nq > 0) return fe_fail(FE_ERR_INVALID_ARG, "w is null");
    cudaStream_t s = (cudaStream_t)stream;
    m->last_stream = p->last_stream = s;
    const int32_t nq = m->nq, nme = m->nme;
    if (nq == 0) return FE_OK;
    if (variant == FE_VARIANT_ATOMIC || nme == 0) {
        FE_CUDA(cudaMemsetAsync(dq, 0, 2 * sizeof(double) * nq, s));
        FE_CUDA(cudaMemsetAsync(dw, 0, sizeof(double) * nq, s));
        if (nme == 0) return FE_OK;
        { FE_PROF("k_adjoint_atomic", s); k_adjoint_atomic<<<fe_grid(nme, 256), 256, 0, s>>>(m->q, m->me, nme, nq, p->map, w, gS, gM, dq, dw, m->err); }
        FE_LAUNCHED("k_adjoint_atomic");
        return FE_OK;
    }
    if (!gM) FE_CUDA(cudaMemsetAsync(dw, 0, sizeof(double) * nq, s));
    { FE_PROF("k_adjoint_stage", s); k_adjoint_stage<<<fe_grid(nme, 256), 256, 0, s>>>(m->q, m->me, nme, p->map, w, gS, gM, p->kg, m->err); }
    FE_LAUNCHED("k_adjoint_stage");
    { FE_PROF("k_adjoint_gather", s); k_adjoint_gather<<<fe_grid(nq, 256), 256, 0, s>>>(p->vptr, p->vel, nq, p->kg, gM != nullptr, dq, dw); }
    FE_LAUNCHED("k_adjoint_gather");
    return FE_OK;
}
