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
#include "ff.cuh"
#include "internal.cuh"

// The element adjoint in double-float arithmetic on the FP32 pipes (ff.cuh). GB300's FP64 rate
// (about 2 operations per clock per SM) made the FP64 form of these ~150 operations per triangle
// the whole cost of the pass. FP64 remains for the coordinate differences and one addition per
// output. The 18 upstream values of a triangle enter linearly, so they are split with a common
// power-of-two scale (magnitude about 1) and the outputs are scaled back exactly.
struct AdjConsts {
    ff c60;        // 1/60
    int64_t nnz;   // stored entries of the upstream arrays (bounds-checked builds)
    int64_t n3;    // incidences, 3 nme (bounds-checked builds)
};

template <bool WS, bool WM>
__device__ __forceinline__ void elem_adjoint(const double2* __restrict__ q, const int32_t* __restrict__ mk,
                                             int32_t v0, int32_t v1, int32_t v2, const double* __restrict__ w,
                                             const double* __restrict__ gS, const double* __restrict__ gM,
                                             const AdjConsts& cs, double dpx[3], double dpy[3], double dw[3],
                                             int& bad, int& orient) {
    double2 p0 = q[v0], p1 = q[v1], p2 = q[v2];
    // edge vectors e_a (opposite vertex a): exact FP64 differences, then split
    ff ex[3] = {ff_from_double(p1.x - p2.x, bad), ff_from_double(p2.x - p0.x, bad), ff_from_double(p0.x - p1.x, bad)};
    ff ey[3] = {ff_from_double(p1.y - p2.y, bad), ff_from_double(p2.y - p0.y, bad), ff_from_double(p0.y - p1.y, bad)};
    ff D = ff_dot2(ex[1], ex[2], ey[2], ff_neg(ey[1]));         // 2A = e1 x e2
    orient |= !(D.h > 0.f);
    ff inv = ff_rcp_fast(D);
    inv = ff{0.5f * inv.h, 0.5f * inv.l};                       // 1 / (2D) = 1 / (4A)
    ff inv4 = ff{4.0f * inv.h, 4.0f * inv.l};                   // 1 / A
    // the triangle's upstream values g[3b + a] (at (a, b)), one common scale 2^k
    double gsr[9], gmr[9];
    unsigned emax = 0;
#pragma unroll
    for (int t = 0; t < 9; t++) {
        if (WS) { gsr[t] = gS[FE_IDX(mk[t], cs.nnz)]; emax = max(emax, fp64_biased_exponent(gsr[t])); }
        if (WM) { gmr[t] = gM[FE_IDX(mk[t], cs.nnz)]; emax = max(emax, fp64_biased_exponent(gmr[t])); }
    }
    const int k = ff_group_scale(emax);
    ff dA = z_ff();                                             // dL/dA (scaled)
    ff dex[3] = {z_ff(), z_ff(), z_ff()}, dey[3] = {z_ff(), z_ff(), z_ff()};
    if (WS) {
        ff g[9];
#pragma unroll
        for (int t = 0; t < 9; t++) g[t] = ff_from_double_scaled(gsr[t], k);
        // dL/de_a = sum_b (g_ab + g_ba) e_b / (4A); dL/dA = -sum_ab g_ab (e_a . e_b) / (4A^2)
        ff h[3][3];
#pragma unroll
        for (int a = 0; a < 3; a++)
#pragma unroll
            for (int b = 0; b < 3; b++) h[a][b] = ff_add(g[3 * b + a], g[3 * a + b]);
        ff sum = z_ff();
#pragma unroll
        for (int a = 0; a < 3; a++) {
            dex[a] = ff_mul(ff_add(ff_add(ff_mul(h[a][0], ex[0]), ff_mul(h[a][1], ex[1])), ff_mul(h[a][2], ex[2])), inv);
            dey[a] = ff_mul(ff_add(ff_add(ff_mul(h[a][0], ey[0]), ff_mul(h[a][1], ey[1])), ff_mul(h[a][2], ey[2])), inv);
#pragma unroll
            for (int b = a; b < 3; b++) {
                ff G = ff_dot2(ex[a], ey[a], ex[b], ey[b]);     // e_a . e_b
                ff_acc(sum, ff_mul(a == b ? g[4 * a] : h[a][b], G));
            }
        }
        dA = ff_neg(ff_mul(ff_mul(sum, inv), inv4));
    }
    if (WM) {
        ff g[9];
#pragma unroll
        for (int t = 0; t < 9; t++) g[t] = ff_from_double_scaled(gmr[t], k);
        ff c = ff_mul(D, cs.c60);                               // A / 30
        ff W[3] = {ff_mul(c, ff_from_double(w[v0], bad)), ff_mul(c, ff_from_double(w[v1], bad)),
                   ff_mul(c, ff_from_double(w[v2], bad))};
        ff sW = ff_add(ff_add(W[0], W[1]), W[2]);
        ff diag = ff_add(ff_add(g[0], g[4]), g[8]);
        ff R[3] = {ff_add(ff_add(g[1], g[3]), ff_add(g[2], g[6])), ff_add(ff_add(g[1], g[3]), ff_add(g[5], g[7])),
                   ff_add(ff_add(g[2], g[6]), ff_add(g[5], g[7]))};
        ff off = ff_add(ff_add(ff_add(g[1], g[3]), ff_add(g[2], g[6])), ff_add(g[5], g[7]));
        // sum_ab g_ab Mw_ab with Mw_aa = s + 2 W_a, Mw_ab = s - W_c / 2 (c the third vertex)
        ff two = ff_add(ff_add(ff_mul(g[0], W[0]), ff_mul(g[4], W[1])), ff_mul(g[8], W[2]));
        ff half = ff_add(ff_add(ff_mul(ff_add(g[1], g[3]), W[2]), ff_mul(ff_add(g[2], g[6]), W[1])),
                         ff_mul(ff_add(g[5], g[7]), W[0]));
        ff Lm = ff_add(ff_add(ff_mul(sW, ff_add(diag, off)), ff_mulf(two, 2.0f)), ff_mulf(half, -0.5f));
        dA = ff_add(dA, ff_mul(Lm, inv4));
        ff gd[3] = {g[0], g[4], g[8]};
#pragma unroll
        for (int t = 0; t < 3; t++) {
            ff v = ff_add(ff_add(ff_mulf(gd[t], 2.0f), diag), ff_add(R[t], ff_mulf(ff_sub(off, R[t]), 0.5f)));
            dw[t] = ff_to_double_scaled(ff_mul(c, v), k);
        }
    } else {
        dw[0] = dw[1] = dw[2] = 0.0;
    }
    // chain rule: dp0 = de2 - de1, dp1 = de0 - de2, dp2 = de1 - de0, plus dA * dA/dp_a with
    // dA/dp_a = (e_a,y, -e_a,x) / 2
    ff hA = ff{0.5f * dA.h, 0.5f * dA.l};
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const int b = a == 2 ? 0 : a + 1, c2 = a == 0 ? 2 : a - 1;
        dpx[a] = ff_to_double_scaled(ff_add(ff_sub(dex[c2], dex[b]), ff_mul(hA, ey[a])), k);
        dpy[a] = ff_to_double_scaled(ff_sub(ff_sub(dey[c2], dey[b]), ff_mul(hA, ex[a])), k);
    }
}

template <bool WS, bool WM>
__global__ void k_adjoint_atomic(const double2* __restrict__ q, const int32_t* __restrict__ me, int32_t nme, int32_t nq,
                                 const int32_t* __restrict__ map, const double* __restrict__ w,
                                 const double* __restrict__ gS, const double* __restrict__ gM, AdjConsts cs,
                                 double* __restrict__ dq, double* __restrict__ dw, int* __restrict__ err) {
    int bad = 0, orient = 0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nme; k += (int64_t)gridDim.x * blockDim.x) {
        int32_t v[3] = {me[k], me[nme + k], me[2 * (int64_t)nme + k]};
        double dpx[3], dpy[3], dwl[3];
        elem_adjoint<WS, WM>(q, map + 9 * k, v[0], v[1], v[2], w, gS, gM, cs, dpx, dpy, dwl, bad, orient);
#pragma unroll
        for (int a = 0; a < 3; a++) {
            atomicAdd(&dq[v[a]], dpx[a]);
            atomicAdd(&dq[nq + v[a]], dpy[a]);
            if (WM) atomicAdd(&dw[v[a]], dwl[a]);
        }
    }
    if (bad) atomicOr(err, 2);
    if (orient) atomicOr(err, 1);
}

// stage[9k + 3 comp + a]: comp 0 = d/dx, 1 = d/dy, 2 = d/dw of local vertex a.
template <bool WS, bool WM>
__global__ void k_adjoint_stage(const double2* __restrict__ q, const int32_t* __restrict__ me, int32_t nme,
                                const int32_t* __restrict__ map, const double* __restrict__ w,
                                const double* __restrict__ gS, const double* __restrict__ gM, AdjConsts cs,
                                double* __restrict__ stage, int* __restrict__ err) {
    int bad = 0, orient = 0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nme; k += (int64_t)gridDim.x * blockDim.x) {
        double dpx[3], dpy[3], dwl[3];
        elem_adjoint<WS, WM>(q, map + 9 * k, me[k], me[nme + k], me[2 * (int64_t)nme + k], w, gS, gM, cs, dpx, dpy, dwl,
                             bad, orient);
        double* o = stage + 9 * k;
#pragma unroll
        for (int a = 0; a < 3; a++) { o[a] = dpx[a]; o[3 + a] = dpy[a]; o[6 + a] = dwl[a]; }
    }
    if (bad) atomicOr(err, 2);
    if (orient) atomicOr(err, 1);
}

__global__ void k_adjoint_gather(const int32_t* __restrict__ vptr, const int32_t* __restrict__ vel, int32_t nq,
                                 const double* __restrict__ stage, bool want_w, double* __restrict__ dq,
                                 double* __restrict__ dw, int64_t n3) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nq; i += (int64_t)gridDim.x * blockDim.x) {
        double sx = 0.0, sy = 0.0, sw = 0.0;
        const int32_t s0 = vptr[i], s1 = vptr[i + 1];
        // four triangles per step: their ids, then their staged values, are loaded together;
        // the sums still take them one by one in ascending order
        for (int32_t b = s0; b < s1; b += 4) {
            int32_t e[4];
            double vx[4], vy[4], vw[4];
#pragma unroll
            for (int u = 0; u < 4; u++) e[u] = b + u < s1 ? FE_IDX(vel[FE_IDX(b + u, n3)], n3) : 0;
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const int32_t k = e[u] / 3, a = e[u] - 3 * k;
                const double* o = stage + 9 * (int64_t)k;
                const bool in = b + u < s1;
                vx[u] = in ? o[a] : 0.0;
                vy[u] = in ? o[3 + a] : 0.0;
                vw[u] = in && want_w ? o[6 + a] : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 4; u++) {
                if (b + u < s1) {
                    sx += vx[u];
                    sy += vy[u];
                    sw += vw[u];
                }
            }
        }
        dq[i] = sx;
        dq[nq + i] = sy;
        if (want_w) dw[i] = sw;
    }
}

extern "C" fe_status fe_adjoint_stiff_wmass(fe_mesh m, fe_pattern p, const double* w, const double* gS,
                                            const double* gM, int variant, double* dq, double* dw, fe_stream stream) {
    FE_RANGE(__func__);
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
    AdjConsts cs;
    {
        double c = 1.0 / 60.0;
        cs.c60.h = (float)c;
        cs.c60.l = (float)(c - (double)cs.c60.h);
    }
    cs.nnz = p->nnz;
    cs.n3 = 3 * (int64_t)nme;
    if (variant == FE_VARIANT_ATOMIC || nme == 0) {
        FE_CUDA(cudaMemsetAsync(dq, 0, 2 * sizeof(double) * nq, s));
        FE_CUDA(cudaMemsetAsync(dw, 0, sizeof(double) * nq, s));
        if (nme == 0) return FE_OK;
        if (!gS && !gM) return FE_OK;
        const unsigned g = fe_grid(nme, 256);
        {
            FE_PROF("k_adjoint_atomic", s);
            if (gS && gM) k_adjoint_atomic<true, true><<<g, 256, 0, s>>>(m->q, m->me, nme, nq, p->map, w, gS, gM, cs, dq, dw, m->err);
            else if (gS) k_adjoint_atomic<true, false><<<g, 256, 0, s>>>(m->q, m->me, nme, nq, p->map, w, gS, gM, cs, dq, dw, m->err);
            else k_adjoint_atomic<false, true><<<g, 256, 0, s>>>(m->q, m->me, nme, nq, p->map, w, gS, gM, cs, dq, dw, m->err);
        }
        FE_LAUNCHED("k_adjoint_atomic");
        return FE_OK;
    }
    if (!gM) FE_CUDA(cudaMemsetAsync(dw, 0, sizeof(double) * nq, s));
    if (!gS && !gM) {
        FE_CUDA(cudaMemsetAsync(dq, 0, 2 * sizeof(double) * nq, s));
        return FE_OK;
    }
    {
        const unsigned g = fe_grid(nme, 256);
        FE_PROF("k_adjoint_stage", s);
        if (gS && gM) k_adjoint_stage<true, true><<<g, 256, 0, s>>>(m->q, m->me, nme, p->map, w, gS, gM, cs, p->kg, m->err);
        else if (gS) k_adjoint_stage<true, false><<<g, 256, 0, s>>>(m->q, m->me, nme, p->map, w, gS, gM, cs, p->kg, m->err);
        else k_adjoint_stage<false, true><<<g, 256, 0, s>>>(m->q, m->me, nme, p->map, w, gS, gM, cs, p->kg, m->err);
    }
    FE_LAUNCHED("k_adjoint_stage");
    { FE_PROF("k_adjoint_gather", s); k_adjoint_gather<<<fe_grid(nq, 256), 256, 0, s>>>(p->vptr, p->vel, nq, p->kg, gM != nullptr, dq, dw, 3 * (int64_t)nme); }
    FE_LAUNCHED("k_adjoint_gather");
    return FE_OK;
}
