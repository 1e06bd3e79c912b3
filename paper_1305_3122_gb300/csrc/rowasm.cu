// rowasm.cu -- FE_VARIANT_ROW: atomic-free, deterministic assembly by row owners.
//
// The paper sums the 9*nme contributions with sparse() (Section 5). Here each CSR row i (vertex
// i) is summed by its owner, which computes just the entries of each element matrix that land in
// row i. For a triangle (i, j, l), counter-clockwise with i at local position a, and relative
// coordinates r_t = p_t - p_i:
//   edge vectors  e_a = r_j - r_l, e_{a+1} = r_l, e_{a+2} = -r_j;   D = 2|T| = r_j x r_l
//   S   (Eq. 3): S_ii += |e_a|^2 / 2D,  S_ij += e_a.r_l / 2D,  S_il += -e_a.r_j / 2D
//   M^w (Eq. 2): with s = w_i + w_j + w_l:
//                Mw_ii += D/60 (s + 2 w_i), Mw_ij += D/60 (s - w_l/2), Mw_il += D/60 (s - w_j/2)
//   M   (Eq. 1): M_ii += D/12, M_ij += D/24, M_il += D/24
//   K   (Sec. 7): the 2 x 2 blocks of rows 2i, 2i+1 of K^e = |T| B^T C B (elas_terms below).
// Every value is written exactly once: no atomics, no zeroing, no staged element matrices.
//
// Simple rows (pattern.cu) list their neighbours n_0, n_1, ... in counter-clockwise fan order,
// so triangle e of the fan is (i, n_e, n_{e+1}); consecutive triangles share a neighbour, whose
// two contributions meet in a register carry and leave as one store. One thread per row, no
// shared memory, each neighbour's coordinates loaded once. The arithmetic is double-float on
// the FP32 pipes (ff.cuh) after an exact FP64 difference per coordinate and neighbour.
// General rows (several chains, long fans, non-manifold) use one block per row: thread t owns
// column t and adds, in the row's stored (sorted) triangle order, every contribution to its
// column, converting each to FP64 and summing with Neumaier's compensated summation.
// Both paths fix the order of every sum, so the result is bit-identical from run to run.
#include "ff.cuh"
#include "internal.cuh"

namespace {

enum { W_S = 1, W_W = 2, W_M = 4 };

struct Consts {
    ff c60, c12, c24;           // 1/60, 1/12, 1/24 as double-floats
    ff l2m, lam, mu;            // lambda + 2 mu, lambda, mu (elasticity)
    double d60, d12, d24;       // the same in FP64 (general rows)
    double dl2m, dlam, dmu;     // elasticity constants in FP64 (badly shaped triangles)
};

// A neighbour of the row's vertex: relative coordinates r = p - p_i and weight as double-floats,
// exact squared length |r|^2 (stiffness only), its approximate float value (for the conditioning
// test), vertex id and column position.
struct Nb {
    ff x, y, w, nn;
    float n;
    int32_t id;
    int pos;
};

// The contributions of one triangle (i, j, l) to row i: columns j and l (and self), for S and
// M^w. The S diagonal is not needed: every row of S sums to zero (Eq. 3 gives S^e 1 = 0), so the
// row owner writes S_ii = -sum_{j != i} S_ij.
struct RowTerms {
    ff d;          // D = 2|T|
    ff s[3];       // S entries (self entry unused)
    ff w[3];       // unscaled M^w entries: D (s + 2 w_i), D (s - w_l / 2), D (s - w_j / 2)
};

// FP64 version of row_terms for badly shaped triangles (an angle below about 14.5 degrees),
// where the double-float path would lose too many bits to cancellation. Rare, so the FP64
// pipe's low rate does not matter; the results are split back into double-floats.
template <int KIND>
__device__ __noinline__ RowTerms row_terms_fp64(const double2* __restrict__ q, const double* __restrict__ w, int32_t i,
                                                int32_t j, int32_t l, int& bad) {
    RowTerms t;
    double2 pi = q[i], pj = q[j], pl = q[l];
    double eax = pj.x - pl.x, eay = pj.y - pl.y;      // e_a
    double e1x = pl.x - pi.x, e1y = pl.y - pi.y;      // e_{a+1} = r_l
    double e2x = pi.x - pj.x, e2y = pi.y - pj.y;      // e_{a+2} = -r_j
    double D = e1x * e2y - e2x * e1y;
    t.d = ff_from_double(D, bad);
    if (KIND & W_S) {
        double inv = 1.0 / (2.0 * D);
        t.s[0] = ff_from_double((eax * eax + eay * eay) * inv, bad);
        t.s[1] = ff_from_double((eax * e1x + eay * e1y) * inv, bad);
        t.s[2] = ff_from_double((eax * e2x + eay * e2y) * inv, bad);
    }
    if (KIND & W_W) {
        double wi = w[i], wj = w[j], wl = w[l];
        double s = wi + wj + wl;
        t.w[0] = ff_from_double(D * (s + 2.0 * wi), bad);
        t.w[1] = ff_from_double(D * (s - 0.5 * wl), bad);
        t.w[2] = ff_from_double(D * (s - 0.5 * wj), bad);
    }
    return t;
}

// 1/a from the approximate float reciprocal and one Newton step in double-float (about 46 bits).
__device__ __forceinline__ ff ff_rcp_fast(ff a) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a.h));
    float r = fmaf(-a.h, y, 1.0f);
    r = fmaf(-a.l, y, r);
    return ff_norm(y, FMUL(y, r));
}

// Shape test: sin^2 of each angle is D^2 over the product of the two adjacent squared edges;
// all three must be at least 1/16 (angles of at least about 14.5 degrees) for the fast path.
__device__ __forceinline__ bool well_shaped(const Nb& j, const Nb& l, float dh) {
    float ex = j.x.h - l.x.h, ey = j.y.h - l.y.h;
    float eaa = ex * ex + ey * ey;
    float d2 = 16.0f * dh * dh;
    return d2 >= j.n * l.n && d2 >= eaa * l.n && d2 >= eaa * j.n;
}

template <int KIND>
__device__ __forceinline__ RowTerms row_terms(const double2* __restrict__ q, const double* __restrict__ w, int32_t i,
                                              const Nb& j, const Nb& l, ff wi, int& bad) {
    RowTerms t;
    t.d = ff_dot2(j.x, l.x, l.y, ff_neg(j.y));                  // r_j x r_l
    if (!well_shaped(j, l, t.d.h)) return row_terms_fp64<KIND>(q, w, i, j.id, l.id, bad);
    if (KIND & W_S) {
        ff inv = ff_mulf(ff_rcp_fast(t.d), 0.5f);              // 1 / 2D
        ff njl = ff_dot2(j.x, j.y, l.x, l.y);
        t.s[1] = ff_mul(ff_sub(njl, l.nn), inv);                // (r_j - r_l) . r_l
        t.s[2] = ff_mul(ff_sub(njl, j.nn), inv);                // (r_j - r_l) . (-r_j)
    }
    if (KIND & W_W) {
        ff s = ff_add(ff_add(wi, j.w), l.w);
        t.w[0] = ff_mul(t.d, ff_add(s, ff_mulf(wi, 2.0f)));
        t.w[1] = ff_mul(t.d, ff_add(s, ff_mulf(l.w, -0.5f)));
        t.w[2] = ff_mul(t.d, ff_add(s, ff_mulf(j.w, -0.5f)));
    }
    return t;
}

// Raw (FP64) data of a neighbour, loaded one triangle ahead of its use.
struct Raw {
    double2 p;
    double w;
    int32_t id;
    int pos;
};

template <int KIND>
__device__ __forceinline__ Raw load_raw(const double2* __restrict__ q, const double* __restrict__ w, int2 rec) {
    Raw r;
    r.p = q[rec.x];
    r.w = (KIND & W_W) ? w[rec.x] : 0.0;
    r.id = rec.x;
    r.pos = rec.y;
    return r;
}

template <int KIND>
__device__ __forceinline__ Nb make_nb(const Raw& r, double2 pi, int& bad) {
    Nb b;
    b.x = ff_from_double(r.p.x - pi.x, bad);
    b.y = ff_from_double(r.p.y - pi.y, bad);
    b.n = b.x.h * b.x.h + b.y.h * b.y.h;
    b.nn = (KIND & W_S) ? ff_dot2(b.x, b.y, b.x, b.y) : ff_make(0.f);
    b.w = (KIND & W_W) ? ff_from_double(r.w, bad) : ff_make(0.f);
    b.id = r.id;
    b.pos = r.pos;
    return b;
}

// General-row helper: a neighbour from its id (no prefetching).
template <int KIND>
__device__ __forceinline__ Nb load_nb(const double2* __restrict__ q, const double* __restrict__ w, double2 pi,
                                      int32_t c, int pos, int& bad) {
    return make_nb<KIND>(load_raw<KIND>(q, w, make_int2(c, pos)), pi, bad);
}

// Value (or pair of values) of one row entry, scaled and converted to FP64.
template <int KIND>
__device__ __forceinline__ void emit(double* __restrict__ out0, double* __restrict__ out1, int32_t at, ff a0, ff a1,
                                     bool diag, const Consts& cs) {
    if (KIND == W_M) a0 = ff_mul(a0, diag ? cs.c12 : cs.c24);
    if (KIND == W_W) a0 = ff_mul(a0, cs.c60);
    out0[at] = ff_to_double(a0);
    if (KIND == (W_S | W_W)) out1[at] = ff_to_double(ff_mul(a1, cs.c60));
}

// per-contribution values of the two outputs (out0: S, else M^w, else M; out1: M^w with S)
template <int KIND>
__device__ __forceinline__ void pick(const RowTerms& t, int which, ff& v0, ff& v1) {
    if (KIND & W_S) v0 = t.s[which];
    else if (KIND & W_W) v0 = t.w[which];
    else v0 = t.d;
    v1 = (KIND == (W_S | W_W)) ? t.w[which] : ff_make(0.f);
}

}  // namespace

template <int KIND>
__global__ void __launch_bounds__(256, 3) k_fan_scalar(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ vptr,
                                                       const int2* __restrict__ fan, const int2* __restrict__ hdr,
                                                       const double2* __restrict__ q, const double* __restrict__ w, int32_t nq,
                                                       Consts cs, double* __restrict__ out0, double* __restrict__ out1,
                                                       int* __restrict__ err) {
    int bad = 0, orient = 0;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nq; r += (int64_t)gridDim.x * blockDim.x) {
        int32_t i = (int32_t)r;
        int2 h = hdr[i];
        int kind = h.y >> 28;
        if (kind > 1) continue;                                  // general row (or no triangle)
        int32_t rb = row_ptr[i], b0 = vptr[i], d = vptr[i + 1] - b0;
        int pself = h.y & 0x3FFF;
        // neighbour k of the fan: k < d from the fan records; k == d is the last neighbour of an
        // open fan (from the header) or n_0 again for a closed fan
        const int2 last = kind == 1 ? make_int2(h.x, (h.y >> 14) & 0x3FFF) : fan[b0];
        double2 pi = q[i];
        ff wi = (KIND & W_W) ? ff_from_double(w[i], bad) : ff_make(0.f);
        Raw rn = load_raw<KIND>(q, w, fan[b0]);
        Raw rp = load_raw<KIND>(q, w, d > 1 ? fan[b0 + 1] : last);
        Nb cur = make_nb<KIND>(rn, pi, bad);
        const int first_pos = cur.pos;
        const ff z = ff_make(0.f);
        ff dg0 = z, dg1 = z, fs0 = z, fs1 = z, ca0 = z, ca1 = z;
        for (int32_t e = 0; e < d; e++) {
            rn = rp;                                             // neighbour e + 1 (already loaded)
            if (e + 2 <= d) rp = load_raw<KIND>(q, w, e + 2 < d ? fan[b0 + e + 2] : last);
            Nb nxt = make_nb<KIND>(rn, pi, bad);
            RowTerms t = row_terms<KIND>(q, w, i, cur, nxt, wi, bad);
            orient |= !(t.d.h > 0.f);
            ff j0, j1, l0, l1;
            pick<KIND>(t, 1, j0, j1);
            pick<KIND>(t, 2, l0, l1);
            if (KIND == W_W || KIND == (W_S | W_W)) ff_acc(KIND == W_W ? dg0 : dg1, t.w[0]);
            if (KIND == W_M) ff_acc(dg0, t.d);
            if (e == 0) {
                fs0 = j0;
                fs1 = j1;
            } else {
                ff v0 = ff_add(ca0, j0);
                if (KIND & W_S) ff_acc(dg0, ff_neg(v0));
                emit<KIND>(out0, out1, rb + cur.pos, v0, ff_add(ca1, j1), false, cs);
            }
            ca0 = l0;
            ca1 = l1;
            cur = nxt;
        }
        if (kind == 0) {
            ff v0 = ff_add(fs0, ca0);
            if (KIND & W_S) ff_acc(dg0, ff_neg(v0));
            emit<KIND>(out0, out1, rb + first_pos, v0, ff_add(fs1, ca1), false, cs);
        } else {
            if (KIND & W_S) { ff_acc(dg0, ff_neg(fs0)); ff_acc(dg0, ff_neg(ca0)); }
            emit<KIND>(out0, out1, rb + first_pos, fs0, fs1, false, cs);
            emit<KIND>(out0, out1, rb + cur.pos, ca0, ca1, false, cs);
        }
        emit<KIND>(out0, out1, rb + pself, dg0, dg1, true, cs);
    }
    if (bad) atomicOr(err, 2);
    if (orient) atomicOr(err, 1);
}

__device__ __forceinline__ void neumaier(double& sum, double& c, double v) {
    double t = sum + v;
    c += fabs(sum) >= fabs(v) ? (sum - t) + v : (v - t) + sum;
    sum = t;
}

template <int KIND>
__global__ void k_general_scalar(const int32_t* __restrict__ gen, const int32_t* __restrict__ row_ptr,
                                 const int32_t* __restrict__ col_idx, const int32_t* __restrict__ vptr,
                                 const int2* __restrict__ fan, const double2* __restrict__ q,
                                 const double* __restrict__ w, Consts cs, double* __restrict__ out0,
                                 double* __restrict__ out1, int* __restrict__ err) {
    int32_t i = gen[blockIdx.x];
    int32_t rb = row_ptr[i], u = row_ptr[i + 1] - rb;
    int32_t b0 = vptr[i], d = vptr[i + 1] - b0;
    double2 pi = q[i];
    int bad = 0, orient = 0;
    ff wi = (KIND & W_W) ? ff_from_double(w[i], bad) : ff_make(0.f);
    for (int t = threadIdx.x; t < u; t += blockDim.x) {
        int32_t col = col_idx[rb + t];
        bool self = col == i;
        double s0 = 0.0, c0 = 0.0, s1 = 0.0, c1 = 0.0;
        for (int32_t e = 0; e < d; e++) {
            int2 p = fan[b0 + e];
            int which = self ? 0 : (p.x == col ? 1 : (p.y == col ? 2 : -1));
            if (which < 0) continue;
            Nb j = load_nb<KIND>(q, w, pi, p.x, 0, bad), l = load_nb<KIND>(q, w, pi, p.y, 0, bad);
            RowTerms rt = row_terms<KIND>(q, w, i, j, l, wi, bad);
            orient |= !(rt.d.h > 0.f);
            // the S diagonal term |e_a|^2 / 2D = -(S_ij + S_il) of the same triangle
            if (KIND & W_S) rt.s[0] = ff_neg(ff_add(rt.s[1], rt.s[2]));
            ff v0, v1;
            pick<KIND>(rt, which, v0, v1);
            neumaier(s0, c0, ff_to_double(v0));
            if (KIND == (W_S | W_W)) neumaier(s1, c1, ff_to_double(v1));
        }
        double v = s0 + c0;
        if (KIND == W_M) v *= self ? cs.d12 : cs.d24;
        if (KIND == W_W) v *= cs.d60;
        out0[rb + t] = v;
        if (KIND == (W_S | W_W)) out1[rb + t] = (s1 + c1) * cs.d60;
    }
    if (bad) atomicOr(err, 2);
    if (orient) atomicOr(err, 1);
}

// ---------------------------------------------------------------- elasticity
//
// With e_a = r_j - r_l and, for the three columns b (self, j, l), e_b = e_a, r_l, -r_j and
// r = 1/2D (K^e = |T| B^T C B with grad(phi_a) = (e_a,y, -e_a,x) / D):
//   K[2a][2b]     =  r ((l+2m) ea_y eb_y + m ea_x eb_x)
//   K[2a][2b+1]   = -r (l ea_y eb_x + m ea_x eb_y)
//   K[2a+1][2b]   = -r (l ea_x eb_y + m ea_y eb_x)
//   K[2a+1][2b+1] =  r ((l+2m) ea_x eb_x + m ea_y eb_y)
// Positions in the block-expanded pattern: row 2i + alpha starts at 4 rb + 2 alpha u (u = the
// scalar row length); scalar column position t gives entries 2t and 2t + 1.

namespace {

struct Block2 {
    ff k00, k01, k10, k11;
};

__device__ __forceinline__ Block2 elas_block(ff ax, ff ay, ff bx, ff by, const Consts& cs) {
    // (ax, ay) = r e_a, already scaled by 1/2D
    ff xx = ff_mul(ax, bx), yy = ff_mul(ay, by), yx = ff_mul(ay, bx), xy = ff_mul(ax, by);
    Block2 k;
    k.k00 = ff_add(ff_mul(cs.l2m, yy), ff_mul(cs.mu, xx));
    k.k01 = ff_neg(ff_add(ff_mul(cs.lam, yx), ff_mul(cs.mu, xy)));
    k.k10 = ff_neg(ff_add(ff_mul(cs.lam, xy), ff_mul(cs.mu, yx)));
    k.k11 = ff_add(ff_mul(cs.l2m, xx), ff_mul(cs.mu, yy));
    return k;
}

__device__ __noinline__ ff elas_terms_fp64(const double2* __restrict__ q, int32_t i, int32_t j, int32_t l,
                                           const Consts& cs, Block2 out[3], int& bad) {
    double2 pi = q[i], pj = q[j], pl = q[l];
    double eax = pj.x - pl.x, eay = pj.y - pl.y;
    double e1x = pl.x - pi.x, e1y = pl.y - pi.y;      // e_{a+1} = r_l
    double e2x = pi.x - pj.x, e2y = pi.y - pj.y;      // e_{a+2} = -r_j
    double D = e1x * e2y - e2x * e1y;
    double r = 1.0 / (2.0 * D);
    double ax = r * eax, ay = r * eay;
    double bx[3] = {eax, e1x, e2x}, by[3] = {eay, e1y, e2y};
    double l2m = cs.dl2m, lam = cs.dlam, mu = cs.dmu;
    for (int b = 0; b < 3; b++) {
        out[b].k00 = ff_from_double(l2m * ay * by[b] + mu * ax * bx[b], bad);
        out[b].k01 = ff_from_double(-(lam * ay * bx[b] + mu * ax * by[b]), bad);
        out[b].k10 = ff_from_double(-(lam * ax * by[b] + mu * ay * bx[b]), bad);
        out[b].k11 = ff_from_double(l2m * ax * bx[b] + mu * ay * by[b], bad);
    }
    return ff_from_double(D, bad);
}

__device__ __forceinline__ ff elas_terms(const double2* __restrict__ q, int32_t i, const Nb& j, const Nb& l,
                                         const Consts& cs, Block2 out[3], int& bad) {
    ff D = ff_dot2(j.x, l.x, l.y, ff_neg(j.y));
    if (!well_shaped(j, l, D.h)) return elas_terms_fp64(q, i, j.id, l.id, cs, out, bad);
    ff r = ff_mulf(ff_rcp_fast(D), 0.5f);
    ff eax = ff_sub(j.x, l.x), eay = ff_sub(j.y, l.y);
    ff sax = ff_mul(eax, r), say = ff_mul(eay, r);
    out[0] = elas_block(sax, say, eax, eay, cs);
    out[1] = elas_block(sax, say, l.x, l.y, cs);
    out[2] = elas_block(sax, say, ff_neg(j.x), ff_neg(j.y), cs);
    return D;
}

__device__ __forceinline__ Block2 badd(const Block2& a, const Block2& b) {
    return Block2{ff_add(a.k00, b.k00), ff_add(a.k01, b.k01), ff_add(a.k10, b.k10), ff_add(a.k11, b.k11)};
}

__device__ __forceinline__ void write_block(double* __restrict__ out, int32_t rb, int32_t u, int t, const Block2& k) {
    int32_t o0 = 4 * rb + 2 * t, o1 = 4 * rb + 2 * u + 2 * t;
    out[o0] = ff_to_double(k.k00);
    out[o0 + 1] = ff_to_double(k.k01);
    out[o1] = ff_to_double(k.k10);
    out[o1 + 1] = ff_to_double(k.k11);
}

}  // namespace

__global__ void __launch_bounds__(256, 2) k_fan_elas(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ vptr,
                                                     const int2* __restrict__ fan, const int2* __restrict__ hdr,
                                                     const double2* __restrict__ q, int32_t nq, Consts cs,
                                                     double* __restrict__ out, int* __restrict__ err) {
    int bad = 0, orient = 0;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nq; r += (int64_t)gridDim.x * blockDim.x) {
        int32_t i = (int32_t)r;
        int2 h = hdr[i];
        int kind = h.y >> 28;
        if (kind > 1) continue;
        int32_t rb = row_ptr[i], u = row_ptr[i + 1] - rb, b0 = vptr[i], d = vptr[i + 1] - b0;
        int pself = h.y & 0x3FFF;
        const int2 last = kind == 1 ? make_int2(h.x, (h.y >> 14) & 0x3FFF) : fan[b0];
        double2 pi = q[i];
        Raw rn = load_raw<0>(q, nullptr, fan[b0]);
        Raw rp = load_raw<0>(q, nullptr, d > 1 ? fan[b0 + 1] : last);
        Nb cur = make_nb<0>(rn, pi, bad);
        const int first_pos = cur.pos;
        const ff z = ff_make(0.f);
        Block2 dg = {z, z, z, z}, fs = dg, ca = dg;
        for (int32_t e = 0; e < d; e++) {
            rn = rp;
            if (e + 2 <= d) rp = load_raw<0>(q, nullptr, e + 2 < d ? fan[b0 + e + 2] : last);
            Nb nxt = make_nb<0>(rn, pi, bad);
            Block2 k[3];
            ff D = elas_terms(q, i, cur, nxt, cs, k, bad);
            orient |= !(D.h > 0.f);
            dg = badd(dg, k[0]);
            if (e == 0) fs = k[1];
            else write_block(out, rb, u, cur.pos, badd(ca, k[1]));
            ca = k[2];
            cur = nxt;
        }
        if (kind == 0) {
            write_block(out, rb, u, first_pos, badd(fs, ca));
        } else {
            write_block(out, rb, u, first_pos, fs);
            write_block(out, rb, u, cur.pos, ca);
        }
        write_block(out, rb, u, pself, dg);
    }
    if (bad) atomicOr(err, 2);
    if (orient) atomicOr(err, 1);
}

__global__ void k_general_elas(const int32_t* __restrict__ gen, const int32_t* __restrict__ row_ptr,
                               const int32_t* __restrict__ col_idx, const int32_t* __restrict__ vptr,
                               const int2* __restrict__ fan, const double2* __restrict__ q, Consts cs,
                               double* __restrict__ out, int* __restrict__ err) {
    int32_t i = gen[blockIdx.x];
    int32_t rb = row_ptr[i], u = row_ptr[i + 1] - rb;
    int32_t b0 = vptr[i], d = vptr[i + 1] - b0;
    double2 pi = q[i];
    int bad = 0, orient = 0;
    for (int t = threadIdx.x; t < u; t += blockDim.x) {
        int32_t col = col_idx[rb + t];
        bool self = col == i;
        double s[4] = {0, 0, 0, 0}, c[4] = {0, 0, 0, 0};
        for (int32_t e = 0; e < d; e++) {
            int2 p = fan[b0 + e];
            int which = self ? 0 : (p.x == col ? 1 : (p.y == col ? 2 : -1));
            if (which < 0) continue;
            Nb j = load_nb<0>(q, nullptr, pi, p.x, 0, bad), l = load_nb<0>(q, nullptr, pi, p.y, 0, bad);
            Block2 k[3];
            ff D = elas_terms(q, i, j, l, cs, k, bad);
            orient |= !(D.h > 0.f);
            neumaier(s[0], c[0], ff_to_double(k[which].k00));
            neumaier(s[1], c[1], ff_to_double(k[which].k01));
            neumaier(s[2], c[2], ff_to_double(k[which].k10));
            neumaier(s[3], c[3], ff_to_double(k[which].k11));
        }
        int32_t o0 = 4 * rb + 2 * t, o1 = 4 * rb + 2 * u + 2 * t;
        out[o0] = s[0] + c[0];
        out[o0 + 1] = s[1] + c[1];
        out[o1] = s[2] + c[2];
        out[o1 + 1] = s[3] + c[3];
    }
    if (bad) atomicOr(err, 2);
    if (orient) atomicOr(err, 1);
}

// ---------------------------------------------------------------- host side

static ff host_ff(double v) {
    ff r;
    r.h = (float)v;
    r.l = (float)(v - (double)r.h);
    return r;
}

static Consts make_consts(double lam, double mu) {
    Consts c;
    c.c60 = host_ff(1.0 / 60.0);
    c.c12 = host_ff(1.0 / 12.0);
    c.c24 = host_ff(1.0 / 24.0);
    c.l2m = host_ff(lam + 2.0 * mu);
    c.lam = host_ff(lam);
    c.mu = host_ff(mu);
    c.d60 = 1.0 / 60.0;
    c.d12 = 1.0 / 12.0;
    c.d24 = 1.0 / 24.0;
    c.dl2m = lam + 2.0 * mu;
    c.dlam = lam;
    c.dmu = mu;
    return c;
}

static constexpr int FAN_BLOCK = 256;
static constexpr int GEN_BLOCK = 64;

template <int KIND>
static fe_status launch_scalar(fe_mesh m, fe_pattern p, const double* w, double* out0, double* out1, cudaStream_t s) {
    Consts cs = make_consts(0.0, 0.0);
    { FE_PROF("k_fan_scalar", s); k_fan_scalar<KIND><<<fe_grid(m->nq, FAN_BLOCK, 8), FAN_BLOCK, 0, s>>>(p->row_ptr, p->vptr, p->fan, p->hdr, m->q, w, m->nq, cs, out0, out1, m->err); }
    FE_LAUNCHED("k_fan_scalar");
    if (p->n_gen > 0) {
        { FE_PROF("k_general_scalar", s); k_general_scalar<KIND><<<p->n_gen, GEN_BLOCK, 0, s>>>(p->gen_rows, p->row_ptr, p->col_idx, p->vptr, p->fan, m->q, w, cs, out0, out1, m->err); }
        FE_LAUNCHED("k_general_scalar");
    }
    return FE_OK;
}

fe_status fe_row_scalar(int kind_bits, fe_mesh m, fe_pattern p, const double* w, double* out0, double* out1,
                        cudaStream_t s) {
    if (m->nq == 0 || p->nnz_scalar == 0) return FE_OK;
    switch (kind_bits) {
        case W_S: return launch_scalar<W_S>(m, p, w, out0, out1, s);
        case W_W: return launch_scalar<W_W>(m, p, w, out0, out1, s);
        case W_M: return launch_scalar<W_M>(m, p, w, out0, out1, s);
        case W_S | W_W: return launch_scalar<W_S | W_W>(m, p, w, out0, out1, s);
    }
    return fe_fail(FE_ERR_INVALID_ARG, "internal: bad row kind");
}

fe_status fe_row_elas(fe_mesh m, fe_pattern p, double lam, double mu, double* out, cudaStream_t s) {
    if (m->nq == 0 || p->nnz_scalar == 0) return FE_OK;
    Consts cs = make_consts(lam, mu);
    { FE_PROF("k_fan_elas", s); k_fan_elas<<<fe_grid(m->nq, FAN_BLOCK, 8), FAN_BLOCK, 0, s>>>(p->row_ptr, p->vptr, p->fan, p->hdr, m->q, m->nq, cs, out, m->err); }
    FE_LAUNCHED("k_fan_elas");
    if (p->n_gen > 0) {
        { FE_PROF("k_general_elas", s); k_general_elas<<<p->n_gen, GEN_BLOCK, 0, s>>>(p->gen_rows, p->row_ptr, p->col_idx, p->vptr, p->fan, m->q, cs, out, m->err); }
        FE_LAUNCHED("k_general_elas");
    }
    return FE_OK;
}
