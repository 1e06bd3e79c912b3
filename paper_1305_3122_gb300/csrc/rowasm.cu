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
// General rows (several chains, long fans, non-manifold) use one block per row. Each triangle's
// contributions to its three columns are computed once (for rows of up to 256 triangles) and kept
// as double-floats. Thread t owns column t: an off-diagonal column adds its few contributions in
// the row's stored (sorted) triangle order, and the diagonal's d contributions are added by a
// fixed-shape pairwise tree over the block, all in double-float. (Longer rows: each column's
// contributions, recomputed, converted to FP64 and added by Neumaier's compensated summation.)
// Both paths fix the order of every sum, so the result is bit-identical from run to run.
#include "ff.cuh"
#include "internal.cuh"

namespace {

enum { W_S = 1, W_W = 2, W_M = 4 };

struct Consts {
    ff c60, c12, c24, c120;     // 1/60, 1/12, 1/24, 1/120 as double-floats
    ff l2m, lam, mu;            // lambda + 2 mu, lambda, mu (elasticity)
    double d60, d12, d24;       // the same in FP64 (general rows)
};

// A neighbour of the row's vertex: relative coordinates r = p - p_i and weight as double-floats,
// the approximate float value of |r|^2 (for the conditioning test), vertex id and column
// position.
struct Nb {
    ff x, y, w;
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

// A badly shaped triangle (i, c, n) (a small angle, see the shape tests): the quantities that
// double-float arithmetic on the split relative coordinates would get wrong by too much come from
// FP64 coordinate differences (each correctly rounded) and are then split: D = r_c x r_n (a
// cancelling difference of products), the edge e_a = p_c - p_n (a difference of nearly equal
// vectors when the angle at i is small), and the stiffness's two dot products e_a . r_n and
// e_a . r_c (which cancel when the angles at n and c are near 90 degrees, as they are when the
// angle at i is small; a row whose only triangle is such a sliver has only such small entries).
// 1/2D and the products by it stay in double-float. 12 FP64 instructions, against about 40 (with
// a division) for the same terms entirely in FP64. Inlined: a call's register and stack handling
// cost the fan kernel 10 registers and 5% of its time. The elasticity blocks take D and e_a from here
// and form their products in double-float: each of their rows keeps entries of the size of
// |e_a| |r| / 2D that do not cancel, so those products' rounding stays small against the row.
__device__ __forceinline__ void thin_terms(const double2* __restrict__ q, int32_t i, int32_t c, int32_t n, ff& D, ff& ax,
                                        ff& ay, ff* dn, ff* dc, int& bad) {
    const double2 pi = q[i], pc = q[c], pn = q[n];
    const double cx = pc.x - pi.x, cy = pc.y - pi.y, nx = pn.x - pi.x, ny = pn.y - pi.y;
    const double ex = pc.x - pn.x, ey = pc.y - pn.y;
    D = ff_from_value(fma(cx, ny, -(cy * nx)), bad);
    ax = ff_from_double(ex, bad);
    ay = ff_from_double(ey, bad);
    if (dn) *dn = ff_from_value(fma(ex, nx, ey * ny), bad);     // e_a . r_n
    if (dc) *dc = ff_from_value(fma(ex, cx, ey * cy), bad);     // e_a . r_c
}

// Shape tests. sin^2 of an angle is D^2 over the product of its two squared edges.
// For the scalar kinds only the angle at the row's own vertex i matters. D, the edge e_a and the
// stiffness's dot products lose bits, relative to the row's largest entry, only when that angle is
// small: D by 1/sin(angle at i); e_a when it is short against r; the dot products when the
// other two angles are near 90 degrees, so that the row's entries are small. A small angle at c
// or n makes the dot products' terms large, but the row's diagonal then grows as 1/sin of that
// angle too. So the fast path needs sin^2(angle at i) >= 1/16 (about 14.5 degrees; scalar_shaped).
// The elasticity blocks' mixed products are not covered by that argument, so they keep the test of
// all three angles (well_shaped).
__device__ __forceinline__ bool scalar_shaped(const Nb& j, const Nb& l, float dh) {
    return 16.0f * dh * dh >= j.n * l.n;
}

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
    ff ax = ff_sub(j.x, l.x), ay = ff_sub(j.y, l.y);            // e_a = r_j - r_l
    ff dl, dj;                                                  // e_a . r_l, e_a . r_j
    if (scalar_shaped(j, l, t.d.h)) {
        if (KIND & W_S) {
            dl = ff_dot2(ax, ay, l.x, l.y);
            dj = ff_dot2(ax, ay, j.x, j.y);
        }
    } else {
        thin_terms(q, i, j.id, l.id, t.d, ax, ay, (KIND & W_S) ? &dl : nullptr, (KIND & W_S) ? &dj : nullptr, bad);
    }
    if (KIND & W_S) {
        ff inv = ff_mulf(ff_rcp_fast(t.d), 0.5f);              // 1 / 2D
        t.s[1] = ff_mul(dl, inv);                               // e_a . r_l / 2D
        t.s[2] = ff_neg(ff_mul(dj, inv));                       // e_a . (-r_j) / 2D
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

// per-contribution values of the two outputs (out0: S, else M^w, else M; out1: M^w or M with S),
// unscaled (M^w by 1/60, M by 1/12 or 1/24 at the end)
template <int KIND>
__device__ __forceinline__ void pick(const RowTerms& t, int which, ff& v0, ff& v1) {
    if (KIND & W_S) v0 = t.s[which];
    else if (KIND & W_W) v0 = t.w[which];
    else v0 = t.d;
    v1 = !(KIND & W_S) ? ff_make(0.f) : (KIND & W_W) ? t.w[which] : (KIND & W_M) ? t.d : ff_make(0.f);
}

}  // namespace

// ---------------------------------------------------------------- scalar fan kernel
//
// Triangle e of a simple row's fan is (i, c, n) with c = n_e, n = n_{e+1} (counter-clockwise),
// D_e = r_c x r_n = 2|T_e| and e_a = r_c - r_n its edge opposite i. Its contributions to row i:
//   S   (Eq. 3):  column c: e_a . r_n / 2D          column n: -e_a . r_c / 2D
//                 (e_a formed first: the Gram form r_c . r_n - |r_n|^2 cancels badly when the
//                 edges at i are long against e_a)
//   M^w (Eq. 2):  column c: (D u_c + B_e) / 120     column n: (D u_n + A_e) / 120
//                 diagonal: (3 w_i D + A_e + B_e) / 60
//                 with A_e = D w_c, B_e = D w_n and u_k = 2 (w_i + w_k) per neighbour
//   M   (Eq. 1):  columns D / 24, diagonal D / 12.
// Column n_e collects triangles e-1 and e; their D's are summed first, so the M^w entry is
// ((D_{e-1} + D_e) u + A_{e-1} + B_e) / 120 with one product by u. The S diagonal is minus the
// sum of the row's off-diagonal S entries (S 1 = 0).

namespace {

// Vertex record of the weighted kinds: coordinates (FP64) and the weight already split into a
// double-float, 32 bytes, so a neighbour's data is one sector (one DRAM access on a miss)
// instead of a 16-byte and an 8-byte gather from two arrays.
struct __align__(16) VRec {
    double x, y;
    float wh, wl, pad0, pad1;
};

__global__ void k_pack_vrec(const double2* __restrict__ q, const double* __restrict__ w, int32_t nq,
                            VRec* __restrict__ vr, int* __restrict__ err) {
    int bad = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < (uint32_t)nq; i += gridDim.x * blockDim.x) {
        ff wf = ff_from_double(w[i], bad);
        VRec r;
        double2 p = q[i];
        r.x = p.x;
        r.y = p.y;
        r.wh = wf.h;
        r.wl = wf.l;
        r.pad0 = r.pad1 = 0.f;
        vr[i] = r;
    }
    if (bad) atomicOr(err, 2);
}

// Coordinates, weight and fan record of one neighbour, loaded one triangle ahead of its use.
struct FanRaw {
    double2 p;
    ff w;
    int32_t id;
    int pos;
};

template <int KIND>
__device__ __forceinline__ FanRaw fan_load(const double2* __restrict__ q, const VRec* __restrict__ vr, int2 rec) {
    FanRaw r;
    if (KIND & W_W) {
        const double2* a2 = reinterpret_cast<const double2*>(vr + rec.x);
        r.p = a2[0];
        float4 t = *reinterpret_cast<const float4*>(a2 + 1);
        r.w = ff{t.x, t.y};
    } else {
        r.p = q[rec.x];
        r.w = z_ff();
    }
    r.id = rec.x;
    r.pos = rec.y;
    return r;
}

// A neighbour of the row's vertex in the scalar fan kernel.
struct FanNb {
    ff x, y;      // r = p - p_i
    float n;      // |r|^2 from the high words (shape test)
    ff w;         // w at the neighbour      (M^w)
    int32_t id;
    int pos;
};

// 2 (w_i + w_k) of a neighbour k (M^w)
__device__ __forceinline__ ff fan_u(ff wi2, const FanNb& k) { return ff_add(wi2, ff{FADD(k.w.h, k.w.h), FADD(k.w.l, k.w.l)}); }

template <int KIND>
__device__ __forceinline__ FanNb fan_nb(const FanRaw& r, double2 pi, int& bad) {
    FanNb b;
    b.x = ff_from_double(r.p.x - pi.x, bad);              // exact FP64 differences, then split
    b.y = ff_from_double(r.p.y - pi.y, bad);
    b.n = b.x.h * b.x.h + b.y.h * b.y.h;
    b.w = r.w;
    b.id = r.id;
    b.pos = r.pos;
    return b;
}

// The scalar shape test (the angle at the row's vertex, as scalar_shaped) on the float parts.
__device__ __forceinline__ bool fan_well_shaped(const FanNb& c, const FanNb& n, float dh) {
    return 16.0f * dh * dh >= c.n * n.n;
}

// FP64 value of a row entry.
__device__ __forceinline__ void put(double* __restrict__ out, int32_t at, ff v) { out[at] = ff_to_double(v); }

// Sizes the bounds-checked build checks derived indices against: vertices, fan records (3 nme),
// stored entries of the output.
struct Lim {
    int32_t nq;
    int64_t n_inc, nnz;
};

// A fan record (neighbour id, column position) at index t of the fan records.
__device__ __forceinline__ int2 fan_rec(const int2* __restrict__ fan, int64_t t, const Lim& lim) {
    int2 r = fan[FE_IDX(t, lim.n_inc)];
    r.x = FE_IDX(r.x, lim.nq);
    return r;
}

}  // namespace

// One simple row of the scalar kinds (S, M^w, M, or two of them): see the header of this section.
// KIND bits: W_S stiffness, W_W weighted mass, W_M mass. The first matrix goes to out0, a second
// one (with W_S) to out1.
template <int KIND>
__device__ __forceinline__ void fan_row(int32_t i, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ vptr,
                                        const int2* __restrict__ fan, const int2* __restrict__ hdr,
                                        const double2* __restrict__ q, const VRec* __restrict__ vr, const Consts& cs,
                                        double* __restrict__ out0, double* __restrict__ out1, int& bad, int& orient,
                                        const Lim& lim) {
    constexpr bool DS = (KIND & W_S) != 0, DW = (KIND & W_W) != 0, DM = (KIND & W_M) != 0;
    double* __restrict__ outX = DS ? out1 : out0;            // M^w or M
    int2 h = hdr[i];
    int kind = h.y >> 28;
    if (kind > 1) return;                                    // general row (or no triangle)
    int32_t rb = row_ptr[i], b0 = vptr[i], d = vptr[i + 1] - b0;
    int pself = h.y & 0x3FFF;
    // neighbour k of the fan: k < d from the fan records; k == d is the last neighbour of an
    // open fan (from the header) or n_0 again for a closed fan
    const int2 rec0 = fan_rec(fan, b0, lim);
    const int2 last = kind == 1 ? make_int2(FE_IDX(h.x, lim.nq), (h.y >> 14) & 0x3FFF) : rec0;
    FanRaw self = fan_load<KIND>(q, vr, make_int2(i, 0));
    double2 pi = self.p;
    ff wi2 = ff{FADD(self.w.h, self.w.h), FADD(self.w.l, self.w.l)};   // 2 w_i (M^w)
    // neighbour data are loaded one triangle ahead of their use and fan records two ahead, so a
    // gather never waits for its own record (N_k = fan[b0 + k] for k < d, N_d = last); loading
    // the data two ahead costs more in occupancy than it gains
    FanRaw rn = fan_load<KIND>(q, vr, rec0);
    FanRaw rp = fan_load<KIND>(q, vr, d > 1 ? fan_rec(fan, b0 + 1, lim) : last);
    int2 recn = d > 2 ? fan_rec(fan, b0 + 2, lim) : last;    // N_2
    FanNb cur = fan_nb<KIND>(rn, pi, bad);
    const int first_pos = cur.pos;
    const ff first_u = DW ? fan_u(wi2, cur) : z_ff();
    ff caS = z_ff(), fsS = z_ff(), dgS = z_ff();                      // S
    ff Dp = z_ff(), Ap = z_ff(), fsD = z_ff(), fsM = z_ff();          // M^w / M carries
    ff sD = z_ff(), sAB = z_ff();                                     // diagonal sums
    for (int32_t e = 0; e < d; e++) {
        rn = rp;                                             // neighbour e + 1 (already loaded)
        if (e + 2 <= d) {
            rp = fan_load<KIND>(q, vr, recn);                // N_{e+2}
            recn = e + 3 < d ? fan_rec(fan, b0 + e + 3, lim) : last;   // N_{e+3}
        }
        FanNb nxt = fan_nb<KIND>(rn, pi, bad);
        ff D = ff_dot2(cur.x, nxt.x, nxt.y, ff_neg(cur.y));          // r_c x r_n
        ff ax = ff_sub(cur.x, nxt.x), ay = ff_sub(cur.y, nxt.y);      // e_a
        ff dn, dc;                                                    // e_a . r_n, e_a . r_c
        if (fan_well_shaped(cur, nxt, D.h)) {
            if (DS) {
                dn = ff_dot2(ax, ay, nxt.x, nxt.y);
                dc = ff_dot2(ax, ay, cur.x, cur.y);
            }
        } else {
            thin_terms(q, i, cur.id, nxt.id, D, ax, ay, DS ? &dn : nullptr, DS ? &dc : nullptr, bad);
        }
        ff sc = z_ff(), sn = z_ff();
        if (DS) {
            ff inv = ff_rcp_fast(D);
            inv = ff{0.5f * inv.h, 0.5f * inv.l};                   // 1 / 2D
            sc = ff_mul(dn, inv);
            sn = ff_neg(ff_mul(dc, inv));
        }
        orient |= !(D.h > 0.f);
        ff A = z_ff(), B = z_ff();
        if (DW) {
            A = ff_mul(D, cur.w);
            B = ff_mul(D, nxt.w);
            ff_acc(sAB, ff_add(A, B));
        }
        ff_acc(sD, D);
        if (e == 0) {
            fsS = sc;
            fsD = D;
            if (DW) fsM = ff_add(ff_mul(D, first_u), B);             // n_0's share of triangle 0
        } else {
            // column n_e is complete: triangles e - 1 and e
            ff sig = ff_add(Dp, D);
            if (DS) {
                ff v = ff_add(caS, sc);
                ff_acc(dgS, ff_neg(v));
                put(out0, FE_IDX(rb + cur.pos, lim.nnz), v);
            }
            if (DW) put(outX, FE_IDX(rb + cur.pos, lim.nnz), ff_mul(ff_add(ff_add(ff_mul(sig, fan_u(wi2, cur)), Ap), B), cs.c120));
            if (DM) put(outX, FE_IDX(rb + cur.pos, lim.nnz), ff_mul(sig, cs.c24));
        }
        caS = sn;
        Dp = D;
        Ap = A;
        cur = nxt;
    }
    if (kind == 0) {                                         // closed: n_0 meets triangle d - 1
        if (DS) {
            ff v = ff_add(caS, fsS);
            ff_acc(dgS, ff_neg(v));
            put(out0, FE_IDX(rb + first_pos, lim.nnz), v);
        }
        if (DW) put(outX, FE_IDX(rb + first_pos, lim.nnz), ff_mul(ff_add(ff_add(ff_mul(Dp, first_u), Ap), fsM), cs.c120));
        if (DM) put(outX, FE_IDX(rb + first_pos, lim.nnz), ff_mul(ff_add(Dp, fsD), cs.c24));
    } else {                                                 // open: n_0 and n_d have one triangle each
        if (DS) {
            ff_acc(dgS, ff_neg(fsS));
            ff_acc(dgS, ff_neg(caS));
            put(out0, FE_IDX(rb + first_pos, lim.nnz), fsS);
            put(out0, FE_IDX(rb + cur.pos, lim.nnz), caS);
        }
        if (DW) {
            put(outX, FE_IDX(rb + first_pos, lim.nnz), ff_mul(fsM, cs.c120));
            put(outX, FE_IDX(rb + cur.pos, lim.nnz), ff_mul(ff_add(ff_mul(Dp, fan_u(wi2, cur)), Ap), cs.c120));
        }
        if (DM) {
            put(outX, FE_IDX(rb + first_pos, lim.nnz), ff_mul(fsD, cs.c24));
            put(outX, FE_IDX(rb + cur.pos, lim.nnz), ff_mul(Dp, cs.c24));
        }
    }
    if (DS) put(out0, FE_IDX(rb + pself, lim.nnz), dgS);
    if (DW) put(outX, FE_IDX(rb + pself, lim.nnz), ff_mul(ff_add(ff_mul(ff_mulf(wi2, 1.5f), sD), sAB), cs.c60));
    if (DM) put(outX, FE_IDX(rb + pself, lim.nnz), ff_mul(sD, cs.c12));
}

// Resident blocks of 128 threads per SM for each kind: as many as fit without register spills
// (measured at 2048 x 2048 cells: S and M run fastest at 7, the weighted kinds at 5).
template <int KIND>
struct FanOcc {
    static constexpr int blocks = (KIND == W_S || KIND == W_M) ? 7 : (KIND == (W_S | W_M) ? 6 : 5);
};

template <int KIND>
__global__ void __launch_bounds__(128, FanOcc<KIND>::blocks) k_fan_scalar(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ vptr,
                                                       const int2* __restrict__ fan, const int2* __restrict__ hdr,
                                                       const double2* __restrict__ q, const VRec* __restrict__ vr, int32_t r0,
                                                       int32_t r1, Consts cs, double* __restrict__ out0, double* __restrict__ out1,
                                                       int* __restrict__ err, Lim lim) {
    int bad = 0, orient = 0;
    for (uint32_t r = r0 + blockIdx.x * blockDim.x + threadIdx.x; r < (uint32_t)r1; r += gridDim.x * blockDim.x)
        fan_row<KIND>((int32_t)r, row_ptr, vptr, fan, hdr, q, vr, cs, out0, out1, bad, orient, lim);
    if (bad) atomicOr(err, 2);
    if (orient) atomicOr(err, 1);
}

__device__ __forceinline__ void neumaier(double& sum, double& c, double v) {
    double t = sum + v;
    c += fabs(sum) >= fabs(v) ? (sum - t) + v : (v - t) + sum;
    sum = t;
}

// One general row, by one block: thread t owns column t of the row.
// General rows: one warp each, GEN_WARPS warps per block. A row of at most GEN_SMEM_TRIS
// triangles keeps its triangles' terms in the warp's part of shared memory; longer rows recompute
// each triangle's terms in every lane that needs them.
constexpr int GEN_WARPS = 4;
constexpr int GEN_SMEM_TRIS = 64;

// Sum of one double-float per lane over the warp, by a fixed-shape tree (the same bits every run;
// for non-negative terms an error of about 7 units of 2^-48 of the sum). Every lane gets it.
__device__ __forceinline__ ff warp_sum_ff(ff a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ff b{__shfl_xor_sync(0xffffffffu, a.h, o), __shfl_xor_sync(0xffffffffu, a.l, o)};
        // both lanes of a pair add the same two values in the same order (lower lane first)
        a = (threadIdx.x & o) ? ff_add(b, a) : ff_add(a, b);
    }
    return a;
}

template <int KIND>
__device__ __forceinline__ void general_row(int32_t i, const int32_t* __restrict__ row_ptr,
                                            const int32_t* __restrict__ col_idx, const int32_t* __restrict__ vptr,
                                            const int2* __restrict__ fan, const double2* __restrict__ q,
                                            const double* __restrict__ w, const Consts& cs, double* __restrict__ out0,
                                            double* __restrict__ out1, int& bad, int& orient) {
    constexpr bool TWO = (KIND & W_S) && (KIND & (W_W | W_M));   // a second matrix in out1
    constexpr int M1 = TWO ? 1 : 0;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int32_t rb = row_ptr[i], u = row_ptr[i + 1] - rb;
    int32_t b0 = vptr[i], d = vptr[i + 1] - b0;
    double2 pi = q[i];
    ff wi = (KIND & W_W) ? ff_from_double(w[i], bad) : ff_make(0.f);
    if (d <= GEN_SMEM_TRIS) {
        // each triangle's contributions to its three columns (self, j, l) computed once by one
        // lane and kept as double-floats; the sums run in double-float too, as on the fast path,
        // and only each entry's value is converted to FP64 (GB300's FP64 rate made FP64 sums the
        // bound of this kernel)
        __shared__ int2 sp_all[GEN_WARPS][GEN_SMEM_TRIS];
        __shared__ ff sv_all[GEN_WARPS][TWO ? 2 : 1][3][GEN_SMEM_TRIS];
        int2* sp = sp_all[wid];
        auto sv = sv_all[wid];
        ff a0 = z_ff(), a1 = z_ff();                                 // this lane's diagonal terms
        for (int e = lane; e < d; e += 32) {
            int2 p = fan[b0 + e];
            sp[e] = p;
            Nb j = load_nb<KIND>(q, w, pi, p.x, 0, bad), l = load_nb<KIND>(q, w, pi, p.y, 0, bad);
            RowTerms rt = row_terms<KIND>(q, w, i, j, l, wi, bad);
            orient |= !(rt.d.h > 0.f);
            if (KIND & W_S) rt.s[0] = ff_neg(ff_add(rt.s[1], rt.s[2]));
#pragma unroll
            for (int which = 0; which < 3; which++) {
                ff v0, v1;
                pick<KIND>(rt, which, v0, v1);
                sv[0][which][e] = v0;
                if (TWO) sv[M1][which][e] = v1;
                if (which == 0) {
                    a0 = ff_add(a0, v0);
                    if (TWO) a1 = ff_add(a1, v1);
                }
            }
        }
        // the diagonal's d terms (all positive for S, M^w and M): each lane's in order, then the
        // warp's tree
        const ff dg0 = warp_sum_ff(a0);
        const ff dg1 = TWO ? warp_sum_ff(a1) : z_ff();
        __syncwarp();
        for (int t = lane; t < u; t += 32) {
            int32_t col = col_idx[rb + t];
            bool self = col == i;
            ff v0 = z_ff(), v1 = z_ff();
            if (self) {
                v0 = dg0;
                v1 = dg1;
            } else {
                // an off-diagonal column takes one term from each triangle on its edge: two for an
                // interior edge of a manifold mesh. Up to four are found by integer compares and
                // added in stored order by the same additions in every lane (absent terms are
                // zeros); more (an edge of more than four triangles) in a loop over them.
                int p0 = -1, p1 = -1, p2 = -1, p3 = -1, n = 0;
                for (int32_t e = 0; e < d; e++) {
                    int2 p = sp[e];
                    int which = p.x == col ? 1 : (p.y == col ? 2 : -1);
                    if (which < 0) continue;
                    int code = 3 * e + which;
                    p0 = n == 0 ? code : p0;
                    p1 = n == 1 ? code : p1;
                    p2 = n == 2 ? code : p2;
                    p3 = n == 3 ? code : p3;
                    n++;
                }
                if (n <= 4) {
                    auto term = [&](int code, int m) { return code < 0 ? z_ff() : sv[m][code % 3][code / 3]; };
                    v0 = ff_add(ff_add(ff_add(term(p0, 0), term(p1, 0)), term(p2, 0)), term(p3, 0));
                    if (TWO) v1 = ff_add(ff_add(ff_add(term(p0, M1), term(p1, M1)), term(p2, M1)), term(p3, M1));
                } else {
                    for (int32_t e = 0; e < d; e++) {
                        int2 p = sp[e];
                        int which = p.x == col ? 1 : (p.y == col ? 2 : -1);
                        if (which < 0) continue;
                        v0 = ff_add(v0, sv[0][which][e]);
                        if (TWO) v1 = ff_add(v1, sv[M1][which][e]);
                    }
                }
            }
            if (KIND == W_M) v0 = ff_mul(v0, self ? cs.c12 : cs.c24);
            if (KIND == W_W) v0 = ff_mul(v0, cs.c60);
            out0[rb + t] = ff_to_double(v0);
            if (TWO) out1[rb + t] = ff_to_double(ff_mul(v1, (KIND & W_W) ? cs.c60 : (self ? cs.c12 : cs.c24)));
        }
        __syncwarp();
        return;
    }
    for (int t = lane; t < u; t += 32) {
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
            if (TWO) neumaier(s1, c1, ff_to_double(v1));
        }
        double v = s0 + c0;
        if (KIND == W_M) v *= self ? cs.d12 : cs.d24;
        if (KIND == W_W) v *= cs.d60;
        const double scale1 = (KIND & W_W) ? cs.d60 : (self ? cs.d12 : cs.d24);
        out0[rb + t] = v;
        if (TWO) out1[rb + t] = (s1 + c1) * scale1;
    }
}

// General rows of the list (n of them) that lie in [r0, r1) (a row window), one warp each.
template <int KIND>
__global__ void __launch_bounds__(32 * GEN_WARPS) k_general_scalar(const int32_t* __restrict__ gen, int32_t n,
                                 const int32_t* __restrict__ row_ptr,
                                 const int32_t* __restrict__ col_idx, const int32_t* __restrict__ vptr,
                                 const int2* __restrict__ fan, const double2* __restrict__ q,
                                 const double* __restrict__ w, Consts cs, double* __restrict__ out0,
                                 double* __restrict__ out1, int* __restrict__ err, int32_t r0, int32_t r1) {
    const int32_t g = blockIdx.x * GEN_WARPS + (threadIdx.x >> 5);
    if (g >= n) return;
    const int32_t i = gen[g];
    if (i < r0 || i >= r1) return;
    int bad = 0, orient = 0;
    general_row<KIND>(i, row_ptr, col_idx, vptr, fan, q, w, cs, out0, out1, bad, orient);
    if (bad) atomicOr(err, 2);
    if (orient) atomicOr(err, 1);
}

// ---------------------------------------------------------------- batches of meshes
//
// S and M (W_S | W_M) of many meshes by row owners: one persistent launch walks a list of row
// tiles (mesh, first row, end row); general rows of all meshes are a second list, one block
// each. Output pointers come from device tables, so new output buffers need no new launch.

__global__ void __launch_bounds__(256) k_batch_rows(const fe_row_mesh* __restrict__ desc,
                                                    const fe_row_tile* __restrict__ tiles, int32_t ntiles,
                                                    double* const* __restrict__ S, double* const* __restrict__ M,
                                                    Consts cs) {
    for (int32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        fe_row_tile tl = tiles[t];
        fe_row_mesh d = desc[tl.mesh];
        double* s = S[tl.mesh];
        double* m = M[tl.mesh];
        int bad = 0, orient = 0;
        for (int32_t i = tl.r0 + threadIdx.x; i < tl.r1; i += blockDim.x)
            fan_row<W_S | W_M>(i, d.row_ptr, d.vptr, d.fan, d.hdr, d.q, nullptr, cs, s, m, bad, orient,
                               Lim{d.nq, d.n_inc, d.nnz});
        if (bad) atomicOr(d.err, 2);
        if (orient) atomicOr(d.err, 1);
    }
}

__global__ void __launch_bounds__(32 * GEN_WARPS) k_batch_general(const fe_row_mesh* __restrict__ desc, const int2* __restrict__ list,
                                                                   int32_t n, double* const* __restrict__ S,
                                                                   double* const* __restrict__ M, Consts cs) {
    const int32_t g = blockIdx.x * GEN_WARPS + (threadIdx.x >> 5);
    if (g >= n) return;
    int2 e = list[g];                                            // (mesh, row), one warp
    fe_row_mesh d = desc[e.x];
    int bad = 0, orient = 0;
    general_row<W_S | W_M>(e.y, d.row_ptr, d.col_idx, d.vptr, d.fan, d.q, nullptr, cs, S[e.x], M[e.x], bad, orient);
    if (bad) atomicOr(d.err, 2);
    if (orient) atomicOr(d.err, 1);
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

// The three 2 x 2 blocks of triangle (i, j, l) in row i: out[0] (column i), out[1] (column j),
// out[2] (column l). (Row owners of simple rows compute only the last two: K annihilates the
// translations, since the gradients of a triangle's basis functions sum to zero, so each 2 x 2
// diagonal block of the assembled K is minus the sum of its row's off-diagonal blocks.)
__device__ __forceinline__ ff elas_terms(const double2* __restrict__ q, int32_t i, const Nb& j, const Nb& l,
                                         const Consts& cs, Block2 out[3], int& bad) {
    ff D = ff_dot2(j.x, l.x, l.y, ff_neg(j.y));
    ff eax = ff_sub(j.x, l.x), eay = ff_sub(j.y, l.y);
    if (!well_shaped(j, l, D.h)) thin_terms(q, i, j.id, l.id, D, eax, eay, nullptr, nullptr, bad);
    ff r = ff_mulf(ff_rcp_fast(D), 0.5f);
    ff sax = ff_mul(eax, r), say = ff_mul(eay, r);
    out[0] = elas_block(sax, say, eax, eay, cs);
    out[1] = elas_block(sax, say, l.x, l.y, cs);
    out[2] = elas_block(sax, say, ff_neg(j.x), ff_neg(j.y), cs);
    return D;
}

__device__ __forceinline__ Block2 badd(const Block2& a, const Block2& b) {
    return Block2{ff_add(a.k00, b.k00), ff_add(a.k01, b.k01), ff_add(a.k10, b.k10), ff_add(a.k11, b.k11)};
}

__device__ __forceinline__ void write_block(double* __restrict__ out, int32_t rb, int32_t u, int t, const Block2& k,
                                            int64_t nnz4 = INT64_MAX) {
    int32_t o0 = FE_IDX(4 * rb + 2 * t, nnz4 - 1), o1 = FE_IDX(4 * rb + 2 * u + 2 * t, nnz4 - 1);
    out[o0] = ff_to_double(k.k00);
    out[o0 + 1] = ff_to_double(k.k01);
    out[o1] = ff_to_double(k.k10);
    out[o1 + 1] = ff_to_double(k.k11);
}

}  // namespace

__device__ __forceinline__ Block2 bneg(const Block2& a) { return Block2{ff_neg(a.k00), ff_neg(a.k01), ff_neg(a.k10), ff_neg(a.k11)}; }

__global__ void __launch_bounds__(256, 2) k_fan_elas(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ vptr,
                                                     const int2* __restrict__ fan, const int2* __restrict__ hdr,
                                                     const double2* __restrict__ q, int32_t nq, Consts cs,
                                                     double* __restrict__ out, int* __restrict__ err, Lim lim) {
    int bad = 0, orient = 0;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nq; r += (int64_t)gridDim.x * blockDim.x) {
        int32_t i = (int32_t)r;
        int2 h = hdr[i];
        int kind = h.y >> 28;
        if (kind > 1) continue;
        int32_t rb = row_ptr[i], u = row_ptr[i + 1] - rb, b0 = vptr[i], d = vptr[i + 1] - b0;
        int pself = h.y & 0x3FFF;
        const int2 rec0 = fan_rec(fan, b0, lim);
        const int2 last = kind == 1 ? make_int2(FE_IDX(h.x, lim.nq), (h.y >> 14) & 0x3FFF) : rec0;
        double2 pi = q[i];
        // neighbour data one triangle ahead of use, fan records two ahead (as in the scalar kernel)
        Raw rn = load_raw<0>(q, nullptr, rec0);
        Raw rp = load_raw<0>(q, nullptr, d > 1 ? fan_rec(fan, b0 + 1, lim) : last);
        int2 recn = d > 2 ? fan_rec(fan, b0 + 2, lim) : last;
        Nb cur = make_nb<0>(rn, pi, bad);
        const int first_pos = cur.pos;
        const ff z = ff_make(0.f);
        Block2 ndg = {z, z, z, z}, fs = ndg, ca = ndg;           // ndg: sum of the off-diagonal blocks
        for (int32_t e = 0; e < d; e++) {
            rn = rp;
            if (e + 2 <= d) {
                rp = load_raw<0>(q, nullptr, recn);
                recn = e + 3 < d ? fan_rec(fan, b0 + e + 3, lim) : last;
            }
            Nb nxt = make_nb<0>(rn, pi, bad);
            // the blocks of columns n_e and n_{e+1} (D and e_a from FP64 for badly shaped triangles)
            ff D = ff_dot2(cur.x, nxt.x, nxt.y, ff_neg(cur.y));
            ff eax = ff_sub(cur.x, nxt.x), eay = ff_sub(cur.y, nxt.y);
            if (!well_shaped(cur, nxt, D.h)) thin_terms(q, i, cur.id, nxt.id, D, eax, eay, nullptr, nullptr, bad);
            ff rr = ff_mulf(ff_rcp_fast(D), 0.5f);
            ff sax = ff_mul(eax, rr), say = ff_mul(eay, rr);
            Block2 kc = elas_block(sax, say, nxt.x, nxt.y, cs);
            Block2 kn = elas_block(sax, say, ff_neg(cur.x), ff_neg(cur.y), cs);
            orient |= !(D.h > 0.f);
            if (e == 0) {
                fs = kc;
            } else {
                Block2 v = badd(ca, kc);
                ndg = badd(ndg, v);
                write_block(out, rb, u, cur.pos, v, 4 * lim.nnz);
            }
            ca = kn;
            cur = nxt;
        }
        if (kind == 0) {
            Block2 v = badd(fs, ca);
            ndg = badd(ndg, v);
            write_block(out, rb, u, first_pos, v, 4 * lim.nnz);
        } else {
            ndg = badd(badd(ndg, fs), ca);
            write_block(out, rb, u, first_pos, fs, 4 * lim.nnz);
            write_block(out, rb, u, cur.pos, ca, 4 * lim.nnz);
        }
        write_block(out, rb, u, pself, bneg(ndg), 4 * lim.nnz);
    }
    if (bad) atomicOr(err, 2);
    if (orient) atomicOr(err, 1);
}

// General rows of K, one warp each (as k_general_scalar).
__global__ void __launch_bounds__(32 * GEN_WARPS) k_general_elas(const int32_t* __restrict__ gen, int32_t ngen,
                                                                 const int32_t* __restrict__ row_ptr,
                                                                 const int32_t* __restrict__ col_idx, const int32_t* __restrict__ vptr,
                                                                 const int2* __restrict__ fan, const double2* __restrict__ q, Consts cs,
                                                                 double* __restrict__ out, int* __restrict__ err) {
    const int32_t g = blockIdx.x * GEN_WARPS + (threadIdx.x >> 5);
    if (g >= ngen) return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int32_t i = gen[g];
    int32_t rb = row_ptr[i], u = row_ptr[i + 1] - rb;
    int32_t b0 = vptr[i], d = vptr[i + 1] - b0;
    double2 pi = q[i];
    int bad = 0, orient = 0;
    if (d <= GEN_SMEM_TRIS) {
        // as general_row: each triangle's three 2 x 2 blocks once, as double-floats (block b of
        // triangle e at sk[4 b + entry][e]); the diagonal block by the warp's tree, each
        // off-diagonal block from at most four terms by the same additions in every lane, more in
        // a loop; all sums in double-float, each entry converted to FP64 once
        __shared__ int2 sp_all[GEN_WARPS][GEN_SMEM_TRIS];
        __shared__ ff sk_all[GEN_WARPS][12][GEN_SMEM_TRIS];
        int2* sp = sp_all[wid];
        auto sk = sk_all[wid];
        ff a[4] = {z_ff(), z_ff(), z_ff(), z_ff()};
        for (int e = lane; e < d; e += 32) {
            int2 p = fan[b0 + e];
            sp[e] = p;
            Nb j = load_nb<0>(q, nullptr, pi, p.x, 0, bad), l = load_nb<0>(q, nullptr, pi, p.y, 0, bad);
            Block2 k[3];
            ff D = elas_terms(q, i, j, l, cs, k, bad);
            orient |= !(D.h > 0.f);
#pragma unroll
            for (int b = 0; b < 3; b++) {
                sk[4 * b][e] = k[b].k00;
                sk[4 * b + 1][e] = k[b].k01;
                sk[4 * b + 2][e] = k[b].k10;
                sk[4 * b + 3][e] = k[b].k11;
            }
            a[0] = ff_add(a[0], k[0].k00);
            a[1] = ff_add(a[1], k[0].k01);
            a[2] = ff_add(a[2], k[0].k10);
            a[3] = ff_add(a[3], k[0].k11);
        }
        ff dg[4];
#pragma unroll
        for (int x = 0; x < 4; x++) dg[x] = warp_sum_ff(a[x]);
        __syncwarp();
        for (int t = lane; t < u; t += 32) {
            int32_t col = col_idx[rb + t];
            ff v[4] = {z_ff(), z_ff(), z_ff(), z_ff()};
            if (col == i) {
#pragma unroll
                for (int x = 0; x < 4; x++) v[x] = dg[x];
            } else {
                int p0 = -1, p1 = -1, p2 = -1, p3 = -1, n = 0;
                for (int32_t e = 0; e < d; e++) {
                    int2 p = sp[e];
                    int which = p.x == col ? 1 : (p.y == col ? 2 : -1);
                    if (which < 0) continue;
                    int code = 3 * e + which;
                    p0 = n == 0 ? code : p0;
                    p1 = n == 1 ? code : p1;
                    p2 = n == 2 ? code : p2;
                    p3 = n == 3 ? code : p3;
                    n++;
                }
                if (n <= 4) {
                    auto term = [&](int code, int x) { return code < 0 ? z_ff() : sk[4 * (code % 3) + x][code / 3]; };
#pragma unroll
                    for (int x = 0; x < 4; x++) v[x] = ff_add(ff_add(ff_add(term(p0, x), term(p1, x)), term(p2, x)), term(p3, x));
                } else {
                    for (int32_t e = 0; e < d; e++) {
                        int2 p = sp[e];
                        int which = p.x == col ? 1 : (p.y == col ? 2 : -1);
                        if (which < 0) continue;
#pragma unroll
                        for (int x = 0; x < 4; x++) v[x] = ff_add(v[x], sk[4 * which + x][e]);
                    }
                }
            }
            int32_t o0 = 4 * rb + 2 * t, o1 = 4 * rb + 2 * u + 2 * t;
            out[o0] = ff_to_double(v[0]);
            out[o0 + 1] = ff_to_double(v[1]);
            out[o1] = ff_to_double(v[2]);
            out[o1 + 1] = ff_to_double(v[3]);
        }
        __syncwarp();
    } else {
        // a long row: each lane's columns, their contributions recomputed and added by
        // compensated FP64 sums
        for (int t = lane; t < u; t += 32) {
            int32_t col = col_idx[rb + t];
            bool self = col == i;
            double sx[4] = {0, 0, 0, 0}, c[4] = {0, 0, 0, 0};
            for (int32_t e = 0; e < d; e++) {
                int2 p = fan[b0 + e];
                int which = self ? 0 : (p.x == col ? 1 : (p.y == col ? 2 : -1));
                if (which < 0) continue;
                Nb j = load_nb<0>(q, nullptr, pi, p.x, 0, bad), l = load_nb<0>(q, nullptr, pi, p.y, 0, bad);
                Block2 k[3];
                ff D = elas_terms(q, i, j, l, cs, k, bad);
                orient |= !(D.h > 0.f);
                neumaier(sx[0], c[0], ff_to_double(k[which].k00));
                neumaier(sx[1], c[1], ff_to_double(k[which].k01));
                neumaier(sx[2], c[2], ff_to_double(k[which].k10));
                neumaier(sx[3], c[3], ff_to_double(k[which].k11));
            }
            int32_t o0 = 4 * rb + 2 * t, o1 = 4 * rb + 2 * u + 2 * t;
            out[o0] = sx[0] + c[0];
            out[o0 + 1] = sx[1] + c[1];
            out[o1] = sx[2] + c[2];
            out[o1 + 1] = sx[3] + c[3];
        }
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
    c.c120 = host_ff(1.0 / 120.0);
    c.l2m = host_ff(lam + 2.0 * mu);
    c.lam = host_ff(lam);
    c.mu = host_ff(mu);
    c.d60 = 1.0 / 60.0;
    c.d12 = 1.0 / 12.0;
    c.d24 = 1.0 / 24.0;
    return c;
}

static constexpr int FAN_BLOCK = 256;
static constexpr int FAN_SCALAR_BLOCK = 128;
static constexpr int GEN_BLOCK = 32 * GEN_WARPS;
static unsigned gen_grid(int32_t n) { return (unsigned)((n + GEN_WARPS - 1) / GEN_WARPS); }

template <int KIND>
static fe_status launch_scalar(fe_mesh m, fe_pattern p, const double* w, double* out0, double* out1, cudaStream_t s) {
    Consts cs = make_consts(0.0, 0.0);
    VRec* vr = nullptr;
    FeStreamScope scope(s);
    if (KIND & W_W) {
        fe_status st = fe_alloc_n(&vr, (size_t)m->nq, "vertex records");
        if (st) return st;
        { FE_PROF("k_pack_vrec", s); k_pack_vrec<<<fe_grid(m->nq, 256), 256, 0, s>>>(m->q, w, m->nq, vr, m->err); }
        cudaError_t e0 = cudaGetLastError();
        if (e0 != cudaSuccess) {
            fe_free(vr);
            return fe_cuda_fail(e0, "k_pack_vrec");
        }
    }
    // a row window (fe_pattern_build_part) assembles its rows only, into an output that holds
    // just them: the output pointers are shifted back by the window's first entry
    const bool win = p->row1 >= 0;
    const int32_t r0 = win ? p->row0 : 0, r1 = win ? p->row1 : m->nq;
    if (win) {
        out0 -= p->base_w;
        if (out1) out1 -= p->base_w;
    }
    if (r1 > r0) { FE_PROF("k_fan_scalar", s); k_fan_scalar<KIND><<<fe_grid(r1 - r0, FAN_SCALAR_BLOCK, FanOcc<KIND>::blocks), FAN_SCALAR_BLOCK, 0, s>>>(p->row_ptr, p->vptr, p->fan, p->hdr, m->q, vr, r0, r1, cs, out0, out1, m->err,
                                                                                                        Lim{m->nq, 3 * (int64_t)m->nme, win ? p->base_w + p->nnz : p->nnz_scalar}); }
    cudaError_t e = cudaGetLastError();
    fe_free(vr);
    if (e != cudaSuccess) return fe_cuda_fail(e, "k_fan_scalar");
    if (p->n_gen > 0) {
        { FE_PROF("k_general_scalar", s); k_general_scalar<KIND><<<gen_grid(p->n_gen), GEN_BLOCK, 0, s>>>(p->gen_rows, p->n_gen, p->row_ptr, p->col_idx, p->vptr, p->fan, m->q, w, cs, out0, out1, m->err, r0, r1); }
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
        case W_S | W_M: return launch_scalar<W_S | W_M>(m, p, w, out0, out1, s);
    }
    return fe_fail(FE_ERR_INVALID_ARG, "internal: bad row kind");
}

fe_status fe_row_elas(fe_mesh m, fe_pattern p, double lam, double mu, double* out, cudaStream_t s) {
    if (m->nq == 0 || p->nnz_scalar == 0) return FE_OK;
    Consts cs = make_consts(lam, mu);
    { FE_PROF("k_fan_elas", s); k_fan_elas<<<fe_grid(m->nq, FAN_BLOCK, 8), FAN_BLOCK, 0, s>>>(p->row_ptr, p->vptr, p->fan, p->hdr, m->q, m->nq, cs, out, m->err,
                                                                                           Lim{m->nq, 3 * (int64_t)m->nme, p->nnz_scalar}); }
    FE_LAUNCHED("k_fan_elas");
    if (p->n_gen > 0) {
        { FE_PROF("k_general_elas", s); k_general_elas<<<gen_grid(p->n_gen), GEN_BLOCK, 0, s>>>(p->gen_rows, p->n_gen, p->row_ptr, p->col_idx, p->vptr, p->fan, m->q, cs, out, m->err); }
        FE_LAUNCHED("k_general_elas");
    }
    return FE_OK;
}

int fe_row_batch_resident(int block) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_rows, block, 0);
    return per_sm > 0 ? per_sm : 1;
}

void fe_row_batch_launch(const fe_row_mesh* desc, const fe_row_tile* tiles, int32_t ntiles, const int2* general,
                         int32_t ngeneral, double* const* S, double* const* M, int block, cudaStream_t s) {
    Consts cs = make_consts(0.0, 0.0);
    if (ntiles > 0) {
        int64_t want = (int64_t)fe_sm_count() * fe_row_batch_resident(block);
        unsigned grid = (unsigned)(ntiles < want ? ntiles : want);
        { FE_PROF("k_batch_rows", s); k_batch_rows<<<grid, block, 0, s>>>(desc, tiles, ntiles, S, M, cs); }
    }
    if (ngeneral > 0) {
        { FE_PROF("k_batch_general", s); k_batch_general<<<gen_grid(ngeneral), GEN_BLOCK, 0, s>>>(desc, general, ngeneral, S, M, cs); }
    }
}

// ---------------------------------------------------------------- end-to-end call
//
// Host arrays in, host CSR arrays out, with the copies overlapped where the data allow it:
//   side stream:  w upload (while the mesh is uploaded and validated) | col_idx download | value
//                 downloads of row block k as soon as block k is assembled
//   main stream:  mesh upload + validation | pattern build | row_ptr download (its entries split
//                 the values into row blocks) | vertex records, general rows, row blocks 0..K-1
// The host link (about 0.2 TB/s each way) is the bound: the value downloads dominate.

namespace {
constexpr int E2E_BLOCKS = 8;

cudaStream_t side_stream() {
    static thread_local int dev = -1;
    static thread_local cudaStream_t st = nullptr;
    int d = 0;
    cudaGetDevice(&d);
    if (!st || d != dev) {
        st = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) st = nullptr;
        dev = d;
    }
    return st;
}

// The call's events, created once per thread and device (creating and destroying nine events per
// call put host-side driver work into every call).
cudaEvent_t* host_call_events() {
    static thread_local int dev = -1;
    static thread_local cudaEvent_t ev[E2E_BLOCKS + 1] = {};
    int d = 0;
    cudaGetDevice(&d);
    if (d != dev) {
        for (auto& e : ev) {
            e = nullptr;                                 // the previous device's events are kept
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
                dev = -1;
                return nullptr;
            }
        }
        dev = d;
    }
    return ev;
}
}  // namespace

extern "C" fe_status fe_assemble_stiff_wmass_host(int32_t nq, int32_t nme, const double* q, const int32_t* me,
                                                  const double* w, int32_t* row_ptr, int32_t* col_idx, double* S,
                                                  double* Mw, int64_t cap, int64_t* nnz_out, fe_stream stream) {
    FE_RANGE(__func__);
    if (!nnz_out || !row_ptr) return fe_fail(FE_ERR_INVALID_ARG, "row_ptr or nnz_out is null");
    *nnz_out = 0;
    if (nq < 0 || nme < 0) return fe_fail(FE_ERR_INVALID_ARG, "nq and nme must be >= 0");
    if (nq > 0 && (!q || !w)) return fe_fail(FE_ERR_INVALID_ARG, "q or w is null");
    cudaStream_t s = (cudaStream_t)stream;
    cudaStream_t s2 = side_stream();
    if (!s2) return fe_fail(FE_ERR_CUDA, "could not create the copy stream");
    FeStreamScope scope(s);
    if (nme > 0 && !me) return fe_fail(FE_ERR_INVALID_ARG, "me is null");
    if ((int64_t)nme * 9 >= INT32_MAX) return fe_fail(FE_ERR_LIMIT, "9*nme must be < 2^31");
    fe_mesh m = nullptr;
    fe_pattern p = nullptr;
    int32_t* med = nullptr;
    double *qd = nullptr, *wd = nullptr, *Sd = nullptr, *Md = nullptr;
    VRec* vr = nullptr;
    cudaEvent_t* ev = host_call_events();
    if (!ev) return fe_fail(FE_ERR_CUDA, "event creation");
    fe_status st = FE_OK;
    auto done = [&](fe_status ret) {
        cudaStreamSynchronize(s2);
        cudaStreamSynchronize(s);
        fe_free(vr);
        fe_free(Sd);
        fe_free(Md);
        fe_free(wd);
        fe_free(qd);
        fe_free(med);
        if (p) fe_pattern_destroy(p);
        if (m) fe_mesh_destroy(m);
        return ret;
    };
    // 1. the connectivity goes up first on the main stream; the coordinates and the weights follow
    //    on the side stream and arrive while the pattern is built (the pattern needs only me)
    if ((st = fe_alloc_n(&med, 3 * (size_t)nme, "mesh connectivity"))) return done(st);
    if ((st = fe_alloc_n(&qd, 2 * (size_t)nq, "coordinate staging"))) return done(st);
    if ((st = fe_alloc_n(&wd, (size_t)nq, "vertex weights"))) return done(st);
    if (nme > 0 && cudaMemcpyAsync(med, me, 3 * sizeof(int32_t) * nme, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return done(fe_fail(FE_ERR_CUDA, "connectivity upload"));
    cudaEventRecord(ev[0], s);                                   // allocations and the me upload come first
    cudaStreamWaitEvent(s2, ev[0]);
    if (nq > 0 && (cudaMemcpyAsync(qd, q, 2 * sizeof(double) * nq, cudaMemcpyHostToDevice, s2) != cudaSuccess ||
                   cudaMemcpyAsync(wd, w, sizeof(double) * nq, cudaMemcpyHostToDevice, s2) != cudaSuccess))
        return done(fe_fail(FE_ERR_CUDA, "coordinate or weight upload"));
    cudaEventRecord(ev[0], s2);                                  // q and w are up
    // 2. mesh (range, repeats, valences) and pattern, each synchronising the main stream; the mesh
    //    owns the connectivity from here on (also when it fails)
    st = fe_mesh_create_topology(nq, nme, med, s, &m);
    med = nullptr;
    if (st) return done(st);
    if ((st = fe_pattern_build(m, 1, FE_PATTERN_DEFAULT, stream, &p))) return done(st);
    // 3. the coordinates: packed, and every triangle's orientation checked
    cudaStreamWaitEvent(s, ev[0]);
    if ((st = fe_mesh_attach_coords(m, qd, s))) return done(st);
    const int64_t nnz = p->nnz;
    *nnz_out = nnz;
    int word[4] = {0, 0, 0, 0};
    auto read_word = [&]() -> fe_status {
        if (cudaMemcpyAsync(word, m->err, sizeof word, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return fe_fail(FE_ERR_CUDA, "validation word read-back");
        return fe_mesh_orientation_status(word);
    };
    if (cap < nnz) {                                             // mesh errors come before buffer errors
        if ((st = read_word())) return done(st);
        return done(fe_fail(FE_ERR_BUFFER_TOO_SMALL, "capacity " + std::to_string(cap) + " < nnz " + std::to_string(nnz)));
    }
    if (nnz > 0 && (!col_idx || !S || !Mw)) return done(fe_fail(FE_ERR_INVALID_ARG, "col_idx, S or Mw is null"));
    // 4. the column indices go down at once (the pattern is complete) while the coordinates are
    //    packed and checked and the values computed
    if (nnz > 0 && cudaMemcpyAsync(col_idx, p->col_idx, sizeof(int32_t) * nnz, cudaMemcpyDeviceToHost, s2) != cudaSuccess)
        return done(fe_fail(FE_ERR_CUDA, "col_idx download"));
    // 5. row_ptr (its entries split the value downloads into row blocks) with the orientation
    //    result; then the error word is cleared for the assembly's own flags
    if (cudaMemcpyAsync(row_ptr, p->row_ptr, sizeof(int32_t) * ((size_t)nq + 1), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return done(fe_fail(FE_ERR_CUDA, "row_ptr download"));
    if ((st = read_word())) return done(st);
    if (cudaMemsetAsync(m->err, 0, 4 * sizeof(int), s) != cudaSuccess) return done(fe_fail(FE_ERR_CUDA, "memset"));
    if (nnz == 0) return done(FE_OK);
    // 6. values: vertex records, general rows, then the row blocks, each downloaded when done
    if ((st = fe_alloc_n(&Sd, (size_t)nnz, "S values")) || (st = fe_alloc_n(&Md, (size_t)nnz, "Mw values")) ||
        (st = fe_alloc_n(&vr, (size_t)nq, "vertex records")))
        return done(st);
    cudaStreamWaitEvent(s, ev[0]);                               // w is on the device
    Consts cs = make_consts(0.0, 0.0);
    { FE_PROF("k_pack_vrec", s); k_pack_vrec<<<fe_grid(nq, 256), 256, 0, s>>>(m->q, wd, nq, vr, m->err); }
    if (p->n_gen > 0) {
        FE_PROF("k_general_scalar", s);
        k_general_scalar<W_S | W_W><<<gen_grid(p->n_gen), GEN_BLOCK, 0, s>>>(p->gen_rows, p->n_gen, p->row_ptr, p->col_idx, p->vptr, p->fan, m->q,
                                                                   wd, cs, Sd, Md, m->err, 0, nq);
    }
    for (int k = 0; k < E2E_BLOCKS; k++) {
        int32_t r0 = (int32_t)((int64_t)nq * k / E2E_BLOCKS), r1 = (int32_t)((int64_t)nq * (k + 1) / E2E_BLOCKS);
        if (r1 > r0) {
            FE_PROF("k_fan_scalar", s);
            k_fan_scalar<W_S | W_W><<<fe_grid(r1 - r0, FAN_SCALAR_BLOCK, FanOcc<W_S | W_W>::blocks), FAN_SCALAR_BLOCK, 0, s>>>(
                p->row_ptr, p->vptr, p->fan, p->hdr, m->q, vr, r0, r1, cs, Sd, Md, m->err, Lim{m->nq, 3 * (int64_t)m->nme, p->nnz_scalar});
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return done(fe_cuda_fail(e, "k_fan_scalar"));
        cudaEventRecord(ev[k + 1], s);
        cudaStreamWaitEvent(s2, ev[k + 1]);
        int64_t v0 = row_ptr[r0], v1 = row_ptr[r1];
        if (v1 > v0 && (cudaMemcpyAsync(S + v0, Sd + v0, sizeof(double) * (v1 - v0), cudaMemcpyDeviceToHost, s2) != cudaSuccess ||
                        cudaMemcpyAsync(Mw + v0, Md + v0, sizeof(double) * (v1 - v0), cudaMemcpyDeviceToHost, s2) != cudaSuccess))
            return done(fe_fail(FE_ERR_CUDA, "value download"));
    }
    if (cudaStreamSynchronize(s2) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
        return done(fe_fail(FE_ERR_CUDA, "end-to-end call"));
    return done(fe_mesh_check(m, stream));
}
