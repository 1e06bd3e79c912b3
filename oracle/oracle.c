/*
 * oracle.c -- plain, slow, FP64 CPU reference for P1 finite-element matrix assembly.
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark may call this library. It shares no code, header, table or helper with the CUDA
 * library; the two meet only through the seeded input arrays.
 *
 * What it computes (Cuvelier, Japhet, Scarella, "An efficient way to perform the assembly of
 * finite element matrices in Matlab and Octave", INRIA RR-8305, 2013):
 *   - element matrices straight from their closed forms: mass M^e (Eq. 1), weighted mass
 *     M^{e,[w]} (Eq. 2), stiffness S^e (Eq. 3), and the plane-elasticity K^e = |T| B^T C B
 *     with the basis-function gradients of Eq. (4) (Section 7);
 *   - the triplet arrays Ig, Jg, Kg in the paper's order: element k's local matrix stored
 *     column-wise, contribution index c = n^2*k + n*jl + il for an n x n element matrix
 *     (Section 5, "Ke = E(:)"; Section 7.1 for n = 6);
 *   - the sparse(I,J,K,m,n) semantics of Section 5: triplets with equal (row, col) are summed.
 *     Result in CSR, columns ascending in each row. Reading kept here: the pattern is
 *     structural, so a sum that happens to be exactly 0.0 is still stored; or_drop_zeros then
 *     gives Matlab's value-dependent result (no zero stored).
 *
 * Conventions: indices are 0-based (the paper is 1-based). q is [2][nq] row-major (x row,
 * then y row); me is [3][nme] row-major. The area |T| is not an input here: it is half the
 * signed cross product D = v_x*w_y - w_x*v_y of the edge vectors v = q3-q1, w = q1-q2, taken
 * from coordinate differences; D <= 0 is rejected (counter-clockwise triangles only).
 * Elasticity dofs are interleaved: vertex i owns rows 2i (x) and 2i+1 (y).
 *
 * Summation: duplicates are summed left to right in ascending contribution index c, in
 * round-to-nearest FP64 with no fused multiply-add (the build passes -ffp-contract=off).
 *
 * The adjoint (dL/dq, dL/dw for L = sum_p G[p]*A.values[p]) is not in the paper; it is the
 * derivative of the element formulas above, written out term by term in or_adjoint().
 * The extensions the paper announces without formulas (P1 tetrahedra, 3-D elasticity on them,
 * P2 and P3 triangles) follow in their own sections below, each from the definitions it states.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { OR_MASS = 0, OR_WMASS = 1, OR_STIFF = 2, OR_ELAS = 3 };
enum { OR_OK = 0, OR_ERR_ARG = 1, OR_ERR_INDEX = 2, OR_ERR_DEGENERATE = 3, OR_ERR_ORIENT = 4,
       OR_ERR_NOMEM = 5, OR_ERR_CAP = 6 };

/* ---------------------------------------------------------------- element matrices ---- */

/* Twice the signed area from the edge vectors v = p2 - p0 and w = p0 - p1 (0-based names of
 * the paper's q^3 - q^1 and q^1 - q^2). */
double or_double_area(const double x[3], const double y[3]) {
    double vx = x[2] - x[0], vy = y[2] - y[0];
    double wx = x[0] - x[1], wy = y[0] - y[1];
    return vx * wy - wx * vy;
}

/* Eq. (1): M^e = |T|/12 * [[2,1,1],[1,2,1],[1,1,2]].  E is row-major E[3*a+b]. */
void or_elem_mass(double area, double E[9]) {
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++)
            E[3 * a + b] = (area / 12.0) * (a == b ? 2.0 : 1.0);
}

/* Eq. (2), entry by entry as printed: |T|/30 times
 *   [3w1+w2+w3,    w1+w2+w3/2,  w1+w2/2+w3 ]
 *   [w1+w2+w3/2,   w1+3w2+w3,   w1/2+w2+w3 ]
 *   [w1+w2/2+w3,   w1/2+w2+w3,  w1+w2+3w3  ]                                             */
void or_elem_wmass(double area, const double w[3], double E[9]) {
    double c = area / 30.0;
    E[0] = c * (3.0 * w[0] + w[1] + w[2]);
    E[1] = c * (w[0] + w[1] + w[2] / 2.0);
    E[2] = c * (w[0] + w[1] / 2.0 + w[2]);
    E[3] = c * (w[0] + w[1] + w[2] / 2.0);
    E[4] = c * (w[0] + 3.0 * w[1] + w[2]);
    E[5] = c * (w[0] / 2.0 + w[1] + w[2]);
    E[6] = c * (w[0] + w[1] / 2.0 + w[2]);
    E[7] = c * (w[0] / 2.0 + w[1] + w[2]);
    E[8] = c * (w[0] + w[1] + 3.0 * w[2]);
}

/* The three edge vectors of Eq. (3): u = q2-q3, v = q3-q1, w = q1-q2 (0-based p1-p2, p2-p0,
 * p0-p1). ex[a], ey[a] are the components of the a-th of (u, v, w). */
static void edges(const double x[3], const double y[3], double ex[3], double ey[3]) {
    ex[0] = x[1] - x[2]; ey[0] = y[1] - y[2];
    ex[1] = x[2] - x[0]; ey[1] = y[2] - y[0];
    ex[2] = x[0] - x[1]; ey[2] = y[0] - y[1];
}

/* Eq. (3): S^e = 1/(4|T|) * Gram(u, v, w). */
void or_elem_stiff(const double x[3], const double y[3], double area, double E[9]) {
    double ex[3], ey[3];
    edges(x, y, ex, ey);
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++)
            E[3 * a + b] = (ex[a] * ex[b] + ey[a] * ey[b]) / (4.0 * area);
}

/* Section 7: K^e = |T| * B^T C B, 6x6 row-major. Gradients (Eq. 4):
 * grad(phi_a) = (e_a,y, -e_a,x) / (2|T|) with e = (u, v, w). Local dof 2a is the x-component
 * of vertex a, 2a+1 the y-component; B has column 2a = (dphi_a/dx, 0, dphi_a/dy) and column
 * 2a+1 = (0, dphi_a/dy, dphi_a/dx). C = [[l+2m, l, 0], [l, l+2m, 0], [0, 0, m]].            */
void or_elem_elas(const double x[3], const double y[3], double area, double lam, double mu,
                  double E[36]) {
    double ex[3], ey[3];
    edges(x, y, ex, ey);
    double B[3][6];
    memset(B, 0, sizeof B);
    for (int a = 0; a < 3; a++) {
        double gx = ey[a] / (2.0 * area);
        double gy = -ex[a] / (2.0 * area);
        B[0][2 * a] = gx;  B[2][2 * a] = gy;
        B[1][2 * a + 1] = gy;  B[2][2 * a + 1] = gx;
    }
    double C[3][3] = {{lam + 2.0 * mu, lam, 0.0}, {lam, lam + 2.0 * mu, 0.0}, {0.0, 0.0, mu}};
    double CB[3][6];
    for (int r = 0; r < 3; r++)
        for (int j = 0; j < 6; j++) {
            double s = 0.0;
            for (int t = 0; t < 3; t++) s += C[r][t] * B[t][j];
            CB[r][j] = s;
        }
    for (int i = 0; i < 6; i++)
        for (int j = 0; j < 6; j++) {
            double s = 0.0;
            for (int t = 0; t < 3; t++) s += B[t][i] * CB[t][j];
            E[6 * i + j] = area * s;
        }
}

/* ------------------------------------------------------------------------ triplets ---- */

static int gather_element(int64_t nq, const double* q, int64_t nme, const int32_t* me, int64_t k,
                          int32_t v[3], double x[3], double y[3]) {
    for (int a = 0; a < 3; a++) {
        v[a] = me[a * nme + k];
        if (v[a] < 0 || v[a] >= nq) return OR_ERR_INDEX;
        x[a] = q[v[a]];
        y[a] = q[nq + v[a]];
    }
    if (v[0] == v[1] || v[1] == v[2] || v[0] == v[2]) return OR_ERR_DEGENERATE;
    return OR_OK;
}

/* The arrays Ig, Jg, Kg of Sections 4-6 for one matrix kind, 0-based. Element k writes
 * entries c = n*n*k + n*jl + il (its matrix column-wise), n = 3 (or 6 for OR_ELAS).
 * w: vertex values (OR_WMASS only). On error, *bad_element receives the element index. */
int or_triplets(int kind, int64_t nq, int64_t nme, const double* q, const int32_t* me,
                const double* w, double lam, double mu, int32_t* I, int32_t* J, double* K,
                int64_t* bad_element) {
    if (kind < OR_MASS || kind > OR_ELAS || nq < 0 || nme < 0) return OR_ERR_ARG;
    int n = (kind == OR_ELAS) ? 6 : 3;
    for (int64_t k = 0; k < nme; k++) {
        int32_t v[3];
        double x[3], y[3], E[36];
        int st = gather_element(nq, q, nme, me, k, v, x, y);
        if (st) { if (bad_element) *bad_element = k; return st; }
        double D = or_double_area(x, y);
        if (!(D > 0.0)) { if (bad_element) *bad_element = k; return OR_ERR_ORIENT; }
        double area = D / 2.0;
        if (kind == OR_MASS) {
            or_elem_mass(area, E);
        } else if (kind == OR_WMASS) {
            double wl[3] = {w[v[0]], w[v[1]], w[v[2]]};
            or_elem_wmass(area, wl, E);
        } else if (kind == OR_STIFF) {
            or_elem_stiff(x, y, area, E);
        } else {
            or_elem_elas(x, y, area, lam, mu, E);
        }
        for (int jl = 0; jl < n; jl++)
            for (int il = 0; il < n; il++) {
                int64_t c = (int64_t)n * n * k + (int64_t)n * jl + il;
                int32_t gi, gj;
                if (n == 3) { gi = v[il]; gj = v[jl]; }
                else { gi = 2 * v[il / 2] + (il % 2); gj = 2 * v[jl / 2] + (jl % 2); }
                I[c] = gi;
                J[c] = gj;
                K[c] = E[n * il + jl];
            }
    }
    return OR_OK;
}

/* -------------------------------------------------------------- sparse(I, J, K) ---- */

static const int32_t* g_I;
static const int32_t* g_J;

static int key_less(int64_t a, int64_t b) {
    if (g_I[a] != g_I[b]) return g_I[a] < g_I[b];
    return g_J[a] < g_J[b];
}

/* Stable bottom-up merge sort of the permutation idx by (I, J): equal keys keep their input
 * order, so every run of duplicates stays in ascending contribution index. */
static int stable_sort_by_key(int64_t n, int64_t* idx) {
    int64_t* tmp = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    if (!tmp) return OR_ERR_NOMEM;
    int64_t* src = idx;
    int64_t* dst = tmp;
    for (int64_t width = 1; width < n; width *= 2) {
        for (int64_t lo = 0; lo < n; lo += 2 * width) {
            int64_t mid = lo + width < n ? lo + width : n;
            int64_t hi = lo + 2 * width < n ? lo + 2 * width : n;
            int64_t i = lo, j = mid, o = lo;
            while (i < mid && j < hi) {
                if (key_less(src[j], src[i])) dst[o++] = src[j++];
                else dst[o++] = src[i++];
            }
            while (i < mid) dst[o++] = src[i++];
            while (j < hi) dst[o++] = src[j++];
        }
        int64_t* t = src; src = dst; dst = t;
    }
    if (src != idx) memcpy(idx, src, (size_t)n * sizeof(int64_t));
    free(tmp);
    return OR_OK;
}

/* sparse(I, J, K, n_rows, n_cols) into CSR: row_ptr[n_rows+1], col_idx[cap], val[cap].
 * Duplicates are summed in ascending input position; exact zeros are kept. */
int or_sparse(int64_t n_rows, int64_t n_cols, int64_t ntrip, const int32_t* I, const int32_t* J,
              const double* K, int32_t* row_ptr, int32_t* col_idx, double* val, int64_t cap,
              int64_t* nnz_out) {
    for (int64_t t = 0; t < ntrip; t++)
        if (I[t] < 0 || I[t] >= n_rows || J[t] < 0 || J[t] >= n_cols) return OR_ERR_INDEX;
    int64_t* idx = (int64_t*)malloc((size_t)(ntrip > 0 ? ntrip : 1) * sizeof(int64_t));
    if (!idx) return OR_ERR_NOMEM;
    for (int64_t t = 0; t < ntrip; t++) idx[t] = t;
    g_I = I;
    g_J = J;
    int st = stable_sort_by_key(ntrip, idx);
    if (st) { free(idx); return st; }
    for (int64_t r = 0; r <= n_rows; r++) row_ptr[r] = 0;
    int64_t nnz = 0;
    for (int64_t s = 0; s < ntrip; ) {
        int64_t e = s + 1;
        double sum = K[idx[s]];
        while (e < ntrip && I[idx[e]] == I[idx[s]] && J[idx[e]] == J[idx[s]]) {
            sum += K[idx[e]];
            e++;
        }
        if (nnz >= cap) { free(idx); return OR_ERR_CAP; }
        col_idx[nnz] = J[idx[s]];
        val[nnz] = sum;
        row_ptr[I[idx[s]] + 1]++;
        nnz++;
        s = e;
    }
    for (int64_t r = 0; r < n_rows; r++) row_ptr[r + 1] += row_ptr[r];
    *nnz_out = nnz;
    free(idx);
    return OR_OK;
}

/* Matlab's sparse() stores no zero: an entry of K that is zero adds nothing, and a position whose
 * sum is zero is not stored (Section 5). or_sparse keeps those positions (the structural
 * reading); this removes every entry that compares equal to 0.0 (+0 and -0) from a CSR matrix,
 * keeping the others in order (NaN compares unequal to 0 and stays). The outputs may not alias
 * the inputs; col_idx_out and val_out need room for row_ptr[n_rows] entries. Returns the number
 * of entries kept. */
int64_t or_drop_zeros(int64_t n_rows, const int32_t* row_ptr, const int32_t* col_idx, const double* val,
                      int32_t* row_ptr_out, int32_t* col_idx_out, double* val_out) {
    int64_t n = 0;
    row_ptr_out[0] = 0;
    for (int64_t i = 0; i < n_rows; i++) {
        for (int64_t s = row_ptr[i]; s < row_ptr[i + 1]; s++) {
            if (val[s] != 0.0) {
                col_idx_out[n] = col_idx[s];
                val_out[n] = val[s];
                n++;
            }
        }
        row_ptr_out[i + 1] = (int32_t)n;
    }
    return n;
}

/* One full assembly: triplets of one kind, then sparse(). n_rows = nq (or 2nq for OR_ELAS).
 * The caller provides row_ptr[n_rows+1] and col_idx/val with capacity cap (9*nme, or 36*nme,
 * always suffices). */
int or_assemble(int kind, int64_t nq, int64_t nme, const double* q, const int32_t* me,
                const double* w, double lam, double mu, int32_t* row_ptr, int32_t* col_idx,
                double* val, int64_t cap, int64_t* nnz_out, int64_t* bad_element) {
    int n = (kind == OR_ELAS) ? 6 : 3;
    int64_t ntrip = (int64_t)n * n * nme;
    int32_t* I = (int32_t*)malloc((size_t)(ntrip > 0 ? ntrip : 1) * sizeof(int32_t));
    int32_t* J = (int32_t*)malloc((size_t)(ntrip > 0 ? ntrip : 1) * sizeof(int32_t));
    double* K = (double*)malloc((size_t)(ntrip > 0 ? ntrip : 1) * sizeof(double));
    int st = (I && J && K) ? OR_OK : OR_ERR_NOMEM;
    if (!st) st = or_triplets(kind, nq, nme, q, me, w, lam, mu, I, J, K, bad_element);
    if (!st) st = or_sparse(n == 6 ? 2 * nq : nq, n == 6 ? 2 * nq : nq, ntrip, I, J, K,
                            row_ptr, col_idx, val, cap, nnz_out);
    free(I); free(J); free(K);
    return st;
}

/* ------------------------------------------------------------------------- adjoint ---- */

/* Position of column j in CSR row i (binary search over the ascending columns), -1 if absent. */
static int64_t csr_find(const int32_t* row_ptr, const int32_t* col_idx, int32_t i, int32_t j) {
    int64_t lo = row_ptr[i], hi = row_ptr[i + 1];
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (col_idx[mid] < j) lo = mid + 1;
        else hi = mid;
    }
    return (lo < row_ptr[i + 1] && col_idx[lo] == j) ? lo : -1;
}

/* Accumulates into dq ([2][nq]) and, for OR_WMASS, dw ([nq]) the gradient of
 *   L = sum_p G[p] * A.values[p]
 * where A is the scalar matrix of the given kind (OR_MASS, OR_WMASS or OR_STIFF) on the CSR
 * pattern (row_ptr, col_idx). The caller zeroes dq and dw. Per element, with A = |T| = D/2,
 * g_ab = G at the position of (me[a], me[b]) and e = (u, v, w) as in Eq. (3):
 *   dA/dp_a = (e_a,y, -e_a,x) / 2                          (derivative of D/2)
 *   mass:     dL/dA = sum_ab g_ab * M_ab / A               (M^e is linear in A)
 *   wmass:    dL/dA = sum_ab g_ab * Mw_ab / A,  dL/dw_c = sum_ab g_ab * dMw_ab/dw_c
 *   stiff:    dL/de_a = sum_b (g_ab + g_ba) e_b / (4A),  dL/dA = -sum_ab g_ab * S_ab / A
 * and, since e_0 = p1-p2, e_1 = p2-p0, e_2 = p0-p1,
 *   dL/dp_0 = dL/de_2 - dL/de_1,  dL/dp_1 = dL/de_0 - dL/de_2,  dL/dp_2 = dL/de_1 - dL/de_0,
 * plus dL/dA * dA/dp_a. Vertex sums run in element order. */
int or_adjoint(int kind, int64_t nq, int64_t nme, const double* q, const int32_t* me,
               const double* w, const int32_t* row_ptr, const int32_t* col_idx, const double* G,
               double* dq, double* dw) {
    if (kind != OR_MASS && kind != OR_WMASS && kind != OR_STIFF) return OR_ERR_ARG;
    for (int64_t k = 0; k < nme; k++) {
        int32_t v[3];
        double x[3], y[3], E[9], g[9];
        int st = gather_element(nq, q, nme, me, k, v, x, y);
        if (st) return st;
        double D = or_double_area(x, y);
        if (!(D > 0.0)) return OR_ERR_ORIENT;
        double area = D / 2.0;
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) {
                int64_t p = csr_find(row_ptr, col_idx, v[a], v[b]);
                if (p < 0) return OR_ERR_INDEX;
                g[3 * a + b] = G[p];
            }
        double ex[3], ey[3];
        edges(x, y, ex, ey);
        double dex[3] = {0, 0, 0}, dey[3] = {0, 0, 0};
        double dA = 0.0;
        if (kind == OR_MASS) {
            or_elem_mass(area, E);
            for (int t = 0; t < 9; t++) dA += g[t] * E[t] / area;
        } else if (kind == OR_WMASS) {
            double wl[3] = {w[v[0]], w[v[1]], w[v[2]]};
            or_elem_wmass(area, wl, E);
            for (int t = 0; t < 9; t++) dA += g[t] * E[t] / area;
            /* dMw/dw_c: Eq. (2) with w replaced by the c-th unit vector. */
            for (int c = 0; c < 3; c++) {
                double unit[3] = {0, 0, 0}, Ec[9];
                unit[c] = 1.0;
                or_elem_wmass(area, unit, Ec);
                double s = 0.0;
                for (int t = 0; t < 9; t++) s += g[t] * Ec[t];
                dw[v[c]] += s;
            }
        } else {
            or_elem_stiff(x, y, area, E);
            for (int t = 0; t < 9; t++) dA -= g[t] * E[t] / area;
            for (int a = 0; a < 3; a++)
                for (int b = 0; b < 3; b++) {
                    double gs = (g[3 * a + b] + g[3 * b + a]) / (4.0 * area);
                    dex[a] += gs * ex[b];
                    dey[a] += gs * ey[b];
                }
        }
        double dpx[3], dpy[3];
        dpx[0] = dex[2] - dex[1]; dpy[0] = dey[2] - dey[1];
        dpx[1] = dex[0] - dex[2]; dpy[1] = dey[0] - dey[2];
        dpx[2] = dex[1] - dex[0]; dpy[2] = dey[1] - dey[0];
        for (int a = 0; a < 3; a++) {
            dpx[a] += dA * (ey[a] / 2.0);
            dpy[a] += dA * (-ex[a] / 2.0);
            dq[v[a]] += dpx[a];
            dq[nq + v[a]] += dpy[a];
        }
    }
    return OR_OK;
}

/* --------------------------------------------------------- tetrahedra (3-D P1) ---- */

/* The paper states that the method extends to three dimensions and gives no formulas (its
 * conclusion); these are the P1 element matrices on a tetrahedron K with vertices p0..p3,
 * written from the standard integrals:
 *   phi_a affine, phi_a(p_b) = delta_ab; grad(phi_1), grad(phi_2), grad(phi_3) are the rows of
 *   J^{-1} with J = [p1-p0 | p2-p0 | p3-p0] (columns), and grad(phi_0) = -(their sum);
 *   integral over K of phi_0^a0 phi_1^a1 phi_2^a2 phi_3^a3 = 6|K| a0! a1! a2! a3! / (a0+a1+a2+a3+3)!
 * so that
 *   mass            M^e_ab   = |K|/20 (1 + delta_ab)
 *   weighted mass   M^{e,[w]}_ab = |K|/120 sum_c kappa_abc w_c, kappa = 6 if a = b = c, 2 if exactly
 *                   two of a, b, c are equal, 1 if all three differ (w_h = sum_c w_c phi_c)
 *   stiffness       S^e_ab   = |K| grad(phi_a) . grad(phi_b)
 * q is [3][nq] (x, y, z rows), me is [4][nme]; element k writes c = 16k + 4*jl + il. The signed
 * volume 6|K| = det J must be > 0. */

/* det [p1-p0 | p2-p0 | p3-p0] = 6 |K| (signed) */
double or_tet_volume6(const double x[4], const double y[4], const double z[4]) {
    double ax = x[1] - x[0], ay = y[1] - y[0], az = z[1] - z[0];
    double bx = x[2] - x[0], by = y[2] - y[0], bz = z[2] - z[0];
    double cx = x[3] - x[0], cy = y[3] - y[0], cz = z[3] - z[0];
    return ax * (by * cz - bz * cy) - bx * (ay * cz - az * cy) + cx * (ay * bz - az * by);
}

void or_tet_elem_mass(double vol, double E[16]) {
    for (int a = 0; a < 4; a++)
        for (int b = 0; b < 4; b++)
            E[4 * a + b] = (vol / 20.0) * (a == b ? 2.0 : 1.0);
}

void or_tet_elem_wmass(double vol, const double w[4], double E[16]) {
    for (int a = 0; a < 4; a++)
        for (int b = 0; b < 4; b++) {
            double s = 0.0;
            for (int c = 0; c < 4; c++) {
                int eq = (a == b) + (a == c) + (b == c);     /* 3: all equal, 1: one pair, 0: distinct */
                double kappa = eq == 3 ? 6.0 : (eq == 1 ? 2.0 : 1.0);
                s += kappa * w[c];
            }
            E[4 * a + b] = (vol / 120.0) * s;
        }
}

/* grad(phi_a), a = 0..3, as g[a][0..2] */
static void tet_gradients(const double x[4], const double y[4], const double z[4], double g[4][3]) {
    double J[3][3] = {{x[1] - x[0], x[2] - x[0], x[3] - x[0]},
                      {y[1] - y[0], y[2] - y[0], y[3] - y[0]},
                      {z[1] - z[0], z[2] - z[0], z[3] - z[0]}};
    double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1])
               - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0])
               + J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    /* J^{-1} = adj(J) / det; row r of J^{-1} is grad(phi_{r+1}) */
    double inv[3][3];
    inv[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
    inv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
    inv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
    inv[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
    inv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
    inv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
    inv[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
    inv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
    inv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
    for (int d = 0; d < 3; d++) {
        g[1][d] = inv[0][d];
        g[2][d] = inv[1][d];
        g[3][d] = inv[2][d];
        g[0][d] = -(inv[0][d] + inv[1][d] + inv[2][d]);
    }
}

void or_tet_elem_stiff(const double x[4], const double y[4], const double z[4], double vol, double E[16]) {
    double g[4][3];
    tet_gradients(x, y, z, g);
    for (int a = 0; a < 4; a++)
        for (int b = 0; b < 4; b++)
            E[4 * a + b] = vol * (g[a][0] * g[b][0] + g[a][1] * g[b][1] + g[a][2] * g[b][2]);
}

/* Ig, Jg, Kg of a tetrahedral mesh for OR_MASS, OR_WMASS or OR_STIFF (c = 16k + 4*jl + il). */
int or_tet_triplets(int kind, int64_t nq, int64_t nme, const double* q, const int32_t* me,
                    const double* w, int32_t* I, int32_t* J, double* K, int64_t* bad_element) {
    if (kind < OR_MASS || kind > OR_STIFF || nq < 0 || nme < 0) return OR_ERR_ARG;
    for (int64_t k = 0; k < nme; k++) {
        int32_t v[4];
        double x[4], y[4], z[4], E[16];
        for (int a = 0; a < 4; a++) {
            v[a] = me[a * nme + k];
            if (v[a] < 0 || v[a] >= nq) { if (bad_element) *bad_element = k; return OR_ERR_INDEX; }
            x[a] = q[v[a]];
            y[a] = q[nq + v[a]];
            z[a] = q[2 * nq + v[a]];
        }
        for (int a = 0; a < 4; a++)
            for (int b = a + 1; b < 4; b++)
                if (v[a] == v[b]) { if (bad_element) *bad_element = k; return OR_ERR_DEGENERATE; }
        double D = or_tet_volume6(x, y, z);
        if (!(D > 0.0)) { if (bad_element) *bad_element = k; return OR_ERR_ORIENT; }
        double vol = D / 6.0;
        if (kind == OR_MASS) {
            or_tet_elem_mass(vol, E);
        } else if (kind == OR_WMASS) {
            double wl[4] = {w[v[0]], w[v[1]], w[v[2]], w[v[3]]};
            or_tet_elem_wmass(vol, wl, E);
        } else {
            or_tet_elem_stiff(x, y, z, vol, E);
        }
        for (int jl = 0; jl < 4; jl++)
            for (int il = 0; il < 4; il++) {
                int64_t c = 16 * k + 4 * jl + il;
                I[c] = v[il];
                J[c] = v[jl];
                K[c] = E[4 * il + jl];
            }
    }
    return OR_OK;
}

/* One full tetrahedral assembly: triplets, then sparse() (cap >= 16 nme always suffices). */
int or_tet_assemble(int kind, int64_t nq, int64_t nme, const double* q, const int32_t* me,
                    const double* w, int32_t* row_ptr, int32_t* col_idx, double* val, int64_t cap,
                    int64_t* nnz_out, int64_t* bad_element) {
    int64_t ntrip = 16 * nme;
    int32_t* I = (int32_t*)malloc((size_t)(ntrip > 0 ? ntrip : 1) * sizeof(int32_t));
    int32_t* J = (int32_t*)malloc((size_t)(ntrip > 0 ? ntrip : 1) * sizeof(int32_t));
    double* K = (double*)malloc((size_t)(ntrip > 0 ? ntrip : 1) * sizeof(double));
    int st = (I && J && K) ? OR_OK : OR_ERR_NOMEM;
    if (!st) st = or_tet_triplets(kind, nq, nme, q, me, w, I, J, K, bad_element);
    if (!st) st = or_sparse(nq, nq, ntrip, I, J, K, row_ptr, col_idx, val, cap, nnz_out);
    free(I); free(J); free(K);
    return st;
}

/* --------------------------------------- 3-D linear elasticity on tetrahedra (P1) ---- */

/* Section 7's construction carried to three dimensions (the paper announces the 3-D extension
 * without formulas): small strains, an isotropic material with constant Lame parameters lambda
 * and mu. Local dof 3a + d is component d (x, y, z) of vertex a. With g = grad(phi_a) (as for
 * the stiffness above), column 3a + d of the 6 x 12 strain matrix B maps that dof to the Voigt
 * strain vector (e_xx, e_yy, e_zz, 2 e_xy, 2 e_yz, 2 e_zx):
 *   column 3a     = (gx, 0,  0,  gy, 0,  gz)
 *   column 3a + 1 = (0,  gy, 0,  gx, gz, 0 )
 *   column 3a + 2 = (0,  0,  gz, 0,  gy, gx)
 * The material matrix is C = lambda (1,1,1,0,0,0)^T (1,1,1,0,0,0) + mu diag(2,2,2,1,1,1), and
 * K^e = |K| B^T C B (12 x 12, row-major E[12 i + j]). Global dofs are interleaved: vertex v owns
 * rows 3v, 3v + 1, 3v + 2. Element k writes c = 144k + 12 jl + il (column-wise, Ke = E(:)). */
void or_tet_elem_elas(const double x[4], const double y[4], const double z[4], double vol,
                      double lam, double mu, double E[144]) {
    double g[4][3];
    tet_gradients(x, y, z, g);
    double B[6][12];
    memset(B, 0, sizeof B);
    for (int a = 0; a < 4; a++) {
        double gx = g[a][0], gy = g[a][1], gz = g[a][2];
        B[0][3 * a] = gx;      B[3][3 * a] = gy;      B[5][3 * a] = gz;
        B[1][3 * a + 1] = gy;  B[3][3 * a + 1] = gx;  B[4][3 * a + 1] = gz;
        B[2][3 * a + 2] = gz;  B[4][3 * a + 2] = gy;  B[5][3 * a + 2] = gx;
    }
    double C[6][6];
    memset(C, 0, sizeof C);
    for (int r = 0; r < 3; r++)
        for (int t = 0; t < 3; t++) C[r][t] = lam + (r == t ? 2.0 * mu : 0.0);
    for (int r = 3; r < 6; r++) C[r][r] = mu;
    double CB[6][12];
    for (int r = 0; r < 6; r++)
        for (int j = 0; j < 12; j++) {
            double s = 0.0;
            for (int t = 0; t < 6; t++) s += C[r][t] * B[t][j];
            CB[r][j] = s;
        }
    for (int i = 0; i < 12; i++)
        for (int j = 0; j < 12; j++) {
            double s = 0.0;
            for (int t = 0; t < 6; t++) s += B[t][i] * CB[t][j];
            E[12 * i + j] = vol * s;
        }
}

/* Ig, Jg, Kg of the 3-D elasticity matrix (144 per tetrahedron, c = 144k + 12 jl + il). */
int or_tet_elas_triplets(int64_t nq, int64_t nme, const double* q, const int32_t* me, double lam,
                         double mu, int32_t* I, int32_t* J, double* K, int64_t* bad_element) {
    if (nq < 0 || nme < 0 || 3 * nq >= INT32_MAX) return OR_ERR_ARG;
    for (int64_t k = 0; k < nme; k++) {
        int32_t v[4];
        double x[4], y[4], z[4], E[144];
        for (int a = 0; a < 4; a++) {
            v[a] = me[a * nme + k];
            if (v[a] < 0 || v[a] >= nq) { if (bad_element) *bad_element = k; return OR_ERR_INDEX; }
            x[a] = q[v[a]];
            y[a] = q[nq + v[a]];
            z[a] = q[2 * nq + v[a]];
        }
        for (int a = 0; a < 4; a++)
            for (int b = a + 1; b < 4; b++)
                if (v[a] == v[b]) { if (bad_element) *bad_element = k; return OR_ERR_DEGENERATE; }
        double D = or_tet_volume6(x, y, z);
        if (!(D > 0.0)) { if (bad_element) *bad_element = k; return OR_ERR_ORIENT; }
        or_tet_elem_elas(x, y, z, D / 6.0, lam, mu, E);
        for (int jl = 0; jl < 12; jl++)
            for (int il = 0; il < 12; il++) {
                int64_t c = 144 * k + 12 * jl + il;
                I[c] = 3 * v[il / 3] + il % 3;
                J[c] = 3 * v[jl / 3] + jl % 3;
                K[c] = E[12 * il + jl];
            }
    }
    return OR_OK;
}

/* The 3-D elasticity matrix (3 nq rows): triplets, then sparse() (cap >= 144 nme suffices). */
int or_tet_elas_assemble(int64_t nq, int64_t nme, const double* q, const int32_t* me, double lam,
                         double mu, int32_t* row_ptr, int32_t* col_idx, double* val, int64_t cap,
                         int64_t* nnz_out, int64_t* bad_element) {
    int64_t ntrip = 144 * nme;
    int32_t* I = (int32_t*)malloc((size_t)(ntrip > 0 ? ntrip : 1) * sizeof(int32_t));
    int32_t* J = (int32_t*)malloc((size_t)(ntrip > 0 ? ntrip : 1) * sizeof(int32_t));
    double* K = (double*)malloc((size_t)(ntrip > 0 ? ntrip : 1) * sizeof(double));
    int st = (I && J && K) ? OR_OK : OR_ERR_NOMEM;
    if (!st) st = or_tet_elas_triplets(nq, nme, q, me, lam, mu, I, J, K, bad_element);
    if (!st) st = or_sparse(3 * nq, 3 * nq, ntrip, I, J, K, row_ptr, col_idx, val, cap, nnz_out);
    free(I); free(J); free(K);
    return st;
}

/* ----------------------------------------------- P2 triangles (quadratic, 6 dofs) ---- */

/* The paper states that the method extends to P_k elements and gives no formulas. These are the P2
 * (quadratic) matrices on a triangle T with vertices p0, p1, p2, written from the definitions:
 *   barycentric coordinates l0, l1, l2 (the P1 functions of Eq. (1)-(3); grad l_a as in Eq. (4));
 *   local dofs 0, 1, 2: the vertex functions phi_a = l_a (2 l_a - 1);
 *   local dofs 3, 4, 5: the edge functions 4 l0 l1, 4 l1 l2, 4 l2 l0 (midpoints of the edges
 *   (0,1), (1,2), (2,0));
 *   mass       M^e_ij = int_T phi_i phi_j
 *   stiffness  S^e_ij = int_T grad phi_i . grad phi_j, grad phi = sum_k (d phi / d l_k) grad l_k
 * with every polynomial in l0, l1, l2 integrated exactly:
 *   int_T l0^a l1^b l2^c = 2|T| a! b! c! / (a + b + c + 2)!.
 * Global dofs: vertex i is dof i; the edges follow, numbered in ascending order of their
 * (smaller vertex id, larger vertex id). Element k writes c = 36k + 6*jl + il (column-wise). */

#define P2_DEG 5      /* exponents 0..4 per barycentric coordinate */
typedef struct { double c[P2_DEG][P2_DEG][P2_DEG]; } p2_poly;

static void p2_zero(p2_poly* p) { memset(p, 0, sizeof *p); }

static void p2_mul(const p2_poly* a, const p2_poly* b, p2_poly* out) {
    p2_zero(out);
    for (int i = 0; i < P2_DEG; i++)
        for (int j = 0; j < P2_DEG - i; j++)
            for (int k = 0; k < P2_DEG - i - j; k++) {
                double x = a->c[i][j][k];
                if (x == 0.0) continue;
                for (int u = 0; u < P2_DEG - i; u++)
                    for (int v = 0; v < P2_DEG - j; v++)
                        for (int w = 0; w < P2_DEG - k; w++) {
                            double y = b->c[u][v][w];
                            if (y != 0.0 && i + u + j + v + k + w < P2_DEG) out->c[i + u][j + v][k + w] += x * y;
                        }
            }
}

/* d/d l_var */
static void p2_diff(const p2_poly* a, int var, p2_poly* out) {
    p2_zero(out);
    for (int i = 0; i < P2_DEG; i++)
        for (int j = 0; j < P2_DEG; j++)
            for (int k = 0; k < P2_DEG; k++) {
                double x = a->c[i][j][k];
                if (x == 0.0) continue;
                if (var == 0 && i > 0) out->c[i - 1][j][k] += i * x;
                if (var == 1 && j > 0) out->c[i][j - 1][k] += j * x;
                if (var == 2 && k > 0) out->c[i][j][k - 1] += k * x;
            }
}

static double p2_fact(int n) { double f = 1.0; for (int i = 2; i <= n; i++) f *= i; return f; }

static double p2_integrate(const p2_poly* a, double area) {
    double s = 0.0;
    for (int i = 0; i < P2_DEG; i++)
        for (int j = 0; j < P2_DEG; j++)
            for (int k = 0; k < P2_DEG; k++)
                if (a->c[i][j][k] != 0.0)
                    s += a->c[i][j][k] * 2.0 * area * p2_fact(i) * p2_fact(j) * p2_fact(k) / p2_fact(i + j + k + 2);
    return s;
}

/* the six basis functions as polynomials in (l0, l1, l2) */
static void p2_basis(p2_poly phi[6]) {
    for (int a = 0; a < 6; a++) p2_zero(&phi[a]);
    for (int a = 0; a < 3; a++) {
        int e[3] = {0, 0, 0};
        e[a] = 2;
        phi[a].c[e[0]][e[1]][e[2]] += 2.0;           /* 2 l_a^2 */
        e[a] = 1;
        phi[a].c[e[0]][e[1]][e[2]] -= 1.0;           /* - l_a */
    }
    phi[3].c[1][1][0] = 4.0;                          /* 4 l0 l1 */
    phi[4].c[0][1][1] = 4.0;                          /* 4 l1 l2 */
    phi[5].c[1][0][1] = 4.0;                          /* 4 l2 l0 */
}

void or_p2_elem_mass(double area, double E[36]) {
    p2_poly phi[6], prod;
    p2_basis(phi);
    for (int i = 0; i < 6; i++)
        for (int j = 0; j < 6; j++) {
            p2_mul(&phi[i], &phi[j], &prod);
            E[6 * i + j] = p2_integrate(&prod, area);
        }
}

void or_p2_elem_stiff(const double x[3], const double y[3], double area, double E[36]) {
    double ex[3], ey[3];
    edges(x, y, ex, ey);
    double g[3][2];                                   /* grad l_a = (e_a,y, -e_a,x) / (2|T|), Eq. (4) */
    for (int a = 0; a < 3; a++) {
        g[a][0] = ey[a] / (2.0 * area);
        g[a][1] = -ex[a] / (2.0 * area);
    }
    p2_poly phi[6], d[6][3], prod;
    p2_basis(phi);
    for (int i = 0; i < 6; i++)
        for (int k = 0; k < 3; k++) p2_diff(&phi[i], k, &d[i][k]);
    for (int i = 0; i < 6; i++)
        for (int j = 0; j < 6; j++) {
            double s = 0.0;
            for (int k = 0; k < 3; k++)
                for (int l = 0; l < 3; l++) {
                    p2_mul(&d[i][k], &d[j][l], &prod);
                    s += (g[k][0] * g[l][0] + g[k][1] * g[l][1]) * p2_integrate(&prod, area);
                }
            E[6 * i + j] = s;
        }
}

static int cmp_i64(const void* a, const void* b) {
    int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
    return x < y ? -1 : x > y;
}

/* Edge keys (smaller id << 32 | larger id) of a triangle mesh, sorted and unique; returns their
 * number (the caller frees *keys). */
int64_t or_p2_edges(int64_t nq, int64_t nme, const int32_t* me, int64_t** keys_out) {
    int64_t* keys = (int64_t*)malloc((size_t)(3 * nme > 0 ? 3 * nme : 1) * sizeof(int64_t));
    if (!keys) return -1;
    for (int64_t k = 0; k < nme; k++)
        for (int a = 0; a < 3; a++) {
            int64_t u = me[a * nme + k], v = me[((a + 1) % 3) * nme + k];
            int64_t lo = u < v ? u : v, hi = u < v ? v : u;
            keys[3 * k + a] = (lo << 32) | hi;
        }
    qsort(keys, (size_t)(3 * nme), sizeof(int64_t), cmp_i64);
    int64_t n = 0;
    for (int64_t t = 0; t < 3 * nme; t++)
        if (n == 0 || keys[t] != keys[n - 1]) keys[n++] = keys[t];
    (void)nq;
    *keys_out = keys;
    return n;
}

static int64_t p2_edge_id(const int64_t* keys, int64_t ne, int64_t u, int64_t v) {
    int64_t key = ((u < v ? u : v) << 32) | (u < v ? v : u);
    int64_t lo = 0, hi = ne - 1;
    while (lo < hi) {
        int64_t mid = (lo + hi) / 2;
        if (keys[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

/* Ig, Jg, Kg of the P2 matrices (OR_MASS or OR_STIFF) of a triangle mesh; *ndof = nq + edges. */
int or_p2_triplets(int kind, int64_t nq, int64_t nme, const double* q, const int32_t* me, int32_t* I, int32_t* J,
                   double* K, int64_t* ndof, int64_t* bad_element) {
    if ((kind != OR_MASS && kind != OR_STIFF) || nq < 0 || nme < 0) return OR_ERR_ARG;
    int64_t* keys = NULL;
    int64_t ne = or_p2_edges(nq, nme, me, &keys);
    if (ne < 0) return OR_ERR_NOMEM;
    *ndof = nq + ne;
    for (int64_t k = 0; k < nme; k++) {
        int32_t v[3];
        double x[3], y[3], E[36];
        int st = gather_element(nq, q, nme, me, k, v, x, y);
        if (st) { if (bad_element) *bad_element = k; free(keys); return st; }
        double D = or_double_area(x, y);
        if (!(D > 0.0)) { if (bad_element) *bad_element = k; free(keys); return OR_ERR_ORIENT; }
        double area = D / 2.0;
        if (kind == OR_MASS) or_p2_elem_mass(area, E);
        else or_p2_elem_stiff(x, y, area, E);
        int32_t dof[6] = {v[0], v[1], v[2], (int32_t)(nq + p2_edge_id(keys, ne, v[0], v[1])),
                          (int32_t)(nq + p2_edge_id(keys, ne, v[1], v[2])), (int32_t)(nq + p2_edge_id(keys, ne, v[2], v[0]))};
        for (int jl = 0; jl < 6; jl++)
            for (int il = 0; il < 6; il++) {
                int64_t c = 36 * k + 6 * jl + il;
                I[c] = dof[il];
                J[c] = dof[jl];
                K[c] = E[6 * il + jl];
            }
    }
    free(keys);
    return OR_OK;
}

/* One full P2 assembly: triplets, then sparse(). row_ptr needs nq + 3 nme + 1 entries (an upper
 * bound on ndof + 1); cap >= 36 nme always suffices. */
int or_p2_assemble(int kind, int64_t nq, int64_t nme, const double* q, const int32_t* me, int32_t* row_ptr,
                   int32_t* col_idx, double* val, int64_t cap, int64_t* nnz_out, int64_t* ndof_out,
                   int64_t* bad_element) {
    int64_t ntrip = 36 * nme;
    int32_t* I = (int32_t*)malloc((size_t)(ntrip > 0 ? ntrip : 1) * sizeof(int32_t));
    int32_t* J = (int32_t*)malloc((size_t)(ntrip > 0 ? ntrip : 1) * sizeof(int32_t));
    double* K = (double*)malloc((size_t)(ntrip > 0 ? ntrip : 1) * sizeof(double));
    int st = (I && J && K) ? OR_OK : OR_ERR_NOMEM;
    int64_t ndof = nq;
    if (!st) st = or_p2_triplets(kind, nq, nme, q, me, I, J, K, &ndof, bad_element);
    if (!st) st = or_sparse(ndof, ndof, ntrip, I, J, K, row_ptr, col_idx, val, cap, nnz_out);
    *ndof_out = ndof;
    free(I); free(J); free(K);
    return st;
}

/* ----------------------------------------------- P3 triangles (cubic, 10 dofs) ---- */

/* The paper states that the method extends to P_k elements and gives no formulas. These are the P3
 * (cubic) matrices on a triangle T with vertices p0, p1, p2, written from the definitions, as for
 * P2 above but with cubic Lagrange functions in the barycentric coordinates l0, l1, l2:
 *   local dofs 0, 1, 2: the vertices, phi_a = l_a (3 l_a - 1)(3 l_a - 2) / 2;
 *   local dofs 3..8: two per edge, for the edges (0,1), (1,2), (2,0) in turn: on edge (a, b) the
 *     node at 2/3 p_a + 1/3 p_b, phi = 9/2 l_a l_b (3 l_a - 1), then the node at 1/3 p_a + 2/3 p_b,
 *     phi = 9/2 l_a l_b (3 l_b - 1);
 *   local dof 9: the centroid, the bubble 27 l0 l1 l2;
 *   mass M^e_ij = int_T phi_i phi_j, stiffness S^e_ij = int_T grad phi_i . grad phi_j, every
 *   product integrated exactly with int_T l0^a l1^b l2^c = 2|T| a! b! c! / (a + b + c + 2)!.
 * Global dofs: vertex i is dof i; edge e (the edges numbered in ascending order of (smaller id,
 * larger id), as for P2) owns dofs nq + 2e (its node nearer the smaller vertex id) and nq + 2e + 1
 * (nearer the larger); element k's bubble is dof nq + 2 ne + k. Element k writes
 * c = 100k + 10*jl + il (column-wise). */

#define P3_DEG 7      /* exponents 0..6 per barycentric coordinate (products of two cubics) */
typedef struct { double c[P3_DEG][P3_DEG][P3_DEG]; } p3_poly;

static void p3_zero(p3_poly* p) { memset(p, 0, sizeof *p); }

static void p3_mul(const p3_poly* a, const p3_poly* b, p3_poly* out) {
    p3_zero(out);
    for (int i = 0; i < P3_DEG; i++)
        for (int j = 0; j < P3_DEG - i; j++)
            for (int k = 0; k < P3_DEG - i - j; k++) {
                double x = a->c[i][j][k];
                if (x == 0.0) continue;
                for (int u = 0; u < P3_DEG - i; u++)
                    for (int v = 0; v < P3_DEG - j; v++)
                        for (int w = 0; w < P3_DEG - k; w++) {
                            double y = b->c[u][v][w];
                            if (y != 0.0 && i + u + j + v + k + w < P3_DEG) out->c[i + u][j + v][k + w] += x * y;
                        }
            }
}

static void p3_diff(const p3_poly* a, int var, p3_poly* out) {
    p3_zero(out);
    for (int i = 0; i < P3_DEG; i++)
        for (int j = 0; j < P3_DEG; j++)
            for (int k = 0; k < P3_DEG; k++) {
                double x = a->c[i][j][k];
                if (x == 0.0) continue;
                if (var == 0 && i > 0) out->c[i - 1][j][k] += i * x;
                if (var == 1 && j > 0) out->c[i][j - 1][k] += j * x;
                if (var == 2 && k > 0) out->c[i][j][k - 1] += k * x;
            }
}

static double p3_fact(int n) { double f = 1.0; for (int i = 2; i <= n; i++) f *= i; return f; }

static double p3_integrate(const p3_poly* a, double area) {
    double s = 0.0;
    for (int i = 0; i < P3_DEG; i++)
        for (int j = 0; j < P3_DEG; j++)
            for (int k = 0; k < P3_DEG; k++)
                if (a->c[i][j][k] != 0.0)
                    s += a->c[i][j][k] * 2.0 * area * p3_fact(i) * p3_fact(j) * p3_fact(k) / p3_fact(i + j + k + 2);
    return s;
}

/* adds coef * l0^e0 l1^e1 l2^e2 to p */
static void p3_add(p3_poly* p, double coef, int e0, int e1, int e2) { p->c[e0][e1][e2] += coef; }

/* the ten basis functions as polynomials in (l0, l1, l2) */
static void p3_basis(p3_poly phi[10]) {
    for (int a = 0; a < 10; a++) p3_zero(&phi[a]);
    for (int a = 0; a < 3; a++) {                     /* l (3l - 1)(3l - 2)/2 = 9/2 l^3 - 9/2 l^2 + l */
        int e[3] = {0, 0, 0};
        e[a] = 3; p3_add(&phi[a], 4.5, e[0], e[1], e[2]);
        e[a] = 2; p3_add(&phi[a], -4.5, e[0], e[1], e[2]);
        e[a] = 1; p3_add(&phi[a], 1.0, e[0], e[1], e[2]);
    }
    const int ea[3] = {0, 1, 2}, eb[3] = {1, 2, 0};
    for (int t = 0; t < 3; t++) {
        for (int side = 0; side < 2; side++) {        /* 9/2 l_a l_b (3 l_n - 1), n = a then b */
            const int n = side == 0 ? ea[t] : eb[t];
            p3_poly* f = &phi[3 + 2 * t + side];
            int e[3] = {0, 0, 0};
            e[ea[t]] += 1; e[eb[t]] += 1; e[n] += 1;
            p3_add(f, 13.5, e[0], e[1], e[2]);
            e[n] -= 1;
            p3_add(f, -4.5, e[0], e[1], e[2]);
        }
    }
    p3_add(&phi[9], 27.0, 1, 1, 1);
}

void or_p3_elem_mass(double area, double E[100]) {
    p3_poly phi[10], prod;
    p3_basis(phi);
    for (int i = 0; i < 10; i++)
        for (int j = 0; j < 10; j++) {
            p3_mul(&phi[i], &phi[j], &prod);
            E[10 * i + j] = p3_integrate(&prod, area);
        }
}

void or_p3_elem_stiff(const double x[3], const double y[3], double area, double E[100]) {
    double ex[3], ey[3];
    edges(x, y, ex, ey);
    double g[3][2];                                   /* grad l_a = (e_a,y, -e_a,x) / (2|T|), Eq. (4) */
    for (int a = 0; a < 3; a++) {
        g[a][0] = ey[a] / (2.0 * area);
        g[a][1] = -ex[a] / (2.0 * area);
    }
    p3_poly phi[10], prod;
    p3_poly(*d)[3] = (p3_poly(*)[3])malloc(sizeof(p3_poly[10][3]));   /* 80 KB: off the stack */
    if (!d) { for (int t = 0; t < 100; t++) E[t] = 0.0; return; }
    p3_basis(phi);
    for (int i = 0; i < 10; i++)
        for (int k = 0; k < 3; k++) p3_diff(&phi[i], k, &d[i][k]);
    for (int i = 0; i < 10; i++)
        for (int j = 0; j < 10; j++) {
            double s = 0.0;
            for (int k = 0; k < 3; k++)
                for (int l = 0; l < 3; l++) {
                    p3_mul(&d[i][k], &d[j][l], &prod);
                    s += (g[k][0] * g[l][0] + g[k][1] * g[l][1]) * p3_integrate(&prod, area);
                }
            E[10 * i + j] = s;
        }
    free(d);
}

/* Ig, Jg, Kg of the P3 matrices (OR_MASS or OR_STIFF); *ndof = nq + 2 ne + nme. */
int or_p3_triplets(int kind, int64_t nq, int64_t nme, const double* q, const int32_t* me, int32_t* I, int32_t* J,
                   double* K, int64_t* ndof, int64_t* bad_element) {
    if ((kind != OR_MASS && kind != OR_STIFF) || nq < 0 || nme < 0) return OR_ERR_ARG;
    int64_t* keys = NULL;
    int64_t ne = or_p2_edges(nq, nme, me, &keys);
    if (ne < 0) return OR_ERR_NOMEM;
    *ndof = nq + 2 * ne + nme;
    for (int64_t k = 0; k < nme; k++) {
        int32_t v[3];
        double x[3], y[3], E[100];
        int st = gather_element(nq, q, nme, me, k, v, x, y);
        if (st) { if (bad_element) *bad_element = k; free(keys); return st; }
        double D = or_double_area(x, y);
        if (!(D > 0.0)) { if (bad_element) *bad_element = k; free(keys); return OR_ERR_ORIENT; }
        double area = D / 2.0;
        if (kind == OR_MASS) or_p3_elem_mass(area, E);
        else or_p3_elem_stiff(x, y, area, E);
        int32_t dof[10];
        for (int a = 0; a < 3; a++) dof[a] = v[a];
        for (int t = 0; t < 3; t++) {
            int32_t a = v[t], b = v[(t + 1) % 3];
            int64_t e = p2_edge_id(keys, ne, a, b);
            dof[3 + 2 * t] = (int32_t)(nq + 2 * e + (a < b ? 0 : 1));       /* the node nearer a */
            dof[4 + 2 * t] = (int32_t)(nq + 2 * e + (a < b ? 1 : 0));       /* the node nearer b */
        }
        dof[9] = (int32_t)(nq + 2 * ne + k);
        for (int jl = 0; jl < 10; jl++)
            for (int il = 0; il < 10; il++) {
                int64_t c = 100 * k + 10 * jl + il;
                I[c] = dof[il];
                J[c] = dof[jl];
                K[c] = E[10 * il + jl];
            }
    }
    free(keys);
    return OR_OK;
}

/* One full P3 assembly: triplets, then sparse(). row_ptr needs nq + 6 nme + nme + 1 entries (an
 * upper bound on ndof + 1); cap >= 100 nme always suffices. */
int or_p3_assemble(int kind, int64_t nq, int64_t nme, const double* q, const int32_t* me, int32_t* row_ptr,
                   int32_t* col_idx, double* val, int64_t cap, int64_t* nnz_out, int64_t* ndof_out,
                   int64_t* bad_element) {
    int64_t ntrip = 100 * nme;
    int32_t* I = (int32_t*)malloc((size_t)(ntrip > 0 ? ntrip : 1) * sizeof(int32_t));
    int32_t* J = (int32_t*)malloc((size_t)(ntrip > 0 ? ntrip : 1) * sizeof(int32_t));
    double* K = (double*)malloc((size_t)(ntrip > 0 ? ntrip : 1) * sizeof(double));
    int st = (I && J && K) ? OR_OK : OR_ERR_NOMEM;
    int64_t ndof = nq;
    if (!st) st = or_p3_triplets(kind, nq, nme, q, me, I, J, K, &ndof, bad_element);
    if (!st) st = or_sparse(ndof, ndof, ntrip, I, J, K, row_ptr, col_idx, val, cap, nnz_out);
    *ndof_out = ndof;
    free(I); free(J); free(K);
    return st;
}
