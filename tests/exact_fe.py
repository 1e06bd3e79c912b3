"""Exact rational P1 element matrices, derived independently of both implementations.

The oracle and the CUDA kernels use the paper's closed forms (Eqs. 1-3 and the B^T C B form
of Section 7, built from edge vectors). This helper starts from the definitions instead:
  - the barycentric coordinates lambda_a(x, y) = alpha_a + beta_a x + gamma_a y are found by
    solving lambda_a(p_b) = delta_ab with exact Gaussian elimination on Fractions;
  - integrals of products of barycentric coordinates use the exact monomial formula
        int_T l0^i l1^j l2^k = 2|T| i! j! k! / (i + j + k + 2)!;
  - the P1 weighted mass integrates w_h = sum_c w_c l_c against l_a l_b;
  - the plane-elasticity matrix integrates eps(phi_I)^T C eps(phi_J) with the strain vector
    (du_x/dx, du_y/dy, du_x/dy + du_y/dx) of each vector basis function.
So a dropped term, a sign error or a swapped index in the closed forms shows up as a mismatch.
"""
from __future__ import annotations

from fractions import Fraction
from math import factorial


def _solve3(A, rhs):
    """Exact solution of a 3x3 linear system (Gaussian elimination with pivot search)."""
    M = [list(A[r]) + [rhs[r]] for r in range(3)]
    for c in range(3):
        p = next(r for r in range(c, 3) if M[r][c] != 0)
        M[c], M[p] = M[p], M[c]
        for r in range(3):
            if r != c and M[r][c] != 0:
                f = M[r][c] / M[c][c]
                M[r] = [M[r][t] - f * M[c][t] for t in range(4)]
    return [M[r][3] / M[r][r] for r in range(3)]


def barycentric(pts):
    """[(alpha, beta, gamma)] of the three barycentric coordinates of triangle pts."""
    A = [[Fraction(1), Fraction(x), Fraction(y)] for (x, y) in pts]
    out = []
    for a in range(3):
        rhs = [Fraction(int(a == b)) for b in range(3)]
        out.append(tuple(_solve3(A, rhs)))
    return out


def area(pts):
    (x0, y0), (x1, y1), (x2, y2) = [(Fraction(x), Fraction(y)) for (x, y) in pts]
    return abs((x1 - x0) * (y2 - y0) - (x2 - x0) * (y1 - y0)) / 2


def mono(area_t, e):
    """int_T l0^e0 l1^e1 l2^e2."""
    return 2 * area_t * Fraction(factorial(e[0]) * factorial(e[1]) * factorial(e[2]),
                                 factorial(sum(e) + 2))


def mass(pts):
    A = area(pts)
    M = [[None] * 3 for _ in range(3)]
    for a in range(3):
        for b in range(3):
            e = [0, 0, 0]
            e[a] += 1
            e[b] += 1
            M[a][b] = mono(A, e)
    return M


def wmass(pts, w):
    A = area(pts)
    M = [[Fraction(0)] * 3 for _ in range(3)]
    for a in range(3):
        for b in range(3):
            for c in range(3):
                e = [0, 0, 0]
                e[a] += 1
                e[b] += 1
                e[c] += 1
                M[a][b] += Fraction(w[c]) * mono(A, e)
    return M


def stiff(pts):
    A = area(pts)
    g = barycentric(pts)
    return [[A * (g[a][1] * g[b][1] + g[a][2] * g[b][2]) for b in range(3)] for a in range(3)]


def elas(pts, lam, mu):
    """6x6, local dof 2a = x-displacement of vertex a, 2a+1 = y-displacement."""
    A = area(pts)
    g = barycentric(pts)
    lam, mu = Fraction(lam), Fraction(mu)
    C = [[lam + 2 * mu, lam, 0], [lam, lam + 2 * mu, 0], [0, 0, mu]]
    eps = []
    for a in range(3):
        dx, dy = g[a][1], g[a][2]
        eps.append((dx, Fraction(0), dy))      # u = (phi_a, 0)
        eps.append((Fraction(0), dy, dx))      # u = (0, phi_a)
    K = [[None] * 6 for _ in range(6)]
    for i in range(6):
        for j in range(6):
            s = Fraction(0)
            for r in range(3):
                for t in range(3):
                    s += eps[i][r] * C[r][t] * eps[j][t]
            K[i][j] = A * s
    return K


def assemble_dense(kind, pts_all, me, w=None, lam=1, mu=Fraction(1, 2)):
    """Exact dense global matrix by direct accumulation (no sorting), for tiny meshes.

    kind in {"mass", "wmass", "stiff", "elas"}; pts_all is a list of (x, y) per vertex;
    me is a list of (v0, v1, v2) per element.
    """
    nq = len(pts_all)
    n = 2 * nq if kind == "elas" else nq
    G = [[Fraction(0)] * n for _ in range(n)]
    for tri in me:
        pts = [pts_all[v] for v in tri]
        if kind == "mass":
            E = mass(pts)
        elif kind == "wmass":
            E = wmass(pts, [w[v] for v in tri])
        elif kind == "stiff":
            E = stiff(pts)
        else:
            E = elas(pts, lam, mu)
        m = 6 if kind == "elas" else 3
        dof = [2 * tri[i // 2] + i % 2 for i in range(6)] if kind == "elas" else list(tri)
        for i in range(m):
            for j in range(m):
                G[dof[i]][dof[j]] += E[i][j]
    return G


# ------------------------------------------------------------------ tetrahedra

def _solve(A, rhs):
    """Exact solution of an n x n linear system (Gaussian elimination with pivot search)."""
    n = len(A)
    M = [list(A[r]) + [rhs[r]] for r in range(n)]
    for c in range(n):
        p = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[p] = M[p], M[c]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c] / M[c][c]
                M[r] = [M[r][t] - f * M[c][t] for t in range(n + 1)]
    return [M[r][n] / M[r][r] for r in range(n)]


def barycentric3(pts):
    """[(alpha, beta_x, beta_y, beta_z)] of the four barycentric coordinates of tetrahedron pts."""
    A = [[Fraction(1), Fraction(x), Fraction(y), Fraction(z)] for (x, y, z) in pts]
    return [tuple(_solve(A, [Fraction(int(a == b)) for b in range(4)])) for a in range(4)]


def volume3(pts):
    """|K| from the barycentric gradients: the coordinate l_0 = 1 - l_1 - l_2 - l_3 has the
    constant gradient; |K| = 1 / (6 |det of the three gradients of l_1, l_2, l_3|)."""
    b = barycentric3(pts)
    G = [[b[a][1], b[a][2], b[a][3]] for a in (1, 2, 3)]
    det = (G[0][0] * (G[1][1] * G[2][2] - G[1][2] * G[2][1]) - G[0][1] * (G[1][0] * G[2][2] - G[1][2] * G[2][0])
           + G[0][2] * (G[1][0] * G[2][1] - G[1][1] * G[2][0]))
    return 1 / (6 * abs(det))


def mono3(vol, e):
    """int_K l0^e0 l1^e1 l2^e2 l3^e3 = 6|K| e0! e1! e2! e3! / (e0+e1+e2+e3+3)!"""
    num = 6 * vol
    for v in e:
        num *= factorial(v)
    return num / factorial(sum(e) + 3)


def tet_mass(pts):
    vol = volume3(pts)
    E = [[Fraction(0)] * 4 for _ in range(4)]
    for a in range(4):
        for b in range(4):
            e = [0] * 4
            e[a] += 1
            e[b] += 1
            E[a][b] = mono3(vol, e)
    return E


def tet_wmass(pts, w):
    vol = volume3(pts)
    E = [[Fraction(0)] * 4 for _ in range(4)]
    for a in range(4):
        for b in range(4):
            for c in range(4):
                e = [0] * 4
                e[a] += 1
                e[b] += 1
                e[c] += 1
                E[a][b] += Fraction(w[c]) * mono3(vol, e)
    return E


def tet_stiff(pts):
    vol = volume3(pts)
    g = [b[1:] for b in barycentric3(pts)]
    return [[vol * sum(g[a][d] * g[b][d] for d in range(3)) for b in range(4)] for a in range(4)]


def tet_elas(pts, lam, mu):
    """12 x 12 3-D elasticity matrix from the bilinear form
        a(u, v) = int_K lam div(u) div(v) + 2 mu eps(u) : eps(v),   eps(u) = (grad u + grad u^T) / 2,
    for the vector basis functions u = phi_a e_alpha (local dof 3a + alpha): grad u has the
    single row alpha equal to grad(phi_a). No strain vector or material matrix is formed."""
    vol = volume3(pts)
    g = [b[1:] for b in barycentric3(pts)]
    lam, mu = Fraction(lam), Fraction(mu)
    grads = []
    for a in range(4):
        for al in range(3):
            G = [[g[a][j] if i == al else Fraction(0) for j in range(3)] for i in range(3)]
            grads.append(G)
    eps = [[[(G[i][j] + G[j][i]) / 2 for j in range(3)] for i in range(3)] for G in grads]
    div = [G[0][0] + G[1][1] + G[2][2] for G in grads]
    return [[vol * (lam * div[I] * div[J] + 2 * mu * sum(eps[I][i][j] * eps[J][i][j] for i in range(3) for j in range(3)))
             for J in range(12)] for I in range(12)]


def tet_assemble_dense(kind, pts_all, me, w=None):
    """Dense global matrix of a tetrahedral mesh, exact (kind in mass, wmass, stiff)."""
    n = len(pts_all)
    G = [[Fraction(0)] * n for _ in range(n)]
    for t in me:
        pts = [pts_all[v] for v in t]
        if kind == "mass":
            E = tet_mass(pts)
        elif kind == "wmass":
            E = tet_wmass(pts, [w[v] for v in t])
        else:
            E = tet_stiff(pts)
        for a in range(4):
            for b in range(4):
                G[t[a]][t[b]] += E[a][b]
    return G
