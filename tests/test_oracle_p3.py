"""Pins of the oracle's P3 (cubic) triangle assembly, the P_k extension the paper announces without
formulas (k = 3). Element matrices are checked against an independent symbolic integration (sympy:
the ten basis functions built in x, y from their nodal values, integrated over the triangle) and a
closed form; the assembled matrices against what cubic functions, which the P3 space contains, fix
exactly on any triangulation of the unit square.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1305_3122_gb300 import meshgen


def _sym_p3(pts):
    """P3 mass and stiffness of the triangle pts (rationals), by sympy: the ten cubic polynomials in
    x, y with phi_i(node_j) = delta_ij (nodes: vertices; on the edges (0,1), (1,2), (2,0) the points
    at 1/3 and 2/3 from the first vertex; the centroid), integrated over the triangle."""
    sp = pytest.importorskip("sympy")
    x, y, s, t = sp.symbols("x y s t")
    P = [sp.Matrix([sp.Rational(px), sp.Rational(py)]) for px, py in pts]
    nodes = list(P)
    for a, b in ((0, 1), (1, 2), (2, 0)):
        nodes += [(2 * P[a] + P[b]) / 3, (P[a] + 2 * P[b]) / 3]
    nodes.append((P[0] + P[1] + P[2]) / 3)
    mono = [sp.Integer(1), x, y, x * x, x * y, y * y, x ** 3, x * x * y, x * y * y, y ** 3]
    V = sp.Matrix([[m.subs({x: n[0], y: n[1]}) for m in mono] for n in nodes])
    C = V.inv()
    phi = [sum(C[r, i] * mono[r] for r in range(10)) for i in range(10)]
    X = P[0] + s * (P[1] - P[0]) + t * (P[2] - P[0])
    jac = abs((P[1] - P[0]).row_join(P[2] - P[0]).det())

    def integ(f):
        g = sp.Poly(sp.expand(f.subs({x: X[0], y: X[1]}, simultaneous=True)), s, t)
        # int over the unit triangle of s^a t^b = a! b! / (a + b + 2)!
        return sum(c * sp.factorial(a) * sp.factorial(b) / sp.factorial(a + b + 2)
                   for (a, b), c in g.terms()) * jac

    M = [[integ(phi[i] * phi[j]) for j in range(10)] for i in range(10)]
    grad = [(sp.diff(f, x), sp.diff(f, y)) for f in phi]
    S = [[integ(grad[i][0] * grad[j][0] + grad[i][1] * grad[j][1]) for j in range(10)] for i in range(10)]
    return np.array(M, dtype=float), np.array(S, dtype=float)


@pytest.mark.parametrize("seed", range(2))
def test_elements_vs_symbolic(seed):
    rng = np.random.default_rng(300 + seed)
    while True:
        p = rng.integers(-20, 21, size=(3, 2)) / 7
        d = (p[1, 0] - p[0, 0]) * (p[2, 1] - p[0, 1]) - (p[2, 0] - p[0, 0]) * (p[1, 1] - p[0, 1])
        if abs(d) > 0.5:
            if d < 0:
                p = p[[0, 2, 1]]
            break
    pts = [(Fraction(int(round(a * 7)), 7), Fraction(int(round(b * 7)), 7)) for a, b in p]
    Ms, Ss = _sym_p3(pts)
    x, y = p[:, 0], p[:, 1]
    area = oracle.double_area(x, y) / 2
    np.testing.assert_allclose(oracle.p3_elem_mass(area), Ms, rtol=0, atol=1e-14 * np.abs(Ms).max())
    np.testing.assert_allclose(oracle.p3_elem_stiff(x, y, area), Ss, rtol=0, atol=1e-13 * np.abs(Ss).max())


def test_reference_triangle_closed_forms():
    """Sum of M = |T| (the basis sums to 1); the bubble's own mass int (27 l0 l1 l2)^2 =
    729 * 2|T| 2!2!2!/8! = 81/280 |T|; M and S symmetric; S 1 = 0 (the gradients of a partition of
    unity sum to zero); the bubble's stiffness diagonal positive."""
    M = oracle.p3_elem_mass(0.5)
    assert M.sum() == pytest.approx(0.5, rel=1e-14)
    assert M[9, 9] == pytest.approx(81 / 280 * 0.5, rel=1e-14)
    np.testing.assert_allclose(M, M.T, rtol=0, atol=1e-16)
    S = oracle.p3_elem_stiff(np.array([0.0, 1.0, 0.0]), np.array([0.0, 0.0, 1.0]), 0.5)
    np.testing.assert_allclose(S @ np.ones(10), 0, atol=1e-13)
    np.testing.assert_allclose(S, S.T, rtol=0, atol=1e-13)
    assert S[9, 9] > 0


def test_dof_numbering_two_triangles():
    """Vertices first; then two dofs per edge, edges in ascending (smaller id, larger id) order and
    the node nearer the smaller id first; then one bubble per triangle."""
    q = np.array([[0.0, 1.0, 1.0, 0.0], [0.0, 0.0, 1.0, 1.0]])
    me = np.array([[0, 0], [1, 2], [2, 3]], np.int32)
    I, J, K, ndof = oracle.p3_triplets(oracle.MASS, q, me)
    # edges (0,1) (0,2) (0,3) (1,2) (2,3) -> dofs 4-5, 6-7, 8-9, 10-11, 12-13; bubbles 14, 15
    assert ndof == 4 + 10 + 2
    # triangle 0 = (0, 1, 2): edge (0,1) near 0, near 1 = 4, 5; (1,2): near 1, near 2 = 10, 11;
    # (2,0): near 2 = 7 (the node of edge (0,2) nearer 2), near 0 = 6; bubble 14
    assert [int(I[il]) for il in range(10)] == [0, 1, 2, 4, 5, 10, 11, 7, 6, 14]
    # triangle 1 = (0, 2, 3): (0,2) -> 6, 7; (2,3) -> 12, 13; (3,0) -> 9 (nearer 3), 8; bubble 15
    assert [int(I[100 + il]) for il in range(10)] == [0, 2, 3, 6, 7, 12, 13, 9, 8, 15]
    for k in (0, 1):
        for c in range(100):
            il, jl = c % 10, c // 10
            assert I[100 * k + c] == I[100 * k + il] and J[100 * k + c] == I[100 * k + jl]
    pts = oracle.p3_dof_points(q, me)
    np.testing.assert_allclose(pts[:, 6], [1 / 3, 1 / 3])           # edge (0,2), nearer 0
    np.testing.assert_allclose(pts[:, 15], [1 / 3, 2 / 3])          # centroid of (0, 2, 3)


@pytest.fixture(scope="module", params=["grid", "unstructured"])
def sq(request):
    if request.param == "grid":
        m = meshgen.square_mesh(7, 4)
    else:
        m = meshgen.square_mesh(8, 6, random_diagonals=True)
    rpM, ciM, vaM = oracle.p3_assemble(oracle.MASS, m.q, m.me)
    rpS, ciS, vaS = oracle.p3_assemble(oracle.STIFF, m.q, m.me)
    n = len(rpM) - 1
    pts = oracle.p3_dof_points(m.q, m.me)
    assert pts.shape[1] == n
    return pts, oracle.csr_to_dense(rpM, ciM, vaM, n), oracle.csr_to_dense(rpS, ciS, vaS, n)


def test_mass_identities(sq):
    """P3 interpolation is exact for cubics on any triangulation of the unit square."""
    pts, M, _ = sq
    X, Y = pts
    one = np.ones(M.shape[0])
    assert one @ M @ one == pytest.approx(1.0, rel=1e-13)
    u = X ** 3
    assert u @ M @ u == pytest.approx(1.0 / 7.0, rel=1e-12)            # int x^6
    v = X * X * Y
    assert v @ M @ v == pytest.approx(1.0 / 15.0, rel=1e-12)           # int x^4 y^2
    assert one @ M @ (X * Y * Y) == pytest.approx(1.0 / 6.0, rel=1e-12)  # int x y^2
    np.testing.assert_allclose(M, M.T, rtol=0, atol=1e-16)


def test_stiffness_identities(sq):
    pts, _, S = sq
    X, Y = pts
    np.testing.assert_allclose(S @ np.ones(S.shape[0]), 0, atol=1e-11)
    u = X ** 3
    assert u @ S @ u == pytest.approx(9.0 / 5.0, rel=1e-11)            # int 9 x^4
    v = X * Y * Y
    assert v @ S @ v == pytest.approx(1.0 / 5.0 + 4.0 / 9.0, rel=1e-11)  # int y^4 + 4 x^2 y^2
    w = 2 * X - 3 * Y
    assert w @ S @ w == pytest.approx(13.0, rel=1e-11)
    np.testing.assert_allclose(S, S.T, rtol=0, atol=1e-11)


def test_row_sampler_matches_full_assembly():
    m = meshgen.square_mesh(6, 5, random_diagonals=True)
    for kind in (oracle.MASS, oracle.STIFF):
        rp, ci, va = oracle.p3_assemble(kind, m.q, m.me)
        n = len(rp) - 1
        rows = [0, 5, m.nq - 1, m.nq, m.nq + 17, n - m.nme - 1, n - m.nme, n - 1]
        for r, (cols, vals) in zip(rows, oracle.p3_row_values(kind, m.q, m.me, rows)):
            np.testing.assert_array_equal(cols, ci[rp[r]:rp[r + 1]])
            np.testing.assert_array_equal(vals, va[rp[r]:rp[r + 1]])
