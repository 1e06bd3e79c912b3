"""Pins of the oracle's P2 (quadratic) triangle assembly, the P_k extension the paper announces
without formulas. Element matrices are checked against an independent symbolic integration (sympy:
the basis functions built in x, y from their nodal values, integrated over the triangle), and the
assembled matrices against what quadratic functions, which the P2 space contains, fix exactly.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1305_3122_gb300 import meshgen


def _sym_p2(pts):
    """P2 mass and stiffness of the triangle pts (rationals), by sympy from the definitions: the six
    basis polynomials a + b x + c y + d x^2 + e x y + f y^2 with phi_i(node_j) = delta_ij (nodes:
    vertices, then the midpoints of (0,1), (1,2), (2,0)), integrated over the triangle."""
    sp = pytest.importorskip("sympy")
    x, y, s, t = sp.symbols("x y s t")
    P = [sp.Matrix([sp.Rational(px), sp.Rational(py)]) for px, py in pts]
    nodes = P + [(P[0] + P[1]) / 2, (P[1] + P[2]) / 2, (P[2] + P[0]) / 2]
    mono = [sp.Integer(1), x, y, x * x, x * y, y * y]
    V = sp.Matrix([[m.subs({x: n[0], y: n[1]}) for m in mono] for n in nodes])
    C = V.inv()                                   # column i: coefficients of phi_i
    phi = [sum(C[r, i] * mono[r] for r in range(6)) for i in range(6)]
    # the triangle as the image of the unit triangle (s, t >= 0, s + t <= 1)
    X = P[0] + s * (P[1] - P[0]) + t * (P[2] - P[0])
    jac = abs((P[1] - P[0]).row_join(P[2] - P[0]).det())

    def integ(f):
        g = sp.expand(f.subs({x: X[0], y: X[1]}, simultaneous=True))
        return sp.integrate(sp.integrate(g, (t, 0, 1 - s)), (s, 0, 1)) * jac

    M = [[integ(phi[i] * phi[j]) for j in range(6)] for i in range(6)]
    grad = [(sp.diff(f, x), sp.diff(f, y)) for f in phi]
    S = [[integ(grad[i][0] * grad[j][0] + grad[i][1] * grad[j][1]) for j in range(6)] for i in range(6)]
    return np.array(M, dtype=float), np.array(S, dtype=float)


@pytest.mark.parametrize("seed", range(3))
def test_elements_vs_symbolic(seed):
    rng = np.random.default_rng(200 + seed)
    while True:
        p = rng.integers(-20, 21, size=(3, 2)) / 7
        d = (p[1, 0] - p[0, 0]) * (p[2, 1] - p[0, 1]) - (p[2, 0] - p[0, 0]) * (p[1, 1] - p[0, 1])
        if abs(d) > 0.5:
            if d < 0:
                p = p[[0, 2, 1]]
            break
    pts = [(Fraction(int(round(a * 7)), 7), Fraction(int(round(b * 7)), 7)) for a, b in p]
    Ms, Ss = _sym_p2(pts)
    x, y = p[:, 0], p[:, 1]
    area = oracle.double_area(x, y) / 2
    np.testing.assert_allclose(oracle.p2_elem_mass(area), Ms, rtol=0, atol=1e-14 * np.abs(Ms).max())
    np.testing.assert_allclose(oracle.p2_elem_stiff(x, y, area), Ss, rtol=0, atol=1e-13 * np.abs(Ss).max())


def test_reference_triangle_exact():
    x, y = np.array([0.0, 1.0, 0.0]), np.array([0.0, 0.0, 1.0])
    M = oracle.p2_elem_mass(0.5)
    np.testing.assert_allclose(360 * M, [[6, -1, -1, 0, -4, 0], [-1, 6, -1, 0, 0, -4], [-1, -1, 6, -4, 0, 0],
                                         [0, 0, -4, 32, 16, 16], [-4, 0, 0, 16, 32, 16], [0, -4, 0, 16, 16, 32]],
                               rtol=0, atol=1e-12)
    S = oracle.p2_elem_stiff(x, y, 0.5)
    np.testing.assert_allclose(S @ np.ones(6), 0, atol=1e-15)


def test_dof_numbering_two_triangles():
    """Vertices first, then the edges in ascending (smaller id, larger id) order."""
    q = np.array([[0.0, 1.0, 1.0, 0.0], [0.0, 0.0, 1.0, 1.0]])
    me = np.array([[0, 0], [1, 2], [2, 3]], np.int32)
    I, J, K, ndof = oracle.p2_triplets(oracle.MASS, q, me)
    assert ndof == 4 + 5                       # edges (0,1) (0,2) (0,3) (1,2) (2,3) -> dofs 4..8
    # triangle 0 = (0, 1, 2): local edge dofs (0,1) -> 4, (1,2) -> 7, (2,0) -> 5
    assert [int(I[36 * 0 + 6 * 0 + il]) for il in range(6)] == [0, 1, 2, 4, 7, 5]
    # triangle 1 = (0, 2, 3): (0,2) -> 5, (2,3) -> 8, (3,0) -> 6
    assert [int(I[36 * 1 + 6 * 0 + il]) for il in range(6)] == [0, 2, 3, 5, 8, 6]
    for k in (0, 1):
        for c in range(36):
            il, jl = c % 6, c // 6
            assert I[36 * k + c] == I[36 * k + il] and J[36 * k + c] == I[36 * k + jl]


@pytest.fixture(scope="module")
def sq():
    m = meshgen.square_mesh(9, 4)
    rpM, ciM, vaM = oracle.p2_assemble(oracle.MASS, m.q, m.me)
    rpS, ciS, vaS = oracle.p2_assemble(oracle.STIFF, m.q, m.me)
    n = len(rpM) - 1
    return m, oracle.csr_to_dense(rpM, ciM, vaM, n), oracle.csr_to_dense(rpS, ciS, vaS, n)


def test_mass_identities(sq):
    """P2 interpolation is exact for quadratics on any mesh of the unit square."""
    m, M, _ = sq
    one = np.ones(M.shape[0])
    assert one @ M @ one == pytest.approx(1.0, rel=1e-13)
    u = oracle.p2_dof_values(m.q, m.me, lambda x, y: x * x)
    assert u @ M @ u == pytest.approx(0.2, rel=1e-13)                  # int x^4
    v = oracle.p2_dof_values(m.q, m.me, lambda x, y: x * y)
    assert v @ M @ v == pytest.approx(1.0 / 9.0, rel=1e-13)            # int x^2 y^2
    assert one @ M @ v == pytest.approx(0.25, rel=1e-13)               # int x y
    np.testing.assert_allclose(M, M.T, rtol=0, atol=1e-16)


def test_stiffness_identities(sq):
    m, _, S = sq
    np.testing.assert_allclose(S @ np.ones(S.shape[0]), 0, atol=1e-12)
    u = oracle.p2_dof_values(m.q, m.me, lambda x, y: x * x)
    assert u @ S @ u == pytest.approx(4.0 / 3.0, rel=1e-12)            # int |grad x^2|^2 = int 4 x^2
    v = oracle.p2_dof_values(m.q, m.me, lambda x, y: x * y)
    assert v @ S @ v == pytest.approx(2.0 / 3.0, rel=1e-12)            # int x^2 + y^2
    w = oracle.p2_dof_values(m.q, m.me, lambda x, y: 2 * x - 3 * y)
    assert w @ S @ w == pytest.approx(13.0, rel=1e-12)                 # int |(2, -3)|^2
    np.testing.assert_allclose(S, S.T, rtol=0, atol=1e-12)


def test_row_sampler_matches_full_assembly():
    m = meshgen.square_mesh(7, 5)
    for kind in (oracle.MASS, oracle.STIFF):
        rp, ci, va = oracle.p2_assemble(kind, m.q, m.me)
        rows = [0, 5, m.nq - 1, m.nq, m.nq + 17, len(rp) - 2]
        for r, (cols, vals) in zip(rows, oracle.p2_row_values(kind, m.q, m.me, rows)):
            np.testing.assert_array_equal(cols, ci[rp[r]:rp[r + 1]])
            np.testing.assert_array_equal(vals, va[rp[r]:rp[r + 1]])
