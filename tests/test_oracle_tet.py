"""Pins of the oracle's tetrahedral (3-D P1) assembly, the extension the paper announces without
formulas. Each element matrix is checked against an exact-rational derivation from the
definitions (barycentric coordinates by exact elimination, the monomial integral formula), and the
assembled matrices against identities that hold on any tetrahedralisation of the unit cube.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1305_3122_gb300 import meshgen
from tests import exact_fe

REF = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)]


def _xyz(pts):
    a = np.array(pts, dtype=float)
    return a[:, 0], a[:, 1], a[:, 2]


def _rand_tet(rng):
    while True:
        p = rng.uniform(-2, 3, size=(4, 3))
        d = np.linalg.det(np.stack([p[1] - p[0], p[2] - p[0], p[3] - p[0]], axis=1))
        if abs(d) > 0.5:
            if d < 0:
                p = p[[0, 1, 3, 2]]
            return p


def test_reference_tetrahedron_exact():
    x, y, z = _xyz(REF)
    d = oracle.tet_volume6(x, y, z)
    assert d == 1.0
    S = oracle.tet_elem_stiff(x, y, z, d / 6)
    np.testing.assert_array_equal(6 * S, [[3, -1, -1, -1], [-1, 1, 0, 0], [-1, 0, 1, 0], [-1, 0, 0, 1]])
    M = oracle.tet_elem_mass(d / 6)
    np.testing.assert_array_equal(120 * M, 1 + np.eye(4))


@pytest.mark.parametrize("seed", range(6))
def test_elements_vs_exact_derivation(seed):
    rng = np.random.default_rng(100 + seed)
    p = _rand_tet(rng)
    pts = [tuple(Fraction(float(c)) for c in row) for row in p]
    w = rng.uniform(0.5, 2.0, 4)
    x, y, z = p[:, 0], p[:, 1], p[:, 2]
    vol = oracle.tet_volume6(x, y, z) / 6
    assert vol == pytest.approx(float(exact_fe.volume3(pts)), rel=1e-14)
    for got, want in ((oracle.tet_elem_mass(vol), exact_fe.tet_mass(pts)),
                      (oracle.tet_elem_wmass(vol, w), exact_fe.tet_wmass(pts, [Fraction(float(v)) for v in w])),
                      (oracle.tet_elem_stiff(x, y, z, vol), exact_fe.tet_stiff(pts))):
        want = np.array([[float(v) for v in row] for row in want])
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-13 * np.abs(want).max())


def test_triplet_layout():
    m = meshgen.cube_mesh(2, 3)
    I, J, K = oracle.tet_triplets(oracle.STIFF, m.q, m.me)
    for k in (0, 7, m.nme - 1):
        v = m.me[:, k]
        for c in range(16):
            il, jl = c % 4, c // 4       # column-wise storage of the element matrix
            assert I[16 * k + c] == v[il] and J[16 * k + c] == v[jl]


def test_brute_force_dense_one_cube():
    """The unjittered unit cube (6 tetrahedra, 8 vertices) against the exact dense assembly."""
    m = meshgen.cube_mesh(1, 1, jitter=0.0, permute=False)
    pts = [tuple(Fraction(float(c)) for c in m.q[:, i]) for i in range(m.nq)]
    tets = [tuple(int(v) for v in m.me[:, k]) for k in range(m.nme)]
    w = [Fraction(v) for v in (1, 2, 3, 4, 5, 6, 7, 8)]
    for kind, name in ((oracle.MASS, "mass"), (oracle.WMASS, "wmass"), (oracle.STIFF, "stiff")):
        rp, ci, va = oracle.tet_assemble(kind, m.q, m.me, np.array([float(v) for v in w]))
        G = exact_fe.tet_assemble_dense(name, pts, tets, w)
        want = np.array([[float(v) for v in row] for row in G])
        got = oracle.csr_to_dense(rp, ci, va, m.nq)
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-15 * np.abs(want).max())
        # the pattern is structural: every pair sharing a tetrahedron, zeros included
        assert len(ci) == int(sum(1 for i in range(8) for j in range(8)
                                  if any(i in t and j in t for t in tets)))


@pytest.fixture(scope="module")
def cube5():
    m = meshgen.cube_mesh(5, 9)
    w = meshgen.vertex_weights3(m, 9)
    return m, w


def test_mass_identities(cube5):
    m, w = cube5
    rp, ci, va = oracle.tet_assemble(oracle.MASS, m.q, m.me)
    A = oracle.csr_to_dense(rp, ci, va, m.nq)
    assert A.sum() == pytest.approx(1.0, rel=1e-13)                      # volume of the cube
    x, y, z = m.q
    assert x @ A @ x == pytest.approx(1.0 / 3.0, rel=1e-13)             # int x^2 (x is in the P1 space)
    assert x @ A @ y == pytest.approx(0.25, rel=1e-13)                  # int x y
    rpw, ciw, vaw = oracle.tet_assemble(oracle.WMASS, m.q, m.me, np.ones(m.nq))
    np.testing.assert_allclose(vaw, va, rtol=1e-14, atol=0)             # w = 1 gives M
    rpw, ciw, vaw = oracle.tet_assemble(oracle.WMASS, m.q, m.me, x)     # w = x: int x * u * v
    Aw = oracle.csr_to_dense(rpw, ciw, vaw, m.nq)
    assert np.ones(m.nq) @ Aw @ np.ones(m.nq) == pytest.approx(0.5, rel=1e-13)   # int x
    assert np.ones(m.nq) @ Aw @ y == pytest.approx(0.25, rel=1e-13)              # int x y


def test_stiffness_identities(cube5):
    m, _ = cube5
    rp, ci, va = oracle.tet_assemble(oracle.STIFF, m.q, m.me)
    A = oracle.csr_to_dense(rp, ci, va, m.nq)
    np.testing.assert_allclose(A @ np.ones(m.nq), 0, atol=1e-12)         # constants in the kernel
    np.testing.assert_allclose(A, A.T, rtol=0, atol=1e-13)
    x, y, z = m.q
    for u, want in ((x, 1.0), (y, 1.0), (z, 1.0), (x + 2 * y - z, 6.0)):
        assert u @ A @ u == pytest.approx(want, rel=1e-12)              # int |grad u|^2 for linear u
    interior = np.all((m.q > 1e-12) & (m.q < 1 - 1e-12), axis=0)
    for u in (x, y, z):
        np.testing.assert_allclose((A @ u)[interior], 0, atol=1e-12)     # patch test at interior rows


def test_rejects_bad_tetrahedra():
    m = meshgen.cube_mesh(1, 1, jitter=0.0, permute=False)
    me = m.me.copy()
    me[2, 3], me[3, 3] = me[3, 3], me[2, 3]
    with pytest.raises(oracle.OracleError, match="counter-clockwise"):
        oracle.tet_assemble(oracle.MASS, m.q, me)
    me = m.me.copy()
    me[1, 0] = me[0, 0]
    with pytest.raises(oracle.OracleError, match="repeated"):
        oracle.tet_assemble(oracle.MASS, m.q, me)
    me = m.me.copy()
    me[0, 2] = m.nq
    with pytest.raises(oracle.OracleError, match="range"):
        oracle.tet_assemble(oracle.MASS, m.q, me)
