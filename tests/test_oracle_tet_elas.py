"""Pins of the oracle's 3-D linear elasticity on tetrahedra: the plane elasticity of Section 7
carried to three dimensions, an extension the paper announces without formulas.

The element matrix (the oracle forms |K| B^T C B with a Voigt strain matrix) is checked three ways:
against the bilinear form lam div u div v + 2 mu eps(u):eps(v), integrated exactly with barycentric
gradients found by exact elimination (no strain vector, no material matrix); against entries worked
by hand on the reference tetrahedron; and for its six rigid modes. The assembled matrix is checked
against what holds on any tetrahedralisation of the unit cube: the energy of every linear
displacement, the rigid modes, and the traces of its 3 x 3 blocks, which equal lam + 4 mu times
the (separately pinned) scalar stiffness.
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


def _rigid_modes(P):
    """The six rigid displacements at points P (n x 3), as 3n vectors (dof 3v + d)."""
    n = P.shape[0]
    modes = []
    for d in range(3):
        t = np.zeros((n, 3))
        t[:, d] = 1.0
        modes.append(t.ravel())
    for d in range(3):
        w = np.zeros(3)
        w[d] = 1.0
        modes.append(np.cross(w, P).ravel())                 # u = w x p, an infinitesimal rotation
    return modes


def test_reference_tetrahedron_by_hand():
    """grad(phi_0) = (-1, -1, -1), grad(phi_a) = e_a (a = 1, 2, 3). With |K| taken as 1, the entry
    of dofs (a, alpha), (b, beta) is lam g_a,alpha g_b,beta + mu (g_a,beta g_b,alpha + [alpha = beta]
    g_a . g_b); lam = 3, mu = 0.75 make every value exact."""
    x, y, z = _xyz(REF)
    lam, mu = 3.0, 0.75
    E = oracle.tet_elem_elas(x, y, z, 1.0, lam, mu)
    assert E[0, 0] == lam + mu * (1 + 3)          # (0,x),(0,x): g0x^2 = 1, |g0|^2 = 3
    assert E[0, 1] == lam + mu                    # (0,x),(0,y)
    assert E[0, 3] == -lam - 2 * mu               # (0,x),(1,x): g0x g1x = -1, g0 . g1 = -1
    assert E[0, 4] == -mu                         # (0,x),(1,y): only mu g0y g1x = -mu
    assert E[1, 3] == -lam                        # (0,y),(1,x): only lam g0y g1x = -lam
    assert E[3, 3] == lam + 2 * mu                # (1,x),(1,x)
    assert E[4, 4] == mu                          # (1,y),(1,y): only mu |g1|^2
    assert E[3, 7] == lam                         # (1,x),(2,y): lam g1x g2y
    assert E[4, 6] == mu                          # (1,y),(2,x): mu g1x g2y
    assert E[3, 6] == 0.0 and E[3, 10] == 0.0     # (1,x),(2,x) and (1,x),(3,y)
    # and the whole matrix against the exact bilinear form (|K| = 1/6 there)
    want = np.array([[float(v) for v in row] for row in exact_fe.tet_elas(REF, Fraction(3), Fraction(3, 4))])
    np.testing.assert_allclose(E / 6.0, want, rtol=0, atol=1e-15 * np.abs(want).max())


@pytest.mark.parametrize("seed", range(4))
def test_element_vs_bilinear_form(seed):
    rng = np.random.default_rng(500 + seed)
    while True:
        p = rng.integers(-12, 13, size=(4, 3)) / 4.0
        d = np.linalg.det(np.stack([p[1] - p[0], p[2] - p[0], p[3] - p[0]], axis=1))
        if abs(d) > 0.5:
            if d < 0:
                p = p[[0, 1, 3, 2]]
            break
    lam, mu = [(1.0, 0.5), (-0.25, 1.0), (7.0, 0.125), (0.0, 2.0)][seed]   # 3 lam + 2 mu > 0, mu > 0
    pts = [tuple(Fraction(float(c)) for c in row) for row in p]
    x, y, z = p[:, 0], p[:, 1], p[:, 2]
    vol = oracle.tet_volume6(x, y, z) / 6
    got = oracle.tet_elem_elas(x, y, z, vol, lam, mu)
    want = np.array([[float(v) for v in row] for row in exact_fe.tet_elas(pts, Fraction(lam), Fraction(mu))])
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-13 * np.abs(want).max())


def test_element_rigid_modes_and_spectrum():
    rng = np.random.default_rng(7)
    p = rng.uniform(-1, 2, size=(4, 3))
    if np.linalg.det(np.stack([p[1] - p[0], p[2] - p[0], p[3] - p[0]], axis=1)) < 0:
        p = p[[0, 1, 3, 2]]
    x, y, z = p[:, 0], p[:, 1], p[:, 2]
    E = oracle.tet_elem_elas(x, y, z, oracle.tet_volume6(x, y, z) / 6, 2.0, 0.7)
    scale = np.abs(E).max()
    for r in _rigid_modes(p):
        assert np.abs(E @ r).max() <= 1e-12 * scale * np.abs(r).max()
    np.testing.assert_allclose(E, E.T, rtol=0, atol=1e-14 * scale)
    ev = np.linalg.eigvalsh(E)
    assert (np.abs(ev[:6]) <= 1e-12 * scale).all() and (ev[6:] > 1e-6 * scale).all()


def test_triplet_layout():
    m = meshgen.cube_mesh(2, 3)
    I, J, K = oracle.tet_elas_triplets(m.q, m.me, 1.0, 0.5)
    for k in (0, 11, m.nme - 1):
        v = m.me[:, k]
        for c in range(144):
            il, jl = c % 12, c // 12             # column-wise storage of the element matrix
            assert I[144 * k + c] == 3 * v[il // 3] + il % 3 and J[144 * k + c] == 3 * v[jl // 3] + jl % 3


def test_brute_force_dense_one_cube():
    """The unjittered unit cube (6 tetrahedra) against the exact dense sum of bilinear forms."""
    m = meshgen.cube_mesh(1, 1, jitter=0.0, permute=False)
    lam, mu = Fraction(5, 4), Fraction(3, 8)
    rp, ci, va = oracle.tet_elas_assemble(m.q, m.me, float(lam), float(mu))
    n = 3 * m.nq
    G = np.zeros((n, n))
    for k in range(m.nme):
        t = [int(v) for v in m.me[:, k]]
        E = exact_fe.tet_elas([tuple(Fraction(float(c)) for c in m.q[:, v]) for v in t], lam, mu)
        for I in range(12):
            for J in range(12):
                G[3 * t[I // 3] + I % 3, 3 * t[J // 3] + J % 3] += float(E[I][J])
    got = oracle.csr_to_dense(rp, ci, va, n)
    np.testing.assert_allclose(got, G, rtol=0, atol=1e-15 * np.abs(G).max())


@pytest.fixture(scope="module")
def cube4():
    m = meshgen.cube_mesh(4, 21)
    lam, mu = 1.5, 0.6
    rp, ci, va = oracle.tet_elas_assemble(m.q, m.me, lam, mu)
    return m, lam, mu, rp, ci, va


def test_pattern_is_the_block_expansion(cube4):
    """Row 3i + d holds columns 3j, 3j+1, 3j+2 for every column j of scalar row i."""
    m, _, _, rp, ci, _ = cube4
    rps, cis, _ = oracle.tet_assemble(oracle.STIFF, m.q, m.me)
    for i in range(m.nq):
        cols = cis[rps[i]:rps[i + 1]]
        want = np.stack([3 * cols, 3 * cols + 1, 3 * cols + 2], axis=1).ravel()
        for d in range(3):
            np.testing.assert_array_equal(ci[rp[3 * i + d]:rp[3 * i + d + 1]], want)


def test_block_traces_are_scaled_stiffness(cube4):
    """sum_d K[3i+d, 3j+d] = (lam + 4 mu) S[i, j]: the trace of a 3 x 3 block of the element
    form is |K| (lam + mu + 3 mu) g_a . g_b."""
    m, lam, mu, rp, ci, va = cube4
    K = oracle.csr_to_dense(rp, ci, va, 3 * m.nq)
    rps, cis, vas = oracle.tet_assemble(oracle.STIFF, m.q, m.me)
    S = oracle.csr_to_dense(rps, cis, vas, m.nq)
    T = K[0::3, 0::3] + K[1::3, 1::3] + K[2::3, 2::3]
    np.testing.assert_allclose(T, (lam + 4 * mu) * S, rtol=0, atol=1e-13 * np.abs(T).max())


def test_linear_displacement_energies(cube4):
    """For u(p) = A p + t (in the P1 space), u^T K u = int lam (tr eps)^2 + 2 mu eps:eps over the unit
    cube = lam (tr A)^2 + 2 mu |sym A|_F^2, on any tetrahedralisation."""
    m, lam, mu, rp, ci, va = cube4
    K = oracle.csr_to_dense(rp, ci, va, 3 * m.nq)
    P = m.q.T
    rng = np.random.default_rng(3)
    for _ in range(4):
        A = rng.normal(size=(3, 3))
        t = rng.normal(size=3)
        u = (P @ A.T + t).ravel()
        sym = (A + A.T) / 2
        want = lam * np.trace(A) ** 2 + 2 * mu * (sym * sym).sum()
        assert u @ K @ u == pytest.approx(want, rel=1e-12)
    np.testing.assert_allclose(K, K.T, rtol=0, atol=1e-13 * np.abs(K).max())


def test_global_rigid_modes(cube4):
    m, _, _, rp, ci, va = cube4
    K = oracle.csr_to_dense(rp, ci, va, 3 * m.nq)
    for r in _rigid_modes(m.q.T):
        assert np.abs(K @ r).max() <= 1e-12 * np.abs(K).max()
