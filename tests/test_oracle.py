"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU needed).

Each test is chosen so that a plausible mistake in the oracle (a dropped term, a wrong sign or
index, a transposed operand, a wrong summation order) fails at least one of them:
  - element matrices vs an independent exact-rational derivation (tests/exact_fe.py);
  - the worked CSC example of Section 4 (non-symmetric, so a transposition shows);
  - the triplet layout of Sections 5-7 (Ig = me([1 2 3 1 2 3 1 2 3],:), Jg = me([1 1 1 2 2 2 ...]));
  - exact rational values on a two-triangle square, brute-force dense assembly on small meshes;
  - integral identities that hold for any mesh of the unit square.
"""
from __future__ import annotations

import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1305_3122_gb300 import meshgen
from tests import exact_fe

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_triangle(rng):
    while True:
        p = rng.uniform(-2, 3, size=(3, 2))
        d = (p[1, 0] - p[0, 0]) * (p[2, 1] - p[0, 1]) - (p[2, 0] - p[0, 0]) * (p[1, 1] - p[0, 1])
        if abs(d) > 0.3:
            if d < 0:
                p = p[[0, 2, 1]]
            return p


def _frac_mat(E):
    return np.array([[float(v) for v in row] for row in E])


# ------------------------------------------------------------------ element level

def test_reference_triangle_exact():
    """Reference triangle (0,0),(1,0),(0,1): every entry is a short binary fraction, so the
    oracle must reproduce the exact rationals bit for bit."""
    x = np.array([0.0, 1.0, 0.0])
    y = np.array([0.0, 0.0, 1.0])
    pts = list(zip([0, 1, 0], [0, 0, 1]))
    D = oracle.double_area(x, y)
    assert D == 1.0
    area = D / 2
    np.testing.assert_array_equal(oracle.elem_mass(area), _frac_mat(exact_fe.mass(pts)))
    np.testing.assert_array_equal(oracle.elem_stiff(x, y, area), _frac_mat(exact_fe.stiff(pts)))
    K = oracle.elem_elas(x, y, area, 1.0, 0.5)
    np.testing.assert_array_equal(K, _frac_mat(exact_fe.elas(pts, 1, Fraction(1, 2))))
    # the K^e rows worked by hand for lambda = 1, mu = 1/2
    hand = np.array([[5, 3, -4, -1, -1, -2], [3, 5, -2, -1, -1, -4], [-4, -2, 4, 0, 0, 2],
                     [-1, -1, 0, 1, 1, 0], [-1, -1, 0, 1, 1, 0], [-2, -4, 2, 0, 0, 4]]) / 4.0
    np.testing.assert_array_equal(K, hand)


@pytest.mark.parametrize("seed", range(8))
def test_elements_vs_exact_derivation(seed):
    rng = np.random.default_rng(seed)
    p = _rand_triangle(rng)
    x, y = p[:, 0].copy(), p[:, 1].copy()
    pts = [(Fraction(float(a)), Fraction(float(b))) for a, b in p]
    area = oracle.double_area(x, y) / 2
    assert area == pytest.approx(float(exact_fe.area(pts)), rel=1e-15)
    w = rng.uniform(0.5, 2.0, 3)
    lam, mu = float(rng.uniform(0.1, 3)), float(rng.uniform(0.1, 3))
    cases = [
        (oracle.elem_mass(area), exact_fe.mass(pts)),
        (oracle.elem_wmass(area, w), exact_fe.wmass(pts, [Fraction(float(v)) for v in w])),
        (oracle.elem_stiff(x, y, area), exact_fe.stiff(pts)),
        (oracle.elem_elas(x, y, area, lam, mu),
         exact_fe.elas(pts, Fraction(lam), Fraction(mu))),
    ]
    for got, want in cases:
        want = _frac_mat(want)
        scale = np.abs(want).max()
        assert np.abs(got - want).max() <= 1e-14 * scale


def test_wmass_with_unit_weight_is_mass():
    rng = np.random.default_rng(3)
    p = _rand_triangle(rng)
    area = oracle.double_area(p[:, 0].copy(), p[:, 1].copy()) / 2
    np.testing.assert_allclose(oracle.elem_wmass(area, np.ones(3)), oracle.elem_mass(area),
                               rtol=1e-15)


# ------------------------------------------------------------------ sparse() semantics

def _load_golden_csc():
    rows = {}
    lines = [l.split() for l in open(os.path.join(GOLDEN, "csc_example.txt"))
             if l.strip() and not l.startswith("#")]
    i = 0
    while i < len(lines):
        tag = lines[i][0]
        if tag in ("A", "A2"):
            m, n = int(lines[i][1]), int(lines[i][2])
            rows[tag] = np.array([[float(v) for v in lines[i + 1 + r]] for r in range(m)])
            i += 1 + m
        else:
            rows[tag] = [float(v) for v in lines[i][1:]]
            i += 1
    return rows


@pytest.mark.parametrize("which", ["", "2"])
def test_paper_csc_example(which):
    """Section 4's 3x4 example. CSC of A equals CSR of A^T, so sparse() is called with the
    roles of rows and columns exchanged; the triplets are fed in a scrambled order with one
    entry split in two, and aa / ia / ja must come out exactly as printed."""
    g = _load_golden_csc()
    A = g["A" + which]
    I, J = np.nonzero(A)
    K = A[I, J]
    # split the largest entry in two pieces (sparse sums duplicates)
    s = int(np.argmax(K))
    I = np.append(I, I[s]); J = np.append(J, J[s]); K = np.append(K, K[s] / 2); K[s] /= 2
    order = np.random.default_rng(0).permutation(len(K))
    rp, ci, va = oracle.sparse(J[order], I[order], K[order], A.shape[1], A.shape[0])
    np.testing.assert_array_equal(va, g["aa" + which])
    np.testing.assert_array_equal(ci + 1, g["ia" + which])
    np.testing.assert_array_equal(rp + 1, g["ja" + which])


def test_sparse_sums_in_ascending_input_order_and_keeps_zeros():
    I = np.array([1, 0, 1, 1, 0, 2], np.int32)
    J = np.array([1, 0, 1, 1, 0, 2], np.int32)
    K = np.array([1e16, 1.0, 1.0, -1e16, -1.0, 0.0])
    rp, ci, va = oracle.sparse(I, J, K, 3, 3)
    np.testing.assert_array_equal(rp, [0, 1, 2, 3])
    np.testing.assert_array_equal(ci, [0, 1, 2])
    # (1e16 + 1) - 1e16 == 0 in round-to-nearest: the left-to-right order is the oracle's
    assert va[1] == 0.0
    assert va[0] == 0.0 and va[2] == 0.0     # exact zeros are stored, not dropped


@pytest.mark.parametrize("which", ["", "2"])
def test_paper_csc_example_drop_zeros(which):
    """Section 4's example with every entry of the dense A fed as a triplet, zeros included, and
    one zero position fed as x and -x: sparse() keeps those positions (structural reading), and
    dropping the zeros must give the printed aa / ia / ja, which store no zero."""
    g = _load_golden_csc()
    A = g["A" + which]
    J, I = np.meshgrid(np.arange(A.shape[1]), np.arange(A.shape[0]))
    I, J = I.ravel(), J.ravel()
    K = A[I, J]
    z = int(np.nonzero(K == 0)[0][0])
    I = np.append(I, I[z]); J = np.append(J, J[z]); K = np.append(K, 3.5); K[z] = -3.5
    order = np.random.default_rng(1).permutation(len(K))
    rp, ci, va = oracle.sparse(J[order], I[order], K[order], A.shape[1], A.shape[0])
    assert len(va) == A.size                         # structural: zeros stored
    rp, ci, va = oracle.drop_zeros(rp, ci, va)
    np.testing.assert_array_equal(va, g["aa" + which])
    np.testing.assert_array_equal(ci + 1, g["ia" + which])
    np.testing.assert_array_equal(rp + 1, g["ja" + which])


def test_drop_zeros_cell_diagonals_of_unjittered_mesh():
    """On the unjittered N x N mesh with N a power of two (exact coordinates) every cell's diagonal
    is opposite a right angle in both of its triangles, so S is exactly 0 there (cot 90 = 0,
    Eq. 3): dropping the zeros removes exactly those 2 N^2 entries, node ids differing by N + 2
    in the unpermuted numbering. M has no zero."""
    N = 8
    m = meshgen.square_mesh(N, 3, jitter=0.0, permute=False)
    rp, ci, va = oracle.assemble(oracle.STIFF, m.q, m.me)
    rp2, ci2, va2 = oracle.drop_zeros(rp, ci, va)
    assert len(ci) - len(ci2) == 2 * N * N
    rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    gone = va == 0.0
    assert np.all(np.abs(rows[gone] - ci[gone]) == N + 2)
    np.testing.assert_array_equal(va2, va[~gone])
    np.testing.assert_array_equal(ci2, ci[~gone])
    rpm, cim, vam = oracle.assemble(oracle.MASS, m.q, m.me)
    rpm2, cim2, vam2 = oracle.drop_zeros(rpm, cim, vam)
    np.testing.assert_array_equal(rpm2, rpm)


def test_drop_zeros_special_values():
    """+0 and -0 go; NaN, subnormals and negative values stay, in order; empty rows stay empty."""
    rp = np.array([0, 3, 3, 7, 8], np.int32)
    ci = np.array([0, 2, 3, 0, 1, 2, 3, 1], np.int32)
    va = np.array([0.0, np.nan, -0.0, 5e-324, -2.0, 0.0, 1.0, 0.0])
    rp2, ci2, va2 = oracle.drop_zeros(rp, ci, va)
    np.testing.assert_array_equal(rp2, [0, 1, 1, 4, 4])
    np.testing.assert_array_equal(ci2, [2, 0, 1, 3])
    assert np.isnan(va2[0]) and va2[1] == 5e-324 and va2[2] == -2.0 and va2[3] == 1.0


def test_drop_zeros_brute_force():
    """Random CSR with about a third of the values zero, against a boolean mask and per-row
    counts."""
    rng = np.random.default_rng(5)
    for n_rows in (0, 1, 17, 300):
        lens = rng.integers(0, 12, n_rows)
        rp = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
        nnz = int(rp[-1])
        ci = rng.integers(0, 50, nnz).astype(np.int32)
        va = rng.standard_normal(nnz) * (rng.random(nnz) > 0.35)
        rp2, ci2, va2 = oracle.drop_zeros(rp, ci, va)
        keep = va != 0
        np.testing.assert_array_equal(ci2, ci[keep])
        np.testing.assert_array_equal(va2, va[keep])
        per_row = np.array([keep[rp[i]:rp[i + 1]].sum() for i in range(n_rows)], dtype=np.int64)
        np.testing.assert_array_equal(np.diff(rp2), per_row)


def test_sparse_rejects_out_of_range():
    with pytest.raises(oracle.OracleError):
        oracle.sparse(np.array([0, 3]), np.array([0, 0]), np.array([1.0, 2.0]), 3, 3)


# ------------------------------------------------------------------ triplet layout

def test_triplet_layout_follows_paper():
    m = meshgen.square_mesh(3, 7)
    for kind, n in ((oracle.STIFF, 3), (oracle.ELAS, 6)):
        I, J, K = oracle.triplets(kind, m.q, m.me)
        for k in (0, 5, m.nme - 1):
            v = m.me[:, k]
            dof = [2 * v[i // 2] + i % 2 for i in range(6)] if n == 6 else list(v)
            for c in range(n * n):
                il, jl = c % n, c // n     # column-wise storage of the element matrix
                assert I[n * n * k + c] == dof[il]
                assert J[n * n * k + c] == dof[jl]


# ------------------------------------------------------------------ two triangles, exact

TWO_Q = np.array([[0.0, 1.0, 1.0, 0.0], [0.0, 0.0, 1.0, 1.0]])
TWO_ME = np.array([[0, 0], [1, 2], [2, 3]], np.int32)


def _csr_equals_exact(rp, ci, va, G, exact=True):
    n = len(G)
    nzs = [(i, j) for i in range(n) for j in range(n)]
    dense = oracle.csr_to_dense(rp, ci, va, n)
    want = np.array([[float(G[i][j]) for j in range(n)] for i in range(n)])
    if exact:
        np.testing.assert_array_equal(dense, want)
    else:
        np.testing.assert_allclose(dense, want, rtol=0, atol=1e-15 * np.abs(want).max())
    return nzs


def test_two_triangles():
    pts = [(0, 0), (1, 0), (1, 1), (0, 1)]
    me = [(0, 1, 2), (0, 2, 3)]
    w = np.array([1.0, 2.0, 3.0, 4.0])
    for kind, name in ((oracle.MASS, "mass"), (oracle.STIFF, "stiff"), (oracle.WMASS, "wmass")):
        rp, ci, va = oracle.assemble(kind, TWO_Q, TWO_ME, w)
        assert len(ci) == 14                 # (1,3) and (3,1) share no element
        assert not any(ci[rp[1]:rp[2]] == 3) and not any(ci[rp[3]:rp[4]] == 1)
        G = exact_fe.assemble_dense(name, pts, me, [Fraction(v) for v in (1, 2, 3, 4)])
        _csr_equals_exact(rp, ci, va, G, exact=(name != "wmass"))
    rp, ci, va = oracle.assemble(oracle.STIFF, TWO_Q, TWO_ME)
    assert va[rp[0] + 2] == 0.0              # S_02 == 0 is stored (structural pattern)
    rpw, ciw, vaw = oracle.assemble(oracle.WMASS, TWO_Q, TWO_ME, w)
    assert vaw.sum() == pytest.approx(7.0 / 3.0, rel=1e-15)
    rpk, cik, vak = oracle.assemble(oracle.ELAS, TWO_Q, TWO_ME, lam=1.0, mu=0.5)
    assert len(cik) == 56
    G = exact_fe.assemble_dense("elas", pts, me, lam=1, mu=Fraction(1, 2))
    _csr_equals_exact(rpk, cik, vak, G)


# ------------------------------------------------------------------ brute force

@pytest.mark.parametrize("N,seed", [(3, 1), (5, 2), (9, 3)])
def test_brute_force_dense(N, seed):
    m = meshgen.square_mesh(N, seed)
    w = meshgen.vertex_weights(m, seed)
    pts = [(Fraction(float(m.q[0, i])), Fraction(float(m.q[1, i]))) for i in range(m.nq)]
    tris = [tuple(int(v) for v in m.me[:, k]) for k in range(m.nme)]
    wf = [Fraction(float(v)) for v in w]
    for kind, name in ((oracle.MASS, "mass"), (oracle.WMASS, "wmass"), (oracle.STIFF, "stiff"),
                       (oracle.ELAS, "elas")):
        if name == "elas" and N > 5:
            continue
        rp, ci, va = oracle.assemble(kind, m.q, m.me, w, lam=1.0, mu=0.5)
        G = exact_fe.assemble_dense(name, pts, tris, wf, lam=1, mu=Fraction(1, 2))
        n = len(G)
        want = np.array([[float(G[i][j]) for j in range(n)] for i in range(n)])
        dense = oracle.csr_to_dense(rp, ci, va, n)
        for i in range(n):
            scale = np.abs(want[i]).max()
            assert np.abs(dense[i] - want[i]).max() <= 1e-13 * scale
        # structural pattern: (i, j) stored iff i, j share an element
        share = np.zeros((m.nq, m.nq), bool)
        for t in tris:
            for a in t:
                for b in t:
                    share[a, b] = True
        if name == "elas":
            share = np.kron(share, np.ones((2, 2), bool))
        stored = np.zeros_like(share)
        for i in range(n):
            stored[i, ci[rp[i]:rp[i + 1]]] = True
            assert np.all(np.diff(ci[rp[i]:rp[i + 1]]) > 0)
        np.testing.assert_array_equal(stored, share)


# ------------------------------------------------------------------ integral identities

@pytest.fixture(scope="module")
def mesh16():
    m = meshgen.square_mesh(16, 11)
    return m, meshgen.vertex_weights(m, 11)


def test_mass_sums_to_area(mesh16):
    m, _ = mesh16
    rp, ci, va = oracle.assemble(oracle.MASS, m.q, m.me)
    assert va.sum() == pytest.approx(1.0, rel=1e-14)


def test_wmass_identities(mesh16):
    m, w = mesh16
    rp1, ci1, va1 = oracle.assemble(oracle.WMASS, m.q, m.me, np.ones(m.nq))
    rp0, ci0, va0 = oracle.assemble(oracle.MASS, m.q, m.me)
    np.testing.assert_array_equal(ci1, ci0)
    np.testing.assert_allclose(va1, va0, rtol=1e-14)
    rp, ci, va = oracle.assemble(oracle.WMASS, m.q, m.me, w)
    x, y = m.q
    me = m.me
    D = (x[me[2]] - x[me[0]]) * (y[me[0]] - y[me[1]]) - (x[me[0]] - x[me[1]]) * (y[me[2]] - y[me[0]])
    expect = np.sum(D / 2 * (w[me[0]] + w[me[1]] + w[me[2]]) / 3)
    assert va.sum() == pytest.approx(expect, rel=1e-13)


def _quad(rp, ci, va, u):
    n = len(rp) - 1
    Au = np.zeros(n)
    for i in range(n):
        Au[i] = np.dot(va[rp[i]:rp[i + 1]], u[ci[rp[i]:rp[i + 1]]])
    return Au


def test_stiffness_identities(mesh16):
    m, _ = mesh16
    rp, ci, va = oracle.assemble(oracle.STIFF, m.q, m.me)
    rowmax = np.array([np.abs(va[rp[i]:rp[i + 1]]).max() for i in range(m.nq)])
    assert np.all(np.abs(_quad(rp, ci, va, np.ones(m.nq))) <= 1e-13 * rowmax)
    dense = oracle.csr_to_dense(rp, ci, va, m.nq)
    np.testing.assert_array_equal(dense, dense.T)
    a, b, c = 0.3, -1.7, 0.6
    u = a + b * m.q[0] + c * m.q[1]
    assert u @ _quad(rp, ci, va, u) == pytest.approx(b * b + c * c, rel=1e-12)
    rpm, cim, vam = oracle.assemble(oracle.MASS, m.q, m.me)
    want = a * a + b * b / 3 + c * c / 3 + a * b + a * c + b * c / 2
    assert u @ _quad(rpm, cim, vam, u) == pytest.approx(want, rel=1e-13)


def test_elasticity_identities():
    m = meshgen.square_mesh(8, 5)
    lam, mu = 1.0, 0.5
    rp, ci, va = oracle.assemble(oracle.ELAS, m.q, m.me, lam=lam, mu=mu)
    x, y = m.q
    n = 2 * m.nq
    scale = np.abs(va).max()
    for rx, ry in ((np.ones_like(x), np.zeros_like(x)), (np.zeros_like(x), np.ones_like(x)),
                   (-y, x)):
        r = np.empty(n)
        r[0::2], r[1::2] = rx, ry
        assert np.abs(_quad(rp, ci, va, r)).max() <= 1e-13 * scale * 20
    b11, b12, b21, b22 = 0.4, -0.3, 0.7, 1.1
    U = np.empty(n)
    U[0::2] = 0.2 + b11 * x + b12 * y
    U[1::2] = -0.1 + b21 * x + b22 * y
    want = (lam + 2 * mu) * (b11 ** 2 + b22 ** 2) + 2 * lam * b11 * b22 + mu * (b12 + b21) ** 2
    assert U @ _quad(rp, ci, va, U) == pytest.approx(want, rel=1e-12)


# ------------------------------------------------------------------ input errors

def test_rejects_bad_elements():
    q = TWO_Q.copy()
    with pytest.raises(oracle.OracleError, match="counter-clockwise"):
        oracle.assemble(oracle.MASS, q, TWO_ME[[0, 2, 1]])
    with pytest.raises(oracle.OracleError, match="range"):
        oracle.assemble(oracle.MASS, q, np.array([[0], [1], [4]], np.int32))
    with pytest.raises(oracle.OracleError, match="repeated"):
        oracle.assemble(oracle.MASS, q, np.array([[0], [1], [1]], np.int32))


def test_row_sampler_matches_full_assembly(mesh16):
    m, w = mesh16
    for kind in (oracle.WMASS, oracle.STIFF, oracle.ELAS):
        rp, ci, va = oracle.assemble(kind, m.q, m.me, w)
        rows = [0, 17, len(rp) - 2]
        for r, (cols, vals) in zip(rows, oracle.csr_row_values(kind, m.q, m.me, rows, w)):
            np.testing.assert_array_equal(cols, ci[rp[r]:rp[r + 1]])
            np.testing.assert_array_equal(vals, va[rp[r]:rp[r + 1]])


def test_sparse_duplicate_order_brute_force():
    """Many duplicate groups of values with wildly different magnitudes: each group's stored
    value must equal a plain left-to-right float loop over the group in input order (any other
    order rounds differently for most groups)."""
    rng = np.random.default_rng(42)
    n_groups, per = 400, 7
    rows = np.repeat(np.arange(n_groups), per)
    vals = rng.choice([-1, 1], rows.size) * 10.0 ** rng.uniform(-8, 8, rows.size)
    order = rng.permutation(rows.size)          # interleave the groups
    I = rows[order].astype(np.int32)
    K = vals[order]
    rp, ci, va = oracle.sparse(I, np.zeros_like(I), K, n_groups, 1)
    for g in range(n_groups):
        s = None
        for t in range(I.size):
            if I[t] == g:
                s = K[t] if s is None else s + K[t]
        assert va[g] == s


# ------------------------------------------------------------------ adjoint

def _loss(m, w, GS, GM, q=None):
    q = m.q if q is None else q
    _, _, s = oracle.assemble(oracle.STIFF, q, m.me)
    _, _, mw = oracle.assemble(oracle.WMASS, q, m.me, w)
    return float(np.dot(GS, s)), float(np.dot(GM, mw))


@pytest.fixture(scope="module")
def adj_case():
    m = meshgen.square_mesh(6, 21)
    w = meshgen.vertex_weights(m, 21)
    rp, ci, _ = oracle.assemble(oracle.STIFF, m.q, m.me)
    GS, GM = meshgen.upstream_gradients(21, len(ci))
    dqS, _ = oracle.adjoint(oracle.STIFF, m.q, m.me, rp, ci, GS)
    dqM, dw = oracle.adjoint(oracle.WMASS, m.q, m.me, rp, ci, GM, w=w)
    return m, w, GS, GM, dqS, dqM, dw


def test_adjoint_central_differences(adj_case):
    m, w, GS, GM, dqS, dqM, dw = adj_case
    h = 1e-6
    dq = dqS + dqM
    for flat in meshgen.sample_indices(5, 40, 2 * m.nq):
        r, i = divmod(int(flat), m.nq)
        qp, qm = m.q.copy(), m.q.copy()
        qp[r, i] += h
        qm[r, i] -= h
        fd = (sum(_loss(m, w, GS, GM, qp)) - sum(_loss(m, w, GS, GM, qm))) / (2 * h)
        assert abs(fd - dq[r, i]) <= 1e-6 * np.abs(dq).max()


def test_adjoint_weights_exact(adj_case):
    """L_M is linear in w, so dL/dw_c is L_M evaluated at the c-th unit vector."""
    m, w, GS, GM, dqS, dqM, dw = adj_case
    for c in (0, 7, m.nq - 1):
        e = np.zeros(m.nq)
        e[c] = 1.0
        _, lm = _loss(m, e, GS, GM)
        assert dw[c] == pytest.approx(lm, rel=1e-13, abs=1e-15)
    assert float(np.dot(w, dw)) == pytest.approx(_loss(m, w, GS, GM)[1], rel=1e-12)


def test_adjoint_invariances(adj_case):
    """S and M^[w] depend on q only through edge vectors (translation invariance) and are
    unchanged by rotations; S is homogeneous of degree 0 in q, M^[w] of degree 2 (Euler)."""
    m, w, GS, GM, dqS, dqM, dw = adj_case
    x, y = m.q
    LS, LM = _loss(m, w, GS, GM)
    for dq, L, deg in ((dqS, LS, 0), (dqM, LM, 2)):
        scale = np.abs(dq).max()
        assert abs(dq[0].sum()) <= 1e-12 * scale * m.nq
        assert abs(dq[1].sum()) <= 1e-12 * scale * m.nq
        assert abs(np.dot(x, dq[1]) - np.dot(y, dq[0])) <= 1e-12 * scale * m.nq
        assert np.dot(x, dq[0]) + np.dot(y, dq[1]) == pytest.approx(deg * L, abs=1e-12 * scale * m.nq)


def test_adjoint_mass(adj_case):
    m, w, GS, GM, *_ = adj_case
    rp, ci, vm = oracle.assemble(oracle.MASS, m.q, m.me)
    dq, _ = oracle.adjoint(oracle.MASS, m.q, m.me, rp, ci, GM)
    h = 1e-6
    for flat in (3, 50, 2 * m.nq - 5):
        r, i = divmod(flat, m.nq)
        qp, qm = m.q.copy(), m.q.copy()
        qp[r, i] += h
        qm[r, i] -= h
        fd = (np.dot(GM, oracle.assemble(oracle.MASS, qp, m.me)[2])
              - np.dot(GM, oracle.assemble(oracle.MASS, qm, m.me)[2])) / (2 * h)
        assert abs(fd - dq[r, i]) <= 1e-7 * np.abs(dq).max()
    L = float(np.dot(GM, vm))
    assert np.dot(m.q[0], dq[0]) + np.dot(m.q[1], dq[1]) == pytest.approx(2 * L, rel=1e-11)
