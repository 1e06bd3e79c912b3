"""P3 (cubic) triangles through the C ABI against the oracle.

Dof numbering, row_ptr / col_idx and the element map are compared bit-exactly, values within 1e-13
of each row's largest |a_ij| for both variants (FP64 atomics, ordered row sums); the ordered variant
must be bit-identical from run to run. Meshes: jittered node-permuted squares (one cell, several
warps and blocks), fans whose centre belongs to 8 triangles, 12 (the last fast row) and 13 or 70
(rows of the long-row passes), five triangles on one edge, the one- and two-triangle meshes,
unstructured squares (random diagonals, a hole, a stretch), the bow-tie, and the 512 x 512-cell
square at full size on sampled rows and identities.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
from paper_1305_3122_gb300 import feasm, meshgen
from tests.gpu_common import assert_csr_equal, assert_values_close
from tests.test_gpu_parity import bowtie_mesh, fan_mesh

pytestmark = pytest.mark.gpu

KINDS = {"mass": (feasm.P3_MASS, oracle.MASS), "stiff": (feasm.P3_STIFF, oracle.STIFF)}
VARIANTS = {"atomic": feasm.ATOMIC, "gather": feasm.GATHER}


def _cases():
    out = {}
    for N, seed in ((1, 1), (5, 2), (23, 3)):
        m = meshgen.square_mesh(N, seed)
        out[f"square{N}"] = (m.q, m.me)
    for n in (8, 12, 13, 70):
        out[f"fan{n}"] = fan_mesh(n)
    qb = np.array([[0.0, 1.0, 0.5, 0.4, 0.6, 0.5, 0.3], [0.0, 0.0, 1.0, 2.0, 3.0, -1.0, -2.0]])
    meb = np.array([[0, 0, 0, 1, 1], [1, 1, 1, 0, 0], [2, 3, 4, 5, 6]], np.int32)
    out["book5"] = (qb, meb)
    q2 = np.array([[0.0, 1.0, 1.0, 0.0], [0.0, 0.0, 1.0, 1.0]])
    me2 = np.array([[0, 0], [1, 2], [2, 3]], np.int32)
    out["two"] = (q2, me2)
    out["one"] = (q2, me2[:, :1].copy())
    m = meshgen.square_mesh(21, 51, random_diagonals=True, hole=True)
    out["rdiag_hole21"] = (m.q, m.me)
    m = meshgen.square_mesh(16, 52, random_diagonals=True, stretch=6.0)
    out["rdiag_stretch16"] = (m.q, m.me)
    out["bowtie"] = bowtie_mesh()
    return out


CASES = _cases()


def _build(q, me, gather=False):
    mesh = feasm.Mesh(q, me)
    pat = feasm.Pattern(mesh)
    return mesh, feasm.P3Pattern(mesh, pat, gather=gather), pat


@pytest.mark.parametrize("case", sorted(CASES))
def test_p3_dofs_pattern_and_map(case):
    q, me = CASES[case]
    mesh, p3, _ = _build(q, me)
    I, J, K, ndof = oracle.p3_triplets(oracle.MASS, q, me)
    assert p3.n_rows == ndof
    nme = me.shape[1]
    edof = p3.edof.cpu().numpy().reshape(nme, 10)
    np.testing.assert_array_equal(edof, I.reshape(nme, 100)[:, :10])      # c = 100k + il (jl = 0)
    rp, ci, _ = oracle.p3_assemble(oracle.MASS, q, me)
    assert_csr_equal(p3.row_ptr.cpu(), p3.col_idx.cpu(), rp, ci)
    mp = p3.map.cpu().numpy().reshape(nme, 10, 10)
    rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    np.testing.assert_array_equal(rows[mp], edof[:, :, None].repeat(10, axis=2))
    np.testing.assert_array_equal(ci[mp], edof[:, None, :].repeat(10, axis=1))


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("kind", sorted(KINDS))
@pytest.mark.parametrize("variant", sorted(VARIANTS))
def test_p3_values(case, kind, variant):
    q, me = CASES[case]
    v = VARIANTS[variant]
    mesh, p3, _ = _build(q, me, gather=v == feasm.GATHER)
    kg, ko = KINDS[kind]
    got = feasm.p3_assemble(mesh, p3, kg, variant=v)
    rp, ci, va = oracle.p3_assemble(ko, q, me)
    assert_csr_equal(p3.row_ptr.cpu(), p3.col_idx.cpu(), rp, ci)
    assert_values_close(rp, got.cpu().numpy(), va)


@pytest.mark.parametrize("case", ["square23", "fan13", "fan70", "rdiag_hole21"])
def test_p3_gather_bit_identical_runs(case):
    q, me = CASES[case]
    mesh, p3, _ = _build(q, me, gather=True)
    first = None
    for _ in range(10):
        cur = feasm.p3_assemble(mesh, p3, feasm.P3_STIFF, variant=feasm.GATHER).cpu().numpy().view(np.int64)
        first = cur if first is None else first
        np.testing.assert_array_equal(cur, first)


def test_p3_cubic_energies():
    """P3 interpolation is exact for cubics: u'Su = int |grad u|^2 and u'Mu = int u^2."""
    m = meshgen.square_mesh(24, 9, random_diagonals=True)
    mesh, p3, _ = _build(m.q, m.me, gather=True)
    X, Y = (torch.tensor(a, device="cuda") for a in oracle.p3_dof_points(m.q, m.me))
    for v in (feasm.ATOMIC, feasm.GATHER):
        Sv = feasm.p3_assemble(mesh, p3, feasm.P3_STIFF, variant=v)
        Mv = feasm.p3_assemble(mesh, p3, feasm.P3_MASS, variant=v)
        A = torch.sparse_csr_tensor(p3.row_ptr.long(), p3.col_idx.long(), Sv, size=(p3.n_rows, p3.n_rows))
        B = torch.sparse_csr_tensor(p3.row_ptr.long(), p3.col_idx.long(), Mv, size=(p3.n_rows, p3.n_rows))
        u = X * Y * Y
        assert float(u @ (A @ u)) == pytest.approx(1.0 / 5.0 + 4.0 / 9.0, rel=1e-11)
        w = X ** 3
        assert float(w @ (B @ w)) == pytest.approx(1.0 / 7.0, rel=1e-11)
        assert float((A @ torch.ones_like(X)).abs().max()) <= 1e-10


def test_p3_full_size_sampled_rows():
    """512 x 512 cells (0.52 M triangles, 2.4 M dofs): sampled vertex, edge and bubble rows against
    the oracle, and on every row S 1 = 0 and the mass total 1, both variants."""
    m = meshgen.square_mesh(512, meshgen.SEED_BASE + 8)
    mesh, p3, _ = _build(m.q, m.me, gather=True)
    rp = p3.row_ptr.cpu().numpy()
    ci = p3.col_idx.cpu().numpy()
    ne = p3.n_edges
    assert p3.n_rows == m.nq + 2 * ne + m.nme
    rows = sorted(set([0, m.nq - 1, m.nq, m.nq + 2 * ne - 1, m.nq + 2 * ne, p3.n_rows - 1] +
                      [int(r) for r in meshgen.sample_indices(11, 24, p3.n_rows)]))
    for v in (feasm.ATOMIC, feasm.GATHER):
        S = feasm.p3_assemble(mesh, p3, feasm.P3_STIFF, variant=v)
        M = feasm.p3_assemble(mesh, p3, feasm.P3_MASS, variant=v)
        vs = S.cpu().numpy()
        for r, (cols, vals) in zip(rows, oracle.p3_row_values(oracle.STIFF, m.q, m.me, rows)):
            np.testing.assert_array_equal(ci[rp[r]:rp[r + 1]], cols)
            assert np.abs(vs[rp[r]:rp[r + 1]] - vals).max() <= 1e-13 * np.abs(vals).max()
        rows_t = torch.repeat_interleave(torch.arange(p3.n_rows, device="cuda"), torch.diff(p3.row_ptr.long()))
        rs = torch.zeros(p3.n_rows, dtype=torch.float64, device="cuda").index_add_(0, rows_t, S)
        rmax = torch.zeros(p3.n_rows, dtype=torch.float64, device="cuda").index_reduce_(0, rows_t, S.abs(), "amax")
        assert bool((rs.abs() <= 32 * 1e-13 * rmax).all())
        assert float(M.sum()) == pytest.approx(1.0, rel=1e-12)


def test_p3_errors():
    q, me = CASES["square5"]
    mesh, p3, pat = _build(q, me)
    with pytest.raises(feasm.FeasmError) as e:
        feasm.p3_assemble(mesh, p3, feasm.P3_STIFF, variant=feasm.GATHER)       # built without the lists
    assert e.value.status == 1
    with pytest.raises(feasm.FeasmError) as e:
        feasm.p3_assemble(mesh, p3, feasm.P3_STIFF, variant=feasm.ROW)
    assert e.value.status == 1
    with pytest.raises(feasm.FeasmError) as e:
        feasm.p3_assemble(mesh, p3, feasm.P3_STIFF, out=torch.empty(3, dtype=torch.float64, device="cuda"))
    assert e.value.status == 5
    with pytest.raises(feasm.FeasmError) as e:
        feasm.P3Pattern(mesh, feasm.Pattern(mesh, rows=(0, 10)))                # a row window
    assert e.value.status == 1
    qf, mef = fan_mesh(401, ring2=False)                                       # a vertex in 401 triangles
    mf = feasm.Mesh(qf, mef)
    with pytest.raises(feasm.FeasmError) as e:
        feasm.P3Pattern(mf, feasm.Pattern(mf))
    assert e.value.status == 9 and b"FE_P3_MAX_VALENCE" in feasm.lib().fe_last_error()
    empty = feasm.Mesh(np.zeros((2, 3)), np.zeros((3, 0), np.int32))
    pe = feasm.P3Pattern(empty, feasm.Pattern(empty))
    assert pe.n_rows == 3 and pe.nnz == 0
    assert feasm.p3_assemble(empty, pe, feasm.P3_MASS).numel() == 0
