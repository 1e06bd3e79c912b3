"""P2 (quadratic) triangles through the C ABI against the oracle.

Dof numbering, row_ptr / col_idx and the element map are compared bit-exactly, values within 1e-13
of each row's largest |a_ij| for both variants (FP64 atomics, ordered row sums); the ordered
variant must be bit-identical from run to run. Meshes: jittered node-permuted squares (several
warps and blocks), fans whose centre belongs to 8 triangles (a 25-column vertex row), 12 (37
columns: a long row from the warp pass) and 70 (the long-row pass), five triangles on one edge
(an 18-column edge row), the one- and two-triangle meshes, unstructured squares (random cell
diagonals, a hole, a stretch) and the bow-tie, and the 1024 x 1024-cell square at full size on
sampled rows.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
from paper_1305_3122_gb300 import feasm, meshgen
from tests.gpu_common import assert_csr_equal, assert_values_close
from tests.test_gpu_parity import fan_mesh

pytestmark = pytest.mark.gpu

KINDS = {"mass": (feasm.P2_MASS, oracle.MASS), "stiff": (feasm.P2_STIFF, oracle.STIFF)}
VARIANTS = {"atomic": feasm.ATOMIC, "gather": feasm.GATHER}


def _cases():
    out = {}
    for N, seed in ((1, 1), (5, 2), (37, 3)):
        m = meshgen.square_mesh(N, seed)
        out[f"square{N}"] = (m.q, m.me)
    out["fan8"] = fan_mesh(8)
    out["fan12"] = fan_mesh(12)
    out["fan70"] = fan_mesh(70)
    # five triangles on one edge (0, 1): the edge's dof row has 18 columns (2 + 5 vertices, 1 + 10
    # edges), longer than an edge row's accumulators: the long-row kernel through the big-row pass
    qb = np.array([[0.0, 1.0, 0.5, 0.4, 0.6, 0.5, 0.3], [0.0, 0.0, 1.0, 2.0, 3.0, -1.0, -2.0]])
    meb = np.array([[0, 0, 0, 1, 1], [1, 1, 1, 0, 0], [2, 3, 4, 5, 6]], np.int32)
    out["book5"] = (qb, meb)
    q2 = np.array([[0.0, 1.0, 1.0, 0.0], [0.0, 0.0, 1.0, 1.0]])
    me2 = np.array([[0, 0], [1, 2], [2, 3]], np.int32)
    out["two"] = (q2, me2)
    out["one"] = (q2, me2[:, :1].copy())
    # unstructured: random cell diagonals (vertex rows of 4 to 8 triangles), a hole with unused
    # vertices and a vertex in two fans, a stretched square, and the bow-tie
    m = meshgen.square_mesh(29, 41, random_diagonals=True, hole=True)
    out["rdiag_hole29"] = (m.q, m.me)
    m = meshgen.square_mesh(24, 42, random_diagonals=True, stretch=6.0)
    out["rdiag_stretch24"] = (m.q, m.me)
    out["bowtie"] = (np.array([[0.0, 1.0, 0.0, -1.0, 0.0], [0.0, 0.0, 1.0, 0.0, -1.0]]),
                     np.array([[0, 0], [1, 3], [2, 4]], np.int32))
    return out


CASES = _cases()


def _build(q, me, gather=False):
    mesh = feasm.Mesh(q, me)
    pat = feasm.Pattern(mesh)
    return mesh, feasm.P2Pattern(mesh, pat, gather=gather), pat


@pytest.mark.parametrize("case", sorted(CASES))
def test_p2_dofs_pattern_and_map(case):
    q, me = CASES[case]
    mesh, p2, _ = _build(q, me)
    I, J, K, ndof = oracle.p2_triplets(oracle.MASS, q, me)
    assert p2.n_rows == ndof
    nme = me.shape[1]
    edof = p2.edof.cpu().numpy().reshape(nme, 6)
    np.testing.assert_array_equal(edof, I.reshape(nme, 36)[:, :6])        # c = 36k + il (jl = 0)
    rp, ci, _ = oracle.p2_assemble(oracle.MASS, q, me)
    assert_csr_equal(p2.row_ptr.cpu(), p2.col_idx.cpu(), rp, ci)
    mp = p2.map.cpu().numpy().reshape(nme, 6, 6)
    rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    np.testing.assert_array_equal(rows[mp], edof[:, :, None].repeat(6, axis=2))
    np.testing.assert_array_equal(ci[mp], edof[:, None, :].repeat(6, axis=1))


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("kind", sorted(KINDS))
@pytest.mark.parametrize("variant", sorted(VARIANTS))
def test_p2_values(case, kind, variant):
    q, me = CASES[case]
    v = VARIANTS[variant]
    mesh, p2, _ = _build(q, me, gather=v == feasm.GATHER)
    kg, ko = KINDS[kind]
    got = feasm.p2_assemble(mesh, p2, kg, variant=v)
    rp, ci, va = oracle.p2_assemble(ko, q, me)
    assert_csr_equal(p2.row_ptr.cpu(), p2.col_idx.cpu(), rp, ci)
    assert_values_close(rp, got.cpu().numpy(), va)


@pytest.mark.parametrize("case", ["square37", "fan12", "fan70", "book5"])
def test_p2_gather_bit_identical_runs(case):
    """The ordered variant sums each non-zero in ascending element order: ten runs, one result,
    and both variants' patterns alike."""
    q, me = CASES[case]
    mesh, p2, pat = _build(q, me, gather=True)
    p2a = feasm.P2Pattern(mesh, pat)
    np.testing.assert_array_equal(p2.col_idx.cpu().numpy(), p2a.col_idx.cpu().numpy())
    np.testing.assert_array_equal(p2.map.cpu().numpy(), p2a.map.cpu().numpy())
    for kind in (feasm.P2_MASS, feasm.P2_STIFF):
        first = feasm.p2_assemble(mesh, p2, kind, variant=feasm.GATHER).cpu().numpy()
        for _ in range(9):
            again = feasm.p2_assemble(mesh, p2, kind, variant=feasm.GATHER).cpu().numpy()
            assert np.array_equal(first.view(np.int64), again.view(np.int64))


def test_p2_quadratic_energy():
    """u^T S u = int |grad u|^2 and u^T M u = int u^2 for u = x y, interpolated exactly by P2."""
    m = meshgen.square_mesh(50, 6)
    mesh, p2, _ = _build(m.q, m.me)
    u = torch.tensor(oracle.p2_dof_values(m.q, m.me, lambda x, y: x * y), device="cuda")
    for kind, want in ((feasm.P2_STIFF, 2.0 / 3.0), (feasm.P2_MASS, 1.0 / 9.0)):
        A = torch.sparse_csr_tensor(p2.row_ptr.long(), p2.col_idx.long(), feasm.p2_assemble(mesh, p2, kind),
                                    size=(p2.n_rows, p2.n_rows))
        assert float(u @ (A @ u)) == pytest.approx(want, rel=1e-12)


def test_p2_empty_mesh_and_isolated_vertex():
    """No triangle: the P2 dofs are the vertices alone and every row is empty. A vertex in no
    triangle keeps an empty row next to a meshed one."""
    q = np.zeros((2, 5))
    mesh = feasm.Mesh(q, np.zeros((3, 0), np.int32))
    p2 = feasm.P2Pattern(mesh, feasm.Pattern(mesh), gather=True)
    assert p2.n_rows == 5 and p2.nnz == 0 and p2.n_edges == 0
    assert p2.row_ptr.cpu().tolist() == [0] * 6
    assert feasm.p2_assemble(mesh, p2, feasm.P2_STIFF).numel() == 0
    assert feasm.p2_assemble(mesh, p2, feasm.P2_STIFF, variant=feasm.GATHER).numel() == 0
    q = np.array([[0.0, 1.0, 0.0, 5.0], [0.0, 0.0, 1.0, 5.0]])           # vertex 3 in no triangle
    me = np.array([[0], [1], [2]], np.int32)
    mesh = feasm.Mesh(q, me)
    p2 = feasm.P2Pattern(mesh, feasm.Pattern(mesh), gather=True)
    rp, ci, va = oracle.p2_assemble(oracle.STIFF, q, me)
    assert_csr_equal(p2.row_ptr.cpu(), p2.col_idx.cpu(), rp, ci)
    assert rp[4] - rp[3] == 0
    for v in (feasm.ATOMIC, feasm.GATHER):
        assert_values_close(rp, feasm.p2_assemble(mesh, p2, feasm.P2_STIFF, variant=v).cpu().numpy(), va)


def test_p2_errors():
    m = meshgen.square_mesh(4, 1)
    mesh, p2, pat = _build(m.q, m.me)
    other = feasm.Mesh(m.q, m.me)
    with pytest.raises(feasm.FeasmError):
        feasm.P2Pattern(other, pat)                       # pattern of another mesh
    with pytest.raises(feasm.FeasmError):
        feasm.p2_assemble(other, p2, feasm.P2_STIFF)
    with pytest.raises(feasm.FeasmError):
        feasm.p2_assemble(mesh, p2, 9)
    with pytest.raises(feasm.FeasmError) as e:
        feasm.p2_assemble(mesh, p2, feasm.P2_MASS, out=torch.empty(p2.nnz - 1, dtype=torch.float64, device="cuda"))
    assert e.value.status == 5
    pat2 = feasm.Pattern(mesh, dofs=2, map=False)
    with pytest.raises(feasm.FeasmError):
        feasm.P2Pattern(mesh, pat2)                       # needs the scalar pattern
    with pytest.raises(feasm.FeasmError):
        feasm.p2_assemble(mesh, p2, feasm.P2_STIFF, variant=feasm.GATHER)    # pattern without the row lists
    with pytest.raises(feasm.FeasmError):
        feasm.p2_assemble(mesh, p2, feasm.P2_STIFF, variant=feasm.ROW)       # no row-owner P2 kernel


def test_p2_full_size_sampled_rows():
    """1024 x 1024 cells (1,050,625 vertices, 3,147,776 edges, 2,097,152 triangles): sampled vertex
    and edge rows of M and S against the oracle's triplets."""
    seed = 13053122 + 7
    m = meshgen.square_mesh(1024, seed)
    mesh = feasm.Mesh(torch.tensor(m.q, device="cuda"), torch.tensor(m.me, device="cuda"))
    pat = feasm.Pattern(mesh, map=False)
    p2 = feasm.P2Pattern(mesh, pat, gather=True)
    assert p2.n_rows == m.nq + 3 * 1024 * 1024 + 2 * 1024
    rows = np.concatenate([meshgen.sample_indices(seed, 6, m.nq), m.nq + meshgen.sample_indices(seed + 1, 6, p2.n_edges)])
    rp = p2.row_ptr.cpu().numpy()
    ci = p2.col_idx.cpu().numpy()
    for kg, ko in KINDS.values():
        want = oracle.p2_row_values(ko, m.q, m.me, rows)
        for v in (feasm.ATOMIC, feasm.GATHER):
            got = feasm.p2_assemble(mesh, p2, kg, variant=v).cpu().numpy()
            for r, (cols, vals) in zip(rows, want):
                np.testing.assert_array_equal(ci[rp[r]:rp[r + 1]], cols)
                assert np.abs(got[rp[r]:rp[r + 1]] - vals).max() <= 1e-13 * np.abs(vals).max()
    # every row, both variants: S 1 = 0 (relative to each row's largest entry) and the entries of
    # M sum to the square's area, 1 (the P2 functions sum to one; the boundary is not jittered)
    row_of = torch.repeat_interleave(torch.arange(p2.n_rows, device="cuda"), torch.diff(p2.row_ptr.long()))
    for v in (feasm.ATOMIC, feasm.GATHER):
        S = feasm.p2_assemble(mesh, p2, feasm.P2_STIFF, variant=v)
        rs = torch.zeros(p2.n_rows, dtype=torch.float64, device="cuda").index_add_(0, row_of, S)
        rmax = torch.zeros(p2.n_rows, dtype=torch.float64, device="cuda").index_reduce_(0, row_of, S.abs(), "amax")
        assert float((rs.abs() / rmax).max()) <= 1e-13
        M = feasm.p2_assemble(mesh, p2, feasm.P2_MASS, variant=v)
        assert abs(float(M.sum()) - 1.0) <= 1e-12
