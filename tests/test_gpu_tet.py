"""Tetrahedral (3-D P1) assembly through the C ABI against the oracle.

row_ptr / col_idx / map are compared bit-exactly; values within 1e-13 of each row's largest |a_ij|;
the gather variant must be bit-identical from run to run. Meshes: jittered, node-permuted cube
meshes (several warps and blocks, ragged tails), stars whose centre belongs to 40 tetrahedra (rows
of 22 and 23 columns: the gather variant's 32-column row sums) or to 80 and 1000 (the long-row
kernels), and the 128^3-cell cube at full size on sampled rows.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
from paper_1305_3122_gb300 import feasm, meshgen
from tests.gpu_common import assert_csr_equal, assert_values_close

pytestmark = pytest.mark.gpu

KINDS = {"mass": (feasm.TET_MASS, oracle.MASS), "wmass": (feasm.TET_WMASS, oracle.WMASS),
         "stiff": (feasm.TET_STIFF, oracle.STIFF)}


def star_mesh(n: int):
    """2n tetrahedra around vertex 0: a ring of n vertices in the plane z = 0 with apexes at z = +-1,
    so vertex 0 has valence 2n and the apexes n."""
    t = np.linspace(0, 2 * np.pi, n, endpoint=False)
    pts = [(0.0, 0.0, 0.0), (0.0, 0.0, 1.0), (0.0, 0.0, -1.0)] + [(np.cos(a), np.sin(a), 0.0) for a in t]
    tets = []
    for j in range(n):
        a, b = 3 + j, 3 + (j + 1) % n
        tets += [(0, a, b, 1), (0, b, a, 2)]
    q = np.array(pts).T.copy()
    me = np.array(tets, dtype=np.int32).T.copy()
    P = q[:, me]
    d = np.einsum("ij,ij->j", P[:, 1] - P[:, 0], np.cross((P[:, 2] - P[:, 0]).T, (P[:, 3] - P[:, 0]).T).T)
    flip = d < 0
    me[2, flip], me[3, flip] = me[3, flip].copy(), me[2, flip].copy()
    return q, me


def _cases():
    out = {}
    for N, seed in ((1, 1), (3, 2), (7, 3), (12, 4)):
        m = meshgen.cube_mesh(N, seed)
        out[f"cube{N}"] = (m.q, m.me)
    out["star20"] = star_mesh(20)      # rows of 22 and 23 columns: the 32-column row sums, no long rows
    out["star40"] = star_mesh(40)
    out["star500"] = star_mesh(500)
    return out


CASES = _cases()


def _weights(q):
    return 1.0 + 0.3 * np.sin(3 * q[0]) * np.cos(2 * q[1]) + 0.1 * q[2]


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("gather", [False, True])
def test_tet_pattern_and_map(case, gather):
    q, me = CASES[case]
    mesh = feasm.TetMesh(q, me)
    pat = feasm.TetPattern(mesh, gather=gather)
    rp_o, ci_o, _ = oracle.tet_assemble(oracle.MASS, q, me)
    assert_csr_equal(pat.row_ptr.cpu(), pat.col_idx.cpu(), rp_o, ci_o)
    mp = pat.map.cpu().numpy()
    rows = np.repeat(np.arange(len(rp_o) - 1), np.diff(rp_o))
    c = np.arange(16 * me.shape[1])
    k, il, jl = c >> 4, (c >> 2) & 3, c & 3
    np.testing.assert_array_equal(rows[mp], me[il, k])
    np.testing.assert_array_equal(ci_o[mp], me[jl, k])


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("kind", sorted(KINDS))
@pytest.mark.parametrize("variant", [feasm.ATOMIC, feasm.GATHER])
def test_tet_values(case, kind, variant):
    q, me = CASES[case]
    w = _weights(q)
    mesh = feasm.TetMesh(q, me)
    pat = feasm.TetPattern(mesh, gather=True)
    kg, ko = KINDS[kind]
    got = feasm.tet_assemble(mesh, pat, kg, torch.tensor(w, device="cuda"), variant)
    rp, ci, va = oracle.tet_assemble(ko, q, me, w)
    assert_values_close(rp, got.cpu().numpy(), va)


@pytest.mark.parametrize("scale,offset", [(1e-9, 0.0), (1e9, 0.0), (1.0, 1000.0)])
def test_tet_scale_and_offset(scale, offset):
    """The double-float dot products work on gradients scaled by a power of two, so a cube shrunk
    to 1e-9, blown up to 1e9 or moved far from the origin still matches the oracle."""
    m = meshgen.cube_mesh(5, 8)
    q = m.q * scale + offset
    w = _weights(m.q)
    mesh = feasm.TetMesh(q, m.me)
    pat = feasm.TetPattern(mesh, gather=True)
    for kg, ko in KINDS.values():
        rp, ci, va = oracle.tet_assemble(ko, q, m.me, w)
        for variant in (feasm.ATOMIC, feasm.GATHER):
            got = feasm.tet_assemble(mesh, pat, kg, torch.tensor(w, device="cuda"), variant)
            assert_values_close(rp, got.cpu().numpy(), va)


def test_tet_gather_bit_identical_runs():
    q, me = CASES["cube12"]
    mesh = feasm.TetMesh(q, me)
    pat = feasm.TetPattern(mesh, gather=True)
    a = feasm.tet_assemble(mesh, pat, feasm.TET_STIFF, None, feasm.GATHER)
    b = feasm.tet_assemble(mesh, pat, feasm.TET_STIFF, None, feasm.GATHER)
    assert torch.equal(a.view(torch.int64), b.view(torch.int64))


def test_tet_drop_zeros_of_unjittered_cube():
    """On the unjittered cube mesh with N a power of two (exact coordinates, so every edge vector,
    cross product and dot product is exact) the stiffness entries between vertices whose gradients
    are orthogonal in every shared tetrahedron are exactly zero on both sides; the zero-dropped
    patterns agree. (With N = 6 whether such an entry rounds to 0.0 depends on the formula.)"""
    m = meshgen.cube_mesh(8, 5, jitter=0.0)
    mesh = feasm.TetMesh(m.q, m.me)
    pat = feasm.TetPattern(mesh, gather=True)
    S = feasm.tet_assemble(mesh, pat, feasm.TET_STIFF, None, feasm.GATHER)
    rpg, cig, vag = feasm.drop_zeros(pat.row_ptr, pat.col_idx, S)
    rpo, cio, vao = oracle.drop_zeros(*oracle.tet_assemble(oracle.STIFF, m.q, m.me))
    assert len(cio) < pat.nnz
    np.testing.assert_array_equal(rpg.cpu().numpy(), rpo)
    np.testing.assert_array_equal(cig.cpu().numpy(), cio)
    assert_values_close(rpo, vag.cpu().numpy(), vao)


def test_tet_errors():
    m = meshgen.cube_mesh(2, 1)
    me = m.me.copy()
    me[2, 5], me[3, 5] = me[3, 5], me[2, 5]
    with pytest.raises(feasm.FeasmError) as e:
        feasm.TetMesh(m.q, me)
    assert e.value.status == 4 and "tetrahedron 5" in str(e.value)
    me = m.me.copy()
    me[1, 3] = me[0, 3]
    with pytest.raises(feasm.FeasmError) as e:
        feasm.TetMesh(m.q, me)
    assert e.value.status == 3
    me = m.me.copy()
    me[0, 2] = m.nq
    with pytest.raises(feasm.FeasmError) as e:
        feasm.TetMesh(m.q, me)
    assert e.value.status == 2
    mesh = feasm.TetMesh(m.q, m.me)
    pat = feasm.TetPattern(mesh, gather=False)
    with pytest.raises(feasm.FeasmError):
        feasm.tet_assemble(mesh, pat, feasm.TET_STIFF, None, feasm.GATHER)      # needs a gather pattern
    with pytest.raises(feasm.FeasmError):
        feasm.tet_assemble(mesh, pat, 7, None, feasm.ATOMIC)                    # unknown kind
    with pytest.raises(feasm.FeasmError) as e:
        feasm.tet_assemble(mesh, pat, feasm.TET_STIFF, None, feasm.ATOMIC,
                           out=torch.empty(pat.nnz - 1, dtype=torch.float64, device="cuda"))
    assert e.value.status == 5
    q, me = star_mesh(600)                                                      # valence 1200 > 1024
    big = feasm.TetMesh(q, me)
    with pytest.raises(feasm.FeasmError) as e:
        feasm.TetPattern(big)
    assert e.value.status == 9


def test_tet_empty_mesh():
    mesh = feasm.TetMesh(np.zeros((3, 5)), np.zeros((4, 0), np.int32))
    pat = feasm.TetPattern(mesh, gather=True)
    assert pat.nnz == 0 and pat.row_ptr.cpu().tolist() == [0] * 6
    v = feasm.tet_assemble(mesh, pat, feasm.TET_STIFF, None, feasm.GATHER)
    assert v.numel() == 0


def _oracle_rows(kind, q, me, rows, w=None):
    out = []
    for r in rows:
        ks = np.nonzero((me == r).any(axis=0))[0]
        I, J, K = oracle.tet_triplets(kind, q, me[:, ks], w)
        sel = I == r
        cols = np.unique(J[sel])
        vals = np.array([K[sel & (J == c)].sum() for c in cols])
        out.append((cols, vals))
    return out


def test_tet_full_size_sampled_rows():
    """128^3 cells (2,146,689 vertices, 12,582,912 tetrahedra), as the benchmark times it: sampled
    rows of S and M^w (both variants) against the oracle."""
    seed = 13053122 + 6
    m = meshgen.cube_mesh(128, seed)
    w = meshgen.vertex_weights3(m, seed)
    mesh = feasm.TetMesh(torch.tensor(m.q, device="cuda"), torch.tensor(m.me, device="cuda"))
    pat = feasm.TetPattern(mesh, gather=True)
    rows = meshgen.sample_indices(seed, 12, m.nq)
    wd = torch.tensor(w, device="cuda")
    rp = pat.row_ptr.cpu().numpy()
    ci = pat.col_idx.cpu().numpy()
    for kg, ko in ((feasm.TET_STIFF, oracle.STIFF), (feasm.TET_WMASS, oracle.WMASS)):
        want = _oracle_rows(ko, m.q, m.me, rows, w)
        for variant in (feasm.ATOMIC, feasm.GATHER):
            got = feasm.tet_assemble(mesh, pat, kg, wd, variant).cpu().numpy()
            for r, (cols, vals) in zip(rows, want):
                np.testing.assert_array_equal(ci[rp[r]:rp[r + 1]], cols)
                g = got[rp[r]:rp[r + 1]]
                assert np.abs(g - vals).max() <= 1e-13 * np.abs(vals).max()
    # every row, both variants: S 1 = 0 (relative to each row's largest entry) and the entries of
    # M sum to the cube's volume, 1 (its boundary nodes are not jittered)
    row_of = torch.repeat_interleave(torch.arange(m.nq, device="cuda"), torch.diff(pat.row_ptr.long()))
    for variant in (feasm.ATOMIC, feasm.GATHER):
        S = feasm.tet_assemble(mesh, pat, feasm.TET_STIFF, None, variant)
        rs = torch.zeros(m.nq, dtype=torch.float64, device="cuda").index_add_(0, row_of, S)
        rmax = torch.zeros(m.nq, dtype=torch.float64, device="cuda").index_reduce_(0, row_of, S.abs(), "amax")
        assert float((rs.abs() / rmax).max()) <= 1e-13
        M = feasm.tet_assemble(mesh, pat, feasm.TET_MASS, None, variant)
        assert abs(float(M.sum()) - 1.0) <= 1e-12
