"""3-D linear elasticity on tetrahedra through the C ABI against the oracle.

The structure (rows 3i + s) is compared bit-exactly; values within 1e-13 of each row's largest
|a_ij|, for both variants (FP64 atomics; staged element matrices summed row by row in ascending
element order, which must be bit-identical from run to run). Meshes: jittered node-permuted cubes
(one cell, several warps and blocks, ragged tails), stars whose centre belongs to 40 tetrahedra
(scalar rows of 22 and 23 columns: the 32-column row sums), 80 and 1000 (the warp-per-row kernel),
several Lame pairs (negative lambda, nearly incompressible), and the 64^3-cell cube at full size on
sampled rows and on identities every row obeys.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1305_3122_gb300 import feasm, meshgen
from tests.gpu_common import assert_csr_equal, assert_values_close
from tests.test_gpu_tet import star_mesh

pytestmark = pytest.mark.gpu

VARIANTS = {"atomic": feasm.ATOMIC, "gather": feasm.GATHER}
LAM, MU = 1.25, 0.4


def _cases():
    out = {}
    for N, seed in ((1, 31), (3, 32), (6, 33)):
        m = meshgen.cube_mesh(N, seed)
        out[f"cube{N}"] = (m.q, m.me)
    out["star20"] = star_mesh(20)
    out["star40"] = star_mesh(40)
    out["star500"] = star_mesh(500)
    return out


CASES = _cases()


def _build(q, me, gather=True):
    mesh = feasm.TetMesh(q, me)
    return mesh, feasm.TetPattern(mesh, gather=gather, elas=True)


@pytest.mark.parametrize("case", sorted(CASES))
def test_elas_structure(case):
    q, me = CASES[case]
    _, pat = _build(q, me)
    rp, ci, _ = oracle.tet_elas_assemble(q, me, LAM, MU)
    assert pat.elas_n_rows == 3 * q.shape[1] and pat.elas_nnz == len(ci) == 9 * pat.nnz
    assert_csr_equal(pat.elas_row_ptr.cpu(), pat.elas_col_idx.cpu(), rp, ci)


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("variant", sorted(VARIANTS))
def test_elas_values(case, variant):
    q, me = CASES[case]
    mesh, pat = _build(q, me)
    got = feasm.tet_assemble_elas(mesh, pat, LAM, MU, VARIANTS[variant])
    rp, ci, va = oracle.tet_elas_assemble(q, me, LAM, MU)
    assert_values_close(rp, got.cpu().numpy(), va)


@pytest.mark.parametrize("lam,mu", [(-0.5, 1.0), (1000.0, 1.0), (0.0, 3.0), (2.0, 1e-3)])
@pytest.mark.parametrize("variant", sorted(VARIANTS))
def test_elas_lame_parameters(lam, mu, variant):
    q, me = CASES["cube3"]
    mesh, pat = _build(q, me)
    got = feasm.tet_assemble_elas(mesh, pat, lam, mu, VARIANTS[variant])
    rp, ci, va = oracle.tet_elas_assemble(q, me, lam, mu)
    assert_values_close(rp, got.cpu().numpy(), va)


@pytest.mark.parametrize("case", ["cube6", "star40", "star500"])
def test_elas_gather_bit_identical_runs(case):
    q, me = CASES[case]
    mesh, pat = _build(q, me)
    first = feasm.tet_assemble_elas(mesh, pat, LAM, MU, feasm.GATHER).cpu().numpy().view(np.int64)
    for _ in range(5):
        cur = feasm.tet_assemble_elas(mesh, pat, LAM, MU, feasm.GATHER).cpu().numpy().view(np.int64)
        np.testing.assert_array_equal(cur, first)


def test_elas_errors():
    q, me = CASES["cube3"]
    mesh, pat = _build(q, me, gather=False)
    plain = feasm.TetPattern(mesh)
    with pytest.raises(ValueError):
        feasm.tet_assemble_elas(mesh, plain, LAM, MU)                           # no elasticity structure
    out = torch.empty(pat.elas_nnz, dtype=torch.float64, device="cuda")
    L = feasm.lib()
    st = L.fe_tet_assemble_elas(mesh.handle, plain.handle, LAM, MU, feasm.ATOMIC, out.data_ptr(), out.numel(), None)
    assert st == 1 and b"FE_TET_PATTERN_ELAS" in L.fe_last_error()
    for lam, mu in ((1.0, 0.0), (-1.0, 1.0), (float("nan"), 1.0), (1.0, float("inf")), (1.0, -1.0)):
        with pytest.raises(feasm.FeasmError) as e:
            feasm.tet_assemble_elas(mesh, pat, lam, mu)
        assert e.value.status == 1
    with pytest.raises(feasm.FeasmError) as e:
        feasm.tet_assemble_elas(mesh, pat, LAM, MU, feasm.GATHER)               # built without the lists
    assert e.value.status == 1
    with pytest.raises(feasm.FeasmError) as e:
        feasm.tet_assemble_elas(mesh, pat, LAM, MU, feasm.ROW)
    assert e.value.status == 1
    with pytest.raises(feasm.FeasmError) as e:
        feasm.tet_assemble_elas(mesh, pat, LAM, MU, out=torch.empty(pat.elas_nnz - 1, dtype=torch.float64, device="cuda"))
    assert e.value.status == 5
    other = feasm.TetMesh(*CASES["cube1"])
    with pytest.raises(feasm.FeasmError) as e:
        feasm.tet_assemble_elas(other, pat, LAM, MU)
    assert e.value.status == 1
    n, z, rp, ci = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_void_p(), ctypes.c_void_p()
    assert L.fe_tet_pattern_elas_info(plain.handle, ctypes.byref(n), ctypes.byref(z), ctypes.byref(rp), ctypes.byref(ci)) == 1


def test_elas_empty_mesh():
    q = np.zeros((3, 5))
    mesh = feasm.TetMesh(q, np.zeros((4, 0), np.int32))
    pat = feasm.TetPattern(mesh, gather=True, elas=True)
    assert pat.elas_n_rows == 15 and pat.elas_nnz == 0
    assert pat.elas_row_ptr.cpu().tolist() == [0] * 16
    for v in VARIANTS.values():
        assert feasm.tet_assemble_elas(mesh, pat, LAM, MU, v).numel() == 0


def test_elas_full_size_64():
    """64^3 cells (274,625 vertices, 1,572,864 tetrahedra, 37 M non-zeros), as the benchmark times it:
    sampled rows against the oracle, and on every row, both variants: the six rigid modes in the
    kernel, the block traces equal to (lambda + 4 mu) S, and the energy of a linear displacement."""
    seed = 13053122 + 9
    m = meshgen.cube_mesh(64, seed)
    mesh = feasm.TetMesh(torch.tensor(m.q, device="cuda"), torch.tensor(m.me, device="cuda"))
    pat = feasm.TetPattern(mesh, gather=True, elas=True)
    rp3 = pat.elas_row_ptr.cpu().numpy()
    ci3 = pat.elas_col_idx.cpu().numpy()
    rows = sorted(set([0, 1, 2, 3 * m.nq - 1] + [int(r) for r in meshgen.sample_indices(seed, 12, 3 * m.nq)]))
    want = oracle.tet_elas_row_values(m.q, m.me, LAM, MU, rows)
    S = feasm.tet_assemble(mesh, pat, feasm.TET_STIFF, None, feasm.GATHER)
    n3 = 3 * m.nq
    P = torch.tensor(m.q.T, device="cuda")
    rng = np.random.default_rng(5)
    Amat = rng.normal(size=(3, 3))
    u = (P @ torch.tensor(Amat.T, device="cuda") + torch.tensor(rng.normal(size=3), device="cuda")).reshape(-1)
    sym = (Amat + Amat.T) / 2
    energy = LAM * np.trace(Amat) ** 2 + 2 * MU * (sym * sym).sum()
    # positions of the block diagonals: scalar entry p of row i (place o) -> 9 rp_i + 3 s len_i + 3 o + s
    rps = pat.row_ptr.long()
    row_of = torch.repeat_interleave(torch.arange(m.nq, device="cuda"), torch.diff(rps))
    place = torch.arange(pat.nnz, device="cuda") - rps[row_of]
    ln = torch.diff(rps)[row_of]
    row3 = torch.repeat_interleave(torch.arange(n3, device="cuda"), torch.diff(pat.elas_row_ptr.long()))
    for variant in VARIANTS.values():
        K = feasm.tet_assemble_elas(mesh, pat, LAM, MU, variant)
        Kh = K.cpu().numpy()
        for r, (cols, vals) in zip(rows, want):
            np.testing.assert_array_equal(ci3[rp3[r]:rp3[r + 1]], cols)
            assert np.abs(Kh[rp3[r]:rp3[r + 1]] - vals).max() <= 1e-13 * np.abs(vals).max()
        A = torch.sparse_csr_tensor(pat.elas_row_ptr.long(), pat.elas_col_idx.long(), K, size=(n3, n3))
        rmax = torch.zeros(n3, dtype=torch.float64, device="cuda").index_reduce_(0, row3, K.abs(), "amax")
        for d in range(3):
            t = torch.zeros(n3, dtype=torch.float64, device="cuda")
            t[d::3] = 1.0
            assert float(((A @ t).abs() / rmax).max()) <= 1e-12
            w = torch.zeros(3, dtype=torch.float64, device="cuda")
            w[d] = 1.0
            rot = torch.linalg.cross(w.expand_as(P), P).reshape(-1)
            assert float(((A @ rot).abs() / rmax).max()) <= 1e-12
        tr = sum(K[9 * rps[row_of] + 3 * s * ln + 3 * place + s] for s in range(3))
        rmax_s = rmax[3 * row_of]
        assert float(((tr - (LAM + 4 * MU) * S).abs() / rmax_s).max()) <= 1e-12
        assert float(u @ (A @ u)) == pytest.approx(energy, rel=1e-11)
