"""fe_csr_drop_zeros (Matlab's sparse() stores no zero, Section 5) against the oracle.

The compaction is exact work: row_ptr, col_idx and the value bits must equal the oracle's for the
same input. On the unjittered power-of-two mesh the assembled S is exactly zero on the cell
diagonals on both sides, so the dropped patterns must agree too.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1305_3122_gb300 import feasm, meshgen
from tests.gpu_common import assert_values_close

pytestmark = pytest.mark.gpu


def _rand_csr(rng, n_rows, max_len, zero_frac):
    lens = rng.integers(0, max_len + 1, n_rows) * (rng.random(n_rows) > 0.15)
    rp = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    nnz = int(rp[-1])
    ci = rng.integers(0, 1 << 20, nnz).astype(np.int32)
    va = rng.standard_normal(nnz) * (rng.random(nnz) > zero_frac)
    if nnz:
        sel = rng.integers(0, nnz, max(nnz // 50, 1))
        va[sel[0::4]] = -0.0
        va[sel[1::4]] = np.nan
        va[sel[2::4]] = 5e-324
    return rp, ci, va


def _gpu(rp, ci, va):
    return feasm.drop_zeros(torch.tensor(rp, device="cuda"), torch.tensor(ci, device="cuda"),
                            torch.tensor(va, device="cuda"))


def _same_bits(a: np.ndarray, b: np.ndarray):
    assert a.shape == b.shape
    np.testing.assert_array_equal(a.view(np.int64), b.view(np.int64))


@pytest.mark.parametrize("n_rows,max_len,zero_frac", [(0, 5, 0.3), (1, 3, 0.5), (33, 7, 0.3), (1000, 9, 0.3),
                                                      (4097, 80, 0.5), (20000, 7, 0.0), (5000, 7, 1.0),
                                                      (300, 3000, 0.3)])
def test_drop_zeros_matches_oracle(n_rows, max_len, zero_frac):
    rng = np.random.default_rng(n_rows + max_len)
    rp, ci, va = _rand_csr(rng, n_rows, max_len, zero_frac)
    rpg, cig, vag = _gpu(rp, ci, va)
    rpo, cio, vao = oracle.drop_zeros(rp, ci, va)
    np.testing.assert_array_equal(rpg.cpu().numpy(), rpo)
    np.testing.assert_array_equal(cig.cpu().numpy(), cio)
    _same_bits(vag.cpu().numpy(), vao)


@pytest.mark.parametrize("variant", [feasm.ROW, feasm.ATOMIC, feasm.GATHER])
def test_drop_zeros_of_assembled_stiffness(variant):
    """Unjittered 64 x 64 mesh (exact coordinates): S is exactly 0 on the 2 * 64^2 cell-diagonal
    entries on both sides; the dropped patterns are equal and the values within the tolerance."""
    m = meshgen.square_mesh(64, 11, jitter=0.0)
    mesh = feasm.Mesh(m.q, m.me)
    pat = feasm.Pattern(mesh, gather=True)
    S = feasm.assemble_stiff(mesh, pat, variant)
    rpg, cig, vag = feasm.drop_zeros(pat.row_ptr, pat.col_idx, S)
    rpo, cio, vao = oracle.drop_zeros(*oracle.assemble(oracle.STIFF, m.q, m.me))
    assert pat.nnz - cig.numel() == 2 * 64 * 64
    np.testing.assert_array_equal(rpg.cpu().numpy(), rpo)
    np.testing.assert_array_equal(cig.cpu().numpy(), cio)
    assert_values_close(rpo, vag.cpu().numpy(), vao)


def test_drop_zeros_full_size_property():
    """2048 x 2048-cell jittered mesh (the size the benchmark times): the kept entries are exactly
    values[values != 0] in order, and each row keeps its non-zero count."""
    m = meshgen.square_mesh(2048, 13053122 + 2)
    mesh = feasm.Mesh(torch.tensor(m.q, device="cuda"), torch.tensor(m.me, device="cuda"))
    pat = feasm.Pattern(mesh, map=False)
    S = feasm.assemble_stiff(mesh, pat, feasm.ROW)
    S[::7] = 0.0                       # zeros at many positions, so rows lose entries
    rpg, cig, vag = feasm.drop_zeros(pat.row_ptr, pat.col_idx, S)
    keep = S != 0
    assert torch.equal(vag, S[keep]) and torch.equal(cig, pat.col_idx[keep])
    per_row = torch.zeros(pat.n_rows, dtype=torch.int64, device="cuda")
    rows = torch.repeat_interleave(torch.arange(pat.n_rows, device="cuda"), torch.diff(pat.row_ptr.long()))
    per_row.index_add_(0, rows, keep.long())
    assert torch.equal(torch.diff(rpg.long()), per_row)


def test_drop_zeros_errors():
    rp = torch.tensor([0, 2, 3], dtype=torch.int32, device="cuda")
    ci = torch.tensor([0, 1, 1], dtype=torch.int32, device="cuda")
    va = torch.tensor([1.0, 0.0, 2.0], dtype=torch.float64, device="cuda")
    L = feasm.lib()
    out_rp = torch.empty(3, dtype=torch.int32, device="cuda")
    out_ci = torch.empty(1, dtype=torch.int32, device="cuda")
    out_va = torch.empty(1, dtype=torch.float64, device="cuda")
    kept = ctypes.c_int64(-1)
    s = torch.cuda.current_stream().cuda_stream
    st = L.fe_csr_drop_zeros(2, rp.data_ptr(), ci.data_ptr(), va.data_ptr(), out_rp.data_ptr(), out_ci.data_ptr(),
                             out_va.data_ptr(), 1, ctypes.byref(kept), s)
    assert st == 5 and kept.value == 2                      # FE_ERR_BUFFER_TOO_SMALL, count reported
    assert out_rp.cpu().tolist() == [0, 1, 2]
    st = L.fe_csr_drop_zeros(2, rp.data_ptr(), ci.data_ptr(), va.data_ptr(), rp.data_ptr(), out_ci.data_ptr(),
                             out_va.data_ptr(), 3, ctypes.byref(kept), s)
    assert st == 1                                          # outputs overlap the inputs
    st = L.fe_csr_drop_zeros(-1, rp.data_ptr(), ci.data_ptr(), va.data_ptr(), out_rp.data_ptr(), out_ci.data_ptr(),
                             out_va.data_ptr(), 3, ctypes.byref(kept), s)
    assert st == 1
    rp0, ci0, va0 = feasm.drop_zeros(torch.zeros(1, dtype=torch.int32, device="cuda"),
                                     torch.empty(0, dtype=torch.int32, device="cuda"),
                                     torch.empty(0, dtype=torch.float64, device="cuda"))
    assert rp0.cpu().tolist() == [0] and ci0.numel() == 0 and va0.numel() == 0
