"""Helpers for the GPU parity tests: CSR comparison at the tolerance the parity bar states."""
from __future__ import annotations

import numpy as np

# values agree within this fraction of the largest |a_ij| of their row (FP64 assembly)
ROW_TOL = 1e-13


def row_max(rp: np.ndarray, va: np.ndarray) -> np.ndarray:
    n = len(rp) - 1
    out = np.zeros(n)
    nz = np.diff(rp) > 0
    out[nz] = np.maximum.reduceat(np.abs(va), rp[:-1][nz])
    return out


def assert_values_close(rp: np.ndarray, got: np.ndarray, want: np.ndarray, tol: float = ROW_TOL):
    """|got - want| <= tol * max_j |want_ij| in every row i."""
    assert got.shape == want.shape
    rm = row_max(rp, want)
    rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    err = np.abs(got - want)
    bad = err > tol * rm[rows]
    if bad.any():
        i = int(np.argmax(err / np.maximum(rm[rows], 1e-300)))
        raise AssertionError(f"{int(bad.sum())} values off; worst at {i} (row {rows[i]}): got {got[i]!r} "
                             f"want {want[i]!r} rowmax {rm[rows[i]]!r}")


def assert_csr_equal(rp_g, ci_g, rp_o, ci_o):
    np.testing.assert_array_equal(np.asarray(rp_g), np.asarray(rp_o))
    np.testing.assert_array_equal(np.asarray(ci_g), np.asarray(ci_o))
