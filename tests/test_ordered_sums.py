"""The summation order of the ordered (deterministic) variants, checked on the CPU.

The tetrahedral and P2 ordered variants sum each row's incidences in ascending element order into
accumulators that start at -0.0. The paper's sparse() order is per non-zero, its contributions in
ascending contribution index c. Two facts make the row form give the same sums bit for bit:
- each element contributes at most once to a non-zero, so ascending element order is ascending c
  for every non-zero;
- -0.0 + x == x for every x, -0.0 and +0.0 included, so the -0.0 start changes nothing.
This test builds the row lists the way the kernels do: each row's incidences sorted by key, the
column positions from the row's sorted columns. It sums by rows as the kernels do and by
non-zeros as the definition says, with random values that include signed zeros, and compares
the bits.
"""
from __future__ import annotations

import numpy as np

from paper_1305_3122_gb300 import meshgen


def _row_form(me: np.ndarray, nq: int, vals: np.ndarray, nv: int):
    """Per-row sums over incidences (key nv*k + a) in ascending key, accumulators from -0.0."""
    nme = me.shape[1]
    rows = [[] for _ in range(nq)]
    for k in range(nme):
        for a in range(nv):
            rows[me[a, k]].append(nv * k + a)
    out = {}
    for i in range(nq):
        if not rows[i]:
            continue
        cols = sorted({int(me[jl, key // nv]) for key in rows[i] for jl in range(nv)})
        pos = {c: p for p, c in enumerate(cols)}
        acc = [-0.0] * len(cols)
        for key in sorted(rows[i]):                       # ascending element order
            k, a = divmod(key, nv)
            for jl in range(nv):
                acc[pos[int(me[jl, k])]] += vals[nv * nv * k + nv * a + jl]
        for c, v in zip(cols, acc):
            out[(i, c)] = v
    return out


def _nnz_form(me: np.ndarray, vals: np.ndarray, nv: int):
    """Per non-zero, its contributions in ascending c = nv^2 k + nv il + jl, the first taken as is."""
    out = {}
    for c in range(vals.size):
        k, r = divmod(c, nv * nv)
        il, jl = divmod(r, nv)
        key = (int(me[il, k]), int(me[jl, k]))
        out[key] = vals[c] if key not in out else out[key] + vals[c]
    return out


def _same_bits(x: dict, y: dict) -> bool:
    if x.keys() != y.keys():
        return False
    a = np.array([x[k] for k in sorted(x)])
    b = np.array([y[k] for k in sorted(x)])
    return np.array_equal(a.view(np.int64), b.view(np.int64))


def _values(rng, n):
    v = rng.standard_normal(n) * 10.0 ** rng.integers(-3, 4, n)
    v[rng.random(n) < 0.05] = -0.0
    v[rng.random(n) < 0.05] = 0.0
    return v


def test_tetrahedral_row_order_equals_the_definition():
    rng = np.random.default_rng(31)
    for N in (1, 2, 4):
        t = meshgen.cube_mesh(N, 5)
        vals = _values(rng, 16 * t.nme)
        assert _same_bits(_row_form(t.me, t.nq, vals, 4), _nnz_form(t.me, vals, 4))


def test_triangle_row_order_equals_the_definition():
    """The same on triangles (the P2 rows follow it with six dofs per element)."""
    rng = np.random.default_rng(32)
    for N in (1, 3, 8):
        m = meshgen.square_mesh(N, 6)
        vals = _values(rng, 9 * m.nme)
        assert _same_bits(_row_form(m.me, m.nq, vals, 3), _nnz_form(m.me, vals, 3))


def test_a_plus_zero_start_would_differ():
    """Pins the reason for the -0.0 start: from +0.0, a sum of -0.0 contributions would come out
    +0.0, unlike the definition."""
    assert np.signbit(-0.0 + -0.0) and not np.signbit(0.0 + -0.0)
