"""Host side of a row partition of one mesh over several ranks (no data-path collective).

Each rank assembles the rows it owns from its halo triangles (``feasm.Mesh.part``,
``feasm.Pattern(..., rows=...)``) and gets a CSR block whose row_ptr starts at 0 and whose
col_idx holds global column ids. These helpers pick the ranks' row ranges and join the blocks,
in rank order, into the global CSR arrays; they move arrays only and compute no matrix entry.
"""
from __future__ import annotations

import numpy as np


def row_ranges(nq: int, world: int) -> list[tuple[int, int]]:
    """Contiguous owned-row ranges [begin, end) of `world` ranks covering 0..nq-1, sizes
    differing by at most one."""
    if world < 1:
        raise ValueError("world must be >= 1")
    edges = [(nq * r) // world for r in range(world + 1)]
    return [(edges[r], edges[r + 1]) for r in range(world)]


def concat_rows(blocks: list[tuple]) -> tuple:
    """Joins per-rank CSR blocks (row_ptr from 0, col_idx, then any number of value arrays), in
    rank order, into (row_ptr, col_idx, values...) of the rows of all blocks."""
    if not blocks:
        raise ValueError("no blocks")
    n_val = len(blocks[0]) - 2
    rps, cis, vals = [np.zeros(1, dtype=np.int64)], [], [[] for _ in range(n_val)]
    base = 0
    for b in blocks:
        rp = np.asarray(b[0], dtype=np.int64)
        if rp[0] != 0 or np.any(np.diff(rp) < 0) or len(b) - 2 != n_val:
            raise ValueError("a block's row_ptr must start at 0 and not decrease")
        rps.append(rp[1:] + base)
        base += int(rp[-1])
        cis.append(np.asarray(b[1])[: rp[-1]])
        for j in range(n_val):
            vals[j].append(np.asarray(b[2 + j])[: rp[-1]])
    row_ptr = np.concatenate(rps).astype(np.int32)
    col_idx = np.concatenate(cis).astype(np.int32)
    return (row_ptr, col_idx, *[np.concatenate(v) for v in vals])
