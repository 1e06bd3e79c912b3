"""Row partition of one mesh over two ranks (gloo, on the CPU): each rank takes the triangles
touching its owned rows (the selection rule of fe_mesh_create_part, restated in numpy), assembles
its rows with the oracle from those triangles alone, and rank 0 joins the blocks
(partition.concat_rows). The result must equal the whole mesh's oracle matrix bit for bit: the
halo triangles are complete for the owned rows, and keeping them in ascending order keeps every
sum's order. This is the property that lets the GPU ranks assemble with no exchange of values."""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from paper_1305_3122_gb300 import meshgen, partition


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _mesh():
    return meshgen.square_mesh(21, 77, random_diagonals=True, hole=True)


def _halo(me, r0, r1):
    return me[:, ((me >= r0) & (me < r1)).any(axis=0)]


def _rank_block(m, w, r0, r1):
    me_part = _halo(m.me, r0, r1)
    out = []
    for kind in (oracle.STIFF, oracle.WMASS):
        rp, ci, va = oracle.assemble(kind, m.q, me_part, w)
        lo, hi = rp[r0], rp[r1]
        out.append((rp[r0:r1 + 1] - lo, ci[lo:hi], va[lo:hi]))
    (rp, ci, vs), (_, _, vm) = out
    return rp, ci, vs, vm


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        m = _mesh()
        w = meshgen.vertex_weights(m, 77)
        r0, r1 = partition.row_ranges(m.nq, world)[rank]
        block = _rank_block(m, w, r0, r1)
        gathered = [None] * world
        dist.all_gather_object(gathered, block)          # the only exchange: results, after assembly
        if rank == 0:
            rp, ci, vs, vm = partition.concat_rows(gathered)
            rpo, cio, vso = oracle.assemble(oracle.STIFF, m.q, m.me)
            _, _, vmo = oracle.assemble(oracle.WMASS, m.q, m.me, w)
            ok = (np.array_equal(rp, rpo) and np.array_equal(ci, cio) and
                  np.array_equal(vs.view(np.int64), vso.view(np.int64)) and
                  np.array_equal(vm.view(np.int64), vmo.view(np.int64)))
            q.put(("ok", ok, len(_halo(m.me, *partition.row_ranges(m.nq, world)[0])[0]), m.nme))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(180)
def test_two_rank_row_partition_equals_whole_matrix():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    tag, ok, n_halo0, nme = q.get(timeout=150)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert tag == "ok" and ok
    assert 0 < n_halo0 < nme                              # a proper subset of the triangles


def test_row_ranges_and_concat():
    assert partition.row_ranges(10, 3) == [(0, 3), (3, 6), (6, 10)]
    assert partition.row_ranges(0, 2) == [(0, 0), (0, 0)]
    rp, ci, v = partition.concat_rows([(np.array([0, 2]), np.array([0, 1]), np.array([1.0, 2.0])),
                                       (np.array([0]), np.array([], np.int32), np.array([])),
                                       (np.array([0, 1, 3]), np.array([1, 0, 2]), np.array([3.0, 4.0, 5.0]))])
    np.testing.assert_array_equal(rp, [0, 2, 3, 5])
    np.testing.assert_array_equal(ci, [0, 1, 1, 0, 2])
    np.testing.assert_array_equal(v, [1, 2, 3, 4, 5])
    with pytest.raises(ValueError):
        partition.concat_rows([(np.array([1, 2]), np.array([0]))])


@pytest.mark.parametrize("world", [3, 5])
def test_partition_blocks_equal_whole_matrix_in_process(world):
    m = _mesh()
    w = meshgen.vertex_weights(m, 77)
    blocks = [_rank_block(m, w, r0, r1) for r0, r1 in partition.row_ranges(m.nq, world)]
    rp, ci, vs, vm = partition.concat_rows(blocks)
    rpo, cio, vso = oracle.assemble(oracle.STIFF, m.q, m.me)
    np.testing.assert_array_equal(rp, rpo)
    np.testing.assert_array_equal(ci, cio)
    np.testing.assert_array_equal(vs.view(np.int64), vso.view(np.int64))
