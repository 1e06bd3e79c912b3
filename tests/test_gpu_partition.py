"""Row partition through the C ABI (fe_mesh_create_part, fe_pattern_build_part): each rank's
owned rows, assembled from its halo triangles alone, must equal the whole mesh's rows of the
row-owner assembly bit for bit (the same fan, the same arithmetic) and the oracle within the
parity tolerance; joined in rank order they are the whole matrix."""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import oracle
from paper_1305_3122_gb300 import feasm, meshgen, partition
from tests.gpu_common import assert_csr_equal, assert_values_close

pytestmark = pytest.mark.gpu


def _mesh():
    return meshgen.square_mesh(45, 91, random_diagonals=True, hole=True, stretch=2.0)


def _block(mesh, rows, w):
    pat = feasm.Pattern(mesh, rows=rows)
    S, Mw = feasm.assemble_stiff_wmass(mesh, pat, w, feasm.ROW)
    M = feasm.assemble_mass(mesh, pat, feasm.ROW)
    return (pat.row_ptr.cpu().numpy(), pat.col_idx.cpu().numpy(), S.cpu().numpy(), Mw.cpu().numpy(),
            M.cpu().numpy())


@pytest.mark.parametrize("world", [1, 3, 4])
@pytest.mark.parametrize("source", ["host", "device"])
def test_parts_join_to_whole_matrix(world, source):
    m = _mesh()
    wh = meshgen.vertex_weights(m, 91)
    w = torch.tensor(wh, device="cuda")
    q, me = (m.q, m.me) if source == "host" else (torch.tensor(m.q, device="cuda"), torch.tensor(m.me, device="cuda"))
    blocks = []
    for r0, r1 in partition.row_ranges(m.nq, world):
        part = feasm.Mesh.part(q, me, r0, r1)
        if world > 1:
            assert part.nme < m.nme                   # a proper subset: the halo of the owned rows
        blocks.append(_block(part, (r0, r1), w))
        part.check()
    rp, ci, vs, vmw, vm = partition.concat_rows(blocks)
    full = feasm.Mesh(m.q, m.me)
    fp = feasm.Pattern(full)
    Sf, Mwf = feasm.assemble_stiff_wmass(full, fp, w, feasm.ROW)
    Mf = feasm.assemble_mass(full, fp, feasm.ROW)
    assert_csr_equal(rp, ci, fp.row_ptr.cpu(), fp.col_idx.cpu())
    for got, ref in ((vs, Sf), (vmw, Mwf), (vm, Mf)):
        np.testing.assert_array_equal(got.view(np.int64), ref.cpu().numpy().view(np.int64))
    rpo, cio, vso = oracle.assemble(oracle.STIFF, m.q, m.me)
    _, _, vmo = oracle.assemble(oracle.WMASS, m.q, m.me, wh)
    assert_csr_equal(rp, ci, rpo, cio)
    assert_values_close(rpo, vs, vso)
    assert_values_close(rpo, vmw, vmo)


def test_band_numbered_parts_join_to_whole_matrix():
    """Nodes numbered row by row, as a partitioner would number them: each of 8 ranks' triangles
    lie in a few of the 40 tiles of 2048 triangles, so most tiles keep nothing (the placement
    skips them), and the parts' local numberings are nearly contiguous ranges."""
    m = meshgen.square_mesh(200, 93, permute=False)
    wh = meshgen.vertex_weights(m, 93)
    w = torch.tensor(wh, device="cuda")
    q, me = torch.tensor(m.q, device="cuda"), torch.tensor(m.me, device="cuda")
    blocks, held = [], 0
    for r0, r1 in partition.row_ranges(m.nq, 8):
        part = feasm.Mesh.part(q, me, r0, r1)
        held += part.nme
        blocks.append(_block(part, (r0, r1), w))
        part.check()
    assert held < 1.05 * m.nme                        # each cut duplicates one or two rows of cells
    rp, ci, vs, vmw, vm = partition.concat_rows(blocks)
    full = feasm.Mesh(m.q, m.me)
    fp = feasm.Pattern(full)
    Sf, Mwf = feasm.assemble_stiff_wmass(full, fp, w, feasm.ROW)
    Mf = feasm.assemble_mass(full, fp, feasm.ROW)
    assert_csr_equal(rp, ci, fp.row_ptr.cpu(), fp.col_idx.cpu())
    for got, ref in ((vs, Sf), (vmw, Mwf), (vm, Mf)):
        np.testing.assert_array_equal(got.view(np.int64), ref.cpu().numpy().view(np.int64))
    rpo, cio, vso = oracle.assemble(oracle.STIFF, m.q, m.me)
    _, _, vmo = oracle.assemble(oracle.WMASS, m.q, m.me, wh)
    assert_csr_equal(rp, ci, rpo, cio)
    assert_values_close(rpo, vs, vso)
    assert_values_close(rpo, vmw, vmo)


def test_windows_of_a_whole_mesh():
    m = _mesh()
    w = torch.tensor(meshgen.vertex_weights(m, 91), device="cuda")
    full = feasm.Mesh(m.q, m.me)
    blocks = [_block(full, rows, w) for rows in partition.row_ranges(m.nq, 5)]
    rp, ci, vs, _, _ = partition.concat_rows(blocks)
    fp = feasm.Pattern(full)
    assert_csr_equal(rp, ci, fp.row_ptr.cpu(), fp.col_idx.cpu())
    Sf, _ = feasm.assemble_stiff_wmass(full, fp, w, feasm.ROW)
    np.testing.assert_array_equal(vs.view(np.int64), Sf.cpu().numpy().view(np.int64))


def test_partition_errors_and_edge_cases():
    m = _mesh()
    w = torch.tensor(meshgen.vertex_weights(m, 91), device="cuda")
    part = feasm.Mesh.part(m.q, m.me, 100, 300)
    pat = feasm.Pattern(part, rows=(100, 300))
    assert pat.n_rows == 200 and pat.map is None
    with pytest.raises(feasm.FeasmError) as e:          # row windows assemble by row owners only
        feasm.assemble_stiff(part, pat, feasm.ATOMIC)
    assert e.value.status == 1
    with pytest.raises(feasm.FeasmError) as e:          # outside the part's owned rows
        feasm.Pattern(part, rows=(50, 300))
    assert e.value.status == 1
    with pytest.raises(feasm.FeasmError) as e:
        feasm.Mesh.part(m.q, m.me, 10, m.nq + 1)
    assert e.value.status == 1
    with pytest.raises(feasm.FeasmError):               # batches take whole-mesh patterns
        feasm.Batch([part], [pat])
    empty = feasm.Pattern(part, rows=(150, 150))        # an empty window
    assert empty.n_rows == 0 and empty.nnz == 0
    assert feasm.assemble_stiff(part, empty, feasm.ROW).numel() == 0
    # an id out of range anywhere is an error; a clockwise triangle only where it is kept
    bad = m.me.copy()
    bad[1, 7] = m.nq
    with pytest.raises(feasm.FeasmError) as e:
        feasm.Mesh.part(m.q, bad, 0, 10)
    assert e.value.status == 2 and b"triangle 7" in feasm.lib().fe_last_error()
    flip = m.me.copy()
    k = int(np.nonzero((flip >= 0).all(axis=0))[0][-1])
    flip[1, k], flip[2, k] = flip[2, k], flip[1, k]
    owner = int(flip[0, k])
    with pytest.raises(feasm.FeasmError) as e:
        feasm.Mesh.part(m.q, flip, owner, owner + 1)
    assert e.value.status == 4 and f"triangle {k}".encode() in feasm.lib().fe_last_error()
    far = next(v for v in range(m.nq) if v not in flip[:, k])
    others = feasm.Mesh.part(m.q, flip, far, far + 1)     # triangle k is not kept: no error
    assert 0 < others.nme < m.nme


def test_part_speaks_global_ids():
    """A part numbers its vertices locally inside the library; what the caller sees stays global:
    the vertex count, the weights, the coordinates of set_coords and the window's columns."""
    m = _mesh()
    wh = meshgen.vertex_weights(m, 91)
    w = torch.tensor(wh, device="cuda")
    r0, r1 = 700, 1300
    part = feasm.Mesh.part(m.q, m.me, r0, r1)
    assert part.nq == m.nq and 0 < part.nme < m.nme
    with pytest.raises(feasm.FeasmError) as e:          # a part builds row windows only
        feasm.Pattern(part)
    assert e.value.status == 1
    # moved points (a shear and a scaling keep every triangle counter-clockwise), global array
    q2 = m.q.copy()
    q2[0] = 1.5 * m.q[0] + 0.25 * m.q[1]
    q2[1] = 0.75 * m.q[1] - 0.1
    part.set_coords(torch.tensor(q2))
    pat = feasm.Pattern(part, rows=(r0, r1))
    S, Mw = feasm.assemble_stiff_wmass(part, pat, w, feasm.ROW)
    part.check()
    full = feasm.Mesh(q2, m.me)
    fp = feasm.Pattern(full)
    Sf, Mwf = feasm.assemble_stiff_wmass(full, fp, w, feasm.ROW)
    rp, ci = fp.row_ptr.cpu().numpy(), fp.col_idx.cpu().numpy()
    lo, hi = rp[r0], rp[r1]
    np.testing.assert_array_equal(pat.row_ptr.cpu().numpy(), rp[r0:r1 + 1] - lo)
    np.testing.assert_array_equal(pat.col_idx.cpu().numpy(), ci[lo:hi])
    np.testing.assert_array_equal(S.cpu().numpy().view(np.int64), Sf.cpu().numpy()[lo:hi].view(np.int64))
    np.testing.assert_array_equal(Mw.cpu().numpy().view(np.int64), Mwf.cpu().numpy()[lo:hi].view(np.int64))
    rpo, cio, vso = oracle.assemble(oracle.STIFF, q2, m.me)
    assert_values_close(rp, Sf.cpu().numpy(), vso)


@pytest.mark.parametrize("rows", [(0, 0), (17, 17), (None, None)])
def test_empty_parts(rows):
    """An empty owned range keeps no triangle and gives an empty window; so does a range at the
    end of the numbering."""
    m = _mesh()
    r0, r1 = (m.nq, m.nq) if rows[0] is None else rows
    part = feasm.Mesh.part(torch.tensor(m.q, device="cuda"), torch.tensor(m.me, device="cuda"), r0, r1)
    assert part.nme == 0 and part.nq == m.nq
    pat = feasm.Pattern(part, rows=(r0, r1))
    assert pat.n_rows == 0 and pat.nnz == 0 and pat.row_ptr.cpu().tolist() == [0]
    w = torch.ones(m.nq, dtype=torch.float64, device="cuda")
    S, Mw = feasm.assemble_stiff_wmass(part, pat, w, feasm.ROW)
    assert S.numel() == 0 and Mw.numel() == 0
    part.check()


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        m = _mesh()
        wh = meshgen.vertex_weights(m, 91)
        w = torch.tensor(wh, device="cuda")
        r0, r1 = partition.row_ranges(m.nq, world)[rank]
        part = feasm.Mesh.part(torch.tensor(m.q, device="cuda"), torch.tensor(m.me, device="cuda"), r0, r1)
        block = _block(part, (r0, r1), w)
        torch.cuda.synchronize()
        got = [None] * world
        dist.all_gather_object(got, block)                 # host arrays, after every kernel is done
        if rank == 0:
            rp, ci, vs, vmw, _ = partition.concat_rows(got)
            rpo, cio, vso = oracle.assemble(oracle.STIFF, m.q, m.me)
            _, _, vmo = oracle.assemble(oracle.WMASS, m.q, m.me, wh)
            ok = np.array_equal(rp, rpo) and np.array_equal(ci, cio)
            rows = np.repeat(np.arange(m.nq), np.diff(rpo))
            rmax = np.zeros(m.nq)
            np.maximum.at(rmax, rows, np.abs(vso))
            ok = ok and bool(np.all(np.abs(vs - vso) <= 1e-13 * rmax[rows]))
            np.maximum.at(rmax, rows, np.abs(vmo))
            ok = ok and bool(np.all(np.abs(vmw - vmo) <= 1e-13 * rmax[rows]))
            out.put(ok)
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_gloo_ranks_assemble_their_rows():
    """Two processes, each assembling its owned rows on the GPU with no exchange of values; the
    blocks collected on rank 0 after the kernels finished form the oracle's matrix. (The ranks'
    kernels never wait on one another, so sharing one GPU is sound.)"""
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    ok = q.get(timeout=280)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert ok
