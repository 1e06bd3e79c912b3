"""GPU tests at the full workload sizes, the adjoint and the batched form.

Full-size meshes are too big for the oracle's whole-matrix assembly in a test, so they are
checked on sampled rows the oracle computes one by one (csr_row_values), on sampled
triangles of the map, and through properties that hold at any size.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
from paper_1305_3122_gb300 import feasm, meshgen
from tests.gpu_common import ROW_TOL, assert_csr_equal, assert_values_close

pytestmark = pytest.mark.gpu


def _structured_nnz(N: int) -> int:
    """Scalar nnz of the N x N two-triangles-per-cell grid: one diagonal entry per vertex and
    two per edge; the grid has 3N^2 + 2N edges."""
    return (N + 1) ** 2 + 2 * (3 * N * N + 2 * N)


def _check_sampled_rows(kind, m, w, rp, ci, va, n_rows_sample=48, seed=3, lam=1.0, mu=0.5):
    n_rows = len(rp) - 1
    rows = sorted(set(int(r) for r in meshgen.sample_indices(seed, n_rows_sample, n_rows)) | {0, n_rows - 1})
    for r, (cols, vals) in zip(rows, oracle.csr_row_values(kind, m.q, m.me, rows, w, lam, mu)):
        np.testing.assert_array_equal(ci[rp[r]:rp[r + 1]], cols)
        got = va[rp[r]:rp[r + 1]]
        assert np.abs(got - vals).max() <= ROW_TOL * np.abs(vals).max()


def _check_map_sampled(m, rp, ci, mp, seed=4, count=4096):
    ks = meshgen.sample_indices(seed, count, m.nme)
    rows_of = lambda p: np.searchsorted(rp, p, side="right") - 1
    for c_local in range(9):
        il, jl = c_local % 3, c_local // 3
        pos = mp[9 * ks + c_local]
        np.testing.assert_array_equal(rows_of(pos), m.me[il, ks])
        np.testing.assert_array_equal(ci[pos], m.me[jl, ks])


@pytest.fixture(scope="module")
def mesh_2048():
    m = meshgen.square_mesh(2048, meshgen.SEED_BASE + 2)
    w = meshgen.vertex_weights(m, meshgen.SEED_BASE + 2)
    return m, w


@pytest.mark.parametrize("variant", [feasm.ATOMIC, feasm.GATHER, feasm.ROW])
def test_stiff_wmass_2048_full_size(mesh_2048, variant):
    m, w = mesh_2048
    mesh = feasm.Mesh(m.q, m.me)
    pat = feasm.Pattern(mesh, gather=(variant == feasm.GATHER))
    assert pat.nnz == _structured_nnz(2048) == 29_372_417
    S, Mw = feasm.assemble_stiff_wmass(mesh, pat, torch.tensor(w, device="cuda"), variant)
    torch.cuda.synchronize()
    rp = pat.row_ptr.cpu().numpy()
    ci = pat.col_idx.cpu().numpy()
    assert np.all(np.diff(rp) > 0)
    d = np.diff(ci)
    starts = rp[1:-1]
    d[starts - 1] = 1                       # row boundaries may go down
    assert np.all(d > 0)
    _check_map_sampled(m, rp, ci, pat.map.cpu().numpy())
    vs, vm = S.cpu().numpy(), Mw.cpu().numpy()
    _check_sampled_rows(oracle.STIFF, m, w, rp, ci, vs)
    _check_sampled_rows(oracle.WMASS, m, w, rp, ci, vm)
    # S 1 = 0 in every row (relative to the row's largest entry)
    rows = torch.repeat_interleave(torch.arange(m.nq, device="cuda"), torch.diff(pat.row_ptr.long()))
    rs = torch.zeros(m.nq, dtype=torch.float64, device="cuda").index_add_(0, rows, S)
    rmax = torch.zeros(m.nq, dtype=torch.float64, device="cuda").index_reduce_(0, rows, S.abs(), "amax")
    assert bool((rs.abs() <= 16 * ROW_TOL * rmax).all())
    # sum of M^[w] = sum over triangles of |T| (w0 + w1 + w2) / 3
    x, y = m.q
    me = m.me
    D = (x[me[2]] - x[me[0]]) * (y[me[0]] - y[me[1]]) - (x[me[0]] - x[me[1]]) * (y[me[2]] - y[me[0]])
    assert vm.sum() == pytest.approx(np.sum(D / 2 * (w[me[0]] + w[me[1]] + w[me[2]]) / 3), rel=1e-12)


@pytest.fixture(scope="module")
def mesh_2048_unstructured():
    seed = meshgen.SEED_BASE + 12
    m = meshgen.square_mesh(2048, seed, random_diagonals=True, hole=True)
    return m, meshgen.vertex_weights(m, seed)


@pytest.mark.parametrize("variant", [feasm.ATOMIC, feasm.GATHER, feasm.ROW])
def test_stiff_wmass_2048_unstructured(mesh_2048_unstructured, variant):
    """The 2048 x 2048-cell square with random cell diagonals, a hole and a pinch vertex: rows of
    every fan size, empty rows; sampled rows against the oracle, S 1 = 0 on every row and the
    weighted-mass total, at the size of the headline workload."""
    m, w = mesh_2048_unstructured
    mesh = feasm.Mesh(m.q, m.me)
    pat = feasm.Pattern(mesh, gather=(variant == feasm.GATHER))
    S, Mw = feasm.assemble_stiff_wmass(mesh, pat, torch.tensor(w, device="cuda"), variant)
    torch.cuda.synchronize()
    rp = pat.row_ptr.cpu().numpy()
    ci = pat.col_idx.cpu().numpy()
    val = np.bincount(m.me.ravel(), minlength=m.nq)
    assert np.array_equal(np.diff(rp) == 0, val == 0)          # empty rows exactly at unused vertices
    # nnz: one diagonal entry per used vertex and two per edge
    e = np.sort(np.concatenate([m.me[[0, 1]], m.me[[1, 2]], m.me[[2, 0]]], axis=1), axis=0)
    n_edges = len(np.unique(e[0].astype(np.int64) * m.nq + e[1]))
    assert pat.nnz == int((val > 0).sum()) + 2 * n_edges
    # sampled rows: random ones, the unused vertices' neighbours and the vertices of each valence
    rows = set(int(r) for r in meshgen.sample_indices(7, 48, m.nq))
    for v in range(1, 9):
        rows |= set(int(r) for r in np.nonzero(val == v)[0][:3])
    rows = sorted(rows)
    vs, vm = S.cpu().numpy(), Mw.cpu().numpy()
    for kind, va in ((oracle.STIFF, vs), (oracle.WMASS, vm)):
        for r, (cols, vals) in zip(rows, oracle.csr_row_values(kind, m.q, m.me, rows, w)):
            np.testing.assert_array_equal(ci[rp[r]:rp[r + 1]], cols)
            if len(cols):
                assert np.abs(va[rp[r]:rp[r + 1]] - vals).max() <= ROW_TOL * np.abs(vals).max()
    _check_map_sampled(m, rp, ci, pat.map.cpu().numpy())
    rows_t = torch.repeat_interleave(torch.arange(m.nq, device="cuda"), torch.diff(pat.row_ptr.long()))
    rs = torch.zeros(m.nq, dtype=torch.float64, device="cuda").index_add_(0, rows_t, S)
    rmax = torch.zeros(m.nq, dtype=torch.float64, device="cuda").index_reduce_(0, rows_t, S.abs(), "amax")
    assert bool((rs.abs() <= 16 * ROW_TOL * rmax).all())
    x, y = m.q
    me = m.me
    D = (x[me[2]] - x[me[0]]) * (y[me[0]] - y[me[1]]) - (x[me[0]] - x[me[1]]) * (y[me[2]] - y[me[0]])
    assert vm.sum() == pytest.approx(np.sum(D / 2 * (w[me[0]] + w[me[1]] + w[me[2]]) / 3), rel=1e-12)


@pytest.fixture(scope="module")
def disk_1m():
    seed = meshgen.SEED_BASE + 20
    m = meshgen.disk_mesh(1 << 20, seed, points="poisson")
    return m, meshgen.vertex_weights(m, seed)


@pytest.mark.parametrize("variant", [feasm.ATOMIC, feasm.GATHER, feasm.ROW])
def test_stiff_wmass_disk_1m(disk_1m, variant):
    """The Delaunay disk of 2^20 random points, as the benchmark's disk leg times it: sampled rows
    (random ones, and rows of every valence from 3 to the largest, so the general-row kernel's
    rows too) against the oracle; S 1 = 0 on every row; the M^[w] total."""
    m, w = disk_1m
    mesh = feasm.Mesh(m.q, m.me)
    pat = feasm.Pattern(mesh, gather=(variant == feasm.GATHER), map=(variant == feasm.ATOMIC))
    S, Mw = feasm.assemble_stiff_wmass(mesh, pat, torch.tensor(w, device="cuda"), variant)
    torch.cuda.synchronize()
    rp = pat.row_ptr.cpu().numpy()
    ci = pat.col_idx.cpu().numpy()
    val = np.bincount(m.me.ravel(), minlength=m.nq)
    rows = set(int(r) for r in meshgen.sample_indices(8, 32, m.nq))
    for v in range(3, int(val.max()) + 1):
        rows |= set(int(r) for r in np.nonzero(val == v)[0][:2])
    rows = sorted(rows)
    vs, vm = S.cpu().numpy(), Mw.cpu().numpy()
    for kind, va in ((oracle.STIFF, vs), (oracle.WMASS, vm)):
        for r, (cols, vals) in zip(rows, oracle.csr_row_values(kind, m.q, m.me, rows, w)):
            np.testing.assert_array_equal(ci[rp[r]:rp[r + 1]], cols)
            assert np.abs(va[rp[r]:rp[r + 1]] - vals).max() <= ROW_TOL * np.abs(vals).max()
    rows_t = torch.repeat_interleave(torch.arange(m.nq, device="cuda"), torch.diff(pat.row_ptr.long()))
    rs = torch.zeros(m.nq, dtype=torch.float64, device="cuda").index_add_(0, rows_t, S)
    rmax = torch.zeros(m.nq, dtype=torch.float64, device="cuda").index_reduce_(0, rows_t, S.abs(), "amax")
    assert bool((rs.abs() <= 16 * ROW_TOL * rmax).all())
    x, y = m.q
    me = m.me
    D = (x[me[2]] - x[me[0]]) * (y[me[0]] - y[me[1]]) - (x[me[0]] - x[me[1]]) * (y[me[2]] - y[me[0]])
    assert vm.sum() == pytest.approx(np.sum(D / 2 * (w[me[0]] + w[me[1]] + w[me[2]]) / 3), rel=1e-12)
    mesh.check()


def test_mass_64_full_oracle():
    m = meshgen.square_mesh(64, meshgen.SEED_BASE + 1)
    mesh = feasm.Mesh(m.q, m.me)
    pat = feasm.Pattern(mesh, gather=True)
    rp, ci, va = oracle.assemble(oracle.MASS, m.q, m.me)
    assert len(ci) == _structured_nnz(64) == 29_057
    assert_csr_equal(pat.row_ptr.cpu(), pat.col_idx.cpu(), rp, ci)
    for v in (feasm.ATOMIC, feasm.GATHER, feasm.ROW):
        got = feasm.assemble_mass(mesh, pat, v).cpu().numpy()
        assert_values_close(rp, got, va)
        assert got.sum() == pytest.approx(1.0, rel=1e-13)


@pytest.mark.parametrize("variant", [feasm.ATOMIC, feasm.GATHER, feasm.ROW])
def test_elasticity_1024_full_size(variant):
    m = meshgen.square_mesh(1024, meshgen.SEED_BASE + 3)
    mesh = feasm.Mesh(m.q, m.me)
    pat = feasm.Pattern(mesh, dofs=2, gather=(variant == feasm.GATHER))
    assert pat.nnz == 4 * _structured_nnz(1024) == 29_384_708
    K = feasm.assemble_elas(mesh, pat, 1.0, 0.5, variant)
    rp = pat.row_ptr.cpu().numpy()
    ci = pat.col_idx.cpu().numpy()
    _check_sampled_rows(oracle.ELAS, m, None, rp, ci, K.cpu().numpy(), n_rows_sample=32)
    # rigid-body modes are in the kernel of K
    A = pat.to_sparse_csr(K)
    x, y = (torch.tensor(v, device="cuda") for v in m.q)
    kmax = K.abs().max()
    for rx, ry in ((torch.ones_like(x), torch.zeros_like(x)), (torch.zeros_like(x), torch.ones_like(x)), (-y, x)):
        r = torch.stack([rx, ry], dim=1).reshape(-1)
        assert float((A @ r).abs().max()) <= 64 * ROW_TOL * float(kmax)


# ------------------------------------------------------------------ adjoint

ADJ_MESHES = {"grid96": {}, "rdiag_hole96": dict(random_diagonals=True, hole=True),
              "rdiag_stretch80": dict(random_diagonals=True, stretch=4.0)}


@pytest.mark.parametrize("mesh_kind", sorted(ADJ_MESHES))
@pytest.mark.parametrize("variant", [feasm.ATOMIC, feasm.GATHER])
def test_adjoint_vs_oracle(variant, mesh_kind):
    kw = ADJ_MESHES[mesh_kind]
    m = meshgen.square_mesh(80 if "stretch" in kw else 96, meshgen.SEED_BASE + 5, **kw)
    w = meshgen.vertex_weights(m, meshgen.SEED_BASE + 5)
    mesh = feasm.Mesh(m.q, m.me)
    pat = feasm.Pattern(mesh, gather=True)
    GS, GM = meshgen.upstream_gradients(meshgen.SEED_BASE + 5, pat.nnz)
    dq, dw = feasm.adjoint_stiff_wmass(mesh, pat, torch.tensor(w, device="cuda"), torch.tensor(GS, device="cuda"),
                                       torch.tensor(GM, device="cuda"), variant)
    rp = pat.row_ptr.cpu().numpy()
    ci = pat.col_idx.cpu().numpy()
    dqS, _ = oracle.adjoint(oracle.STIFF, m.q, m.me, rp, ci, GS)
    dqM, dwo = oracle.adjoint(oracle.WMASS, m.q, m.me, rp, ci, GM, w=w)
    dqo = dqS + dqM
    assert np.abs(dq.cpu().numpy() - dqo).max() <= 1e-12 * np.abs(dqo).max()
    assert np.abs(dw.cpu().numpy() - dwo).max() <= 1e-12 * np.abs(dwo).max()


def test_adjoint_gather_bit_identical():
    m = meshgen.square_mesh(64, 9)
    w = torch.tensor(meshgen.vertex_weights(m, 9), device="cuda")
    mesh = feasm.Mesh(m.q, m.me)
    pat = feasm.Pattern(mesh, gather=True)
    GS, GM = (torch.tensor(g, device="cuda") for g in meshgen.upstream_gradients(9, pat.nnz))
    ref = None
    for _ in range(10):
        dq, dw = feasm.adjoint_stiff_wmass(mesh, pat, w, GS, GM, feasm.GATHER)
        cur = torch.cat([dq.reshape(-1), dw]).cpu().numpy().view(np.int64)
        ref = cur if ref is None else ref
        np.testing.assert_array_equal(cur, ref)


def test_adjoint_1024_finite_differences():
    """Central differences (h = 1e-6) of L = sum(G_S S.values) + sum(G_M M^[w].values) on 64
    sampled coordinates of the 1024 x 1024 mesh. The forward uses the deterministic variant,
    so values of the non-zeros a move does not touch are bit-identical and drop out exactly."""
    seed = meshgen.SEED_BASE + 5
    m = meshgen.square_mesh(1024, seed)
    w = torch.tensor(meshgen.vertex_weights(m, seed), device="cuda")
    mesh = feasm.Mesh(m.q, m.me)
    pat = feasm.Pattern(mesh, gather=True)
    GS, GM = (torch.tensor(g, device="cuda") for g in meshgen.upstream_gradients(seed, pat.nnz))
    dq, dw = feasm.adjoint_stiff_wmass(mesh, pat, w, GS, GM, feasm.ATOMIC)
    dq = dq.cpu().numpy()
    scale = np.abs(dq).max()
    q0 = torch.tensor(m.q, device="cuda")
    h = 1e-6
    for flat in meshgen.sample_indices(seed, 64, 2 * m.nq):
        r, i = divmod(int(flat), m.nq)
        vals = []
        for sgn in (1.0, -1.0):
            qq = q0.clone()
            qq[r, i] += sgn * h
            mesh.set_coords(qq)
            S, Mw = feasm.assemble_stiff_wmass(mesh, pat, w, feasm.GATHER)
            vals.append((S, Mw))
        dL = float(torch.dot(GS, vals[0][0] - vals[1][0]) + torch.dot(GM, vals[0][1] - vals[1][1]))
        assert abs(dL / (2 * h) - dq[r, i]) <= 1e-6 * scale
    mesh.set_coords(q0)
    mesh.check()
    # dL/dw is exact: L_M is linear in w
    for c in meshgen.sample_indices(seed + 1, 4, m.nq):
        e = torch.zeros(m.nq, dtype=torch.float64, device="cuda")
        e[int(c)] = 1.0
        _, Mw = feasm.assemble_stiff_wmass(mesh, pat, e, feasm.GATHER)
        assert float(torch.dot(GM, Mw)) == pytest.approx(float(dw[int(c)]), rel=1e-12, abs=1e-18)


# ------------------------------------------------------------------ batched

@pytest.fixture(scope="module")
def batch4():
    seed = meshgen.SEED_BASE + 4
    meshes = meshgen.batch_meshes(seed)
    fm = [feasm.Mesh(m.q, m.me) for m in meshes]
    fp = [feasm.Pattern(x) for x in fm]
    return meshes, fm, fp


@pytest.fixture(scope="module")
def batch4_oracle(batch4):
    """The oracle's S and M for 64 meshes of the batch spanning its size range: every fourth mesh
    in order of size, from the smallest to the largest."""
    meshes = batch4[0]
    order = np.argsort([m.nme for m in meshes], kind="stable")
    picked = sorted(set(int(i) for i in order[::4]) | {int(order[-1])})
    out = {}
    for idx in picked:
        m = meshes[idx]
        rp, ci, vs = oracle.assemble(oracle.STIFF, m.q, m.me)
        _, _, vm = oracle.assemble(oracle.MASS, m.q, m.me)
        out[idx] = (rp, ci, vs, vm)
    return out


@pytest.mark.parametrize("variant", [feasm.ROW, feasm.ATOMIC])
def test_batch_matches_plain_and_oracle(batch4, batch4_oracle, variant):
    meshes, fm, fp = batch4
    assert len(meshes) == 256
    b = feasm.Batch(fm, fp)
    b.configure(variant, 256, 1024)
    assert b.config() == (variant, 256, 1024)
    S, M = b.assemble()
    S = [t.clone() for t in S]
    M = [t.clone() for t in M]
    # every mesh against the oracle where it was computed, element by element
    assert len(batch4_oracle) >= 64
    for idx, (rp, ci, vs, vm) in batch4_oracle.items():
        assert_csr_equal(fp[idx].row_ptr.cpu(), fp[idx].col_idx.cpu(), rp, ci)
        assert_values_close(rp, S[idx].cpu().numpy(), vs)
        assert_values_close(rp, M[idx].cpu().numpy(), vm)
    # and all 256 against the per-mesh launches of the same scheme
    Sp, Mp = b.assemble_plain()
    for m, s0, s1, m0, m1, p in zip(meshes, S, Sp, M, Mp, fp):
        rp = p.row_ptr.cpu().numpy()
        assert_values_close(rp, s0.cpu().numpy(), s1.cpu().numpy())
        assert_values_close(rp, m0.cpu().numpy(), m1.cpu().numpy())


@pytest.mark.parametrize("variant", [feasm.ROW, feasm.ATOMIC])
def test_batch_of_unstructured_meshes_matches_oracle(variant):
    """A batch of random-diagonal meshes, with holes and stretches, of uneven sizes: every mesh
    against the oracle."""
    from tests.test_gpu_parity import bowtie_mesh
    ms = [meshgen.square_mesh(n, 500 + n, random_diagonals=True, hole=(n >= 8 and n % 2 == 0),
                              stretch=1.0 + (n % 5)) for n in (3, 8, 17, 40, 64, 130, 211)]
    cases = [(m.q, m.me) for m in ms] + [bowtie_mesh()]
    fm = [feasm.Mesh(q, me) for q, me in cases]
    fp = [feasm.Pattern(x) for x in fm]
    b = feasm.Batch(fm, fp)
    for block, tile in ((128, 256), (256, 4096)):
        b.configure(variant, block, tile)
        S, M = b.assemble()
        for (q, me), s, mm, p in zip(cases, S, M, fp):
            rp, ci, vs = oracle.assemble(oracle.STIFF, q, me)
            _, _, vm = oracle.assemble(oracle.MASS, q, me)
            assert_csr_equal(p.row_ptr.cpu(), p.col_idx.cpu(), rp, ci)
            assert_values_close(rp, s.cpu().numpy(), vs)
            assert_values_close(rp, mm.cpu().numpy(), vm)
    for x in fm:
        x.check()


def test_batch_row_variant_is_deterministic(batch4):
    meshes, fm, fp = batch4
    b = feasm.Batch(fm[:16], fp[:16])
    b.configure(feasm.ROW, 128, 256)
    ref = [t.clone() for t in b.assemble()[0]]
    for _ in range(3):
        for x, y in zip(ref, b.assemble()[0]):
            assert torch.equal(x, y)


def test_batch_tune_and_replay(batch4):
    meshes, fm, fp = batch4
    b = feasm.Batch(fm[:32], fp[:32])
    block, tile = b.tune()
    variant, block2, tile2 = b.config()
    assert (block2, tile2) == (block, tile)
    assert variant in (feasm.ROW, feasm.ATOMIC)
    assert block in (128, 256, 512) and tile in (256, 1024, 4096)
    S1 = [t.clone() for t in b.assemble()[0]]
    S2 = b.assemble()[0]
    for p, x, y in zip(fp[:32], S1, S2):
        assert_values_close(p.row_ptr.cpu().numpy(), y.cpu().numpy(), x.cpu().numpy())


def test_batch_without_map_uses_row_owners():
    ms = [meshgen.square_mesh(n, 40 + n) for n in (3, 17, 40)]
    fm = [feasm.Mesh(m.q, m.me) for m in ms]
    fp = [feasm.Pattern(x, map=False) for x in fm]
    b = feasm.Batch(fm, fp)
    assert b.config()[0] == feasm.ROW
    with pytest.raises(feasm.FeasmError):
        b.configure(feasm.ATOMIC, 256, 1024)
    S, M = b.assemble()
    for m, s, mm, p in zip(ms, S, M, fp):
        rp, _, vs = oracle.assemble(oracle.STIFF, m.q, m.me)
        _, _, vm = oracle.assemble(oracle.MASS, m.q, m.me)
        assert_values_close(rp, s.cpu().numpy(), vs)
        assert_values_close(rp, mm.cpu().numpy(), vm)


def test_batch_general_rows_match_oracle():
    """A batch whose meshes contain general rows (a vertex of valence 70, and a vertex shared by
    two separate fans): the row-owner scheme routes them through its general-row list."""
    from tests.test_gpu_parity import bowtie_mesh, fan_mesh
    qf, mef = fan_mesh(70)
    q2, me2 = bowtie_mesh()                                      # two triangles touching at vertex 0 only
    sq = meshgen.square_mesh(9, 77)
    cases = [(qf, mef), (sq.q, sq.me), (q2, me2)]
    fm = [feasm.Mesh(q, me) for q, me in cases]
    fp = [feasm.Pattern(x, map=False) for x in fm]
    b = feasm.Batch(fm, fp)
    for variant_shape in [(128, 256), (256, 4096)]:
        b.configure(feasm.ROW, *variant_shape)
        S, M = b.assemble()
        for (q, me), s, mm in zip(cases, S, M):
            rp, _, vs = oracle.assemble(oracle.STIFF, q, me)
            _, _, vm = oracle.assemble(oracle.MASS, q, me)
            assert_values_close(rp, s.cpu().numpy(), vs)
            assert_values_close(rp, mm.cpu().numpy(), vm)
    for x in fm:
        x.check()
