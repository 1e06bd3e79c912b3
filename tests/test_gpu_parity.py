"""Parity of the CUDA path (through the C ABI) with the CPU oracle, element by element.

row_ptr / col_idx / map are compared bit-exactly; values within 1e-13 of each row's largest
|a_ij|; the deterministic variant must be bit-identical from run to run. Meshes span several
thread blocks with ragged tails, plus the edge cases (empty mesh, one triangle, a vertex of
high valence that takes the shared-memory path, the two-triangle square), and unstructured
meshes: random cell diagonals (closed fans of every size 4..8), a hole with unused vertices
and a vertex in two fans, a stretched square with angles from about 4 to 168 degrees, and the
bow-tie (two triangles touching at one vertex).
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
from paper_1305_3122_gb300 import feasm, meshgen
from tests.gpu_common import assert_csr_equal, assert_values_close

pytestmark = pytest.mark.gpu

KINDS = {"mass": oracle.MASS, "wmass": oracle.WMASS, "stiff": oracle.STIFF}
VARIANTS = [feasm.ATOMIC, feasm.GATHER, feasm.ROW]


def fan_mesh(n_out: int, ring2: bool = True):
    """A vertex of valence n_out (center 0 on a circle of n_out vertices), so the pattern build
    takes its high-valence path; optionally a second ring to mix in ordinary rows."""
    t = np.linspace(0, 2 * np.pi, n_out, endpoint=False)
    pts = [(0.0, 0.0)] + [(np.cos(a), np.sin(a)) for a in t]
    tris = [(0, 1 + i, 1 + (i + 1) % n_out) for i in range(n_out)]
    if ring2:
        base = len(pts)
        pts += [(2 * np.cos(a + np.pi / n_out), 2 * np.sin(a + np.pi / n_out)) for a in t]
        for i in range(n_out):
            a, b = 1 + i, 1 + (i + 1) % n_out
            c = base + i
            tris.append((a, c, b))
    q = np.array(pts).T.copy()
    me = np.array(tris, dtype=np.int32).T.copy()
    # make every triangle counter-clockwise
    x, y = q
    D = (x[me[2]] - x[me[0]]) * (y[me[0]] - y[me[1]]) - (x[me[0]] - x[me[1]]) * (y[me[2]] - y[me[0]])
    flip = D < 0
    me[1, flip], me[2, flip] = me[2, flip].copy(), me[1, flip].copy()
    return q, me


def fans_mesh(n_fans: int, n_out: int):
    """n_fans disjoint fans of valence n_out whose centres are vertices 0 .. n_fans - 1: one vertex
    block of the pattern build's two-level placement then holds more incidences than its
    shared-memory staging area, so that block is placed directly in global memory."""
    pts, tris = [], []
    for c in range(n_fans):
        pts.append((3.0 * c, 0.0))
    t = np.linspace(0, 2 * np.pi, n_out, endpoint=False)
    for c in range(n_fans):
        base = n_fans + c * n_out
        pts += [(3.0 * c + np.cos(a), np.sin(a)) for a in t]
        tris += [(c, base + i, base + (i + 1) % n_out) for i in range(n_out)]
    return np.array(pts).T.copy(), np.array(tris, dtype=np.int32).T.copy()


def bowtie_mesh():
    """Two triangles that touch at vertex 0 only: vertex 0's row holds two separate fans."""
    q = np.array([[0.0, 1.0, 0.0, -1.0, 0.0], [0.0, 0.0, 1.0, 0.0, -1.0]])
    me = np.array([[0, 0], [1, 3], [2, 4]], np.int32)
    return q, me


def unstructured_cases():
    """Meshes beyond the valence-6 grid: random cell diagonals (closed fans of 4 to 8 triangles,
    open fans of 1 to 4), a hole (open fans around it, unused vertices, and a vertex where two
    fans touch), a stretched square (angles of about 4 to 168 degrees, so rows mix the
    double-float and FP64 fan terms), the bow-tie, and Delaunay meshes of the unit disk."""
    out = {}
    m = meshgen.square_mesh(40, 31, random_diagonals=True)
    out["rdiag40"] = (m.q, m.me)
    m = meshgen.square_mesh(33, 32, random_diagonals=True, hole=True)
    out["rdiag_hole33"] = (m.q, m.me)
    m = meshgen.square_mesh(30, 33, random_diagonals=True, stretch=7.0)
    out["rdiag_stretch30"] = (m.q, m.me)
    m = meshgen.square_mesh(64, 34, random_diagonals=True, hole=True, stretch=2.5)
    out["rdiag_hole_stretch64"] = (m.q, m.me)
    out["bowtie"] = bowtie_mesh()
    # Delaunay meshes of the unit disk (the paper's domain): random points (valences 3 to about
    # 13, rows of more than 8 triangles for the general-row kernel, thin slivers for the FP64 fan
    # terms) and a jittered hexagonal lattice
    m = meshgen.disk_mesh(3000, 35, points="poisson")
    out["disk_poisson3000"] = (m.q, m.me)
    m = meshgen.disk_mesh(900, 36, points="lattice")
    out["disk_lattice900"] = (m.q, m.me)
    return out


def _mesh_cases():
    m64 = meshgen.square_mesh(64, meshgen.SEED_BASE + 1)
    m37 = meshgen.square_mesh(37, 5)
    qf, mef = fan_mesh(70)
    q12, me12 = fan_mesh(12)
    q2 = np.array([[0.0, 1.0, 1.0, 0.0], [0.0, 0.0, 1.0, 1.0]])
    me2 = np.array([[0, 0], [1, 2], [2, 3]], np.int32)
    qb, meb = fans_mesh(5, 4000)
    return {"square64": (m64.q, m64.me), "square37": (m37.q, m37.me), "fan70": (qf, mef), "fan12": (q12, me12),
            "fans5x4000": (qb, meb),
            "two": (q2, me2),
            "one": (q2, me2[:, :1].copy()),
            **unstructured_cases()}


CASES = _mesh_cases()


def _weights(q):
    x, y = q
    return 1.0 + 0.5 * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y) + 0.05 * np.cos(7 * x)


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("gather", [False, True])
def test_pattern_and_map(case, gather):
    q, me = CASES[case]
    mesh = feasm.Mesh(q, me)
    pat = feasm.Pattern(mesh, gather=gather)
    rp_o, ci_o, _ = oracle.assemble(oracle.MASS, q, me)
    assert_csr_equal(pat.row_ptr.cpu(), pat.col_idx.cpu(), rp_o, ci_o)
    # map[9k + 3 jl + il] is the stored position of (me[il][k], me[jl][k])
    I, J, _ = oracle.triplets(oracle.MASS, q, me)
    mp = pat.map.cpu().numpy()
    rows = np.repeat(np.arange(len(rp_o) - 1), np.diff(rp_o))
    np.testing.assert_array_equal(rows[mp], I)
    np.testing.assert_array_equal(ci_o[mp], J)


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("kind", sorted(KINDS))
@pytest.mark.parametrize("variant", VARIANTS)
def test_scalar_values(case, kind, variant):
    q, me = CASES[case]
    w = _weights(q)
    mesh = feasm.Mesh(q, me)
    pat = feasm.Pattern(mesh, gather=True)
    wd = torch.tensor(w, device="cuda")
    if kind == "mass":
        got = feasm.assemble_mass(mesh, pat, variant)
    elif kind == "wmass":
        got = feasm.assemble_wmass(mesh, pat, wd, variant)
    else:
        got = feasm.assemble_stiff(mesh, pat, variant)
    rp, ci, va = oracle.assemble(KINDS[kind], q, me, w)
    assert_values_close(rp, got.cpu().numpy(), va)


@pytest.mark.parametrize("case", ["square64", "rdiag_hole33", "rdiag_stretch30", "bowtie"])
@pytest.mark.parametrize("variant", VARIANTS)
def test_stiff_wmass_fused(case, variant):
    q, me = CASES[case]
    w = _weights(q)
    mesh = feasm.Mesh(q, me)
    pat = feasm.Pattern(mesh, gather=True)
    S, Mw = feasm.assemble_stiff_wmass(mesh, pat, torch.tensor(w, device="cuda"), variant)
    rp, _, vs = oracle.assemble(oracle.STIFF, q, me)
    _, _, vm = oracle.assemble(oracle.WMASS, q, me, w)
    assert_values_close(rp, S.cpu().numpy(), vs)
    assert_values_close(rp, Mw.cpu().numpy(), vm)


@pytest.mark.parametrize("case", ["square37", "fan70", "fan12", "two", "one", "rdiag40", "rdiag_hole33",
                                  "rdiag_stretch30", "bowtie"])
@pytest.mark.parametrize("variant", VARIANTS)
def test_elasticity(case, variant):
    q, me = CASES[case]
    mesh = feasm.Mesh(q, me)
    pat = feasm.Pattern(mesh, dofs=2, gather=True)
    rp, ci, va = oracle.assemble(oracle.ELAS, q, me, lam=1.0, mu=0.5)
    assert_csr_equal(pat.row_ptr.cpu(), pat.col_idx.cpu(), rp, ci)
    got = feasm.assemble_elas(mesh, pat, 1.0, 0.5, variant)
    assert_values_close(rp, got.cpu().numpy(), va)


@pytest.mark.parametrize("case", ["square64", "rdiag_hole_stretch64"])
@pytest.mark.parametrize("variant", [feasm.GATHER, feasm.ROW])
def test_deterministic_bit_identical_runs(case, variant):
    q, me = CASES[case]
    w = torch.tensor(_weights(q), device="cuda")
    mesh = feasm.Mesh(q, me)
    pat = feasm.Pattern(mesh, gather=True)
    first = None
    for _ in range(10):
        S, Mw = feasm.assemble_stiff_wmass(mesh, pat, w, variant)
        cur = torch.cat([S, Mw]).cpu().numpy().view(np.int64)
        if first is None:
            first = cur
        np.testing.assert_array_equal(cur, first)


def test_empty_mesh():
    q = np.zeros((2, 5))
    me = np.zeros((3, 0), np.int32)
    mesh = feasm.Mesh(q, me)
    pat = feasm.Pattern(mesh, gather=True)
    assert pat.nnz == 0
    np.testing.assert_array_equal(pat.row_ptr.cpu().numpy(), np.zeros(6, np.int32))
    for v in VARIANTS:
        assert feasm.assemble_stiff(mesh, pat, v).numel() == 0


# ------------------------------------------------------------------ error paths

def test_input_errors():
    q = np.array([[0.0, 1.0, 1.0, 0.0], [0.0, 0.0, 1.0, 1.0]])
    with pytest.raises(feasm.FeasmError) as e:
        feasm.Mesh(q, np.array([[0], [1], [4]], np.int32))
    assert e.value.status == 2
    with pytest.raises(feasm.FeasmError) as e:
        feasm.Mesh(q, np.array([[0], [1], [1]], np.int32))
    assert e.value.status == 3
    with pytest.raises(feasm.FeasmError) as e:
        feasm.Mesh(q, np.array([[0], [2], [1]], np.int32))
    assert e.value.status == 4
    mesh = feasm.Mesh(q, np.array([[0, 0], [1, 2], [2, 3]], np.int32))
    pat = feasm.Pattern(mesh)
    with pytest.raises(feasm.FeasmError) as e:
        feasm.assemble_mass(mesh, pat, out=torch.empty(5, dtype=torch.float64, device="cuda"))
    assert e.value.status == 5
    with pytest.raises(feasm.FeasmError) as e:
        feasm.assemble_mass(mesh, pat, feasm.GATHER)      # pattern built without FE_PATTERN_GATHER
    assert e.value.status == 1
    other = feasm.Mesh(q, np.array([[0, 0], [1, 2], [2, 3]], np.int32))
    with pytest.raises(feasm.FeasmError) as e:
        feasm.assemble_mass(other, pat)                   # pattern of another mesh
    assert e.value.status == 1
    with pytest.raises(feasm.FeasmError) as e:
        feasm.assemble_elas(mesh, pat, 1.0, 0.5)          # scalar pattern
    assert e.value.status == 1
    pat2 = feasm.Pattern(mesh, dofs=2)
    with pytest.raises(feasm.FeasmError) as e:
        feasm.assemble_elas(mesh, pat2, 1.0, -1.0)        # lambda + mu <= 0
    assert e.value.status == 1


def test_orientation_flag_after_set_coords():
    q = np.array([[0.0, 1.0, 1.0, 0.0], [0.0, 0.0, 1.0, 1.0]])
    mesh = feasm.Mesh(q, np.array([[0, 0], [1, 2], [2, 3]], np.int32))
    pat = feasm.Pattern(mesh)
    mesh.check()
    bad = torch.tensor(q[:, [0, 3, 2, 1]], device="cuda")    # mirror: every triangle turns clockwise
    mesh.set_coords(bad)
    feasm.assemble_stiff(mesh, pat)
    with pytest.raises(feasm.FeasmError) as e:
        mesh.check()
    assert e.value.status == 4
    mesh.check()   # the word was cleared


def test_host_one_shot_matches_device_path():
    q, me = CASES["square37"]
    w = _weights(q)
    out = feasm.assemble_host("stiff_wmass", q, me, w)
    rp, ci, vs = oracle.assemble(oracle.STIFF, q, me)
    _, _, vm = oracle.assemble(oracle.WMASS, q, me, w)
    assert_csr_equal(out["row_ptr"].numpy(), out["col_idx"].numpy(), rp, ci)
    assert_values_close(rp, out["S"].numpy(), vs)
    assert_values_close(rp, out["Mw"].numpy(), vm)


@pytest.mark.parametrize("case", ["rdiag_hole33", "rdiag_stretch30"])
def test_host_one_shot_on_unstructured_meshes(case):
    """The pipelined host call (row blocks, empty rows inside the hole) equals the device-resident
    row-owner call bit for bit and the oracle within tolerance."""
    q, me = CASES[case]
    w = _weights(q)
    out = feasm.assemble_stiff_wmass_host(q, me, w)
    rp, ci, vs = oracle.assemble(oracle.STIFF, q, me)
    _, _, vm = oracle.assemble(oracle.WMASS, q, me, w)
    assert_csr_equal(out["row_ptr"], out["col_idx"], rp, ci)
    assert_values_close(rp, out["S"].numpy(), vs)
    assert_values_close(rp, out["Mw"].numpy(), vm)
    mesh = feasm.Mesh(q, me)
    pat = feasm.Pattern(mesh, map=False)
    S, Mw = feasm.assemble_stiff_wmass(mesh, pat, torch.tensor(w, device="cuda"), feasm.ROW)
    assert torch.equal(S.cpu(), out["S"]) and torch.equal(Mw.cpu(), out["Mw"])


def test_row_variant_needs_no_map():
    q, me = CASES["square37"]
    mesh = feasm.Mesh(q, me)
    pat = feasm.Pattern(mesh, map=False)
    assert pat.map is None
    rp, ci, va = oracle.assemble(oracle.STIFF, q, me)
    assert_values_close(rp, feasm.assemble_stiff(mesh, pat, feasm.ROW).cpu().numpy(), va)
    with pytest.raises(feasm.FeasmError) as e:
        feasm.assemble_stiff(mesh, pat, feasm.ATOMIC)
    assert e.value.status == 1
    pat2 = feasm.Pattern(mesh, dofs=2, map=False)
    rp, ci, va = oracle.assemble(oracle.ELAS, q, me, lam=2.0, mu=0.25)
    assert_values_close(rp, feasm.assemble_elas(mesh, pat2, 2.0, 0.25, feasm.ROW).cpu().numpy(), va)


def test_row_variant_scale_invariance():
    """Coordinates scaled by 2^40 and 2^-30: S is unchanged, M scales with the area; the
    double-float range covers both (edge components stay within [2^-74, 2^128))."""
    m = meshgen.square_mesh(12, 3)
    for sc in (2.0 ** 40, 2.0 ** -30):
        q = m.q * sc
        mesh = feasm.Mesh(q, m.me)
        pat = feasm.Pattern(mesh, map=False)
        for kind, fn in ((oracle.STIFF, lambda: feasm.assemble_stiff(mesh, pat, feasm.ROW)),
                         (oracle.MASS, lambda: feasm.assemble_mass(mesh, pat, feasm.ROW))):
            rp, ci, va = oracle.assemble(kind, q, m.me)
            assert_values_close(rp, fn().cpu().numpy(), va)
        mesh.check()


def test_row_variant_flags_out_of_range():
    m = meshgen.square_mesh(4, 3)
    q = m.q * 2.0 ** -80                     # edge components below 2^-74
    mesh = feasm.Mesh(q, m.me)
    pat = feasm.Pattern(mesh, map=False)
    feasm.assemble_stiff(mesh, pat, feasm.ROW)
    with pytest.raises(feasm.FeasmError) as e:
        mesh.check()
    assert e.value.status == 9


def test_borrowed_connectivity_matches_copied():
    """FE_PTR_DEVICE_BORROW: the mesh reads the caller's me in place; results equal the copying
    mesh's, and the caller's array is left unchanged."""
    m = meshgen.square_mesh(37, 5)
    w = torch.tensor(_weights(m.q), device="cuda")
    q_d, me_d = torch.tensor(m.q, device="cuda"), torch.tensor(m.me, device="cuda")
    me_before = me_d.clone()
    ref = feasm.Mesh(q_d, me_d)
    bor = feasm.Mesh(q_d, me_d, borrow=True)
    pr, pb = feasm.Pattern(ref, gather=True), feasm.Pattern(bor, gather=True)
    assert torch.equal(pr.row_ptr, pb.row_ptr) and torch.equal(pr.col_idx, pb.col_idx)
    for variant in VARIANTS:
        Sr, Mr = feasm.assemble_stiff_wmass(ref, pr, w, variant)
        Sb, Mb = feasm.assemble_stiff_wmass(bor, pb, w, variant)
        rp = pr.row_ptr.cpu().numpy()
        assert_values_close(rp, Sb.cpu().numpy(), Sr.cpu().numpy())
        assert_values_close(rp, Mb.cpu().numpy(), Mr.cpu().numpy())
    bor.close()
    assert torch.equal(me_d, me_before)


def test_end_to_end_host_call():
    """fe_assemble_stiff_wmass_host: host arrays in, host CSR out, pipelined over row blocks; equal
    (bit for bit) to the device-resident row-owner call, and within tolerance of the oracle."""
    m = meshgen.square_mesh(61, 8)
    w = _weights(m.q)
    out = feasm.assemble_stiff_wmass_host(m.q, m.me, w)
    rp, ci, vs = oracle.assemble(oracle.STIFF, m.q, m.me)
    _, _, vm = oracle.assemble(oracle.WMASS, m.q, m.me, w)
    assert out["nnz"] == len(ci)
    assert_csr_equal(out["row_ptr"], out["col_idx"], rp, ci)
    assert_values_close(rp, out["S"].numpy(), vs)
    assert_values_close(rp, out["Mw"].numpy(), vm)
    mesh = feasm.Mesh(m.q, m.me)
    pat = feasm.Pattern(mesh)
    S, Mw = feasm.assemble_stiff_wmass(mesh, pat, torch.tensor(w, device="cuda"), feasm.ROW)
    assert torch.equal(S.cpu(), out["S"]) and torch.equal(Mw.cpu(), out["Mw"])
    # reusing the pinned buffers on a second, smaller mesh
    buf = {}
    feasm.assemble_stiff_wmass_host(m.q, m.me, w, pinned_out=buf)
    m2 = meshgen.square_mesh(13, 9)
    out2 = feasm.assemble_stiff_wmass_host(m2.q, m2.me, _weights(m2.q), pinned_out=buf)
    rp2, ci2, vs2 = oracle.assemble(oracle.STIFF, m2.q, m2.me)
    assert_csr_equal(out2["row_ptr"], out2["col_idx"], rp2, ci2)
    assert_values_close(rp2, out2["S"].numpy(), vs2)


def test_end_to_end_host_call_errors():
    import ctypes
    m = meshgen.square_mesh(9, 3)
    q = np.ascontiguousarray(m.q)
    me = np.ascontiguousarray(m.me)
    w = np.ones(m.nq)
    rp = np.zeros(m.nq + 1, np.int32)
    ci = np.zeros(8, np.int32)
    S = np.zeros(8)
    M = np.zeros(8)
    nnz = ctypes.c_int64()
    L = feasm.lib()
    st = L.fe_assemble_stiff_wmass_host(m.nq, m.nme, q.ctypes.data, me.ctypes.data, w.ctypes.data, rp.ctypes.data,
                                        ci.ctypes.data, S.ctypes.data, M.ctypes.data, 8, ctypes.byref(nnz), None)
    assert st == 5 and nnz.value == (m.nq + 2 * (3 * 81 + 18))       # FE_ERR_BUFFER_TOO_SMALL, nnz reported
    # pageable outputs of the right size work (without overlap)
    n = nnz.value
    ci, S, M = np.zeros(n, np.int32), np.zeros(n), np.zeros(n)
    st = L.fe_assemble_stiff_wmass_host(m.nq, m.nme, q.ctypes.data, me.ctypes.data, w.ctypes.data, rp.ctypes.data,
                                        ci.ctypes.data, S.ctypes.data, M.ctypes.data, n, ctypes.byref(nnz), None)
    assert st == 0
    rpo, cio, vso = oracle.assemble(oracle.STIFF, m.q, m.me)
    np.testing.assert_array_equal(rp, rpo)
    np.testing.assert_array_equal(ci, cio)
    assert_values_close(rpo, S, vso)
    # a clockwise triangle is an orientation error
    bad = me.copy()
    bad[1, 0], bad[2, 0] = bad[2, 0], bad[1, 0]
    st = L.fe_assemble_stiff_wmass_host(m.nq, m.nme, q.ctypes.data, bad.ctypes.data, w.ctypes.data, rp.ctypes.data,
                                        ci.ctypes.data, S.ctypes.data, M.ctypes.data, n, ctypes.byref(nnz), None)
    assert st == 4                                                      # FE_ERR_ORIENTATION
    # the connectivity is checked before the coordinates arrive: range and repeats
    bad = me.copy()
    bad[2, 5] = m.nq
    st = L.fe_assemble_stiff_wmass_host(m.nq, m.nme, q.ctypes.data, bad.ctypes.data, w.ctypes.data, rp.ctypes.data,
                                        ci.ctypes.data, S.ctypes.data, M.ctypes.data, n, ctypes.byref(nnz), None)
    assert st == 2 and b"triangle 5" in L.fe_last_error()              # FE_ERR_INDEX_RANGE
    bad = me.copy()
    bad[1, 7] = bad[0, 7]
    st = L.fe_assemble_stiff_wmass_host(m.nq, m.nme, q.ctypes.data, bad.ctypes.data, w.ctypes.data, rp.ctypes.data,
                                        ci.ctypes.data, S.ctypes.data, M.ctypes.data, n, ctypes.byref(nnz), None)
    assert st == 3 and b"triangle 7" in L.fe_last_error()              # FE_ERR_DEGENERATE
    # an orientation error takes precedence over a buffer that is too small
    bad = me.copy()
    bad[1, 3], bad[2, 3] = bad[2, 3], bad[1, 3]
    st = L.fe_assemble_stiff_wmass_host(m.nq, m.nme, q.ctypes.data, bad.ctypes.data, w.ctypes.data, rp.ctypes.data,
                                        ci.ctypes.data, S.ctypes.data, M.ctypes.data, 8, ctypes.byref(nnz), None)
    assert st == 4 and b"triangle 3" in L.fe_last_error()


# The double-float row owners' error budget: each double-float operation errs by a few units of
# 2^-48 of its operands and a row sums at most about 14 terms (fans of up to 8 triangles; longer
# rows and thin triangles take the paths built for them), so the assembled values agree with FP64
# to about 2^-44 of each row's maximum (the parity tolerance, 1e-13, leaves room above it).
ROW_BUDGET = 2.0 ** -44


@pytest.mark.parametrize("case", sorted(c for c in CASES if c != "fans5x4000"))
def test_row_owner_error_budget(case):
    """The row-owner variant's S, M^[w], M and K on every parity mesh stay within the error budget
    of the double-float arithmetic, which is tighter than the parity tolerance: a change that
    loses bits (in the thin-triangle or general-row paths, say) shows here first. (fans5x4000 is
    left out: its rows sum 4000 contributions, beyond the budget's premise; there even the FP64
    variants differ from the oracle by 3.2e-14 through the order of the sums.)"""
    q, me = CASES[case]
    w = _weights(q)
    mesh = feasm.Mesh(q, me)
    pat = feasm.Pattern(mesh, map=False)
    wd = torch.tensor(w, device="cuda")
    S, Mw = feasm.assemble_stiff_wmass(mesh, pat, wd, feasm.ROW)
    M = feasm.assemble_mass(mesh, pat, feasm.ROW)
    for kind, got in ((oracle.STIFF, S), (oracle.WMASS, Mw), (oracle.MASS, M)):
        rp, _, va = oracle.assemble(kind, q, me, w)
        assert_values_close(rp, got.cpu().numpy(), va, tol=ROW_BUDGET)
    pat2 = feasm.Pattern(mesh, dofs=2, map=False)
    rpk, _, vk = oracle.assemble(oracle.ELAS, q, me, lam=1.0, mu=0.5)
    assert_values_close(rpk, feasm.assemble_elas(mesh, pat2, 1.0, 0.5, feasm.ROW).cpu().numpy(), vk, tol=ROW_BUDGET)
