"""The bounds-checked build: the library compiled with -DFEASM_BOUNDS_CHECK checks every index it
derives itself (map, permutation and incidence entries, fan records, bucket slots, in-row
positions) and counts those out of range instead of trapping. The small parity cases run once on
that build, in a child process that loads it, and must give the oracle's values with no index out
of range. (This stands in for a memory checker, which is not available here.)"""
from __future__ import annotations

import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys
sys.path.insert(0, {root!r})
import numpy as np, torch
import oracle
from paper_1305_3122_gb300 import feasm, meshgen, partition
from tests.gpu_common import assert_csr_equal, assert_values_close
from tests.test_gpu_parity import CASES, _weights
checked, n0 = feasm.debug_bounds(reset=True)
assert checked, "the loaded library is not the bounds-checked build"
for name, (q, me) in sorted(CASES.items()):
    w = _weights(q)
    wd = torch.tensor(w, device="cuda")
    mesh = feasm.Mesh(q, me)
    pat = feasm.Pattern(mesh, gather=True)
    rp, ci, vs = oracle.assemble(oracle.STIFF, q, me)
    _, _, vm = oracle.assemble(oracle.WMASS, q, me, w)
    assert_csr_equal(pat.row_ptr.cpu(), pat.col_idx.cpu(), rp, ci)
    for v in (feasm.ROW, feasm.ATOMIC, feasm.GATHER):
        S, Mw = feasm.assemble_stiff_wmass(mesh, pat, wd, v)
        assert_values_close(rp, S.cpu().numpy(), vs)
        assert_values_close(rp, Mw.cpu().numpy(), vm)
    pat2 = feasm.Pattern(mesh, dofs=2, gather=True)
    rpk, _, vk = oracle.assemble(oracle.ELAS, q, me, lam=1.0, mu=0.5)
    for v in (feasm.ROW, feasm.ATOMIC, feasm.GATHER):
        assert_values_close(rpk, feasm.assemble_elas(mesh, pat2, 1.0, 0.5, v).cpu().numpy(), vk)
    GS, GM = (torch.tensor(g, device="cuda") for g in meshgen.upstream_gradients(3, pat.nnz))
    for v in (feasm.ATOMIC, feasm.GATHER):
        feasm.adjoint_stiff_wmass(mesh, pat, wd, GS, GM, v)
    if mesh.nme > 0 and name != "fans5x4000":                 # P2 takes valences up to 680
        p2 = feasm.P2Pattern(mesh, feasm.Pattern(mesh), gather=True)
        rp2, _, va2 = oracle.p2_assemble(oracle.STIFF, q, me)
        for v in (feasm.ATOMIC, feasm.GATHER):
            assert_values_close(rp2, feasm.p2_assemble(mesh, p2, feasm.P2_STIFF, variant=v).cpu().numpy(), va2)
    if mesh.nme > 0 and name != "fans5x4000":                 # P3 takes valences up to 400
        p3 = feasm.P3Pattern(mesh, feasm.Pattern(mesh), gather=True)
        rp3, _, va3 = oracle.p3_assemble(oracle.STIFF, q, me)
        for v in (feasm.ATOMIC, feasm.GATHER):
            assert_values_close(rp3, feasm.p3_assemble(mesh, p3, feasm.P3_STIFF, variant=v).cpu().numpy(), va3)
    for r0, r1 in partition.row_ranges(mesh.nq, 2):
        part = feasm.Mesh.part(q, me, r0, r1)
        pp = feasm.Pattern(part, rows=(r0, r1))
        feasm.assemble_stiff_wmass(part, pp, wd, feasm.ROW)
    mesh.check()
t = meshgen.cube_mesh(5, 4)
tm = feasm.TetMesh(t.q, t.me)
tp = feasm.TetPattern(tm, gather=True)
rpt, _, vt = oracle.tet_assemble(oracle.STIFF, t.q, t.me)
for v in (feasm.ATOMIC, feasm.GATHER):
    assert_values_close(rpt, feasm.tet_assemble(tm, tp, feasm.TET_STIFF, None, v).cpu().numpy(), vt)
from tests.test_gpu_tet import star_mesh
for tq, tme in ((t.q, t.me), star_mesh(20), star_mesh(40)):
    em = feasm.TetMesh(tq, tme)
    ep = feasm.TetPattern(em, gather=True, elas=True)
    rpe, _, ve = oracle.tet_elas_assemble(tq, tme, 1.25, 0.4)
    for v in (feasm.ATOMIC, feasm.GATHER):
        assert_values_close(rpe, feasm.tet_assemble_elas(em, ep, 1.25, 0.4, v).cpu().numpy(), ve)
ms = [meshgen.square_mesh(n, 60 + n, random_diagonals=True) for n in (5, 12, 30)]
fm = [feasm.Mesh(x.q, x.me) for x in ms]
fp = [feasm.Pattern(x) for x in fm]
b = feasm.Batch(fm, fp)
for var in (feasm.ROW, feasm.ATOMIC):
    b.configure(var, 128, 256)
    b.assemble()
torch.cuda.synchronize()
_, n = feasm.debug_bounds()
print("violations", n)
assert n == 0, f"{{n}} derived indices out of range"
"""


@pytest.mark.timeout(1200)
def test_bounds_checked_build_runs_parity_cases_clean():
    from paper_1305_3122_gb300 import build
    lib = build.build(checked=True)
    env = dict(os.environ, FEASM_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT)], capture_output=True, text=True, env=env,
                       cwd=ROOT, timeout=1100)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "violations 0" in r.stdout


def test_ordinary_build_reports_no_checks():
    from paper_1305_3122_gb300 import feasm
    if os.environ.get("FEASM_LIBRARY"):
        pytest.skip("another build of the library is loaded")
    checked, n = feasm.debug_bounds()
    assert not checked and n == 0
