"""Every entry point fails cleanly when a device allocation fails.

fe_debug_fail_alloc(n) makes the n-th device allocation of the library from then on fail as if the
device were out of memory. For each call below, n = 1, 2, ... is tried until the call makes fewer
than n allocations and succeeds. Every earlier try must:
- raise FE_ERR_OOM, naming the injected failure;
- leave the library's memory pool as it was, so that nothing the failed call allocated stays
  allocated;
- leave the library usable: the successful call gives the result of a call without injection.
The failure is made on the host, in the allocator, before any kernel could use the memory.
"""
from __future__ import annotations

import gc

import numpy as np
import pytest
import torch

from paper_1305_3122_gb300 import feasm, meshgen

pytestmark = pytest.mark.gpu

OOM = 6          # FE_ERR_OOM
MAX_TRIES = 80   # more than any call's number of allocations


class _Fixtures:
    def __init__(self):
        m = meshgen.square_mesh(12, 3)
        self.m = m
        self.w = torch.tensor(meshgen.vertex_weights(m, 3), device="cuda")
        self.mesh = feasm.Mesh(m.q, m.me)
        self.pat = feasm.Pattern(mesh=self.mesh)
        self.pat_g = feasm.Pattern(self.mesh, gather=True)
        self.pat_m = feasm.Pattern(self.mesh, map=True)
        self.pat2 = feasm.Pattern(self.mesh, dofs=2)
        self.S = feasm.assemble_stiff(self.mesh, self.pat_g, feasm.GATHER)
        self.GS, self.GM = (torch.tensor(g, device="cuda") for g in meshgen.upstream_gradients(3, self.pat_g.nnz))
        t = meshgen.cube_mesh(3, 3)
        self.t = t
        self.tmesh = feasm.TetMesh(t.q, t.me)
        self.tpat = feasm.TetPattern(self.tmesh, gather=True)
        self.p2 = feasm.P2Pattern(self.mesh, self.pat, gather=True)
        small = [meshgen.square_mesh(n, 5 + n) for n in (3, 6)]
        self.bmesh = [feasm.Mesh(x.q, x.me) for x in small]
        self.bpat = [feasm.Pattern(x) for x in self.bmesh]
        self.part = feasm.Mesh.part(m.q, m.me, 20, 90)
        self.part_pat = feasm.Pattern(self.part, rows=(20, 90))
        self.p3 = feasm.P3Pattern(self.mesh, self.pat, gather=True)
        self.tpat_e = feasm.TetPattern(self.tmesh, gather=True, elas=True)


def _scenarios(fx: _Fixtures) -> dict:
    m = fx.m

    def batch():
        b = feasm.Batch(fx.bmesh, fx.bpat)
        b.assemble()
        torch.cuda.synchronize()
        return [s.clone() for s in b.S] + [x.clone() for x in b.M]

    return {
        "mesh": lambda: feasm.Mesh(m.q, m.me),
        "pattern": lambda: feasm.Pattern(fx.mesh),
        "pattern_gather": lambda: feasm.Pattern(fx.mesh, gather=True),
        "pattern_dofs2": lambda: feasm.Pattern(fx.mesh, dofs=2),
        "assemble_row": lambda: feasm.assemble_stiff_wmass(fx.mesh, fx.pat, fx.w, feasm.ROW),
        "assemble_atomic": lambda: feasm.assemble_stiff_wmass(fx.mesh, fx.pat_m, fx.w, feasm.ATOMIC),
        "assemble_gather": lambda: feasm.assemble_stiff_wmass(fx.mesh, fx.pat_g, fx.w, feasm.GATHER),
        "elasticity": lambda: feasm.assemble_elas(fx.mesh, fx.pat2, 1.0, 0.5, feasm.ROW),
        "adjoint_gather": lambda: feasm.adjoint_stiff_wmass(fx.mesh, fx.pat_g, fx.w, fx.GS, fx.GM, feasm.GATHER),
        "adjoint_atomic": lambda: feasm.adjoint_stiff_wmass(fx.mesh, fx.pat_g, fx.w, fx.GS, fx.GM, feasm.ATOMIC),
        "drop_zeros": lambda: feasm.drop_zeros(fx.pat_g.row_ptr, fx.pat_g.col_idx, fx.S),
        "tet_mesh": lambda: feasm.TetMesh(fx.t.q, fx.t.me),
        "tet_pattern": lambda: feasm.TetPattern(fx.tmesh, gather=True),
        "tet_gather": lambda: feasm.tet_assemble(fx.tmesh, fx.tpat, feasm.TET_STIFF, None, feasm.GATHER),
        "p2_pattern": lambda: feasm.P2Pattern(fx.mesh, fx.pat, gather=True),
        "p2_gather": lambda: feasm.p2_assemble(fx.mesh, fx.p2, feasm.P2_STIFF, variant=feasm.GATHER),
        "host_call": lambda: feasm.assemble_host("stiff_wmass", m.q, m.me, fx.w.cpu().numpy(), variant=feasm.ROW),
        "batch": batch,
        "mesh_part": lambda: feasm.Mesh.part(m.q, m.me, 20, 90),
        "pattern_part": lambda: feasm.Pattern(fx.part, rows=(30, 80)),
        "assemble_part": lambda: feasm.assemble_stiff_wmass(fx.part, fx.part_pat, fx.w, feasm.ROW),
        "p3_pattern": lambda: feasm.P3Pattern(fx.mesh, fx.pat, gather=True),
        "p3_gather": lambda: feasm.p3_assemble(fx.mesh, fx.p3, feasm.P3_STIFF, variant=feasm.GATHER),
        "p3_atomic": lambda: feasm.p3_assemble(fx.mesh, fx.p3, feasm.P3_MASS, variant=feasm.ATOMIC),
        "tet_pattern_elas": lambda: feasm.TetPattern(fx.tmesh, gather=True, elas=True),
        "tet_elas_gather": lambda: feasm.tet_assemble_elas(fx.tmesh, fx.tpat_e, 1.25, 0.4, feasm.GATHER),
        "tet_elas_atomic": lambda: feasm.tet_assemble_elas(fx.tmesh, fx.tpat_e, 1.25, 0.4, feasm.ATOMIC),
    }


def _arrays(res) -> list[np.ndarray]:
    """The numbers a result carries (tensors, tuples or dicts of them, or a handle's CSR arrays)."""
    if isinstance(res, torch.Tensor):
        return [res.detach().cpu().numpy()]
    if isinstance(res, (tuple, list)):
        return [a for r in res for a in _arrays(r)]
    if isinstance(res, dict):
        return [a for k in sorted(res) if k != "nnz" for a in _arrays(res[k])]
    if hasattr(res, "row_ptr"):
        return _arrays([res.row_ptr, res.col_idx])
    return []


def _close(res):
    if hasattr(res, "close"):
        res.close()
    elif isinstance(res, (tuple, list)):
        for r in res:
            _close(r)


FX = None


def _fx() -> _Fixtures:
    global FX
    if FX is None:
        FX = _Fixtures()
    return FX


NAMES = ["mesh", "pattern", "pattern_gather", "pattern_dofs2", "assemble_row", "assemble_atomic", "assemble_gather",
         "elasticity", "adjoint_gather", "adjoint_atomic", "drop_zeros", "tet_mesh", "tet_pattern", "tet_gather",
         "p2_pattern", "p2_gather", "host_call", "batch", "mesh_part", "pattern_part", "assemble_part", "p3_pattern",
         "p3_gather", "p3_atomic", "tet_pattern_elas", "tet_elas_gather", "tet_elas_atomic"]
# calls that certainly allocate device memory (assembly calls may work in the pattern's buffers)
ALLOCATING = {"mesh", "pattern", "pattern_gather", "pattern_dofs2", "drop_zeros", "tet_mesh", "tet_pattern",
              "p2_pattern", "host_call", "batch", "mesh_part", "pattern_part", "p3_pattern", "tet_pattern_elas",
              "tet_elas_gather"}


@pytest.mark.parametrize("name", NAMES)
def test_allocation_failure_is_clean(name):
    fx = _fx()
    fn = _scenarios(fx)[name]
    ref = fn()
    want = _arrays(ref)
    _close(ref)
    del ref
    gc.collect()
    torch.cuda.synchronize()
    base = feasm.debug_pool_used()
    failures = 0
    try:
        for n in range(1, MAX_TRIES + 1):
            feasm.debug_fail_alloc(n)
            try:
                res = fn()
            except feasm.FeasmError as e:
                feasm.debug_fail_alloc(0)
                assert e.status == OOM, str(e)
                assert "injected failure" in str(e)
                failures += 1
                gc.collect()
                torch.cuda.synchronize()
                assert feasm.debug_pool_used() == base, f"allocation {n} of {name}: memory left behind"
                continue
            feasm.debug_fail_alloc(0)
            got = _arrays(res)
            assert len(got) == len(want)
            for g, w in zip(got, want):
                assert g.shape == w.shape and g.dtype == w.dtype
                if g.dtype.kind == "f":
                    scale = max(float(np.abs(w).max()) if w.size else 0.0, 1e-300)
                    assert np.abs(g - w).max(initial=0.0) <= 1e-12 * scale
                else:
                    np.testing.assert_array_equal(g, w)
            _close(res)
            break
        else:
            pytest.fail(f"{name} still failing after {MAX_TRIES} injected failures")
    finally:
        feasm.debug_fail_alloc(0)
    if name in ALLOCATING:
        assert failures >= 1, f"{name} made no device allocation"
