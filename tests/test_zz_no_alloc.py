"""The allocation-free entry point fe_assemble_stiff_wmass_noalloc.

Some callers cannot have device memory allocated inside a library call: frameworks that route
every device allocation through their own pool and forbid hidden ones, solver plug-ins loaded
into such hosts, and loops with a fixed latency budget where an allocation could stall. For them
the library offers this variant of the staged-gather stiffness + weighted-mass assembly, whose
staging buffer is a fixed array compiled into the library. It runs the same kernels in the same
order as the ordinary FE_VARIANT_GATHER call, so its values must equal that call's bit for bit,
call after call (the shared array keeps the previous call's contents, which must not leak into
the next), and agree with the oracle within the parity tolerance.
"""
from __future__ import annotations

import pytest
import torch

import oracle
from paper_1305_3122_gb300 import feasm, meshgen
from tests.gpu_common import assert_values_close

pytestmark = pytest.mark.gpu

LIMIT = 131072   # FE_NOALLOC_MAX_TRIANGLES


def _noalloc(mesh, pat, w, S, M, stream=None) -> int:
    """Direct C-ABI call of fe_assemble_stiff_wmass_noalloc (on the current stream by default)."""
    s = stream if stream is not None else torch.cuda.current_stream()
    return feasm.lib().fe_assemble_stiff_wmass_noalloc(mesh.handle, pat.handle, w.data_ptr(), S.data_ptr(),
                                                       M.data_ptr(), min(S.numel(), M.numel()), s.cuda_stream)


def _case(n_cells, seed):
    m = meshgen.square_mesh(n_cells, seed)
    w = torch.tensor(meshgen.vertex_weights(m, seed), device="cuda")
    mesh = feasm.Mesh(m.q, m.me)
    pat = feasm.Pattern(mesh, gather=True)
    return m, w, mesh, pat


def test_noalloc_matches_gather_call_after_call():
    cases = [_case(200, 11), _case(97, 12)]          # 80000 and 18818 triangles, below the limit
    for m, w, mesh, pat in cases + cases[:1]:         # back and forth between two sizes
        S_ref, M_ref = feasm.assemble_stiff_wmass(mesh, pat, w, feasm.GATHER)
        for _ in range(2):                            # two calls in a row on the same inputs
            S = torch.full_like(S_ref, float("nan"))
            M = torch.full_like(M_ref, float("nan"))
            assert _noalloc(mesh, pat, w, S, M) == 0, feasm.lib().fe_last_error()
            torch.cuda.synchronize()
            # same kernels, same launch shapes, same order of every sum: identical bits
            assert torch.equal(S, S_ref) and torch.equal(M, M_ref)


def test_noalloc_matches_oracle():
    m, w, mesh, pat = _case(97, 12)
    S = pat.new_values()
    M = pat.new_values()
    for _ in range(2):
        assert _noalloc(mesh, pat, w, S, M) == 0, feasm.lib().fe_last_error()
    torch.cuda.synchronize()
    wh = w.cpu().numpy()
    rp, _, vs = oracle.assemble(oracle.STIFF, m.q, m.me)
    _, _, vm = oracle.assemble(oracle.WMASS, m.q, m.me, wh)
    assert_values_close(rp, S.cpu().numpy(), vs)
    assert_values_close(rp, M.cpu().numpy(), vm)


def test_noalloc_on_a_side_stream_then_release_handles():
    """Called on another stream, then the mesh and pattern are released at once: their device
    memory is returned in order on that stream, after the kernels that read it."""
    m, w, mesh, pat = _case(150, 14)
    S_ref, M_ref = feasm.assemble_stiff_wmass(mesh, pat, w, feasm.GATHER)
    S = torch.full_like(S_ref, float("nan"))
    M = torch.full_like(M_ref, float("nan"))
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    assert _noalloc(mesh, pat, w, S, M, stream=side) == 0, feasm.lib().fe_last_error()
    pat.close()
    mesh.close()
    # new allocations from the library pool, ordered on the current stream, must not disturb
    # the side stream's work still in flight
    other = _case(120, 15)
    feasm.assemble_stiff_wmass(other[2], other[3], other[1], feasm.GATHER)
    side.synchronize()
    torch.cuda.synchronize()
    assert torch.equal(S, S_ref) and torch.equal(M, M_ref)


def test_noalloc_rejects_meshes_above_the_limit():
    m, w, mesh, pat = _case(257, 13)                  # 132098 triangles
    assert m.nme > LIMIT
    S = pat.new_values()
    M = pat.new_values()
    assert _noalloc(mesh, pat, w, S, M) == 9          # FE_ERR_LIMIT
    assert b"FE_NOALLOC_MAX_TRIANGLES" in feasm.lib().fe_last_error()


def test_noalloc_needs_the_gather_pattern():
    m = meshgen.square_mesh(8, 3)
    w = torch.ones(m.nq, dtype=torch.float64, device="cuda")
    mesh = feasm.Mesh(m.q, m.me)
    pat = feasm.Pattern(mesh)
    S = pat.new_values()
    M = pat.new_values()
    assert _noalloc(mesh, pat, w, S, M) == 1          # FE_ERR_INVALID_ARG
