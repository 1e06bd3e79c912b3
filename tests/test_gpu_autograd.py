"""The torch.autograd wrapper (paper_1305_3122_gb300.autograd) over the assembly and its adjoint.

Checked against the oracle's adjoint, against torch.autograd.gradcheck (central differences of
the whole Jacobian on a tiny mesh) and against the direct C-ABI adjoint call.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
from paper_1305_3122_gb300 import feasm, meshgen
from paper_1305_3122_gb300.autograd import StiffWMass

pytestmark = pytest.mark.gpu


def _setup(n_cells, seed, gather=True):
    m = meshgen.square_mesh(n_cells, seed)
    w = meshgen.vertex_weights(m, seed)
    mesh = feasm.Mesh(m.q, m.me)
    pat = feasm.Pattern(mesh, gather=gather)
    return m, w, mesh, pat


@pytest.mark.parametrize("gather", [True, False])
def test_autograd_matches_oracle_adjoint(gather):
    m, w, mesh, pat = _setup(40, 21, gather)
    GS, GM = meshgen.upstream_gradients(21, pat.nnz)
    q = torch.tensor(m.q, device="cuda", requires_grad=True)
    wt = torch.tensor(w, device="cuda", requires_grad=True)
    S, M = StiffWMass(mesh, pat)(q, wt)
    loss = (torch.tensor(GS, device="cuda") * S).sum() + (torch.tensor(GM, device="cuda") * M).sum()
    loss.backward()
    rp, ci = pat.row_ptr.cpu().numpy(), pat.col_idx.cpu().numpy()
    dqS, _ = oracle.adjoint(oracle.STIFF, m.q, m.me, rp, ci, GS)
    dqM, dwo = oracle.adjoint(oracle.WMASS, m.q, m.me, rp, ci, GM, w=w)
    dqo = dqS + dqM
    assert np.abs(q.grad.cpu().numpy() - dqo).max() <= 1e-12 * np.abs(dqo).max()
    assert np.abs(wt.grad.cpu().numpy() - dwo).max() <= 1e-12 * np.abs(dwo).max()


def test_autograd_gradcheck_tiny_mesh():
    """Full Jacobian by central differences (torch.autograd.gradcheck, FP64) on a 3 x 3-cell
    mesh: 16 vertices, 18 triangles, 32 coordinates and 16 weights."""
    m, w, mesh, pat = _setup(3, 22, gather=True)
    asm = StiffWMass(mesh, pat, variant=feasm.GATHER)
    q = torch.tensor(m.q, device="cuda", requires_grad=True)
    wt = torch.tensor(w, device="cuda", requires_grad=True)
    assert torch.autograd.gradcheck(lambda a, b: asm(a, b), (q, wt), eps=1e-6, atol=1e-7, rtol=1e-6)


def test_autograd_equals_direct_adjoint_call():
    """At a larger size the wrapper's gradients are exactly those of the C-ABI adjoint (the
    gather adjoint is deterministic)."""
    m, w, mesh, pat = _setup(256, 23, gather=True)
    GS, GM = (torch.tensor(g, device="cuda") for g in meshgen.upstream_gradients(23, pat.nnz))
    q = torch.tensor(m.q, device="cuda", requires_grad=True)
    wt = torch.tensor(w, device="cuda", requires_grad=True)
    S, M = StiffWMass(mesh, pat)(q, wt)
    torch.autograd.backward([S, M], [GS, GM])
    dq, dw = feasm.adjoint_stiff_wmass(mesh, pat, wt.detach(), GS, GM, feasm.GATHER)
    assert torch.equal(q.grad, dq) and torch.equal(wt.grad, dw)


def test_autograd_only_one_output_used():
    """A loss on S alone: the M gradient is None, dL/dw must be zero."""
    m, w, mesh, pat = _setup(16, 24, gather=True)
    q = torch.tensor(m.q, device="cuda", requires_grad=True)
    wt = torch.tensor(w, device="cuda", requires_grad=True)
    S, _ = StiffWMass(mesh, pat)(q, wt)
    S.square().sum().backward()
    assert torch.count_nonzero(wt.grad) == 0
    assert torch.isfinite(q.grad).all() and torch.count_nonzero(q.grad) > 0


def test_autograd_needs_the_map():
    m = meshgen.square_mesh(4, 25)
    mesh = feasm.Mesh(m.q, m.me)
    pat = feasm.Pattern(mesh, map=False)
    with pytest.raises(ValueError):
        StiffWMass(mesh, pat)
