"""torch.autograd wrapper of the stiffness + weighted-mass assembly and its adjoint kernel.

Not in the paper. S(q) (Eq. 3) and M^[w](q, w) (Eq. 2) are differentiable in the vertex
coordinates q (through the edge vectors and the area |T| = D/2) and linear in the vertex weights
w. The forward pass runs fe_assemble_stiff_wmass; the backward pass runs fe_adjoint_stiff_wmass,
which turns the upstream gradients on the CSR values (G_S, G_M) into dL/dq [2, nq] and
dL/dw [nq] in one launch. Both run on the GPU; there is no CPU path.

    mesh = feasm.Mesh(q0, me)
    pat = feasm.Pattern(mesh, gather=True)           # the adjoint needs the element-to-nnz map
    asm = StiffWMass(mesh, pat)
    S, M = asm(q, w)                                 # q [2, nq], w [nq] float64 CUDA, requires_grad
    loss = (G_S * S).sum() + (G_M * M).sum()
    loss.backward()                                  # q.grad, w.grad
"""
from __future__ import annotations

import torch

from . import feasm


class _StiffWMassFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, q, w, mesh, pattern, variant, adjoint_variant):
        if not (q.is_cuda and w.is_cuda):
            raise ValueError("q and w must be CUDA tensors")
        q = q.detach().contiguous()
        w = w.detach().contiguous()
        if q.shape != (2, mesh.nq) or w.shape != (mesh.nq,):
            raise ValueError("q must be [2, nq] and w [nq]")
        mesh.set_coords(q)
        S, M = feasm.assemble_stiff_wmass(mesh, pattern, w, variant)
        ctx.save_for_backward(q, w)
        ctx.mesh, ctx.pattern, ctx.adjoint_variant = mesh, pattern, adjoint_variant
        return S, M

    @staticmethod
    def backward(ctx, gS, gM):
        q, w = ctx.saved_tensors
        mesh, pattern = ctx.mesh, ctx.pattern
        mesh.set_coords(q)                   # the mesh may have been moved since the forward pass
        gS = None if gS is None else gS.contiguous()
        gM = None if gM is None else gM.contiguous()
        dq, dw = feasm.adjoint_stiff_wmass(mesh, pattern, w, gS, gM, ctx.adjoint_variant)
        return (dq if ctx.needs_input_grad[0] else None, dw if ctx.needs_input_grad[1] else None,
                None, None, None, None)


class StiffWMass:
    """Differentiable (q, w) -> (S.values, M^[w].values) on a fixed mesh topology and pattern.

    variant: the forward scatter (FE_VARIANT_ROW by default). The backward pass uses the
    deterministic gather adjoint when the pattern was built with gather=True, else the atomic one.
    The pattern must carry the element-to-nnz map (Pattern(..., map=True), the default).
    """

    def __init__(self, mesh: feasm.Mesh, pattern: feasm.Pattern, variant: int = feasm.ROW):
        if pattern.map is None:
            raise ValueError("the adjoint needs a pattern built with map=True")
        self.mesh, self.pattern, self.variant = mesh, pattern, variant
        self.adjoint_variant = feasm.GATHER if pattern.gather else feasm.ATOMIC

    def __call__(self, q: torch.Tensor, w: torch.Tensor):
        return _StiffWMassFn.apply(q, w, self.mesh, self.pattern, self.variant, self.adjoint_variant)
