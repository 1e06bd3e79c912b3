"""GB300-native P1 finite-element matrix assembly (mass, weighted mass, stiffness, plane
elasticity) behind a C-ABI CUDA library, after Cuvelier, Japhet and Scarella's vectorised
assembly (INRIA RR-8305).

Submodules: ``meshgen`` (seeded synthetic inputs), ``feasm`` (binding of the CUDA library),
``autograd`` (torch.autograd.Function around assembly and its adjoint).
"""
__all__ = ["meshgen", "feasm", "autograd"]
