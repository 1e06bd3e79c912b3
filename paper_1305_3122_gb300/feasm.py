"""Python binding of ``libfeasm.so`` (the C ABI declared in ``include/feasm.h``).

Argument marshalling only: every step of the assembly runs in the CUDA library. PyTorch
provides device memory (tensors) and streams (``torch.cuda.current_stream()``); the CSR
structure owned by a pattern is exposed as zero-copy int32 CUDA tensors.

If the library has not been built (``paper_1305_3122_gb300.build.build()``), or no GPU is
present, the calls raise; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# FEASM_LIBRARY selects another build of the same library (the bounds-checked one, say)
LIB_PATH = os.environ.get("FEASM_LIBRARY") or os.path.join(_HERE, "libfeasm.so")

FE_OK = 0
PTR_HOST, PTR_DEVICE, PTR_DEVICE_BORROW = 0, 1, 2
ATOMIC, GATHER, ROW = 0, 1, 2
PATTERN_DEFAULT, PATTERN_GATHER, PATTERN_MAP = 0, 1, 2

_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_D = ctypes.c_double
_INT = ctypes.c_int

# name -> (restype, argtypes); mirrors include/feasm.h
SIGNATURES = {
    "fe_mesh_create": (_INT, [_I32, _I32, _P, _P, _INT, _P, ctypes.POINTER(_P)]),
    "fe_mesh_set_coords": (_INT, [_P, _P, _INT, _P]),
    "fe_mesh_check": (_INT, [_P, _P]),
    "fe_mesh_info": (_INT, [_P, ctypes.POINTER(_I32), ctypes.POINTER(_I32)]),
    "fe_mesh_destroy": (None, [_P]),
    "fe_pattern_build": (_INT, [_P, _INT, _INT, _P, ctypes.POINTER(_P)]),
    "fe_pattern_info": (_INT, [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64), ctypes.POINTER(_P), ctypes.POINTER(_P)]),
    "fe_pattern_map": (_INT, [_P, ctypes.POINTER(_P), ctypes.POINTER(_I64)]),
    "fe_pattern_destroy": (None, [_P]),
    "fe_mesh_create_part": (_INT, [_I32, _I32, _P, _P, _INT, _I32, _I32, _P, ctypes.POINTER(_P)]),
    "fe_pattern_build_part": (_INT, [_P, _I32, _I32, _P, ctypes.POINTER(_P)]),
    "fe_assemble_mass": (_INT, [_P, _P, _INT, _P, _I64, _P]),
    "fe_assemble_wmass": (_INT, [_P, _P, _P, _INT, _P, _I64, _P]),
    "fe_assemble_stiff": (_INT, [_P, _P, _INT, _P, _I64, _P]),
    "fe_assemble_stiff_wmass": (_INT, [_P, _P, _P, _INT, _P, _P, _I64, _P]),
    "fe_assemble_elas": (_INT, [_P, _P, _D, _D, _INT, _P, _I64, _P]),
    "fe_assemble_stiff_wmass_noalloc": (_INT, [_P, _P, _P, _P, _P, _I64, _P]),
    "fe_adjoint_stiff_wmass": (_INT, [_P, _P, _P, _P, _P, _INT, _P, _P, _P]),
    "fe_csr_drop_zeros": (_INT, [_I64, _P, _P, _P, _P, _P, _P, _I64, ctypes.POINTER(_I64), _P]),
    "fe_tet_mesh_create": (_INT, [_I32, _I32, _P, _P, _INT, _P, ctypes.POINTER(_P)]),
    "fe_tet_mesh_destroy": (None, [_P]),
    "fe_tet_pattern_build": (_INT, [_P, _INT, _P, ctypes.POINTER(_P)]),
    "fe_tet_pattern_info": (_INT, [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64), ctypes.POINTER(_P), ctypes.POINTER(_P)]),
    "fe_tet_pattern_map": (_INT, [_P, ctypes.POINTER(_P), ctypes.POINTER(_I64)]),
    "fe_tet_pattern_destroy": (None, [_P]),
    "fe_tet_assemble": (_INT, [_P, _P, _INT, _P, _INT, _P, _I64, _P]),
    "fe_tet_pattern_elas_info": (_INT, [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64), ctypes.POINTER(_P), ctypes.POINTER(_P)]),
    "fe_tet_assemble_elas": (_INT, [_P, _P, _D, _D, _INT, _P, _I64, _P]),
    "fe_p2_pattern_build": (_INT, [_P, _P, _INT, _P, ctypes.POINTER(_P)]),
    "fe_p2_pattern_info": (_INT, [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64), ctypes.POINTER(_P), ctypes.POINTER(_P)]),
    "fe_p2_pattern_dofs": (_INT, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_I64)]),
    "fe_p2_pattern_destroy": (None, [_P]),
    "fe_p2_assemble": (_INT, [_P, _P, _INT, _INT, _P, _I64, _P]),
    "fe_p3_pattern_build": (_INT, [_P, _P, _INT, _P, ctypes.POINTER(_P)]),
    "fe_p3_pattern_info": (_INT, [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64), ctypes.POINTER(_P), ctypes.POINTER(_P)]),
    "fe_p3_pattern_dofs": (_INT, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_I64)]),
    "fe_p3_pattern_destroy": (None, [_P]),
    "fe_p3_assemble": (_INT, [_P, _P, _INT, _INT, _P, _I64, _P]),
    "fe_assemble_stiff_wmass_host": (_INT, [_I32, _I32, _P, _P, _P, _P, _P, _P, _P, _I64, ctypes.POINTER(_I64), _P]),
    "fe_batch_create": (_INT, [_I32, _P, _P, ctypes.POINTER(_P)]),
    "fe_batch_tune": (_INT, [_P, _P, _P, _P, ctypes.POINTER(_I32), ctypes.POINTER(_I32)]),
    "fe_batch_tune_cached": (_INT, [_P, ctypes.c_char_p, _P, _P, _P, ctypes.POINTER(_I32), ctypes.POINTER(_I32),
                                    ctypes.POINTER(_I32)]),
    "fe_batch_set_shape": (_INT, [_P, _I32, _I32]),
    "fe_batch_configure": (_INT, [_P, _I32, _I32, _I32]),
    "fe_batch_get_config": (_INT, [_P, ctypes.POINTER(_I32), ctypes.POINTER(_I32), ctypes.POINTER(_I32)]),
    "fe_batch_assemble_stiff_mass": (_INT, [_P, _P, _P, _P]),
    "fe_batch_assemble_stiff_mass_plain": (_INT, [_P, _P, _P, _P]),
    "fe_batch_destroy": (None, [_P]),
    "fe_profile_enable": (_INT, [_INT]),
    "fe_profile_reset": (_INT, []),
    "fe_profile_read": (_INT, [_I32, _P, _P, _P, ctypes.POINTER(_I32)]),
    "fe_measure_fp64_rate": (_INT, [ctypes.POINTER(_D), _P]),
    "fe_debug_fail_alloc": (None, [_I64]),
    "fe_debug_pool_used": (_INT, [ctypes.POINTER(_I64)]),
    "fe_debug_bounds": (_INT, [ctypes.POINTER(_I32), ctypes.POINTER(_I64), _I32]),
    "fe_status_string": (ctypes.c_char_p, [_INT]),
    "fe_last_error": (ctypes.c_char_p, []),
}


class FeasmError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(message)
        self.status = status


_lib = None


def lib() -> ctypes.CDLL:
    """The loaded CUDA library (raises if it is missing: build it first)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build the CUDA library with "
                               "paper_1305_3122_gb300.build.build() (needs nvcc)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status: int, what: str):
    if status != FE_OK:
        L = lib()
        raise FeasmError(status, f"{what}: {L.fe_status_string(status).decode()}: {L.fe_last_error().decode()}")


_raw_stream = getattr(torch._C, "_cuda_getCurrentRawStream", None)


def _stream(stream=None) -> int:
    """The cudaStream_t to pass: the given torch stream's, else the current stream's (read
    without building a torch.cuda.Stream object when PyTorch offers that, which saves host time
    in every call)."""
    if stream is not None:
        return stream.cuda_stream
    if _raw_stream is not None:
        return _raw_stream(torch.cuda.current_device())
    return torch.cuda.current_stream().cuda_stream


def _dptr(t: torch.Tensor | None, dtype: torch.dtype, what: str) -> int | None:
    if t is None:
        return None
    if not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"{what} must be a contiguous CUDA tensor of dtype {dtype}")
    return t.data_ptr()


class _DevView:
    """Zero-copy view of library-owned device memory (keeps its owner alive)."""

    def __init__(self, ptr: int, n: int, typestr: str, owner):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr or 0, False),
                                         "version": 3, "strides": None}
        self.owner = owner


def _view_i32(ptr: int, n: int, owner) -> torch.Tensor:
    if n == 0:
        return torch.empty(0, dtype=torch.int32, device="cuda")
    return torch.as_tensor(_DevView(ptr, n, "<i4", owner), device="cuda")


class Mesh:
    """A triangulation: q [2, nq] float64 and me [3, nme] int32 (0-based, counter-clockwise).

    q and me may be CUDA tensors, CPU tensors or numpy arrays; host inputs are copied by the
    library (FE_PTR_HOST). Section 2 of the paper.
    """

    def __init__(self, q, me, stream=None, borrow: bool = False):
        """borrow: with CUDA tensors, use me in place (FE_PTR_DEVICE_BORROW) instead of copying
        it; the mesh keeps a reference to the tensor, which must not be modified meanwhile."""
        L = lib()
        self._h = None
        self._me_ref = None
        if isinstance(q, torch.Tensor) and q.is_cuda:
            qd = q.contiguous()
            med = me.contiguous()
            kind = PTR_DEVICE_BORROW if borrow else PTR_DEVICE
            if borrow:
                self._me_ref = med
            qp = _dptr(qd, torch.float64, "q")
            mp = _dptr(med, torch.int32, "me")
        else:
            qd = np.ascontiguousarray(q.cpu().numpy() if isinstance(q, torch.Tensor) else q, dtype=np.float64)
            med = np.ascontiguousarray(me.cpu().numpy() if isinstance(me, torch.Tensor) else me, dtype=np.int32)
            kind = PTR_HOST
            qp = qd.ctypes.data
            mp = med.ctypes.data
        if qd.shape[0] != 2 or med.shape[0] != 3:
            raise ValueError("q must be [2, nq] and me must be [3, nme]")
        self.nq, self.nme = int(qd.shape[1]), int(med.shape[1])
        h = _P()
        _check(L.fe_mesh_create(self.nq, self.nme, qp, mp, kind, _stream(stream), ctypes.byref(h)), "fe_mesh_create")
        self._h = h

    @classmethod
    def part(cls, q, me, row_begin: int, row_end: int, stream=None) -> "Mesh":
        """A rank's share of a row partition (fe_mesh_create_part): the triangles of the global
        mesh (q [2, nq], me [3, nme], host or CUDA) that touch the owned vertices
        [row_begin, row_end). The library numbers the part's vertices locally; every id it takes
        or returns is global (nq is the global count, weights have nq entries, set_coords takes
        the global q, windows list global columns)."""
        self = cls.__new__(cls)
        self._h = None
        self._me_ref = None
        if isinstance(q, torch.Tensor) and q.is_cuda:
            qd, med = q.contiguous(), me.contiguous()
            qp, mp, kind = _dptr(qd, torch.float64, "q"), _dptr(med, torch.int32, "me"), PTR_DEVICE
        else:
            qd = np.ascontiguousarray(q.cpu().numpy() if isinstance(q, torch.Tensor) else q, dtype=np.float64)
            med = np.ascontiguousarray(me.cpu().numpy() if isinstance(me, torch.Tensor) else me, dtype=np.int32)
            qp, mp, kind = qd.ctypes.data, med.ctypes.data, PTR_HOST
        if qd.shape[0] != 2 or med.shape[0] != 3:
            raise ValueError("q must be [2, nq] and me must be [3, nme]")
        nq, nme_global = int(qd.shape[1]), int(med.shape[1])
        h = _P()
        _check(lib().fe_mesh_create_part(nq, nme_global, qp, mp, kind, int(row_begin), int(row_end), _stream(stream),
                                         ctypes.byref(h)), "fe_mesh_create_part")
        self._h = h
        n1, n2 = _I32(), _I32()
        _check(lib().fe_mesh_info(h, ctypes.byref(n1), ctypes.byref(n2)), "fe_mesh_info")
        self.nq, self.nme = n1.value, n2.value
        self.rows = (int(row_begin), int(row_end))
        return self

    @property
    def handle(self):
        return self._h

    def set_coords(self, q: torch.Tensor, stream=None):
        if q.is_cuda:
            _check(lib().fe_mesh_set_coords(self._h, _dptr(q.contiguous(), torch.float64, "q"), PTR_DEVICE,
                                            _stream(stream)), "fe_mesh_set_coords")
        else:
            qh = np.ascontiguousarray(q.numpy(), dtype=np.float64)
            _check(lib().fe_mesh_set_coords(self._h, qh.ctypes.data, PTR_HOST, _stream(stream)), "fe_mesh_set_coords")

    def check(self, stream=None):
        _check(lib().fe_mesh_check(self._h, _stream(stream)), "fe_mesh_check")

    def close(self):
        """Release the device copies now (also done on garbage collection)."""
        if getattr(self, "_h", None) and _lib is not None:
            _lib.fe_mesh_destroy(self._h)
        self._h = None
        self._me_ref = None

    def __del__(self):
        self.close()


class Pattern:
    """CSR structure and element-to-nnz map of a mesh (fe_pattern_build)."""

    def __init__(self, mesh: Mesh, dofs: int = 1, gather: bool = False, map: bool = True, stream=None,
                 rows: tuple[int, int] | None = None):
        """gather: also build what FE_VARIANT_GATHER needs; map: also the element-to-nnz map
        (FE_VARIANT_ATOMIC, the adjoint, atomic batches). FE_VARIANT_ROW works with any pattern.
        rows=(begin, end): only those rows (fe_pattern_build_part; scalar, no map, FE_VARIANT_ROW)."""
        h = _P()
        if rows is not None:
            gather, map = False, False
            _check(lib().fe_pattern_build_part(mesh.handle, int(rows[0]), int(rows[1]), _stream(stream),
                                               ctypes.byref(h)), "fe_pattern_build_part")
        else:
            flags = (PATTERN_GATHER if gather else 0) | (PATTERN_MAP if map else 0)
            _check(lib().fe_pattern_build(mesh.handle, dofs, flags, _stream(stream), ctypes.byref(h)), "fe_pattern_build")
        self.rows = rows
        self._h = h
        self.mesh = mesh
        self.dofs = dofs
        self.gather = gather
        n_rows, nnz, rp, ci = _I64(), _I64(), _P(), _P()
        _check(lib().fe_pattern_info(h, ctypes.byref(n_rows), ctypes.byref(nnz), ctypes.byref(rp), ctypes.byref(ci)),
               "fe_pattern_info")
        self.n_rows, self.nnz = n_rows.value, nnz.value
        self._rp, self._ci = rp.value, ci.value
        self._map = None
        if map or gather:
            mp, ml = _P(), _I64()
            _check(lib().fe_pattern_map(h, ctypes.byref(mp), ctypes.byref(ml)), "fe_pattern_map")
            self._map = (mp.value, ml.value)
        self._views = {}

    # The CSR arrays and the map are zero-copy views of the pattern's device memory, made on
    # first access (making a view costs tens of microseconds of host time, which a build that is
    # only used through the library's own calls need not pay).
    def _view(self, key, ptr, n):
        v = self._views.get(key)
        if v is None:
            v = self._views[key] = _view_i32(ptr, n, self)
        return v

    @property
    def row_ptr(self) -> torch.Tensor:
        return self._view("row_ptr", self._rp, self.n_rows + 1)

    @property
    def col_idx(self) -> torch.Tensor:
        return self._view("col_idx", self._ci, self.nnz)

    @property
    def map(self) -> torch.Tensor | None:
        return None if self._map is None else self._view("map", *self._map)

    @property
    def handle(self):
        return self._h

    def new_values(self) -> torch.Tensor:
        return torch.empty(self.nnz, dtype=torch.float64, device="cuda")

    def to_sparse_csr(self, values: torch.Tensor) -> torch.Tensor:
        n_cols = self.mesh.nq * self.dofs if self.rows is not None else self.n_rows
        return torch.sparse_csr_tensor(self.row_ptr.long(), self.col_idx.long(), values,
                                       size=(self.n_rows, n_cols))

    def close(self):
        """Release the pattern's device arrays now (views of them become invalid)."""
        if getattr(self, "_h", None) and _lib is not None:
            _lib.fe_pattern_destroy(self._h)
        self._h = None

    def __del__(self):
        self.close()


def _values(pattern: Pattern, out: torch.Tensor | None) -> torch.Tensor:
    out = pattern.new_values() if out is None else out
    _dptr(out, torch.float64, "values")
    return out


TET_MASS, TET_WMASS, TET_STIFF = 0, 1, 2
TET_PATTERN_ELAS = 4


class TetMesh:
    """A tetrahedral mesh: q [3, nq] float64 and me [4, nme] int32 (0-based, positive volume
    det[p1-p0 | p2-p0 | p3-p0] > 0). Inputs as for Mesh (CUDA tensors, CPU tensors or numpy)."""

    def __init__(self, q, me, stream=None, borrow: bool = False):
        L = lib()
        self._h = None
        self._me_ref = None
        if isinstance(q, torch.Tensor) and q.is_cuda:
            qd, med = q.contiguous(), me.contiguous()
            kind = PTR_DEVICE_BORROW if borrow else PTR_DEVICE
            if borrow:
                self._me_ref = med
            qp, mp = _dptr(qd, torch.float64, "q"), _dptr(med, torch.int32, "me")
        else:
            qd = np.ascontiguousarray(q.cpu().numpy() if isinstance(q, torch.Tensor) else q, dtype=np.float64)
            med = np.ascontiguousarray(me.cpu().numpy() if isinstance(me, torch.Tensor) else me, dtype=np.int32)
            kind = PTR_HOST
            qp, mp = qd.ctypes.data, med.ctypes.data
        if qd.shape[0] != 3 or med.shape[0] != 4:
            raise ValueError("q must be [3, nq] and me must be [4, nme]")
        self.nq, self.nme = int(qd.shape[1]), int(med.shape[1])
        h = _P()
        _check(L.fe_tet_mesh_create(self.nq, self.nme, qp, mp, kind, _stream(stream), ctypes.byref(h)),
               "fe_tet_mesh_create")
        self._h = h

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.fe_tet_mesh_destroy(self._h)
        self._h = None
        self._me_ref = None

    def __del__(self):
        self.close()


class TetPattern:
    """CSR structure and element-to-nnz map (map[16k + 4 il + jl]) of a tetrahedral mesh; with
    elas=True also the 3-D elasticity structure (rows 3i + s): elas_row_ptr, elas_col_idx."""

    def __init__(self, mesh: TetMesh, gather: bool = False, stream=None, elas: bool = False):
        h = _P()
        flags = (PATTERN_GATHER if gather else 0) | (TET_PATTERN_ELAS if elas else 0)
        _check(lib().fe_tet_pattern_build(mesh.handle, flags, _stream(stream), ctypes.byref(h)), "fe_tet_pattern_build")
        self._h = h
        self.mesh = mesh
        self.gather = gather
        self.elas = elas
        if elas:
            n3, z3, rp3, ci3 = _I64(), _I64(), _P(), _P()
            _check(lib().fe_tet_pattern_elas_info(h, ctypes.byref(n3), ctypes.byref(z3), ctypes.byref(rp3), ctypes.byref(ci3)),
                   "fe_tet_pattern_elas_info")
            self.elas_n_rows, self.elas_nnz = n3.value, z3.value
            self.elas_row_ptr = _view_i32(rp3.value, self.elas_n_rows + 1, self)
            self.elas_col_idx = _view_i32(ci3.value, self.elas_nnz, self)
        n_rows, nnz, rp, ci = _I64(), _I64(), _P(), _P()
        _check(lib().fe_tet_pattern_info(h, ctypes.byref(n_rows), ctypes.byref(nnz), ctypes.byref(rp), ctypes.byref(ci)),
               "fe_tet_pattern_info")
        self.n_rows, self.nnz = n_rows.value, nnz.value
        self.row_ptr = _view_i32(rp.value, self.n_rows + 1, self)
        self.col_idx = _view_i32(ci.value, self.nnz, self)
        mp, ml = _P(), _I64()
        _check(lib().fe_tet_pattern_map(h, ctypes.byref(mp), ctypes.byref(ml)), "fe_tet_pattern_map")
        self.map = _view_i32(mp.value, ml.value, self)

    @property
    def handle(self):
        return self._h

    def new_values(self) -> torch.Tensor:
        return torch.empty(self.nnz, dtype=torch.float64, device="cuda")

    def close(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.fe_tet_pattern_destroy(self._h)
        self._h = None

    def __del__(self):
        self.close()


def tet_assemble(mesh: TetMesh, pattern: TetPattern, kind: int, w: torch.Tensor | None = None, variant: int = ATOMIC,
                 out=None, stream=None) -> torch.Tensor:
    """Values of M (TET_MASS), M^w (TET_WMASS, w [nq] float64 CUDA) or S (TET_STIFF) of a
    tetrahedral mesh on the pattern's CSR structure (fe_tet_assemble)."""
    out = pattern.new_values() if out is None else out
    if out.dtype != torch.float64 or not out.is_cuda or not out.is_contiguous():
        raise ValueError("out must be a contiguous float64 CUDA tensor")
    _check(lib().fe_tet_assemble(mesh.handle, pattern.handle, kind, _dptr(w, torch.float64, "w"), variant,
                                 out.data_ptr(), out.numel(), _stream(stream)), "fe_tet_assemble")
    return out


def tet_assemble_elas(mesh: TetMesh, pattern: TetPattern, lam: float, mu: float, variant: int = ATOMIC, out=None,
                      stream=None) -> torch.Tensor:
    """Values of the 3-D elasticity matrix (dofs 3v + s) on the pattern's elasticity structure
    (fe_tet_assemble_elas; the pattern needs elas=True, and gather=True for GATHER)."""
    if not getattr(pattern, "elas", False):
        raise ValueError("the pattern was built without elas=True")
    out = torch.empty(pattern.elas_nnz, dtype=torch.float64, device="cuda") if out is None else out
    if out.dtype != torch.float64 or not out.is_cuda or not out.is_contiguous():
        raise ValueError("out must be a contiguous float64 CUDA tensor")
    _check(lib().fe_tet_assemble_elas(mesh.handle, pattern.handle, float(lam), float(mu), variant, out.data_ptr(),
                                      out.numel(), _stream(stream)), "fe_tet_assemble_elas")
    return out


P2_MASS, P2_STIFF = 0, 1


class P2Pattern:
    """P2 (quadratic) dofs, CSR structure and map of a triangle mesh (fe_p2_pattern_build): vertex i
    is dof i, the edges follow in ascending (smaller id, larger id) order. Built from the mesh's
    scalar pattern, whose structure numbers the edges. gather=True adds the row lists of the
    deterministic variant (GATHER)."""

    def __init__(self, mesh: Mesh, pattern: Pattern, gather: bool = False, stream=None):
        h = _P()
        flags = PATTERN_GATHER if gather else 0
        _check(lib().fe_p2_pattern_build(mesh.handle, pattern.handle, flags, _stream(stream), ctypes.byref(h)),
               "fe_p2_pattern_build")
        self._h = h
        self.mesh = mesh
        n, nnz, rp, ci = _I64(), _I64(), _P(), _P()
        _check(lib().fe_p2_pattern_info(h, ctypes.byref(n), ctypes.byref(nnz), ctypes.byref(rp), ctypes.byref(ci)),
               "fe_p2_pattern_info")
        self.n_rows, self.nnz = n.value, nnz.value
        self.row_ptr = _view_i32(rp.value, self.n_rows + 1, self)
        self.col_idx = _view_i32(ci.value, self.nnz, self)
        ed, mp, ne = _P(), _P(), _I64()
        _check(lib().fe_p2_pattern_dofs(h, ctypes.byref(ed), ctypes.byref(mp), ctypes.byref(ne)), "fe_p2_pattern_dofs")
        self.n_edges = ne.value
        self.edof = _view_i32(ed.value, 6 * mesh.nme, self)
        self.map = _view_i32(mp.value, 36 * mesh.nme, self)

    @property
    def handle(self):
        return self._h

    def new_values(self) -> torch.Tensor:
        return torch.empty(self.nnz, dtype=torch.float64, device="cuda")

    def close(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.fe_p2_pattern_destroy(self._h)
        self._h = None

    def __del__(self):
        self.close()


def p2_assemble(mesh: Mesh, pattern: P2Pattern, kind: int, out=None, stream=None, variant: int = ATOMIC) -> torch.Tensor:
    """Values of the P2 mass (P2_MASS) or stiffness (P2_STIFF) on the P2 pattern (fe_p2_assemble),
    by FP64 atomics (ATOMIC) or by ordered row sums (GATHER, a pattern built with gather=True)."""
    out = pattern.new_values() if out is None else out
    if out.dtype != torch.float64 or not out.is_cuda or not out.is_contiguous():
        raise ValueError("out must be a contiguous float64 CUDA tensor")
    _check(lib().fe_p2_assemble(mesh.handle, pattern.handle, kind, variant, out.data_ptr(), out.numel(),
                                _stream(stream)), "fe_p2_assemble")
    return out


P3_MASS, P3_STIFF = 0, 1


class P3Pattern:
    """P3 (cubic) dofs, CSR structure and map of a triangle mesh (fe_p3_pattern_build): vertex i is
    dof i; edge e owns dofs nq + 2e and nq + 2e + 1 (the node nearer its smaller vertex id first);
    triangle k's bubble is dof nq + 2 nE + k. Built from the mesh's scalar pattern, whose structure
    numbers the edges. gather=True adds the row lists of the deterministic variant (GATHER)."""

    def __init__(self, mesh: Mesh, pattern: Pattern, gather: bool = False, stream=None):
        h = _P()
        flags = PATTERN_GATHER if gather else 0
        _check(lib().fe_p3_pattern_build(mesh.handle, pattern.handle, flags, _stream(stream), ctypes.byref(h)),
               "fe_p3_pattern_build")
        self._h = h
        self.mesh = mesh
        n, nnz, rp, ci = _I64(), _I64(), _P(), _P()
        _check(lib().fe_p3_pattern_info(h, ctypes.byref(n), ctypes.byref(nnz), ctypes.byref(rp), ctypes.byref(ci)),
               "fe_p3_pattern_info")
        self.n_rows, self.nnz = n.value, nnz.value
        self.row_ptr = _view_i32(rp.value, self.n_rows + 1, self)
        self.col_idx = _view_i32(ci.value, self.nnz, self)
        ed, mp, ne = _P(), _P(), _I64()
        _check(lib().fe_p3_pattern_dofs(h, ctypes.byref(ed), ctypes.byref(mp), ctypes.byref(ne)), "fe_p3_pattern_dofs")
        self.n_edges = ne.value
        self.edof = _view_i32(ed.value, 10 * mesh.nme, self)
        self.map = _view_i32(mp.value, 100 * mesh.nme, self)

    @property
    def handle(self):
        return self._h

    def new_values(self) -> torch.Tensor:
        return torch.empty(self.nnz, dtype=torch.float64, device="cuda")

    def close(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.fe_p3_pattern_destroy(self._h)
        self._h = None

    def __del__(self):
        self.close()


def p3_assemble(mesh: Mesh, pattern: P3Pattern, kind: int, out=None, stream=None, variant: int = ATOMIC) -> torch.Tensor:
    """Values of the P3 mass (P3_MASS) or stiffness (P3_STIFF) on the P3 pattern (fe_p3_assemble),
    by FP64 atomics (ATOMIC) or by ordered row sums (GATHER, a pattern built with gather=True)."""
    out = pattern.new_values() if out is None else out
    if out.dtype != torch.float64 or not out.is_cuda or not out.is_contiguous():
        raise ValueError("out must be a contiguous float64 CUDA tensor")
    _check(lib().fe_p3_assemble(mesh.handle, pattern.handle, kind, variant, out.data_ptr(), out.numel(),
                                _stream(stream)), "fe_p3_assemble")
    return out


def drop_zeros(row_ptr: torch.Tensor, col_idx: torch.Tensor, values: torch.Tensor, stream=None):
    """CSR (row_ptr, col_idx, values) without the entries equal to 0.0, as Matlab's sparse()
    stores them (fe_csr_drop_zeros): int32 / int32 / float64 CUDA tensors in, new ones out."""
    n_rows = row_ptr.numel() - 1
    if n_rows < 0 or col_idx.numel() != values.numel():
        raise ValueError("row_ptr must have n_rows + 1 entries and col_idx / values the same length")
    rp = torch.empty(n_rows + 1, dtype=torch.int32, device="cuda")
    cap = values.numel()
    ci = torch.empty(max(cap, 1), dtype=torch.int32, device="cuda")
    va = torch.empty(max(cap, 1), dtype=torch.float64, device="cuda")
    kept = _I64(0)
    if cap == 0:   # no entry: pass one-element buffers rather than null pointers
        col_idx = torch.zeros(1, dtype=torch.int32, device="cuda")
        values = torch.zeros(1, dtype=torch.float64, device="cuda")
    _check(lib().fe_csr_drop_zeros(n_rows, _dptr(row_ptr, torch.int32, "row_ptr"), _dptr(col_idx, torch.int32, "col_idx"),
                                   _dptr(values, torch.float64, "values"), rp.data_ptr(), ci.data_ptr(), va.data_ptr(),
                                   cap, ctypes.byref(kept), _stream(stream)), "fe_csr_drop_zeros")
    return rp, ci[:kept.value], va[:kept.value]


def assemble_mass(mesh: Mesh, pattern: Pattern, variant: int = ATOMIC, out=None, stream=None) -> torch.Tensor:
    """Values of M (Eq. 1) on the pattern's CSR structure."""
    out = _values(pattern, out)
    _check(lib().fe_assemble_mass(mesh.handle, pattern.handle, variant, out.data_ptr(), out.numel(), _stream(stream)),
           "fe_assemble_mass")
    return out


def assemble_wmass(mesh: Mesh, pattern: Pattern, w: torch.Tensor, variant: int = ATOMIC, out=None,
                   stream=None) -> torch.Tensor:
    """Values of M^[w] (Eq. 2), w = vertex values [nq] float64 on the GPU."""
    out = _values(pattern, out)
    _check(lib().fe_assemble_wmass(mesh.handle, pattern.handle, _dptr(w, torch.float64, "w"), variant, out.data_ptr(),
                                   out.numel(), _stream(stream)), "fe_assemble_wmass")
    return out


def assemble_stiff(mesh: Mesh, pattern: Pattern, variant: int = ATOMIC, out=None, stream=None) -> torch.Tensor:
    """Values of S (Eq. 3)."""
    out = _values(pattern, out)
    _check(lib().fe_assemble_stiff(mesh.handle, pattern.handle, variant, out.data_ptr(), out.numel(),
                                   _stream(stream)), "fe_assemble_stiff")
    return out


def assemble_stiff_wmass(mesh: Mesh, pattern: Pattern, w: torch.Tensor, variant: int = ATOMIC, out_S=None,
                         out_M=None, stream=None) -> tuple[torch.Tensor, torch.Tensor]:
    """Values of S and M^[w] in one pass over the triangles."""
    out_S = _values(pattern, out_S)
    out_M = _values(pattern, out_M)
    cap = min(out_S.numel(), out_M.numel())
    _check(lib().fe_assemble_stiff_wmass(mesh.handle, pattern.handle, _dptr(w, torch.float64, "w"), variant,
                                         out_S.data_ptr(), out_M.data_ptr(), cap, _stream(stream)),
           "fe_assemble_stiff_wmass")
    return out_S, out_M


def assemble_elas(mesh: Mesh, pattern: Pattern, lam: float, mu: float, variant: int = ATOMIC, out=None,
                  stream=None) -> torch.Tensor:
    """Values of the plane-elasticity K (Section 7); pattern built with dofs=2."""
    out = _values(pattern, out)
    _check(lib().fe_assemble_elas(mesh.handle, pattern.handle, float(lam), float(mu), variant, out.data_ptr(),
                                  out.numel(), _stream(stream)), "fe_assemble_elas")
    return out


def adjoint_stiff_wmass(mesh: Mesh, pattern: Pattern, w: torch.Tensor, gS: torch.Tensor | None,
                        gM: torch.Tensor | None, variant: int = ATOMIC, stream=None):
    """(dL/dq [2, nq], dL/dw [nq]) of L = sum(gS * S.values) + sum(gM * M^[w].values)."""
    dq = torch.empty((2, mesh.nq), dtype=torch.float64, device="cuda")
    dw = torch.empty(mesh.nq, dtype=torch.float64, device="cuda")
    _check(lib().fe_adjoint_stiff_wmass(mesh.handle, pattern.handle, _dptr(w, torch.float64, "w"),
                                        _dptr(gS, torch.float64, "gS"), _dptr(gM, torch.float64, "gM"), variant,
                                        dq.data_ptr(), dw.data_ptr(), _stream(stream)), "fe_adjoint_stiff_wmass")
    return dq, dw


def measure_fp64_rate(stream=None) -> float:
    """Measured FP64 instructions per second of this GPU (fe_measure_fp64_rate)."""
    v = _D()
    _check(lib().fe_measure_fp64_rate(ctypes.byref(v), _stream(stream)), "fe_measure_fp64_rate")
    return v.value


def debug_fail_alloc(n: int):
    """Make the n-th device allocation of the library from now on fail with FE_ERR_OOM (n <= 0:
    off); a test hook for the error paths (fe_debug_fail_alloc)."""
    lib().fe_debug_fail_alloc(int(n))


def debug_pool_used() -> int:
    """Bytes currently allocated from the library's device memory pool (fe_debug_pool_used)."""
    v = _I64()
    _check(lib().fe_debug_pool_used(ctypes.byref(v)), "fe_debug_pool_used")
    return v.value


def debug_bounds(reset: bool = False) -> tuple[bool, int]:
    """(built with bounds checks, out-of-range derived indices counted so far) (fe_debug_bounds)."""
    c, v = _I32(), _I64()
    _check(lib().fe_debug_bounds(ctypes.byref(c), ctypes.byref(v), 1 if reset else 0), "fe_debug_bounds")
    return bool(c.value), v.value


def profile_enable(on: bool = True):
    """Turn the library's per-kernel event timing on or off (process-wide)."""
    _check(lib().fe_profile_enable(1 if on else 0), "fe_profile_enable")


def profile_reset():
    _check(lib().fe_profile_reset(), "fe_profile_reset")


def profile_read() -> dict[str, tuple[float, int]]:
    """{kernel name: (total device ms, launches)} accumulated since the last reset."""
    L = lib()
    n = _I32()
    _check(L.fe_profile_read(0, None, None, None, ctypes.byref(n)), "fe_profile_read")
    cap = max(n.value, 1)
    names = ctypes.create_string_buffer(64 * cap)
    ms = (_D * cap)()
    cnt = (_I64 * cap)()
    _check(L.fe_profile_read(cap, names, ms, cnt, ctypes.byref(n)), "fe_profile_read")
    out = {}
    for i in range(min(n.value, cap)):
        nm = names.raw[64 * i:64 * (i + 1)].split(b"\0", 1)[0].decode()
        out[nm] = (ms[i], cnt[i])
    return out


class Batch:
    """S and M of many meshes in one persistent, graph-replayed launch (fe_batch_*)."""

    def __init__(self, meshes: list[Mesh], patterns: list[Pattern]):
        n = len(meshes)
        mh = (_P * max(n, 1))(*[m.handle for m in meshes])
        ph = (_P * max(n, 1))(*[p.handle for p in patterns])
        h = _P()
        _check(lib().fe_batch_create(n, mh, ph, ctypes.byref(h)), "fe_batch_create")
        self._h = h
        self.meshes, self.patterns = meshes, patterns
        self.n = n
        self.S = [p.new_values() for p in patterns]
        self.M = [p.new_values() for p in patterns]
        self._tables = ((_P * max(n, 1))(*[t.data_ptr() for t in self.S]),
                        (_P * max(n, 1))(*[t.data_ptr() for t in self.M]))

    def tune(self, stream=None, cache: str | None = None) -> tuple[int, int]:
        """Times the candidates and keeps the fastest (fe_batch_tune). With cache (a file path, or
        "" for the path in FEASM_TUNE_CACHE) a cached choice for this device and batch shape is
        used without timing (fe_batch_tune_cached); self.from_cache tells which happened."""
        b, t, fc = _I32(), _I32(), _I32()
        if cache is None:
            _check(lib().fe_batch_tune(self._h, self._tables[0], self._tables[1], _stream(stream), ctypes.byref(b),
                                       ctypes.byref(t)), "fe_batch_tune")
        else:
            _check(lib().fe_batch_tune_cached(self._h, cache.encode(), self._tables[0], self._tables[1],
                                              _stream(stream), ctypes.byref(b), ctypes.byref(t), ctypes.byref(fc)),
                   "fe_batch_tune_cached")
        self.from_cache = bool(fc.value)
        return b.value, t.value

    def set_shape(self, block: int, tile: int):
        _check(lib().fe_batch_set_shape(self._h, block, tile), "fe_batch_set_shape")

    def configure(self, variant: int, block: int, tile: int):
        """Scheme (ROW or ATOMIC), block size and tile size; recaptures the graph."""
        _check(lib().fe_batch_configure(self._h, variant, block, tile), "fe_batch_configure")

    def config(self) -> tuple[int, int, int]:
        """(variant, block, tile) currently captured."""
        v, b, t = _I32(), _I32(), _I32()
        _check(lib().fe_batch_get_config(self._h, ctypes.byref(v), ctypes.byref(b), ctypes.byref(t)),
               "fe_batch_get_config")
        return v.value, b.value, t.value

    def assemble(self, stream=None):
        _check(lib().fe_batch_assemble_stiff_mass(self._h, self._tables[0], self._tables[1], _stream(stream)),
               "fe_batch_assemble_stiff_mass")
        return self.S, self.M

    def assemble_plain(self, stream=None):
        _check(lib().fe_batch_assemble_stiff_mass_plain(self._h, self._tables[0], self._tables[1], _stream(stream)),
               "fe_batch_assemble_stiff_mass_plain")
        return self.S, self.M

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.fe_batch_destroy(self._h)
            self._h = None


def _host_f64(a) -> np.ndarray:
    return np.ascontiguousarray(a.numpy() if isinstance(a, torch.Tensor) else a, dtype=np.float64)


def assemble_stiff_wmass_host(q, me, w, pinned_out: dict | None = None, stream=None) -> dict:
    """S and M^[w] from host arrays to host CSR arrays in one pipelined library call
    (fe_assemble_stiff_wmass_host). pinned_out may hold reusable pinned torch tensors "row_ptr",
    "col_idx", "S", "Mw" (int32 / float64); missing or too small ones are allocated (pinned)."""
    qh = _host_f64(q)
    meh = np.ascontiguousarray(me.numpy() if isinstance(me, torch.Tensor) else me, dtype=np.int32)
    wh = _host_f64(w)
    nq, nme = int(qh.shape[1]), int(meh.shape[1])
    cap = 6 * nme + nq
    outs = dict(pinned_out or {})
    want = {"row_ptr": (nq + 1, torch.int32), "col_idx": (cap, torch.int32), "S": (cap, torch.float64),
            "Mw": (cap, torch.float64)}
    for name, (n, dt) in want.items():
        t = outs.get(name)
        if t is None or t.numel() < n or t.dtype != dt:
            outs[name] = torch.empty(n, dtype=dt, pin_memory=True)
    nnz = _I64()
    _check(lib().fe_assemble_stiff_wmass_host(nq, nme, qh.ctypes.data, meh.ctypes.data, wh.ctypes.data,
                                              outs["row_ptr"].data_ptr(), outs["col_idx"].data_ptr(),
                                              outs["S"].data_ptr(), outs["Mw"].data_ptr(), cap,
                                              ctypes.byref(nnz), _stream(stream)), "fe_assemble_stiff_wmass_host")
    n = nnz.value
    res = {"row_ptr": outs["row_ptr"][: nq + 1], "col_idx": outs["col_idx"][:n], "S": outs["S"][:n],
           "Mw": outs["Mw"][:n], "nnz": n}
    if pinned_out is not None:
        pinned_out.update({k: outs[k] for k in want})
    return res


def assemble_host(kind: str, q: np.ndarray, me: np.ndarray, w: np.ndarray | None = None, lam: float = 1.0,
                  mu: float = 0.5, variant: int = ROW, pinned_out: dict | None = None, stream=None):
    """One-shot assembly from host arrays to host CSR arrays (the end-to-end call).

    kind in {"mass", "wmass", "stiff", "elas", "stiff_wmass"}. The mesh is created from host
    memory (copied by the library), the pattern built, the values assembled, and row_ptr,
    col_idx and values read back to (pinned, if given) host tensors. Returns a dict.
    "stiff_wmass" with FE_VARIANT_ROW is one pipelined library call (assemble_stiff_wmass_host).
    """
    if kind == "stiff_wmass" and variant == ROW:
        return assemble_stiff_wmass_host(q, me, w, pinned_out, stream)
    mesh = Mesh(q, me, stream=stream)
    pat = Pattern(mesh, dofs=2 if kind == "elas" else 1, gather=(variant == GATHER), map=(variant == ATOMIC),
                  stream=stream)
    vals = {}
    if kind in ("wmass", "stiff_wmass"):
        wd = torch.as_tensor(w).to("cuda", non_blocking=True)
    if kind == "mass":
        vals["values"] = assemble_mass(mesh, pat, variant, stream=stream)
    elif kind == "wmass":
        vals["values"] = assemble_wmass(mesh, pat, wd, variant, stream=stream)
    elif kind == "stiff":
        vals["values"] = assemble_stiff(mesh, pat, variant, stream=stream)
    elif kind == "elas":
        vals["values"] = assemble_elas(mesh, pat, lam, mu, variant, stream=stream)
    elif kind == "stiff_wmass":
        vals["S"], vals["Mw"] = assemble_stiff_wmass(mesh, pat, wd, variant, stream=stream)
    else:
        raise ValueError(kind)
    out = {}
    src = {"row_ptr": pat.row_ptr, "col_idx": pat.col_idx, **vals}
    for name, t in src.items():
        dst = (pinned_out or {}).get(name)
        if dst is None or dst.numel() < t.numel() or dst.dtype != t.dtype:
            dst = torch.empty(t.numel(), dtype=t.dtype, pin_memory=True)
            if pinned_out is not None:
                pinned_out[name] = dst
        dst = dst[: t.numel()]
        dst.copy_(t, non_blocking=True)
        out[name] = dst
    (stream or torch.cuda.current_stream()).synchronize()
    out["nnz"] = pat.nnz
    # release the device arrays now: the pattern's index views refer back to the pattern, so
    # without an explicit close they would wait for Python's cycle collector
    pat.close()
    mesh.close()
    return out
