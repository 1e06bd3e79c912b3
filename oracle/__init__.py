"""CPU FP64 oracle for P1 assembly (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` use this
package. It loads ``liboracle.so`` built from ``oracle.c`` with gcc (``-O2 -ffp-contract=off``,
so no multiply-add contraction changes the rounding) and wraps it for numpy arrays. It shares
nothing with the CUDA library; see ``oracle.c`` for what each routine follows in the paper.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

MASS, WMASS, STIFF, ELAS = 0, 1, 2, 3
_ERRORS = {1: "invalid argument", 2: "index out of range", 3: "repeated vertex in an element",
           4: "element not counter-clockwise (D <= 0)", 5: "out of memory", 6: "capacity"}


class OracleError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"oracle {where}: {_ERRORS.get(code, code)}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source (plain C, gcc)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        D = ctypes.c_double
        _lib.or_double_area.argtypes = [P, P]
        _lib.or_double_area.restype = D
        _lib.or_elem_mass.argtypes = [D, P]
        _lib.or_elem_wmass.argtypes = [D, P, P]
        _lib.or_elem_stiff.argtypes = [P, P, D, P]
        _lib.or_elem_elas.argtypes = [P, P, D, D, D, P]
        _lib.or_triplets.argtypes = [ctypes.c_int, I64, I64, P, P, P, D, D, P, P, P, P]
        _lib.or_sparse.argtypes = [I64, I64, I64, P, P, P, P, P, P, I64, P]
        _lib.or_assemble.argtypes = [ctypes.c_int, I64, I64, P, P, P, D, D, P, P, P, I64, P, P]
        _lib.or_adjoint.argtypes = [ctypes.c_int, I64, I64, P, P, P, P, P, P, P, P]
        _lib.or_drop_zeros.argtypes = [I64, P, P, P, P, P, P]
        _lib.or_drop_zeros.restype = I64
        _lib.or_tet_volume6.argtypes = [P, P, P]
        _lib.or_tet_volume6.restype = D
        _lib.or_tet_elem_mass.argtypes = [D, P]
        _lib.or_tet_elem_wmass.argtypes = [D, P, P]
        _lib.or_tet_elem_stiff.argtypes = [P, P, P, D, P]
        _lib.or_tet_triplets.argtypes = [ctypes.c_int, I64, I64, P, P, P, P, P, P, P]
        _lib.or_tet_assemble.argtypes = [ctypes.c_int, I64, I64, P, P, P, P, P, P, I64, P, P]
        for f in ("or_tet_triplets", "or_tet_assemble"):
            getattr(_lib, f).restype = ctypes.c_int
        _lib.or_tet_elem_elas.argtypes = [P, P, P, D, D, D, P]
        _lib.or_tet_elas_triplets.argtypes = [I64, I64, P, P, D, D, P, P, P, P]
        _lib.or_tet_elas_assemble.argtypes = [I64, I64, P, P, D, D, P, P, P, I64, P, P]
        for f in ("or_tet_elas_triplets", "or_tet_elas_assemble"):
            getattr(_lib, f).restype = ctypes.c_int
        _lib.or_p2_elem_mass.argtypes = [D, P]
        _lib.or_p2_elem_stiff.argtypes = [P, P, D, P]
        _lib.or_p2_triplets.argtypes = [ctypes.c_int, I64, I64, P, P, P, P, P, P, P]
        _lib.or_p2_assemble.argtypes = [ctypes.c_int, I64, I64, P, P, P, P, P, I64, P, P, P]
        for f in ("or_p2_triplets", "or_p2_assemble"):
            getattr(_lib, f).restype = ctypes.c_int
        _lib.or_p3_elem_mass.argtypes = [D, P]
        _lib.or_p3_elem_stiff.argtypes = [P, P, D, P]
        _lib.or_p3_triplets.argtypes = [ctypes.c_int, I64, I64, P, P, P, P, P, P, P]
        _lib.or_p3_assemble.argtypes = [ctypes.c_int, I64, I64, P, P, P, P, P, I64, P, P, P]
        for f in ("or_p3_triplets", "or_p3_assemble"):
            getattr(_lib, f).restype = ctypes.c_int
        for f in ("or_triplets", "or_sparse", "or_assemble", "or_adjoint"):
            getattr(_lib, f).restype = ctypes.c_int
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int32)


# ------------------------------------------------------------------ element matrices

def double_area(x, y) -> float:
    return lib().or_double_area(_p(_f64(x)), _p(_f64(y)))


def elem_mass(area: float) -> np.ndarray:
    E = np.empty(9)
    lib().or_elem_mass(area, _p(E))
    return E.reshape(3, 3)


def elem_wmass(area: float, w) -> np.ndarray:
    E = np.empty(9)
    lib().or_elem_wmass(area, _p(_f64(w)), _p(E))
    return E.reshape(3, 3)


def elem_stiff(x, y, area: float) -> np.ndarray:
    E = np.empty(9)
    lib().or_elem_stiff(_p(_f64(x)), _p(_f64(y)), area, _p(E))
    return E.reshape(3, 3)


def elem_elas(x, y, area: float, lam: float, mu: float) -> np.ndarray:
    E = np.empty(36)
    lib().or_elem_elas(_p(_f64(x)), _p(_f64(y)), area, lam, mu, _p(E))
    return E.reshape(6, 6)


# ------------------------------------------------------------------ assembly

def triplets(kind: int, q, me, w=None, lam: float = 1.0, mu: float = 0.5):
    """(Ig, Jg, Kg) with entry c = n*n*k + n*jl + il (element matrices stored column-wise)."""
    q, me = _f64(q), _i32(me)
    nq, nme = q.shape[1], me.shape[1]
    n = 6 if kind == ELAS else 3
    I = np.empty(n * n * nme, np.int32)
    J = np.empty_like(I)
    K = np.empty(n * n * nme)
    w = _f64(w) if w is not None else np.zeros(max(nq, 1))
    bad = ctypes.c_int64(-1)
    st = lib().or_triplets(kind, nq, nme, _p(q), _p(me), _p(w), lam, mu, _p(I), _p(J), _p(K),
                           ctypes.byref(bad))
    if st:
        raise OracleError(st, f"triplets (element {bad.value})")
    return I, J, K


def sparse(I, J, K, n_rows: int, n_cols: int):
    """CSR (row_ptr, col_idx, val) of sparse(I, J, K, n_rows, n_cols), 0-based."""
    I, J, K = _i32(I), _i32(J), _f64(K)
    nt = I.shape[0]
    row_ptr = np.empty(n_rows + 1, np.int32)
    col_idx = np.empty(max(nt, 1), np.int32)
    val = np.empty(max(nt, 1))
    nnz = ctypes.c_int64(0)
    st = lib().or_sparse(n_rows, n_cols, nt, _p(I), _p(J), _p(K), _p(row_ptr), _p(col_idx),
                         _p(val), max(nt, 1), ctypes.byref(nnz))
    if st:
        raise OracleError(st, "sparse")
    return row_ptr, col_idx[:nnz.value].copy(), val[:nnz.value].copy()


def drop_zeros(row_ptr, col_idx, val):
    """CSR without the entries equal to 0.0 (Matlab's sparse() stores no zero), order kept."""
    row_ptr, col_idx, val = _i32(row_ptr), _i32(col_idx), _f64(val)
    n_rows = row_ptr.shape[0] - 1
    nnz = int(row_ptr[-1]) if n_rows >= 0 else 0
    rp = np.empty(n_rows + 1, np.int32)
    ci = np.empty(max(nnz, 1), np.int32)
    va = np.empty(max(nnz, 1))
    n = lib().or_drop_zeros(n_rows, _p(row_ptr), _p(col_idx), _p(val), _p(rp), _p(ci), _p(va))
    return rp, ci[:n].copy(), va[:n].copy()


def assemble(kind: int, q, me, w=None, lam: float = 1.0, mu: float = 0.5):
    """Global CSR matrix (row_ptr, col_idx, val) of one kind: triplets then sparse()."""
    q, me = _f64(q), _i32(me)
    nq, nme = q.shape[1], me.shape[1]
    n = 6 if kind == ELAS else 3
    n_rows = 2 * nq if kind == ELAS else nq
    cap = max(n * n * nme, 1)
    row_ptr = np.empty(n_rows + 1, np.int32)
    col_idx = np.empty(cap, np.int32)
    val = np.empty(cap)
    w = _f64(w) if w is not None else np.zeros(max(nq, 1))
    nnz = ctypes.c_int64(0)
    bad = ctypes.c_int64(-1)
    st = lib().or_assemble(kind, nq, nme, _p(q), _p(me), _p(w), lam, mu, _p(row_ptr),
                           _p(col_idx), _p(val), cap, ctypes.byref(nnz), ctypes.byref(bad))
    if st:
        raise OracleError(st, f"assemble (element {bad.value})")
    return row_ptr, col_idx[:nnz.value].copy(), val[:nnz.value].copy()


def adjoint(kind: int, q, me, row_ptr, col_idx, G, w=None, dq=None, dw=None):
    """Accumulate dL/dq ([2, nq]) and dL/dw ([nq]) of L = sum(G * A.values) for one kind."""
    q, me = _f64(q), _i32(me)
    nq, nme = q.shape[1], me.shape[1]
    if dq is None:
        dq = np.zeros((2, nq))
    if dw is None:
        dw = np.zeros(nq)
    w = _f64(w) if w is not None else np.zeros(max(nq, 1))
    st = lib().or_adjoint(kind, nq, nme, _p(q), _p(me), _p(w), _p(_i32(row_ptr)),
                          _p(_i32(col_idx)), _p(_f64(G)), _p(dq), _p(dw))
    if st:
        raise OracleError(st, "adjoint")
    return dq, dw


def csr_to_dense(row_ptr, col_idx, val, n_cols: int) -> np.ndarray:
    n_rows = len(row_ptr) - 1
    A = np.zeros((n_rows, n_cols))
    for i in range(n_rows):
        A[i, col_idx[row_ptr[i]:row_ptr[i + 1]]] = val[row_ptr[i]:row_ptr[i + 1]]
    return A


def csr_row_values(kind: int, q, me, rows, w=None, lam: float = 1.0, mu: float = 0.5):
    """Oracle values of selected rows only, for meshes too large to assemble whole.

    For each requested row r (vertex r, or dof r for ELAS) it finds the elements containing
    the vertex, assembles just their triplets with the oracle, and applies sparse() to the
    triplets whose row is r. Returns a list of (cols, vals) in ascending column order.
    """
    q, me = _f64(q), _i32(me)
    out = []
    for r in rows:
        v = r // 2 if kind == ELAS else r
        ks = np.nonzero((me == v).any(axis=0))[0]
        sub = me[:, ks]
        I, J, K = triplets(kind, q, sub, w, lam, mu)
        sel = I == r
        n_rows = 2 * q.shape[1] if kind == ELAS else q.shape[1]
        rp, ci, va = sparse(I[sel], J[sel], K[sel], n_rows, n_rows)
        out.append((ci[rp[r]:rp[r + 1]], va[rp[r]:rp[r + 1]]))
    return out


# ------------------------------------------------------------------ tetrahedra (3-D P1)

def tet_volume6(x, y, z) -> float:
    """det [p1-p0 | p2-p0 | p3-p0] = 6 |K| (signed)."""
    return lib().or_tet_volume6(_p(_f64(x)), _p(_f64(y)), _p(_f64(z)))


def tet_elem_mass(vol: float) -> np.ndarray:
    E = np.empty(16)
    lib().or_tet_elem_mass(vol, _p(E))
    return E.reshape(4, 4)


def tet_elem_wmass(vol: float, w) -> np.ndarray:
    E = np.empty(16)
    lib().or_tet_elem_wmass(vol, _p(_f64(w)), _p(E))
    return E.reshape(4, 4)


def tet_elem_stiff(x, y, z, vol: float) -> np.ndarray:
    E = np.empty(16)
    lib().or_tet_elem_stiff(_p(_f64(x)), _p(_f64(y)), _p(_f64(z)), vol, _p(E))
    return E.reshape(4, 4)


def tet_triplets(kind: int, q, me, w=None):
    """(Ig, Jg, Kg) of a tetrahedral mesh, entry c = 16k + 4*jl + il."""
    q, me = _f64(q), _i32(me)
    nq, nme = q.shape[1], me.shape[1]
    I = np.empty(16 * nme, np.int32)
    J = np.empty_like(I)
    K = np.empty(16 * nme)
    w = _f64(w) if w is not None else np.zeros(max(nq, 1))
    bad = ctypes.c_int64(-1)
    st = lib().or_tet_triplets(kind, nq, nme, _p(q), _p(me), _p(w), _p(I), _p(J), _p(K), ctypes.byref(bad))
    if st:
        raise OracleError(st, f"tet_triplets (element {bad.value})")
    return I, J, K


def tet_assemble(kind: int, q, me, w=None):
    """Global CSR (row_ptr, col_idx, val) of a tetrahedral mesh: triplets then sparse()."""
    q, me = _f64(q), _i32(me)
    nq, nme = q.shape[1], me.shape[1]
    cap = max(16 * nme, 1)
    row_ptr = np.empty(nq + 1, np.int32)
    col_idx = np.empty(cap, np.int32)
    val = np.empty(cap)
    w = _f64(w) if w is not None else np.zeros(max(nq, 1))
    nnz = ctypes.c_int64(0)
    bad = ctypes.c_int64(-1)
    st = lib().or_tet_assemble(kind, nq, nme, _p(q), _p(me), _p(w), _p(row_ptr), _p(col_idx), _p(val), cap,
                               ctypes.byref(nnz), ctypes.byref(bad))
    if st:
        raise OracleError(st, f"tet_assemble (element {bad.value})")
    return row_ptr, col_idx[:nnz.value].copy(), val[:nnz.value].copy()


def tet_elem_elas(x, y, z, vol: float, lam: float, mu: float) -> np.ndarray:
    """12 x 12 3-D elasticity matrix |K| B^T C B of one tetrahedron (local dof 3a + d)."""
    E = np.empty(144)
    lib().or_tet_elem_elas(_p(_f64(x)), _p(_f64(y)), _p(_f64(z)), vol, lam, mu, _p(E))
    return E.reshape(12, 12)


def tet_elas_triplets(q, me, lam: float, mu: float):
    """(Ig, Jg, Kg) of the 3-D elasticity matrix, entry c = 144k + 12*jl + il, dofs 3v + d."""
    q, me = _f64(q), _i32(me)
    nq, nme = q.shape[1], me.shape[1]
    I = np.empty(144 * nme, np.int32)
    J = np.empty_like(I)
    K = np.empty(144 * nme)
    bad = ctypes.c_int64(-1)
    st = lib().or_tet_elas_triplets(nq, nme, _p(q), _p(me), lam, mu, _p(I), _p(J), _p(K), ctypes.byref(bad))
    if st:
        raise OracleError(st, f"tet_elas_triplets (element {bad.value})")
    return I, J, K


def tet_elas_assemble(q, me, lam: float, mu: float):
    """Global CSR (row_ptr, col_idx, val) of the 3-D elasticity matrix (3 nq rows)."""
    q, me = _f64(q), _i32(me)
    nq, nme = q.shape[1], me.shape[1]
    cap = max(144 * nme, 1)
    row_ptr = np.empty(3 * nq + 1, np.int32)
    col_idx = np.empty(cap, np.int32)
    val = np.empty(cap)
    nnz = ctypes.c_int64(0)
    bad = ctypes.c_int64(-1)
    st = lib().or_tet_elas_assemble(nq, nme, _p(q), _p(me), lam, mu, _p(row_ptr), _p(col_idx), _p(val), cap,
                                    ctypes.byref(nnz), ctypes.byref(bad))
    if st:
        raise OracleError(st, f"tet_elas_assemble (element {bad.value})")
    return row_ptr, col_idx[:nnz.value].copy(), val[:nnz.value].copy()


def tet_elas_row_values(q, me, lam: float, mu: float, rows):
    """Oracle values of selected rows (dofs 3v + d) of the 3-D elasticity matrix, for meshes too
    large to assemble whole: the triplets of the tetrahedra containing vertex v, then sparse()
    of those whose row is r. Returns a list of (cols, vals) in ascending column order."""
    q, me = _f64(q), _i32(me)
    n = 3 * q.shape[1]
    out = []
    for r in rows:
        ks = np.nonzero((me == r // 3).any(axis=0))[0]
        I, J, K = tet_elas_triplets(q, me[:, ks], lam, mu)
        sel = I == r
        rp, ci, va = sparse(I[sel], J[sel], K[sel], n, n)
        out.append((ci[rp[r]:rp[r + 1]], va[rp[r]:rp[r + 1]]))
    return out


# ------------------------------------------------------------------ P2 triangles

def p2_elem_mass(area: float) -> np.ndarray:
    E = np.empty(36)
    lib().or_p2_elem_mass(area, _p(E))
    return E.reshape(6, 6)


def p2_elem_stiff(x, y, area: float) -> np.ndarray:
    E = np.empty(36)
    lib().or_p2_elem_stiff(_p(_f64(x)), _p(_f64(y)), area, _p(E))
    return E.reshape(6, 6)


def p2_triplets(kind: int, q, me):
    """(Ig, Jg, Kg, ndof) of the P2 matrices, entry c = 36k + 6*jl + il; dofs: vertices, then edges
    in ascending (smaller id, larger id) order."""
    q, me = _f64(q), _i32(me)
    nq, nme = q.shape[1], me.shape[1]
    I = np.empty(36 * nme, np.int32)
    J = np.empty_like(I)
    K = np.empty(36 * nme)
    ndof = ctypes.c_int64(0)
    bad = ctypes.c_int64(-1)
    st = lib().or_p2_triplets(kind, nq, nme, _p(q), _p(me), _p(I), _p(J), _p(K), ctypes.byref(ndof), ctypes.byref(bad))
    if st:
        raise OracleError(st, f"p2_triplets (element {bad.value})")
    return I, J, K, ndof.value


def p2_assemble(kind: int, q, me):
    """Global P2 CSR (row_ptr, col_idx, val) of a triangle mesh (kind MASS or STIFF)."""
    q, me = _f64(q), _i32(me)
    nq, nme = q.shape[1], me.shape[1]
    cap = max(36 * nme, 1)
    row_ptr = np.empty(nq + 3 * nme + 1, np.int32)
    col_idx = np.empty(cap, np.int32)
    val = np.empty(cap)
    nnz, ndof, bad = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int64(-1)
    st = lib().or_p2_assemble(kind, nq, nme, _p(q), _p(me), _p(row_ptr), _p(col_idx), _p(val), cap,
                              ctypes.byref(nnz), ctypes.byref(ndof), ctypes.byref(bad))
    if st:
        raise OracleError(st, f"p2_assemble (element {bad.value})")
    return row_ptr[:ndof.value + 1].copy(), col_idx[:nnz.value].copy(), val[:nnz.value].copy()


def p2_dof_values(q, me, f):
    """f at the P2 dofs of a triangle mesh: the vertices, then the edge midpoints in the oracle's
    edge order (for interpolating test functions)."""
    q, me = _f64(q), _i32(me)
    nq = q.shape[1]
    e = np.sort(np.concatenate([me[[0, 1]], me[[1, 2]], me[[2, 0]]], axis=1), axis=0)
    keys = np.unique((e[0].astype(np.int64) << 32) | e[1])
    lo, hi = keys >> 32, keys & 0xFFFFFFFF
    mid = 0.5 * (q[:, lo] + q[:, hi])
    return np.concatenate([f(q[0], q[1]), f(mid[0], mid[1])])


def _p2_edge_keys(me):
    """Sorted unique edge keys (smaller id << 32 | larger id): the edge numbering of the P2 dofs."""
    e = np.sort(np.concatenate([me[[0, 1]], me[[1, 2]], me[[2, 0]]], axis=1), axis=0)
    return np.unique((e[0].astype(np.int64) << 32) | e[1])


def p2_row_values(kind: int, q, me, rows):
    """Oracle values of selected P2 rows only, for meshes too large to assemble whole: the element
    matrices of the triangles containing each row's dof (vertex, or both ends of the edge), summed
    per column in ascending element order (the order of sparse() over c = 36k + 6 jl + il).
    Returns a list of (cols, vals) in ascending column order."""
    q, me = _f64(q), _i32(me)
    nq = q.shape[1]
    keys = _p2_edge_keys(me)
    out = []
    for r in rows:
        r = int(r)
        if r < nq:
            ks = np.nonzero((me == r).any(axis=0))[0]
        else:
            lo, hi = int(keys[r - nq] >> 32), int(keys[r - nq] & 0xFFFFFFFF)
            ks = np.nonzero((me == lo).any(axis=0) & (me == hi).any(axis=0))[0]
        acc = {}
        for k in ks:
            v = [int(t) for t in me[:, k]]
            x, y = q[0, v], q[1, v]
            area = double_area(x, y) / 2
            E = p2_elem_mass(area) if kind == MASS else p2_elem_stiff(x, y, area)
            ek = [(min(v[a], v[(a + 1) % 3]) << 32) | max(v[a], v[(a + 1) % 3]) for a in range(3)]
            dof = v + [nq + int(np.searchsorted(keys, key)) for key in ek]
            for il in range(6):
                if dof[il] != r:
                    continue
                for jl in range(6):
                    acc[dof[jl]] = acc.get(dof[jl], 0.0) + E[il, jl]
        cols = np.array(sorted(acc), dtype=np.int64)
        out.append((cols, np.array([acc[c] for c in cols])))
    return out


# ------------------------------------------------------------------ P3 triangles

def p3_elem_mass(area: float) -> np.ndarray:
    E = np.empty(100)
    lib().or_p3_elem_mass(area, _p(E))
    return E.reshape(10, 10)


def p3_elem_stiff(x, y, area: float) -> np.ndarray:
    E = np.empty(100)
    lib().or_p3_elem_stiff(_p(_f64(x)), _p(_f64(y)), area, _p(E))
    return E.reshape(10, 10)


def p3_triplets(kind: int, q, me):
    """(Ig, Jg, Kg, ndof) of the P3 matrices, entry c = 100k + 10*jl + il; dofs: vertices, two per
    edge (edges in ascending (smaller id, larger id) order, the node nearer the smaller id first),
    then one bubble per triangle."""
    q, me = _f64(q), _i32(me)
    nq, nme = q.shape[1], me.shape[1]
    I = np.empty(100 * nme, np.int32)
    J = np.empty_like(I)
    K = np.empty(100 * nme)
    ndof = ctypes.c_int64(0)
    bad = ctypes.c_int64(-1)
    st = lib().or_p3_triplets(kind, nq, nme, _p(q), _p(me), _p(I), _p(J), _p(K), ctypes.byref(ndof), ctypes.byref(bad))
    if st:
        raise OracleError(st, f"p3_triplets (element {bad.value})")
    return I, J, K, ndof.value


def p3_assemble(kind: int, q, me):
    """Global P3 CSR (row_ptr, col_idx, val) of a triangle mesh (kind MASS or STIFF)."""
    q, me = _f64(q), _i32(me)
    nq, nme = q.shape[1], me.shape[1]
    cap = max(100 * nme, 1)
    row_ptr = np.empty(nq + 7 * nme + 1, np.int32)
    col_idx = np.empty(cap, np.int32)
    val = np.empty(cap)
    nnz, ndof, bad = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int64(-1)
    st = lib().or_p3_assemble(kind, nq, nme, _p(q), _p(me), _p(row_ptr), _p(col_idx), _p(val), cap,
                              ctypes.byref(nnz), ctypes.byref(ndof), ctypes.byref(bad))
    if st:
        raise OracleError(st, f"p3_assemble (element {bad.value})")
    return row_ptr[:ndof.value + 1].copy(), col_idx[:nnz.value].copy(), val[:nnz.value].copy()


def p3_dof_points(q, me):
    """Coordinates [2, ndof] of the P3 dofs in the oracle's numbering: the vertices, the two nodes
    of each edge at 1/3 and 2/3 (nearer the smaller id first), the centroids (for interpolating
    test functions)."""
    q, me = _f64(q), _i32(me)
    keys = _p2_edge_keys(me)
    lo, hi = keys >> 32, keys & 0xFFFFFFFF
    n1 = (2 * q[:, lo] + q[:, hi]) / 3
    n2 = (q[:, lo] + 2 * q[:, hi]) / 3
    edge_nodes = np.empty((2, 2 * len(keys)))
    edge_nodes[:, 0::2], edge_nodes[:, 1::2] = n1, n2
    cen = (q[:, me[0]] + q[:, me[1]] + q[:, me[2]]) / 3
    return np.concatenate([q, edge_nodes, cen], axis=1)


def p3_row_values(kind: int, q, me, rows):
    """Oracle values of selected P3 rows only (for meshes too large to assemble whole): the element
    matrices of the triangles containing each row's dof, summed per column in ascending element
    order. Returns a list of (cols, vals) in ascending column order."""
    q, me = _f64(q), _i32(me)
    nq, nme = q.shape[1], me.shape[1]
    keys = _p2_edge_keys(me)
    ne = len(keys)
    out = []
    for r in rows:
        r = int(r)
        if r < nq:
            ks = np.nonzero((me == r).any(axis=0))[0]
        elif r < nq + 2 * ne:
            e = (r - nq) // 2
            lo, hi = int(keys[e] >> 32), int(keys[e] & 0xFFFFFFFF)
            ks = np.nonzero((me == lo).any(axis=0) & (me == hi).any(axis=0))[0]
        else:
            ks = np.array([r - nq - 2 * ne])
        acc = {}
        for k in ks:
            v = [int(t) for t in me[:, k]]
            x, y = q[0, v], q[1, v]
            area = double_area(x, y) / 2
            E = p3_elem_mass(area) if kind == MASS else p3_elem_stiff(x, y, area)
            dof = list(v)
            for t in range(3):
                a, b = v[t], v[(t + 1) % 3]
                e = int(np.searchsorted(keys, (min(a, b) << 32) | max(a, b)))
                dof += [nq + 2 * e + (0 if a < b else 1), nq + 2 * e + (1 if a < b else 0)]
            dof.append(nq + 2 * ne + int(k))
            for il in range(10):
                if dof[il] != r:
                    continue
                for jl in range(10):
                    acc[dof[jl]] = acc.get(dof[jl], 0.0) + E[il, jl]
        cols = np.array(sorted(acc), dtype=np.int64)
        out.append((cols, np.array([acc[c] for c in cols])))
    return out
