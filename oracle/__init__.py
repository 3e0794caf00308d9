"""FP64 CPU oracle for the regularised traveltime least-squares solve.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
CPU-baseline leg may import this package; the product (the CUDA library and
its Python binding) never does, and this package never imports the product.
Inputs come from the seeded generator; everything else here is computed from
the paper's definitions:

* ``build_G``       sensitivity matrix of Eq. 5-7 (synthetic form, see oracle.c)
* ``transpose``     CSR of G^T
* ``laplacian``     3-D 7-point graph Laplacian
* ``lsqr``          Paige & Saunders (1982) LSQR with damping / column scaling
* ``aug_colnorm2``  squared column norms of [G; w L; lam I]
* ``blockprec``     per-cell depth blocks of [G; w L; lam I]^T [G; w L; lam I]
                    and the inverse Cholesky factors that precondition LSQR

Parity status: every function here is pinned by tests/test_oracle_*.py
(closed forms, dense Householder QR, SciPy's LSQR, exact recovery, LSQR
invariants).  See ``mlp.py`` and ``features.py`` for the preconditioner parts.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

_d = ctypes.POINTER(ctypes.c_double)
_i32 = ctypes.POINTER(ctypes.c_int32)
_i64 = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile oracle.c (gcc, -ffp-contract=off, OpenMP) into liboracle.so."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC",
                               "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        lib.oracle_G_count.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                       ctypes.c_int, ctypes.c_int64, _d, _i32]
        lib.oracle_G_count.restype = ctypes.c_int
        lib.oracle_G_fill.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                      ctypes.c_int, ctypes.c_int64, _d, _i32, _d, _d,
                                      ctypes.c_int, _i64, _i32, _d]
        lib.oracle_G_fill.restype = ctypes.c_int
        lib.oracle_transpose.argtypes = [ctypes.c_int64, ctypes.c_int32, _i64, _i32, _d,
                                         _i64, _i32, _d]
        lib.oracle_transpose.restype = None
        lib.oracle_spmv.argtypes = [ctypes.c_int64, _i64, _i32, _d, _d, _d]
        lib.oracle_spmv.restype = None
        lib.oracle_laplacian.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _d, _d]
        lib.oracle_laplacian.restype = None
        lib.oracle_aug_colnorm2.argtypes = [ctypes.c_int32, _i64, _d, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_int, ctypes.c_double, ctypes.c_double, _d]
        lib.oracle_aug_colnorm2.restype = None
        lib.oracle_apply_A.argtypes = [ctypes.c_int64, ctypes.c_int32, _i64, _i32, _d,
                                       ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                       _d, ctypes.c_double, _d, _d, _d]
        lib.oracle_apply_A.restype = None
        lib.oracle_apply_At.argtypes = lib.oracle_apply_A.argtypes
        lib.oracle_apply_At.restype = None
        lib.oracle_lsqr.argtypes = [ctypes.c_int64, ctypes.c_int32, _i64, _i32, _d, _i64, _i32, _d,
                                    ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                    _d, ctypes.c_double, ctypes.c_double, _d, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_double, ctypes.c_int, _d, _d,
                                    ctypes.c_int, _d, _d, _d, ctypes.c_int, _d, _d, _i32, _d]
        lib.oracle_lsqr.restype = ctypes.c_int
        lib.oracle_num_threads.argtypes = []
        lib.oracle_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _p(a: Optional[np.ndarray], ty):
    if a is None:
        return ctypes.cast(None, ty)
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ty)


def num_threads() -> int:
    return int(_load().oracle_num_threads())


@dataclass
class CSR:
    """A CSR matrix: ptr (rows+1, int64), idx (nnz, int32), val (nnz, float64)."""
    ptr: np.ndarray
    idx: np.ndarray
    val: np.ndarray
    n_cols: int

    @property
    def n_rows(self) -> int:
        return self.ptr.shape[0] - 1

    @property
    def nnz(self) -> int:
        return int(self.ptr[-1])

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val, self.idx, self.ptr), shape=(self.n_rows, self.n_cols))


def build_G(nx: int, ny: int, nz: int, dx_km: float, ctrl: np.ndarray,
            row_period: np.ndarray, kdz: np.ndarray, kdz_cells=None, interp: int = 0) -> CSR:
    """Sensitivity matrix G (rows = paths in the order given) as CSR; with
    kdz_cells (nx*ny, periods, nz) a depth kernel per horizontal cell; interp 1:
    bilinear node coefficients instead of cell lengths."""
    if interp not in (0, 1) or (interp == 1 and (nx < 2 or ny < 2)):
        raise ValueError("interp must be 0, or 1 on a grid of at least 2 x 2 nodes")
    lib = _load()
    ctrl = np.ascontiguousarray(ctrl, dtype=np.float64).reshape(-1, 6)
    row_period = np.ascontiguousarray(row_period, dtype=np.int32)
    kdz = np.ascontiguousarray(kdz, dtype=np.float64)
    m = ctrl.shape[0]
    if kdz.shape[1] != nz:
        raise ValueError("kdz must be n_periods x nz")
    if m and (row_period.min() < 0 or row_period.max() >= kdz.shape[0]):
        raise ValueError("period index out of range")
    cells = np.zeros(m, dtype=np.int32)
    if lib.oracle_G_count(nx, ny, dx_km, interp, m, _p(ctrl, _d), _p(cells, _i32)) != 0:
        raise MemoryError("oracle_G_count")
    ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(cells.astype(np.int64) * nz, out=ptr[1:])
    nnz = int(ptr[-1])
    col = np.zeros(nnz, dtype=np.int32)
    val = np.zeros(nnz, dtype=np.float64)
    kc = None
    if kdz_cells is not None:
        kc = np.ascontiguousarray(kdz_cells, dtype=np.float64)
        if kc.shape != (nx * ny, kdz.shape[0], nz):
            raise ValueError("kdz_cells must be (nx*ny, periods, nz)")
    if lib.oracle_G_fill(nx, ny, nz, dx_km, interp, m, _p(ctrl, _d), _p(row_period, _i32),
                         _p(kdz, _d),
                         _p(kc, _d), int(kdz.shape[0]), _p(ptr, _i64), _p(col, _i32),
                         _p(val, _d)) != 0:
        raise MemoryError("oracle_G_fill")
    return CSR(ptr, col, val, nx * ny * nz)


def build_G_problem(p) -> CSR:
    return build_G(p.nx, p.ny, p.nz, p.dx_km, p.ctrl, p.row_period, p.kdz,
                   getattr(p, "kdz_cells", None), getattr(p, "interp", 0))


def transpose(G: CSR) -> CSR:
    lib = _load()
    n = G.n_cols
    cp = np.zeros(n + 1, dtype=np.int64)
    ri = np.zeros(G.nnz, dtype=np.int32)
    vt = np.zeros(G.nnz, dtype=np.float64)
    lib.oracle_transpose(G.n_rows, n, _p(G.ptr, _i64), _p(G.idx, _i32), _p(G.val, _d),
                         _p(cp, _i64), _p(ri, _i32), _p(vt, _d))
    return CSR(cp, ri, vt, G.n_rows)


def spmv(S: CSR, x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.zeros(S.n_rows, dtype=np.float64)
    _load().oracle_spmv(S.n_rows, _p(S.ptr, _i64), _p(S.idx, _i32), _p(S.val, _d),
                        _p(x, _d), _p(y, _d))
    return y


def laplacian(nx: int, ny: int, nz: int, x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.zeros_like(x)
    _load().oracle_laplacian(nx, ny, nz, _p(x, _d), _p(y, _d))
    return y


def aug_colnorm2(GT: CSR, nx: int, ny: int, nz: int, w: float, lam: float) -> np.ndarray:
    out = np.zeros(GT.n_rows, dtype=np.float64)
    _load().oracle_aug_colnorm2(GT.n_rows, _p(GT.ptr, _i64), _p(GT.val, _d), nx, ny, nz,
                                w, lam, _p(out, _d))
    return out


def _blocks(P, n: int, nz: int):
    if P is None:
        return None
    P = np.ascontiguousarray(P, dtype=np.float64)
    assert P.shape == (n // nz, nz, nz), "P: one nz x nz block per horizontal cell"
    return P


def apply_A(G: CSR, grid, w: float, v: np.ndarray, D=None, lam_rows: float = 0.0, P=None):
    """y = A v with A = [G; w L], [G D; w L D; lam D] or [G P; w L P; lam P]."""
    nx, ny, nz = grid
    n = G.n_cols
    assert D is None or P is None
    M = G.n_rows + n + (n if lam_rows > 0 else 0)
    y = np.zeros(M, dtype=np.float64)
    v = np.ascontiguousarray(v, dtype=np.float64)
    D = None if D is None else np.ascontiguousarray(D, dtype=np.float64)
    P = _blocks(P, n, nz)
    _load().oracle_apply_A(G.n_rows, n, _p(G.ptr, _i64), _p(G.idx, _i32), _p(G.val, _d),
                           nx, ny, nz, w, _p(D, _d), lam_rows, _p(v, _d), _p(y, _d), _p(P, _d))
    return y


def apply_At(GT: CSR, grid, w: float, u: np.ndarray, D=None, lam_rows: float = 0.0, P=None):
    """z = A^T u for the operators of apply_A."""
    nx, ny, nz = grid
    n = GT.n_rows
    assert D is None or P is None
    z = np.zeros(n, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    D = None if D is None else np.ascontiguousarray(D, dtype=np.float64)
    P = _blocks(P, n, nz)
    _load().oracle_apply_At(GT.n_cols, n, _p(GT.ptr, _i64), _p(GT.idx, _i32), _p(GT.val, _d),
                            nx, ny, nz, w, _p(D, _d), lam_rows, _p(u, _d), _p(z, _d), _p(P, _d))
    return z


@dataclass
class LSQRResult:
    x: np.ndarray
    itn: int
    istop: int
    rnorm: float
    arnorm: float
    anorm: float
    acond: float
    xnorm: float
    bnorm: float
    U: Optional[np.ndarray] = None
    V: Optional[np.ndarray] = None
    rhist: Optional[np.ndarray] = None
    ck_itn: Optional[np.ndarray] = None   # per checkpoint tolerance: stopping iteration (0: never)
    ck_x: Optional[np.ndarray] = None     # per checkpoint tolerance: the iterate there


def lsqr(G: CSR, GT: CSR, grid, w: float, damp: float, b: np.ndarray,
         atol: float = 1e-8, btol: float = 1e-8, conlim: float = 1e8, itmax: int = 300,
         D: Optional[np.ndarray] = None, lam_rows: float = 0.0, record: int = 0,
         history: bool = False, checkpoints=None, P: Optional[np.ndarray] = None) -> LSQRResult:
    """LSQR on [G; w L] (or [G D; w L D; lam_rows D] when D is given, or
    [G P; w L P; lam_rows P] with P the per-cell depth blocks, (nx*ny, nz, nz));
    x is the solution in the scaled variables (the model is D x or P x).

    checkpoints: tolerances t; for each, the iterate and iteration at which a
    solve with atol = btol = t stops on S1 or S2 (the same run serves all)."""
    lib = _load()
    nx, ny, nz = grid
    m, n = G.n_rows, G.n_cols
    b = np.ascontiguousarray(b, dtype=np.float64)
    assert b.shape[0] == m
    D = None if D is None else np.ascontiguousarray(D, dtype=np.float64)
    assert D is None or P is None
    P = _blocks(P, n, nz)
    M = m + n + (n if lam_rows > 0 else 0)
    x = np.zeros(n, dtype=np.float64)
    est = np.zeros(8, dtype=np.float64)
    U = np.zeros((record, M)) if record > 0 else None
    V = np.zeros((record, n)) if record > 0 else None
    rh = np.zeros(max(itmax, 1)) if history else None
    ck = None if checkpoints is None else np.ascontiguousarray(checkpoints, dtype=np.float64)
    nck = 0 if ck is None else int(ck.shape[0])
    ck_x = np.zeros((nck, n)) if nck else None
    ck_itn = np.zeros(nck, dtype=np.int32) if nck else None
    rc = lib.oracle_lsqr(m, n, _p(G.ptr, _i64), _p(G.idx, _i32), _p(G.val, _d),
                         _p(GT.ptr, _i64), _p(GT.idx, _i32), _p(GT.val, _d),
                         nx, ny, nz, w, _p(D, _d), lam_rows, damp, _p(b, _d),
                         atol, btol, conlim, itmax, _p(x, _d), _p(est, _d),
                         record, _p(U, _d), _p(V, _d), _p(rh, _d),
                         nck, _p(ck, _d), _p(ck_x, _d), _p(ck_itn, _i32), _p(P, _d))
    if rc != 0:
        raise MemoryError("oracle_lsqr")
    itn = int(est[0])
    return LSQRResult(x=x, itn=itn, istop=int(est[1]), rnorm=est[2], arnorm=est[3],
                      anorm=est[4], acond=est[5], xnorm=est[6], bnorm=est[7],
                      U=U, V=V, rhist=None if rh is None else rh[:itn],
                      ck_itn=ck_itn, ck_x=ck_x)


def rhs_for(p, G: CSR, m_model=None, noise=None, frac=None) -> np.ndarray:
    """d = G m + frac * RMS(G m) * z for a generator problem (oracle-side G)."""
    m_model = p.m_true if m_model is None else m_model
    noise = p.noise if noise is None else noise
    frac = p.noise_frac if frac is None else frac
    gm = spmv(G, m_model)
    rms = float(np.sqrt(np.mean(gm * gm))) if gm.size else 0.0
    return gm + frac * rms * noise
