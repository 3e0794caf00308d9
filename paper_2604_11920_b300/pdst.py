"""Python binding of the C ABI in include/pdst.h (argument marshalling only).

Every step of the solve runs in the CUDA library libpdst.so built in-tree by
``paper_2604_11920_b300.build``; this module only converts arguments.  There
is no fallback: if the library is missing or fails to load, calls raise.
PyTorch is used for device memory and streams (``torch.Tensor.data_ptr()``,
``torch.cuda.current_stream()``).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpdst.so")

F64, F32, BF16, DF64 = 0, 1, 2, 3
FMT_ELEMENT, FMT_BLOCKED = 0, 1
DTYPES = {"f64": F64, "f32": F32, "bf16": BF16, "df64": DF64}
METHODS = {"lsqr": 0, "lsmr": 1}
FORMATS = {"element": FMT_ELEMENT, "blocked": FMT_BLOCKED}

STATUS = {0: "PDST_OK", 1: "PDST_ERR_ARG", 2: "PDST_ERR_CUDA", 3: "PDST_ERR_OOM",
          4: "PDST_ERR_BREAKDOWN", 5: "PDST_ERR_TIMEOUT", 6: "PDST_ERR_NOT_CONVERGED",
          7: "PDST_ERR_LIMIT", 8: "PDST_ERR_STATE"}


class PdstError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("dx_km", ctypes.c_double), ("dz_km", ctypes.c_double)]


class BuildOpts(ctypes.Structure):
    _fields_ = [("value_dtypes", ctypes.c_uint32), ("formats", ctypes.c_uint32),
                ("kdz_cells", ctypes.c_void_p), ("interp", ctypes.c_int32),
                ("keep_lengths", ctypes.c_int32)]


class LsqrOpts(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int32), ("format", ctypes.c_int32),
                ("atol", ctypes.c_double), ("btol", ctypes.c_double),
                ("conlim", ctypes.c_double), ("precond", ctypes.c_int32),
                ("kblock", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("profile", ctypes.c_int32), ("rnorm_hist_dev", ctypes.c_void_p),
                ("refine", ctypes.c_int32), ("refine_dtype", ctypes.c_int32),
                ("refine_tol", ctypes.c_double), ("method", ctypes.c_int32),
                ("reserved0", ctypes.c_int32)]


class BatchedOpts(ctypes.Structure):
    _fields_ = [("tile_rows", ctypes.c_int32), ("kblock", ctypes.c_int32),
                ("chosen_tile_rows", ctypes.c_int32), ("kernel_launches", ctypes.c_int32),
                ("tune_ms", ctypes.c_double * 4), ("precond", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class OuterOpts(ctypes.Structure):
    _fields_ = [("max_outer", ctypes.c_int32), ("reserved0", ctypes.c_int32),
                ("rms_tol", ctypes.c_double), ("min_decrease", ctypes.c_double),
                ("z0_factor", ctypes.c_double), ("kernel_power", ctypes.c_double),
                ("inner", LsqrOpts)]


class OuterInfo(ctypes.Structure):
    _fields_ = [("updates", ctypes.c_int32), ("reason", ctypes.c_int32),
                ("inner_iters", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("rms_first", ctypes.c_double), ("rms_final", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


class LsqrInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("istop", ctypes.c_int32),
                ("rnorm", ctypes.c_double), ("arnorm", ctypes.c_double),
                ("anorm", ctypes.c_double), ("acond", ctypes.c_double),
                ("xnorm", ctypes.c_double), ("bnorm", ctypes.c_double),
                ("kernel_launches", ctypes.c_int32), ("profiled_iters", ctypes.c_int32),
                ("fwd_ms", ctypes.c_double), ("adj_ms", ctypes.c_double),
                ("upd_ms", ctypes.c_double), ("sweeps", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("correction", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None
_vp = ctypes.c_void_p
_i32, _i64, _d = ctypes.c_int32, ctypes.c_int64, ctypes.c_double

# name -> (restype, argtypes); must match include/pdst.h
SIGNATURES = {
    "pdst_build_G": (_i32, [ctypes.POINTER(Grid), _i64, _vp, _vp, _i32, _vp,
                            ctypes.POINTER(BuildOpts), _vp, ctypes.POINTER(_vp)]),
    "pdst_destroy": (_i32, [_vp]),
    "pdst_G_info": (_i32, [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i32),
                           ctypes.POINTER(_i64)]),
    "pdst_G_export_csr": (_i32, [_vp, _i32, _vp, _vp, _vp]),
    "pdst_G_export_csc": (_i32, [_vp, _i32, _vp, _vp, _vp]),
    "pdst_apply_G": (_i32, [_vp, _i32, _i32, _vp, _vp, _vp]),
    "pdst_lsqr_opts_default": (None, [ctypes.POINTER(LsqrOpts)]),
    "pdst_lsqr": (_i32, [_vp, _vp, _d, _d, _i32, _d, _vp, ctypes.POINTER(LsqrInfo),
                         ctypes.POINTER(LsqrOpts), _vp]),
    "pdst_lsqr_host": (_i32, [_vp, _vp, _d, _d, _i32, _d, _vp, ctypes.POINTER(LsqrInfo),
                              ctypes.POINTER(LsqrOpts), _vp]),
    "pdst_lsqr_damping_sweep": (_i32, [_vp, _vp, _d, _i32, _vp, _i32, _d, _vp,
                                       ctypes.POINTER(LsqrInfo), ctypes.POINTER(LsqrOpts), _vp]),
    "pdst_lsqr_noalloc": (_i32, [_vp, _vp, _d, _d, _i32, _d, _vp, ctypes.POINTER(LsqrInfo),
                                 ctypes.POINTER(LsqrOpts), _vp]),
    "pdst_set_col_scaling": (_i32, [_vp, _vp, _d, _d, _vp]),
    "pdst_col_norms": (_i32, [_vp, _d, _d, _vp, _vp]),
    "pdst_set_col_scaling_power": (_i32, [_vp, _d, _d, _d, _vp]),
    "pdst_precond_features": (_i32, [_vp, _vp, _vp, _vp]),
    "pdst_depth_blocks": (_i32, [_vp, _d, _d, _vp, _vp]),
    "pdst_set_block_precond": (_i32, [_vp, _vp, _d, _d, _vp]),
    "pdst_get_block_precond": (_i32, [_vp, _vp, _vp]),
    "pdst_mlp_forward": (_i32, [_vp, _vp, _i64, _vp, _vp, _vp]),
    "pdst_mlp_grad": (_i32, [_vp, _vp, _vp, _vp, _i32, _vp, _vp]),
    "pdst_mlp_adam": (_i32, [_vp, _vp, _vp, _vp, _i64, _d, _d, _d, _d, _vp]),
    "pdst_batched_opts_default": (None, [ctypes.POINTER(BatchedOpts)]),
    "pdst_lsqr_batched": (_i32, [_i32, _vp, _vp, _vp, _vp, _vp, _i32, _d, _i32, _vp,
                                 ctypes.POINTER(LsqrInfo), ctypes.POINTER(BatchedOpts), _vp]),
    "pdst_depth_kernels_from_model": (_i32, [_vp, _vp, _d, _d, _vp, _vp, _vp]),
    "pdst_set_depth_kernels": (_i32, [_vp, _vp, _vp]),
    "pdst_outer_opts_default": (None, [ctypes.POINTER(OuterOpts)]),
    "pdst_outer_loop": (_i32, [_vp, _vp, _vp, _d, _d, _i32, _d, ctypes.POINTER(OuterOpts), _vp,
                               _vp, ctypes.POINTER(OuterInfo), _vp]),
    "pdst_stream_read": (_i32, [_vp, _i64, _vp]),
    "pdst_last_error_string": (ctypes.c_char_p, []),
    "pdst_version": (_i32, []),
}


def load(path: str = LIB_PATH):
    """Load libpdst.so (raises if it is missing; run build() first)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with paper_2604_11920_b300.build")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(status: int):
    if status != 0:
        raise PdstError(status, load().pdst_last_error_string().decode())


def _stream(stream=None):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _dev_ptr(t, numel=None, dtype=None, name="tensor"):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, has {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


def _np_ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def stream_read(buf, stream=None):
    """pdst_stream_read: one sequential read of a CUDA tensor's bytes (a
    measurement aid: the streaming ceiling beside the sweeps' rates)."""
    nbytes = buf.numel() * buf.element_size()
    _check(load().pdst_stream_read(ctypes.c_void_p(buf.data_ptr()), nbytes, _stream(stream)))


def lsqr_opts(dtype="f64", fmt="element", atol=-1.0, btol=-1.0, conlim=0.0, precond=0,
              kblock=16, use_graph=True, hist=None, profile=False, refine=0,
              refine_tol=1e-5, refine_dtype=None, method="lsqr") -> LsqrOpts:
    o = LsqrOpts()
    load().pdst_lsqr_opts_default(ctypes.byref(o))
    o.dtype = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
    o.format = FORMATS[fmt] if isinstance(fmt, str) else int(fmt)
    o.atol, o.btol, o.conlim = atol, btol, conlim
    o.precond, o.kblock, o.use_graph = int(precond), int(kblock), int(bool(use_graph))
    o.profile = int(profile) if not isinstance(profile, bool) else int(profile)
    o.refine, o.refine_tol = int(refine), float(refine_tol)
    o.refine_dtype = -1 if refine_dtype is None else (DTYPES[refine_dtype]
                                                      if isinstance(refine_dtype, str)
                                                      else int(refine_dtype))
    o.rnorm_hist_dev = None if hist is None else hist.data_ptr()
    o.method = METHODS[method] if isinstance(method, str) else int(method)
    return o


@dataclass
class Result:
    m: object
    info: dict


class Handle:
    """Owns one device-resident G (CSR + transpose) built by pdst_build_G."""

    def __init__(self, ptr: ctypes.c_void_p, grid: Grid):
        self._ptr = ptr
        self.grid = grid
        m, n, nnz = _i64(), _i32(), _i64()
        _check(load().pdst_G_info(self._ptr, ctypes.byref(m), ctypes.byref(n),
                                  ctypes.byref(nnz)))
        self.m, self.n, self.nnz = m.value, n.value, nnz.value

    def close(self):
        if self._ptr is not None and _lib is not None:
            _lib.pdst_destroy(self._ptr)
        self._ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def ptr(self):
        if self._ptr is None:
            raise ValueError("handle is closed")
        return self._ptr

    # -- inspection -------------------------------------------------------
    def export_csr(self, dtype="f64", ptr_only=False):
        """(row_ptr, col, val) on the host; ptr_only: row_ptr alone (idx, val = None)."""
        ptr = np.zeros(self.m + 1, np.int64)
        idx = None if ptr_only else np.zeros(self.nnz, np.int32)
        val = None if ptr_only else np.zeros(self.nnz, np.float64)
        _check(load().pdst_G_export_csr(self.ptr, DTYPES[dtype], _np_ptr(ptr),
                                        None if idx is None else _np_ptr(idx),
                                        None if val is None else _np_ptr(val)))
        return ptr, idx, val

    def export_csc(self, dtype="f64"):
        ptr = np.zeros(self.n + 1, np.int64)
        idx = np.zeros(self.nnz, np.int32)
        val = np.zeros(self.nnz, np.float64)
        _check(load().pdst_G_export_csc(self.ptr, DTYPES[dtype], _np_ptr(ptr), _np_ptr(idx),
                                        _np_ptr(val)))
        return ptr, idx, val

    def apply_G(self, x, y, trans=False, dtype="f64", stream=None):
        import torch
        nin, nout = (self.m, self.n) if trans else (self.n, self.m)
        _check(load().pdst_apply_G(self.ptr, DTYPES[dtype], int(trans),
                                   _dev_ptr(x, nin, torch.float64, "x"),
                                   _dev_ptr(y, nout, torch.float64, "y"), _stream(stream)))
        return y

    # -- solves ---------------------------------------------------------------
    def lsqr(self, d, w, lam, itmax, tol, m_out=None, stream=None, **opt_kw) -> Result:
        import torch
        if m_out is None:
            m_out = torch.empty(self.n, dtype=torch.float64, device=d.device)
        info = LsqrInfo()
        o = lsqr_opts(**opt_kw)
        _check(load().pdst_lsqr(self.ptr, _dev_ptr(d, self.m, torch.float64, "d"), w, lam,
                                int(itmax), tol, _dev_ptr(m_out, self.n, torch.float64, "m_out"),
                                ctypes.byref(info), ctypes.byref(o), _stream(stream)))
        return Result(m_out, info.as_dict())

    def lsqr_damping_sweep(self, d, w, lambdas, itmax, tol, stream=None, **opt_kw):
        """Solutions for several damping values from one bidiagonalisation:
        a list of Result, one per value of `lambdas`."""
        import torch
        lam = np.ascontiguousarray(lambdas, dtype=np.float64)
        L = lam.shape[0]
        outs = [torch.empty(self.n, dtype=torch.float64, device=d.device) for _ in range(L)]
        ptrs = (ctypes.c_void_p * L)(*[o.data_ptr() for o in outs])
        infos = (LsqrInfo * L)()
        o = lsqr_opts(**opt_kw)
        _check(load().pdst_lsqr_damping_sweep(
            self.ptr, _dev_ptr(d, self.m, torch.float64, "d"), float(w), L, _np_ptr(lam),
            int(itmax), float(tol), ptrs, infos, ctypes.byref(o), _stream(stream)))
        return [Result(outs[i], infos[i].as_dict()) for i in range(L)]

    def lsqr_noalloc(self, d, w, lam, itmax, tol, m_out, stream=None, **opt_kw) -> Result:
        """pdst_lsqr_noalloc: the same solve with no device allocation (the
        caller passes the output buffer; scratch is the library's static array)."""
        import torch
        info = LsqrInfo()
        o = lsqr_opts(**opt_kw)
        _check(load().pdst_lsqr_noalloc(self.ptr, _dev_ptr(d, self.m, torch.float64, "d"), w,
                                        lam, int(itmax), tol,
                                        _dev_ptr(m_out, self.n, torch.float64, "m_out"),
                                        ctypes.byref(info), ctypes.byref(o), _stream(stream)))
        return Result(m_out, info.as_dict())

    def lsqr_host(self, d: np.ndarray, w, lam, itmax, tol, m_out: Optional[np.ndarray] = None,
                  stream=None, **opt_kw) -> Result:
        if d.dtype != np.float64 or not d.flags["C_CONTIGUOUS"] or d.shape != (self.m,):
            raise ValueError("d must be a contiguous float64 vector of length m")
        if m_out is None:
            m_out = np.zeros(self.n, np.float64)
        info = LsqrInfo()
        o = lsqr_opts(**opt_kw)
        _check(load().pdst_lsqr_host(self.ptr, _np_ptr(d), w, lam, int(itmax), tol,
                                     _np_ptr(m_out), ctypes.byref(info), ctypes.byref(o),
                                     _stream(stream)))
        return Result(m_out, info.as_dict())

    def col_norms(self, w, lam, stream=None):
        import torch
        c = torch.empty(self.n, dtype=torch.float64, device="cuda")
        _check(load().pdst_col_norms(self.ptr, w, lam, _dev_ptr(c, self.n), _stream(stream)))
        return c

    def set_col_scaling_power(self, w, lam, p, stream=None):
        _check(load().pdst_set_col_scaling_power(self.ptr, w, lam, float(p), _stream(stream)))

    def features(self, log_periods, stream=None):
        """pdst_precond_features: (n, 8) float32 CUDA tensor."""
        import torch
        lp = np.ascontiguousarray(log_periods, dtype=np.float64)
        f = torch.empty((self.n, MLP_NFEAT), dtype=torch.float32, device="cuda")
        _check(load().pdst_precond_features(self.ptr, _np_ptr(lp), _dev_ptr(f), _stream(stream)))
        return f

    def depth_kernels_from_model(self, periods, m, z0_factor=1.2, kernel_power=1.0,
                                 out=None, stream=None):
        """pdst_depth_kernels_from_model: (nx*ny, T, nz) float64 CUDA tensor."""
        import torch
        per = np.ascontiguousarray(periods, dtype=np.float64)
        T = per.shape[0]
        H = self.grid.nx * self.grid.ny
        if out is None:
            out = torch.empty((H, T, self.grid.nz), dtype=torch.float64, device="cuda")
        _check(load().pdst_depth_kernels_from_model(
            self.ptr, _np_ptr(per), float(z0_factor), float(kernel_power),
            _dev_ptr(m, self.n, torch.float64, "m"),
            _dev_ptr(out, H * T * self.grid.nz, torch.float64, "out"), _stream(stream)))
        return out

    def set_depth_kernels(self, kdz_cells, stream=None):
        import torch
        _check(load().pdst_set_depth_kernels(self.ptr, _dev_ptr(kdz_cells, None, torch.float64,
                                                                "kdz_cells"), _stream(stream)))

    def outer_loop(self, d_obs, periods, w, lam, itmax, tol, max_outer=8, rms_tol=0.0,
                   min_decrease=0.01, z0_factor=1.2, kernel_power=1.0, m_out=None,
                   stream=None, **inner_kw):
        """pdst_outer_loop: returns (m, rms history (numpy), info dict)."""
        import torch
        per = np.ascontiguousarray(periods, dtype=np.float64)
        if m_out is None:
            m_out = torch.empty(self.n, dtype=torch.float64, device=d_obs.device)
        o = OuterOpts()
        load().pdst_outer_opts_default(ctypes.byref(o))
        o.max_outer, o.rms_tol, o.min_decrease = int(max_outer), float(rms_tol), \
            float(min_decrease)
        o.z0_factor, o.kernel_power = float(z0_factor), float(kernel_power)
        o.inner = lsqr_opts(**inner_kw)
        hist = np.zeros(int(max_outer) + 1)
        info = OuterInfo()
        _check(load().pdst_outer_loop(self.ptr, _dev_ptr(d_obs, self.m, torch.float64, "d_obs"),
                                      _np_ptr(per), float(w), float(lam), int(itmax), float(tol),
                                      ctypes.byref(o), _dev_ptr(m_out, self.n, torch.float64,
                                                                "m_out"),
                                      _np_ptr(hist), ctypes.byref(info), _stream(stream)))
        inf = info.as_dict()
        return m_out, hist[: inf["updates"] + 1], inf

    def set_col_scaling(self, D=None, w=0.0, lam=0.0, stream=None):
        import torch
        p = ctypes.c_void_p(None) if D is None else _dev_ptr(D, self.n, torch.float64, "D")
        _check(load().pdst_set_col_scaling(self.ptr, p, w, lam, _stream(stream)))

    def _block_count(self):
        nz = self.grid.nz
        return (self.n // nz) * nz * nz if nz else 0

    def depth_blocks(self, w, lam, stream=None):
        """pdst_depth_blocks: (nx*ny, nz, nz) float64 CUDA tensor of B_h."""
        import torch
        B = torch.empty(self._block_count(), dtype=torch.float64, device="cuda")
        _check(load().pdst_depth_blocks(self.ptr, float(w), float(lam),
                                        _dev_ptr(B, B.numel(), torch.float64, "B"),
                                        _stream(stream)))
        return B.view(-1, self.grid.nz, self.grid.nz)

    def set_block_precond(self, P=None, w=0.0, lam=0.0, stream=None):
        """pdst_set_block_precond: P (nx*ny, nz, nz) float64 CUDA tensor, or
        None to compute P_h = R_h^{-1} from the depth blocks for w, lam."""
        import torch
        if P is None:
            p = ctypes.c_void_p(None)
        else:
            P = P.contiguous()
            p = _dev_ptr(P.view(-1), self._block_count(), torch.float64, "P")
        _check(load().pdst_set_block_precond(self.ptr, p, float(w), float(lam), _stream(stream)))

    def get_block_precond(self, stream=None):
        import torch
        P = torch.empty(self._block_count(), dtype=torch.float64, device="cuda")
        _check(load().pdst_get_block_precond(self.ptr, _dev_ptr(P, P.numel(), torch.float64, "P"),
                                             _stream(stream)))
        return P.view(-1, self.grid.nz, self.grid.nz)


def build_G(nx, ny, nz, dx_km, dz_km, ctrl, row_period, n_periods, kdz, dtypes=("f64", "f32"),
            formats=("element", "blocked"), stream=None, kdz_cells=None, interp=0,
            keep_lengths=False) -> Handle:
    ctrl = np.ascontiguousarray(ctrl, dtype=np.float64).reshape(-1, 6)
    row_period = np.ascontiguousarray(row_period, dtype=np.int32)
    kdz = np.ascontiguousarray(kdz, dtype=np.float64)
    grid = Grid(nx, ny, nz, dx_km, dz_km)
    kc = None
    if kdz_cells is not None:
        kc = np.ascontiguousarray(kdz_cells, dtype=np.float64)
        if kc.shape != (nx * ny, int(n_periods), nz):
            raise ValueError("kdz_cells must be (nx*ny, n_periods, nz)")
    opts = BuildOpts(sum(1 << DTYPES[d] for d in dtypes), sum(1 << FORMATS[f] for f in formats),
                     None if kc is None else kc.ctypes.data, int(interp), int(bool(keep_lengths)))
    out = ctypes.c_void_p()
    _check(load().pdst_build_G(ctypes.byref(grid), ctrl.shape[0], _np_ptr(ctrl),
                               _np_ptr(row_period), int(n_periods), _np_ptr(kdz),
                               ctypes.byref(opts), _stream(stream), ctypes.byref(out)))
    return Handle(out, grid)


def build_G_problem(p, **kw) -> Handle:
    """pdst_build_G for a generator problem (see synth.py)."""
    kw.setdefault("kdz_cells", getattr(p, "kdz_cells", None))
    kw.setdefault("interp", getattr(p, "interp", 0))
    return build_G(p.nx, p.ny, p.nz, p.dx_km, p.dz_km, p.ctrl, p.row_period, p.n_periods,
                   p.kdz, **kw)


def lsqr_batched(handles, ds, w, lams, itmax, tol, dtype="f32", tile_rows=0, kblock=8,
                 m_outs=None, stream=None, precond=0):
    """pdst_lsqr_batched.  ds[s]: (m_s, R_s) float64 CUDA tensors (right-hand
    sides in columns); lams[s]: R_s damping values.  Returns (m_outs, infos,
    opts) with m_outs[s] of shape (n_s, R_s)."""
    import torch
    lib = load()
    nsys = len(handles)
    R = [int(d.shape[1]) for d in ds]
    if m_outs is None:
        m_outs = [torch.empty((h.n, r), dtype=torch.float64, device=ds[0].device)
                  for h, r in zip(handles, R)]
    hs = (ctypes.c_void_p * nsys)(*[h.ptr.value if isinstance(h.ptr, ctypes.c_void_p) else h.ptr
                                    for h in handles])
    nr = (ctypes.c_int32 * nsys)(*R)
    dp = (ctypes.c_void_p * nsys)(*[_dev_ptr(d, h.m * r, torch.float64, "d").value
                                    for d, h, r in zip(ds, handles, R)])
    mp = (ctypes.c_void_p * nsys)(*[_dev_ptr(m, h.n * r, torch.float64, "m_out").value
                                    for m, h, r in zip(m_outs, handles, R)])
    wv = (ctypes.c_double * nsys)(*[float(x) for x in w])
    lam_arrs = [(ctypes.c_double * r)(*[float(x) for x in l]) for l, r in zip(lams, R)]
    lp = (ctypes.c_void_p * nsys)(*[ctypes.cast(a, ctypes.c_void_p).value for a in lam_arrs])
    infos = (LsqrInfo * sum(R))()
    o = BatchedOpts()
    lib.pdst_batched_opts_default(ctypes.byref(o))
    o.tile_rows, o.kblock, o.precond = int(tile_rows), int(kblock), int(precond)
    _check(lib.pdst_lsqr_batched(nsys, hs, nr, dp, wv, lp, int(itmax), float(tol), DTYPES[dtype],
                                 mp, infos, ctypes.byref(o), _stream(stream)))
    out_infos, k = [], 0
    for r in R:
        out_infos.append([infos[k + i].as_dict() for i in range(r)])
        k += r
    return m_outs, out_infos, {"chosen_tile_rows": o.chosen_tile_rows,
                               "kernel_launches": o.kernel_launches,
                               "tune_ms": list(o.tune_ms)}


MLP_NFEAT, MLP_HIDDEN = 8, 64
MLP_NPARAM = 2 * 8 + 64 * 8 + 64 + 64 * 64 + 64 + 64 + 1
MLP_NTRAIN = MLP_NPARAM - 16


def mlp_forward(params, feat, want_D=True, want_logD=False, stream=None):
    """pdst_mlp_forward: returns (D float64, logD float32) CUDA tensors (or None)."""
    import torch
    n = feat.shape[0]
    D = torch.empty(n, dtype=torch.float64, device="cuda") if want_D else None
    L = torch.empty(n, dtype=torch.float32, device="cuda") if want_logD else None
    _check(load().pdst_mlp_forward(_dev_ptr(params, MLP_NPARAM, torch.float32, "params"),
                                   _dev_ptr(feat, n * MLP_NFEAT, torch.float32, "feat"), n,
                                   None if D is None else _dev_ptr(D),
                                   None if L is None else _dev_ptr(L), _stream(stream)))
    return D, L


def mlp_grad(params, feat, idx, target, grad=None, stream=None):
    """pdst_mlp_grad: gradient of the mean loss over the batch idx; returns the
    (NTRAIN + 1) float32 tensor whose last entry is the loss."""
    import torch
    if grad is None:
        grad = torch.empty(MLP_NTRAIN + 1, dtype=torch.float32, device="cuda")
    _check(load().pdst_mlp_grad(_dev_ptr(params, MLP_NPARAM, torch.float32, "params"),
                                _dev_ptr(feat, None, torch.float32, "feat"),
                                _dev_ptr(idx, None, torch.int32, "idx"),
                                _dev_ptr(target, None, torch.float32, "target"),
                                int(idx.numel()), _dev_ptr(grad, MLP_NTRAIN + 1), _stream(stream)))
    return grad


def mlp_adam(params, grad, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    import torch
    _check(load().pdst_mlp_adam(_dev_ptr(params, MLP_NPARAM, torch.float32, "params"),
                                _dev_ptr(grad, None, torch.float32, "grad"),
                                _dev_ptr(m, MLP_NTRAIN, torch.float32, "m"),
                                _dev_ptr(v, MLP_NTRAIN, torch.float32, "v"), int(step),
                                lr, beta1, beta2, eps, _stream(stream)))
