"""Python binding of the GB300 Block Krylov-Schur library (libbks_gb300.so).

Argument marshalling only: every step runs in the library's CUDA kernels.
The names follow the C ABI in include/bks.h.  PyTorch supplies device
memory and streams; dense matrices are torch CUDA tensors in column-major
layout (shape (rows, cols), stride (1, ld)).  The library must be built
(``paper_2012_07595_gb300._build.build()``); importing this package never
falls back to another implementation: a missing library raises.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
from typing import Optional

import numpy as np

from . import _build

__all__ = [
    "lib", "BKS_OK", "BKS_F32", "BKS_F64", "BKS_MIRROR", "BKS_VALIDATE_SYMMETRIC",
    "BKS_INPUT_ON_DEVICE", "BKS_PREC_FP64", "BKS_PREC_MIXED", "BKS_VARIANT_BK",
    "BKS_VARIANT_MIN", "BKS_VARIANT_MAX", "BksError", "Tensor", "bks_tensor_create_coo",
    "bks_tensor_destroy", "bks_tensor_info", "bks_tensor_export_coo", "bks_contract_mode1",
    "bks_contract_mode3", "bks_core", "bks_solve", "hooi_solve", "BksParams", "HooiParams",
    "col_major", "library_path", "bks_launch_count", "bks_tensor_autotune",
    "bks_tensor_set_tiles", "bks_batch_solve", "Server", "BKS_ECANCELED", "BKS_EPENDING",
    "BKS_EBUDGET", "BKS_NORM_FRO", "BKS_NORM_LMAX", "bks_s_values", "bks_slice_norms",
    "bks_tensor_scale_slices", "BKS_INNER_PAPER", "BKS_INNER_FAST", "bks_contract_mode1_noalloc",
    "bks_gen_tensor_create_coo", "bks_gen_tensor_dims", "bks_gen_contract", "bks_gen_core",
    "BksGenParams", "bks_gen_solve", "BksGenHooiParams", "bks_gen_hooi_solve",
]

BKS_OK = 0
BKS_EINVAL, BKS_ENOMEM, BKS_ECUDA, BKS_EASYM = -1, -2, -3, -4
BKS_ENOTCONV, BKS_EBREAKDOWN, BKS_ENUMERIC, BKS_EUNSUPPORTED = -5, -6, -7, -8
BKS_ECANCELED, BKS_EPENDING, BKS_EBUDGET = -9, -10, -11
BKS_NORM_FRO, BKS_NORM_LMAX = 0, 1
BKS_BATCH_AUTOTUNE = 1
BKS_SERVE_AUTOTUNE = 1
BKS_F32, BKS_F64 = 1, 2
BKS_MIRROR, BKS_VALIDATE_SYMMETRIC, BKS_INPUT_ON_DEVICE = 1, 2, 4
BKS_PREC_FP64, BKS_PREC_MIXED = 0, 1
BKS_VARIANT_BK, BKS_VARIANT_MIN, BKS_VARIANT_MAX = 0, 1, 2
BKS_INNER_PAPER, BKS_INNER_FAST = 0, 1

_ERRNAMES = {BKS_EINVAL: "BKS_EINVAL", BKS_ENOMEM: "BKS_ENOMEM", BKS_ECUDA: "BKS_ECUDA",
             BKS_EASYM: "BKS_EASYM", BKS_ENOTCONV: "BKS_ENOTCONV",
             BKS_EBREAKDOWN: "BKS_EBREAKDOWN", BKS_ENUMERIC: "BKS_ENUMERIC",
             BKS_EUNSUPPORTED: "BKS_EUNSUPPORTED", BKS_ECANCELED: "BKS_ECANCELED",
             BKS_EPENDING: "BKS_EPENDING", BKS_EBUDGET: "BKS_EBUDGET"}


class BksError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


class _Params(ctypes.Structure):
    _fields_ = [("r1", ctypes.c_int), ("r3", ctypes.c_int), ("stages", ctypes.c_int),
                ("block_p", ctypes.c_int), ("tol", ctypes.c_double),
                ("max_outer", ctypes.c_int), ("max_inner", ctypes.c_int),
                ("variant", ctypes.c_int), ("precision", ctypes.c_int),
                ("refine_sweeps", ctypes.c_int), ("seed", ctypes.c_uint64),
                ("drop_tol", ctypes.c_double), ("inner_tol", ctypes.c_double),
                ("tol_scale_free", ctypes.c_int), ("mixed_tol", ctypes.c_double),
                ("inner_schedule", ctypes.c_int)]


class _Info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("converged", ctypes.c_int),
                ("grad_rel", ctypes.c_double), ("normF", ctypes.c_double),
                ("k1", ctypes.c_int), ("k3", ctypes.c_int), ("inner_sweeps", ctypes.c_int),
                ("fp32_iters", ctypes.c_int), ("seconds", ctypes.c_double),
                ("phase_ms", ctypes.c_double * 5),
                ("history", ctypes.POINTER(ctypes.c_double)), ("history_cap", ctypes.c_int),
                ("history_len", ctypes.c_int), ("k2", ctypes.c_int)]


class _GenParams(ctypes.Structure):
    _fields_ = [("r1", ctypes.c_int), ("r2", ctypes.c_int), ("r3", ctypes.c_int),
                ("stages", ctypes.c_int), ("block_p", ctypes.c_int), ("tol", ctypes.c_double),
                ("max_outer", ctypes.c_int), ("max_inner", ctypes.c_int),
                ("variant", ctypes.c_int), ("tol_scale_free", ctypes.c_int),
                ("seed", ctypes.c_uint64), ("drop_tol", ctypes.c_double),
                ("inner_tol", ctypes.c_double), ("inner_schedule", ctypes.c_int)]


class _GenHooiParams(ctypes.Structure):
    _fields_ = [("r1", ctypes.c_int), ("r2", ctypes.c_int), ("r3", ctypes.c_int),
                ("tol", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("grad_every", ctypes.c_int), ("seed", ctypes.c_uint64)]


class _HooiParams(ctypes.Structure):
    _fields_ = [("r1", ctypes.c_int), ("r3", ctypes.c_int), ("tol", ctypes.c_double),
                ("max_iter", ctypes.c_int), ("grad_every", ctypes.c_int),
                ("precision", ctypes.c_int), ("seed", ctypes.c_uint64),
                ("mixed_tol", ctypes.c_double)]


_lib = None


def bks_launch_count() -> int:
    """Kernels launched by the library since it was loaded."""
    return int(lib().bks_launch_count())


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libbks_gb300.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: run paper_2012_07595_gb300._build.build()")
    L = ctypes.CDLL(path)
    vp, i64, c_int, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    L.bks_tensor_create_coo.argtypes = [i64, i64, i64, vp, vp, vp, vp, c_int, c_int, vp,
                                        ctypes.POINTER(vp)]
    L.bks_tensor_create_coo.restype = c_int
    L.bks_tensor_destroy.argtypes = [vp]
    L.bks_tensor_destroy.restype = None
    L.bks_tensor_info.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64),
                                  ctypes.POINTER(i64), ctypes.POINTER(dbl)]
    L.bks_tensor_info.restype = c_int
    L.bks_tensor_export_coo.argtypes = [vp, vp, vp, vp, vp, vp]
    L.bks_tensor_export_coo.restype = c_int
    L.bks_contract_mode1.argtypes = [vp, vp, i64, c_int, vp, i64, c_int, vp, i64, c_int, vp]
    L.bks_contract_mode1.restype = c_int
    L.bks_contract_mode1_noalloc.argtypes = [vp, vp, i64, c_int, vp, i64, c_int, vp, i64, c_int,
                                             vp]
    L.bks_contract_mode1_noalloc.restype = c_int
    L.bks_contract_mode3.argtypes = [vp, vp, i64, c_int, vp, i64, c_int, vp, i64, c_int, vp]
    L.bks_contract_mode3.restype = c_int
    L.bks_core.argtypes = [vp, vp, i64, c_int, vp, i64, c_int, vp, c_int, vp]
    L.bks_core.restype = c_int
    L.bks_params_default.argtypes = [ctypes.POINTER(_Params)]
    L.bks_params_default.restype = None
    L.hooi_params_default.argtypes = [ctypes.POINTER(_HooiParams)]
    L.hooi_params_default.restype = None
    L.bks_solve.argtypes = [vp, ctypes.POINTER(_Params), vp, vp, vp, vp, vp,
                            ctypes.POINTER(_Info), vp]
    L.bks_solve.restype = c_int
    L.hooi_solve.argtypes = [vp, ctypes.POINTER(_HooiParams), vp, vp, vp, vp, vp,
                             ctypes.POINTER(_Info), vp]
    L.hooi_solve.restype = c_int
    L.bks_tensor_autotune.argtypes = [vp, ctypes.POINTER(c_int), ctypes.POINTER(c_int), vp]
    L.bks_tensor_autotune.restype = c_int
    L.bks_tensor_set_tiles.argtypes = [vp, c_int, c_int, vp]
    L.bks_tensor_set_tiles.restype = c_int
    L.bks_batch_solve.argtypes = [c_int, ctypes.POINTER(vp), ctypes.POINTER(_Params),
                                  ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                  ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(_Info),
                                  ctypes.POINTER(c_int), c_int, c_int, vp]
    L.bks_batch_solve.restype = c_int
    L.bks_server_create.argtypes = [ctypes.c_size_t, c_int, c_int]
    L.bks_server_create.restype = vp
    L.bks_server_submit.argtypes = [vp, i64, i64, i64, vp, vp, vp, vp, c_int, c_int,
                                    ctypes.POINTER(_Params), ctypes.POINTER(ctypes.c_uint64)]
    L.bks_server_submit.restype = c_int
    L.bks_server_poll.argtypes = [vp, ctypes.c_uint64, c_int, vp, vp, vp, ctypes.POINTER(_Info),
                                  ctypes.POINTER(c_int), ctypes.POINTER(dbl)]
    L.bks_server_poll.restype = c_int
    L.bks_server_cancel.argtypes = [vp, ctypes.c_uint64]
    L.bks_server_cancel.restype = c_int
    L.bks_server_stats.argtypes = [vp, ctypes.POINTER(c_int), ctypes.POINTER(c_int),
                                   ctypes.POINTER(c_int), ctypes.POINTER(ctypes.c_size_t)]
    L.bks_server_stats.restype = c_int
    L.bks_server_destroy.argtypes = [vp]
    L.bks_server_destroy.restype = None
    L.bks_s_values.argtypes = [vp, vp, i64, c_int, vp, i64, c_int, vp, vp, vp]
    L.bks_s_values.restype = c_int
    L.bks_slice_norms.argtypes = [vp, c_int, vp, vp]
    L.bks_slice_norms.restype = c_int
    L.bks_tensor_scale_slices.argtypes = [vp, vp, vp, ctypes.POINTER(vp)]
    L.bks_tensor_scale_slices.restype = c_int
    L.bks_gen_tensor_create_coo.argtypes = [i64, i64, i64, i64, vp, vp, vp, vp, c_int, c_int, vp,
                                            ctypes.POINTER(vp)]
    L.bks_gen_tensor_create_coo.restype = c_int
    L.bks_gen_tensor_dims.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64),
                                      ctypes.POINTER(i64), ctypes.POINTER(c_int)]
    L.bks_gen_tensor_dims.restype = c_int
    L.bks_gen_contract.argtypes = [vp, c_int, vp, i64, c_int, vp, i64, c_int, vp, i64, c_int, vp]
    L.bks_gen_contract.restype = c_int
    L.bks_gen_core.argtypes = [vp, vp, i64, c_int, vp, i64, c_int, vp, i64, c_int, vp, vp]
    L.bks_gen_core.restype = c_int
    L.bks_gen_params_default.argtypes = [ctypes.POINTER(_GenParams)]
    L.bks_gen_params_default.restype = None
    L.bks_gen_solve.argtypes = [vp, ctypes.POINTER(_GenParams), vp, vp, vp, vp, vp, vp, vp,
                                ctypes.POINTER(_Info), vp]
    L.bks_gen_solve.restype = c_int
    L.bks_gen_hooi_params_default.argtypes = [ctypes.POINTER(_GenHooiParams)]
    L.bks_gen_hooi_params_default.restype = None
    L.bks_gen_hooi_solve.argtypes = [vp, ctypes.POINTER(_GenHooiParams), vp, vp, vp, vp, vp, vp,
                                     vp, ctypes.POINTER(_Info), vp]
    L.bks_gen_hooi_solve.restype = c_int
    L.bks_launch_count.argtypes = []
    L.bks_launch_count.restype = ctypes.c_uint64
    L.bks_last_error_string.argtypes = []
    L.bks_last_error_string.restype = ctypes.c_char_p
    _lib = L
    return L


def _check(rc: int, allow=()):
    if rc != BKS_OK and rc not in allow:
        raise BksError(rc, lib().bks_last_error_string().decode())
    return rc


def _stream(stream):
    import torch
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def col_major(x):
    """The same torch matrix with column-major strides (a copy if needed)."""
    if x.dim() == 1:
        x = x.reshape(-1, 1)
    if x.stride(0) == 1 and x.stride(1) >= max(1, x.shape[0]):
        return x
    return x.t().contiguous().t()


def _ld(x) -> int:
    return max(int(x.stride(1)), int(x.shape[0]), 1)


def _dtype_code(x) -> int:
    import torch
    if x.dtype == torch.float64:
        return BKS_F64
    if x.dtype == torch.float32:
        return BKS_F32
    raise TypeError(f"unsupported dtype {x.dtype}")


def _empty_cm(rows, cols, dtype, device):
    import torch
    return torch.empty((cols, rows), dtype=dtype, device=device).t()


class Tensor:
    """Owning handle of a stored tensor: (1,2)-symmetric m x m x n
    (general False, l == m) or general l x m x n (general True)."""

    def __init__(self, handle: ctypes.c_void_p, vdtype: int):
        self._h = handle
        self.vdtype = vdtype
        m, n, nnz, f2 = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double()
        _check(lib().bks_tensor_info(self._h, ctypes.byref(m), ctypes.byref(n), ctypes.byref(nnz),
                                     ctypes.byref(f2)))
        self.m, self.n, self.nnz, self.fro2 = m.value, n.value, nnz.value, f2.value
        l, gen = ctypes.c_int64(), ctypes.c_int()
        _check(lib().bks_gen_tensor_dims(self._h, ctypes.byref(l), None, None, ctypes.byref(gen)))
        self.l, self.general = l.value, bool(gen.value)

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h is not None and self._h.value:
            lib().bks_tensor_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def bks_tensor_create_coo(m: int, n: int, i, j, k, v, mirror: bool = True,
                          validate: bool = False, stream=None) -> Tensor:
    """Create a stored tensor from COO entries.  i, j, k, v are numpy arrays
    (host) or torch CUDA tensors (device); v is float32 or float64."""
    import torch
    flags = (BKS_MIRROR if mirror else 0) | (BKS_VALIDATE_SYMMETRIC if validate else 0)
    keep = []
    if isinstance(i, torch.Tensor):
        flags |= BKS_INPUT_ON_DEVICE
        ii, jj, kk = (x.to(torch.int32).contiguous() for x in (i, j, k))
        vv = v.contiguous()
        vdt = _dtype_code(vv)
        ptrs = [x.data_ptr() for x in (ii, jj, kk, vv)]
        keep = [ii, jj, kk, vv]
        nnz = ii.numel()
    else:
        ii, jj, kk = (np.ascontiguousarray(x, dtype=np.int32) for x in (i, j, k))
        vv = np.ascontiguousarray(v)
        if vv.dtype == np.float64:
            vdt = BKS_F64
        elif vv.dtype == np.float32:
            vdt = BKS_F32
        else:
            raise TypeError(f"unsupported value dtype {vv.dtype}")
        ptrs = [x.ctypes.data if x.size else 0 for x in (ii, jj, kk, vv)]
        keep = [ii, jj, kk, vv]
        nnz = ii.size
    h = ctypes.c_void_p()
    _check(lib().bks_tensor_create_coo(m, n, nnz, *[ctypes.c_void_p(p) for p in ptrs], vdt, flags,
                                       _stream(stream), ctypes.byref(h)))
    del keep
    return Tensor(h, vdt)


def bks_tensor_destroy(t: Tensor):
    t.close()


def bks_tensor_info(t: Tensor):
    return {"m": t.m, "n": t.n, "nnz_stored": t.nnz, "fro2": t.fro2}


def bks_tensor_export_coo(t: Tensor, stream=None):
    """Canonical stored entries (sorted by (i,j,k)) as torch CUDA tensors."""
    import torch
    dt = torch.float64 if t.vdtype == BKS_F64 else torch.float32
    i = torch.empty(t.nnz, dtype=torch.int32, device="cuda")
    j = torch.empty_like(i)
    k = torch.empty_like(i)
    v = torch.empty(t.nnz, dtype=dt, device="cuda")
    _check(lib().bks_tensor_export_coo(t.handle, ctypes.c_void_p(i.data_ptr()),
                                       ctypes.c_void_p(j.data_ptr()),
                                       ctypes.c_void_p(k.data_ptr()),
                                       ctypes.c_void_p(v.data_ptr()), _stream(stream)))
    return i, j, k, v


def bks_s_values(t: Tensor, U, W, stream=None):
    """S-values of Section 2.6 at (U, U, W): (s1, s3, gap1, gap3) with s1
    holding the r1 S-values of mode 1 and s_{r1+1}^(1) last (numpy), s3
    likewise for mode 3, gap_k = s_{r_k}^(k) - s_{r_k+1}^(k)."""
    import torch
    U = col_major(U.to(device="cuda", dtype=torch.float64))
    W = col_major(W.to(device="cuda", dtype=torch.float64))
    r1, r3 = U.shape[1], W.shape[1]
    s1 = np.zeros(r1 + 1)
    s3 = np.zeros(r3 + 1)
    _check(lib().bks_s_values(t.handle, ctypes.c_void_p(U.data_ptr()), _ld(U), r1,
                              ctypes.c_void_p(W.data_ptr()), _ld(W), r3,
                              s1.ctypes.data_as(ctypes.c_void_p), s3.ctypes.data_as(ctypes.c_void_p),
                              _stream(stream)))
    return s1, s3, float(s1[-2] - s1[-1]), float(s3[-2] - s3[-1])


def bks_slice_norms(t: Tensor, kind: str = "fro", stream=None):
    """Per-slice norms (Section 7) as a torch CUDA FP64 tensor of n values:
    kind "fro" (Frobenius) or "lmax" (largest eigenvalue)."""
    import torch
    code = {"fro": BKS_NORM_FRO, "lmax": BKS_NORM_LMAX}[kind]
    out = torch.empty(t.n, dtype=torch.float64, device="cuda")
    _check(lib().bks_slice_norms(t.handle, code, ctypes.c_void_p(out.data_ptr()), _stream(stream)))
    return out


def bks_tensor_scale_slices(t: Tensor, scales, stream=None) -> Tensor:
    """A new tensor with slice k scaled by scales[k] (n values)."""
    import torch
    sc = torch.as_tensor(scales, dtype=torch.float64).to("cuda").contiguous()
    if sc.numel() != t.n:
        raise ValueError("scales must have n entries")
    h = ctypes.c_void_p()
    _check(lib().bks_tensor_scale_slices(t.handle, ctypes.c_void_p(sc.data_ptr()), _stream(stream),
                                         ctypes.byref(h)))
    return Tensor(h, t.vdtype)


def bks_contract_mode1(t: Tensor, X, Y, out=None, stream=None):
    """unfold_1(A.(X,Y)_{2,3}): m x (p q), column a + p b."""
    X, Y = col_major(X), col_major(Y)
    p, q = X.shape[1], Y.shape[1]
    if out is None:
        out = _empty_cm(t.m, p * q, X.dtype, X.device)
    _check(lib().bks_contract_mode1(t.handle, ctypes.c_void_p(X.data_ptr()), _ld(X), p,
                                    ctypes.c_void_p(Y.data_ptr()), _ld(Y), q,
                                    ctypes.c_void_p(out.data_ptr()), _ld(out), _dtype_code(X),
                                    _stream(stream)))
    return out


def bks_contract_mode1_noalloc(t: Tensor, X, Y, out, stream=None):
    """bks_contract_mode1 for callers that cannot allocate device memory: the
    library uses its fixed 32 MiB device scratch array instead of
    allocating, and this wrapper allocates nothing either.  X (m x p), Y
    (n x q) and `out` (m x p q) must be column-major CUDA tensors (stride
    (1, ld), ld >= rows) of one dtype (float32 or float64) on one device;
    anything else raises instead of being copied."""
    import torch
    for name, x, rows in (("X", X, t.m), ("Y", Y, t.n), ("out", out, t.m)):
        if not isinstance(x, torch.Tensor) or x.dim() != 2 or not x.is_cuda:
            raise ValueError(f"{name} must be a 2-D CUDA tensor")
        if x.shape[0] != rows or x.stride(0) != 1 or (x.shape[1] > 1 and x.stride(1) < rows):
            raise ValueError(f"{name} must be column-major with {rows} rows (stride (1, ld), "
                             f"ld >= {rows}); got shape {tuple(x.shape)}, "
                             f"stride {tuple(x.stride())}")
    if not (X.dtype == Y.dtype == out.dtype) or X.dtype not in (torch.float32, torch.float64):
        raise ValueError("X, Y and out must share one dtype, float32 or float64")
    if not (X.device == Y.device == out.device):
        raise ValueError("X, Y and out must be on one device")
    p, q = X.shape[1], Y.shape[1]
    if out.shape[1] != p * q:
        raise ValueError(f"out must have p*q = {p * q} columns, not {out.shape[1]}")
    _check(lib().bks_contract_mode1_noalloc(t.handle, ctypes.c_void_p(X.data_ptr()), _ld(X), p,
                                            ctypes.c_void_p(Y.data_ptr()), _ld(Y), q,
                                            ctypes.c_void_p(out.data_ptr()), _ld(out),
                                            _dtype_code(X), _stream(stream)))
    return out


def bks_contract_mode3(t: Tensor, X, X2=None, out=None, stream=None):
    """unfold_3(A.(X,X2)_{1,2}): n x (p q); X2 None -> triangle n x p(p+1)/2."""
    X = col_major(X)
    p = X.shape[1]
    if X2 is not None:
        X2 = col_major(X2)
        q = X2.shape[1]
        w = p * q
        x2p, ld2 = ctypes.c_void_p(X2.data_ptr()), _ld(X2)
    else:
        q, w = p, p * (p + 1) // 2
        x2p, ld2 = ctypes.c_void_p(0), t.m
    if out is None:
        out = _empty_cm(t.n, w, X.dtype, X.device)
    _check(lib().bks_contract_mode3(t.handle, ctypes.c_void_p(X.data_ptr()), _ld(X), p, x2p, ld2,
                                    q, ctypes.c_void_p(out.data_ptr()), _ld(out),
                                    _dtype_code(X), _stream(stream)))
    return out


def bks_core(t: Tensor, U, W, stream=None):
    """A.(U,U,W) as an r1 x r1 x r3 tensor (torch, column-major flattening)."""
    import torch
    U, W = col_major(U), col_major(W)
    r1, r3 = U.shape[1], W.shape[1]
    F = torch.empty(r1 * r1 * r3, dtype=U.dtype, device=U.device)
    _check(lib().bks_core(t.handle, ctypes.c_void_p(U.data_ptr()), _ld(U), r1,
                          ctypes.c_void_p(W.data_ptr()), _ld(W), r3,
                          ctypes.c_void_p(F.data_ptr()), _dtype_code(U), _stream(stream)))
    return F.reshape(r3, r1, r1).permute(2, 1, 0)


@dataclasses.dataclass
class BksParams:
    r1: int = 2
    r3: int = 2
    stages: int = 2
    block_p: int = 4
    tol: float = 1e-10
    max_outer: int = 500
    max_inner: int = 1000
    variant: int = BKS_VARIANT_BK
    precision: int = BKS_PREC_FP64
    refine_sweeps: int = 1
    seed: int = 1
    drop_tol: float = 1e-14
    inner_tol: float = 0.0
    tol_scale_free: int = 0
    mixed_tol: float = 1e-4
    inner_schedule: int = BKS_INNER_PAPER

    def to_c(self) -> _Params:
        p = _Params()
        for f in dataclasses.fields(self):
            setattr(p, f.name, getattr(self, f.name))
        return p


@dataclasses.dataclass
class HooiParams:
    r1: int = 2
    r3: int = 2
    tol: float = 1e-10
    max_iter: int = 5000
    grad_every: int = 10
    precision: int = BKS_PREC_FP64
    seed: int = 1
    mixed_tol: float = 1e-4

    def to_c(self) -> _HooiParams:
        p = _HooiParams()
        for f in dataclasses.fields(self):
            setattr(p, f.name, getattr(self, f.name))
        return p


def _solve(fn, t: Tensor, cparams, r1, r3, U0, W0, stream, history_cap, raise_notconv):
    import torch
    U = _empty_cm(t.m, r1, torch.float64, "cuda")
    W = _empty_cm(t.n, r3, torch.float64, "cuda")
    F = torch.empty(r1 * r1 * r3, dtype=torch.float64, device="cuda")
    hist = (ctypes.c_double * (2 * max(history_cap, 1)))()
    info = _Info()
    info.history = ctypes.cast(hist, ctypes.POINTER(ctypes.c_double))
    info.history_cap = history_cap
    # starts must be column-major with ld = rows
    u0 = U0.to(device="cuda", dtype=torch.float64).t().contiguous().t() if U0 is not None else None
    w0 = W0.to(device="cuda", dtype=torch.float64).t().contiguous().t() if W0 is not None else None
    rc = fn(t.handle, ctypes.byref(cparams),
            ctypes.c_void_p(u0.data_ptr() if u0 is not None else 0),
            ctypes.c_void_p(w0.data_ptr() if w0 is not None else 0),
            ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(W.data_ptr()),
            ctypes.c_void_p(F.data_ptr()), ctypes.byref(info), _stream(stream))
    _check(rc, allow=() if raise_notconv else (BKS_ENOTCONV,))
    out = {"iters": info.iters, "converged": bool(info.converged), "grad_rel": info.grad_rel,
           "normF": info.normF, "k1": info.k1, "k3": info.k3,
           "inner_sweeps": info.inner_sweeps, "fp32_iters": info.fp32_iters,
           "seconds": info.seconds, "status": rc,
           "phase_ms": dict(zip(["stage1", "expand", "core", "inner", "restart"],
                                list(info.phase_ms))),
           "history": [(hist[2 * q], hist[2 * q + 1]) for q in range(info.history_len)]}
    return U, W, F.reshape(r3, r1, r1).permute(2, 1, 0), out


def bks_solve(t: Tensor, params: Optional[BksParams] = None, U0=None, W0=None, stream=None,
              history_cap: int = 1000, raise_notconv: bool = False):
    """Tensor Krylov-Schur (Algorithm 5).  Returns (U, W, F, info) with U
    (m x r1), W (n x r3) FP64 CUDA tensors and F (r1 x r1 x r3)."""
    params = params or BksParams()
    return _solve(lib().bks_solve, t, params.to_c(), params.r1, params.r3, U0, W0, stream,
                  history_cap, raise_notconv)


def hooi_solve(t: Tensor, params: Optional[HooiParams] = None, U0=None, W0=None, stream=None,
               history_cap: int = 1000, raise_notconv: bool = False):
    """HOOI for (1,2)-symmetric tensors (Section 6.1)."""
    params = params or HooiParams()
    return _solve(lib().hooi_solve, t, params.to_c(), params.r1, params.r3, U0, W0, stream,
                  history_cap, raise_notconv)


def bks_tensor_autotune(t: Tensor, stream=None):
    """Pick the contraction work tiles of this tensor by timing; returns
    (tile, split)."""
    tile, split = ctypes.c_int(), ctypes.c_int()
    _check(lib().bks_tensor_autotune(t.handle, ctypes.byref(tile), ctypes.byref(split),
                                     _stream(stream)))
    return tile.value, split.value


def bks_tensor_set_tiles(t: Tensor, tile: int, split: int, stream=None):
    _check(lib().bks_tensor_set_tiles(t.handle, tile, split, _stream(stream)))


def bks_batch_solve(tensors, params, U0s=None, W0s=None, nstreams: int = 4,
                    autotune: bool = True, stream=None):
    """Independent BKS solves run concurrently on `nstreams` streams.
    Returns a list of (U, W, F, info, status) per job."""
    import torch
    n = len(tensors)
    params = list(params) if isinstance(params, (list, tuple)) else [params] * n
    Ts = (ctypes.c_void_p * n)(*[t.handle.value for t in tensors])
    Ps = (_Params * n)(*[p.to_c() for p in params])
    outs = []
    keep = []
    for q in range(n):
        r1, r3 = params[q].r1, params[q].r3
        U = _empty_cm(tensors[q].m, r1, torch.float64, "cuda")
        W = _empty_cm(tensors[q].n, r3, torch.float64, "cuda")
        F = torch.empty(r1 * r1 * r3, dtype=torch.float64, device="cuda")
        outs.append((U, W, F))

    def ptrs(xs):
        return (ctypes.c_void_p * n)(*[(x.data_ptr() if x is not None else 0) for x in xs])

    u0 = w0 = None
    if U0s is not None:
        keep = [x.to(device="cuda", dtype=torch.float64).t().contiguous().t() for x in U0s]
        u0 = ptrs(keep)
    if W0s is not None:
        keepw = [x.to(device="cuda", dtype=torch.float64).t().contiguous().t() for x in W0s]
        keep += keepw
        w0 = ptrs(keepw)
    infos = (_Info * n)()
    status = (ctypes.c_int * n)()
    lib().bks_batch_solve(n, Ts, Ps, u0, w0, ptrs([o[0] for o in outs]),
                          ptrs([o[1] for o in outs]), ptrs([o[2] for o in outs]), infos, status,
                          nstreams, BKS_BATCH_AUTOTUNE if autotune else 0, _stream(stream))
    res = []
    for q in range(n):
        r1, r3 = params[q].r1, params[q].r3
        i = infos[q]
        d = {"iters": i.iters, "converged": bool(i.converged), "grad_rel": i.grad_rel,
             "normF": i.normF, "k1": i.k1, "k3": i.k3, "fp32_iters": i.fp32_iters,
             "seconds": i.seconds}
        U, W, F = outs[q]
        res.append((U, W, F.reshape(r3, r1, r1).permute(2, 1, 0), d, status[q]))
    return res


class Server:
    """Continuous-batching BKS server: jobs wait in a FIFO queue and are
    admitted as slots and device memory (the budget) free up."""

    def __init__(self, hbm_budget: int, max_slots: int = 4, autotune: bool = True):
        h = lib().bks_server_create(int(hbm_budget), int(max_slots),
                                    BKS_SERVE_AUTOTUNE if autotune else 0)
        if not h:
            raise BksError(BKS_EINVAL, lib().bks_last_error_string().decode())
        self._h = ctypes.c_void_p(h)
        self._shapes = {}

    def submit(self, m, n, i, j, k, v, params: BksParams, mirror: bool = True) -> int:
        ii, jj, kk = (np.ascontiguousarray(x, dtype=np.int32) for x in (i, j, k))
        vv = np.ascontiguousarray(v)
        vdt = BKS_F64 if vv.dtype == np.float64 else BKS_F32
        if vv.dtype not in (np.float64, np.float32):
            raise TypeError("values must be float32 or float64")
        t = ctypes.c_uint64()
        cp = params.to_c()
        _check(lib().bks_server_submit(self._h, m, n, ii.size,
                                       *[ctypes.c_void_p(x.ctypes.data if x.size else 0)
                                         for x in (ii, jj, kk, vv)],
                                       vdt, BKS_MIRROR if mirror else 0, ctypes.byref(cp),
                                       ctypes.byref(t)))
        self._shapes[t.value] = (m, n, params.r1, params.r3)
        return t.value

    def poll(self, ticket: int, wait: bool = True):
        """None while pending (wait=False); else a dict with U, W, F (numpy),
        info, status and latency."""
        m, n, r1, r3 = self._shapes[ticket]
        U = np.empty((m, r1), order="F")
        W = np.empty((n, r3), order="F")
        F = np.empty(r1 * r1 * r3)
        info = _Info()
        st = ctypes.c_int()
        lat = ctypes.c_double()
        rc = lib().bks_server_poll(self._h, ticket, 1 if wait else 0,
                                   ctypes.c_void_p(U.ctypes.data), ctypes.c_void_p(W.ctypes.data),
                                   ctypes.c_void_p(F.ctypes.data), ctypes.byref(info),
                                   ctypes.byref(st), ctypes.byref(lat))
        if rc == BKS_EPENDING:
            return None
        _check(rc)
        del self._shapes[ticket]
        return {"U": U, "W": W, "F": F.reshape(r1, r1, r3, order="F"), "status": st.value,
                "latency_s": lat.value, "iters": info.iters, "converged": bool(info.converged),
                "normF": info.normF, "grad_rel": info.grad_rel,
                "error": lib().bks_last_error_string().decode() if st.value else ""}

    def cancel(self, ticket: int):
        _check(lib().bks_server_cancel(self._h, ticket))

    def stats(self):
        q, r, f = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        b = ctypes.c_size_t()
        _check(lib().bks_server_stats(self._h, ctypes.byref(q), ctypes.byref(r), ctypes.byref(f),
                                      ctypes.byref(b)))
        return {"queued": q.value, "running": r.value, "finished": f.value,
                "resident_bytes": b.value}

    def close(self):
        if self._h is not None and self._h.value:
            lib().bks_server_destroy(self._h)
        self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- general (nonsymmetric) l x m x n tensors (Section 5) --------------------
def _coo_ptrs(i, j, k, v):
    import torch
    if isinstance(i, torch.Tensor):
        ii, jj, kk = (x.to(torch.int32).contiguous() for x in (i, j, k))
        vv = v.contiguous()
        return BKS_INPUT_ON_DEVICE, _dtype_code(vv), [x.data_ptr() for x in (ii, jj, kk, vv)], \
            [ii, jj, kk, vv], ii.numel()
    ii, jj, kk = (np.ascontiguousarray(x, dtype=np.int32) for x in (i, j, k))
    vv = np.ascontiguousarray(v)
    if vv.dtype == np.float64:
        vdt = BKS_F64
    elif vv.dtype == np.float32:
        vdt = BKS_F32
    else:
        raise TypeError(f"unsupported value dtype {vv.dtype}")
    return 0, vdt, [x.ctypes.data if x.size else 0 for x in (ii, jj, kk, vv)], \
        [ii, jj, kk, vv], ii.size


def bks_gen_tensor_create_coo(l: int, m: int, n: int, i, j, k, v, stream=None) -> Tensor:
    """Store a general l x m x n tensor from COO entries (numpy host arrays
    or torch CUDA tensors); duplicates are summed, nothing is mirrored."""
    flags, vdt, ptrs, keep, nnz = _coo_ptrs(i, j, k, v)
    h = ctypes.c_void_p()
    _check(lib().bks_gen_tensor_create_coo(l, m, n, nnz, *[ctypes.c_void_p(p) for p in ptrs], vdt,
                                           flags, _stream(stream), ctypes.byref(h)))
    del keep
    return Tensor(h, vdt)


def bks_gen_tensor_dims(t: Tensor):
    return {"l": t.l, "m": t.m, "n": t.n, "general": t.general}


def bks_gen_contract(t: Tensor, mode: int, B1, B2, out=None, stream=None):
    """The mode-`mode` block contraction of a general tensor: mode 1 ->
    l x p q from (B1 m x p, B2 n x q), mode 2 -> m x p q from (B1 l x p,
    B2 n x q), mode 3 -> n x p q from (B1 l x p, B2 m x q); column a + p b."""
    B1, B2 = col_major(B1), col_major(B2)
    p, q = B1.shape[1], B2.shape[1]
    rows = {1: t.l, 2: t.m, 3: t.n}.get(mode, 1)  # the library rejects other modes
    if out is None:
        out = _empty_cm(rows, p * q, B1.dtype, B1.device)
    _check(lib().bks_gen_contract(t.handle, mode, ctypes.c_void_p(B1.data_ptr()), _ld(B1), p,
                                  ctypes.c_void_p(B2.data_ptr()), _ld(B2), q,
                                  ctypes.c_void_p(out.data_ptr()), _ld(out), _dtype_code(B1),
                                  _stream(stream)))
    return out


def bks_gen_core(t: Tensor, X, Y, Z, stream=None):
    """C = A.(X,Y,Z) of a general tensor as a k1 x k2 x k3 torch FP64 tensor."""
    import torch
    X, Y, Z = (col_major(x.to(torch.float64)) for x in (X, Y, Z))
    k1, k2, k3 = X.shape[1], Y.shape[1], Z.shape[1]
    C = torch.empty(k1 * k2 * k3, dtype=torch.float64, device=X.device)
    _check(lib().bks_gen_core(t.handle, ctypes.c_void_p(X.data_ptr()), _ld(X), k1,
                              ctypes.c_void_p(Y.data_ptr()), _ld(Y), k2,
                              ctypes.c_void_p(Z.data_ptr()), _ld(Z), k3,
                              ctypes.c_void_p(C.data_ptr()), _stream(stream)))
    return C.reshape(k3, k2, k1).permute(2, 1, 0)


@dataclasses.dataclass
class BksGenParams:
    r1: int = 2
    r2: int = 2
    r3: int = 2
    stages: int = 2
    block_p: int = 4
    tol: float = 1e-10
    max_outer: int = 500
    max_inner: int = 1000
    variant: int = BKS_VARIANT_BK
    tol_scale_free: int = 0
    seed: int = 1
    drop_tol: float = 1e-14
    inner_tol: float = 0.0
    inner_schedule: int = BKS_INNER_PAPER

    def to_c(self) -> _GenParams:
        p = _GenParams()
        for f in dataclasses.fields(self):
            setattr(p, f.name, getattr(self, f.name))
        return p


@dataclasses.dataclass
class BksGenHooiParams:
    r1: int = 2
    r2: int = 2
    r3: int = 2
    tol: float = 1e-10
    max_iter: int = 5000
    grad_every: int = 10
    seed: int = 1

    def to_c(self) -> _GenHooiParams:
        p = _GenHooiParams()
        for f in dataclasses.fields(self):
            setattr(p, f.name, getattr(self, f.name))
        return p


def bks_gen_solve(t: Tensor, params: Optional[BksGenParams] = None, U0=None, V0=None, W0=None,
                  stream=None, history_cap: int = 1000, raise_notconv: bool = False):
    """Tensor Krylov-Schur for a general tensor (Algorithm 5, Section 5).
    Returns (U, V, W, F, info): U l x r1, V m x r2, W n x r3 FP64 CUDA
    tensors and F r1 x r2 x r3."""
    return _gen_solve(lib().bks_gen_solve, t, params or BksGenParams(), U0, V0, W0, stream,
                      history_cap, raise_notconv)


def bks_gen_hooi_solve(t: Tensor, params: Optional[BksGenHooiParams] = None, U0=None, V0=None,
                       W0=None, stream=None, history_cap: int = 1000,
                       raise_notconv: bool = False):
    """HOOI for a general tensor (Section 6.1).  Returns (U, V, W, F, info)
    as bks_gen_solve."""
    return _gen_solve(lib().bks_gen_hooi_solve, t, params or BksGenHooiParams(), U0, V0, W0,
                      stream, history_cap, raise_notconv)


def _gen_solve(fn, t: Tensor, prm, U0, V0, W0, stream, history_cap, raise_notconv):
    import torch
    r = (prm.r1, prm.r2, prm.r3)
    dims = (t.l, t.m, t.n)
    outs = [_empty_cm(dims[q], r[q], torch.float64, "cuda") for q in range(3)]
    F = torch.empty(r[0] * r[1] * r[2], dtype=torch.float64, device="cuda")
    hist = (ctypes.c_double * (2 * max(history_cap, 1)))()
    info = _Info()
    info.history = ctypes.cast(hist, ctypes.POINTER(ctypes.c_double))
    info.history_cap = history_cap
    starts = [x.to(device="cuda", dtype=torch.float64).t().contiguous().t() if x is not None
              else None for x in (U0, V0, W0)]
    cp = prm.to_c()
    rc = fn(t.handle, ctypes.byref(cp),
            *[ctypes.c_void_p(x.data_ptr() if x is not None else 0) for x in starts],
            *[ctypes.c_void_p(x.data_ptr()) for x in outs],
            ctypes.c_void_p(F.data_ptr()), ctypes.byref(info), _stream(stream))
    _check(rc, allow=() if raise_notconv else (BKS_ENOTCONV,))
    out = {"iters": info.iters, "converged": bool(info.converged), "grad_rel": info.grad_rel,
           "normF": info.normF, "k1": info.k1, "k2": info.k2, "k3": info.k3,
           "inner_sweeps": info.inner_sweeps, "seconds": info.seconds, "status": rc,
           "history": [(hist[2 * q], hist[2 * q + 1]) for q in range(info.history_len)]}
    return outs[0], outs[1], outs[2], F.reshape(r[2], r[1], r[0]).permute(2, 1, 0), out
