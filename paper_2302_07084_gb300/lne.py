"""Python binding of the C ABI in ``include/lne.h`` (argument marshalling only).

Every computation runs in the CUDA library ``_build/liblne.so``; PyTorch only
provides device memory and streams. There is no CPU fallback: if the library
is missing or fails to load, every entry point raises.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
from typing import Optional, Sequence

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "liblne.so")

LNE_OK = 0
ERRORS = {-1: "LNE_ERR_INVALID", -2: "LNE_ERR_OOM", -3: "LNE_ERR_CUDA", -4: "LNE_ERR_TIMEOUT",
          -5: "LNE_ERR_UNSUPPORTED", -6: "LNE_ERR_NUMERIC"}
PREC_FP32 = 0
PREC_BF16_MIXED = 1
SKETCH_GAUSSIAN = 0
SKETCH_SPARSE_SIGN = 1
SKETCH_VERY_SPARSE = 2

EXPORTED = [
    "lne_create", "lne_destroy", "lne_last_error", "lne_workspace_bytes", "lne_trim",
    "lne_sample_pairs", "lne_sparsifier_counts", "lne_sparsifier_csr", "lne_gaussian_sketch",
    "lne_sparse_sign_sketch", "lne_sparse_sign_spmm", "lne_very_sparse_sketch", "lne_very_sparse_spmm",
    "lne_spmm", "lne_cholqr2", "lne_rsvd", "lne_propagate", "lne_embed",
    "lne_kernel_launches", "lne_trace_enable", "lne_trace_read", "lne_set_option",
    "lne_svd_small", "lne_svd_small_noalloc", "lne_macro_f1", "lne_tune_batch", "lne_tune_tasks",
    "lne_surrogate_init", "lne_surrogate_fit_scaling", "lne_surrogate_set_params", "lne_surrogate_get_params",
    "lne_surrogate_train", "lne_surrogate_predict", "lne_surrogate_grad",
]
SURROGATE_INPUTS = 30
SURROGATE_PARAMS = 73_985
OPT_AGGREGATION = 1
OPT_SPMM_THREADS = 2
OPT_TUNE_WORKERS = 3
OPT_DENSE_PRODUCT = 4
OPT_STRATIFIED = 5
OPT_SPMM_COLBLOCK = 6
OPT_SPMM_VBLOCK = 7
AGG_AUTO, AGG_TABLE, AGG_BUCKET, AGG_SORT = 0, 1, 2, 3


class LneError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class _Graph(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("indptr", ctypes.c_void_p),
                ("indices", ctypes.c_void_p), ("weights", ctypes.c_void_p)]


class _Task(ctypes.Structure):
    _fields_ = [("graph", _Graph), ("labels", ctypes.c_void_p), ("L", ctypes.c_int32), ("train", ctypes.c_void_p),
                ("n_train", ctypes.c_int64), ("test", ctypes.c_void_p), ("n_test", ctypes.c_int64)]


class _Params(ctypes.Structure):
    _fields_ = [("T", ctypes.c_int32), ("s", ctypes.POINTER(ctypes.c_double)), ("samples", ctypes.c_double),
                ("b", ctypes.c_double), ("d", ctypes.c_int32), ("oversample", ctypes.c_int32),
                ("q", ctypes.c_int32), ("k", ctypes.c_int32), ("theta", ctypes.c_double),
                ("mu", ctypes.c_double), ("seed", ctypes.c_uint64), ("precision", ctypes.c_int32),
                ("downsample_C", ctypes.c_double), ("sketch", ctypes.c_int32), ("sketch_zeta", ctypes.c_int32)]


class _Csr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("indptr", ctypes.c_void_p),
                ("indices", ctypes.c_void_p), ("data", ctypes.c_void_p)]


class _TraceEntry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 40), ("regions", ctypes.c_int64), ("launches", ctypes.c_int64),
                ("total_ms", ctypes.c_double)]


class _Counts(ctypes.Structure):
    _fields_ = [("nnz", ctypes.c_int64), ("x", ctypes.c_void_p), ("y", ctypes.c_void_p),
                ("count", ctypes.c_void_p), ("total_samples", ctypes.c_int64), ("weight", ctypes.c_void_p),
                ("window", ctypes.c_void_p)]


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not found at {path}; build it with __graft_entry__.build() "
                           "or python paper_2302_07084_gb300/build.py")
    L = ctypes.CDLL(path)
    vp, i64, i32, u64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64
    L.lne_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int]
    L.lne_destroy.argtypes = [vp]
    L.lne_destroy.restype = None
    L.lne_last_error.argtypes = [vp]
    L.lne_last_error.restype = ctypes.c_char_p
    L.lne_workspace_bytes.argtypes = [vp]
    L.lne_workspace_bytes.restype = i64
    L.lne_trim.argtypes = [vp]
    gp, pp = ctypes.POINTER(_Graph), ctypes.POINTER(_Params)
    L.lne_sample_pairs.argtypes = [vp, gp, pp, i64, i64, vp, vp, i64, ctypes.POINTER(i64), vp]
    L.lne_sparsifier_counts.argtypes = [vp, gp, pp, ctypes.POINTER(_Counts), vp]
    L.lne_sparsifier_csr.argtypes = [vp, gp, pp, ctypes.POINTER(_Csr), vp]
    L.lne_gaussian_sketch.argtypes = [vp, i64, i32, u64, vp, i64, vp]
    L.lne_sparse_sign_sketch.argtypes = [vp, i64, i32, i32, u64, vp, i64, vp]
    L.lne_sparse_sign_spmm.argtypes = [vp, ctypes.POINTER(_Csr), i32, i32, u64, vp, i64, vp]
    L.lne_very_sparse_sketch.argtypes = [vp, i64, i32, ctypes.c_double, u64, vp, i64, vp]
    L.lne_very_sparse_spmm.argtypes = [vp, ctypes.POINTER(_Csr), i32, ctypes.c_double, u64, vp, i64, vp]
    L.lne_spmm.argtypes = [vp, ctypes.POINTER(_Csr), vp, i64, i32, vp, i64, i32, vp]
    L.lne_cholqr2.argtypes = [vp, vp, i64, i32, i64, vp, vp]
    L.lne_rsvd.argtypes = [vp, ctypes.POINTER(_Csr), pp, vp, vp, vp, vp]
    L.lne_propagate.argtypes = [vp, gp, pp, vp, vp, vp, vp, vp]
    L.lne_embed.argtypes = [vp, gp, pp, vp, vp]
    L.lne_kernel_launches.argtypes = []
    L.lne_kernel_launches.restype = i64
    L.lne_trace_enable.argtypes = [vp, ctypes.c_int]
    L.lne_set_option.argtypes = [vp, ctypes.c_int, i64]
    L.lne_svd_small.argtypes = [vp, vp, i32, vp, vp, vp]
    L.lne_svd_small_noalloc.argtypes = [vp, i32, vp, vp, vp]
    L.lne_macro_f1.argtypes = [vp, vp, i64, i32, i64, vp, i32, vp, i64, vp, i64, ctypes.c_double, i32,
                               ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), vp]
    L.lne_tune_batch.argtypes = [vp, gp, vp, i32, vp, i32, vp, i64, vp, i64, ctypes.c_double, i32,
                                 ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), vp, vp]
    L.lne_tune_tasks.argtypes = [vp, vp, i32, vp, i32, ctypes.c_double, i32, ctypes.POINTER(ctypes.c_double),
                                 ctypes.POINTER(ctypes.c_double), vp]
    dp = ctypes.POINTER(ctypes.c_double)
    L.lne_surrogate_init.argtypes = [vp, u64, vp]
    L.lne_surrogate_fit_scaling.argtypes = [vp, vp, i64, vp]
    L.lne_surrogate_set_params.argtypes = [vp, vp, vp, vp, vp]
    L.lne_surrogate_get_params.argtypes = [vp, vp, vp, vp, vp]
    L.lne_surrogate_train.argtypes = [vp, vp, vp, i64, i32, i32, ctypes.c_float, u64, dp, vp]
    L.lne_surrogate_predict.argtypes = [vp, vp, i64, vp, vp]
    L.lne_surrogate_grad.argtypes = [vp, vp, vp, i64, vp, dp, vp]
    L.lne_trace_read.argtypes = [vp, ctypes.POINTER(_TraceEntry), ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    _lib = L
    return L


@dataclasses.dataclass
class Params:
    """Method parameters in the paper's notation."""
    T: int = 10
    s: Sequence[float] = dataclasses.field(default_factory=lambda: [0.1] * 10)
    samples: float = 1.0          # S, total edge samples
    b: float = 1.0
    d: int = 128
    oversample: int = 16
    q: int = 1
    k: int = 10
    theta: float = 0.5
    mu: float = 0.2
    seed: int = 0
    precision: int = PREC_FP32
    downsample_C: float = 0.0     # edge downsampling constant C (0 = off)
    sketch: int = SKETCH_GAUSSIAN  # test matrix of the randomized SVD
    sketch_zeta: int = 0          # sparse sign: nonzeros per row (0 = min(8, c)); very sparse: s (0 = sqrt(n))

    def _c(self):
        s = np.ascontiguousarray(np.asarray(self.s, dtype=np.float64))
        arr = (ctypes.c_double * max(1, len(s)))(*s.tolist())
        p = _Params(int(self.T), ctypes.cast(arr, ctypes.POINTER(ctypes.c_double)), float(self.samples),
                    float(self.b), int(self.d), int(self.oversample), int(self.q), int(self.k),
                    float(self.theta), float(self.mu), int(self.seed) & 0xFFFFFFFFFFFFFFFF,
                    int(self.precision), float(self.downsample_C), int(self.sketch), int(self.sketch_zeta))
        return p, arr


def _check_tensor(name, t, device, dtype=None, shape=None, min_rows=None, cols=None, min_numel=None):
    """Checks a tensor whose raw pointer goes to the library: on `device`,
    contiguous, of the given dtype (or one of a tuple of them), and at least as
    large as what the library reads or writes through it. A mismatch raises
    ValueError before anything is launched."""
    if not isinstance(t, torch.Tensor):
        raise ValueError(f"{name} must be a tensor, got {type(t).__name__}")
    if t.device != device:
        raise ValueError(f"{name} is on {t.device}; the library needs it on {device}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None:
        ok = dtype if isinstance(dtype, tuple) else (dtype,)
        if t.dtype not in ok:
            raise ValueError(f"{name} must be {' or '.join(str(x) for x in ok)}, got {t.dtype}")
    if shape is not None and tuple(t.shape) != tuple(int(x) for x in shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if min_rows is not None and (t.dim() < 1 or t.shape[0] < min_rows):
        raise ValueError(f"{name} needs at least {min_rows} rows, got shape {tuple(t.shape)}")
    if cols is not None and (t.dim() != 2 or t.shape[1] != cols):
        raise ValueError(f"{name} must be 2-D with {cols} columns, got shape {tuple(t.shape)}")
    if min_numel is not None and t.numel() < min_numel:
        raise ValueError(f"{name} needs at least {min_numel} elements, got {t.numel()}")
    return t


class DeviceGraph:
    """A CSR graph resident on the GPU (int64 indptr, int32 indices, optional
    positive integer arc weights held as their uint32 bits)."""

    def __init__(self, indptr, indices, device="cuda", weights=None):
        self.indptr = torch.as_tensor(np.asarray(indptr, dtype=np.int64)).to(device)
        self.indices = torch.as_tensor(np.asarray(indices, dtype=np.int32)).to(device)
        self.n = int(self.indptr.numel() - 1)
        self.nnz = int(self.indices.numel())
        self.weights = None
        if weights is not None:
            w = np.ascontiguousarray(weights, dtype=np.uint32)
            self.weights = torch.as_tensor(w.view(np.int32)).to(device)

    @classmethod
    def from_graph(cls, g, device="cuda", weights=None):
        return cls(g.indptr, g.indices, device, weights=weights)

    @classmethod
    def from_tensors(cls, indptr: torch.Tensor, indices: torch.Tensor):
        """Wrap CSR arrays already on the device (int64 indptr, int32 indices)."""
        g = cls.__new__(cls)
        g.indptr = indptr.contiguous()
        g.indices = indices.contiguous()
        g.n = int(indptr.numel() - 1)
        g.nnz = int(indices.numel())
        g.weights = None
        return g

    def _c(self, device):
        """The C struct; the arrays are checked against n and nnz first (the
        library reads indptr[0..n] and indices / weights [0..nnz))."""
        _check_tensor("graph indptr", self.indptr, device, torch.int64, min_numel=self.n + 1)
        _check_tensor("graph indices", self.indices, device, torch.int32, min_numel=self.nnz)
        if self.weights is not None:
            _check_tensor("graph weights", self.weights, device, torch.int32, min_numel=self.nnz)
        w = self.weights.data_ptr() if self.weights is not None and self.nnz else None
        return _Graph(self.n, self.nnz, self.indptr.data_ptr(), self.indices.data_ptr() if self.nnz else None, w)


class _DevView:
    """Zero-copy view of context-owned device memory for torch.as_tensor."""

    def __init__(self, ptr, n, typestr):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": typestr, "data": (int(ptr or 0), False),
                                         "version": 3, "strides": None}


def _view(ptr, n, typestr, dtype, device):
    if n == 0:
        return torch.empty(0, dtype=dtype, device=device)
    return torch.as_tensor(_DevView(ptr, n, typestr), device=device)


def _own(ptr, n, typestr, dtype, device):
    if n == 0:
        return torch.empty(0, dtype=dtype, device=device)
    return torch.as_tensor(_DevView(ptr, n, typestr), device=device).clone()


def default_downsample_C(n: int) -> float:
    """The downsampling constant the paper takes, C = ln n (Sec. 4.1)."""
    return float(np.log(max(int(n), 2)))


def svd_small_noalloc(R: torch.Tensor, U: torch.Tensor, sigma: torch.Tensor) -> int:
    """lne_svd_small_noalloc: writes U (c x c) and sigma (c) of the FP64 matrix R
    without allocating device memory; returns the library's status code.

    The library reads c x c doubles from R and writes c x c into U and c into
    sigma through raw pointers, so the shapes, dtypes and device are checked
    here before the call (a mismatch raises ValueError, nothing is launched)."""
    L = load_library()
    if R.dim() != 2 or R.shape[0] != R.shape[1]:
        raise ValueError(f"R must be square, got shape {tuple(R.shape)}")
    c = int(R.shape[0])
    for name, t, shape in (("R", R, (c, c)), ("U", U, (c, c)), ("sigma", sigma, (c,))):
        if t.dtype != torch.float64:
            raise ValueError(f"{name} must be float64, got {t.dtype}")
        if tuple(t.shape) != shape:
            raise ValueError(f"{name} must have shape {shape}, got {tuple(t.shape)}")
        if not (t.is_cuda and t.is_contiguous()):
            raise ValueError(f"{name} must be a contiguous CUDA tensor")
        if t.device.index != torch.cuda.current_device():
            raise ValueError(f"{name} is on {t.device}, not on the current device")
    return int(L.lne_svd_small_noalloc(_ptr(R), c, _ptr(U), _ptr(sigma), _stream()))


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    if not (t.is_cuda and t.is_contiguous()):
        raise ValueError(f"the library needs a contiguous CUDA tensor, got one on {t.device}")
    return ctypes.c_void_p(t.data_ptr())


class Context:
    """One library context (workspace owner) on a CUDA device."""

    def __init__(self, device: int = 0):
        self.lib = load_library()
        self.device = device
        h = ctypes.c_void_p()
        rc = self.lib.lne_create(ctypes.byref(h), device)
        if rc != 0:
            raise LneError(rc, f"lne_create failed on device {device}")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.lne_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != 0:
            raise LneError(rc, self.lib.lne_last_error(self.h).decode())

    def workspace_bytes(self) -> int:
        return int(self.lib.lne_workspace_bytes(self.h))

    def trim(self):
        self._check(self.lib.lne_trim(self.h))

    def set_option(self, option: int, value: int):
        self._check(self.lib.lne_set_option(self.h, option, value))

    def kernel_launches(self) -> int:
        return int(self.lib.lne_kernel_launches())

    def trace(self, on: bool = True):
        self._check(self.lib.lne_trace_enable(self.h, 1 if on else 0))

    def trace_read(self) -> list[dict]:
        """Per region name: regions run, kernels launched, summed CUDA-event ms."""
        cap = 128
        buf = (_TraceEntry * cap)()
        cnt = ctypes.c_int()
        self._check(self.lib.lne_trace_read(self.h, buf, cap, ctypes.byref(cnt)))
        return [dict(name=buf[i].name.decode(), regions=int(buf[i].regions), launches=int(buf[i].launches),
                     ms=float(buf[i].total_ms)) for i in range(min(cnt.value, cap))]

    @property
    def dev(self):
        return torch.device("cuda", self.device)

    # ---- sparsifier ---------------------------------------------------------
    def sample_pairs(self, g: DeviceGraph, p: Params, arc_begin: int = 0, arc_end: Optional[int] = None,
                     capacity: Optional[int] = None):
        arc_end = g.nnz if arc_end is None else arc_end
        if capacity is None:
            if getattr(g, "weights", None) is not None:   # per-arc rates vary: S + one per arc bounds them
                capacity = int(np.ceil(float(p.samples))) + (arc_end - arc_begin) + 1
            else:
                rate = float(p.samples) / max(g.nnz, 1)
                capacity = int((arc_end - arc_begin) * (np.floor(rate) + 1)) + 1
        u1 = torch.empty(capacity, dtype=torch.int32, device=self.dev)
        v1 = torch.empty(capacity, dtype=torch.int32, device=self.dev)
        cnt = ctypes.c_int64()
        gc = g._c(self.dev)
        pc, keep = p._c()
        self._check(self.lib.lne_sample_pairs(self.h, ctypes.byref(gc), ctypes.byref(pc), arc_begin, arc_end,
                                              _ptr(u1), _ptr(v1), capacity, ctypes.byref(cnt), _stream()))
        return u1[: cnt.value], v1[: cnt.value]

    def sparsifier_counts(self, g: DeviceGraph, p: Params):
        out = _Counts()
        gc = g._c(self.dev)
        pc, keep = p._c()
        self._check(self.lib.lne_sparsifier_counts(self.h, ctypes.byref(gc), ctypes.byref(pc), ctypes.byref(out),
                                                   _stream()))
        # with edge downsampling `weight` (uint64 bit patterns held in int64)
        # replaces `count`
        res = dict(x=_own(out.x, out.nnz, "<i4", torch.int32, self.dev),
                   y=_own(out.y, out.nnz, "<i4", torch.int32, self.dev),
                   total_samples=int(out.total_samples))
        if out.weight:
            res["weight"] = _own(out.weight, out.nnz, "<i8", torch.int64, self.dev)
        else:
            res["count"] = _own(out.count, out.nnz, "<u4", torch.uint32, self.dev)
        if out.window:   # window-stratified counts: (x, y, r, count) entries
            res["window"] = _own(out.window, out.nnz, "|u1", torch.uint8, self.dev)
        return res

    def sparsifier_csr(self, g: DeviceGraph, p: Params, copy: bool = True):
        """The trunc_log sparsifier as a CSR dict. copy=False returns views of
        the context's buffers, valid until the next call on this context."""
        out = _Csr()
        gc = g._c(self.dev)
        pc, keep = p._c()
        self._check(self.lib.lne_sparsifier_csr(self.h, ctypes.byref(gc), ctypes.byref(pc), ctypes.byref(out),
                                                _stream()))
        wrap = _own if copy else _view
        return dict(n=int(out.n), nnz=int(out.nnz),
                    indptr=wrap(out.indptr, out.n + 1, "<i8", torch.int64, self.dev),
                    indices=wrap(out.indices, out.nnz, "<i4", torch.int32, self.dev),
                    data=wrap(out.data, out.nnz, "<f4", torch.float32, self.dev))

    # ---- linear algebra -----------------------------------------------------
    def gaussian_sketch(self, n: int, c: int, seed: int) -> torch.Tensor:
        out = torch.empty((n, c), dtype=torch.float32, device=self.dev)
        self._check(self.lib.lne_gaussian_sketch(self.h, n, c, int(seed) & 0xFFFFFFFFFFFFFFFF, _ptr(out), c,
                                                 _stream()))
        return out

    def sparse_sign_sketch(self, n: int, c: int, zeta: int, seed: int) -> torch.Tensor:
        """The sparse sign test matrix written out densely (n x c)."""
        out = torch.empty((n, c), dtype=torch.float32, device=self.dev)
        self._check(self.lib.lne_sparse_sign_sketch(self.h, n, c, zeta, int(seed) & 0xFFFFFFFFFFFFFFFF, _ptr(out),
                                                    c, _stream()))
        return out

    def sparse_sign_spmm(self, csr: dict, c: int, zeta: int, seed: int) -> torch.Tensor:
        """Y = M Omega for the sparse sign Omega (never formed)."""
        m = self._csr(csr)
        Y = torch.empty((int(csr["n"]), c), dtype=torch.float32, device=self.dev)
        self._check(self.lib.lne_sparse_sign_spmm(self.h, ctypes.byref(m), c, zeta, int(seed) & 0xFFFFFFFFFFFFFFFF,
                                                  _ptr(Y), c, _stream()))
        return Y

    def very_sparse_sketch(self, n: int, c: int, s: float, seed: int) -> torch.Tensor:
        """The very sparse projection written out densely (n x c); s <= 0: sqrt(n)."""
        out = torch.empty((n, c), dtype=torch.float32, device=self.dev)
        self._check(self.lib.lne_very_sparse_sketch(self.h, n, c, float(s), int(seed) & 0xFFFFFFFFFFFFFFFF, _ptr(out),
                                                    c, _stream()))
        return out

    def very_sparse_spmm(self, csr: dict, c: int, s: float, seed: int) -> torch.Tensor:
        """Y = M Omega for the very sparse Omega (never formed)."""
        m = self._csr(csr)
        Y = torch.empty((int(csr["n"]), c), dtype=torch.float32, device=self.dev)
        self._check(self.lib.lne_very_sparse_spmm(self.h, ctypes.byref(m), c, float(s),
                                                  int(seed) & 0xFFFFFFFFFFFFFFFF, _ptr(Y), c, _stream()))
        return Y

    def _csr(self, csr: dict) -> _Csr:
        n, nnz = int(csr["n"]), int(csr["nnz"])
        _check_tensor("CSR indptr", csr["indptr"], self.dev, torch.int64, min_numel=n + 1)
        if nnz:
            _check_tensor("CSR indices", csr["indices"], self.dev, torch.int32, min_numel=nnz)
            _check_tensor("CSR data", csr["data"], self.dev, torch.float32, min_numel=nnz)
        return _Csr(n, nnz, csr["indptr"].data_ptr(), csr["indices"].data_ptr() if nnz else None,
                    csr["data"].data_ptr() if nnz else None)

    def spmm(self, csr: dict, X: torch.Tensor) -> torch.Tensor:
        """Y = M X; X float32 or bfloat16 (FP32 accumulation either way)."""
        X = X.contiguous()
        if X.dim() != 2:
            raise ValueError(f"X must be 2-D, got shape {tuple(X.shape)}")
        n, c = X.shape
        prec = PREC_BF16_MIXED if X.dtype == torch.bfloat16 else PREC_FP32
        if prec == PREC_FP32:
            X = X.float()
        m = self._csr(csr)
        # the product gathers X rows by column index (< csr n)
        _check_tensor("X", X, self.dev, min_rows=int(csr["n"]))
        Y = torch.empty((int(csr["n"]), c), dtype=torch.float32, device=self.dev)
        self._check(self.lib.lne_spmm(self.h, ctypes.byref(m), _ptr(X), c, c, _ptr(Y), c, prec, _stream()))
        return Y

    def cholqr2(self, Y: torch.Tensor):
        """Returns (Q, R): Q overwrites a copy of Y; R is FP64 upper triangular."""
        _check_tensor("Y", Y.contiguous(), self.dev, torch.float32)
        if Y.dim() != 2:
            raise ValueError(f"Y must be 2-D, got shape {tuple(Y.shape)}")
        Q = Y.contiguous().clone()
        n, c = Q.shape
        R = torch.zeros((c, c), dtype=torch.float64, device=self.dev)
        self._check(self.lib.lne_cholqr2(self.h, _ptr(Q), n, c, c, _ptr(R), _stream()))
        return Q, R

    def svd_small(self, R: torch.Tensor):
        """(U, sigma) of a small FP64 matrix R."""
        R = R.to(torch.float64).contiguous()
        if R.dim() != 2 or R.shape[0] != R.shape[1]:
            raise ValueError(f"R must be square, got shape {tuple(R.shape)}")
        _check_tensor("R", R, self.dev)
        c = R.shape[0]
        U = torch.empty((c, c), dtype=torch.float64, device=self.dev)
        sig = torch.empty(c, dtype=torch.float64, device=self.dev)
        self._check(self.lib.lne_svd_small(self.h, _ptr(R), c, _ptr(U), _ptr(sig), _stream()))
        return U, sig

    def rsvd(self, csr: dict, p: Params):
        n = int(csr["n"])
        m = self._csr(csr)
        U = torch.empty((n, p.d), dtype=torch.float32, device=self.dev)
        X0 = torch.empty((n, p.d), dtype=torch.float32, device=self.dev)
        sig = torch.empty(p.d, dtype=torch.float64, device=self.dev)
        pc, keep = p._c()
        self._check(self.lib.lne_rsvd(self.h, ctypes.byref(m), ctypes.byref(pc), _ptr(U), _ptr(sig), _ptr(X0),
                                      _stream()))
        return dict(U=U, sigma=sig, X0=X0)

    def propagate(self, g: DeviceGraph, p: Params, X0: torch.Tensor, want_intermediates: bool = False):
        X0 = X0.contiguous()
        gc = g._c(self.dev)
        _check_tensor("X0", X0, self.dev, torch.float32, shape=(g.n, p.d))
        X = torch.empty_like(X0)
        F = torch.empty_like(X0) if want_intermediates else None
        P = torch.empty_like(X0) if want_intermediates else None
        pc, keep = p._c()
        self._check(self.lib.lne_propagate(self.h, ctypes.byref(gc), ctypes.byref(pc), _ptr(X0), _ptr(X), _ptr(F),
                                           _ptr(P), _stream()))
        return dict(X=X, F=F, P=P)

    def macro_f1(self, X: torch.Tensor, labels: torch.Tensor, train_idx: torch.Tensor, test_idx: torch.Tensor,
                 C: float = 1.0, iters: int = 10):
        """(Macro-F1, Micro-F1) of one-vs-rest logistic regression on X."""
        X = X.contiguous().float()
        lab = labels.contiguous().to(torch.uint8)
        tr = train_idx.contiguous().to(torch.int32)
        te = test_idx.contiguous().to(torch.int32)
        if X.dim() != 2 or lab.dim() != 2:
            raise ValueError("X and labels must be 2-D")
        n, d = X.shape
        _check_tensor("X", X, self.dev)
        _check_tensor("labels", lab, self.dev, min_rows=n)
        _check_tensor("train_idx", tr, self.dev)
        _check_tensor("test_idx", te, self.dev)
        ma, mi = ctypes.c_double(), ctypes.c_double()
        self._check(self.lib.lne_macro_f1(self.h, _ptr(X), n, d, d, _ptr(lab), lab.shape[1], _ptr(tr), tr.numel(),
                                          _ptr(te), te.numel(), float(C), int(iters), ctypes.byref(ma),
                                          ctypes.byref(mi), _stream()))
        return float(ma.value), float(mi.value)

    def tune_batch(self, g: DeviceGraph, cands: Sequence[Params], labels: torch.Tensor, train_idx: torch.Tensor,
                   test_idx: torch.Tensor, C: float = 1.0, iters: int = 10, want_embeddings: bool = False):
        """Macro-F1 / Micro-F1 of every candidate parameter set (lne_tune_batch):
        numpy arrays of len(cands), plus the embeddings [ncand][n][d] if asked."""
        nc = len(cands)
        built = [p._c() for p in cands]
        arr = (_Params * nc)(*[b[0] for b in built])
        lab = labels.contiguous().to(torch.uint8)
        tr = train_idx.contiguous().to(torch.int32)
        te = test_idx.contiguous().to(torch.int32)
        if lab.dim() != 2:
            raise ValueError("labels must be 2-D")
        gc = g._c(self.dev)
        _check_tensor("labels", lab, self.dev, min_rows=g.n)
        _check_tensor("train_idx", tr, self.dev)
        _check_tensor("test_idx", te, self.dev)
        ma = (ctypes.c_double * nc)()
        mi = (ctypes.c_double * nc)()
        X = torch.empty((nc, g.n, cands[0].d), dtype=torch.float32, device=self.dev) if want_embeddings else None
        self._check(self.lib.lne_tune_batch(self.h, ctypes.byref(gc), ctypes.cast(arr, ctypes.c_void_p), nc,
                                            _ptr(lab), lab.shape[1], _ptr(tr), tr.numel(), _ptr(te), te.numel(),
                                            float(C), int(iters), ma, mi, _ptr(X) if X is not None else None,
                                            _stream()))
        del built
        out = (np.array(ma[:]), np.array(mi[:]))
        return out + (X,) if want_embeddings else out

    def tune_tasks(self, tasks, cands, C: float = 1.0, iters: int = 10):
        """Scores of many tuning tasks (lne_tune_tasks). tasks: list of
        (DeviceGraph, labels, train_idx, test_idx) with device tensors;
        cands: one list of Params per task, all of the same length.
        Returns (macro, micro) numpy arrays [ntasks][ncand]."""
        nt, nc = len(tasks), len(cands[0])
        assert len(cands) == nt and all(len(c) == nc for c in cands)
        keep = []
        tarr = (_Task * nt)()
        for t, (g, lab, tr, te) in enumerate(tasks):
            lab = lab.contiguous().to(torch.uint8)
            tr = tr.contiguous().to(torch.int32)
            te = te.contiguous().to(torch.int32)
            if lab.dim() != 2:
                raise ValueError(f"task {t}: labels must be 2-D")
            _check_tensor(f"task {t} labels", lab, self.dev, min_rows=g.n)
            _check_tensor(f"task {t} train_idx", tr, self.dev)
            _check_tensor(f"task {t} test_idx", te, self.dev)
            keep += [lab, tr, te]
            tarr[t] = _Task(g._c(self.dev), lab.data_ptr(), lab.shape[1], tr.data_ptr(), tr.numel(), te.data_ptr(),
                            te.numel())
        built = [p._c() for row in cands for p in row]
        parr = (_Params * (nt * nc))(*[b[0] for b in built])
        ma = (ctypes.c_double * (nt * nc))()
        mi = (ctypes.c_double * (nt * nc))()
        self._check(self.lib.lne_tune_tasks(self.h, ctypes.cast(tarr, ctypes.c_void_p), nt,
                                            ctypes.cast(parr, ctypes.c_void_p), nc, float(C), int(iters), ma, mi,
                                            _stream()))
        del built, keep
        return np.array(ma[:]).reshape(nt, nc), np.array(mi[:]).reshape(nt, nc)

    # ---- surrogate network ----------------------------------------------------
    def surrogate_init(self, seed: int = 0):
        self._check(self.lib.lne_surrogate_init(self.h, int(seed) & 0xFFFFFFFFFFFFFFFF, _stream()))

    def surrogate_fit_scaling(self, X: torch.Tensor):
        X = X.contiguous().float()
        _check_tensor("X", X, self.dev, cols=SURROGATE_INPUTS)
        self._check(self.lib.lne_surrogate_fit_scaling(self.h, _ptr(X), X.shape[0], _stream()))

    def surrogate_set_params(self, theta, mean, std):
        th = torch.as_tensor(np.asarray(theta, np.float32)).to(self.dev)
        mu = torch.as_tensor(np.asarray(mean, np.float32)).to(self.dev)
        sd = torch.as_tensor(np.asarray(std, np.float32)).to(self.dev)
        assert th.numel() == SURROGATE_PARAMS and mu.numel() == SURROGATE_INPUTS == sd.numel()
        self._check(self.lib.lne_surrogate_set_params(self.h, _ptr(th), _ptr(mu), _ptr(sd), _stream()))

    def surrogate_get_params(self):
        th = torch.empty(SURROGATE_PARAMS, dtype=torch.float32, device=self.dev)
        mu = torch.empty(SURROGATE_INPUTS, dtype=torch.float32, device=self.dev)
        sd = torch.empty(SURROGATE_INPUTS, dtype=torch.float32, device=self.dev)
        self._check(self.lib.lne_surrogate_get_params(self.h, _ptr(th), _ptr(mu), _ptr(sd), _stream()))
        return th.cpu().numpy(), mu.cpu().numpy(), sd.cpu().numpy()

    def surrogate_train(self, X: torch.Tensor, y: torch.Tensor, epochs: int, batch: int = 256, lr: float = 1e-3,
                        seed: int = 0) -> float:
        X = X.contiguous().float()
        y = y.contiguous().float()
        _check_tensor("X", X, self.dev, cols=SURROGATE_INPUTS)
        _check_tensor("y", y, self.dev, min_numel=X.shape[0])
        loss = ctypes.c_double()
        self._check(self.lib.lne_surrogate_train(self.h, _ptr(X), _ptr(y), X.shape[0], int(epochs), int(batch),
                                                 float(lr), int(seed) & 0xFFFFFFFFFFFFFFFF, ctypes.byref(loss),
                                                 _stream()))
        return float(loss.value)

    def surrogate_predict(self, X: torch.Tensor) -> torch.Tensor:
        X = X.contiguous().float()
        _check_tensor("X", X, self.dev, cols=SURROGATE_INPUTS)
        out = torch.empty(X.shape[0], dtype=torch.float32, device=self.dev)
        self._check(self.lib.lne_surrogate_predict(self.h, _ptr(X), X.shape[0], _ptr(out), _stream()))
        return out

    def surrogate_grad(self, X: torch.Tensor, y: torch.Tensor):
        X = X.contiguous().float()
        y = y.contiguous().float()
        _check_tensor("X", X, self.dev, cols=SURROGATE_INPUTS)
        _check_tensor("y", y, self.dev, min_numel=X.shape[0])
        g = torch.empty(SURROGATE_PARAMS, dtype=torch.float32, device=self.dev)
        loss = ctypes.c_double()
        self._check(self.lib.lne_surrogate_grad(self.h, _ptr(X), _ptr(y), X.shape[0], _ptr(g), ctypes.byref(loss),
                                                _stream()))
        return g, float(loss.value)

    def embed(self, g: DeviceGraph, p: Params, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        gc = g._c(self.dev)
        if out is not None:
            _check_tensor("out", out, self.dev, torch.float32, shape=(g.n, p.d))
        X = out if out is not None else torch.empty((g.n, p.d), dtype=torch.float32, device=self.dev)
        pc, keep = p._c()
        self._check(self.lib.lne_embed(self.h, ctypes.byref(gc), ctypes.byref(pc), _ptr(X), _stream()))
        return X
