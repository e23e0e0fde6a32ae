"""ctypes binding of libtwed.so with the entry-point names of include/twed.h.

Argument marshalling only: every step of the computation runs in the CUDA
library.  Device entry points take torch CUDA tensors (PyTorch is used only
for device memory and streams); host entry points take numpy arrays.  If the
library has not been built, or no GPU is present, calls raise -- there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libtwed.so")

TWED_OK = 0
TWED_ERR_INVALID_ARG = 1
TWED_ERR_CUDA = 2
TWED_ERR_ALLOC = 3
TWED_ERR_TIMEOUT = 4
TWED_ERR_UNSUPPORTED = 5
_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "CUDA", 3: "ALLOC", 4: "TIMEOUT", 5: "UNSUPPORTED"}

ACCUM_AUTO, ACCUM_F32, ACCUM_KAHAN = 0, 1, 2

# Every symbol include/twed.h declares (checked by the CPU test suite).
EXPORTS = (
    "twed_create", "twed_destroy", "twed_last_error", "twed_version", "twed_sync_status",
    "twed_f64", "twed_f32", "twed_f32_ex",
    "twed_dev_f64", "twed_dev_f32", "twed_dev_f64_ex", "twed_dev_f32_ex",
    "twed_batch_f64", "twed_batch_f32", "twed_batch_f64_ex", "twed_batch_f32_ex",
    "twed_batch_f32_noalloc",
    "twed_allpairs_plan_create_f64", "twed_allpairs_plan_create_f32", "twed_plan_execute",
    "twed_plan_cells", "twed_plan_pairs", "twed_plan_kernel_ms", "twed_plan_describe", "twed_plan_status",
    "twed_plan_destroy",
    "twed_allpairs_host_f32",
    "twed_knn_config_default", "twed_knn_create", "twed_knn_train", "twed_knn_search",
    "twed_knn_exact", "twed_knn_search_host", "twed_knn_search_profile", "twed_knn_get_stats", "twed_knn_get_params", "twed_knn_set_params",
    "twed_knn_get_embeddings", "twed_knn_destroy",
    "twed_encoder_param_count", "twed_encoder_stats_f32", "twed_encoder_forward_f32",
    "twed_encoder_loss_grad_f32", "twed_adam_f32", "twed_embed_search_f32", "twed_topk_rows_f32",
    "twed_pipe_peak",
    "twed_path_f64", "twed_path_f32", "twed_path_batch_f64", "twed_path_batch_f32",
    "twed_lcs_batch", "twed_lcs_pairs", "twed_dtw_batch_f64", "twed_dtw_batch_f32",
    "twed_dtw_f64", "twed_dtw_f32",
)


class TwedError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"TWED_ERR_{_NAMES.get(status, status)}: {msg}")
        self.status = status


XTERM_OFF, XTERM_TF32, XTERM_BF16 = 0, 1, 2


class Opts(ctypes.Structure):
    _fields_ = [("accum", ctypes.c_int), ("rows_per_lane", ctypes.c_int),
                ("autotune", ctypes.c_int), ("timeout_s", ctypes.c_double),
                ("stall_strip", ctypes.c_int64), ("xterm", ctypes.c_int)]


def make_opts(accum=0, rows_per_lane=0, autotune=0, timeout_s=0.0, stall_strip=-1,
              xterm=0) -> Opts:
    return Opts(accum, rows_per_lane, autotune, timeout_s, stall_strip, xterm)


class _SetF64(ctypes.Structure):
    _fields_ = [("vals", ctypes.c_void_p), ("ts", ctypes.c_void_p), ("offs", ctypes.c_void_p),
                ("offs_host", ctypes.c_void_p), ("n", ctypes.c_int64)]


_SetF32 = _SetF64  # identical layout: four pointers and a count

_lib = None
_lock = threading.Lock()


def load(path: str | None = None):
    """Load libtwed.so (raises if it is missing: build it first)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"libtwed.so not built ({p}); run paper_2007_16135_gb300/build.py")
        lib = ctypes.CDLL(p)
        P, i64, ci = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        d, f = ctypes.c_double, ctypes.c_float
        sig = {
            "twed_create": (ci, [P]),
            "twed_destroy": (None, [P]),
            "twed_last_error": (ctypes.c_char_p, [P]),
            "twed_version": (ctypes.c_char_p, []),
            "twed_sync_status": (ci, [P, P]),
            "twed_f64": (ci, [P, P, P, i64, P, P, i64, ci, d, d, ci, P]),
            "twed_f32": (ci, [P, P, P, i64, P, P, i64, ci, f, f, ci, P]),
            "twed_f32_ex": (ci, [P, P, P, i64, P, P, i64, ci, f, f, ci, P, P]),
            "twed_dev_f64": (ci, [P, P, P, i64, P, P, i64, ci, d, d, ci, P, P]),
            "twed_dev_f32": (ci, [P, P, P, i64, P, P, i64, ci, f, f, ci, P, P]),
            "twed_dev_f64_ex": (ci, [P, P, P, i64, P, P, i64, ci, d, d, ci, P, P, P]),
            "twed_dev_f32_ex": (ci, [P, P, P, i64, P, P, i64, ci, f, f, ci, P, P, P]),
            "twed_batch_f64": (ci, [P, P, P, P, i64, ci, d, d, ci, P, P]),
            "twed_batch_f32": (ci, [P, P, P, P, i64, ci, f, f, ci, P, P]),
            "twed_batch_f64_ex": (ci, [P, P, P, P, i64, ci, d, d, ci, ci, P, P]),
            "twed_batch_f32_ex": (ci, [P, P, P, P, i64, ci, f, f, ci, ci, P, P]),
            "twed_batch_f32_noalloc": (ci, [P, P, P, i64, ci, f, f, ci, P, P]),
            "twed_allpairs_plan_create_f64": (ci, [P, P, P, ci, d, d, ci, P, P]),
            "twed_allpairs_plan_create_f32": (ci, [P, P, P, ci, f, f, ci, P, P]),
            "twed_plan_execute": (ci, [P, P, P]),
            "twed_plan_cells": (i64, [P]),
            "twed_plan_pairs": (i64, [P]),
            "twed_plan_kernel_ms": (ci, [P, P]),
            "twed_plan_status": (ci, [P, P]),
            "twed_plan_describe": (ctypes.c_char_p, [P]),
            "twed_plan_destroy": (None, [P]),
            "twed_allpairs_host_f32": (ci, [P, P, P, P, i64, P, P, P, i64, ci, f, f, ci, P]),
            "twed_knn_config_default": (None, [P]),
            "twed_knn_create": (ci, [P, P, ci, f, f, ci, P, P]),
            "twed_knn_train": (ci, [P]),
            "twed_knn_search": (ci, [P, P, ci, ci, P, P, P]),
            "twed_knn_exact": (ci, [P, P, ci, P, P, P]),
            "twed_knn_search_host": (ci, [P, P, P, P, i64, ci, ci, P, P]),
            "twed_knn_search_profile": (ci, [P, P, P]),
            "twed_knn_get_stats": (ci, [P, P]),
            "twed_knn_get_params": (ci, [P, P, i64]),
            "twed_knn_set_params": (ci, [P, P, i64]),
            "twed_knn_get_embeddings": (ci, [P, P, P]),
            "twed_knn_destroy": (None, [P]),
            "twed_encoder_param_count": (i64, [ci]),
            "twed_encoder_stats_f32": (ci, [P, P, ci, f, f, ci, P, P]),
            "twed_encoder_forward_f32": (ci, [P, P, ci, f, f, ci, P, P, P, f, P]),
            "twed_encoder_loss_grad_f32": (ci, [P, P, ci, f, f, ci, P, P, P, f, P, i64, ci, P, f,
                                                P, P]),
            "twed_adam_f32": (ci, [P, P, P, P, P, i64, i64, f, f, f, f]),
            "twed_embed_search_f32": (ci, [P, P, i64, P, i64, ci, P, P]),
            "twed_topk_rows_f32": (ci, [P, P, i64, i64, i64, ci, P, P, P]),
            "twed_pipe_peak": (ci, [P, ci, P]),
            "twed_path_f64": (ci, [P, P, P, i64, P, P, i64, ci, d, d, ci, P, P, P]),
            "twed_path_f32": (ci, [P, P, P, i64, P, P, i64, ci, f, f, ci, P, P, P]),
            "twed_path_batch_f64": (ci, [P, P, P, P, i64, ci, d, d, ci, P, P, P, P, P]),
            "twed_path_batch_f32": (ci, [P, P, P, P, i64, ci, f, f, ci, P, P, P, P, P]),
            "twed_lcs_batch": (ci, [P, P, P, P, i64, P, P]),
            "twed_lcs_pairs": (ci, [P, P, i64, P, i64, P, P, P]),
            "twed_dtw_batch_f64": (ci, [P, P, P, P, i64, ci, ci, P, P]),
            "twed_dtw_batch_f32": (ci, [P, P, P, P, i64, ci, ci, P, P]),
            "twed_dtw_f64": (ci, [P, P, i64, P, i64, ci, ci, P]),
            "twed_dtw_f32": (ci, [P, P, i64, P, i64, ci, ci, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def version() -> str:
    return load().twed_version().decode()


def _np_ptr(x: np.ndarray):
    return ctypes.c_void_p(x.ctypes.data)


def _t_ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _stream_ptr(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


class Handle:
    """twed_create / twed_destroy.  One handle per host thread."""

    def __init__(self):
        self.lib = load()
        h = ctypes.c_void_p()
        st = self.lib.twed_create(ctypes.byref(h))
        if st != TWED_OK:
            raise TwedError(st, "twed_create failed (no usable CUDA device?)")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.twed_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, st: int):
        if st != TWED_OK:
            raise TwedError(st, self.lib.twed_last_error(self.h).decode(errors="replace"))

    def sync_status(self, stream=None):
        self.check(self.lib.twed_sync_status(self.h, _stream_ptr(stream)))


_default = threading.local()


def default_handle() -> Handle:
    h = getattr(_default, "h", None)
    if h is None:
        h = Handle()
        _default.h = h
    return h


def _series_np(a, ta, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    if a.ndim == 1:
        a = a[:, None]
    ta = np.ascontiguousarray(ta, dtype=dtype)
    return a, ta


# ------------------------------------------------------------------ one pair
def twed_f64(a, ta, b, tb, nu, lam, p=2, handle: Handle | None = None) -> float:
    """Host arrays in, TWED out (blocking).  a: [n, dim] or [n]."""
    h = handle or default_handle()
    a, ta = _series_np(a, ta, np.float64)
    b, tb = _series_np(b, tb, np.float64)
    out = ctypes.c_double()
    h.check(h.lib.twed_f64(h.h, _np_ptr(a), _np_ptr(ta), a.shape[0], _np_ptr(b), _np_ptr(tb),
                           b.shape[0], a.shape[1], nu, lam, p, ctypes.byref(out)))
    return out.value


def twed_f32(a, ta, b, tb, nu, lam, p=2, handle: Handle | None = None, opts: Opts | None = None) -> float:
    h = handle or default_handle()
    a, ta = _series_np(a, ta, np.float32)
    b, tb = _series_np(b, tb, np.float32)
    out = ctypes.c_float()
    if opts is None:
        st = h.lib.twed_f32(h.h, _np_ptr(a), _np_ptr(ta), a.shape[0], _np_ptr(b), _np_ptr(tb),
                            b.shape[0], a.shape[1], nu, lam, p, ctypes.byref(out))
    else:
        st = h.lib.twed_f32_ex(h.h, _np_ptr(a), _np_ptr(ta), a.shape[0], _np_ptr(b), _np_ptr(tb),
                               b.shape[0], a.shape[1], nu, lam, p, ctypes.byref(opts),
                               ctypes.byref(out))
    h.check(st)
    return out.value


def twed_dev(a, ta, b, tb, nu, lam, p=2, out=None, stream=None, handle: Handle | None = None,
             opts: Opts | None = None):
    """Device tensors in (float32 or float64, a: [n, dim]), out: 1-element
    device tensor.  Enqueued on `stream` (default: torch's current stream)."""
    import torch
    h = handle or default_handle()
    if a.dim() == 1:
        a = a[:, None]
    if b.dim() == 1:
        b = b[:, None]
    a, b, ta, tb = (x.contiguous() for x in (a, b, ta, tb))
    f64 = a.dtype == torch.float64
    if out is None:
        out = torch.empty(1, dtype=a.dtype, device=a.device)
    sp = _stream_ptr(stream)
    op = ctypes.byref(opts) if opts is not None else None
    if f64:
        st = h.lib.twed_dev_f64_ex(h.h, _t_ptr(a), _t_ptr(ta), a.shape[0], _t_ptr(b), _t_ptr(tb),
                                   b.shape[0], a.shape[1], float(nu), float(lam), p, op,
                                   _t_ptr(out), sp)
    else:
        st = h.lib.twed_dev_f32_ex(h.h, _t_ptr(a), _t_ptr(ta), a.shape[0], _t_ptr(b), _t_ptr(tb),
                                   b.shape[0], a.shape[1], float(nu), float(lam), p, op,
                                   _t_ptr(out), sp)
    h.check(st)
    return out


twed_dev_f64 = twed_dev
twed_dev_f32 = twed_dev


# ------------------------------------------------------------------ sets
@dataclass
class DeviceSet:
    """A packed set on the device plus the host copy of its offsets."""
    vals: "object"  # torch [sum_len, dim]
    ts: "object"  # torch [sum_len]
    offs: "object"  # torch int64 [n + 1] (device)
    offs_host: np.ndarray  # int64 [n + 1]

    @classmethod
    def from_numpy(cls, vals, ts, offs, dtype, device="cuda"):
        import torch
        v = np.ascontiguousarray(vals)
        if v.ndim == 1:
            v = v[:, None]
        return cls(torch.as_tensor(v, device=device).to(dtype).contiguous(),
                   torch.as_tensor(np.ascontiguousarray(ts), device=device).to(dtype).contiguous(),
                   torch.as_tensor(np.ascontiguousarray(offs, dtype=np.int64), device=device),
                   np.ascontiguousarray(offs, dtype=np.int64))

    @property
    def n(self) -> int:
        return int(self.offs_host.shape[0] - 1)

    @property
    def dim(self) -> int:
        return int(self.vals.shape[1])

    def cstruct(self):
        return _SetF64(self.vals.data_ptr(), self.ts.data_ptr(), self.offs.data_ptr(),
                       self.offs_host.ctypes.data, self.n)


# run orders of twed_batch (twed.h TWED_ORDER_*)
ORDER_LIST, ORDER_LONGEST_FIRST = 0, 1


def twed_batch(A: DeviceSet, B: DeviceSet, pairs, nu, lam, p=2, out=None, stream=None,
               handle: Handle | None = None, order: int = ORDER_LIST):
    """TWED of listed pairs (device int64 [k, 2]) -> device tensor [k].
    `order` picks the run order (ORDER_*); out[k] is pair k's value in any."""
    import torch
    h = handle or default_handle()
    pairs = pairs.contiguous()
    k = pairs.shape[0]
    if out is None:
        out = torch.empty(k, dtype=A.vals.dtype, device=A.vals.device)
    sa, sb = A.cstruct(), B.cstruct()
    args = (h.h, ctypes.byref(sa), ctypes.byref(sb), _t_ptr(pairs), k, A.dim, float(nu),
            float(lam), p)
    f64 = A.vals.dtype == torch.float64
    if order == ORDER_LIST:
        fn = h.lib.twed_batch_f64 if f64 else h.lib.twed_batch_f32
        h.check(fn(*args, _t_ptr(out), _stream_ptr(stream)))
    else:
        fn = h.lib.twed_batch_f64_ex if f64 else h.lib.twed_batch_f32_ex
        h.check(fn(*args, int(order), _t_ptr(out), _stream_ptr(stream)))
    return out


twed_batch_f64 = twed_batch
twed_batch_f32 = twed_batch


# ---------------------------------------------------------------- edit paths
MOVE_CHARS = "MAB"  # 0 match, 1 delete in a, 2 delete in b


def twed_path(a, ta, b, tb, nu, lam, p=2, dtype="f64", handle: Handle | None = None):
    """TWED of one pair and an optimal edit path, ``(value, moves)`` with
    ``moves`` a string over 'M' (match), 'A' (delete in a), 'B' (delete in b),
    the steps after the forced first match (twed_path_f64 / _f32)."""
    h = handle or default_handle()
    npd = np.float64 if dtype == "f64" else np.float32
    a, ta = _series_np(a, ta, npd)
    b, tb = _series_np(b, tb, npd)
    if a.shape[1] != b.shape[1]:
        raise ValueError("series dimensions differ")
    moves = np.zeros(max(a.shape[0] + b.shape[0] - 2, 1), dtype=np.int8)
    out = np.zeros(1, dtype=npd)
    n = np.zeros(1, dtype=np.int64)
    fn = h.lib.twed_path_f64 if dtype == "f64" else h.lib.twed_path_f32
    h.check(fn(h.h, _np_ptr(a), _np_ptr(ta), a.shape[0], _np_ptr(b), _np_ptr(tb), b.shape[0], a.shape[1],
               float(nu), float(lam), int(p), _np_ptr(out), _np_ptr(moves), _np_ptr(n)))
    return float(out[0]), "".join(MOVE_CHARS[x] for x in moves[:int(n[0])])


def path_batch_buffers(A: DeviceSet, B: DeviceSet, pairs):
    """Output buffers for :func:`twed_path_batch`: ``(dist, moves, move_offs,
    lens)``, with room for n + m - 2 moves per pair."""
    import torch
    k = pairs.shape[0]
    la = torch.as_tensor(np.diff(A.offs_host), device=pairs.device)
    lb = torch.as_tensor(np.diff(B.offs_host), device=pairs.device)
    cap = (la[pairs[:, 0]] + lb[pairs[:, 1]] - 2).clamp(min=1)
    offs = torch.zeros(k, dtype=torch.int64, device=pairs.device)
    if k > 1:
        offs[1:] = torch.cumsum(cap, 0)[:-1]
    moves = torch.zeros(int(cap.sum().item()) if k else 1, dtype=torch.int8, device=pairs.device)
    dist = torch.empty(k, dtype=A.vals.dtype, device=pairs.device)
    lens = torch.empty(k, dtype=torch.int64, device=pairs.device)
    return dist, moves, offs, lens


def twed_path_batch(A: DeviceSet, B: DeviceSet, pairs, nu, lam, p=2, stream=None,
                    handle: Handle | None = None, out=None):
    """Distances and edit paths of listed pairs (device int64 [k, 2]):
    ``(dist [k], moves int8, move_offs [k], lens [k])`` on the device; pair
    k's moves are ``moves[move_offs[k] : move_offs[k] + lens[k]]``.  ``out``
    reuses buffers from :func:`path_batch_buffers` (no allocation, no
    synchronization)."""
    import torch
    h = handle or default_handle()
    pairs = pairs.contiguous()
    k = pairs.shape[0]
    dist, moves, offs, lens = out if out is not None else path_batch_buffers(A, B, pairs)
    sa, sb = A.cstruct(), B.cstruct()
    f64 = A.vals.dtype == torch.float64
    fn = h.lib.twed_path_batch_f64 if f64 else h.lib.twed_path_batch_f32
    h.check(fn(h.h, ctypes.byref(sa), ctypes.byref(sb), _t_ptr(pairs), k, A.dim, float(nu), float(lam), p,
               _t_ptr(dist), _t_ptr(moves), _t_ptr(offs), _t_ptr(lens), _stream_ptr(stream)))
    return dist, moves, offs, lens


# ---------------------------------------------------------------- LCS and DTW
class _Seq(ctypes.Structure):
    _fields_ = [("sym", ctypes.c_void_p), ("offs", ctypes.c_void_p), ("offs_host", ctypes.c_void_p),
                ("n", ctypes.c_int64)]


@dataclass
class DeviceSeqs:
    """Packed int32 symbol sequences on the device (may be empty)."""
    sym: "object"  # torch int32 [sum_len]
    offs: "object"  # torch int64 [n + 1]
    offs_host: np.ndarray

    @classmethod
    def from_lists(cls, seqs, device="cuda"):
        import torch
        lens = [len(x) for x in seqs]
        offs = np.zeros(len(seqs) + 1, dtype=np.int64)
        offs[1:] = np.cumsum(lens)
        flat = np.concatenate([np.asarray(x, dtype=np.int32).ravel() for x in seqs]) if offs[-1] else \
            np.zeros(1, dtype=np.int32)
        return cls(torch.as_tensor(flat, device=device), torch.as_tensor(offs, device=device), offs)

    @property
    def n(self) -> int:
        return int(self.offs_host.shape[0] - 1)

    def cstruct(self):
        return _Seq(self.sym.data_ptr(), self.offs.data_ptr(), self.offs_host.ctypes.data, self.n)


def lcs_batch(X: DeviceSeqs, Y: DeviceSeqs, pairs, stream=None, handle: Handle | None = None):
    """LCS lengths of listed pairs (device int64 [k, 2]) -> device int32 [k]."""
    import torch
    h = handle or default_handle()
    pairs = pairs.contiguous()
    out = torch.empty(pairs.shape[0], dtype=torch.int32, device=pairs.device)
    sx, sy = X.cstruct(), Y.cstruct()
    h.check(h.lib.twed_lcs_batch(h.h, ctypes.byref(sx), ctypes.byref(sy), _t_ptr(pairs), pairs.shape[0],
                                 _t_ptr(out), _stream_ptr(stream)))
    return out


def lcs_pairs(x, y, handle: Handle | None = None):
    """One longest common subsequence as matched positions ``(xi, yj)``."""
    h = handle or default_handle()
    x = np.ascontiguousarray(np.asarray(x, dtype=np.int32).ravel())
    y = np.ascontiguousarray(np.asarray(y, dtype=np.int32).ravel())
    k = max(min(x.size, y.size), 1)
    xi = np.zeros(k, dtype=np.int64)
    yj = np.zeros(k, dtype=np.int64)
    n = np.zeros(1, dtype=np.int64)
    h.check(h.lib.twed_lcs_pairs(h.h, _np_ptr(x) if x.size else None, x.size, _np_ptr(y) if y.size else None,
                                 y.size, _np_ptr(xi), _np_ptr(yj), _np_ptr(n)))
    return xi[:int(n[0])].copy(), yj[:int(n[0])].copy()


def dtw_batch(A: DeviceSet, B: DeviceSet, pairs, p=2, stream=None, handle: Handle | None = None):
    """DTW of listed pairs (device int64 [k, 2]) -> device tensor [k]."""
    import torch
    h = handle or default_handle()
    pairs = pairs.contiguous()
    out = torch.empty(pairs.shape[0], dtype=A.vals.dtype, device=pairs.device)
    sa, sb = A.cstruct(), B.cstruct()
    fn = h.lib.twed_dtw_batch_f64 if A.vals.dtype == torch.float64 else h.lib.twed_dtw_batch_f32
    h.check(fn(h.h, ctypes.byref(sa), ctypes.byref(sb), _t_ptr(pairs), pairs.shape[0], A.dim, int(p),
               _t_ptr(out), _stream_ptr(stream)))
    return out


def dtw(a, b, p=2, dtype="f64", handle: Handle | None = None) -> float:
    """DTW of one pair of ``[len, dim]`` host arrays (twed_dtw_f64 / _f32)."""
    h = handle or default_handle()
    npd = np.float64 if dtype == "f64" else np.float32
    a = np.ascontiguousarray(np.asarray(a, dtype=npd))
    b = np.ascontiguousarray(np.asarray(b, dtype=npd))
    a = a[:, None] if a.ndim == 1 else a
    b = b[:, None] if b.ndim == 1 else b
    out = np.zeros(1, dtype=npd)
    fn = h.lib.twed_dtw_f64 if dtype == "f64" else h.lib.twed_dtw_f32
    h.check(fn(h.h, _np_ptr(a), a.shape[0], _np_ptr(b), b.shape[0], a.shape[1], int(p), _np_ptr(out)))
    return float(out[0])


def twed_batch_f32_noalloc(A: DeviceSet, B: DeviceSet, pairs, nu, lam, p=2, out=None,
                           stream=None):
    """As twed_batch for float32 sets, for callers that cannot allocate: the
    library works in its one static device array (no handle, no cudaMalloc).
    `out` (float32 device [k]) is allocated here only if not given."""
    import torch
    lib = load()
    pairs = pairs.contiguous()
    k = pairs.shape[0]
    if out is None:
        out = torch.empty(k, dtype=torch.float32, device=A.vals.device)
    sa, sb = A.cstruct(), B.cstruct()
    st = lib.twed_batch_f32_noalloc(ctypes.byref(sa), ctypes.byref(sb), _t_ptr(pairs), k, A.dim,
                                    float(nu), float(lam), p, _t_ptr(out), _stream_ptr(stream))
    if st != TWED_OK:
        raise TwedError(st, "twed_batch_f32_noalloc failed")
    return out


class Plan:
    """twed_allpairs_plan_create_* / twed_plan_execute / twed_plan_destroy."""

    def __init__(self, A: DeviceSet, B: DeviceSet | None, nu, lam, p=2,
                 opts: Opts | None = None, handle: Handle | None = None):
        import torch
        self.handle = handle or default_handle()
        self.A, self.B = A, B  # keep the device buffers alive
        self.f64 = A.vals.dtype == torch.float64
        self._sa = A.cstruct()
        self._sb = B.cstruct() if B is not None else None
        plan = ctypes.c_void_p()
        lib = self.handle.lib
        fn = lib.twed_allpairs_plan_create_f64 if self.f64 else lib.twed_allpairs_plan_create_f32
        self.handle.check(fn(self.handle.h, ctypes.byref(self._sa),
                             ctypes.byref(self._sb) if self._sb is not None else None, A.dim,
                             float(nu), float(lam), p,
                             ctypes.byref(opts) if opts is not None else None,
                             ctypes.byref(plan)))
        self.plan = plan
        self.na = A.n
        self.nb = A.n if B is None else B.n

    @property
    def cells(self) -> int:
        return int(self.handle.lib.twed_plan_cells(self.plan))

    @property
    def pairs(self) -> int:
        return int(self.handle.lib.twed_plan_pairs(self.plan))

    def kernel_ms(self) -> float:
        """Device time of the pairs launch in the last completed execute."""
        ms = ctypes.c_float()
        self.handle.check(self.handle.lib.twed_plan_kernel_ms(self.plan, ctypes.byref(ms)))
        return ms.value

    def describe(self) -> str:
        return self.handle.lib.twed_plan_describe(self.plan).decode()

    def status(self, stream=None):
        """Wait for `stream`; raise TwedError if a kernel of this plan failed
        (a bounded wait expired) since the last call."""
        self.handle.check(self.handle.lib.twed_plan_status(self.plan, _stream_ptr(stream)))

    def new_output(self):
        import torch
        return torch.empty((self.na, self.nb), dtype=self.A.vals.dtype, device=self.A.vals.device)

    def execute(self, out=None, stream=None):
        if out is None:
            out = self.new_output()
        self.handle.check(self.handle.lib.twed_plan_execute(self.plan, _t_ptr(out),
                                                            _stream_ptr(stream)))
        return out

    def close(self):
        if getattr(self, "plan", None):
            self.handle.lib.twed_plan_destroy(self.plan)
            self.plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


twed_allpairs_plan_create_f64 = Plan
twed_allpairs_plan_create_f32 = Plan


def twed_allpairs_host_f32(a_vals, a_ts, a_offs, b=None, nu=1.0, lam=1.0, p=2,
                           handle: Handle | None = None, out: np.ndarray | None = None):
    """All-pairs matrix from host arrays (blocking).  b = (vals, ts, offs) or
    None for the symmetric self-matrix.  Returns a float32 [na, nb] array."""
    h = handle or default_handle()
    av = np.ascontiguousarray(a_vals, dtype=np.float32)
    if av.ndim == 1:
        av = av[:, None]
    at = np.ascontiguousarray(a_ts, dtype=np.float32)
    ao = np.ascontiguousarray(a_offs, dtype=np.int64)
    na = ao.shape[0] - 1
    if b is None:
        bv = bt = bo = None
        nb = na
    else:
        bv = np.ascontiguousarray(b[0], dtype=np.float32)
        if bv.ndim == 1:
            bv = bv[:, None]
        bt = np.ascontiguousarray(b[1], dtype=np.float32)
        bo = np.ascontiguousarray(b[2], dtype=np.int64)
        nb = bo.shape[0] - 1
    if out is None:
        out = np.empty((na, nb), dtype=np.float32)
    ptr = lambda x: None if x is None else _np_ptr(x)
    h.check(h.lib.twed_allpairs_host_f32(h.h, _np_ptr(av), _np_ptr(at), _np_ptr(ao), na, ptr(bv),
                                         ptr(bt), ptr(bo), nb if b is not None else 0,
                                         av.shape[1], float(nu), float(lam), p, _np_ptr(out)))
    return out


# ------------------------------------------------------- learned k-NN filter
class KnnConfig(ctypes.Structure):
    _fields_ = [("group_size", ctypes.c_int), ("groups_per_step", ctypes.c_int),
                ("epochs", ctypes.c_int), ("train_pairs", ctypes.c_int64), ("lr", ctypes.c_float),
                ("seed", ctypes.c_uint64), ("mine_fraction", ctypes.c_float),
                ("rel_floor", ctypes.c_float)]


class KnnStats(ctypes.Structure):
    _fields_ = [("sigma", ctypes.c_double), ("mean_len", ctypes.c_double),
                ("first_loss", ctypes.c_double), ("last_loss", ctypes.c_double),
                ("label_pairs", ctypes.c_int64), ("mined_pairs", ctypes.c_int64),
                ("label_cells", ctypes.c_int64),
                ("steps", ctypes.c_int64), ("label_ms", ctypes.c_double),
                ("train_ms", ctypes.c_double), ("embed_ms", ctypes.c_double),
                ("rerank_rows_per_lane", ctypes.c_int32), ("rerank_blocks_per_sm", ctypes.c_int32),
                ("tune_ms", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


def knn_config(**kw) -> KnnConfig:
    c = KnnConfig()
    load().twed_knn_config_default(ctypes.byref(c))
    for k, v in kw.items():
        setattr(c, k, v)
    return c


def encoder_param_count(dim: int) -> int:
    return int(load().twed_encoder_param_count(dim))


class KnnIndex:
    """twed_knn_create / train / search / exact / destroy over a float32
    DeviceSet database (kept alive by the index)."""

    def __init__(self, db: DeviceSet, nu, lam, p=2, config: KnnConfig | None = None,
                 handle: Handle | None = None):
        self.handle = handle or default_handle()
        self.db = db
        self._sdb = db.cstruct()
        k = ctypes.c_void_p()
        self.handle.check(self.handle.lib.twed_knn_create(
            self.handle.h, ctypes.byref(self._sdb), db.dim, float(nu), float(lam), p,
            ctypes.byref(config) if config is not None else None, ctypes.byref(k)))
        self.k = k
        self.dim = db.dim

    def train(self):
        self.handle.check(self.handle.lib.twed_knn_train(self.k))
        return self.stats()

    def stats(self) -> dict:
        st = KnnStats()
        self.handle.check(self.handle.lib.twed_knn_get_stats(self.k, ctypes.byref(st)))
        return st.as_dict()

    def params(self) -> np.ndarray:
        n = encoder_param_count(self.dim)
        out = np.empty(n, dtype=np.float32)
        self.handle.check(self.handle.lib.twed_knn_get_params(self.k, _np_ptr(out), n))
        return out

    def set_params(self, w):
        w = np.ascontiguousarray(w, dtype=np.float32)
        self.handle.check(self.handle.lib.twed_knn_set_params(self.k, _np_ptr(w), w.size))

    def embeddings(self, stream=None):
        import torch
        out = torch.empty((self.db.n, 32), dtype=torch.float32, device=self.db.vals.device)
        self.handle.check(self.handle.lib.twed_knn_get_embeddings(self.k, _t_ptr(out),
                                                                  _stream_ptr(stream)))
        return out

    def _outputs(self, nq, k):
        import torch
        dev = self.db.vals.device
        return (torch.empty((nq, k), dtype=torch.int64, device=dev),
                torch.empty((nq, k), dtype=torch.float32, device=dev))

    def search(self, queries: DeviceSet, k=10, n_candidates=200, stream=None, out=None):
        idx, dist = out if out is not None else self._outputs(queries.n, k)
        sq = queries.cstruct()
        self.handle.check(self.handle.lib.twed_knn_search(self.k, ctypes.byref(sq), k,
                                                          n_candidates, _t_ptr(idx),
                                                          _t_ptr(dist), _stream_ptr(stream)))
        return idx, dist

    def search_host(self, vals, ts, offs, k=10, n_candidates=200, out=None):
        """Host arrays in, host arrays out (blocking)."""
        v = np.ascontiguousarray(vals, dtype=np.float32)
        t = np.ascontiguousarray(ts, dtype=np.float32)
        o = np.ascontiguousarray(offs, dtype=np.int64)
        nq = o.shape[0] - 1
        if out is None:
            out = (np.empty((nq, k), dtype=np.int64), np.empty((nq, k), dtype=np.float32))
        self.handle.check(self.handle.lib.twed_knn_search_host(
            self.k, _np_ptr(v), _np_ptr(t), _np_ptr(o), nq, k, n_candidates, _np_ptr(out[0]),
            _np_ptr(out[1])))
        return out

    def search_profile(self):
        """(phase_ms [embed, candidates, re-rank, select], re-rank cells) of
        the last search."""
        ms = (ctypes.c_double * 4)()
        cells = ctypes.c_int64()
        self.handle.check(self.handle.lib.twed_knn_search_profile(self.k, ms, ctypes.byref(cells)))
        return list(ms), cells.value

    def exact(self, queries: DeviceSet, k=10, stream=None, out=None):
        idx, dist = out if out is not None else self._outputs(queries.n, k)
        sq = queries.cstruct()
        self.handle.check(self.handle.lib.twed_knn_exact(self.k, ctypes.byref(sq), k, _t_ptr(idx),
                                                         _t_ptr(dist), _stream_ptr(stream)))
        return idx, dist

    def close(self):
        if getattr(self, "k", None):
            self.handle.lib.twed_knn_destroy(self.k)
            self.k = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


twed_knn_create = KnnIndex


def encoder_stats(S: DeviceSet, nu, lam, p=2, handle: Handle | None = None):
    import torch
    h = handle or default_handle()
    mu = torch.empty(S.dim + 2, dtype=torch.float32, device=S.vals.device)
    sd = torch.empty_like(mu)
    s = S.cstruct()
    h.check(h.lib.twed_encoder_stats_f32(h.h, ctypes.byref(s), S.dim, float(nu), float(lam), p,
                                         _t_ptr(mu), _t_ptr(sd)))
    return mu, sd


def encoder_forward(S: DeviceSet, nu, lam, p, params, mu, sd, mean_len,
                    handle: Handle | None = None):
    import torch
    h = handle or default_handle()
    out = torch.empty((S.n, 32), dtype=torch.float32, device=S.vals.device)
    s = S.cstruct()
    h.check(h.lib.twed_encoder_forward_f32(h.h, ctypes.byref(s), S.dim, float(nu), float(lam), p,
                                           _t_ptr(params), _t_ptr(mu), _t_ptr(sd),
                                           float(mean_len), _t_ptr(out)))
    return out


def encoder_loss_grad(S: DeviceSet, nu, lam, p, params, mu, sd, mean_len, groups, labels,
                      inv_sigma, handle: Handle | None = None):
    """groups: host int array [ngroups, group_size]; labels: device float32
    [ngroups, npg].  Returns (loss, grad) on the device."""
    import torch
    h = handle or default_handle()
    groups = np.ascontiguousarray(groups, dtype=np.int64)
    ng, gs = groups.shape
    grad = torch.empty(encoder_param_count(S.dim), dtype=torch.float32, device=S.vals.device)
    loss = torch.empty(1, dtype=torch.float32, device=S.vals.device)
    s = S.cstruct()
    labels = labels.contiguous()
    h.check(h.lib.twed_encoder_loss_grad_f32(h.h, ctypes.byref(s), S.dim, float(nu), float(lam), p,
                                             _t_ptr(params), _t_ptr(mu), _t_ptr(sd),
                                             float(mean_len), _np_ptr(groups), ng, gs,
                                             _t_ptr(labels), float(inv_sigma), _t_ptr(grad),
                                             _t_ptr(loss)))
    return loss, grad


def adam_step(theta, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8,
              handle: Handle | None = None):
    h = handle or default_handle()
    h.check(h.lib.twed_adam_f32(h.h, _t_ptr(theta), _t_ptr(grad), _t_ptr(m), _t_ptr(v),
                                theta.numel(), int(step), float(lr), float(beta1), float(beta2),
                                float(eps)))


def embed_search(db_emb, q_emb, k, handle: Handle | None = None):
    import torch
    h = handle or default_handle()
    db_emb = db_emb.contiguous()
    q_emb = q_emb.contiguous()
    nq = q_emb.shape[0]
    idx = torch.empty((nq, k), dtype=torch.int64, device=db_emb.device)
    val = torch.empty((nq, k), dtype=torch.float32, device=db_emb.device)
    h.check(h.lib.twed_embed_search_f32(h.h, _t_ptr(db_emb), db_emb.shape[0], _t_ptr(q_emb), nq, k,
                                        _t_ptr(idx), _t_ptr(val)))
    return idx, val


def topk_rows(D, k, cols=None, stream=None, handle: Handle | None = None):
    """k smallest per row of a float32 device matrix (ties by smaller column)."""
    import torch
    h = handle or default_handle()
    rows, ld = D.shape
    cols = ld if cols is None else cols
    idx = torch.empty((rows, k), dtype=torch.int64, device=D.device)
    val = torch.empty((rows, k), dtype=torch.float32, device=D.device)
    h.check(h.lib.twed_topk_rows_f32(h.h, _t_ptr(D), rows, cols, ld, k, _t_ptr(idx), _t_ptr(val),
                                     _stream_ptr(stream)))
    return idx, val


PEAK_FFMA32, PEAK_DFMA64, PEAK_IALU32 = 0, 1, 2


def pipe_peak(kind=PEAK_FFMA32, handle: Handle | None = None) -> float:
    """Measured lane operations per second: FP32 or FP64 FMA, or 32-bit
    integer xor/max (the integer ALU pipe)."""
    h = handle or default_handle()
    v = ctypes.c_double()
    h.check(h.lib.twed_pipe_peak(h.h, int(kind), ctypes.byref(v)))
    return v.value
