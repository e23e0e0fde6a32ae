"""CPU oracle for Time Warp Edit Distance -- TEST INFRASTRUCTURE ONLY.

Plain FP64 statement of the TWED dynamic program (paper: section "Time Warp
Edit Distance", steps 1-6; recurrence restated in ``twed_oracle.c``).  It is
compiled with gcc from ``twed_oracle.c`` and loaded with ctypes.  Only the
tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this package; the library in ``paper_2007_16135_gb300`` never
does, and the two share no code.

Entry points (all values float64; series are ``[len, dim]`` arrays):

* ``twed(a, ta, b, tb, nu, lam, p)`` -- full (n+1)x(m+1) matrix, C order.
* ``twed_rolling(...)`` -- same operations, two rows of memory (O(m)).
* ``delete_costs(a, ta, nu, lam, p)`` -- dA(1..n) of one series.
* ``twed_pairs(setA, setB, pairs, dim, nu, lam, p, nthreads)`` -- rolling
  oracle over listed pairs of two packed sets, threads over pairs.
* ``twed_path(a, ta, b, tb, nu, lam, p)`` -- TWED and an optimal edit path
  (full matrix, walk back with a fixed tie-break), as a string of moves.
* ``lcs_length(x, y)``, ``lcs_length_rolling(x, y)``, ``lcs_pairs(x, y)`` --
  longest common subsequence of int32 sequences (``lcs_oracle.c``): its
  length (full matrix / two rows) and one subsequence.
* ``dtw(a, b, p)`` -- dynamic time warping distance (``dtw_oracle.c``).

Parity pins for these functions live in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "twed_oracle.c")
_SRC_LCS = os.path.join(_HERE, "lcs_oracle.c")
_SRC_DTW = os.path.join(_HERE, "dtw_oracle.c")
_SOURCES = [_SRC, _SRC_LCS, _SRC_DTW]
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

# -ffp-contract=off: no FMA contraction (gcc on aarch64 contracts by default),
# so every operation rounds exactly as written in twed_oracle.c.
CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c99"]


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (seconds)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(f) for f in _SOURCES)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, *_SOURCES, "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


def _declare(lib):
    d, i64, ci = ctypes.c_double, ctypes.c_int64, ctypes.c_int
    P = ctypes.c_void_p
    for name in ("oracle_twed", "oracle_twed_rolling"):
        f = getattr(lib, name)
        f.restype = ci
        f.argtypes = [P, P, i64, P, P, i64, ci, d, d, ci, P]
    lib.oracle_delete_costs.restype = ci
    lib.oracle_delete_costs.argtypes = [P, P, i64, ci, d, d, ci, P]
    lib.oracle_twed_path.restype = ci
    lib.oracle_twed_path.argtypes = [P, P, i64, P, P, i64, ci, d, d, ci, P, P, P]
    for name in ("oracle_lcs_length", "oracle_lcs_length_rolling"):
        f = getattr(lib, name)
        f.restype = ci
        f.argtypes = [P, i64, P, i64, P]
    lib.oracle_dtw.restype = ci
    lib.oracle_dtw.argtypes = [P, i64, P, i64, ci, ci, P]
    lib.oracle_lcs_pairs.restype = ci
    lib.oracle_lcs_pairs.argtypes = [P, i64, P, i64, P, P, P]
    lib.oracle_twed_pairs.restype = ci
    lib.oracle_twed_pairs.argtypes = [P, P, P, P, P, P, P, i64, ci, d, d, ci, ci, P]
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _declare(ctypes.CDLL(build()))
    return _lib


def compile_library(out_path: str, sources) -> ctypes.CDLL:
    """Compile the given oracle sources (the files of ``SOURCE_FILES``,
    possibly from another directory) with the oracle's own flags into
    ``out_path`` and load them.  Used by the pin-strength tests, which build
    private copies with planted mistakes."""
    subprocess.check_call(["gcc", *CFLAGS, "-o", out_path, *sources, "-lm", "-lpthread"])
    return _declare(ctypes.CDLL(out_path))


SOURCE_FILES = [os.path.basename(f) for f in _SOURCES]
SOURCE_DIR = _HERE


def twed_of(lib) -> "callable":
    """The full-matrix ``twed`` of a library from :func:`compile_library`."""
    return lambda a, ta, b, tb, nu, lam, p=2: _call(lib.oracle_twed, a, ta, b, tb, nu, lam, p)


def twed_path_of(lib) -> "callable":
    """As :func:`twed_of`, for ``twed_path``."""
    return lambda a, ta, b, tb, nu, lam, p=2: _path_call(lib, a, ta, b, tb, nu, lam, p)


def _series(a, ta):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.ndim == 1:
        a = a[:, None]
    ta = np.ascontiguousarray(ta, dtype=np.float64)
    if ta.shape != (a.shape[0],):
        raise ValueError("timestamps must have one entry per point")
    return a, ta


def _ptr(x):
    return x.ctypes.data_as(ctypes.c_void_p) if x is not None else None


class OracleError(RuntimeError):
    pass


def _call(fn, a, ta, b, tb, nu, lam, p):
    a, ta = _series(a, ta)
    b, tb = _series(b, tb)
    if a.shape[1] != b.shape[1]:
        raise ValueError("series dimensions differ")
    out = np.zeros(1, dtype=np.float64)
    rc = fn(_ptr(a), _ptr(ta), a.shape[0], _ptr(b), _ptr(tb), b.shape[0], a.shape[1],
            float(nu), float(lam), int(p), _ptr(out))
    if rc:
        raise OracleError(f"oracle rejected its arguments (status {rc})")
    return float(out[0])


def twed(a, ta, b, tb, nu, lam, p=2):
    """TWED by the full-matrix dynamic program (C order)."""
    return _call(_load().oracle_twed, a, ta, b, tb, nu, lam, p)


def twed_rolling(a, ta, b, tb, nu, lam, p=2):
    """TWED with two rolling rows; bit-identical to :func:`twed`."""
    return _call(_load().oracle_twed_rolling, a, ta, b, tb, nu, lam, p)


def twed_path(a, ta, b, tb, nu, lam, p=2):
    """TWED and one optimal edit path, ``(value, moves)``.

    ``moves`` lists the steps after the forced first match (0,0) -> (1,1), in
    order: ``'M'`` match (i+1, j+1), ``'A'`` delete in a (i+1, j), ``'B'``
    delete in b (i, j+1).  Among optimal paths the one returned is fixed by
    the walk back from (n,m): at each cell the first of match, delete in a,
    delete in b whose candidate equals D(i,j)."""
    return _path_call(_load(), a, ta, b, tb, nu, lam, p)


def _path_call(lib, a, ta, b, tb, nu, lam, p):
    a, ta = _series(a, ta)
    b, tb = _series(b, tb)
    if a.shape[1] != b.shape[1]:
        raise ValueError("series dimensions differ")
    out = np.zeros(1, dtype=np.float64)
    moves = np.zeros(max(a.shape[0] + b.shape[0] - 2, 1), dtype=np.int8)
    length = np.zeros(1, dtype=np.int64)
    rc = lib.oracle_twed_path(_ptr(a), _ptr(ta), a.shape[0], _ptr(b), _ptr(tb), b.shape[0],
                              a.shape[1], float(nu), float(lam), int(p), _ptr(out),
                              _ptr(moves), _ptr(length))
    if rc:
        raise OracleError(f"oracle path failed (status {rc})")
    return float(out[0]), "".join("MAB"[x] for x in moves[:int(length[0])])


def _symbols(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.int32).ravel())


def _lcs_call(fn, x, y):
    x, y = _symbols(x), _symbols(y)
    out = np.zeros(1, dtype=np.int64)
    rc = fn(_ptr(x), x.size, _ptr(y), y.size, _ptr(out))
    if rc:
        raise OracleError(f"LCS oracle failed (status {rc})")
    return int(out[0])


def lcs_length(x, y, lib=None):
    """Length of a longest common subsequence of two int32 symbol sequences
    (full matrix).  `lib`: a variant library (pin-strength tests only)."""
    return _lcs_call((lib or _load()).oracle_lcs_length, x, y)


def lcs_length_rolling(x, y, lib=None):
    """As :func:`lcs_length` on two rows of memory."""
    return _lcs_call((lib or _load()).oracle_lcs_length_rolling, x, y)


def lcs_pairs(x, y, lib=None):
    """One longest common subsequence as matched positions ``(xi, yj)``
    (0-based, increasing), by the textbook walk back: diagonal on a match,
    else up when L(i-1,j) >= L(i,j-1), else left."""
    lib = lib or _load()
    x, y = _symbols(x), _symbols(y)
    k = max(min(x.size, y.size), 1)
    xi = np.zeros(k, dtype=np.int64)
    yj = np.zeros(k, dtype=np.int64)
    length = np.zeros(1, dtype=np.int64)
    rc = lib.oracle_lcs_pairs(_ptr(x), x.size, _ptr(y), y.size, _ptr(xi), _ptr(yj), _ptr(length))
    if rc:
        raise OracleError(f"LCS oracle failed (status {rc})")
    n = int(length[0])
    return xi[:n].copy(), yj[:n].copy()


def dtw(a, b, p=2, lib=None):
    """Dynamic time warping distance of two ``[len, dim]`` series with the lp
    point distance (full matrix, ``dtw_oracle.c``).  `lib`: a variant
    library (pin-strength tests only)."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    a = a[:, None] if a.ndim == 1 else a
    b = b[:, None] if b.ndim == 1 else b
    if a.shape[1] != b.shape[1]:
        raise ValueError("series dimensions differ")
    out = np.zeros(1, dtype=np.float64)
    rc = (lib or _load()).oracle_dtw(_ptr(a), a.shape[0], _ptr(b), b.shape[0], a.shape[1], int(p),
                                     _ptr(out))
    if rc:
        raise OracleError(f"DTW oracle rejected its arguments (status {rc})")
    return float(out[0])


def delete_costs(a, ta, nu, lam, p=2):
    """dA(i) = d(a_i, a_{i-1}) + nu |t_i - t_{i-1}| + lambda for i = 1..n."""
    a, ta = _series(a, ta)
    out = np.zeros(a.shape[0], dtype=np.float64)
    rc = _load().oracle_delete_costs(_ptr(a), _ptr(ta), a.shape[0], a.shape[1], float(nu),
                                     float(lam), int(p), _ptr(out))
    if rc:
        raise OracleError(f"oracle rejected its arguments (status {rc})")
    return out


def twed_pairs(setA, setB, pairs, nu, lam, p=2, nthreads=None):
    """Rolling oracle over ``pairs`` ([k, 2] int64 indices into A and B).

    A set is a tuple ``(vals [sum_len, dim], ts [sum_len], offs [n+1])``.
    """
    va, ta, oa = setA
    vb, tb, ob = setB
    va = np.ascontiguousarray(va, dtype=np.float64)
    vb = np.ascontiguousarray(vb, dtype=np.float64)
    if va.ndim == 1:
        va = va[:, None]
    if vb.ndim == 1:
        vb = vb[:, None]
    ta = np.ascontiguousarray(ta, dtype=np.float64)
    tb = np.ascontiguousarray(tb, dtype=np.float64)
    oa = np.ascontiguousarray(oa, dtype=np.int64)
    ob = np.ascontiguousarray(ob, dtype=np.int64)
    pairs = np.ascontiguousarray(pairs, dtype=np.int64).reshape(-1, 2)
    if nthreads is None:
        nthreads = os.cpu_count() or 1
    out = np.zeros(pairs.shape[0], dtype=np.float64)
    rc = _load().oracle_twed_pairs(_ptr(va), _ptr(ta), _ptr(oa), _ptr(vb), _ptr(tb), _ptr(ob),
                                   _ptr(pairs), pairs.shape[0], va.shape[1], float(nu),
                                   float(lam), int(p), int(nthreads), _ptr(out))
    if rc:
        raise OracleError(f"oracle rejected its arguments (status {rc})")
    return out
