"""FP64 CPU oracle of LBG vector-quantizer design -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``lbg_oracle.c`` (plain C,
double precision, index-order sums) with ctypes and numpy marshalling; it
shares no code with the CUDA library and never imports it.

Each function follows a step of Annaji & Rao, "Parallelization of the LBG
Vector Quantization Algorithm for Shared Memory Systems":

* :func:`mean`     -- initial codebook = centroid of the training set (Alg. 1, Table 1)
* :func:`split`    -- codebook splitting c+delta, c-delta (Alg. 1, Sec. 3.2)
* :func:`assign`   -- cell allocation / nearest codevector (Alg. 1, Sec. 2.2 step 1)
* :func:`update`   -- updation: centroid of every cell (Alg. 1, Sec. 2.2 step 3)
* :func:`lloyd_step` -- allocation + distortion integration + updation
* :func:`lbg_train`  -- the whole split/iterate design with the Sec. 2.2 stop test
* :func:`grad`, :func:`distortion_fixed` -- D at a fixed cell table and its gradient

The readings taken where the paper is silent or inconsistent are listed at
the top of ``lbg_oracle.c``.  Every function is pinned by ``tests/test_oracle.py``
(exact brute force, closed forms, hand-worked cases, invariants, scipy, finite
differences), and ``tests/test_oracle_mutants.py`` checks that those pins fail
on copies of ``lbg_oracle.c`` with plausible mistakes planted in them; no
function is left with its parity unpinned.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbg_oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "liblbgoracle.so")
_lock = threading.Lock()
_lib = None

OK, WARN_MAXPASS = 0, 1


#: Environment variable naming another compiled copy of the oracle to load
#: instead of ``_lib/liblbgoracle.so`` (the mutation test of the pins loads
#: copies of ``lbg_oracle.c`` with planted mistakes through it).
LIBRARY_ENV = "LBG_ORACLE_LIBRARY"


def compile_source(src: str, out: str) -> str:
    """Compile one C source of the oracle into the shared library ``out``.

    ``-ffp-contract=off`` keeps a*b+c unfused so x86 and aarch64 give the
    same bits; OpenMP parallelises only the independent rows of the cell
    allocation.
    """
    tmp = out + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp",
           src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile ``lbg_oracle.c`` into ``_lib/liblbgoracle.so`` (if out of date)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    return compile_source(_SRC, _LIB)


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(os.environ.get(LIBRARY_ENV) or build())
        P = ctypes.c_void_p
        i64, i32, f64 = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
        lib.oracle_max_threads.restype = ctypes.c_int
        lib.oracle_mean.argtypes = [P, i64, i32, P]
        lib.oracle_split.argtypes = [P, i32, i32, f64, P]
        lib.oracle_split_mode.argtypes = [P, i32, i32, f64, i32, P]
        lib.oracle_reseed.argtypes = [P, P, i32, i32, f64]
        lib.oracle_assign.argtypes = [P, i64, i32, P, i32, P, P, P, i32]
        lib.oracle_sum.argtypes = [P, i64]
        lib.oracle_sum.restype = f64
        lib.oracle_update.argtypes = [P, i64, i32, P, i32, P, P, P]
        lib.oracle_lloyd_step.argtypes = [P, i64, i32, P, i32, P, P, P, P, P, P, i32]
        lib.oracle_distortion_fixed.argtypes = [P, i64, i32, P, P]
        lib.oracle_distortion_fixed.restype = f64
        lib.oracle_grad.argtypes = [P, i64, i32, P, i32, P, P, P]
        lib.oracle_lbg_train.argtypes = [P, i64, i32, i32, f64, f64, i32, i32, i32, i32, P, i32,
                                         P, P, P, P, P, P, P, f64, i32, P]
        _lib = lib
        return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _x(X):
    X = np.ascontiguousarray(X, dtype=np.float32)
    if X.ndim != 2:
        raise ValueError("X must be [M, L]")
    return X


def _c(C):
    C = np.ascontiguousarray(C, dtype=np.float64)
    if C.ndim != 2:
        raise ValueError("C must be [N, L]")
    return C


def _check(rc, what):
    if rc < 0:
        raise ValueError(f"oracle {what} failed with status {rc}")
    return rc


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def mean(X) -> np.ndarray:
    """Centroid of all training vectors, [1, L] float64."""
    X = _x(X)
    out = np.empty((1, X.shape[1]), np.float64)
    _check(_load().oracle_mean(_ptr(X), X.shape[0], X.shape[1], _ptr(out)), "mean")
    return out


def split(C, delta: float, multiplicative: bool = False) -> np.ndarray:
    """[2n, L]: row 2i = c_i + delta, row 2i+1 = c_i - delta (or c_i (1 +- delta))."""
    C = _c(C)
    out = np.empty((2 * C.shape[0], C.shape[1]), np.float64)
    _check(_load().oracle_split_mode(_ptr(C), C.shape[0], C.shape[1], float(delta),
                                     int(bool(multiplicative)), _ptr(out)), "split")
    return out


def reseed(C, counts, delta: float):
    """Variant V2 (see lbg_oracle.c): (C', counts') with the empty cells re-seeded."""
    C = _c(C).copy()
    counts = np.ascontiguousarray(counts, dtype=np.int64).copy()
    _check(_load().oracle_reseed(_ptr(C), _ptr(counts), C.shape[0], C.shape[1], float(delta)),
           "reseed")
    return C, counts


def assign(X, C, nthreads: int = 0):
    """Nearest codevector of every row: (a int32[M], e float64[M], gap float64[M])."""
    X, C = _x(X), _c(C)
    if X.shape[1] != C.shape[1]:
        raise ValueError("dimension mismatch")
    M = X.shape[0]
    a = np.empty(M, np.int32)
    e = np.empty(M, np.float64)
    g = np.empty(M, np.float64)
    _check(_load().oracle_assign(_ptr(X), M, X.shape[1], _ptr(C), C.shape[0], _ptr(a), _ptr(e),
                                 _ptr(g), int(nthreads)), "assign")
    return a, e, g


def update(X, a, C_in):
    """Cell centroids: (C_out float64[N, L], counts int64[N]); empty cells keep C_in."""
    X, C_in = _x(X), _c(C_in)
    a = np.ascontiguousarray(a, dtype=np.int32)
    N, L = C_in.shape
    out = np.empty((N, L), np.float64)
    counts = np.empty(N, np.int64)
    _check(_load().oracle_update(_ptr(X), X.shape[0], L, _ptr(a), N, _ptr(C_in), _ptr(out),
                                 _ptr(counts)), "update")
    return out, counts


@dataclass
class Step:
    a: np.ndarray
    e: np.ndarray
    gap: np.ndarray
    D: float
    C: np.ndarray
    counts: np.ndarray


def lloyd_step(X, C_in, nthreads: int = 0) -> Step:
    """One pass: allocation, distortion, updation (no stop test)."""
    X, C_in = _x(X), _c(C_in)
    M, L = X.shape
    N = C_in.shape[0]
    a = np.empty(M, np.int32)
    e = np.empty(M, np.float64)
    g = np.empty(M, np.float64)
    D = ctypes.c_double()
    out = np.empty((N, L), np.float64)
    counts = np.empty(N, np.int64)
    _check(_load().oracle_lloyd_step(_ptr(X), M, L, _ptr(C_in), N, _ptr(a), _ptr(e), _ptr(g),
                                     ctypes.byref(D), _ptr(out), _ptr(counts), int(nthreads)),
           "lloyd_step")
    return Step(a, e, g, D.value, out, counts)


def distortion_fixed(X, C, a) -> float:
    X, C = _x(X), _c(C)
    a = np.ascontiguousarray(a, dtype=np.int32)
    return float(_load().oracle_distortion_fixed(_ptr(X), X.shape[0], X.shape[1], _ptr(C), _ptr(a)))


def grad(X, C, a):
    """(dD/dC float64[N, L], dD/dX float64[M, L]) at the fixed cell table a."""
    X, C = _x(X), _c(C)
    a = np.ascontiguousarray(a, dtype=np.int32)
    gC = np.empty_like(C)
    gX = np.empty(X.shape, np.float64)
    _check(_load().oracle_grad(_ptr(X), X.shape[0], X.shape[1], _ptr(C), C.shape[0], _ptr(a),
                               _ptr(gC), _ptr(gX)), "grad")
    return gC, gX


@dataclass
class Train:
    status: int
    C: np.ndarray
    a: np.ndarray
    D: float
    trace_n: np.ndarray = field(default_factory=lambda: np.empty(0, np.int32))
    trace_pass: np.ndarray = field(default_factory=lambda: np.empty(0, np.int32))
    trace_D: np.ndarray = field(default_factory=lambda: np.empty(0, np.float64))
    trace_near: np.ndarray = field(default_factory=lambda: np.empty(0, np.int32))

    def near_ties(self) -> int:
        """Rows that were near-ties (gap <= near_tol), summed over all passes."""
        return int(self.trace_near.sum())

    def passes_per_stage(self):
        """Number of passes run at each stage size, in stage order."""
        out = []
        for n, p in zip(self.trace_n.tolist(), self.trace_pass.tolist()):
            if p == 0:
                out.append(0)
            out[-1] += 1
        return out


def lbg_train(X, N: int, delta: float, theta: float, max_passes: int = 1000,
              nthreads: int = 0, trace_cap: int = 100000, C_init=None,
              near_tol: float = 1e-5, split_multiplicative: bool = False,
              reseed_empty: bool = False) -> Train:
    """The whole LBG design up to N codevectors, from the centroid of X or,
    if C_init ([n_init, L]) is given, from that initial alphabet (Sec. 2.2)."""
    X = _x(X)
    Ci = None if C_init is None else _c(C_init)
    n_init = 0 if Ci is None else Ci.shape[0]
    M, L = X.shape
    C = np.empty((N, L), np.float64)
    a = np.empty(M, np.int32)
    D = ctypes.c_double()
    rn = np.empty(trace_cap, np.int32)
    rp = np.empty(trace_cap, np.int32)
    rD = np.empty(trace_cap, np.float64)
    rnear = np.empty(trace_cap, np.int32)
    cnt = ctypes.c_int32()
    rc = _load().oracle_lbg_train(_ptr(X), M, L, int(N), float(delta), float(theta),
                                  int(max_passes), int(nthreads), int(bool(split_multiplicative)),
                                  int(bool(reseed_empty)), _ptr(Ci), n_init, _ptr(C),
                                  _ptr(a),
                                  ctypes.byref(D), _ptr(rn), _ptr(rp), _ptr(rD), _ptr(rnear),
                                  float(near_tol), trace_cap, ctypes.byref(cnt))
    _check(rc, "lbg_train")
    k = min(cnt.value, trace_cap)
    return Train(rc, C, a, D.value, rn[:k].copy(), rp[:k].copy(), rD[:k].copy(), rnear[:k].copy())
