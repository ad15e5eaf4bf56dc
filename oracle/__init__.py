"""FP64 CPU oracle for dictionary learning with Jacobi atom updates.

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The GPU library never
imports this package and this package never imports the GPU library; the two
share only the seeded input generators of ``paper_1509_05054_gb300.synth``.

The arithmetic lives in ``dl_oracle.c`` (plain C, double precision, OpenMP
over signals / atoms).  This module compiles it with gcc on first use (or via
:func:`build`) and wraps it with ctypes.  Layout conventions follow the paper's
problem statement (Section 1, Eq. 1):

* ``Y`` is given as an ``(m, p)`` C-contiguous array: row i is signal i, which
  is the column-major ``p x m`` matrix of the paper;
* ``D`` is ``(n, p)``: row j is atom d_j;
* the sparse ``X`` is returned in per-signal slots ``idx (m, s)`` int32,
  ``val (m, s)`` float64 and ``cnt (m,)`` int32, atoms ascending, unused slots
  ``idx = -1``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dl_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

RULE_AKSVD = 0
RULE_SGK = 1
RULE_NSGK = 2  # oracle_dl only: P-NSGK (Eq. 7), see atom_update_nsgk


def build(force: bool = False) -> str:
    """Compile ``dl_oracle.c`` into ``oracle/_build/liboracle.so`` with gcc."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            P = ctypes.c_void_p
            i32, i64 = ctypes.c_int, ctypes.c_int64
            lib.oracle_gram.argtypes = [i32, i32, P, P, i32]
            lib.oracle_omp.argtypes = [i32, i32, i64, P, P, i32, P, P, P, P, i32]
            lib.oracle_omp_naive.argtypes = [i32, i32, i64, P, P, i32, P, P, P, i32]
            lib.oracle_error_energy.argtypes = [i32, i64, P, P, i32, P, P, P, P, i32]
            lib.oracle_atom_update.argtypes = [i32, i32, i64, P, P, i32, P, P, P, i32, i32, i32,
                                               P, i32]
            lib.oracle_atom_update_nsgk.argtypes = [i32, i32, i64, P, P, i32, P, P, P, P, P, P,
                                                    i32, P, i32]
            lib.oracle_dl.argtypes = [i32, i32, i64, P, P, i32, i32, i32, i32, P, P, P, P, i32]
            lib.oracle_max_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def gram(D, nthreads: int = 0):
    """G = D^T D for D given as (n, p) rows = atoms."""
    D = _f64(D)
    n, p = D.shape
    G = np.empty((n, n))
    _load().oracle_gram(p, n, _ptr(D), _ptr(G), nthreads)
    return G


def omp(Y, D, s: int, nthreads: int = 0, return_gaps: bool = False):
    """Batch-OMP (Cholesky form) of every signal. Returns (idx, val, cnt[, gaps])."""
    Y, D = _f64(Y), _f64(D)
    m, p = Y.shape
    n = D.shape[0]
    assert D.shape[1] == p
    idx = np.empty((m, s), np.int32)
    val = np.empty((m, s))
    cnt = np.empty(m, np.int32)
    gaps = np.empty((m, s)) if return_gaps else None
    _load().oracle_omp(p, n, m, _ptr(Y), _ptr(D), s, _ptr(idx), _ptr(val), _ptr(cnt),
                       _ptr(gaps) if return_gaps else None, nthreads)
    return (idx, val, cnt, gaps) if return_gaps else (idx, val, cnt)


def omp_naive(Y, D, s: int, nthreads: int = 0):
    """Textbook residual-form OMP, written independently of :func:`omp`."""
    Y, D = _f64(Y), _f64(D)
    m, p = Y.shape
    n = D.shape[0]
    idx = np.empty((m, s), np.int32)
    val = np.empty((m, s))
    cnt = np.empty(m, np.int32)
    _load().oracle_omp_naive(p, n, m, _ptr(Y), _ptr(D), s, _ptr(idx), _ptr(val), _ptr(cnt),
                             nthreads)
    return idx, val, cnt


def error_energy(Y, D, idx, val, cnt, nthreads: int = 0):
    """Return (||Y - D X||_F^2, ||Y||_F^2)."""
    Y, D = _f64(Y), _f64(D)
    m, p = Y.shape
    s = idx.shape[1]
    idx = np.ascontiguousarray(idx, np.int32)
    val = _f64(val)
    cnt = np.ascontiguousarray(cnt, np.int32)
    out = np.empty(2)
    _load().oracle_error_energy(p, m, _ptr(Y), _ptr(D), s, _ptr(idx), _ptr(val), _ptr(cnt),
                                _ptr(out), nthreads)
    return float(out[0]), float(out[1])


def rmse(Y, D, idx, val, cnt, nthreads: int = 0) -> float:
    """Relative error ||Y - D X||_F / ||Y||_F."""
    ee, yy = error_energy(Y, D, idx, val, cnt, nthreads)
    return float(np.sqrt(ee / yy)) if yy > 0 else 0.0


def atom_update(Y, D, idx, val, cnt, ntilde: int | None = None, rule: int = RULE_AKSVD,
                only_atom: int = -1, nthreads: int = 0):
    """Atom-update stage (Algorithm 1 steps 2-5). Returns (D_new, val_new, n_unused)."""
    Y = _f64(Y)
    D = _f64(D).copy()
    m, p = Y.shape
    n = D.shape[0]
    s = idx.shape[1]
    idx = np.ascontiguousarray(idx, np.int32)
    val = _f64(val).copy()
    cnt = np.ascontiguousarray(cnt, np.int32)
    unused = ctypes.c_int(0)
    _load().oracle_atom_update(p, n, m, _ptr(Y), _ptr(D), s, _ptr(idx), _ptr(val), _ptr(cnt),
                               n if ntilde is None else int(ntilde), int(rule), int(only_atom),
                               ctypes.cast(ctypes.pointer(unused), ctypes.c_void_p), nthreads)
    return D, val, int(unused.value)


def atom_update_nsgk(Y, D, idx, val, cnt, pidx, pval, pcnt, ntilde: int | None = None,
                     nthreads: int = 0):
    """P-NSGK atom-update stage (Eq. 7): SGK on Z = Y + D X_prev - D X with the
    representations X_prev.  Returns (D_new, n_unused); X and X_prev unchanged."""
    Y = _f64(Y)
    D = _f64(D).copy()
    m, p = Y.shape
    n = D.shape[0]
    s = idx.shape[1]
    unused = ctypes.c_int(0)
    args = [np.ascontiguousarray(idx, np.int32), _f64(val), np.ascontiguousarray(cnt, np.int32),
            np.ascontiguousarray(pidx, np.int32), _f64(pval), np.ascontiguousarray(pcnt, np.int32)]
    _load().oracle_atom_update_nsgk(p, n, m, _ptr(Y), _ptr(D), s, *[_ptr(a) for a in args],
                                    n if ntilde is None else int(ntilde),
                                    ctypes.cast(ctypes.pointer(unused), ctypes.c_void_p), nthreads)
    return D, unused.value


def jau(Y, D, idx, val, cnt, nthreads: int = 0):
    """PAK-SVD with full parallelism (ntilde = n): returns (D_new, val_new, n_unused)."""
    return atom_update(Y, D, idx, val, cnt, ntilde=None, rule=RULE_AKSVD, nthreads=nthreads)


def dl(Y, D, s: int, iters: int, ntilde: int | None = None, rule: int = RULE_AKSVD,
       nthreads: int = 0):
    """Algorithm 1 repeated `iters` times. Returns (D, idx, val, cnt, rmse[iters, 2])."""
    Y = _f64(Y)
    D = _f64(D).copy()
    m, p = Y.shape
    n = D.shape[0]
    idx = np.empty((m, s), np.int32)
    val = np.empty((m, s))
    cnt = np.empty(m, np.int32)
    r = np.empty((iters, 2))
    _load().oracle_dl(p, n, m, _ptr(Y), _ptr(D), s, iters, n if ntilde is None else int(ntilde),
                      int(rule), _ptr(idx), _ptr(val), _ptr(cnt), _ptr(r), nthreads)
    return D, idx, val, cnt, r


def slots_to_dense(idx, val, cnt, n: int):
    """Dense X (n x m) from slots; for small test cases."""
    m, s = idx.shape
    X = np.zeros((n, m))
    for i in range(m):
        for t in range(int(cnt[i])):
            X[idx[i, t], i] = val[i, t]
    return X
