"""Thin Python binding of the C ABI in ``include/dl_gb300.h``.

Argument marshalling only: every step of the computation runs in the CUDA
kernels of ``libdl_gb300.so``.  The functions keep the C names
(``dl_init``, ``omp_code``, ``jau_update``, ``dl_iterate``, ...) and accept
either torch tensors (device or host) or raw integer pointers.  There is no
CPU fallback: if the library is missing, loading raises.

Layouts follow the C header: ``Y`` is an ``(m, p)`` float32 tensor (row i is
signal i, i.e. the column-major ``p x m`` matrix), ``D`` is ``(n, p)``
(row j is atom j), ``X`` is CSC (``colptr`` int64 ``m+1``, ``rowidx`` int32,
``val`` float32, capacity ``s*m``).
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libdl_gb300.so")

DL_OK, DL_EINVAL, DL_ECUDA, DL_ENUMERIC, DL_ETIMEOUT, DL_ENOMEM, DL_ENOTIMPL = 0, -1, -2, -3, -4, -5, -6
DL_FP32, DL_BF16, DL_FP8 = 0, 1, 2

_lib = None
_lock = threading.Lock()


class DLProblem(ctypes.Structure):
    """struct dl_problem of the C header."""
    _fields_ = [("p", ctypes.c_int), ("n", ctypes.c_int), ("s", ctypes.c_int),
                ("m", ctypes.c_int64), ("Y", ctypes.c_void_p), ("D", ctypes.c_void_p),
                ("colptr", ctypes.c_void_p), ("rowidx", ctypes.c_void_p), ("val", ctypes.c_void_p)]


class DLError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {dl_strerror(status)} (status {status})")


def load(build_if_missing: bool = True):
    """Load ``libdl_gb300.so`` (building it with nvcc first if it is missing)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            if not build_if_missing:
                raise RuntimeError(f"CUDA library not built: {LIB_PATH}")
            from . import build as _build
            _build.build()
        lib = ctypes.CDLL(LIB_PATH)
        P, i32, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
        lib.dl_init.argtypes = [ctypes.POINTER(P), i32, i32, i64, i32, i32, P]
        lib.dl_set_stream.argtypes = [P, P]
        lib.dl_destroy.argtypes = [P]
        lib.dl_strerror.argtypes = [i32]
        lib.dl_strerror.restype = ctypes.c_char_p
        lib.omp_code.argtypes = [P, P, i64, P, i32, P, P, P]
        lib.jau_update.argtypes = [P, P, i64, P, P, P, P, P]
        lib.dl_iterate.argtypes = [P, P, i64, P, i32, i32, P, P, P, P]
        lib.dl_sync.argtypes = [P]
        lib.dl_kernel_launches.argtypes = [P]
        lib.dl_kernel_launches.restype = i64
        lib.dl_set_profiling.argtypes = [P, i32]
        lib.dl_set_group_size.argtypes = [P, i32]
        lib.dl_set_deterministic.argtypes = [P, i32]
        lib.dl_set_update_rule.argtypes = [P, i32]
        lib.dl_check_bounded_wait.argtypes = [P]
        lib.dl_check_bounded_wait.restype = i32
        lib.dl_batch_set_update_rule.argtypes = [P, i32]
        lib.dl_batch_set_group_size.argtypes = [P, i32]
        lib.dl_gram.argtypes = [P, P, P]
        lib.dl_correlate.argtypes = [P, P, i64, P, P]
        lib.dl_uses_tensor_cores.argtypes = [P]
        lib.dl_correlate_noalloc.argtypes = [P, i64, P, i32, i32, P, P]
        lib.dl_correlate_noalloc_status.argtypes = [P]
        lib.dl_fp32_probe.argtypes = [i32, i64, P, P, P]
        lib.dl_last_resolved.argtypes = [P]
        lib.dl_last_resolved.restype = i64
        lib.dl_phase_times.argtypes = [P, P, i32]
        lib.dl_autotune.argtypes = [P, P, i64, P, i32]
        lib.dl_get_config.argtypes = [P, P]
        lib.dl_last_omp_kernel.argtypes = [P, ctypes.POINTER(ctypes.c_int)]
        lib.dl_batch_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(DLProblem), i32, i32, i32, P]
        lib.dl_batch_iterate.argtypes = [P, i32, P]
        lib.dl_batch_destroy.argtypes = [P]
        lib.dl_batch_kernel_launches.argtypes = [P]
        lib.dl_batch_kernel_launches.restype = i64
        lib.dl_batch_config.argtypes = [P, i32, P]
        lib.dl_proposer_create.argtypes = [ctypes.POINTER(P), i32, i32, i32, i64, P]
        lib.dl_proposer_destroy.argtypes = [P]
        lib.dl_proposer_set_weights.argtypes = [P] + [P] * 6
        lib.dl_proposer_get.argtypes = [P, i32] + [P] * 6
        lib.dl_proposer_train.argtypes = [P, P, i64, P, i32, P, i64, ctypes.c_float, P]
        lib.dl_proposer_forward.argtypes = [P, P, i64, P, P, i32]
        lib.dl_attach_proposer.argtypes = [P, P, i32, i32, ctypes.c_double]
        lib.dl_attach_correlation_proposer.argtypes = [P, i32, i32, ctypes.c_double]
        lib.dl_last_fallbacks.argtypes = [P]
        lib.dl_last_fallbacks.restype = i64
        for name in ("dl_autotune", "dl_get_config", "dl_batch_create", "dl_batch_iterate",
                     "dl_batch_destroy", "dl_batch_config", "dl_proposer_create",
                     "dl_proposer_destroy", "dl_proposer_set_weights", "dl_proposer_get",
                     "dl_proposer_train", "dl_proposer_forward", "dl_attach_proposer"):
            getattr(lib, name).restype = i32
        for name in ("dl_init", "dl_set_stream", "dl_destroy", "omp_code", "jau_update", "dl_iterate",
                     "dl_sync", "dl_set_profiling", "dl_phase_times", "dl_gram", "dl_correlate",
                     "dl_uses_tensor_cores", "dl_correlate_noalloc", "dl_correlate_noalloc_status", "dl_fp32_probe", "dl_set_deterministic", "dl_attach_correlation_proposer",
                     "dl_set_group_size",
                     "dl_set_update_rule", "dl_batch_set_update_rule", "dl_batch_set_group_size"):
            getattr(lib, name).restype = i32
        _lib = lib
        return lib


def _ptr(x):
    """Pointer of a torch tensor / numpy array / int / None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        assert x.is_contiguous(), "arrays must be contiguous"
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        assert x.flags["C_CONTIGUOUS"], "arrays must be contiguous"
        return x.ctypes.data
    raise TypeError(f"cannot take a pointer of {type(x)}")


def _check(rc: int, where: str):
    if rc != DL_OK:
        raise DLError(rc, where)


def dl_strerror(status: int) -> str:
    return load().dl_strerror(int(status)).decode()


def dl_init(p: int, n: int, m_max: int, s_max: int, precision: int = DL_FP32, stream=None) -> int:
    ctx = ctypes.c_void_p()
    _check(load().dl_init(ctypes.byref(ctx), p, n, m_max, s_max, precision, _stream_ptr(stream)),
           "dl_init")
    return ctx.value


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def dl_set_stream(ctx: int, stream) -> None:
    _check(load().dl_set_stream(ctx, _stream_ptr(stream)), "dl_set_stream")


def dl_destroy(ctx: int) -> None:
    load().dl_destroy(ctx)


def dl_sync(ctx: int) -> None:
    _check(load().dl_sync(ctx), "dl_sync")


def dl_kernel_launches(ctx: int) -> int:
    return int(load().dl_kernel_launches(ctx))


PHASES = ("gram", "correlations", "omp", "colptr_scan", "accumulate", "atoms", "rows", "finalize")


DL_RULE_AKSVD, DL_RULE_SGK, DL_RULE_NSGK = 0, 1, 2


def dl_set_update_rule(ctx: int, rule: int) -> None:
    _check(load().dl_set_update_rule(ctx, rule), "dl_set_update_rule")


def dl_check_bounded_wait(ctx: int) -> int:
    """Status of the bounded-wait failure path (DL_ETIMEOUT when it works)."""
    return load().dl_check_bounded_wait(ctx)


def dl_set_deterministic(ctx: int, on: bool = True) -> None:
    _check(load().dl_set_deterministic(ctx, int(bool(on))), "dl_set_deterministic")


def dl_set_group_size(ctx: int, ntilde: int) -> None:
    _check(load().dl_set_group_size(ctx, ntilde), "dl_set_group_size")


def dl_set_profiling(ctx: int, on: bool) -> None:
    _check(load().dl_set_profiling(ctx, 1 if on else 0), "dl_set_profiling")


def dl_phase_times(ctx: int) -> dict:
    import numpy as np
    out = np.zeros(8)
    rc = load().dl_phase_times(ctx, out.ctypes.data, 8)
    if rc < 0:
        raise DLError(rc, "dl_phase_times")
    return dict(zip(PHASES, out.tolist()))


def dl_gram(ctx: int, D, G) -> None:
    _check(load().dl_gram(ctx, _ptr(D), _ptr(G)), "dl_gram")


def dl_correlate(ctx: int, Y, m: int, D, A) -> None:
    _check(load().dl_correlate(ctx, _ptr(Y), m, _ptr(D), _ptr(A)), "dl_correlate")


def dl_correlate_noalloc(Y, m: int, D, p: int, n: int, A, stream=None) -> None:
    """A = Y^T D with no device allocation (for callers that cannot allocate:
    their memory is reserved by another allocator, or an allocation's implicit
    synchronisation is not acceptable).  p <= 64, n <= 512."""
    _check(load().dl_correlate_noalloc(_ptr(Y), m, _ptr(D), p, n, _ptr(A), _stream_ptr(stream)),
           "dl_correlate_noalloc")


def dl_correlate_noalloc_status(stream=None) -> int:
    """Synchronise ``stream`` and return (and clear) the device-side status of the
    allocation-free correlations: DL_OK, DL_ETIMEOUT or DL_ENUMERIC."""
    return int(load().dl_correlate_noalloc_status(_stream_ptr(stream)))


def dl_fp32_probe(packed: int, iters: int, out, stream=None) -> float:
    """Enqueue the FP32 multiply-add probe on ``stream``; returns its FLOP count."""
    flops = ctypes.c_double(0.0)
    _check(load().dl_fp32_probe(int(packed), int(iters), _ptr(out), ctypes.byref(flops),
                                _stream_ptr(stream)), "dl_fp32_probe")
    return flops.value


def dl_last_resolved(ctx: int) -> int:
    rc = int(load().dl_last_resolved(ctx))
    if rc < 0:
        raise DLError(rc, "dl_last_resolved")
    return rc


def dl_uses_tensor_cores(ctx: int) -> int:
    rc = load().dl_uses_tensor_cores(ctx)
    if rc < 0:
        raise DLError(rc, "dl_uses_tensor_cores")
    return rc


def omp_code(ctx: int, Y, m: int, D, s: int, colptr, rowidx, val) -> None:
    _check(load().omp_code(ctx, _ptr(Y), m, _ptr(D), s, _ptr(colptr), _ptr(rowidx), _ptr(val)),
           "omp_code")


def jau_update(ctx: int, Y, m: int, D, colptr, rowidx, val, rmse2=None) -> None:
    _check(load().jau_update(ctx, _ptr(Y), m, _ptr(D), _ptr(colptr), _ptr(rowidx), _ptr(val),
                             _ptr(rmse2)), "jau_update")


def dl_iterate(ctx: int, Y, m: int, D, s: int, iters: int, colptr, rowidx, val, rmse=None) -> None:
    _check(load().dl_iterate(ctx, _ptr(Y), m, _ptr(D), s, iters, _ptr(colptr), _ptr(rowidx),
                             _ptr(val), _ptr(rmse)), "dl_iterate")


def dl_autotune(ctx: int, Y, m: int, D, s: int) -> None:
    _check(load().dl_autotune(ctx, _ptr(Y), m, _ptr(D), s), "dl_autotune")


def dl_last_omp_kernel(ctx: int) -> int:
    """The coding kernel of the last pass: 0 Batch-OMP (warp), 1 Batch-OMP (TMEM),
    2 residual-form tensor-core OMP, 3 restricted to proposed candidates, -1 none."""
    out = ctypes.c_int(0)
    _check(load().dl_last_omp_kernel(ctx, ctypes.byref(out)), "dl_last_omp_kernel")
    return int(out.value)


def dl_get_config(ctx: int) -> dict:
    import numpy as np
    out = np.zeros(4, np.int32)
    _check(load().dl_get_config(ctx, out.ctypes.data), "dl_get_config")
    return dict(zip(("corr_tensor_cores", "omp_warps", "accum_mult", "rows_per_sm"), out.tolist()))


def dl_batch_create(problems, precision: int = DL_FP32, autotune: bool = True, stream=None):
    """problems: list of dicts with p, n, s, m and device tensors Y, D, colptr, rowidx, val."""
    arr = (DLProblem * len(problems))()
    for k, q in enumerate(problems):
        arr[k] = DLProblem(q["p"], q["n"], q["s"], q["m"], _ptr(q["Y"]), _ptr(q["D"]),
                           _ptr(q["colptr"]), _ptr(q["rowidx"]), _ptr(q["val"]))
    b = ctypes.c_void_p()
    _check(load().dl_batch_create(ctypes.byref(b), arr, len(problems), precision,
                                  1 if autotune else 0, _stream_ptr(stream)), "dl_batch_create")
    return b.value


def dl_batch_iterate(batch: int, iters: int, rmse=None) -> None:
    _check(load().dl_batch_iterate(batch, iters, _ptr(rmse)), "dl_batch_iterate")


def dl_batch_set_update_rule(batch: int, rule: int) -> None:
    _check(load().dl_batch_set_update_rule(batch, rule), "dl_batch_set_update_rule")


def dl_batch_set_group_size(batch: int, ntilde: int) -> None:
    _check(load().dl_batch_set_group_size(batch, ntilde), "dl_batch_set_group_size")


def dl_batch_destroy(batch: int) -> None:
    load().dl_batch_destroy(batch)


def dl_batch_kernel_launches(batch: int) -> int:
    return int(load().dl_batch_kernel_launches(batch))


def dl_batch_config(batch: int, k: int) -> dict:
    import numpy as np
    out = np.zeros(4, np.int32)
    _check(load().dl_batch_config(batch, k, out.ctypes.data), "dl_batch_config")
    return dict(zip(("corr_tensor_cores", "omp_warps", "accum_mult", "rows_per_sm"), out.tolist()))


def dl_proposer_create(p: int, n: int, hidden: int = 512, batch: int = 4096, stream=None) -> int:
    h = ctypes.c_void_p()
    _check(load().dl_proposer_create(ctypes.byref(h), p, n, hidden, batch, _stream_ptr(stream)),
           "dl_proposer_create")
    return h.value


def dl_proposer_destroy(prop: int) -> None:
    load().dl_proposer_destroy(prop)


def dl_proposer_set_weights(prop: int, params) -> None:
    """params: [W1 (h,p), b1, W2 (h,h), b2, W3 (n,h), b3] numpy arrays."""
    import numpy as np
    arrs = [np.ascontiguousarray(a, np.float32) for a in params]
    _check(load().dl_proposer_set_weights(prop, *[a.ctypes.data for a in arrs]),
           "dl_proposer_set_weights")


def dl_proposer_get(prop: int, which: int, shapes):
    import numpy as np
    outs = [np.zeros(sh, np.float32) for sh in shapes]
    _check(load().dl_proposer_get(prop, which, *[a.ctypes.data for a in outs]), "dl_proposer_get")
    return outs


def dl_proposer_train(prop: int, Y, m: int, sup, s: int, perm=None, batch: int = 4096,
                      lr: float = 1e-3) -> float:
    import numpy as np
    loss = np.zeros(1)
    _check(load().dl_proposer_train(prop, _ptr(Y), m, _ptr(sup), s, _ptr(perm), batch, lr,
                                    loss.ctypes.data), "dl_proposer_train")
    return float(loss[0])


def dl_proposer_forward(prop: int, Y, m: int, logits=None, cand=None, K: int = 16) -> None:
    _check(load().dl_proposer_forward(prop, _ptr(Y), m, _ptr(logits), _ptr(cand), K),
           "dl_proposer_forward")


def dl_attach_proposer(ctx: int, prop, K: int = 16, full_every: int = 10, tol: float = 0.01) -> None:
    _check(load().dl_attach_proposer(ctx, prop, K, full_every, tol), "dl_attach_proposer")


def dl_attach_correlation_proposer(ctx: int, K: int, full_every: int = 10, tol: float = 0.01) -> None:
    """Candidates = the K largest |D^T y| (no network); otherwise as dl_attach_proposer."""
    _check(load().dl_attach_correlation_proposer(ctx, K, full_every, tol),
           "dl_attach_correlation_proposer")


def dl_last_fallbacks(ctx: int) -> int:
    return int(load().dl_last_fallbacks(ctx))


class Context:
    """Owns one ``dl_ctx`` and the CSC output tensors for convenience."""

    def __init__(self, p: int, n: int, m_max: int, s_max: int, precision: int = DL_FP32,
                 device=None, stream=None):
        import torch
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else device
        with torch.cuda.device(self.device):
            if stream is None:
                stream = torch.cuda.current_stream(self.device)
            self.ctx = dl_init(p, n, m_max, s_max, precision, stream)
        self.p, self.n, self.m_max, self.s_max = p, n, m_max, s_max

    def close(self):
        if getattr(self, "ctx", None):
            dl_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def alloc_csc(self, m: int, s: int, device=None):
        import torch
        dev = self.device if device is None else device
        colptr = torch.zeros(m + 1, dtype=torch.int64, device=dev)
        rowidx = torch.zeros(max(1, m * s), dtype=torch.int32, device=dev)
        val = torch.zeros(max(1, m * s), dtype=torch.float32, device=dev)
        return colptr, rowidx, val
