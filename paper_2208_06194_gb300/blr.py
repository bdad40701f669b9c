"""Thin Python binding of the BLR-QR C ABI (include/blr.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Function names follow the C entry points.  Device matrices are
torch float64 CUDA tensors in column-major layout (shape (rows, cols),
stride (1, ld)); ``fortran_empty``/``to_fortran`` make them.  The library
must have been built (``paper_2208_06194_gb300.build.build()``); importing
works without it, but the first call raises if it is missing.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libblrqr.so")

BLR_PREC_FP64 = 0
BLR_PREC_MIXED = 1
KERNEL_IDS = {"inv1d": 0, "yukawa3d": 1, "laplace3d": 2}
ERRORS = {1: "INVALID", 2: "OOM", 3: "CUDA", 4: "TIMEOUT", 5: "NUMERIC", 6: "RANK_OVERFLOW"}


class BLRError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"BLR_ERR_{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Opts(ctypes.Structure):
    _fields_ = [("b", ctypes.c_int), ("fixed_rank", ctypes.c_int), ("tol", ctypes.c_double),
                ("rec_tol", ctypes.c_double), ("dense_rank", ctypes.c_int),
                ("precision", ctypes.c_int), ("sched_ctas", ctypes.c_int),
                ("watchdog_ms", ctypes.c_int), ("scratch_b2", ctypes.c_int), ("trace", ctypes.c_int),
                ("eta", ctypes.c_double), ("test_withhold", ctypes.c_int), ("prep_slots", ctypes.c_int),
                ("reserved", ctypes.c_int * 2)]


class TraceEvent(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int), ("i", ctypes.c_int), ("j", ctypes.c_int), ("k", ctypes.c_int),
                ("matrix", ctypes.c_int), ("cta", ctypes.c_int), ("sm", ctypes.c_int), ("reserved", ctypes.c_int),
                ("t_start_ns", ctypes.c_longlong), ("t_end_ns", ctypes.c_longlong)]


class Stats(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int), ("n", ctypes.c_int), ("b", ctypes.c_int), ("p", ctypes.c_int),
                ("q", ctypes.c_int), ("n_dense", ctypes.c_int), ("max_rank", ctypes.c_int),
                ("mean_rank", ctypes.c_double), ("device_bytes", ctypes.c_longlong),
                ("flops", ctypes.c_double * 5), ("tasks", ctypes.c_longlong * 4),
                ("task_seconds", ctypes.c_double * 4), ("seconds", ctypes.c_double),
                ("tpmqrt_kind", ctypes.c_longlong * 8), ("tpmqrt_kind_seconds", ctypes.c_double * 8),
                ("tpmqrt_kind_flops", ctypes.c_double * 8), ("scratch_peak_bytes", ctypes.c_longlong),
                ("scratch_bytes", ctypes.c_longlong), ("prep_slots", ctypes.c_longlong),
                ("prep_misses", ctypes.c_longlong)]


_lib = None
_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_DP = ctypes.POINTER(ctypes.c_double)
_IP = ctypes.POINTER(ctypes.c_int)

_SIGS = {
    "blr_opts_default": (None, [ctypes.POINTER(Opts)]),
    "blr_last_error": (ctypes.c_char_p, []),
    "blr_compress_kernel": (_I, [_DP, _DP, _I, _I, _I, _I, _DP, ctypes.POINTER(Opts), ctypes.POINTER(_P), _P]),
    "blr_compress_dense": (_I, [_P, _I, _I, _I, ctypes.POINTER(Opts), ctypes.POINTER(_P), _P]),
    "blr_matrix_import": (_I, [_I, _I, _I, _IP, _DP, ctypes.POINTER(_P), _P]),
    "blr_matrix_import_device": (_I, [_I, _I, _I, _IP, _P, ctypes.POINTER(_P), _P]),
    "blr_matrix_export": (_I, [_P, _I, _IP, _DP, _P]),
    "blr_matrix_clone": (_I, [_P, ctypes.POINTER(_P), _P]),
    "blr_qr": (_I, [_P, ctypes.POINTER(Opts), ctypes.POINTER(_P), _P]),
    "blr_qr_batched": (_I, [ctypes.POINTER(_P), _I, ctypes.POINTER(Opts), ctypes.POINTER(_P), _P]),
    "blr_batch_plan_create": (_I, [ctypes.POINTER(_P), _I, ctypes.POINTER(Opts), ctypes.POINTER(_P), _P]),
    "blr_batch_plan_launch": (_I, [_P, _P]),
    "blr_batch_plan_finish": (_I, [_P, _P]),
    "blr_batch_plan_factor": (_P, [_P, _I]),
    "blr_batch_plan_destroy": (None, [_P]),
    "blr_apply_qt": (_I, [_P, _P, _I, _I, _I, _P]),
    "blr_apply_qt_noalloc": (_I, [_P, _P, _I, _I, _I, _P]),
    "blr_lstsq": (_I, [_P, _P, _P, _I, _P, _I, _I, _I, _P]),
    "blr_matmul": (_I, [_P, _P, _I, _P, _I, _I, _P]),
    "blr_apply_r": (_I, [_P, _P, _I, _P, _I, _I, _P]),
    "blr_solve_r": (_I, [_P, _P, _I, _P, _I, _I, _I, _P]),
    "blr_lstsq_backward": (_I, [_P, _P, _P, _I, _P, _I, _P, _I, _I, _P, _I, _P, _P]),
    "blr_factor_export_t": (_I, [_P, _DP, _P]),
    "blr_stats": (_I, [_P, _I, ctypes.POINTER(Stats)]),
    "blr_trace_export": (_I, [_P, ctypes.POINTER(TraceEvent), _I, ctypes.POINTER(ctypes.c_longlong)]),
    "blr_densify": (_I, [_P, _I, _I, _P, _I, _P]),
    "blr_destroy_matrix": (None, [_P]),
    "blr_destroy_factor": (None, [_P]),
    "blr_dag_selfcheck": (_I, [_I, _I, ctypes.c_uint]),
    "blr_batch_selfcheck": (_I, [_IP, _IP, _I, ctypes.c_uint]),
    "blr_dag_task": (_I, [_I, _I, _I, _IP, _IP, _I]),
    "blr_tc_gemm_selftest": (_I, [_P, _I, _P, _I, _P, _I, _I, _I, _I, _P]),
    "blr_tc_update_bench": (_I, [_I, _I, _I, _I, _DP, _DP]),
}
EXPORTED = tuple(_SIGS)


def lib() -> ctypes.CDLL:
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2208_06194_gb300.build.build()")
        handle = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        _lib = handle
    return _lib


def blr_last_error() -> str:
    return lib().blr_last_error().decode()


def _check(rc: int) -> None:
    if rc != 0:
        raise BLRError(rc, blr_last_error())


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return ctypes.c_void_p(int(stream))


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_DP)


def blr_opts_default(**kw) -> Opts:
    o = Opts()
    lib().blr_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise AttributeError(k)
        setattr(o, k, v)
    return o


def fortran_empty(rows: int, cols: int, device="cuda"):
    import torch
    return torch.empty((cols, rows), dtype=torch.float64, device=device).t()


def to_fortran(a):
    """Column-major float64 copy of a 2-D tensor or array on the GPU."""
    import torch
    t = torch.as_tensor(a, dtype=torch.float64)
    if t.dim() == 1:
        t = t[:, None]
    out = fortran_empty(t.shape[0], t.shape[1], device="cuda")
    out.copy_(t)
    return out


def _ld(t) -> int:
    if t.dtype.is_floating_point is False or t.element_size() != 8:
        raise TypeError("float64 tensor required")
    if t.stride(0) != 1:
        raise ValueError("column-major tensor required (stride (1, ld))")
    return max(t.stride(1), t.shape[0]) if t.shape[1] > 1 else t.shape[0]


class Matrix:
    """Owning wrapper of a blr_matrix handle."""

    def __init__(self, handle: ctypes.c_void_p, m: int, n: int, b: int):
        self.handle, self.m, self.n, self.b = handle, m, n, b
        self.p, self.q = m // b, n // b

    def destroy(self):
        if self.handle:
            lib().blr_destroy_matrix(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


class Factor:
    """Owning wrapper of a blr_factor handle."""

    def __init__(self, handle: ctypes.c_void_p, m: int, n: int, b: int):
        self.handle, self.m, self.n, self.b = handle, m, n, b
        self.p, self.q = m // b, n // b

    def destroy(self):
        if self.handle:
            lib().blr_destroy_factor(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def blr_compress_kernel(x: np.ndarray, y: np.ndarray, kernel: str | int, opts: Opts,
                        col_scale: np.ndarray | None = None, stream=None) -> Matrix:
    """x: (dim, m), y: (dim, n) host point arrays (already ordered)."""
    kid = KERNEL_IDS[kernel] if isinstance(kernel, str) else int(kernel)
    dim, m = x.shape
    n = y.shape[1]
    xc = np.ascontiguousarray(np.asarray(x, dtype=np.float64).T)   # column i = point i
    yc = np.ascontiguousarray(np.asarray(y, dtype=np.float64).T)
    sc = None if col_scale is None else np.ascontiguousarray(col_scale, dtype=np.float64)
    h = ctypes.c_void_p()
    _check(lib().blr_compress_kernel(_dptr(xc), _dptr(yc), dim, m, n, kid,
                                     None if sc is None else _dptr(sc), ctypes.byref(opts),
                                     ctypes.byref(h), _stream(stream)))
    return Matrix(h, m, n, opts.b)


def blr_compress_dense(a, opts: Opts, stream=None) -> Matrix:
    """a: column-major float64 CUDA tensor (m, n)."""
    m, n = a.shape
    h = ctypes.c_void_p()
    _check(lib().blr_compress_dense(ctypes.c_void_p(a.data_ptr()), _ld(a), m, n, ctypes.byref(opts),
                                    ctypes.byref(h), _stream(stream)))
    return Matrix(h, m, n, opts.b)


def blr_matrix_import(m: int, n: int, b: int, ranks: np.ndarray, tiles: np.ndarray, stream=None) -> Matrix:
    """ranks: (p*q,) int32 in (j*p + i) order; tiles: (p*q*b*b,) float64 (library layout)."""
    r = np.ascontiguousarray(ranks, dtype=np.int32)
    t = np.ascontiguousarray(tiles, dtype=np.float64)
    h = ctypes.c_void_p()
    _check(lib().blr_matrix_import(m, n, b, r.ctypes.data_as(_IP), _dptr(t), ctypes.byref(h),
                                   _stream(stream)))
    return Matrix(h, m, n, b)


def blr_matrix_import_device(m: int, n: int, b: int, ranks: np.ndarray, tiles, stream=None) -> Matrix:
    """As blr_matrix_import with tiles a float64 CUDA tensor of p*q*b*b elements."""
    r = np.ascontiguousarray(ranks, dtype=np.int32)
    if tiles.dtype != __import__("torch").float64 or not tiles.is_cuda or not tiles.is_contiguous():
        raise TypeError("tiles must be a contiguous float64 CUDA tensor")
    if tiles.numel() != (m // b) * (n // b) * b * b:
        raise ValueError("tiles has the wrong size")
    h = ctypes.c_void_p()
    _check(lib().blr_matrix_import_device(m, n, b, r.ctypes.data_as(_IP), ctypes.c_void_p(tiles.data_ptr()),
                                          ctypes.byref(h), _stream(stream)))
    return Matrix(h, m, n, b)


def blr_matrix_export(obj, stream=None) -> tuple[np.ndarray, np.ndarray]:
    """(ranks (p*q,), tiles (p*q*b*b,)) of a Matrix or the in-place storage of a Factor."""
    p, q, b = obj.p, obj.q, obj.b
    ranks = np.empty(p * q, dtype=np.int32)
    tiles = np.empty(p * q * b * b, dtype=np.float64)
    _check(lib().blr_matrix_export(obj.handle, 1 if isinstance(obj, Factor) else 0,
                                   ranks.ctypes.data_as(_IP), _dptr(tiles), _stream(stream)))
    return ranks, tiles


def blr_matrix_clone(a: Matrix, stream=None) -> Matrix:
    h = ctypes.c_void_p()
    _check(lib().blr_matrix_clone(a.handle, ctypes.byref(h), _stream(stream)))
    return Matrix(h, a.m, a.n, a.b)


def blr_qr(a: Matrix, opts: Opts, stream=None) -> Factor:
    """Consumes a (its storage becomes the factor's)."""
    h = ctypes.c_void_p()
    handle, a.handle = a.handle, None
    _check(lib().blr_qr(handle, ctypes.byref(opts), ctypes.byref(h), _stream(stream)))
    return Factor(h, a.m, a.n, a.b)


def blr_qr_batched(mats: list, opts: Opts, stream=None) -> list:
    """One persistent launch for all matrices; consumes them (like blr_qr)."""
    n = len(mats)
    arr = (_P * n)(*[m.handle for m in mats])
    out = (_P * n)()
    for m in mats:
        m.handle = None
    _check(lib().blr_qr_batched(arr, n, ctypes.byref(opts), out, _stream(stream)))
    return [Factor(ctypes.c_void_p(out[i]), mats[i].m, mats[i].n, mats[i].b) for i in range(n)]


class BatchPlan:
    """A launch plan (blr_batch_plan_*): launch() is capturable in a CUDA
    graph; the matrices must outlive the plan and stay unchanged."""

    def __init__(self, mats: list, opts: Opts, stream=None):
        n = len(mats)
        arr = (_P * n)(*[m.handle for m in mats])
        h = ctypes.c_void_p()
        _check(lib().blr_batch_plan_create(arr, n, ctypes.byref(opts), ctypes.byref(h), _stream(stream)))
        self.handle, self.mats = h, list(mats)

    def launch(self, stream=None):
        _check(lib().blr_batch_plan_launch(self.handle, _stream(stream)))

    def finish(self, stream=None):
        _check(lib().blr_batch_plan_finish(self.handle, _stream(stream)))

    def factor(self, i: int) -> "Factor":
        """A non-owning view of the plan's factor i."""
        h = lib().blr_batch_plan_factor(self.handle, i)
        m = self.mats[i]
        f = Factor(ctypes.c_void_p(h), m.m, m.n, m.b)
        f.destroy = lambda: None          # owned by the plan
        f.__del__ = lambda: None
        return f

    def destroy(self):
        if self.handle:
            lib().blr_batch_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def blr_apply_qt(f: Factor, bmat, trans: int = 0, stream=None) -> None:
    """In place: trans=0 -> Q^T B, trans=1 -> Q B (B column-major m x nrhs)."""
    _check(lib().blr_apply_qt(f.handle, ctypes.c_void_p(bmat.data_ptr()), _ld(bmat), bmat.shape[1],
                              trans, _stream(stream)))


def blr_apply_qt_noalloc(f: Factor, bmat, trans: int = 0, stream=None) -> None:
    """blr_apply_qt without device allocation (static library scratch; see
    include/blr.h for the size limit and the serialisation rule)."""
    _check(lib().blr_apply_qt_noalloc(f.handle, ctypes.c_void_p(bmat.data_ptr()), _ld(bmat), bmat.shape[1],
                                      trans, _stream(stream)))


def blr_lstsq(f: Factor, bmat, a_orig: Matrix | None = None, refine_steps: int = 0, x=None, stream=None):
    nrhs = bmat.shape[1]
    if x is None:
        x = fortran_empty(f.n, nrhs)
    _check(lib().blr_lstsq(f.handle, None if a_orig is None else a_orig.handle,
                           ctypes.c_void_p(bmat.data_ptr()), _ld(bmat), ctypes.c_void_p(x.data_ptr()),
                           _ld(x), nrhs, refine_steps, _stream(stream)))
    return x


def blr_matmul(a: Matrix, x, stream=None):
    y = fortran_empty(a.m, x.shape[1])
    _check(lib().blr_matmul(a.handle, ctypes.c_void_p(x.data_ptr()), _ld(x), ctypes.c_void_p(y.data_ptr()),
                            _ld(y), x.shape[1], _stream(stream)))
    return y


def blr_apply_r(f: Factor, x, stream=None):
    y = fortran_empty(f.n, x.shape[1])
    _check(lib().blr_apply_r(f.handle, ctypes.c_void_p(x.data_ptr()), _ld(x), ctypes.c_void_p(y.data_ptr()),
                             _ld(y), x.shape[1], _stream(stream)))
    return y


def blr_solve_r(f: Factor, c, trans: int = 0, stream=None):
    """X = R^{-1} C (trans=0) or R^{-T} C (trans=1); C column-major n x nrhs."""
    x = fortran_empty(f.n, c.shape[1])
    _check(lib().blr_solve_r(f.handle, ctypes.c_void_p(c.data_ptr()), _ld(c), ctypes.c_void_p(x.data_ptr()),
                             _ld(x), c.shape[1], trans, _stream(stream)))
    return x


def blr_lstsq_backward(f: Factor, a_orig: Matrix, bmat, x, xbar, stream=None):
    """(dL/dB (m x nrhs), dL/dtiles (p*q*b*b)) for x = argmin ||A~ x - B||."""
    import torch
    nrhs = bmat.shape[1]
    bbar = fortran_empty(f.m, nrhs)
    grad = torch.empty(a_orig.p * a_orig.q * a_orig.b * a_orig.b, dtype=torch.float64, device=bmat.device)
    _check(lib().blr_lstsq_backward(f.handle, a_orig.handle, ctypes.c_void_p(bmat.data_ptr()), _ld(bmat),
                                    ctypes.c_void_p(x.data_ptr()), _ld(x), ctypes.c_void_p(xbar.data_ptr()),
                                    _ld(xbar), nrhs, ctypes.c_void_p(bbar.data_ptr()), _ld(bbar),
                                    ctypes.c_void_p(grad.data_ptr()), _stream(stream)))
    return bbar, grad


def blr_factor_export_t(f: Factor, stream=None) -> np.ndarray:
    nt = sum(f.p - k for k in range(f.q))
    out = np.empty(nt * 32 * f.b, dtype=np.float64)
    _check(lib().blr_factor_export_t(f.handle, _dptr(out), _stream(stream)))
    return out


def blr_stats(obj) -> dict:
    s = Stats()
    _check(lib().blr_stats(obj.handle, 1 if isinstance(obj, Factor) else 0, ctypes.byref(s)))
    d = {k: getattr(s, k) for k, _ in Stats._fields_}
    d["flops"] = list(s.flops)
    d["tasks"] = list(s.tasks)
    d["task_seconds"] = list(s.task_seconds)
    for k in ("tpmqrt_kind", "tpmqrt_kind_seconds", "tpmqrt_kind_flops"):
        d[k] = list(getattr(s, k))
    return d


TASK_NAMES = ("GEQRT", "LARFB", "TSQRT", "TPMQRT")


def blr_trace_export(f: Factor) -> tuple[list[dict], int]:
    """(events, tasks run) of a factorization made with opts.trace > 0; each
    event a dict with the fields of blr_trace_event."""
    total = ctypes.c_longlong(0)
    n = lib().blr_trace_export(f.handle, None, 0, ctypes.byref(total))
    if n < 0:
        raise BLRError(1, blr_last_error())
    cap = int(total.value)
    buf = (TraceEvent * max(cap, 1))()
    n = lib().blr_trace_export(f.handle, buf, cap, ctypes.byref(total))
    if n < 0:
        raise BLRError(1, blr_last_error())
    return [{k: getattr(buf[e], k) for k, _ in TraceEvent._fields_ if k != "reserved"} for e in range(n)], \
        int(total.value)


def chrome_trace(events: list[dict]) -> dict:
    """The task trace in the Chrome trace-event format (one row per
    scheduler CTA, times in microseconds from the first task's start)."""
    t0 = min((e["t_start_ns"] for e in events), default=0)
    out = []
    for e in events:
        name = f"{TASK_NAMES[e['type']]}({e['i']},{e['j']},{e['k']})"
        out.append({"name": name, "cat": TASK_NAMES[e["type"]], "ph": "X", "pid": e["matrix"], "tid": e["cta"],
                    "ts": (e["t_start_ns"] - t0) / 1e3, "dur": (e["t_end_ns"] - e["t_start_ns"]) / 1e3,
                    "args": {"sm": e["sm"]}})
    return {"traceEvents": out, "displayTimeUnit": "ms"}


def blr_densify(obj, which: int = 0, stream=None):
    """Dense column-major CUDA tensor of a Matrix (which 0: A~) or of a
    Factor (0: in-place storage, 1: R (n x n), 2: reflector tails Y~)."""
    rows = obj.n if which == 1 else obj.m
    cols = obj.n
    out = fortran_empty(rows, cols)
    _check(lib().blr_densify(obj.handle, 1 if isinstance(obj, Factor) else 0, which, ctypes.c_void_p(out.data_ptr()),
                             rows, _stream(stream)))
    return out


def blr_batch_selfcheck(ps, qs, seed: int = 0) -> int:
    """Host-only check of a batch's task numbering and protocol (0 = pass)."""
    p = np.ascontiguousarray(ps, dtype=np.int32)
    q = np.ascontiguousarray(qs, dtype=np.int32)
    return lib().blr_batch_selfcheck(p.ctypes.data_as(_IP), q.ctypes.data_as(_IP), len(p), seed)


def blr_dag_task(p: int, q: int, task_id: int) -> tuple[tuple[int, int, int, int], list[int]]:
    """(type, i, j, k) of a scheduler task id and the ids it releases (host only)."""
    task = (ctypes.c_int * 4)()
    succ = (ctypes.c_int * (q + 1))()
    n = lib().blr_dag_task(p, q, task_id, task, succ, q + 1)
    if n < 0:
        raise BLRError(1, blr_last_error())
    return tuple(task), list(succ[:n])


def blr_dag_selfcheck(p: int, q: int, seed: int = 0) -> int:
    """Host-only check of the scheduler's DAG formulas (0 = pass)."""
    return lib().blr_dag_selfcheck(p, q, seed)


def blr_tc_gemm_selftest(a, bm, stream=None):
    """D = A B through the tensor-core building block (3xTF32, FP32
    accumulation); a, bm are column-major float64 CUDA tensors."""
    m, k = a.shape
    k2, n = bm.shape
    if k2 != k:
        raise ValueError("inner dimensions differ")
    d = fortran_empty(m, n, device=a.device)
    _check(lib().blr_tc_gemm_selftest(a.data_ptr(), a.stride(1), bm.data_ptr(), bm.stride(1), d.data_ptr(),
                                      d.stride(1), m, n, k, _stream(stream)))
    return d


def blr_tc_update_bench(b: int = 512, ctas: int | None = None, reps: int = 8, variant: int = 0) -> dict:
    """Diagnostic timing of the dense prepared update (ms per update per CTA,
    aggregate algorithmic TFLOP/s); ctas defaults to the SM count."""
    if ctas is None:
        import torch
        ctas = torch.cuda.get_device_properties(0).multi_processor_count
    ms, tf = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(lib().blr_tc_update_bench(b, ctas, reps, variant, ctypes.byref(ms), ctypes.byref(tf)))
    return {"b": b, "ctas": ctas, "reps": reps, "variant": variant, "ms_per_update": ms.value,
            "aggregate_tflops": tf.value}
