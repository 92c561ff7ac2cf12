"""Python binding of libesom (ctypes).

The functions named like the C ABI (``esom_create``, ``esom_project``, ...)
only marshal arguments: pointers are passed as integers (for example
``tensor.data_ptr()``) and each returns the C status code.  ``Projector`` is
a convenience wrapper for torch CUDA tensors that checks shapes, dtypes and
devices and raises ``EsomError`` on a non-OK status.  Every computation runs
in the CUDA library; there is no CPU path, and loading fails loudly when the
library has not been built.
"""
from __future__ import annotations

import ctypes
import os
import re

from . import build as _build

ESOM_OK = 0
ESOM_EINVAL = -1
ESOM_ENOMEM = -2
ESOM_EALIGN = -3
ESOM_ENOLANDMARKS = -4
ESOM_ECUDA = -5
ESOM_EUNSUPPORTED = -6
ESOM_EDEVICE = -7
ESOM_SCREEN_FP32 = 0
ESOM_SCREEN_TF32 = 1
ESOM_SCREEN_BF16 = 2
ESOM_SCREEN_AUTO = 3
ESOM_PLAN_FUSED = 0
ESOM_PLAN_SPLIT = 1
ESOM_PLAN_TF32 = 2
ESOM_PLAN_BF16 = 3
ESOM_KNN_BASE = 1
ESOM_KNN_BITONIC = 2
ESOM_PROJ_TABLE = 0
ESOM_PROJ_REGISTERS = 1
PLAN_NAMES = {ESOM_PLAN_FUSED: "fused", ESOM_PLAN_SPLIT: "split", ESOM_PLAN_TF32: "tf32",
              ESOM_PLAN_BF16: "bf16"}

HEADER = os.path.join(_build.INCLUDE, "esom.h")


class EsomError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{status_string(status)}: {message}")
        self.status = status


class _Stats(ctypes.Structure):
    _fields_ = [("points", ctypes.c_uint64), ("rescans", ctypes.c_uint64),
                ("refines", ctypes.c_uint64), ("launches", ctypes.c_uint64)]


ESOM_KERNEL_KINDS = 8
KERNEL_NAMES = ["order", "tc_knn", "rerank_project", "rerank", "rescan", "project", "refine",
                "fused"]


class _KernelTimes(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_uint64 * ESOM_KERNEL_KINDS),
                ("ms", ctypes.c_double * ESOM_KERNEL_KINDS)]


class BatchItem(ctypes.Structure):
    _fields_ = [("landmarks", ctypes.c_void_p), ("points", ctypes.c_void_p),
                ("n", ctypes.c_int64), ("out", ctypes.c_void_p),
                ("boost", ctypes.c_float), ("adjust", ctypes.c_float)]


class SessionDesc(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("L", ctypes.c_int), ("k", ctypes.c_int),
                ("n", ctypes.c_int64), ("boost", ctypes.c_float), ("adjust", ctypes.c_float),
                ("alpha", ctypes.c_float), ("sigma", ctypes.c_float),
                ("minibatch", ctypes.c_int), ("seed", ctypes.c_uint64)]


class FrameDone(ctypes.Structure):
    _fields_ = [("session", ctypes.c_int), ("frame", ctypes.c_uint64),
                ("arrival", ctypes.c_double), ("completion", ctypes.c_double)]


class _Config(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int) for n in
                ("d", "L", "k", "kc", "threads_per_block", "blocks_per_sm", "num_sms",
                 "landmark_chunk", "landmark_chunks", "shared_bytes", "screening", "plan")]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Loads libesom.so (building it first only if asked)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        if not build_if_missing:
            raise RuntimeError(
                f"libesom.so is not built ({_build.LIB}); run "
                "`python -c 'import __graft_entry__ as g; g.build()'`")
        _build.build()
    lib = ctypes.CDLL(_build.LIB)
    P, I, I64, F = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_float
    sigs = {
        "esom_create": ([I, I, I, ctypes.POINTER(P)], I),
        "esom_set_landmarks": ([P, P, P, P], I),
        "esom_landmark_version": ([P], ctypes.c_uint64),
        "esom_project": ([P, P, I64, P, F, F, P], I),
        "esom_knn": ([P, P, I64, P, P, P], I),
        "esom_knn_variant": ([P, I, P, I64, P, P, P], I),
        "esom_project_knn": ([P, I, P, I64, P, P, P, F, F, P], I),
        "esom_project_host": ([P, P, I64, P, F, F, P], I),
        "esom_device_status": ([P, P], I),
        "esom_set_landmark_chunk": ([P, I], I),
        "esom_get_config": ([P, ctypes.POINTER(_Config)], I),
        "esom_project_noalloc": ([P, I64, P, P, I, I, I, P, F, F, P], I),
        "esom_get_stats": ([P, P, ctypes.POINTER(_Stats), I], I),
        "esom_set_timing": ([P, I], I),
        "esom_get_timing": ([P, P, ctypes.POINTER(_KernelTimes), I], I),
        "esom_set_screening": ([P, I, P], I),
        "esom_set_split": ([P, I], I),
        "esom_set_centering": ([P, I], I),
        "esom_tune": ([P, P, I64, P, F, F, P, ctypes.POINTER(I)], I),
        "esom_batch_create": ([ctypes.POINTER(BatchItem), I, I, ctypes.POINTER(P)], I),
        "esom_batch_run": ([P, P], I),
        "esom_batch_run_graph": ([P, P], I),
        "esom_batch_plan": ([P], ctypes.c_char_p),
        "esom_batch_destroy": ([P], I),
        "esom_som_update": ([P, P, I, I, P, P, I, I64, F, F, P], I),
        "esom_server_create": ([ctypes.c_uint64, I, ctypes.POINTER(P)], I),
        "esom_server_add_session": ([P, ctypes.POINTER(SessionDesc), P, P, P,
                                     ctypes.POINTER(I)], I),
        "esom_server_now": ([P], ctypes.c_double),
        "esom_server_set_coalescing": ([P, I], I),
        "esom_server_set_screening": ([P, I], I),
        "esom_server_submit": ([P, I, ctypes.c_double], I),
        "esom_server_poll": ([P, I, ctypes.POINTER(FrameDone), I, ctypes.POINTER(I)], I),
        "esom_server_session_output": ([P, I, ctypes.POINTER(P), ctypes.POINTER(ctypes.c_uint64)], I),
        "esom_server_memory": ([P, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)], I),
        "esom_server_destroy": ([P], I),
        "esom_test_stall": ([P, I64], I),
        "esom_selftest_drcp": ([P, I64, P, P, P], I),
        "esom_selftest_tc_products": ([P, P, I64, P, P], I),
        "esom_destroy": ([P], I),
        "esom_last_error": ([], ctypes.c_char_p),
        "esom_status_string": ([I], ctypes.c_char_p),
    }
    for name, (args, res) in sigs.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def declared_functions() -> list[str]:
    """Names of the functions include/esom.h declares."""
    with open(HEADER) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(esom_[a-z_]+)\s*\(", text)))


# --- the C ABI, one to one -------------------------------------------------

def esom_create(d: int, L: int, k: int):
    """Returns (status, handle)."""
    h = ctypes.c_void_p()
    st = load().esom_create(d, L, k, ctypes.byref(h))
    return st, h.value


def esom_set_landmarks(h, hi_ptr: int, lo_ptr: int, stream: int = 0) -> int:
    return load().esom_set_landmarks(h, hi_ptr, lo_ptr, stream)


def esom_landmark_version(h) -> int:
    return int(load().esom_landmark_version(h))


def esom_project(h, points_ptr: int, n: int, out_ptr: int, boost: float, adjust: float,
                 stream: int = 0) -> int:
    return load().esom_project(h, points_ptr, n, out_ptr, boost, adjust, stream)


def esom_knn(h, points_ptr: int, n: int, idx_ptr: int, dist2_ptr: int | None,
             stream: int = 0) -> int:
    return load().esom_knn(h, points_ptr, n, idx_ptr, dist2_ptr, stream)


def esom_knn_variant(h, variant: int, points_ptr: int, n: int, idx_ptr: int,
                     dist2_ptr: int | None, stream: int = 0) -> int:
    """The k-NN by one of the paper's alternative kernels (ablation)."""
    return load().esom_knn_variant(h, variant, points_ptr, n, idx_ptr, dist2_ptr, stream)


def esom_project_knn(h, variant: int, points_ptr: int, n: int, idx_ptr: int, dist2_ptr: int,
                     out_ptr: int, boost: float, adjust: float, stream: int = 0) -> int:
    """Steps 2-4 from given neighbours, by the library's or the paper's kernel."""
    return load().esom_project_knn(h, variant, points_ptr, n, idx_ptr, dist2_ptr, out_ptr,
                                   boost, adjust, stream)


def esom_project_host(h, points_ptr: int, n: int, out_ptr: int, boost: float, adjust: float,
                      stream: int = 0) -> int:
    return load().esom_project_host(h, points_ptr, n, out_ptr, boost, adjust, stream)


def esom_device_status(h, stream: int = 0) -> int:
    return load().esom_device_status(h, stream)


def esom_set_landmark_chunk(h, chunk: int) -> int:
    return load().esom_set_landmark_chunk(h, chunk)


def esom_get_config(h):
    """Returns (status, dict)."""
    cfg = _Config()
    st = load().esom_get_config(h, ctypes.byref(cfg))
    return st, {name: getattr(cfg, name) for name, _ in _Config._fields_}


def esom_get_stats(h, stream: int = 0, reset: bool = False):
    """Returns (status, {"points": ..., "rescans": ...})."""
    st_ = _Stats()
    st = load().esom_get_stats(h, stream, ctypes.byref(st_), int(reset))
    return st, {"points": int(st_.points), "rescans": int(st_.rescans),
                "refines": int(st_.refines), "launches": int(st_.launches)}


def esom_set_timing(h, on: bool) -> int:
    return load().esom_set_timing(h, int(on))


def esom_get_timing(h, stream: int = 0, reset: bool = False):
    """Returns (status, {kernel kind: (launches, total ms)})."""
    t = _KernelTimes()
    st = load().esom_get_timing(h, stream, ctypes.byref(t), int(reset))
    return st, {name: (int(t.launches[i]), float(t.ms[i]))
                for i, name in enumerate(KERNEL_NAMES)}


def esom_set_screening(h, mode: int, stream: int = 0) -> int:
    """ESOM_SCREEN_FP32 (0), ESOM_SCREEN_TF32 (1) or ESOM_SCREEN_BF16 (2)."""
    return load().esom_set_screening(h, mode, stream)


def esom_set_split(h, on: bool) -> int:
    """Two kernels (k-NN, then projection from neighbours) instead of one."""
    return load().esom_set_split(h, int(on))


def esom_set_centering(h, on: bool) -> int:
    """Centre the data on the landmarks' rounded mean (next set_landmarks on)."""
    return load().esom_set_centering(h, int(on))


def esom_tune(h, points_ptr: int, n: int, out_ptr: int, boost: float, adjust: float,
              stream: int = 0):
    """Returns (status, plan): ESOM_PLAN_FUSED / _SPLIT / _TF32 / _BF16, now set."""
    plan = ctypes.c_int(-1)
    st = load().esom_tune(h, points_ptr, n, out_ptr, boost, adjust, stream, ctypes.byref(plan))
    return st, plan.value


def esom_project_noalloc(points_ptr: int, n: int, hi_ptr: int, lo_ptr: int, d: int, L: int,
                         k: int, out_ptr: int, boost: float, adjust: float,
                         stream: int = 0) -> int:
    """Projection with no device allocation (scratch in a fixed device array)."""
    return load().esom_project_noalloc(points_ptr, n, hi_ptr, lo_ptr, d, L, k, out_ptr, boost,
                                       adjust, stream)


def esom_test_stall(h, limit_ns: int) -> int:
    """Arms the next fused-kernel launch to run out a bounded wait (tests)."""
    return load().esom_test_stall(h, limit_ns)


def esom_selftest_drcp(x_ptr: int, n: int, rcp_ptr: int, div_ptr: int, stream: int = 0) -> int:
    """The solve's FP64 reciprocal and CUDA's 1.0 / x of n doubles (tests)."""
    return load().esom_selftest_drcp(x_ptr, n, rcp_ptr, div_ptr, stream)


def esom_selftest_tc_products(h, points_ptr: int, n: int, T_ptr: int, stream: int = 0) -> int:
    """Raw tensor-core dot products x . l of the screening (tests)."""
    return load().esom_selftest_tc_products(h, points_ptr, n, T_ptr, stream)


def esom_batch_create(items, autotune: bool = False):
    """items: sequence of BatchItem.  Returns (status, batch)."""
    arr = (BatchItem * len(items))(*items)
    b = ctypes.c_void_p()
    st = load().esom_batch_create(arr, len(items), int(autotune), ctypes.byref(b))
    return st, b.value


def esom_batch_run(b, stream: int = 0) -> int:
    return load().esom_batch_run(b, stream)


def esom_batch_run_graph(b, stream: int = 0) -> int:
    return load().esom_batch_run_graph(b, stream)


def esom_batch_plan(b) -> str:
    return load().esom_batch_plan(b).decode()


def esom_batch_destroy(b) -> int:
    return load().esom_batch_destroy(b)


def esom_som_update(hi_ptr: int, lo_ptr: int, d: int, L: int, batch_ptr: int, bmu_ptr: int,
                    bmu_stride: int, b: int, alpha: float, sigma: float, stream: int = 0) -> int:
    return load().esom_som_update(hi_ptr, lo_ptr, d, L, batch_ptr, bmu_ptr, bmu_stride, b, alpha,
                                  sigma, stream)


def esom_server_create(budget_bytes: int, max_inflight: int):
    s = ctypes.c_void_p()
    st = load().esom_server_create(int(budget_bytes), max_inflight, ctypes.byref(s))
    return st, s.value


def esom_server_add_session(s, desc: "SessionDesc", points_ptr: int, hi_ptr: int, lo_ptr: int):
    sid = ctypes.c_int(-1)
    st = load().esom_server_add_session(s, ctypes.byref(desc), points_ptr, hi_ptr, lo_ptr,
                                        ctypes.byref(sid))
    return st, sid.value


def esom_server_now(s) -> float:
    return float(load().esom_server_now(s))


def esom_server_set_coalescing(s, on: bool) -> int:
    return load().esom_server_set_coalescing(s, int(on))


def esom_server_set_screening(s, mode: int) -> int:
    return load().esom_server_set_screening(s, mode)


def esom_server_submit(s, session: int, arrival: float) -> int:
    return load().esom_server_submit(s, session, arrival)


def esom_server_poll(s, wait_all: bool = False, max_records: int = 1024):
    """Returns (status, [FrameDone, ...])."""
    buf = (FrameDone * max_records)()
    cnt = ctypes.c_int(0)
    st = load().esom_server_poll(s, int(wait_all), buf, max_records, ctypes.byref(cnt))
    return st, [buf[i] for i in range(cnt.value)]


def esom_server_session_output(s, session: int):
    """Returns (status, device pointer, frames completed)."""
    p = ctypes.c_void_p()
    f = ctypes.c_uint64(0)
    st = load().esom_server_session_output(s, session, ctypes.byref(p), ctypes.byref(f))
    return st, p.value, int(f.value)


def esom_server_memory(s):
    u, b = ctypes.c_uint64(0), ctypes.c_uint64(0)
    st = load().esom_server_memory(s, ctypes.byref(u), ctypes.byref(b))
    return st, int(u.value), int(b.value)


def esom_server_destroy(s) -> int:
    return load().esom_server_destroy(s)


def esom_destroy(h) -> int:
    return load().esom_destroy(h)


def esom_last_error() -> str:
    return load().esom_last_error().decode()


def status_string(status: int) -> str:
    return load().esom_status_string(status).decode()


def check(status: int) -> None:
    if status != ESOM_OK:
        raise EsomError(status, esom_last_error())


# --- torch convenience wrapper ----------------------------------------------

class Projector:
    """A handle for (d, L, k) bound to the current CUDA device."""

    def __init__(self, d: int, L: int, k: int):
        st, h = esom_create(d, L, k)
        check(st)
        self.h, self.d, self.L, self.k = h, d, L, k

    def close(self):
        if self.h:
            esom_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @staticmethod
    def _stream():
        import torch
        return torch.cuda.current_stream().cuda_stream

    def _points(self, X):
        import torch
        if not (X.is_cuda and X.dtype == torch.float32 and X.dim() == 2
                and X.shape[1] == self.d and X.is_contiguous()):
            raise ValueError(f"points must be a contiguous CUDA float32 tensor n x {self.d}")
        return X

    def set_landmarks(self, hi, lo):
        import torch
        if hi.shape != (self.L, self.d) or lo.shape != (self.L, 2):
            raise ValueError("landmark shapes must be L x d and L x 2")
        if hi.dtype != torch.float32 or lo.dtype != torch.float32:
            raise ValueError("landmarks must be float32")
        hi, lo = hi.contiguous(), lo.contiguous()
        check(esom_set_landmarks(self.h, hi.data_ptr(), lo.data_ptr(), self._stream()))
        self._keep = (hi, lo)  # alive until the asynchronous copy has run

    def project(self, X, boost: float = 1.0, adjust: float = 1.0, out=None):
        import torch
        X = self._points(X)
        if out is None:
            out = torch.empty((X.shape[0], 2), dtype=torch.float32, device=X.device)
        check(esom_project(self.h, X.data_ptr(), X.shape[0], out.data_ptr(), boost, adjust,
                           self._stream()))
        return out

    def knn(self, X, with_dist: bool = True):
        import torch
        X = self._points(X)
        idx = torch.empty((X.shape[0], self.k), dtype=torch.int32, device=X.device)
        d2 = (torch.empty((X.shape[0], self.k), dtype=torch.float32, device=X.device)
              if with_dist else None)
        check(esom_knn(self.h, X.data_ptr(), X.shape[0], idx.data_ptr(),
                       d2.data_ptr() if d2 is not None else None, self._stream()))
        return idx, d2

    def knn_variant(self, X, variant: int, with_dist: bool = True):
        """esom_knn by ESOM_KNN_BASE or ESOM_KNN_BITONIC (same results)."""
        import torch
        X = self._points(X)
        idx = torch.empty((X.shape[0], self.k), dtype=torch.int32, device=X.device)
        d2 = (torch.empty((X.shape[0], self.k), dtype=torch.float32, device=X.device)
              if with_dist else None)
        check(esom_knn_variant(self.h, variant, X.data_ptr(), X.shape[0], idx.data_ptr(),
                               d2.data_ptr() if d2 is not None else None, self._stream()))
        return idx, d2

    def project_knn(self, X, idx, d2, variant: int = ESOM_PROJ_TABLE, boost: float = 1.0,
                    adjust: float = 1.0, out=None):
        """Steps 2-4 from the neighbours idx / d2 (n x k, as knn returns)."""
        import torch
        X = self._points(X)
        n = X.shape[0]
        for t, dt in ((idx, torch.int32), (d2, torch.float32)):
            if not (t.is_cuda and t.dtype == dt and t.shape == (n, self.k) and t.is_contiguous()):
                raise ValueError(f"neighbours must be contiguous CUDA {dt} tensors n x {self.k}")
        if out is None:
            out = torch.empty((n, 2), dtype=torch.float32, device=X.device)
        check(esom_project_knn(self.h, variant, X.data_ptr(), n, idx.data_ptr(), d2.data_ptr(),
                               out.data_ptr(), boost, adjust, self._stream()))
        return out

    def project_host(self, X_host, boost: float = 1.0, adjust: float = 1.0, out_host=None):
        """Host (CPU) tensors in and out; pinned memory overlaps the copies."""
        import torch
        if X_host.is_cuda or X_host.dtype != torch.float32 or not X_host.is_contiguous():
            raise ValueError("points must be a contiguous CPU float32 tensor")
        if out_host is None:
            out_host = torch.empty((X_host.shape[0], 2), dtype=torch.float32,
                                   pin_memory=X_host.is_pinned())
        check(esom_project_host(self.h, X_host.data_ptr(), X_host.shape[0],
                                out_host.data_ptr(), boost, adjust, self._stream()))
        return out_host

    def device_status(self) -> int:
        return esom_device_status(self.h, self._stream())

    def stats(self, reset: bool = False) -> dict:
        st, out = esom_get_stats(self.h, self._stream(), reset)
        check(st)
        return out

    def set_timing(self, on: bool):
        """Per-kernel CUDA-event timing of this handle's launches (off by default)."""
        check(esom_set_timing(self.h, on))

    def timing(self, reset: bool = False) -> dict:
        """{kernel kind: (launches, total ms)} since the last reset."""
        st, out = esom_get_timing(self.h, self._stream(), reset)
        check(st)
        return out

    def set_screening(self, mode: int):
        """ESOM_SCREEN_FP32 or ESOM_SCREEN_TF32; same results, different speed."""
        check(esom_set_screening(self.h, mode, self._stream()))

    def set_split(self, on: bool):
        check(esom_set_split(self.h, on))

    def set_centering(self, on: bool):
        check(esom_set_centering(self.h, on))

    def set_plan(self, plan: int):
        """ESOM_PLAN_FUSED, _SPLIT, _TF32 or _BF16."""
        self.set_screening({ESOM_PLAN_TF32: ESOM_SCREEN_TF32,
                            ESOM_PLAN_BF16: ESOM_SCREEN_BF16}.get(plan, ESOM_SCREEN_FP32))
        self.set_split(plan == ESOM_PLAN_SPLIT)

    def tune(self, X, boost: float = 1.0, adjust: float = 1.0) -> int:
        """Times the execution plans on X and keeps the fastest; returns it."""
        X = self._points(X)
        import torch
        out = torch.empty((X.shape[0], 2), dtype=torch.float32, device=X.device)
        st, plan = esom_tune(self.h, X.data_ptr(), X.shape[0], out.data_ptr(), boost, adjust,
                             self._stream())
        check(st)
        return plan

    def set_landmark_chunk(self, chunk: int):
        check(esom_set_landmark_chunk(self.h, chunk))

    def config(self) -> dict:
        st, cfg = esom_get_config(self.h)
        check(st)
        return cfg


def device_view(ptr: int, shape, typestr: str = "<f4"):
    """A torch tensor viewing device memory the library owns (no copy)."""
    import torch

    class _View:
        pass

    v = _View()
    v.__cuda_array_interface__ = {"shape": tuple(int(s) for s in shape), "typestr": typestr,
                                  "data": (int(ptr), False), "version": 2, "strides": None}
    return torch.as_tensor(v, device="cuda")


class Server:
    """The frame server (esom_server_*) on the current CUDA device."""

    def __init__(self, budget_bytes: int, max_inflight: int):
        st, s = esom_server_create(budget_bytes, max_inflight)
        check(st)
        self.s = s
        self.n = {}

    def close(self):
        if self.s:
            esom_server_destroy(self.s)
            self.s = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def add_session(self, X, hi, lo, k: int, boost: float = 1.0, adjust: float = 1.0,
                    alpha: float = 0.0, sigma: float = 1.0, minibatch: int = 0,
                    seed: int = 0) -> int:
        """X, hi, lo: contiguous float32 tensors (host or device); copied.
        Raises EsomError (status ESOM_ENOMEM when the budget refuses it)."""
        n, d = X.shape
        desc = SessionDesc(d, hi.shape[0], k, n, boost, adjust, alpha, sigma, minibatch, seed)
        st, sid = esom_server_add_session(self.s, desc, X.data_ptr(), hi.data_ptr(),
                                          lo.data_ptr())
        check(st)
        self.n[sid] = n
        return sid

    def now(self) -> float:
        return esom_server_now(self.s)

    def set_coalescing(self, on: bool):
        check(esom_server_set_coalescing(self.s, on))

    def set_timing(self, on: bool):
        """Per-kernel CUDA-event timing of this handle's launches (off by default)."""
        check(esom_set_timing(self.h, on))

    def timing(self, reset: bool = False) -> dict:
        """{kernel kind: (launches, total ms)} since the last reset."""
        st, out = esom_get_timing(self.h, self._stream(), reset)
        check(st)
        return out

    def set_screening(self, mode: int):
        check(esom_server_set_screening(self.s, mode))

    def submit(self, session: int, arrival: float | None = None):
        check(esom_server_submit(self.s, session, self.now() if arrival is None else arrival))

    def poll(self, wait_all: bool = False, max_records: int = 4096):
        st, recs = esom_server_poll(self.s, wait_all, max_records)
        check(st)
        return [(r.session, int(r.frame), r.arrival, r.completion) for r in recs]

    def output(self, session: int):
        """(copy of the session's latest n x 2 coordinates, frames completed)."""
        st, ptr, frames = esom_server_session_output(self.s, session)
        check(st)
        return device_view(ptr, (self.n[session], 2)).clone(), frames

    def memory(self):
        st, used, budget = esom_server_memory(self.s)
        check(st)
        return used, budget
