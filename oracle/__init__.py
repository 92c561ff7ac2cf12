"""ctypes front end of the FP64 CPU oracle (``esom_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the
benchmark's CPU-baseline leg use it to check and to time against.  The CUDA
library never imports, links or calls it, and this module imports nothing
from the CUDA package.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "esom_oracle.c")
BUILD_DIR = os.path.join(HERE, "_build")
SO = os.path.join(BUILD_DIR, "libesom_oracle.so")
CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-fno-fast-math"]


def compile_source(src: str, out: str) -> str:
    """Compile one oracle source file into a shared object (atomic rename)."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=os.path.dirname(out))
    os.close(fd)
    subprocess.run(["gcc", *CFLAGS, src, "-o", tmp, "-lm"], check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no fast-math) into oracle/_build."""
    if not force and os.path.exists(SO) and os.path.getmtime(SO) >= os.path.getmtime(SRC):
        return SO
    return compile_source(SRC, SO)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


class Oracle:
    """One loaded build of the oracle."""

    def __init__(self, so_path: str):
        lib = ctypes.CDLL(so_path)
        P = ctypes.c_void_p
        lib.esom_oracle_knn.argtypes = [P, ctypes.c_int64, P, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, P, P, ctypes.c_int]
        lib.esom_oracle_knn.restype = ctypes.c_int
        lib.esom_oracle_project.argtypes = [P, ctypes.c_int64, P, P, ctypes.c_int,
                                            ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                            ctypes.c_double, P, P, P, ctypes.c_int]
        lib.esom_oracle_project.restype = ctypes.c_int
        lib.esom_oracle_scores.argtypes = [P, ctypes.c_int, ctypes.c_double, P]
        lib.esom_oracle_scores.restype = None
        lib.esom_oracle_fit.argtypes = [P, P, P, ctypes.c_int, ctypes.c_int, P, P,
                                        ctypes.c_double, P, P, P]
        lib.esom_oracle_fit.restype = None
        lib.esom_oracle_som_step.argtypes = [P, P, ctypes.c_int, ctypes.c_int, P, P,
                                             ctypes.c_int, ctypes.c_double, ctypes.c_double, P]
        lib.esom_oracle_som_step.restype = None
        lib.esom_oracle_default_threads.argtypes = []
        lib.esom_oracle_default_threads.restype = ctypes.c_int
        self.lib = lib

    def default_threads(self) -> int:
        return int(self.lib.esom_oracle_default_threads())

    def knn(self, X, hi, k: int, threads: int = 0):
        """k nearest landmarks: (idx int32 n x k, squared distances float64 n x k)."""
        X, hi = _f32(X), _f32(hi)
        n, d = X.shape
        idx = np.empty((n, k), np.int32)
        d2 = np.empty((n, k), np.float64)
        rc = self.lib.esom_oracle_knn(_ptr(X), n, _ptr(hi), hi.shape[0], d, k, _ptr(idx),
                                      _ptr(d2), threads)
        if rc != 0:
            raise ValueError(f"esom_oracle_knn failed ({rc})")
        return idx, d2

    def scores(self, d2, boost: float):
        """Scores of k neighbours from their ascending squared distances."""
        d2 = np.ascontiguousarray(d2, dtype=np.float64)
        s = np.empty_like(d2)
        self.lib.esom_oracle_scores(_ptr(d2), d2.shape[0], float(boost), _ptr(s))
        return s

    def fit(self, x, hi, lo, idx, s, adjust: float):
        """Pair terms and solve for one point with given neighbours and scores.
        Returns (xy float64[2], diag float64[6], branch int)."""
        x, hi, lo = _f32(x), _f32(hi), _f32(lo)
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        s = np.ascontiguousarray(s, dtype=np.float64)
        out = np.empty(2, np.float64)
        diag = np.empty(6, np.float64)
        br = ctypes.c_int(0)
        self.lib.esom_oracle_fit(_ptr(x), _ptr(hi), _ptr(lo), hi.shape[1], idx.shape[0],
                                 _ptr(idx), _ptr(s), float(adjust), _ptr(out), _ptr(diag),
                                 ctypes.byref(br))
        return out, diag, int(br.value)

    def som_step(self, hi, lo, batch, bmu, alpha: float, sigma: float):
        """One batch SOM step; returns the new L x d landmarks (float64)."""
        hi, lo, batch = _f32(hi), _f32(lo), _f32(batch)
        bmu = np.ascontiguousarray(bmu, dtype=np.int32)
        out = np.empty(hi.shape, np.float64)
        self.lib.esom_oracle_som_step(_ptr(hi), _ptr(lo), hi.shape[1], hi.shape[0], _ptr(batch),
                                      _ptr(bmu), batch.shape[0], float(alpha), float(sigma),
                                      _ptr(out))
        return out

    def project(self, X, hi, lo, k: int, boost: float, adjust: float, threads: int = 0,
                diagnostics: bool = False):
        """Full projection of n points -> n x 2 float64.  With diagnostics=True
        also returns det/trace^2 per point (-1 when A = 0) and the solve branch
        (0 Cramer's rule, 1 rank one, 2 centroid)."""
        X, hi, lo = _f32(X), _f32(hi), _f32(lo)
        n, d = X.shape
        out = np.empty((n, 2), np.float64)
        ratio = np.empty(n, np.float64)
        branch = np.empty(n, np.int32)
        rc = self.lib.esom_oracle_project(_ptr(X), n, _ptr(hi), _ptr(lo), hi.shape[0], d, k,
                                          float(boost), float(adjust), _ptr(out), _ptr(ratio),
                                          _ptr(branch), threads)
        if rc != 0:
            raise ValueError(f"esom_oracle_project failed ({rc})")
        if diagnostics:
            return out, ratio, branch
        return out


_default = None


def get() -> Oracle:
    global _default
    if _default is None:
        _default = Oracle(build())
    return _default


def default_threads() -> int:
    return get().default_threads()


def knn(X, hi, k, threads=0):
    return get().knn(X, hi, k, threads)


def scores(d2, boost):
    return get().scores(d2, boost)


def fit(x, hi, lo, idx, s, adjust):
    return get().fit(x, hi, lo, idx, s, adjust)


def project(X, hi, lo, k, boost, adjust, threads=0, diagnostics=False):
    return get().project(X, hi, lo, k, boost, adjust, threads, diagnostics)


def som_step(hi, lo, batch, bmu, alpha, sigma):
    return get().som_step(hi, lo, batch, bmu, alpha, sigma)
