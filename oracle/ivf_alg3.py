"""ctypes front end of oracle/ivf_alg3.c: Algorithm 3 (IVF) in C, FP64.

Test infrastructure and the timed CPU baseline of the paper's own method
(Section 3, Algorithm 3; Section 5 runs it single-threaded in C).  It
computes what oracle/inverted_file.py computes, in the same FP64 operation
order, but fast enough for the benchmark's workloads; the objects loop of
the assignment and the clusters loop of the update run on OpenMP threads.

Only tests/, the smoke check and bench.py's CPU legs use it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ivf_alg3.c")
_LIB = os.path.join(_HERE, "libivf_alg3.so")
# -ffp-contract=off: no fused multiply-add, so every product and sum rounds
# as written (the order the Python module uses)
CFLAGS = ["-O3", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.run(["gcc", *CFLAGS, _SRC, "-o", tmp, "-lm"], check=True)
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        vp, i64, i32, cint = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int
        lib.alg3_assign.argtypes = [i64, vp, vp, vp, i32, i64, vp, vp, vp, vp, i64, vp, vp, vp, cint]
        lib.alg3_assign.restype = cint
        lib.alg3_update.argtypes = [i64, vp, vp, vp, i32, i64, vp, vp, vp, vp, i32, i32, i32, vp, vp, vp, i64, vp,
                                    cint]
        lib.alg3_update.restype = cint
        lib.alg3_threads_available.argtypes = []
        lib.alg3_threads_available.restype = cint
        _lib = lib
    return _lib


def threads_available() -> int:
    return int(_load().alg3_threads_available())


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


class InvertedFile:
    """Term-major means: xi_s = (c, u) pairs in xi_ptr[s]:xi_ptr[s+1], ascending c."""

    def __init__(self, ptr, c, u):
        self.ptr = np.ascontiguousarray(ptr, dtype=np.int64)
        self.c = np.ascontiguousarray(c, dtype=np.int32)
        self.u = np.ascontiguousarray(u, dtype=np.float64)

    @classmethod
    def from_means(cls, means):
        """From cluster-major means (oracle.spherical_kmeans.Means)."""
        counts = np.bincount(means.term, minlength=means.n_terms)
        ptr = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
        owner = np.repeat(np.arange(means.k, dtype=np.int32), np.diff(means.ptr))
        order = np.argsort(means.term, kind="stable")  # by term; rows are in ascending cluster order
        return cls(ptr, owner[order], means.val[order])

    @classmethod
    def from_lists(cls, xi):
        """From the list form of oracle.inverted_file ([(c, u), ...] per term)."""
        ptr = np.concatenate([[0], np.cumsum([len(x) for x in xi])]).astype(np.int64)
        c = np.array([cu[0] for x in xi for cu in x], dtype=np.int32)
        u = np.array([cu[1] for x in xi for cu in x], dtype=np.float64)
        return cls(ptr, c, u)


def _corpus_arrays(corpus):
    return (np.ascontiguousarray(corpus.row_ptr, dtype=np.int64), np.ascontiguousarray(corpus.term, dtype=np.int32),
            np.ascontiguousarray(corpus.val, dtype=np.float32))


def assignment_step(corpus, xi: InvertedFile, k: int, rows=None, threads: int = 0):
    """Algorithm 3's assignment: (assign, best, multiplications) for all objects or `rows`."""
    rp, tm, vl = _corpus_arrays(corpus)
    rows_a = None if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    n_out = corpus.n_docs if rows_a is None else rows_a.size
    assign = np.empty(n_out, dtype=np.int32)
    best = np.empty(n_out, dtype=np.float64)
    mults = ctypes.c_int64(0)
    st = _load().alg3_assign(corpus.n_docs, _p(rp), _p(tm), _p(vl), int(k), int(corpus.n_terms), _p(xi.ptr),
                             _p(xi.c), _p(xi.u), _p(rows_a), int(n_out), _p(assign), _p(best),
                             ctypes.byref(mults), int(threads))
    if st != 0:
        raise RuntimeError(f"alg3_assign failed with status {st}")
    return assign, best, int(mults.value)


def update_step(corpus, assign, k: int, prev: InvertedFile | None = None, empty_policy: int = 0,
                threads: int = 0, clusters: tuple[int, int] | None = None) -> InvertedFile:
    """Algorithm 3's update: the new inverted file from the assignment
    (clusters = (j0, j1): only those clusters' rows, for timing a sample)."""
    j0, j1 = (0, int(k)) if clusters is None else (int(clusters[0]), int(clusters[1]))
    rp, tm, vl = _corpus_arrays(corpus)
    a = np.ascontiguousarray(assign, dtype=np.int32)
    out_ptr = np.empty(corpus.n_terms + 1, dtype=np.int64)
    cap = int(min(corpus.nnz, int(k) * corpus.n_terms)) + (0 if prev is None else int(prev.ptr[-1]))
    out_c = np.empty(max(cap, 1), dtype=np.int32)
    out_u = np.empty(max(cap, 1), dtype=np.float64)
    out_len = ctypes.c_int64(0)
    st = _load().alg3_update(corpus.n_docs, _p(rp), _p(tm), _p(vl), int(k), int(corpus.n_terms), _p(a),
                             _p(prev.ptr) if prev else None, _p(prev.c) if prev else None,
                             _p(prev.u) if prev else None, int(empty_policy), j0, j1, _p(out_ptr), _p(out_c),
                             _p(out_u),
                             int(cap), ctypes.byref(out_len), int(threads))
    if st != 0:
        raise RuntimeError(f"alg3_update failed with status {st}")
    e = int(out_len.value)
    return InvertedFile(out_ptr, out_c[:e].copy(), out_u[:e].copy())
