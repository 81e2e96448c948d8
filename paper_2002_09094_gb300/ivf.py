"""Python binding of libivfkm (include/ivf.h) via ctypes.

Argument marshalling only: every step of the clustering runs in the CUDA
kernels of the library.  Arrays may be numpy arrays, CPU torch tensors or CUDA
torch tensors; they are passed to the library as raw pointers (it copies what
it keeps).  The CUDA stream defaults to torch's current stream.

If the shared library is missing this module raises at import time of the
first context: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Any

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libivfkm.so")

IVF_OK, IVF_E_INVALID, IVF_E_STATE, IVF_E_OOM, IVF_E_CUDA, IVF_E_TIMEOUT, IVF_E_UNSUPPORTED = range(7)
STATUS_NAMES = {0: "IVF_OK", 1: "IVF_E_INVALID", 2: "IVF_E_STATE", 3: "IVF_E_OOM", 4: "IVF_E_CUDA",
                5: "IVF_E_TIMEOUT", 6: "IVF_E_UNSUPPORTED"}
STORAGE = {"f32": 0, "f16": 1, "bf16": 2}
IVF_FLAG_VALIDATE = 1
IVF_FLAG_NO_GRAPH = 2
IVF_FLAG_DENSE_HEAD = 4
IVF_FLAG_SPARSE_ONLY = 8
IVF_FLAG_TENSOR_HEAD = 16
IVF_FLAG_TILE_MAJOR = 32
IVF_FLAG_OBJECT_MAJOR = 64
IVF_FLAG_IVFD = 128
SCHEDULE_FLAGS = {"auto": 0, "tile_major": IVF_FLAG_TILE_MAJOR, "object_major": IVF_FLAG_OBJECT_MAJOR}
KERNEL_FLAGS = {"auto": 0, "dense_head": IVF_FLAG_DENSE_HEAD, "sparse": IVF_FLAG_SPARSE_ONLY,
                "tensor_head": IVF_FLAG_TENSOR_HEAD, "ivfd": IVF_FLAG_IVFD}

# Every symbol include/ivf.h declares.
EXPORTS = ["ivf_create", "ivf_load_objects", "ivf_set_means", "ivf_set_means_from_docs", "ivf_assign",
           "ivf_update", "ivf_iterate", "ivf_get_assign", "ivf_get_best", "ivf_get_gap", "ivf_get_info",
           "ivf_get_err_bound", "ivf_get_means", "ivf_get_inverted_file", "ivf_get_members", "ivf_set_assign", "ivf_restore_means",
           "ivf_last_error", "ivf_destroy", "ivf_launch_count", "ivf_version", "ivfb_create", "ivfb_get_changed",
           "ivf_timing_reset", "ivf_get_timing", "ivf_assign_static", "ivf_probe_l2_read", "ivf_head_product",
           "ivf_get_partial_sums", "ivf_update_from_partials"]
IVF_STATIC_MAX_DOCS = 16384
IVF_STATIC_MAX_K = 12288


class IvfError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status
        self.message = message


class Config(ctypes.Structure):
    _fields_ = [("n_docs", ctypes.c_int64), ("n_terms", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("k", ctypes.c_int32), ("storage", ctypes.c_int32), ("rescore", ctypes.c_int32),
                ("empty_policy", ctypes.c_int32), ("k_tile", ctypes.c_int32), ("warps_per_block", ctypes.c_int32),
                ("flags", ctypes.c_uint32), ("means_capacity", ctypes.c_int32),
                ("dense_head_bytes", ctypes.c_int64)]


class IterStats(ctypes.Structure):
    _fields_ = [("n_changed", ctypes.c_int64), ("entries_visited", ctypes.c_int64),
                ("ivf_entries", ctypes.c_int64), ("n_zero_sim", ctypes.c_int64), ("n_flagged", ctypes.c_int64),
                ("n_rescored", ctypes.c_int64), ("objective", ctypes.c_double), ("t_assign_ms", ctypes.c_float),
                ("t_update_ms", ctypes.c_float)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class Timing(ctypes.Structure):
    _fields_ = [("n_assign", ctypes.c_int32), ("n_update", ctypes.c_int32), ("assign_kernel_ms", ctypes.c_double),
                ("assign_step_ms", ctypes.c_double), ("update_ms", ctypes.c_double),
                ("entries_visited", ctypes.c_int64), ("n_rescored", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class Info(ctypes.Structure):
    _fields_ = [("n_docs", ctypes.c_int64), ("n_terms", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("k", ctypes.c_int32), ("n_instances", ctypes.c_int32), ("ivf_entries", ctypes.c_int64),
                ("ivf_capacity", ctypes.c_int64), ("k_tile", ctypes.c_int32), ("warps_per_block", ctypes.c_int32),
                ("iteration", ctypes.c_int32), ("storage", ctypes.c_int32), ("device_bytes", ctypes.c_int64),
                ("dense_head_r", ctypes.c_int32), ("dense_head_sub", ctypes.c_int32),
                ("dense_head_tensor", ctypes.c_int32),
                ("dense_head_theta", ctypes.c_float),
                ("dense_head_rows", ctypes.c_int64), ("tile_major", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libivfkm.so and declare its signatures (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: run `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(path)
    vp, i32, i64, st = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_int
    P = ctypes.POINTER
    sig = {
        "ivf_create": ([P(Config), vp, vp, vp, vp, P(vp)], st),
        "ivf_load_objects": ([vp, vp, vp, vp], st),
        "ivf_set_means": ([vp, vp, vp, vp], st),
        "ivf_set_means_from_docs": ([vp, vp], st),
        "ivf_assign": ([vp, vp, vp, vp, P(IterStats)], st),
        "ivf_update": ([vp], st),
        "ivf_iterate": ([vp, i32, P(i32), P(i32), P(IterStats)], st),
        "ivf_get_assign": ([vp, vp], st),
        "ivf_get_best": ([vp, vp], st),
        "ivf_get_gap": ([vp, vp], st),
        "ivf_get_err_bound": ([vp, vp], st),
        "ivf_get_info": ([vp, P(Info)], st),
        "ivf_get_means": ([vp, vp, vp, vp], st),
        "ivf_get_inverted_file": ([vp, vp, vp, vp], st),
        "ivf_get_members": ([vp, vp, vp], st),
        "ivf_set_assign": ([vp, vp], st),
        "ivf_restore_means": ([vp, vp, vp, vp, i32], st),
        "ivf_last_error": ([vp], ctypes.c_char_p),
        "ivf_destroy": ([vp], None),
        "ivf_launch_count": ([], i64),
        "ivf_version": ([], ctypes.c_char_p),
        "ivfb_create": ([P(Config), i32, vp, vp, vp, vp, vp, vp, vp, P(vp)], st),
        "ivfb_get_changed": ([vp, vp], st),
        "ivf_timing_reset": ([vp, i32], st),
        "ivf_get_timing": ([vp, P(Timing)], st),
        "ivf_assign_static": ([i64, vp, vp, vp, i64, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp], st),
        "ivf_probe_l2_read": ([i64, i32, vp, ctypes.POINTER(ctypes.c_double)], st),
        "ivf_head_product": ([i64, i32, i32, vp, i64, vp, i64, vp, i64, i32, vp], st),
        "ivf_get_partial_sums": ([vp, i64, vp, vp, vp, ctypes.POINTER(i64)], st),
        "ivf_update_from_partials": ([vp, i64, vp, vp, vp], st),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def launch_count() -> int:
    return int(load_library().ivf_launch_count())


def head_product(a, b, d, storage: str, stream=None) -> None:
    """d = a @ b.T on the tensor cores (ivf_head_product); a (m x k), b (n x k),
    d (m x n): 16-bit CUDA tensors (torch) with unit column stride."""
    for t in (a, b, d):
        if not t.is_cuda or t.stride(1) != 1:
            raise ValueError("head_product takes row-major CUDA tensors")
    s = _default_stream() if stream is None else stream
    st = load_library().ivf_head_product(int(a.shape[0]), int(b.shape[0]), int(a.shape[1]), a.data_ptr(), a.stride(0),
                                         b.data_ptr(), b.stride(0), d.data_ptr(), d.stride(0), STORAGE[storage],
                                         ctypes.c_void_p(s))
    if st != 0:
        raise IvfError(st, "ivf_head_product failed")


def probe_l2_read_gbs(nbytes: int = 48 << 20, reps: int = 64, stream=None) -> float:
    """Read bandwidth (GB/s) of a resident set served by L2 (ivf_probe_l2_read)."""
    out = ctypes.c_double(0.0)
    s = _default_stream() if stream is None else stream
    st = load_library().ivf_probe_l2_read(int(nbytes), int(reps), ctypes.c_void_p(s), ctypes.byref(out))
    if st != 0:
        raise IvfError(st, "ivf_probe_l2_read failed")
    return float(out.value)


def _ptr(x: Any, dtype) -> tuple[int, Any]:
    """(address, keep-alive object) of a contiguous array of the given numpy dtype."""
    if x is None:
        return 0, None
    try:
        import torch

        if isinstance(x, torch.Tensor):
            tdt = {np.int64: torch.int64, np.int32: torch.int32, np.float32: torch.float32,
                   np.float64: torch.float64}[np.dtype(dtype).type]
            if x.dtype != tdt:
                raise TypeError(f"expected {tdt}, got {x.dtype}")
            x = x.contiguous()
            return x.data_ptr(), x
    except ImportError:
        pass
    a = np.ascontiguousarray(x, dtype=dtype)
    return a.ctypes.data, a


def _default_stream():
    try:
        import torch

        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except ImportError:
        pass
    return 0


class IVF:
    """One inverted-file spherical k-means problem on the GPU (or a batch of them).

    Arguments mirror ``ivf_config`` (include/ivf.h): ``storage`` is "f32",
    "f16" or "bf16" (the streamed value type; accumulation is FP32, near-ties
    are re-scored in FP64 when ``rescore``); ``kernel`` restricts the
    autotuner to one family -- "auto", "sparse", "dense_head" (CUDA-core dense
    rows), "tensor_head" (FP16/BF16: dense rows as a tensor-core GEMM) or
    "ivfd" (the comparison algorithm IVFD: Algorithm 4's loop order over an
    inverted file of the objects);
    ``schedule`` restricts it to "tile_major" (one launch per cluster tile
    over all objects) or "object_major" shapes (default "auto": either);
    ``k_tile`` / ``warps_per_block`` fix the launch shape instead of tuning
    it; ``means_capacity`` and ``dense_head_bytes`` size the first
    allocations (both grow on demand); ``use_graph`` lets ``iterate`` replay
    CUDA graphs.  Arrays may be numpy arrays or torch tensors (host or
    device).
    """

    def __init__(self, row_ptr, term, val, n_terms: int, k: int, storage: str = "f32", rescore: bool = True,
                 empty_policy: int = 0, k_tile: int = 0, warps_per_block: int = 0, validate: bool = False,
                 use_graph: bool = True, stream=None, kernel: str = "auto", means_capacity: int = 0,
                 dense_head_bytes: int = 0, schedule: str = "auto", _batched=None):
        self._lib = load_library()
        self._ctx = ctypes.c_void_p(0)
        self._loading = None
        rp, rk = _ptr(row_ptr, np.int64)
        tp, tk = _ptr(term, np.int32)
        vptr, vk = _ptr(val, np.float32)
        n_docs = int(len(row_ptr) - 1)
        nnz = int(len(term))
        flags = ((IVF_FLAG_VALIDATE if validate else 0) | (0 if use_graph else IVF_FLAG_NO_GRAPH) |
                 KERNEL_FLAGS[kernel] | SCHEDULE_FLAGS[schedule])
        cfg = Config(n_docs=n_docs, n_terms=int(n_terms), nnz=nnz, k=int(k), storage=STORAGE[storage],
                     rescore=1 if rescore else 0, empty_policy=int(empty_policy), k_tile=int(k_tile),
                     warps_per_block=int(warps_per_block), flags=flags, means_capacity=int(means_capacity),
                     dense_head_bytes=int(dense_head_bytes))
        self.stream = _default_stream() if stream is None else stream
        if _batched is None:
            s = self._lib.ivf_create(ctypes.byref(cfg), rp, tp, vptr, ctypes.c_void_p(self.stream),
                                     ctypes.byref(self._ctx))
        else:
            inst_docs, inst_terms, inst_k = _batched
            dp, dk = _ptr(inst_docs, np.int64)
            ip, ik = _ptr(inst_terms, np.int32)
            kp, kk = _ptr(inst_k, np.int32)
            s = self._lib.ivfb_create(ctypes.byref(cfg), int(len(inst_k)), dp, ip, kp, rp, tp, vptr,
                                      ctypes.c_void_p(self.stream), ctypes.byref(self._ctx))
        if s != IVF_OK:
            raise IvfError(s, "ivf_create failed (see stderr)")
        self.n_docs = n_docs
        self.nnz = nnz
        self.storage = storage
        info = self.info()
        self.k = info["k"]
        self.n_terms = info["n_terms"]
        self.n_instances = info["n_instances"]

    # -- plumbing
    def _check(self, status: int):
        if status != IVF_OK:
            msg = self._lib.ivf_last_error(self._ctx)
            raise IvfError(status, msg.decode() if msg else "")

    def close(self):
        if self._ctx:
            self._lib.ivf_destroy(self._ctx)
            self._ctx = ctypes.c_void_p(0)
        self._loading = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- calls
    def load_objects(self, row_ptr, term, val):
        """New objects (same N and nnz), copied on a second stream; they take
        effect at the next assign / iterate / set_means_from_docs, and update()
        keeps working on the objects of the last assignment.  The sources are
        held until then (a pinned host buffer is read asynchronously)."""
        rp, rk = _ptr(row_ptr, np.int64)
        tp, tk = _ptr(term, np.int32)
        vp, vk = _ptr(val, np.float32)
        self._check(self._lib.ivf_load_objects(self._ctx, rp, tp, vp))
        self._loading = (rk, tk, vk)

    def set_means(self, mean_ptr, mean_term, mean_val):
        pp, pk = _ptr(mean_ptr, np.int64)
        tp, tk = _ptr(mean_term, np.int32)
        vp, vk = _ptr(mean_val, np.float32)
        self._check(self._lib.ivf_set_means(self._ctx, pp, tp, vp))

    def set_means_from_docs(self, doc_ids):
        dp, dk = _ptr(doc_ids, np.int32)
        self._check(self._lib.ivf_set_means_from_docs(self._ctx, dp))
        self._loading = None

    def assign(self, assign_out=None, best_out=None, gap_out=None, stats: bool = True):
        """Assignment step; outputs are optional CUDA tensors. Returns stats dict (or None)."""
        st = IterStats()
        ap = assign_out.data_ptr() if assign_out is not None else 0
        bp = best_out.data_ptr() if best_out is not None else 0
        gp = gap_out.data_ptr() if gap_out is not None else 0
        self._check(self._lib.ivf_assign(self._ctx, ap, bp, gp, ctypes.byref(st) if stats else None))
        self._loading = None
        return st.as_dict() if stats else None

    def update(self):
        self._check(self._lib.ivf_update(self._ctx))

    def iterate(self, max_iter: int):
        done, conv = ctypes.c_int32(0), ctypes.c_int32(0)
        st = IterStats()
        self._check(self._lib.ivf_iterate(self._ctx, int(max_iter), ctypes.byref(done), ctypes.byref(conv),
                                          ctypes.byref(st)))
        self._loading = None
        return int(done.value), bool(conv.value), st.as_dict()

    def get_assign(self, out=None) -> np.ndarray:
        if out is not None:
            self._check(self._lib.ivf_get_assign(self._ctx, out.data_ptr()))
            return out
        a = np.empty(self.n_docs, dtype=np.int32)
        self._check(self._lib.ivf_get_assign(self._ctx, a.ctypes.data))
        return a

    def get_best(self) -> np.ndarray:
        a = np.empty(self.n_docs, dtype=np.float32)
        self._check(self._lib.ivf_get_best(self._ctx, a.ctypes.data))
        return a

    def get_gap(self) -> np.ndarray:
        a = np.empty(self.n_docs, dtype=np.float32)
        self._check(self._lib.ivf_get_gap(self._ctx, a.ctypes.data))
        return a

    def get_partial_sums(self):
        """This context's member sums of its last assignment, before
        normalisation: (cluster int32[U], term int32[U], sum float64[U]) in
        ascending (cluster, term) (ivf_get_partial_sums)."""
        n = ctypes.c_int64(0)
        self._check(self._lib.ivf_get_partial_sums(self._ctx, 0, None, None, None, ctypes.byref(n)))
        u = int(n.value)
        cl = np.empty(u, dtype=np.int32)
        tm = np.empty(u, dtype=np.int32)
        sm = np.empty(u, dtype=np.float64)
        if u:
            self._check(self._lib.ivf_get_partial_sums(self._ctx, u, cl.ctypes.data, tm.ctypes.data, sm.ctypes.data,
                                                       ctypes.byref(n)))
        return cl, tm, sm

    def update_from_partials(self, cluster, term, sums) -> None:
        """The update step from member sums of every shard, concatenated in
        shard order (ivf_update_from_partials)."""
        cp, ck = _ptr(cluster, np.int32)
        tp, tk = _ptr(term, np.int32)
        sp, sk = _ptr(sums, np.float64)
        self._check(self._lib.ivf_update_from_partials(self._ctx, int(len(cluster)), cp, tp, sp))

    def get_err_bound(self) -> np.ndarray:
        """Per object: a bound on |best - rho| against the FP64 means (ivf_get_err_bound)."""
        a = np.empty(self.n_docs, dtype=np.float32)
        self._check(self._lib.ivf_get_err_bound(self._ctx, a.ctypes.data))
        return a

    def info(self) -> dict:
        i = Info()
        self._check(self._lib.ivf_get_info(self._ctx, ctypes.byref(i)))
        return i.as_dict()

    def get_means(self):
        """FP64 master means, cluster-major: (ptr int64[K+1], term int32[E], val float64[E])."""
        ptr = np.empty(self.k + 1, dtype=np.int64)
        self._check(self._lib.ivf_get_means(self._ctx, ptr.ctypes.data, None, None))
        e = int(ptr[-1])
        term = np.empty(e, dtype=np.int32)
        val = np.empty(e, dtype=np.float64)
        self._check(self._lib.ivf_get_means(self._ctx, None, term.ctypes.data, val.ctypes.data))
        return ptr, term, val

    def get_inverted_file(self):
        """(term_ptr int64[D+1], cid int32[E], w float32[E]) as streamed by the assignment."""
        tp = np.empty(self.n_terms + 1, dtype=np.int64)
        self._check(self._lib.ivf_get_inverted_file(self._ctx, tp.ctypes.data, None, None))
        e = int(tp[-1])
        cid = np.empty(e, dtype=np.int32)
        w = np.empty(e, dtype=np.float32)
        self._check(self._lib.ivf_get_inverted_file(self._ctx, None, cid.ctypes.data, w.ctypes.data))
        return tp, cid, w

    def get_members(self):
        cl = np.empty(self.k + 1, dtype=np.int64)
        mem = np.empty(self.n_docs, dtype=np.int32)
        self._check(self._lib.ivf_get_members(self._ctx, cl.ctypes.data, mem.ctypes.data))
        return cl, mem

    def set_assign(self, assign):
        p, kp = _ptr(assign, np.int32)
        self._check(self._lib.ivf_set_assign(self._ctx, p))

    def restore_means(self, ptr, term, val, iteration: int = 0):
        pp, pk = _ptr(ptr, np.int64)
        tp, tk = _ptr(term, np.int32)
        vp, vk = _ptr(val, np.float64)
        self._check(self._lib.ivf_restore_means(self._ctx, pp, tp, vp, int(iteration)))

    def timing_reset(self, enable: bool = True):
        self._check(self._lib.ivf_timing_reset(self._ctx, 1 if enable else 0))

    def get_timing(self) -> dict:
        t = Timing()
        self._check(self._lib.ivf_get_timing(self._ctx, ctypes.byref(t)))
        return t.as_dict()

    def get_changed_per_instance(self) -> np.ndarray:
        a = np.empty(self.n_instances, dtype=np.int64)
        self._check(self._lib.ivfb_get_changed(self._ctx, a.ctypes.data))
        return a


class BatchedIVF(IVF):
    """Many independent problems in one context (each instance's own N, D, K).

    row_ptr/term/val concatenate the instances' CSR rows (row_ptr global, term
    ids local to each instance); inst_docs int64[n+1] object offsets,
    inst_terms int32[n], inst_k int32[n].
    """

    def __init__(self, row_ptr, term, val, inst_docs, inst_terms, inst_k, **kw):
        super().__init__(row_ptr, term, val, n_terms=int(np.sum(inst_terms)), k=int(np.sum(inst_k)),
                         _batched=(inst_docs, inst_terms, inst_k), **kw)
        self.inst_docs = np.asarray(inst_docs, dtype=np.int64)
        self.inst_k = np.asarray(inst_k, dtype=np.int32)
        self.inst_terms = np.asarray(inst_terms, dtype=np.int32)


def version() -> str:
    return load_library().ivf_version().decode()
