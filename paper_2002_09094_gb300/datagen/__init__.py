"""Seeded synthetic inputs for inverted-file spherical k-means.

This module makes the object set of the paper's problem statement (Section
2.2: N L2-normalised sparse document vectors; Section 2.3 / Fig. 1: each
object stored as sorted (term id, value) tuples) with the shape of its tf-idf
corpora (Section 5.1: PubMed and NYT, which are not available here): Zipf term
ids without repeats inside a document, lognormal weights, unit L2 norm.  It
also draws the K distinct documents that seed the initial means.

It holds none of the clustering method's arithmetic: the FP64 oracle and the
CUDA path both take their inputs from here and from nowhere else.  The heavy
lifting is in ``corpus.c`` (counter-based SplitMix64 streams per document,
OpenMP), so a corpus depends only on its spec and seed, not on thread count.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field, replace

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "corpus.c")
_LIB = os.path.join(_HERE, "_libcorpus.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile corpus.c into a shared library beside it (gcc, OpenMP)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                   _SRC, "-o", tmp, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        i64, f64, u64, cint = ctypes.c_int64, ctypes.c_double, ctypes.c_uint64, ctypes.c_int
        vp = ctypes.c_void_p
        lib.corpus_lengths.argtypes = [i64, i64, cint, f64, f64, i64, i64, u64, vp]
        lib.corpus_lengths.restype = cint
        lib.corpus_zipf_cdf.argtypes = [i64, f64, vp]
        lib.corpus_zipf_cdf.restype = cint
        lib.corpus_fill.argtypes = [i64, i64, vp, u64, vp, vp, vp]
        lib.corpus_fill.restype = cint
        _lib = lib
    return _lib


@dataclass(frozen=True)
class CorpusSpec:
    """Recipe of one synthetic document collection.

    length_kind: "poisson" (mean length_mean) or "lognormal" (unclipped mean
    length_mean, log-space sigma length_sigma); lengths are clipped to
    [length_lo, min(length_hi, n_terms)].  Term ids follow a Zipf law with
    exponent zipf_s over ranks 1..n_terms (rank r -> id r-1).
    """

    n_docs: int
    n_terms: int
    length_kind: str
    length_mean: float
    length_lo: int
    length_hi: int
    zipf_s: float
    seed: int
    length_sigma: float = 0.75


@dataclass
class Corpus:
    """CSR object set: row i is object x_i with sorted unique term ids."""

    row_ptr: np.ndarray  # int64 [N+1]
    term: np.ndarray  # int32 [nnz], ascending within a row
    val: np.ndarray  # float32 [nnz], each row has unit L2 norm
    n_terms: int
    spec: CorpusSpec | None = field(default=None, repr=False)

    @property
    def n_docs(self) -> int:
        return int(self.row_ptr.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])


def make_corpus(spec: CorpusSpec) -> Corpus:
    lib = _load()
    n, d = int(spec.n_docs), int(spec.n_terms)
    kind = {"poisson": 0, "lognormal": 1}[spec.length_kind]
    lengths = np.empty(n, dtype=np.int64)
    rc = lib.corpus_lengths(n, d, kind, float(spec.length_mean), float(spec.length_sigma),
                            int(spec.length_lo), int(spec.length_hi), int(spec.seed) & (2**64 - 1),
                            lengths.ctypes.data)
    if rc != 0:
        raise ValueError(f"bad corpus spec {spec}")
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lengths, out=row_ptr[1:])
    nnz = int(row_ptr[-1])
    cdf = np.empty(d, dtype=np.float64)
    if lib.corpus_zipf_cdf(d, float(spec.zipf_s), cdf.ctypes.data) != 0:
        raise ValueError("bad Zipf parameters")
    term = np.empty(nnz, dtype=np.int32)
    val = np.empty(nnz, dtype=np.float32)
    rc = lib.corpus_fill(n, d, cdf.ctypes.data, int(spec.seed) & (2**64 - 1), row_ptr.ctypes.data,
                         term.ctypes.data, val.ctypes.data)
    if rc != 0:
        raise RuntimeError("corpus_fill failed")
    return Corpus(row_ptr=row_ptr, term=term, val=val, n_terms=d, spec=spec)


def corpus_from_rows(rows, n_terms: int) -> Corpus:
    """Build a Corpus from explicit rows [(terms, values), ...] (hand-made cases).

    Terms are sorted per row; values are stored as given (no normalisation).
    """
    row_ptr = [0]
    terms, vals = [], []
    for t, v in rows:
        t = np.asarray(t, dtype=np.int64)
        v = np.asarray(v, dtype=np.float64)
        order = np.argsort(t, kind="stable")
        terms.append(t[order])
        vals.append(v[order])
        row_ptr.append(row_ptr[-1] + len(t))
    term = np.concatenate(terms).astype(np.int32) if terms else np.zeros(0, np.int32)
    val = np.concatenate(vals).astype(np.float32) if vals else np.zeros(0, np.float32)
    return Corpus(row_ptr=np.asarray(row_ptr, dtype=np.int64), term=term, val=val, n_terms=int(n_terms))


def init_doc_ids(n_docs: int, k: int, seed: int) -> np.ndarray:
    """K distinct document ids d_0..d_{K-1}; initial mean j is object d_j."""
    if not 1 <= k <= n_docs:
        raise ValueError("need 1 <= k <= n_docs")
    rng = np.random.default_rng(seed)
    return rng.choice(n_docs, size=k, replace=False).astype(np.int32)


@dataclass(frozen=True)
class Workload:
    """A named clustering workload: corpus recipe, K, init seed, iterations."""

    name: str
    corpus: CorpusSpec
    k: int
    init_seed: int
    iterations: int

    def scaled(self, n_docs: int | None = None, n_terms: int | None = None, k: int | None = None,
               name: str | None = None) -> "Workload":
        c = replace(self.corpus, n_docs=n_docs or self.corpus.n_docs, n_terms=n_terms or self.corpus.n_terms)
        return replace(self, corpus=c, k=k or self.k, name=name or f"{self.name}-scaled")


_SEED0 = 20020909

# 10,000 Poisson(50)-length docs over 20,000 terms, Zipf 1.1, K = 100, 10 iterations.
SMALL = Workload(
    name="ivf-small-n10k-d20k-k100",
    corpus=CorpusSpec(n_docs=10_000, n_terms=20_000, length_kind="poisson", length_mean=50.0,
                      length_lo=5, length_hi=200, zipf_s=1.1, seed=_SEED0),
    k=100, init_seed=_SEED0 + 1, iterations=10)

# 1,000,000 lognormal(mean 120)-length docs over 500,000 terms, Zipf 1.05, K = 10,000.
SCALE = Workload(
    name="ivf-scale-n1m-d500k-k10k",
    corpus=CorpusSpec(n_docs=1_000_000, n_terms=500_000, length_kind="lognormal", length_mean=120.0,
                      length_lo=10, length_hi=2_000, zipf_s=1.05, seed=_SEED0 + 1),
    k=10_000, init_seed=_SEED0 + 2, iterations=30)

# 8,000,000 lognormal(mean 80)-length docs over 2,000,000 terms, Zipf 1.0, K = 80,000.
LARGE = Workload(
    name="ivf-large-n8m-d2m-k80k",
    corpus=CorpusSpec(n_docs=8_000_000, n_terms=2_000_000, length_kind="lognormal", length_mean=80.0,
                      length_lo=5, length_hi=1_500, zipf_s=1.0, seed=_SEED0 + 2),
    k=80_000, init_seed=_SEED0 + 3, iterations=10)

WORKLOADS = {w.name: w for w in (SMALL, SCALE, LARGE)}


def batched_workloads(n_instances: int = 256, seed: int = _SEED0 + 4,
                      n_range=(2_000, 200_000), k_range=(16, 2_000), d_range=(10_000, 100_000),
                      nnz_range=(20.0, 150.0), iterations: int = 15) -> list[Workload]:
    """Independent instances of uneven N, K and D (Poisson lengths, Zipf 1.1)."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(n_instances):
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        k = int(rng.integers(k_range[0], k_range[1] + 1))
        d = int(rng.integers(d_range[0], d_range[1] + 1))
        m = float(rng.uniform(nnz_range[0], nnz_range[1]))
        k = min(k, n)
        spec = CorpusSpec(n_docs=n, n_terms=d, length_kind="poisson", length_mean=m, length_lo=5,
                          length_hi=int(min(d, 4 * m)), zipf_s=1.1, seed=seed + 1000 * (b + 1))
        out.append(Workload(name=f"batch{b}-n{n}-d{d}-k{k}", corpus=spec, k=k,
                            init_seed=seed + 1000 * (b + 1) + 1, iterations=iterations))
    return out
