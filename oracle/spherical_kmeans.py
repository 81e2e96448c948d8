"""Spherical k-means (Lloyd iteration) in FP64: the oracle's definition.

Test infrastructure only: imported by tests, ``__graft_entry__.smoke()`` and
the CPU legs of ``bench.py``; never by the product path.

What it computes, and where the paper says so:
  * Objects x_i are unit L2 vectors stored sparsely as (t_(i,h), v_(i,h)),
    h = 1..(nt)_i, ascending t (Section 2.3, Fig. 1(a)).  FP32 input values are
    promoted to FP64 unchanged.
  * Assignment (Algorithm 2, Eq. 4): a(x_i) = argmax_j x_i . mu_j, with the
    similarity of a sparse object and a full mean written as Eq. 8:
        rho_ij = sum_h v_(i,h) * mu_(j, t_(i,h))      (summed in ascending h)
  * Update (Algorithm 2, last two steps): mu_j = normalise(mean of C_j).
    Dividing by |C_j| only rescales before the normalisation, so the oracle
    forms s_j = sum_{i in C_j} x_i (members in ascending i) and
    mu_j = s_j / ||s_j||_2.
  * Objective (Eq. 5): J = sum_i x_i . mu_{a(x_i)} with the means the
    assignment used.  Lloyd never decreases it.
  * Multiplication count of IVF (Eq. 15): sum_i sum_h (nc)_{t_(i,h)}.

Readings where the paper is silent or inconsistent (the CUDA path takes the same):
  R1 ties: the smallest cluster id among all maxima.  Algorithm 3 scans j
     upward with a strict '>' (first maximum wins); Algorithm 2 starts from
     the current assignment.  The stateless lowest-id rule is used.
  R2 an object sharing no term with any mean has rho = 0 everywhere and so
     goes to cluster 0 under R1 (Algorithm 3 would leave it unassigned);
     n_zero_sim counts these objects (zero_similarity_objects).
  R3 a cluster with no members, or whose member sum is exactly zero, keeps
     its previous mean (empty_policy 0) or becomes an empty mean with no
     terms (empty_policy 1); the paper's w/|C_j| would be 0/0.
  R4 a mean element whose FP64 sum is exactly 0 is dropped (Algorithm 3's
     w_p != 0 test).
  R5 initial means (K distinct objects) and means given by the caller are
     divided by their FP64 L2 norm, so every mean is unit length.
  R6 0-based ids (the paper counts from 1).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

# Means are held dense (K x D FP64) when that takes at most this many bytes;
# above it the same definition runs on sparse per-cluster means.
DENSE_LIMIT_BYTES = 1 << 30


@dataclass
class Means:
    """Cluster-major sparse means: row j holds the nonzero (term, value) of mu_j."""

    ptr: np.ndarray  # int64 [K+1]
    term: np.ndarray  # int64 [E], ascending within a row
    val: np.ndarray  # float64 [E]
    n_terms: int

    @property
    def k(self) -> int:
        return int(self.ptr.shape[0] - 1)

    def row(self, j: int):
        a, b = int(self.ptr[j]), int(self.ptr[j + 1])
        return self.term[a:b], self.val[a:b]

    def to_csr(self) -> sp.csr_matrix:
        return sp.csr_matrix((self.val, self.term, self.ptr), shape=(self.k, self.n_terms))

    def dense(self) -> np.ndarray:
        m = np.zeros((self.k, self.n_terms), dtype=np.float64)
        rows = np.repeat(np.arange(self.k), np.diff(self.ptr))
        m[rows, self.term] = self.val
        return m


def object_matrix(corpus, rows=None) -> sp.csr_matrix:
    """The objects as an N x D FP64 CSR matrix (optionally a subset of rows)."""
    x = sp.csr_matrix((corpus.val.astype(np.float64), corpus.term.astype(np.int64), corpus.row_ptr),
                      shape=(corpus.n_docs, corpus.n_terms))
    return x if rows is None else x[np.asarray(rows)]


def normalize_rows(ptr, term, val) -> Means:
    """Reading R5: mu_j = m_j / ||m_j||_2 in FP64; a zero row is an error."""
    ptr = np.asarray(ptr, dtype=np.int64)
    term = np.asarray(term, dtype=np.int64)
    val = np.asarray(val, dtype=np.float64)
    k = ptr.shape[0] - 1
    owner = np.repeat(np.arange(k), np.diff(ptr))
    sq = np.bincount(owner, weights=val * val, minlength=k)
    if np.any(sq == 0.0):
        raise ValueError("a mean row has zero norm")
    nrm = np.sqrt(sq)
    return Means(ptr=ptr.copy(), term=term.copy(), val=val / nrm[owner], n_terms=-1)


def initial_means(corpus, doc_ids) -> Means:
    """mu_j^[0] = x_{d_j} / ||x_{d_j}|| for K distinct seeded documents d_j (R5)."""
    doc_ids = np.asarray(doc_ids, dtype=np.int64)
    lens = corpus.row_ptr[doc_ids + 1] - corpus.row_ptr[doc_ids]
    ptr = np.zeros(len(doc_ids) + 1, dtype=np.int64)
    np.cumsum(lens, out=ptr[1:])
    idx = np.concatenate([np.arange(corpus.row_ptr[d], corpus.row_ptr[d + 1]) for d in doc_ids]) \
        if len(doc_ids) else np.zeros(0, np.int64)
    m = normalize_rows(ptr, corpus.term[idx], corpus.val[idx].astype(np.float64))
    m.n_terms = corpus.n_terms
    return m


def means_from_rows(ptr, term, val, n_terms: int) -> Means:
    """Means given cluster-major by the caller, each row normalised (R5)."""
    m = normalize_rows(ptr, term, val)
    m.n_terms = int(n_terms)
    return m


def similarities(corpus, means: Means, rows=None, chunk: int = 2048) -> np.ndarray:
    """rho[i, j] = sum_h v_(i,h) mu_(j, t_(i,h)) in FP64 (Eq. 8), ascending h.

    Dense means (K x D) when they fit DENSE_LIMIT_BYTES, else sparse means;
    both sum the nonzero products of each (i, j) in ascending h, and the dense
    form only adds exact zeros besides, so the two agree bit for bit.
    """
    x = object_matrix(corpus, rows)
    k = means.k
    out = np.empty((x.shape[0], k), dtype=np.float64)
    if k * corpus.n_terms * 8 <= DENSE_LIMIT_BYTES:
        mt = np.ascontiguousarray(means.dense().T)  # D x K
        for a in range(0, x.shape[0], chunk):
            out[a:a + chunk] = x[a:a + chunk] @ mt
    else:
        mt = means.to_csr().T.tocsr()  # D x K
        for a in range(0, x.shape[0], chunk):
            out[a:a + chunk] = (x[a:a + chunk] @ mt).toarray()
    return out


def assign_from_similarities(rho: np.ndarray):
    """a_i = lowest j among the maxima of rho_i (R1, R2); best_i; gap_i.

    gap_i = best_i minus the second largest value of rho_i counted with
    multiplicity (0 on a tie; +inf when K = 1).
    """
    n, k = rho.shape
    a = np.argmax(rho, axis=1).astype(np.int32)  # first maximum = lowest id
    best = rho[np.arange(n), a]
    if k >= 2:
        second = np.partition(rho, k - 2, axis=1)[:, k - 2]
        gap = best - second
    else:
        gap = np.full(n, np.inf)
    return a, best, gap


def cluster_sums(corpus, assign, k: int) -> sp.csr_matrix:
    """s_j = sum_{i : a_i = j} x_i in FP64 (members in ascending i) as K x D CSR.

    Computed as P X with P the K x N membership matrix.  Exact zeros are
    removed (R4) and column indices sorted.
    """
    n = corpus.n_docs
    assign = np.asarray(assign, dtype=np.int64)
    p = sp.csr_matrix((np.ones(n), (assign, np.arange(n))), shape=(k, n))
    p.sort_indices()
    s = (p @ object_matrix(corpus)).tocsr()
    s.eliminate_zeros()
    s.sort_indices()
    return s


def update(corpus, assign, prev: Means, empty_policy: int = 0):
    """New means mu_j = s_j / ||s_j||, empty clusters per R3.

    Returns (means, sum_norm, sizes): sum_norm[j] = ||s_j||_2 (0 when empty),
    sizes[j] = |C_j|.
    """
    k = prev.k
    s = cluster_sums(corpus, assign, k)
    sizes = np.bincount(np.asarray(assign, dtype=np.int64), minlength=k)
    s_ptr = s.indptr.astype(np.int64)
    owner = np.repeat(np.arange(k), np.diff(s_ptr))
    sq = np.bincount(owner, weights=s.data * s.data, minlength=k)
    norm = np.sqrt(sq)
    live = norm > 0.0
    if empty_policy == 0:
        lens = np.where(live, np.diff(s_ptr), np.diff(prev.ptr))
    elif empty_policy == 1:
        lens = np.where(live, np.diff(s_ptr), 0)
    else:
        raise ValueError("empty_policy must be 0 or 1")
    ptr = np.zeros(k + 1, dtype=np.int64)
    np.cumsum(lens, out=ptr[1:])
    term = np.empty(int(ptr[-1]), dtype=np.int64)
    val = np.empty(int(ptr[-1]), dtype=np.float64)
    for j in range(k):
        a, b = int(ptr[j]), int(ptr[j + 1])
        if live[j]:
            sa, sb = int(s_ptr[j]), int(s_ptr[j + 1])
            term[a:b] = s.indices[sa:sb]
            val[a:b] = s.data[sa:sb] / norm[j]
        elif empty_policy == 0:
            pt, pv = prev.row(j)
            term[a:b] = pt
            val[a:b] = pv
    return Means(ptr=ptr, term=term, val=val, n_terms=prev.n_terms), norm, sizes


def zero_similarity_objects(corpus, means: Means) -> np.ndarray:
    """Mask of the objects that share no term with any mean (reading R2).

    These are the objects for which Algorithm 3's inner loop over posting
    entries never runs, so it never assigns them: sum_h (nc)_{t_(i,h)} = 0.
    An object that shares terms but whose similarities all come out 0 (signed
    values that cancel) is not one of them.
    """
    nc = np.bincount(means.term, minlength=corpus.n_terms).astype(np.int64)
    owner = np.repeat(np.arange(corpus.n_docs), np.diff(corpus.row_ptr))
    per_obj = np.bincount(owner, weights=nc[corpus.term], minlength=corpus.n_docs)
    return per_obj == 0


def objective(best) -> float:
    """J = sum_i x_i . mu_{a_i} (Eq. 5) accumulated in FP64."""
    return float(np.sum(np.asarray(best, dtype=np.float64)))


def multiplication_count(corpus, means: Means) -> int:
    """IVF's number of multiplications, Eq. 15: sum_i sum_h (nc)_{t_(i,h)}.

    (nc)_p = number of means with a nonzero element at term p.
    """
    nc = np.bincount(means.term, minlength=corpus.n_terms).astype(np.int64)
    return int(nc[corpus.term].sum())


@dataclass
class Iteration:
    r: int
    assign: np.ndarray
    best: np.ndarray
    gap: np.ndarray
    objective: float
    n_changed: int
    n_zero_sim: int
    mult_count: int
    means_before: Means
    means_after: Means
    sum_norm: np.ndarray
    sizes: np.ndarray


def iterate(corpus, means0: Means, max_iter: int, empty_policy: int = 0,
            stop_on_convergence: bool = True, prev_assign=None) -> list[Iteration]:
    """Run spherical Lloyd iterations r = 1..max_iter from means0.

    Stops after the first iteration r >= 2 with no assignment change
    ("until convergence", Section 5.2).  n_changed at r = 1 counts objects
    whose assignment differs from prev_assign (all N when it is None).
    """
    out = []
    means = means0
    prev = None if prev_assign is None else np.asarray(prev_assign, dtype=np.int32)
    for r in range(1, max_iter + 1):
        rho = similarities(corpus, means)
        a, best, gap = assign_from_similarities(rho)
        n_changed = corpus.n_docs if prev is None else int(np.count_nonzero(a != prev))
        n_zero = int(np.count_nonzero(zero_similarity_objects(corpus, means)))
        mc = multiplication_count(corpus, means)
        new_means, norm, sizes = update(corpus, a, means, empty_policy)
        out.append(Iteration(r=r, assign=a, best=best, gap=gap, objective=objective(best),
                             n_changed=n_changed, n_zero_sim=n_zero, mult_count=mc,
                             means_before=means, means_after=new_means, sum_norm=norm, sizes=sizes))
        means = new_means
        if stop_on_convergence and r >= 2 and n_changed == 0:
            break
        prev = a
    return out


def lockstep_check(corpus, means_prev: Means, gpu_assign, gpu_best=None, rows=None,
                   gap_exclusion: float = 1e-6, best_tol: float = 1e-5) -> dict:
    """Compare one GPU assignment with the FP64 argmax under the same means.

    rows: object ids to check (all when None); gpu_assign / gpu_best are the
    full-length GPU outputs.  Objects whose FP64 top-2 gap is below
    gap_exclusion are excluded from the assignment comparison.
    """
    rows_arr = np.arange(corpus.n_docs) if rows is None else np.asarray(rows, dtype=np.int64)
    rho = similarities(corpus, means_prev, rows_arr)
    a, best, gap = assign_from_similarities(rho)
    ga = np.asarray(gpu_assign)[rows_arr]
    excluded = gap < gap_exclusion
    mism = (ga != a) & ~excluded
    rep = {"checked": int(rows_arr.size), "excluded": int(excluded.sum()),
           "mismatches": int(mism.sum()), "mismatch_rows": rows_arr[mism][:20].tolist()}
    if gpu_best is not None:
        gb = np.asarray(gpu_best, dtype=np.float64)[rows_arr]
        rep["max_best_err"] = float(np.max(np.abs(gb - best))) if rows_arr.size else 0.0
        rep["best_ok"] = rep["max_best_err"] <= best_tol
    rep["oracle_assign"] = a
    rep["oracle_best"] = best
    rep["oracle_gap"] = gap
    return rep
