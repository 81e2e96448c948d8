"""The C Algorithm 3 (oracle/ivf_alg3.c) against the Python one (CPU only).

oracle/inverted_file.py is Algorithm 3 in plain Python loops, pinned to the
Lloyd definition by tests/test_oracle_pins.py.  The C version performs the
same FP64 operations in the same order, so its assignment (rho, argmax,
Eq. 15 count) must equal the Python one bit for bit; its update differs only
in how ||w||_2 is summed (Python's sum() is compensated), so the mean values
agree to 1e-15 and the list structure exactly.
"""
import numpy as np
import pytest

import oracle.inverted_file as pyivf
import oracle.ivf_alg3 as calg3
import oracle.spherical_kmeans as sk
from paper_2002_09094_gb300 import datagen as dg


def small_corpus(seed, n_docs=300, n_terms=120, mean_len=8.0):
    spec = dg.CorpusSpec(n_docs=n_docs, n_terms=n_terms, length_kind="poisson", length_mean=mean_len,
                         length_lo=2, length_hi=20, zipf_s=0.9, seed=seed)
    return dg.make_corpus(spec)


def _same_xi(xi_c, xi_py, atol=1e-15):
    ref = calg3.InvertedFile.from_lists(xi_py)
    assert np.array_equal(xi_c.ptr, ref.ptr)
    assert np.array_equal(xi_c.c, ref.c)
    assert np.allclose(xi_c.u, ref.u, rtol=0, atol=atol)


@pytest.mark.parametrize("threads", [1, 3])
def test_assignment_bit_equal_to_python_algorithm3(threads):
    c = small_corpus(41)
    k = 17
    m0 = sk.initial_means(c, dg.init_doc_ids(c.n_docs, k, 41))
    xi_py = pyivf.inverted_file_from_means(m0)
    a_py, b_py, _, mults_py = pyivf.assignment_step(c, xi_py, k)
    xi = calg3.InvertedFile.from_means(m0)
    _same_xi(xi, xi_py, atol=0.0)
    a, b, mults = calg3.assignment_step(c, xi, k, threads=threads)
    assert a.tolist() == a_py
    assert np.array_equal(b, np.array(b_py))
    assert mults == mults_py == sk.multiplication_count(c, m0)


def test_sampled_rows_equal_full_run():
    c = small_corpus(42)
    k = 9
    xi = calg3.InvertedFile.from_means(sk.initial_means(c, dg.init_doc_ids(c.n_docs, k, 42)))
    a, b, _ = calg3.assignment_step(c, xi, k)
    rows = np.array([0, 5, 77, 299, 5])
    a2, b2, _ = calg3.assignment_step(c, xi, k, rows=rows)
    assert np.array_equal(a2, a[rows]) and np.array_equal(b2, b[rows])


@pytest.mark.parametrize("empty_policy", [0, 1])
def test_iterations_equal_python_algorithm3(empty_policy):
    """Several full iterations, with clusters emptied on purpose (duplicate
    initial means leave the higher id empty), both empty-cluster policies."""
    c = small_corpus(43, n_docs=200, n_terms=80)
    k = 12
    ids = dg.init_doc_ids(c.n_docs, k, 43)
    m0 = sk.initial_means(c, ids)
    # cluster 7 duplicates cluster 3: it loses every tie and stays empty
    rows = [(m0.row(j) if j != 7 else m0.row(3)) for j in range(k)]
    ptr = np.concatenate([[0], np.cumsum([len(t) for t, _ in rows])])
    m0 = sk.means_from_rows(ptr, np.concatenate([t for t, _ in rows]), np.concatenate([v for _, v in rows]),
                            c.n_terms)
    xi_py = pyivf.inverted_file_from_means(m0)
    xi = calg3.InvertedFile.from_means(m0)
    saw_empty = False
    for _ in range(5):
        a_py, b_py, _, _ = pyivf.assignment_step(c, xi_py, k)
        a, b, _ = calg3.assignment_step(c, xi, k, threads=2)
        assert a.tolist() == a_py
        assert np.allclose(b, b_py, rtol=0, atol=1e-15)
        saw_empty |= np.bincount(a, minlength=k).min() == 0
        xi_py = pyivf.update_step(c, a_py, k, c.n_terms, prev_xi=xi_py, empty_policy=empty_policy)
        xi = calg3.update_step(c, a, k, prev=xi, empty_policy=empty_policy, threads=2)
        _same_xi(xi, xi_py)
    assert saw_empty


def test_trajectory_equals_lloyd_oracle():
    """From the same initial means the C Algorithm 3 follows the FP64 Lloyd
    oracle's trajectory (the Lloyd-type property of Section 2.1)."""
    c = small_corpus(44, n_docs=600, n_terms=200, mean_len=10.0)
    k = 20
    m0 = sk.initial_means(c, dg.init_doc_ids(c.n_docs, k, 44))
    lloyd = sk.iterate(c, m0, max_iter=6, stop_on_convergence=False)
    xi = calg3.InvertedFile.from_means(m0)
    for it in lloyd:
        a, b, _ = calg3.assignment_step(c, xi, k)
        ok = (a == it.assign) | (it.gap < 1e-9)
        assert ok.all()
        assert np.allclose(b, it.best, rtol=0, atol=1e-13)
        xi = calg3.update_step(c, a, k, prev=xi)


def test_invalid_inputs_are_statuses():
    c = small_corpus(45, n_docs=20, n_terms=30)
    xi = calg3.InvertedFile.from_means(sk.initial_means(c, dg.init_doc_ids(c.n_docs, 3, 45)))
    with pytest.raises(RuntimeError):
        calg3.assignment_step(c, xi, 3, rows=np.array([0, 20]))
    with pytest.raises(RuntimeError):
        calg3.update_step(c, np.full(c.n_docs, 3, np.int32), 3)


def test_cluster_range_update_is_the_slice_of_the_full_update():
    c = small_corpus(46, n_docs=200, n_terms=90)
    k = 10
    m0 = sk.initial_means(c, dg.init_doc_ids(c.n_docs, k, 46))
    xi = calg3.InvertedFile.from_means(m0)
    a, _, _ = calg3.assignment_step(c, xi, k)
    full = calg3.update_step(c, a, k, prev=xi)
    part = calg3.update_step(c, a, k, prev=xi, clusters=(3, 7))
    sel = (full.c >= 3) & (full.c < 7)
    assert np.array_equal(part.c, full.c[sel]) and np.array_equal(part.u, full.u[sel])
