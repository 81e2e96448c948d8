"""The seeded input generator: determinism and the stated distributions."""
import numpy as np
import pytest

from paper_2002_09094_gb300 import datagen as dg


def small_spec(**kw):
    base = dict(n_docs=3000, n_terms=5000, length_kind="poisson", length_mean=30.0, length_lo=5,
                length_hi=120, zipf_s=1.1, seed=7)
    base.update(kw)
    return dg.CorpusSpec(**base)


def test_same_seed_same_bytes_and_different_seed_differs():
    a = dg.make_corpus(small_spec())
    b = dg.make_corpus(small_spec())
    c = dg.make_corpus(small_spec(seed=8))
    assert np.array_equal(a.row_ptr, b.row_ptr)
    assert np.array_equal(a.term, b.term)
    assert np.array_equal(a.val.view(np.uint32), b.val.view(np.uint32))
    assert not np.array_equal(a.term[:1000], c.term[:1000])


def test_rows_sorted_unique_in_range_and_unit_norm():
    c = dg.make_corpus(small_spec(length_kind="lognormal", length_mean=40.0))
    r = c.row_ptr
    lens = np.diff(r)
    assert lens.min() >= 5 and lens.max() <= 120
    row_of = np.repeat(np.arange(c.n_docs), lens)
    # strictly ascending inside each row
    same_row = row_of[1:] == row_of[:-1]
    assert np.all(np.diff(c.term.astype(np.int64))[same_row] > 0)
    assert c.term.min() >= 0 and c.term.max() < c.n_terms
    assert np.all(c.val > 0)
    nrm2 = np.bincount(row_of, weights=c.val.astype(np.float64) ** 2)
    assert np.max(np.abs(nrm2 - 1.0)) < 1e-6


def test_zipf_head_and_length_mean():
    c = dg.make_corpus(small_spec(n_docs=20000, length_mean=20.0))
    df = np.bincount(c.term, minlength=c.n_terms)
    # document frequency falls with rank over the head
    assert np.all(np.diff(df[:8]) < 0)
    lens = np.diff(c.row_ptr)
    assert abs(lens.mean() - 20.0) < 0.5  # Poisson(20), clipping at 5 and 120 moves it a little


def test_init_doc_ids_distinct_and_seeded():
    a = dg.init_doc_ids(1000, 100, 3)
    assert len(set(a.tolist())) == 100
    assert np.array_equal(a, dg.init_doc_ids(1000, 100, 3))
    with pytest.raises(ValueError):
        dg.init_doc_ids(10, 11, 0)


def test_batched_instances_within_ranges():
    ws = dg.batched_workloads(n_instances=16)
    for w in ws:
        assert 2000 <= w.corpus.n_docs <= 200000
        assert 16 <= w.k <= 2000 and w.k <= w.corpus.n_docs
        assert 10000 <= w.corpus.n_terms <= 100000
        assert 20.0 <= w.corpus.length_mean <= 150.0
