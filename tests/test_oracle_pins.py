"""Pins of the FP64 oracle to facts other than itself.

Each ``check_*`` states a fact fixed by the paper or by plain mathematics and
checks the oracle against it: a hand-derived worked example (tests/golden),
brute force through a different formula (Euclidean distance, Section 2.2),
closed forms (K = 1, N = K, disjoint supports, duplicate means), Lloyd
invariants (objective never decreases, unit means), the paper's claim that
IVF (Algorithm 3) keeps the Lloyd solution, and its multiplication count
(Eq. 15).  ``test_planted_mistakes_are_caught`` plants plausible mistakes in
the oracle (on the CPU) and requires that some check fails for each.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle.inverted_file as ivf
import oracle.spherical_kmeans as sk
from paper_2002_09094_gb300 import datagen as dg

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "worked_examples.json")


def tiny_corpus(seed, n_docs=60, n_terms=40, mean_len=6.0, zipf_s=0.8):
    spec = dg.CorpusSpec(n_docs=n_docs, n_terms=n_terms, length_kind="poisson", length_mean=mean_len,
                         length_lo=2, length_hi=12, zipf_s=zipf_s, seed=seed)
    return dg.make_corpus(spec)


def dense_rows(corpus):
    rows = []
    for i in range(corpus.n_docs):
        x = [0.0] * corpus.n_terms
        for h in range(int(corpus.row_ptr[i]), int(corpus.row_ptr[i + 1])):
            x[int(corpus.term[h])] = float(corpus.val[h])
        rows.append(x)
    return rows


# ---------------------------------------------------------------- checks


def check_golden():
    spec = json.load(open(GOLDEN))
    for ex in spec["examples"]:
        c = dg.corpus_from_rows(ex["rows"], ex["n_terms"])
        m0 = sk.initial_means(c, ex["init_doc_ids"])
        its = sk.iterate(c, m0, max_iter=len(ex["iterations"]) + 2, empty_policy=ex["empty_policy"])
        tol = ex["tolerance"]
        assert len(its) == len(ex["iterations"]), ex["name"]
        for it, exp in zip(its, ex["iterations"]):
            assert it.assign.tolist() == exp["assign"], ex["name"]
            assert np.allclose(it.best, exp["best"], rtol=0, atol=tol), ex["name"]
            assert np.allclose(it.gap, exp["gap"], rtol=0, atol=tol), ex["name"]
            assert abs(it.objective - exp["objective"]) <= 4 * tol, ex["name"]
            if "n_changed" in exp:
                assert it.n_changed == exp["n_changed"]
            if "sum_norm" in exp:
                assert np.allclose(it.sum_norm, exp["sum_norm"], rtol=0, atol=tol)
            if "means_after" in exp:
                for j, (t, v) in enumerate(exp["means_after"]):
                    mt, mv = it.means_after.row(j)
                    assert mt.tolist() == t, (ex["name"], j)
                    assert np.allclose(mv, v, rtol=0, atol=tol), (ex["name"], j)


def check_euclidean_brute_force(seed=11):
    """argmax_j x.mu_j = argmin_j ||x - mu_j||^2 for unit means (Section 2.2),
    with every distance and mean computed densely in plain Python."""
    c = tiny_corpus(seed)
    k = 7
    ids = dg.init_doc_ids(c.n_docs, k, seed)
    X = dense_rows(c)
    mus = []
    for d in ids:
        nrm = math.sqrt(sum(v * v for v in X[d]))
        mus.append([v / nrm for v in X[d]])
    rho = sk.similarities(c, sk.initial_means(c, ids))
    a, best, gap = sk.assign_from_similarities(rho)
    checked = 0
    for i, x in enumerate(X):
        xx = sum(v * v for v in x)
        dist = [sum((xv - mv) ** 2 for xv, mv in zip(x, mu)) for mu in mus]
        for j in range(k):  # ||x - mu||^2 = ||x||^2 - 2 x.mu + 1
            assert abs(rho[i, j] - (xx + 1.0 - dist[j]) / 2.0) < 1e-12
        order = sorted(range(k), key=lambda j: (dist[j], j))
        if dist[order[1]] - dist[order[0]] > 1e-9:
            assert a[i] == order[0]
            checked += 1
    assert checked > c.n_docs // 2
    # update: normalised member sums, densely in plain Python
    new, norm, sizes = sk.update(c, a, sk.initial_means(c, ids))
    dense_new = new.dense()
    for j in range(k):
        s = [0.0] * c.n_terms
        for i in range(c.n_docs):
            if a[i] == j:
                s = [p + q for p, q in zip(s, X[i])]
        n2 = math.sqrt(sum(v * v for v in s))
        assert sizes[j] == int(np.sum(a == j))
        if n2 > 0:
            assert abs(norm[j] - n2) < 1e-12
            assert np.allclose(dense_new[j], [v / n2 for v in s], rtol=0, atol=1e-12)


def check_dense_equals_sparse(seed=5):
    c = tiny_corpus(seed, n_docs=80)
    m = sk.initial_means(c, dg.init_doc_ids(c.n_docs, 9, seed))
    dense = sk.similarities(c, m)
    old = sk.DENSE_LIMIT_BYTES
    try:
        sk.DENSE_LIMIT_BYTES = 0
        sparse = sk.similarities(c, m)
    finally:
        sk.DENSE_LIMIT_BYTES = old
    assert np.array_equal(dense, sparse)


def check_k1(seed=3):
    c = tiny_corpus(seed)
    its = sk.iterate(c, sk.initial_means(c, [4]), max_iter=3)
    assert all(np.all(it.assign == 0) for it in its)
    total = np.zeros(c.n_terms)
    np.add.at(total, c.term, c.val.astype(np.float64))
    expect = total / np.linalg.norm(total)
    assert np.allclose(its[0].means_after.dense()[0], expect, rtol=0, atol=1e-13)
    assert np.all(np.isinf(its[0].gap))


def check_n_equals_k(seed=4):
    """Every (distinct) object is its own initial mean: by Cauchy-Schwarz it
    keeps itself, with similarity ||x|| = 1."""
    c = tiny_corpus(seed, n_docs=30)
    X = np.array(dense_rows(c))
    # drop duplicate objects so that Cauchy-Schwarz is strict
    _, first = np.unique(X.round(12), axis=0, return_index=True)
    keep = np.sort(first)
    rows = [(c.term[c.row_ptr[i]:c.row_ptr[i + 1]], c.val[c.row_ptr[i]:c.row_ptr[i + 1]]) for i in keep]
    c2 = dg.corpus_from_rows(rows, c.n_terms)
    n = c2.n_docs
    rho = sk.similarities(c2, sk.initial_means(c2, np.arange(n)))
    a, best, _ = sk.assign_from_similarities(rho)
    assert np.array_equal(a, np.arange(n))
    assert np.allclose(best, 1.0, atol=1e-6)


def check_disjoint_supports():
    """Objects on disjoint term sets have similarity exactly 0 across groups."""
    rows = [([0, 1], [0.6, 0.8]), ([1, 2], [0.8, 0.6]), ([5, 6], [0.6, 0.8]), ([6, 7], [0.8, 0.6])]
    c = dg.corpus_from_rows(rows, 8)
    rho = sk.similarities(c, sk.initial_means(c, [0, 2]))
    assert rho[0, 1] == 0.0 and rho[1, 1] == 0.0 and rho[2, 0] == 0.0 and rho[3, 0] == 0.0
    a, _, _ = sk.assign_from_similarities(rho)
    assert a.tolist() == [0, 0, 1, 1]


def check_duplicate_means_tie():
    c = tiny_corpus(21, n_docs=40)
    ids = dg.init_doc_ids(c.n_docs, 3, 21)
    m = sk.initial_means(c, [ids[0], ids[1], ids[0], ids[2]])  # means 0 and 2 identical
    rho = sk.similarities(c, m)
    assert np.array_equal(rho[:, 0], rho[:, 2])
    a, best, gap = sk.assign_from_similarities(rho)
    assert not np.any(a == 2)  # the lower id of the tied pair always wins
    tied = a == 0
    assert np.all(gap[tied] == 0.0)
    # cluster 2 is therefore empty: policy 0 keeps its previous mean exactly,
    # policy 1 leaves it with no terms; the other rows are the same in both
    m0, norm0, sizes0 = sk.update(c, a, m, empty_policy=0)
    m1, norm1, sizes1 = sk.update(c, a, m, empty_policy=1)
    assert sizes0[2] == 0 and norm0[2] == 0.0
    pt, pv = m0.row(2)
    qt, qv = m.row(2)
    assert np.array_equal(pt, qt) and np.array_equal(pv, qv)
    assert m1.row(2)[0].size == 0
    for j in (0, 1, 3):
        assert np.array_equal(m0.row(j)[0], m1.row(j)[0]) and np.array_equal(m0.row(j)[1], m1.row(j)[1])


def check_zero_similarity_object():
    rows = [([0], [1.0]), ([1], [1.0]), ([3], [1.0])]
    c = dg.corpus_from_rows(rows, 4)
    m = sk.initial_means(c, [1, 0])
    rho = sk.similarities(c, m)
    a, best, gap = sk.assign_from_similarities(rho)
    assert a.tolist() == [1, 0, 0] and best[2] == 0.0 and gap[2] == 0.0
    assert sk.zero_similarity_objects(c, m).tolist() == [False, False, True]
    # signed values: object 0 shares both terms with mean 0 = (1, -1)/sqrt(2)
    # and one with mean 1 = (-1, 0), yet 0.5 a - 0.5 a = 0 exactly and
    # 0.5 * (-1) < 0, so its best is 0; it met posting entries and is not
    # counted.  Object 1 (term 5) shares nothing, object 2 (no terms) neither.
    c2 = dg.corpus_from_rows([([0, 1], [0.5, 0.5]), ([5], [1.0]), ([], [])], 6)
    m2 = sk.means_from_rows([0, 2, 3], [0, 1, 0], [1.0, -1.0, -1.0], 6)
    rho2 = sk.similarities(c2, m2)
    assert rho2[0, 0] == 0.0 and rho2[0, 1] < 0.0
    its = sk.iterate(c2, m2, max_iter=1)
    assert sk.zero_similarity_objects(c2, m2).tolist() == [False, True, True]
    assert its[0].n_zero_sim == 2 and its[0].best[0] == 0.0


def check_lloyd_invariants(seed=8):
    """J^r <= sum_j ||s_j^r|| <= J^(r+1); means unit; sum_norm identity."""
    c = tiny_corpus(seed, n_docs=300, n_terms=60, mean_len=8.0)
    its = sk.iterate(c, sk.initial_means(c, dg.init_doc_ids(c.n_docs, 12, seed)), max_iter=12)
    for r, it in enumerate(its):
        jp = float(np.sum(it.sum_norm))
        assert it.objective <= jp + 1e-12
        if r + 1 < len(its):
            assert jp <= its[r + 1].objective + 1e-12
        # closed form: sum_{i in C_j} x_i . (s_j/||s_j||) = ||s_j||
        rho_new = sk.similarities(c, it.means_after)
        own = rho_new[np.arange(c.n_docs), it.assign]
        per = np.bincount(it.assign, weights=own, minlength=12)
        live = it.sizes > 0
        assert np.allclose(per[live], it.sum_norm[live], rtol=0, atol=1e-12)
        nrm = np.sqrt(np.bincount(np.repeat(np.arange(12), np.diff(it.means_after.ptr)),
                                  weights=it.means_after.val ** 2, minlength=12))
        assert np.allclose(nrm, 1.0, rtol=0, atol=1e-12)
        assert np.all(np.diff(its[r].assign.shape) == 0)


def check_ivf_equals_lloyd(seed=9):
    """Algorithm 3 keeps the Lloyd solution from the same initial state; with
    identical means its rho equals Eq. 8's bit for bit (it only skips exact
    zero products)."""
    c = tiny_corpus(seed, n_docs=120, n_terms=50)
    k = 6
    m0 = sk.initial_means(c, dg.init_doc_ids(c.n_docs, k, seed))
    xi0 = ivf.inverted_file_from_means(m0)
    a_ivf, best_ivf, rho_ivf, _ = ivf.assignment_step(c, xi0, k)
    rho = sk.similarities(c, m0)
    assert np.array_equal(np.array(rho_ivf), rho)
    lloyd = sk.iterate(c, m0, max_iter=8)
    alg3 = ivf.iterate(c, xi0, k, max_iter=8)
    assert len(lloyd) == len(alg3)
    for it, (a3, b3, xi3) in zip(lloyd, alg3):
        assert it.assign.tolist() == a3
        assert np.allclose(it.best, b3, rtol=0, atol=1e-13)
        g = it.gap[np.isfinite(it.gap)]
        assert np.all((g == 0.0) | (g > 1e-9))  # exact ties or clear gaps: no near-ties blur it
        # same means (Algorithm 3 divides by |C_j| before normalising)
        mine = it.means_after
        for j in range(k):
            mt, mv = mine.row(j)
            t3 = [p for p in range(c.n_terms) for (cc, _) in xi3[p] if cc == j]
            u3 = [u for p in range(c.n_terms) for (cc, u) in xi3[p] if cc == j]
            assert mt.tolist() == t3
            assert np.allclose(mv, u3, rtol=0, atol=1e-14)


def check_multiplication_count(seed=13):
    """Eq. 15 equals Algorithm 3's counted multiplications and sum_p (no)_p (nc)_p."""
    c = tiny_corpus(seed, n_docs=100, n_terms=45)
    m = sk.initial_means(c, dg.init_doc_ids(c.n_docs, 8, seed))
    xi = ivf.inverted_file_from_means(m)
    _, _, _, mults = ivf.assignment_step(c, xi, 8)
    no = np.bincount(c.term, minlength=c.n_terms)
    nc = np.array([len(xi[p]) for p in range(c.n_terms)])
    assert sk.multiplication_count(c, m) == mults == int(np.sum(no * nc))
    # memory identity: sum_p (nc)_p = sum_j (ntm)_j (Section 5.3)
    assert int(nc.sum()) == int(m.ptr[-1])


def _brute_force_assignment(rows_dense, mus):
    """Plain-Python similarities, lowest-id argmax, best and top-2 gap."""
    out = []
    for x in rows_dense:
        rho = [sum(a * b for a, b in zip(x, mu)) for mu in mus]
        order = sorted(range(len(mus)), key=lambda j: (-rho[j], j))
        out.append((order[0], rho[order[0]], rho[order[0]] - rho[order[1]]))
    return out


def check_lockstep_checker(seed=17):
    """The lockstep comparison of a GPU assignment with the FP64 argmax under
    the same means (the per-iteration protocol on Algorithm 2's assignment,
    Eq. 4) counts exactly the planted disagreements.

    Expected values come from a plain-Python brute force: means
    mu_j = x_{d_j} / ||x_{d_j}|| with a duplicated mean (exact ties, gap 0),
    plus a hand-built pair of means 5e-9 apart in similarity (a near-tie
    below the 1e-6 exclusion) and an object sharing no term with any mean.
    """
    c = tiny_corpus(seed, n_docs=70)
    ids = [int(d) for d in dg.init_doc_ids(c.n_docs, 5, seed)]
    ids = ids + [ids[1]]                                   # mean 5 duplicates mean 1
    X = dense_rows(c)
    mus = []
    for d in ids:
        nrm = math.sqrt(sum(v * v for v in X[d]))
        mus.append([v / nrm for v in X[d]])
    bf = _brute_force_assignment(X, mus)
    a_bf = np.array([t[0] for t in bf], dtype=np.int32)
    best_bf = np.array([t[1] for t in bf])
    gap_bf = np.array([t[2] for t in bf])
    excl_bf = gap_bf < 1e-6
    assert excl_bf.any() and (~excl_bf).sum() > 20
    means = sk.initial_means(c, ids)

    # 1. the true assignment: nothing flagged; exactly the near-ties excluded
    rep = sk.lockstep_check(c, means, a_bf, best_bf)
    assert rep["checked"] == c.n_docs and rep["mismatches"] == 0
    assert rep["excluded"] == int(excl_bf.sum())
    assert rep["best_ok"] and rep["max_best_err"] <= 1e-12

    # 2. wrong clusters on clear objects are counted, on excluded ones ignored
    clear = np.flatnonzero(~excl_bf)
    wrong = clear[::4]
    ga = a_bf.copy()
    ga[wrong] = (ga[wrong] + 1) % len(ids)
    ga[np.flatnonzero(excl_bf)] = (a_bf[excl_bf] + 2) % len(ids)
    rep = sk.lockstep_check(c, means, ga, best_bf)
    assert rep["mismatches"] == wrong.size
    assert rep["mismatch_rows"] == sorted(wrong.tolist())[:20]

    # 3. a row subset reads the full-length outputs at those rows: every other
    #    position holds an invalid cluster id and a wrong best
    rows = np.arange(c.n_docs - 1, -1, -3)
    ga = np.full(c.n_docs, -1, dtype=np.int32)
    gb = np.full(c.n_docs, 5.0)
    ga[rows] = a_bf[rows]
    gb[rows] = best_bf[rows]
    rep = sk.lockstep_check(c, means, ga, gb, rows=rows)
    assert rep["checked"] == rows.size and rep["mismatches"] == 0 and rep["best_ok"]
    assert rep["excluded"] == int(excl_bf[rows].sum())
    ga[rows[1]] = (a_bf[rows[1]] + 1) % len(ids)
    if not excl_bf[rows[1]]:
        assert sk.lockstep_check(c, means, ga, gb, rows=rows)["mismatches"] == 1

    # 4. the best-similarity tolerance: 2e-5 off fails, 5e-6 off passes
    j = int(clear[0])
    gb = best_bf.copy()
    gb[j] += 2e-5
    rep = sk.lockstep_check(c, means, a_bf, gb)
    assert not rep["best_ok"] and abs(rep["max_best_err"] - 2e-5) < 1e-12
    gb[j] = best_bf[j] - 5e-6
    assert sk.lockstep_check(c, means, a_bf, gb)["best_ok"]

    # 5. a hand-built near-tie (gap 1 - 1/sqrt(1 + 1e-8) ~ 5e-9) and an
    #    object with no shared term (gap 0) are excluded; a gap of ~8e-5 is not
    c2 = dg.corpus_from_rows([([0], [1.0]), ([0, 1], [0.6, 0.8]), ([2], [1.0])], 3)
    m2 = sk.means_from_rows([0, 1, 3], [0, 0, 1], [1.0, 1.0, 1e-4], 3)
    rep = sk.lockstep_check(c2, m2, [1, 0, 1], [1.0, 0.6, 0.0])
    assert rep["excluded"] == 2 and rep["mismatches"] == 1 and rep["mismatch_rows"] == [1]


CHECKS = [check_golden, check_euclidean_brute_force, check_dense_equals_sparse, check_k1,
          check_n_equals_k, check_disjoint_supports, check_duplicate_means_tie,
          check_zero_similarity_object, check_lloyd_invariants, check_ivf_equals_lloyd,
          check_multiplication_count, check_lockstep_checker]


@pytest.mark.parametrize("check", CHECKS, ids=[f.__name__ for f in CHECKS])
def test_oracle_pin(check):
    check()


# ------------------------------------------------------- planted mistakes


def _mut_drop_last_term(orig):
    def similarities(corpus, means, rows=None, chunk=2048):
        keep = np.ones(corpus.nnz, dtype=bool)
        keep[corpus.row_ptr[1:][np.diff(corpus.row_ptr) > 0] - 1] = False
        lens = np.diff(corpus.row_ptr) - (np.diff(corpus.row_ptr) > 0)
        rp = np.zeros_like(corpus.row_ptr)
        np.cumsum(lens, out=rp[1:])
        c2 = dg.Corpus(row_ptr=rp, term=corpus.term[keep], val=corpus.val[keep], n_terms=corpus.n_terms)
        return orig(c2, means, rows, chunk)
    return "similarities", similarities


def _mut_highest_id_ties(orig):
    def assign_from_similarities(rho):
        a, best, gap = orig(rho)
        k = rho.shape[1]
        a2 = (k - 1 - np.argmax(rho[:, ::-1], axis=1)).astype(np.int32)
        return a2, best, gap
    return "assign_from_similarities", assign_from_similarities


def _mut_no_normalisation(orig):
    def update(corpus, assign, prev, empty_policy=0):
        m, norm, sizes = orig(corpus, assign, prev, empty_policy)
        owner = np.repeat(np.arange(m.k), np.diff(m.ptr))
        scale = np.where(norm > 0, norm, 1.0)[owner]
        return sk.Means(ptr=m.ptr, term=m.term, val=m.val * scale, n_terms=m.n_terms), norm, sizes
    return "update", update


def _mut_shifted_cluster(orig):
    def cluster_sums(corpus, assign, k):
        return orig(corpus, (np.asarray(assign) + 1) % k, k)
    return "cluster_sums", cluster_sums


def _mut_reversed_means(orig):
    def similarities(corpus, means, rows=None, chunk=2048):
        return orig(corpus, means, rows, chunk)[:, ::-1].copy()
    return "similarities", similarities


def _mut_gap_sign(orig):
    def assign_from_similarities(rho):
        a, best, gap = orig(rho)
        return a, best, -gap
    return "assign_from_similarities", assign_from_similarities


def _mut_empty_loses_mean(orig):
    def update(corpus, assign, prev, empty_policy=0):
        return orig(corpus, assign, prev, 1)   # empty clusters never keep their previous mean
    return "update", update


def _mut_shifted_object(orig):
    def cluster_sums(corpus, assign, k):
        a = np.asarray(assign)
        return orig(corpus, np.roll(a, 1), k)  # x_{i} summed into the cluster of x_{i-1}
    return "cluster_sums", cluster_sums


def _mut_negated_similarity(orig):
    def similarities(corpus, means, rows=None, chunk=2048):
        return -orig(corpus, means, rows, chunk)
    return "similarities", similarities


def _mut_count_per_term_not_per_entry(orig):
    def multiplication_count(corpus, means):
        return int(corpus.nnz)                 # one product per object term instead of per posting entry
    return "multiplication_count", multiplication_count


def _mut_no_update(orig):
    def update(corpus, assign, prev, empty_policy=0):
        m, norm, sizes = orig(corpus, assign, prev, empty_policy)
        return prev, norm, sizes               # means never move
    return "update", update


def _lockstep_with(bug):
    """lockstep_check restated with one planted slip."""
    def lockstep_check(corpus, means_prev, gpu_assign, gpu_best=None, rows=None,
                       gap_exclusion=1e-6, best_tol=1e-5):
        rows_arr = np.arange(corpus.n_docs) if rows is None else np.asarray(rows, dtype=np.int64)
        a, best, gap = sk.assign_from_similarities(sk.similarities(corpus, means_prev, rows_arr))
        if bug == "unindexed":
            ga = np.asarray(gpu_assign)[:rows_arr.size]
        else:
            ga = np.asarray(gpu_assign)[rows_arr]
        excluded = gap >= gap_exclusion if bug == "inverted_exclusion" else gap < gap_exclusion
        mism = (ga != a) & ~excluded
        rep = {"checked": int(rows_arr.size), "excluded": int(excluded.sum()),
               "mismatches": int(mism.sum()), "mismatch_rows": rows_arr[mism][:20].tolist()}
        if gpu_best is not None:
            gb = np.asarray(gpu_best, dtype=np.float64)
            gb = gb[:rows_arr.size] if bug == "unindexed" else gb[rows_arr]
            rep["max_best_err"] = float(np.max(np.abs(gb - best))) if rows_arr.size else 0.0
            rep["best_ok"] = True if bug == "best_tol_ignored" else rep["max_best_err"] <= best_tol
        rep["oracle_assign"], rep["oracle_best"], rep["oracle_gap"] = a, best, gap
        return rep
    return lockstep_check


def _mut_zero_sim_by_best_value(orig):
    def zero_similarity_objects(corpus, means):
        _, best, _ = sk.assign_from_similarities(sk.similarities(corpus, means))
        return best == 0.0                     # counts cancelling signed objects too
    return "zero_similarity_objects", zero_similarity_objects


def _mut_lockstep_inverted_exclusion(orig):
    return "lockstep_check", _lockstep_with("inverted_exclusion")


def _mut_lockstep_unindexed_rows(orig):
    return "lockstep_check", _lockstep_with("unindexed")


def _mut_lockstep_best_tol_ignored(orig):
    return "lockstep_check", _lockstep_with("best_tol_ignored")


MUTANTS = [_mut_drop_last_term, _mut_highest_id_ties, _mut_no_normalisation, _mut_shifted_cluster,
           _mut_reversed_means, _mut_gap_sign, _mut_empty_loses_mean, _mut_shifted_object,
           _mut_negated_similarity, _mut_count_per_term_not_per_entry, _mut_no_update,
           _mut_lockstep_inverted_exclusion, _mut_lockstep_unindexed_rows, _mut_lockstep_best_tol_ignored,
           _mut_zero_sim_by_best_value]


@pytest.mark.parametrize("mutant", MUTANTS, ids=[m.__name__ for m in MUTANTS])
def test_planted_mistakes_are_caught(mutant, monkeypatch):
    name, fn = mutant(getattr(sk, name_of(mutant)))
    monkeypatch.setattr(sk, name, fn)
    failed = []
    for check in CHECKS:
        try:
            check()
        except (AssertionError, ValueError, IndexError):
            failed.append(check.__name__)
    assert failed, f"no pin caught {mutant.__name__}"


def name_of(mutant):
    return {
        _mut_drop_last_term: "similarities", _mut_highest_id_ties: "assign_from_similarities",
        _mut_no_normalisation: "update", _mut_shifted_cluster: "cluster_sums",
        _mut_reversed_means: "similarities", _mut_gap_sign: "assign_from_similarities",
        _mut_empty_loses_mean: "update", _mut_shifted_object: "cluster_sums",
        _mut_negated_similarity: "similarities", _mut_count_per_term_not_per_entry: "multiplication_count",
        _mut_no_update: "update", _mut_lockstep_inverted_exclusion: "lockstep_check",
        _mut_lockstep_unindexed_rows: "lockstep_check", _mut_lockstep_best_tol_ignored: "lockstep_check",
        _mut_zero_sim_by_best_value: "zero_similarity_objects",
    }[mutant]
