"""Lockstep comparison of the CUDA path (through the C ABI) with the FP64 oracle.

At iteration r the oracle takes the GPU's previous assignment, forms its own
FP64 means from it, and checks that the GPU's assignment equals the FP64
argmax for every object whose FP64 top-2 gap is at least 1e-6, that the
GPU's best similarity is within 1e-5 of the FP64 one, and that the GPU's FP64
master means equal the oracle's.  Each checked object's best is also held
to the library's own per-result error statement (ivf_get_err_bound):
|best_i - rho_i| <= E_i, with rho_i the FP64 similarity to the returned
cluster, and the count of objects sharing no term with any mean is compared
with the oracle's.
"""
from __future__ import annotations

import numpy as np

import oracle.spherical_kmeans as sk
from paper_2002_09094_gb300 import ivf

GAP_EXCLUSION = 1e-6
BEST_TOL = 1e-5
MEAN_TOL = 1e-12


def means_report(gpu_means, oracle_means) -> dict:
    gp, gt, gv = gpu_means
    same = np.array_equal(gp, oracle_means.ptr) and np.array_equal(gt, oracle_means.term)
    diff = float(np.max(np.abs(gv - oracle_means.val))) if same and gv.size else (0.0 if same else np.inf)
    return {"structure_equal": bool(same), "max_diff": diff}


def lockstep(corpus, k, doc_ids, iters, rows=None, best_tol=BEST_TOL, means_rows=None, **kw):
    """Run `iters` GPU iterations (assign + update) with oracle checks; returns reports.

    Initial means: documents doc_ids, or explicit cluster-major rows
    means_rows = (ptr, term, val32) when given.
    """
    m = ivf.IVF(corpus.row_ptr, corpus.term, corpus.val, corpus.n_terms, k, **kw)
    empty_policy = kw.get("empty_policy", 0)
    try:
        if means_rows is None:
            m.set_means_from_docs(doc_ids)
            means = sk.initial_means(corpus, doc_ids)
        else:
            mp, mt, mv = means_rows
            m.set_means(mp, np.asarray(mt, np.int32), np.asarray(mv, np.float32))
            means = sk.means_from_rows(mp, mt, np.asarray(mv, np.float32).astype(np.float64), corpus.n_terms)
        prev = None
        reports = []
        for r in range(1, iters + 1):
            st = m.assign()
            a, b, g = m.get_assign(), m.get_best(), m.get_gap()
            e = m.get_err_bound()
            sample = rows
            if rows is not None:  # sampled objects plus every object the GPU flagged as a near-tie
                flagged = np.flatnonzero(g <= 1e-3)
                sample = np.unique(np.concatenate([np.asarray(rows, dtype=np.int64), flagged]))
            rep = sk.lockstep_check(corpus, means, a, b, rows=sample, gap_exclusion=GAP_EXCLUSION,
                                    best_tol=best_tol)
            rep["r"] = r
            rep["best_tol"] = best_tol
            rep["stats"] = st
            rep["mult_count"] = sk.multiplication_count(corpus, means)
            rep["n_changed_expected"] = corpus.n_docs if prev is None else int(np.count_nonzero(a != prev))
            rep["objective_expected"] = float(np.sum(rep["oracle_best"])) if sample is None else None
            rep["gpu_assign"] = a
            rep["gpu_best"] = b
            rep["gpu_gap"] = g
            rep["n_zero_sim_expected"] = int(np.count_nonzero(sk.zero_similarity_objects(corpus, means)))
            rep.update(err_bound_report(corpus, means, rep, sample, a, b, e))
            m.update()
            new, norm, sizes = sk.update(corpus, a, means, empty_policy)
            rep["means"] = means_report(m.get_means(), new)
            rep["oracle_means_after"] = new
            means = new
            prev = a
            reports.append(rep)
        return reports
    finally:
        m.close()


def err_bound_report(corpus, means, rep, rows, gpu_assign, gpu_best, gpu_err) -> dict:
    """|best_i - rho_i(a_i)| against the GPU's stated bound E_i on the checked
    rows, rho in FP64 for the cluster the GPU returned (which differs from the
    oracle's only for excluded near-ties)."""
    rows = np.arange(corpus.n_docs) if rows is None else np.asarray(rows, dtype=np.int64)
    oa = rep["oracle_assign"]
    rho_gpu_cluster = np.array(rep["oracle_best"], dtype=np.float64)
    ga = np.asarray(gpu_assign)[rows]
    diff = np.flatnonzero(ga != oa)
    if diff.size:
        rho = sk.similarities(corpus, means, rows[diff])
        rho_gpu_cluster[diff] = rho[np.arange(diff.size), ga[diff]]
    err = np.abs(np.asarray(gpu_best, np.float64)[rows] - rho_gpu_cluster)
    bound = np.asarray(gpu_err, np.float64)[rows]
    ratio = err / np.maximum(bound, 1e-30)
    return {"err_within_bound": bool(np.all(err <= bound + 1e-12)),
            "max_err_over_bound": float(ratio.max()) if rows.size else 0.0,
            "max_abs_err": float(err.max()) if rows.size else 0.0,
            "max_bound": float(bound.max()) if rows.size else 0.0}


def assert_report_ok(rep, check_best=True, check_means=True, check_objective=True):
    assert rep["mismatches"] == 0, (rep["r"], rep["mismatches"], rep["mismatch_rows"])
    assert rep["err_within_bound"], (rep["r"], rep["max_err_over_bound"], rep["max_abs_err"])
    assert rep["stats"]["n_zero_sim"] == rep["n_zero_sim_expected"], (rep["stats"]["n_zero_sim"],
                                                                       rep["n_zero_sim_expected"])
    if check_best:
        assert rep["best_ok"], (rep["r"], rep["max_best_err"])
    st = rep["stats"]
    assert st["entries_visited"] == rep["mult_count"], (st["entries_visited"], rep["mult_count"])
    assert st["n_changed"] == rep["n_changed_expected"]
    if check_objective and rep["objective_expected"] is not None:
        n = rep["checked"]
        assert abs(st["objective"] - rep["objective_expected"]) / n <= rep["best_tol"]
    if check_means:
        assert rep["means"]["structure_equal"], rep["r"]
        assert rep["means"]["max_diff"] <= MEAN_TOL, rep["means"]
