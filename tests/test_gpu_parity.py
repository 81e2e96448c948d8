"""CUDA path vs the FP64 oracle, through the C ABI (GPU only).

Bar: assignments equal to the FP64 argmax for every object whose FP64 top-2
gap is >= 1e-6; best similarity within 1e-5 absolute (FP32 storage); the
objective per object within 1e-5; FP64 master means equal to the oracle's
update of the same assignment within 1e-12; the visited-entry counter equal
to Eq. 15's multiplication count exactly.
"""
import numpy as np
import pytest

import oracle.spherical_kmeans as sk
from paper_2002_09094_gb300 import datagen as dg
from paper_2002_09094_gb300 import ivf
from tests.parity_util import assert_report_ok, lockstep

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()


def corpus_for(n_docs, n_terms, mean_len=30.0, zipf=1.1, seed=1, kind="poisson", lo=3, hi=200):
    return dg.make_corpus(dg.CorpusSpec(n_docs=n_docs, n_terms=n_terms, length_kind=kind, length_mean=mean_len,
                                        length_lo=lo, length_hi=hi, zipf_s=zipf, seed=seed))


# ------------------------------------------------------------ trajectories


def test_small_workload_ten_iterations_lockstep():
    """10,000 Poisson(50) docs, 20,000 terms, Zipf 1.1, K = 100, 10 iterations."""
    w = dg.SMALL
    c = dg.make_corpus(w.corpus)
    ids = dg.init_doc_ids(c.n_docs, w.k, w.init_seed)
    reps = lockstep(c, w.k, ids, w.iterations)
    for rep in reps:
        assert_report_ok(rep)
    # free-running: with no excluded object assigned differently, the GPU
    # trajectory is the oracle's own trajectory from the same initial state
    free = sk.iterate(c, sk.initial_means(c, ids), w.iterations, stop_on_convergence=False)
    diverged = False
    for rep, it in zip(reps, free):
        if not diverged:
            same = np.array_equal(rep["gpu_assign"], it.assign)
            if not same:
                excl = it.gap < 1e-6
                assert np.all((rep["gpu_assign"] == it.assign) | excl)
                diverged = True


@pytest.mark.parametrize("k_tile", [512, 1024, 2048])
def test_tiled_accumulator_equals_untiled(k_tile):
    c = corpus_for(4000, 6000, mean_len=40.0)
    k = 3000
    ids = dg.init_doc_ids(c.n_docs, k, 5)
    out = {}
    for kt in (0, k_tile):
        with ivf.IVF(c.row_ptr, c.term, c.val, c.n_terms, k, k_tile=kt if kt else 65536) as m:
            m.set_means_from_docs(ids)
            st = m.assign()
            out[kt] = (m.get_assign(), m.get_best(), m.get_gap(), st["entries_visited"], m.info()["k_tile"])
    assert out[k_tile][4] == k_tile
    for q in range(3):
        assert np.array_equal(out[0][q].view(np.uint32), out[k_tile][q].view(np.uint32))
    assert out[0][3] == out[k_tile][3]
    reps = lockstep(c, k, ids, 2, k_tile=k_tile)
    for rep in reps:
        assert_report_ok(rep)


@pytest.mark.parametrize("k", [1023, 1024, 1025, 4095, 4096, 4097])
def test_cluster_counts_around_tile_edges(k):
    c = corpus_for(6000, 5000, mean_len=25.0, seed=k)
    ids = dg.init_doc_ids(c.n_docs, k, k)
    for kt in (0, 1024):
        for rep in lockstep(c, k, ids, 2, k_tile=kt):
            assert_report_ok(rep)


@pytest.mark.parametrize("storage,tol", [("f16", 3e-3), ("bf16", 2.5e-2)])
def test_mixed_precision_assignments_equal_fp64(storage, tol):
    c = corpus_for(6000, 8000, mean_len=40.0, seed=3)
    k = 150
    ids = dg.init_doc_ids(c.n_docs, k, 9)
    reps = lockstep(c, k, ids, 3, storage=storage, best_tol=tol)
    for rep in reps:
        assert_report_ok(rep)
    assert sum(r["stats"]["n_rescored"] for r in reps) > 0


def test_rescore_off_still_close():
    c = corpus_for(3000, 4000, seed=4)
    k = 60
    ids = dg.init_doc_ids(c.n_docs, k, 4)
    rep = lockstep(c, k, ids, 1, rescore=False)[0]
    assert rep["best_ok"]
    assert rep["stats"]["n_flagged"] == 0 and rep["stats"]["n_rescored"] == 0


# ------------------------------------------------------------- batched


def test_batched_equals_single_instances():
    ws = dg.batched_workloads(n_instances=6, n_range=(500, 3000), k_range=(4, 300), d_range=(1000, 6000),
                              nnz_range=(10.0, 60.0), iterations=4)
    cs = [dg.make_corpus(w.corpus) for w in ws]
    ids = [dg.init_doc_ids(c.n_docs, w.k, w.init_seed) for w, c in zip(ws, cs)]
    single = []
    for w, c, d in zip(ws, cs, ids):
        with ivf.IVF(c.row_ptr, c.term, c.val, c.n_terms, w.k) as m:
            m.set_means_from_docs(d)
            done, conv, _ = m.iterate(4)
            single.append((m.get_assign(), m.get_means()))
    inst_docs = np.concatenate([[0], np.cumsum([c.n_docs for c in cs])]).astype(np.int64)
    offs = np.concatenate([[0], np.cumsum([c.nnz for c in cs])])
    row_ptr = np.concatenate([c.row_ptr[:-1] + o for c, o in zip(cs, offs)] + [[offs[-1]]]).astype(np.int64)
    term = np.concatenate([c.term for c in cs])
    val = np.concatenate([c.val for c in cs])
    with ivf.BatchedIVF(row_ptr, term, val, inst_docs, [c.n_terms for c in cs], [w.k for w in ws]) as m:
        m.set_means_from_docs(np.concatenate(ids))
        for _ in range(4):
            m.assign(stats=False)
            m.update()
        a = m.get_assign()
        ptr, mt, mv = m.get_means()
    kof = np.concatenate([[0], np.cumsum([w.k for w in ws])])
    for b, (sa, (sp, st_, sv)) in enumerate(single):
        assert np.array_equal(a[inst_docs[b]:inst_docs[b + 1]], sa)
        lo, hi = ptr[kof[b]], ptr[kof[b + 1]]
        assert np.array_equal(ptr[kof[b]:kof[b + 1] + 1] - lo, sp)
        assert np.array_equal(mt[lo:hi], st_)
        assert np.array_equal(mv[lo:hi], sv)


@pytest.mark.parametrize("kernel,seed,n_inst", [("sparse", 77, 4), ("dense_head", 77, 4), ("auto", 85, 5),
                                                ("dense_head", 88, 5), ("auto", 98, 32)])
def test_batched_lockstep_against_oracle(kernel, seed, n_inst):
    """Seed 77: K in two of the classes the batched assignment launches
    separately (<= 1,024 and larger); seeds 85 and 88: three classes; seed 98:
    32 instances with K in six classes (<= 128, <= 256, <= 512, <= 1,024,
    <= 1,536, <= 2,048)."""
    k_hi = {4: 1500, 5: 1600, 32: 2000}[n_inst]
    ws = dg.batched_workloads(n_instances=n_inst, n_range=(800, 2000), k_range=(8, k_hi),
                              d_range=(2000, 5000), nnz_range=(15.0, 50.0), iterations=3, seed=seed)
    if n_inst == 32:
        ks = [w.k for w in ws]
        assert all(any(lo < k <= hi for k in ks) for lo, hi in [(0, 128), (128, 256), (256, 512), (512, 1024),
                                                                (1024, 1536), (1536, 2048)])
    cs = [dg.make_corpus(w.corpus) for w in ws]
    ids = [dg.init_doc_ids(c.n_docs, w.k, w.init_seed) for w, c in zip(ws, cs)]
    inst_docs = np.concatenate([[0], np.cumsum([c.n_docs for c in cs])]).astype(np.int64)
    offs = np.concatenate([[0], np.cumsum([c.nnz for c in cs])])
    row_ptr = np.concatenate([c.row_ptr[:-1] + o for c, o in zip(cs, offs)] + [[offs[-1]]]).astype(np.int64)
    with ivf.BatchedIVF(row_ptr, np.concatenate([c.term for c in cs]), np.concatenate([c.val for c in cs]),
                        inst_docs, [c.n_terms for c in cs], [w.k for w in ws], kernel=kernel) as m:
        m.set_means_from_docs(np.concatenate(ids))
        means = [sk.initial_means(c, d) for c, d in zip(cs, ids)]
        for r in range(3):
            st = m.assign()
            a, bst = m.get_assign(), m.get_best()
            total_mult = 0
            for b, c in enumerate(cs):
                sl = slice(inst_docs[b], inst_docs[b + 1])
                rep = sk.lockstep_check(c, means[b], a[sl], bst[sl])
                assert rep["mismatches"] == 0 and rep["best_ok"]
                total_mult += sk.multiplication_count(c, means[b])
                means[b] = sk.update(c, a[sl], means[b])[0]
            assert st["entries_visited"] == total_mult
            changed = m.get_changed_per_instance()
            assert changed.sum() == st["n_changed"]
            m.update()


# ------------------------------------------------------------ edge cases


def test_k_equals_one_closed_form():
    c = corpus_for(500, 300, seed=8)
    with ivf.IVF(c.row_ptr, c.term, c.val, c.n_terms, 1) as m:
        m.set_means_from_docs([7])
        m.iterate(3)
        assert np.all(m.get_assign() == 0)
        ptr, term, val = m.get_means()
    total = np.zeros(c.n_terms)
    np.add.at(total, c.term, c.val.astype(np.float64))
    nz = np.flatnonzero(total)
    assert np.array_equal(term, nz)
    assert np.allclose(val, total[nz] / np.linalg.norm(total), atol=1e-13, rtol=0)


def test_each_document_its_own_cluster():
    c = corpus_for(400, 50000, mean_len=20.0, zipf=0.6, seed=10)  # distinct docs (wide vocabulary)
    n = c.n_docs
    with ivf.IVF(c.row_ptr, c.term, c.val, c.n_terms, n) as m:
        m.set_means_from_docs(np.arange(n, dtype=np.int32))
        m.assign()
        assert np.array_equal(m.get_assign(), np.arange(n))
        assert np.allclose(m.get_best(), 1.0, atol=1e-6)


def test_duplicate_means_tie_lowest_id_and_empty_cluster_policies():
    c = corpus_for(800, 500, seed=12)
    ids = dg.init_doc_ids(c.n_docs, 5, 12)
    dup = [ids[0], ids[1], ids[2], ids[0], ids[3]]  # mean 3 == mean 0
    lens = [c.row_ptr[d + 1] - c.row_ptr[d] for d in dup]
    ptr = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    term = np.concatenate([c.term[c.row_ptr[d]:c.row_ptr[d + 1]] for d in dup])
    val = np.concatenate([c.val[c.row_ptr[d]:c.row_ptr[d + 1]] for d in dup])
    for policy in (0, 1):
        reps = lockstep(c, 5, None, 3, empty_policy=policy, means_rows=(ptr, term, val))
        for rep in reps:
            assert_report_ok(rep)
        assert not np.any(reps[0]["gpu_assign"] == 3)  # the higher id of a tie never wins
        kept = reps[0]["oracle_means_after"].row(3)[0]
        assert np.array_equal(kept, term[ptr[3]:ptr[4]]) if policy == 0 else kept.size == 0


def test_zero_similarity_objects_and_empty_rows():
    rows = [([0, 1], [0.6, 0.8]), ([2], [1.0]), ([5, 6], [0.8, 0.6]), ([], []), ([9], [1.0]), ([1, 2], [0.6, 0.8])]
    c = dg.corpus_from_rows(rows, 10)
    with ivf.IVF(c.row_ptr, c.term, c.val, c.n_terms, 2) as m:
        m.set_means_from_docs([0, 1])
        st = m.assign()
        a, b = m.get_assign(), m.get_best()
    assert a.tolist() == [0, 1, 0, 0, 0, 1]
    assert b[2] == 0.0 and b[3] == 0.0 and b[4] == 0.0
    assert st["n_zero_sim"] == 3


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_zero_similarity_counts_objects_without_entries(storage):
    """Signed values: object 0 shares both terms with mean 0 = (1, -1)/sqrt(2)
    and 0.5 a - 0.5 a cancels exactly, while mean 1 gives -0.5, so its best is
    0 although it met posting entries; it is not counted.  Objects 1 (a term
    no mean has) and 2 (no terms) are."""
    c = dg.corpus_from_rows([([0, 1], [0.5, 0.5]), ([5], [1.0]), ([], [])], 6)
    rows = (np.array([0, 2, 3], np.int64), np.array([0, 1, 0], np.int32), np.array([1.0, -1.0, -1.0], np.float32))
    reps = lockstep(c, 2, None, 2, means_rows=rows, storage=storage, best_tol=1e-5 if storage == "f32" else 2.5e-2)
    for rep in reps:
        assert_report_ok(rep)
    assert reps[0]["gpu_best"][0] == 0.0 and reps[0]["stats"]["n_zero_sim"] == 2


@pytest.mark.parametrize("n", [1, 2, 33, 1000])
def test_ragged_tiny_collections(n):
    c = corpus_for(n, 64, mean_len=5.0, seed=n, lo=1, hi=20)
    k = max(1, min(n, 7))
    ids = dg.init_doc_ids(n, k, n)
    for rep in lockstep(c, k, ids, 3):
        assert_report_ok(rep)


def test_long_posting_lists():
    """A head term in every document: its list is as long as K (here 20,000)."""
    c = corpus_for(30000, 3000, mean_len=30.0, zipf=1.3, seed=14)
    k = 20000
    ids = dg.init_doc_ids(c.n_docs, k, 14)
    rows = np.random.default_rng(0).choice(c.n_docs, 500, replace=False)
    for rep in lockstep(c, k, ids, 2, rows=rows):
        assert_report_ok(rep, check_objective=False)


# ------------------------------------------------------ state and layout


def test_checkpoint_resume_bit_exact():
    c = corpus_for(5000, 6000, seed=15)
    k = 80
    ids = dg.init_doc_ids(c.n_docs, k, 15)
    with ivf.IVF(c.row_ptr, c.term, c.val, c.n_terms, k) as m:
        m.set_means_from_docs(ids)
        m.iterate(10)
        a10, means10 = m.get_assign(), m.get_means()
    with ivf.IVF(c.row_ptr, c.term, c.val, c.n_terms, k) as m:
        m.set_means_from_docs(ids)
        m.iterate(5)
        a5, (p5, t5, v5) = m.get_assign(), m.get_means()
        it5 = m.info()["iteration"]
    with ivf.IVF(c.row_ptr, c.term, c.val, c.n_terms, k) as m:
        m.restore_means(p5, t5, v5, it5)
        m.set_assign(a5)
        m.iterate(5)
        assert m.info()["iteration"] == 10
        b10, bm = m.get_assign(), m.get_means()
    assert np.array_equal(a10, b10)
    for x, y in zip(means10, bm):
        assert np.array_equal(x, y)


def test_graph_iterations_equal_eager():
    c = corpus_for(4000, 5000, seed=16)
    k = 64
    ids = dg.init_doc_ids(c.n_docs, k, 16)
    res = []
    for g in (True, False):
        with ivf.IVF(c.row_ptr, c.term, c.val, c.n_terms, k, use_graph=g) as m:
            m.set_means_from_docs(ids)
            done, conv, st = m.iterate(8)
            res.append((done, conv, m.get_assign(), m.get_best(), m.get_means()))
    with ivf.IVF(c.row_ptr, c.term, c.val, c.n_terms, k) as m:
        m.set_means_from_docs(ids)
        for _ in range(res[0][0]):
            m.assign(stats=False)
            m.update()
        res.append((res[0][0], res[0][1], m.get_assign(), m.get_best(), m.get_means()))
    for other in res[1:]:
        assert other[0] == res[0][0] and other[1] == res[0][1]
        assert np.array_equal(other[2], res[0][2])
        assert np.array_equal(other[3].view(np.uint32), res[0][3].view(np.uint32))
        for x, y in zip(other[4], res[0][4]):
            assert np.array_equal(x, y)


def test_runs_are_bit_reproducible():
    c = corpus_for(6000, 7000, seed=17)
    k = 120
    ids = dg.init_doc_ids(c.n_docs, k, 17)
    outs = []
    for _ in range(2):
        with ivf.IVF(c.row_ptr, c.term, c.val, c.n_terms, k) as m:
            m.set_means_from_docs(ids)
            m.iterate(4)
            m.assign(stats=False)
            outs.append((m.get_best().view(np.uint32), m.get_gap().view(np.uint32)))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


def test_inverted_file_layout_and_members():
    c = corpus_for(3000, 4000, seed=18)
    k = 50
    ids = dg.init_doc_ids(c.n_docs, k, 18)
    with ivf.IVF(c.row_ptr, c.term, c.val, c.n_terms, k) as m:
        m.set_means_from_docs(ids)
        m.assign(stats=False)
        a = m.get_assign()
        m.update()
        tp, cid, w = m.get_inverted_file()
        ptr, term, val = m.get_means()
        cl, mem = m.get_members()
    # every list ascends strictly in cluster id; E = sum_p (nc)_p = sum_j (ntm)_j
    assert tp[0] == 0 and tp[-1] == ptr[-1] == cid.size
    owner = np.repeat(np.arange(c.n_terms), np.diff(tp))
    same = owner[1:] == owner[:-1]
    assert np.all(np.diff(cid.astype(np.int64))[same] > 0)
    # the inverted file is the transpose of the cluster-major means, values cast once to FP32
    rows = np.repeat(np.arange(k), np.diff(ptr))
    order = np.lexsort((rows, term))
    assert np.array_equal(cid, rows[order])
    assert np.array_equal(w, val[order].astype(np.float32))
    # C_j: objects grouped by cluster in ascending id
    assert np.array_equal(mem, np.argsort(a, kind="stable"))
    assert np.array_equal(cl, np.concatenate([[0], np.cumsum(np.bincount(a, minlength=k))]))


def test_set_means_rows_normalised():
    c = corpus_for(2000, 3000, seed=19)
    k = 30
    ids = dg.init_doc_ids(c.n_docs, k, 19)
    # means given as raw rows scaled by 3: the library divides by the norm
    m0 = sk.initial_means(c, ids)
    with ivf.IVF(c.row_ptr, c.term, c.val, c.n_terms, k) as m:
        m.set_means(m0.ptr, m0.term.astype(np.int32), (3.0 * m0.val).astype(np.float32))
        m.assign()
        a = m.get_assign()
    ref = sk.means_from_rows(m0.ptr, m0.term, (3.0 * m0.val).astype(np.float32).astype(np.float64), c.n_terms)
    rep = sk.lockstep_check(c, ref, a)
    assert rep["mismatches"] == 0


# -------------------------------------------------------------- errors


def test_errors_are_statuses_not_crashes():
    c = corpus_for(200, 100, seed=20)
    with pytest.raises(ivf.IvfError) as e:
        ivf.IVF(c.row_ptr, c.term, c.val, c.n_terms, c.n_docs + 1)
    assert e.value.status == ivf.IVF_E_INVALID
    bad = c.row_ptr.copy()
    bad[5] = bad[6] + 1
    with pytest.raises(ivf.IvfError):
        ivf.IVF(bad, c.term, c.val, c.n_terms, 4)
    t2 = c.term.copy()
    t2[c.row_ptr[3]], t2[c.row_ptr[3] + 1] = t2[c.row_ptr[3] + 1], t2[c.row_ptr[3]]  # unsorted row
    with pytest.raises(ivf.IvfError) as e:
        ivf.IVF(c.row_ptr, t2, c.val, c.n_terms, 4, validate=True)
    assert e.value.status == ivf.IVF_E_INVALID
    with ivf.IVF(c.row_ptr, c.term, c.val, c.n_terms, 4) as m:
        with pytest.raises(ivf.IvfError) as e:
            m.assign()
        assert e.value.status == ivf.IVF_E_STATE
        with pytest.raises(ivf.IvfError) as e:
            m.update()
        assert e.value.status == ivf.IVF_E_STATE
        with pytest.raises(ivf.IvfError) as e:
            m.set_means_from_docs([1, 1, 2, 3])
        assert e.value.status == ivf.IVF_E_INVALID
        with pytest.raises(ivf.IvfError):
            m.set_means_from_docs([1, 2, 3, 999])
        with pytest.raises(ivf.IvfError) as e:
            m.set_means(np.array([0, 1, 1, 2, 3]), np.array([0, 1, 2], np.int32), np.array([1, 1, 1], np.float32))
        assert e.value.status == ivf.IVF_E_INVALID  # an empty (zero-norm) mean row
        # still usable after the errors
        m.set_means_from_docs([1, 2, 3, 4])
        m.assign()
        m.update()


# ----------------------------------------------- full-size sampled parity


def test_scale_workload_sampled_lockstep():
    """1,000,000 docs x 500,000 terms, K = 10,000, in the benchmark's launch
    shape: two iterations, 2,000 sampled objects plus every near-tie the GPU
    flagged, means checked in full, Eq. 15 exact at full size."""
    w = dg.SCALE
    c = dg.make_corpus(w.corpus)
    ids = dg.init_doc_ids(c.n_docs, w.k, w.init_seed)
    rows = np.random.default_rng(123).choice(c.n_docs, 2000, replace=False)
    reps = lockstep(c, w.k, ids, 2, rows=rows)
    for rep in reps:
        assert_report_ok(rep, check_objective=False)


def test_scale_workload_bf16_sampled_lockstep():
    """The mixed-precision bench configuration (BF16 storage; after the first
    update the autotuner picks the tensor-core head there) at full size:
    sampled objects and every flagged near-tie equal the FP64 argmax, the
    FP64 master means equal the oracle's update, Eq. 15 exact."""
    w = dg.SCALE
    c = dg.make_corpus(w.corpus)
    ids = dg.init_doc_ids(c.n_docs, w.k, w.init_seed)
    rows = np.random.default_rng(321).choice(c.n_docs, 2000, replace=False)
    reps = lockstep(c, w.k, ids, 2, rows=rows, storage="bf16", best_tol=2.5e-2)
    for rep in reps:
        assert_report_ok(rep, check_objective=False)


def test_large_workload_full_size_sampled():
    """8,000,000 docs x 2,000,000 terms, K = 80,000 in the benchmark's launch
    configuration: 500 sampled objects equal the FP64 argmax at the first
    assignment and, against the GPU's own FP64 means, at the second; 16
    sampled non-empty clusters of the update equal the oracle's member sums
    normalised; Eq. 15 exact at the first assignment."""
    w = dg.LARGE
    c = dg.make_corpus(w.corpus)
    ids = dg.init_doc_ids(c.n_docs, w.k, w.init_seed)
    rng = np.random.default_rng(808)
    rows = rng.choice(c.n_docs, 500, replace=False)
    m0 = sk.initial_means(c, ids)
    with ivf.IVF(c.row_ptr, c.term, c.val, c.n_terms, w.k) as m:
        m.set_means_from_docs(ids)
        st = m.assign()
        a1, b1 = m.get_assign(), m.get_best()
        rep = sk.lockstep_check(c, m0, a1, b1, rows=np.unique(np.concatenate([rows, np.flatnonzero(m.get_gap() <= 1e-3)[:500]])))
        assert rep["mismatches"] == 0 and rep["best_ok"], (rep["mismatches"], rep["max_best_err"])
        assert st["entries_visited"] == sk.multiplication_count(c, m0)
        m.update()
        gp, gt, gv = m.get_means()
        # sampled clusters: the oracle's update restricted to their members
        sizes = np.bincount(a1, minlength=w.k)
        picks = rng.choice(np.flatnonzero(sizes > 0), 16, replace=False)
        members = np.flatnonzero(np.isin(a1, picks))
        sub_ptr = np.concatenate([[0], np.cumsum(np.diff(c.row_ptr)[members])]).astype(np.int64)
        sel = np.concatenate([np.arange(c.row_ptr[i], c.row_ptr[i + 1]) for i in members])
        sub = dg.Corpus(sub_ptr, c.term[sel], c.val[sel], c.n_terms)
        new, _, _ = sk.update(sub, a1[members], m0)
        for j in picks:
            t_o, v_o = new.row(int(j))
            t_g, v_g = gt[gp[j]:gp[j + 1]], gv[gp[j]:gp[j + 1]]
            assert np.array_equal(t_o, t_g)
            assert np.max(np.abs(v_o - v_g)) <= 1e-12
        # second assignment (the tuned kernel) against the GPU's FP64 means
        st2 = m.assign()
        a2, b2 = m.get_assign(), m.get_best()
        gm = sk.Means(ptr=gp, term=gt.astype(np.int64), val=gv, n_terms=c.n_terms)
        rep2 = sk.lockstep_check(c, gm, a2, b2, rows=rows)
        assert rep2["mismatches"] == 0 and rep2["best_ok"], (rep2["mismatches"], rep2["max_best_err"])
        assert st2["n_changed"] > 0


def test_large_k_tiled_sampled_lockstep():
    """K = 80,000 (> 65,536: tiled accumulator and 16-bit tile-local ids) on
    200,000 docs x 2,000,000 terms, lognormal(80) lengths, Zipf 1.0."""
    w = dg.LARGE.scaled(n_docs=200_000, name="large-k-200k-docs")
    c = dg.make_corpus(w.corpus)
    ids = dg.init_doc_ids(c.n_docs, w.k, w.init_seed)
    rows = np.random.default_rng(7).choice(c.n_docs, 1000, replace=False)
    reps = lockstep(c, w.k, ids, 2, rows=rows)
    for rep in reps:
        assert_report_ok(rep, check_objective=False)


# ------------------------------------------------ dense-head kernel (IFN rows)


@pytest.mark.parametrize("kernel", ["dense_head", "sparse"])
def test_kernel_family_lockstep_small_workload(kernel):
    """Both kernel families meet the bar on the 10k-doc workload, and the
    dense-head kernel really stores dense rows there."""
    w = dg.SMALL
    c = dg.make_corpus(w.corpus)
    ids = dg.init_doc_ids(c.n_docs, w.k, w.init_seed)
    reps = lockstep(c, w.k, ids, 5, kernel=kernel)
    for rep in reps:
        assert_report_ok(rep)
    with ivf.IVF(c.row_ptr, c.term, c.val, c.n_terms, w.k, kernel=kernel) as m:
        m.set_means_from_docs(ids)
        m.iterate(3)
        info = m.info()
    if kernel == "dense_head":
        assert info["dense_head_r"] > 0 and info["dense_head_rows"] > 0
    else:
        assert info["dense_head_r"] == 0


@pytest.mark.parametrize("k", [700, 3000, 5000])
def test_dense_head_tiled_lockstep(k):
    c = corpus_for(8000, 6000, mean_len=45.0, seed=k + 1)
    ids = dg.init_doc_ids(c.n_docs, k, k + 1)
    reps = lockstep(c, k, ids, 3, kernel="dense_head")
    for rep in reps:
        assert_report_ok(rep)


@pytest.mark.parametrize("storage,tol", [("f16", 3e-3), ("bf16", 2.5e-2)])
def test_dense_head_mixed_precision(storage, tol):
    c = corpus_for(6000, 8000, mean_len=40.0, seed=23)
    k = 1500
    ids = dg.init_doc_ids(c.n_docs, k, 23)
    for rep in lockstep(c, k, ids, 3, storage=storage, best_tol=tol, kernel="dense_head"):
        assert_report_ok(rep)


def test_dense_head_and_sparse_kernels_agree():
    c = corpus_for(5000, 5000, mean_len=40.0, seed=24)
    k = 2000
    ids = dg.init_doc_ids(c.n_docs, k, 24)
    out = {}
    for kernel in ("dense_head", "sparse"):
        with ivf.IVF(c.row_ptr, c.term, c.val, c.n_terms, k, kernel=kernel) as m:
            m.set_means_from_docs(ids)
            m.iterate(3)
            st = m.assign()
            out[kernel] = (m.get_assign(), m.get_best(), st["entries_visited"])
    assert np.array_equal(out["dense_head"][0], out["sparse"][0])
    assert np.allclose(out["dense_head"][1], out["sparse"][1], rtol=0, atol=1e-6)
    assert out["dense_head"][2] == out["sparse"][2]


@pytest.mark.parametrize("use_graph", [True, False])
def test_means_capacity_grows_on_demand(use_graph):
    """A context that starts with room for 1,000 mean entries grows while the
    means fill up, and ends with the same result as a roomy context."""
    c = corpus_for(3000, 4000, mean_len=30.0, seed=25)
    k = 40
    ids = dg.init_doc_ids(c.n_docs, k, 25)
    out = []
    for cap in (0, 1000):
        with ivf.IVF(c.row_ptr, c.term, c.val, c.n_terms, k, means_capacity=cap, use_graph=use_graph,
                     kernel="sparse") as m:
            m.set_means_from_docs(ids)
            m.iterate(3)
            m.assign(stats=False)
            m.update()
            out.append((m.get_assign(), m.get_means(), m.info()["ivf_capacity"]))
    assert out[1][2] > 1000
    assert np.array_equal(out[0][0], out[1][0])
    for x, y in zip(out[0][1], out[1][1]):
        assert np.array_equal(x, y)


# ------------------------------------------------ signs and reloaded objects


def _signed(c, frac, seed):
    """The corpus with a seeded fraction of its values negated (norms unchanged)."""
    flip = np.random.default_rng(seed).random(c.nnz) < frac
    val = np.where(flip, -c.val, c.val).astype(np.float32)
    return dg.Corpus(c.row_ptr, c.term, val, c.n_terms)


@pytest.mark.parametrize("kernel,storage,tol", [("sparse", "f32", 1e-5), ("sparse", "bf16", 2.5e-2),
                                                ("dense_head", "f32", 1e-5), ("dense_head", "bf16", 2.5e-2),
                                                ("tensor_head", "bf16", 2.5e-2)])
def test_mixed_sign_objects_lockstep(kernel, storage, tol):
    """Values of both signs: similarities can be negative, so unvisited
    clusters (similarity 0) compete for the argmax, and the error bound of the
    near-tie test is the absolute one."""
    c = _signed(corpus_for(5000, 5000, mean_len=35.0, seed=31), 0.3, 31)
    k = 1200
    ids = dg.init_doc_ids(c.n_docs, k, 31)
    for rep in lockstep(c, k, ids, 3, storage=storage, best_tol=tol, kernel=kernel):
        assert_report_ok(rep)


def test_negative_mean_rows_lockstep():
    """Non-negative objects, caller means with negative values; empty
    clusters keep their (negative) rows across the update."""
    c = corpus_for(3000, 3000, mean_len=30.0, seed=32)
    k = 200
    rng = np.random.default_rng(32)
    ptr = [0]
    terms, vals = [], []
    for _ in range(k):
        t = np.sort(rng.choice(c.n_terms, 12, replace=False))
        terms.append(t)
        vals.append(rng.standard_normal(12))
        ptr.append(ptr[-1] + 12)
    rows = (np.array(ptr, np.int64), np.concatenate(terms).astype(np.int32),
            np.concatenate(vals).astype(np.float32))
    for rep in lockstep(c, k, None, 3, means_rows=rows):
        assert_report_ok(rep)


@pytest.mark.parametrize("empty_policy", [0, 1])
def test_exactly_cancelling_member_sums_are_dropped(empty_policy):
    """Signed objects in pairs whose values on one term cancel exactly inside
    their cluster: that term's member sum is 0 and leaves the new mean
    (Algorithm 3 keeps w_p != 0 only).  Clusters 0-9 hold such pairs (their
    rows come from the per-cluster writer), 10-29 none (the per-run writer),
    30-31 no member (kept or emptied).  The update of a given assignment
    equals the oracle's: row structure exactly, values to 1e-12."""
    rng = np.random.default_rng(71)
    d, k, n_pairs, n_rand = 50, 32, 40, 360
    rows, assign = [], []
    for m in range(n_pairs):  # pair m: 5 shared terms of 0..39 and term 40 + m % 10 with +w / -w
        t = np.sort(np.append(rng.choice(40, 5, replace=False), 40 + m % 10))
        v = rng.lognormal(0.0, 1.0, t.size)
        v /= np.sqrt(np.sum(v * v))
        v32 = v.astype(np.float32)
        neg = v32.copy()
        neg[-1] = -neg[-1]
        rows += [(t, v32), (t, neg)]
        assign += [m % 10, m % 10]
    for i in range(n_rand):
        t = np.sort(rng.choice(40, 6, replace=False))
        v = rng.lognormal(0.0, 1.0, t.size)
        v /= np.sqrt(np.sum(v * v))
        rows.append((t, v.astype(np.float32)))
        assign.append(int(rng.integers(0, 30)))  # clusters 0-9 also get objects without terms 40-49
    rp = np.concatenate([[0], np.cumsum([t.size for t, _ in rows])]).astype(np.int64)
    tm = np.concatenate([t for t, _ in rows]).astype(np.int32)
    vl = np.concatenate([v for _, v in rows]).astype(np.float32)
    c = dg.Corpus(row_ptr=rp, term=tm, val=vl, n_terms=d)
    a = np.array(assign, np.int32)
    ids = rng.choice(c.n_docs, k, replace=False).astype(np.int32)
    with ivf.IVF(rp, tm, vl, d, k, empty_policy=empty_policy) as m:
        m.set_means_from_docs(ids)
        p0, t0, v0 = m.get_means()
        m.set_assign(a)
        m.update()
        gp, gt, gv = m.get_means()
    want, _, _ = sk.update(c, a, sk.Means(ptr=p0, term=t0.astype(np.int64), val=v0, n_terms=d),
                           empty_policy=empty_policy)
    assert np.array_equal(gp, want.ptr) and np.array_equal(gt, want.term)
    assert np.max(np.abs(gv - want.val)) <= 1e-12
    for j in range(10):  # the cancelling terms are gone, the others are there
        row = set(gt[gp[j]:gp[j + 1]].tolist())
        assert 40 + j not in row and len(row) > 0


def test_load_objects_equals_fresh_context():
    """Objects reloaded into a context (values of a different sign pattern)
    give bit for bit what a context created on them gives."""
    base = corpus_for(4000, 4000, mean_len=30.0, seed=33)
    c2 = _signed(base, 0.4, 33)
    k = 300
    ids = dg.init_doc_ids(base.n_docs, k, 33)
    out = []
    with ivf.IVF(base.row_ptr, base.term, base.val, base.n_terms, k) as m:
        m.set_means_from_docs(ids)
        m.iterate(2)
        m.load_objects(c2.row_ptr, c2.term, c2.val)
        m.set_means_from_docs(ids)
        m.iterate(2)
        m.assign()
        out.append((m.get_assign(), m.get_best(), m.get_gap()))
        # and back to the non-negative objects
        m.load_objects(base.row_ptr, base.term, base.val)
        m.set_means_from_docs(ids)
        m.assign()
        out.append((m.get_assign(), m.get_best(), m.get_gap()))
    for corpus, got in zip((c2, base), out):
        with ivf.IVF(corpus.row_ptr, corpus.term, corpus.val, corpus.n_terms, k) as m:
            m.set_means_from_docs(ids)
            if corpus is c2:
                m.iterate(2)
            m.assign()
            ref = (m.get_assign(), m.get_best(), m.get_gap())
        for x, y in zip(got, ref):
            assert np.array_equal(x.view(np.uint32), y.view(np.uint32))


def test_load_objects_rejects_bad_row_ptr_and_stays_usable():
    c = corpus_for(2000, 2000, mean_len=20.0, seed=34)
    k = 50
    ids = dg.init_doc_ids(c.n_docs, k, 34)
    with ivf.IVF(c.row_ptr, c.term, c.val, c.n_terms, k) as m:
        m.set_means_from_docs(ids)
        m.assign()
        a0 = m.get_assign()
        shifted = c.row_ptr + 1                 # does not start at 0
        decreasing = c.row_ptr.copy()
        decreasing[5] = decreasing[6] + 1       # row 5 ends before it starts
        short = c.row_ptr.copy()
        short[-1] -= 1                          # does not end at nnz
        for bad in (shifted, decreasing, short):
            with pytest.raises(ivf.IvfError) as e:
                m.load_objects(bad, c.term, c.val)
            assert e.value.status == ivf.IVF_E_INVALID
        # the context still holds the original objects
        m.assign()
        assert np.array_equal(m.get_assign(), a0)


@pytest.mark.parametrize("source", ["numpy", "pinned", "device"])
def test_load_objects_overlapped_with_the_iteration(source):
    """A load issued right after an assignment is enqueued (its copy runs on
    the context's copy stream meanwhile) takes effect at the next assignment;
    the update in between works on the objects its assignment ran on, and of
    two loads the second wins.  Bit-equal to the same calls made one after
    the other with nothing pending."""
    import torch

    a = corpus_for(3000, 3000, mean_len=25.0, seed=35)
    # the same rows in another order: same N and nnz, other objects per id
    perm = np.random.default_rng(35).permutation(a.n_docs)
    lens = np.diff(a.row_ptr)
    b_ptr = np.concatenate([[0], np.cumsum(lens[perm])]).astype(np.int64)
    b_term = np.concatenate([a.term[a.row_ptr[i]:a.row_ptr[i + 1]] for i in perm]).astype(np.int32)
    b_val = np.concatenate([a.val[a.row_ptr[i]:a.row_ptr[i + 1]] for i in perm]).astype(np.float32)
    half = (a.val * 0.5).astype(np.float32)
    k = 80
    ids = dg.init_doc_ids(a.n_docs, k, 35)

    def src(x):
        if source == "numpy":
            return x
        t = torch.from_numpy(np.ascontiguousarray(x))
        return t.pin_memory() if source == "pinned" else t.cuda()

    def run(mode):
        with ivf.IVF(a.row_ptr, a.term, a.val, a.n_terms, k) as m:
            m.set_means_from_docs(ids)
            m.assign()
            if mode == "overlapped":
                m.load_objects(src(a.row_ptr), src(a.term), src(half))  # replaced by the next load
                m.load_objects(src(b_ptr), src(b_term), src(b_val))
            m.update()
            if mode == "sequential":
                m.load_objects(b_ptr, b_term, b_val)
            m.assign()
            out = [m.get_assign(), m.get_best()]
            m.update()
            m.assign()
            out.append(m.get_assign())
            return out

    got, ref, none = run("overlapped"), run("sequential"), run("no load")
    for x, y in zip(got, ref):
        assert np.array_equal(x.view(np.uint32), y.view(np.uint32))
    assert not np.array_equal(got[0], none[0])


@pytest.mark.parametrize("k,kind", [(1500, "poisson"), (4500, "poisson"), (3000, "lognormal")])
def test_dense_head_wide_tiles_bit_equal(k, kind):
    """Shared-memory tiles of 1, 2 and 4 head sub-tiles (the sparse lists
    scattered once per wide tile, the dense rows per 1,024-cluster sub-tile)
    sum every rho_c in the same order, so their results are identical; K =
    1,500 with a 2,048 tile runs untiled, K = 4,500 ends in a ragged tile, the
    lognormal lengths reach 400 terms (13 chunks of 32)."""
    if kind == "lognormal":
        c = corpus_for(5000, 5000, mean_len=90.0, seed=k + 7, kind="lognormal", lo=5, hi=400)
        assert np.diff(c.row_ptr).max() > 128
    else:
        c = corpus_for(5000, 5000, mean_len=40.0, seed=k + 7)
    ids = dg.init_doc_ids(c.n_docs, k, k + 7)
    out = {}
    for kt in (1024, 2048, 4096):
        if kt == 4096 and k <= 2048:
            continue
        with ivf.IVF(c.row_ptr, c.term, c.val, c.n_terms, k, kernel="dense_head", k_tile=kt) as m:
            m.set_means_from_docs(ids)
            m.iterate(2)
            st = m.assign()
            inf = m.info()
            assert inf["dense_head_r"] == 32 and inf["dense_head_sub"] == kt // 1024
            out[kt] = (m.get_assign(), m.get_best(), m.get_gap(), st["entries_visited"])
    ref = out[1024]
    for kt, got in out.items():
        for x, y in zip(got[:3], ref[:3]):
            assert np.array_equal(x.view(np.uint32), y.view(np.uint32)), kt
        assert got[3] == ref[3]
    wide = max(out)
    for rep in lockstep(c, k, ids, 2, kernel="dense_head", k_tile=wide):
        assert_report_ok(rep)


@pytest.mark.parametrize("use_graph", [True, False])
def test_dense_head_rows_grow_on_demand(use_graph):
    """A context that starts with room for a single dense row grows its rows
    when more lists qualify (at the kernel choice and after updates) and ends
    with exactly the results of a roomy context."""
    c = corpus_for(4000, 4000, mean_len=35.0, seed=35)
    k = 1500
    ids = dg.init_doc_ids(c.n_docs, k, 35)
    out = []
    for budget in (0, 1024 * 4):
        with ivf.IVF(c.row_ptr, c.term, c.val, c.n_terms, k, kernel="dense_head", k_tile=1024,
                     use_graph=use_graph, dense_head_bytes=budget) as m:
            m.set_means_from_docs(ids)
            m.iterate(3)
            st = m.assign()
            out.append((m.get_assign(), m.get_best(), m.get_gap(), st["entries_visited"],
                        m.info()["dense_head_rows"]))
    assert out[1][4] == out[0][4] > 1
    for x, y in zip(out[0][:3], out[1][:3]):
        assert np.array_equal(x.view(np.uint32), y.view(np.uint32))
    assert out[0][3] == out[1][3]


# ----------------------------------------------------- tensor-core head


@pytest.mark.parametrize("storage,tol", [("f16", 3e-3), ("bf16", 2.5e-2)])
def test_tensor_head_lockstep(storage, tol):
    """Head part from the tensor-core GEMM (16-bit operands, FP32
    accumulation), tail and argmax by the CUDA-core kernel: assignments equal
    the FP64 argmax at every iteration, the Eq. 15 count is exact."""
    c = corpus_for(6000, 6000, mean_len=40.0, seed=37)
    k = 2500
    ids = dg.init_doc_ids(c.n_docs, k, 37)
    reps = lockstep(c, k, ids, 3, storage=storage, best_tol=tol, kernel="tensor_head")
    for rep in reps:
        assert_report_ok(rep)


def test_tensor_head_several_batches_equal_cuda_core_head():
    """K = 30,000 makes the GEMM output of 40,000 objects span two batches;
    the assignments equal those of the CUDA-core head (both are the FP64
    argmax), sampled objects are checked against the oracle, and two runs
    give identical bits."""
    c = corpus_for(40000, 20000, mean_len=30.0, seed=38)
    k = 30000
    ids = dg.init_doc_ids(c.n_docs, k, 38)
    out = {}
    for kernel in ("tensor_head", "tensor_head", "dense_head"):
        with ivf.IVF(c.row_ptr, c.term, c.val, c.n_terms, k, storage="bf16", kernel=kernel) as m:
            m.set_means_from_docs(ids)
            m.iterate(2)
            st = m.assign()
            inf = m.info()
            res = (m.get_assign(), m.get_best(), m.get_gap(), st["entries_visited"], inf["dense_head_tensor"])
        if kernel in out:
            for x, y in zip(out[kernel][:3], res[:3]):
                assert np.array_equal(x.view(np.uint32), y.view(np.uint32))
        out[kernel] = res
    assert out["tensor_head"][4] == 1 and out["dense_head"][4] == 0
    assert np.array_equal(out["tensor_head"][0], out["dense_head"][0])
    assert out["tensor_head"][3] == out["dense_head"][3]
    rows = np.random.default_rng(38).choice(c.n_docs, 1500, replace=False)
    for rep in lockstep(c, k, ids, 2, rows=rows, storage="bf16", best_tol=2.5e-2, kernel="tensor_head"):
        assert_report_ok(rep, check_objective=False)


def test_tensor_head_needs_16bit_storage():
    c = corpus_for(3000, 3000, seed=39)
    with ivf.IVF(c.row_ptr, c.term, c.val, c.n_terms, 1500, kernel="tensor_head") as m:
        m.set_means_from_docs(dg.init_doc_ids(c.n_docs, 1500, 39))
        with pytest.raises(ivf.IvfError) as e:
            m.assign()
        assert e.value.status == ivf.IVF_E_UNSUPPORTED


@pytest.mark.parametrize("kernel,k_tile,storage", [("dense_head", 2048, "f32"), ("dense_head", 1024, "f32"),
                                                   ("sparse", 512, "f32"), ("dense_head", 2048, "bf16"),
                                                   ("tensor_head", 2048, "bf16"), ("tensor_head", 1024, "f16")])
def test_tile_major_equals_object_major(kernel, k_tile, storage):
    """One launch per cluster tile over all objects, with (best, id, second)
    carried in device memory, sums every rho_c in the same order as the
    object-major launch: identical assignments, best, gap and error bounds,
    the same Eq. 15 count, and the near-ties it hands to the object-major
    candidate pass are re-scored to the same FP64 argmax.  Duplicated means
    make exact ties (near-ties in every tile)."""
    c = corpus_for(6000, 5000, mean_len=60.0, seed=41, kind="lognormal", lo=5, hi=400)
    k = 4500  # 2.2 / 4.4 / 8.8 tiles: the last one ragged
    ids = dg.init_doc_ids(c.n_docs, k, 41)
    ids[k - 1] = ids[0]
    ids[k // 2] = ids[1]
    lens = [c.row_ptr[d + 1] - c.row_ptr[d] for d in ids]
    rows = (np.concatenate([[0], np.cumsum(lens)]).astype(np.int64),
            np.concatenate([c.term[c.row_ptr[d]:c.row_ptr[d + 1]] for d in ids]),
            np.concatenate([c.val[c.row_ptr[d]:c.row_ptr[d + 1]] for d in ids]))
    out = {}
    for sched in ("object_major", "tile_major"):
        with ivf.IVF(c.row_ptr, c.term, c.val, c.n_terms, k, kernel=kernel, k_tile=k_tile, schedule=sched,
                     storage=storage) as m:
            m.set_means(*rows)
            sts = [m.assign()]
            m.update()
            sts.append(m.assign())
            assert m.info()["tile_major"] == (sched == "tile_major")
            out[sched] = (m.get_assign(), m.get_best(), m.get_gap(), m.get_err_bound(),
                          [s["entries_visited"] for s in sts], [s["n_rescored"] for s in sts],
                          [s["n_zero_sim"] for s in sts])
    ref, got = out["object_major"], out["tile_major"]
    for x, y in zip(got[:4], ref[:4]):
        assert np.array_equal(np.asarray(x).view(np.uint32), np.asarray(y).view(np.uint32))
    assert got[4] == ref[4] and got[5] == ref[5] and got[6] == ref[6]
    assert ref[5][0] > 0  # the duplicated means were re-scored
    for rep in lockstep(c, k, None, 2, means_rows=rows, kernel=kernel, k_tile=k_tile, schedule="tile_major",
                        storage=storage, best_tol=1e-5 if storage == "f32" else 2.5e-2):
        assert_report_ok(rep)


@pytest.mark.parametrize("k", [37, 700, 3000])
def test_ivfd_equals_sparse_ivf(k):
    """IVFD (Algorithm 4: the objects as an inverted file, the assignment
    looping over the means) multiplies the same posting entries as IVF (Eq. 15)
    and sums every rho_c in the same ascending term order, so without the
    re-score its FP32 results equal the sparse IVF kernel's bit for bit; with
    it, the lockstep check against the FP64 oracle holds."""
    c = corpus_for(5000, 4000, mean_len=40.0, seed=k, kind="lognormal", lo=3, hi=300)
    ids = dg.init_doc_ids(c.n_docs, k, k)
    out = {}
    for kernel in ("sparse", "ivfd"):
        with ivf.IVF(c.row_ptr, c.term, c.val, c.n_terms, k, kernel=kernel, rescore=False) as m:
            m.set_means_from_docs(ids)
            sts = [m.assign()]
            m.update()
            sts.append(m.assign())
            out[kernel] = (m.get_assign(), m.get_best(), m.get_gap(), [s["entries_visited"] for s in sts],
                           [s["n_zero_sim"] for s in sts])
    for x, y in zip(out["ivfd"][:3], out["sparse"][:3]):
        assert np.array_equal(np.asarray(x).view(np.uint32), np.asarray(y).view(np.uint32))
    assert out["ivfd"][3] == out["sparse"][3] and out["ivfd"][4] == out["sparse"][4]
    for rep in lockstep(c, k, ids, 3, kernel="ivfd"):
        assert_report_ok(rep)


def test_ivfd_object_reload_and_unsupported_forms():
    """The object inverted file follows ivf_load_objects; FP16/BF16 storage is
    not offered for IVFD."""
    c = corpus_for(3000, 3000, mean_len=30.0, seed=77)
    k = 150
    ids = dg.init_doc_ids(c.n_docs, k, 77)
    flip = np.where(np.random.default_rng(77).random(c.nnz) < 0.3, -c.val, c.val).astype(np.float32)
    res = {}
    for kernel in ("sparse", "ivfd"):
        with ivf.IVF(c.row_ptr, c.term, c.val, c.n_terms, k, kernel=kernel) as m:
            m.set_means_from_docs(ids)
            m.iterate(2)
            m.load_objects(c.row_ptr, c.term, flip)
            m.assign()
            res[kernel] = m.get_assign()
    assert np.array_equal(res["ivfd"], res["sparse"])
    with pytest.raises(ivf.IvfError):
        ivf.IVF(c.row_ptr, c.term, c.val, c.n_terms, k, kernel="ivfd", storage="bf16")
