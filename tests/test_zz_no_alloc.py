"""ivf_assign_static: the assignment step for callers that cannot allocate (GPU).

Some callers cannot allocate device memory where they run the assignment:
their device memory belongs to their own pool or framework allocator, or their
loop must not pay for (or synchronise the device on) a cudaMalloc after
start-up.  ivf_assign_static serves them: every buffer is the caller's, and
the step's scratch sits in a fixed static device array inside the library.
These tests call it through the C ABI and check its output against
ivf_assign on the same means and against the FP64 oracle, on several calls in
a row (each call starts from whatever the previous one left in the shared
scratch array), and check that repeated calls leave the device's free memory
unchanged.  The file is named to be collected last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

BEST_TOL = 1e-5  # the tolerance of the other GPU parity tests


def test_static_assignment_matches_context_assignment_twice():
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_2002_09094_gb300 import datagen as dg
    from paper_2002_09094_gb300 import ivf

    lib = ivf.load_library()
    c = dg.make_corpus(dg.CorpusSpec(n_docs=6000, n_terms=8000, length_kind="poisson", length_mean=40.0,
                                     length_lo=3, length_hi=200, zipf_s=1.1, seed=31))
    k = 200
    ids = dg.init_doc_ids(c.n_docs, k, 31)
    with ivf.IVF(c.row_ptr, c.term, c.val, c.n_terms, k) as m:
        m.set_means_from_docs(ids)
        m.iterate(2)  # means after two update steps
        m.assign(stats=False)  # the existing entry point on the same means
        a_ref, b_ref, g_ref = m.get_assign(), m.get_best(), m.get_gap()
        tp, cid, w = m.get_inverted_file()
        mp, mt, mv = m.get_means()

    def dev(x):
        return torch.from_numpy(np.ascontiguousarray(x)).cuda()

    rp, tm, vl = dev(c.row_ptr), dev(c.term), dev(c.val)
    d_tp, d_cid, d_w = dev(tp), dev(cid), dev(w)
    d_mp, d_mt, d_mv = dev(mp), dev(mt), dev(mv)
    stream = torch.cuda.current_stream().cuda_stream
    n = c.n_docs

    def call(a, b, g, n_docs=n, kk=k):
        return lib.ivf_assign_static(n_docs, rp.data_ptr(), tm.data_ptr(), vl.data_ptr(), c.n_terms, kk,
                                     d_tp.data_ptr(), d_cid.data_ptr(), d_w.data_ptr(), d_mp.data_ptr(),
                                     d_mt.data_ptr(), d_mv.data_ptr(), a.data_ptr(),
                                     b.data_ptr() if b is not None else None,
                                     g.data_ptr() if g is not None else None, stream)

    for _ in range(2):
        a = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        b = torch.full((n,), float("nan"), dtype=torch.float32, device="cuda")
        g = torch.full((n,), float("nan"), dtype=torch.float32, device="cuda")
        assert call(a, b, g) == ivf.IVF_OK
        torch.cuda.synchronize()
        assert np.array_equal(a.cpu().numpy(), a_ref)
        assert np.allclose(b.cpu().numpy(), b_ref, rtol=0, atol=BEST_TOL)
        assert np.allclose(g.cpu().numpy(), g_ref, rtol=0, atol=BEST_TOL)

    # best/gap outputs are optional
    a = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    assert call(a, None, None) == ivf.IVF_OK
    torch.cuda.synchronize()
    assert np.array_equal(a.cpu().numpy(), a_ref)

    # the FP64 argmax (lowest id on ties) under the same means, from the oracle
    import oracle.spherical_kmeans as sk

    means = sk.Means(ptr=mp, term=mt.astype(np.int64), val=mv, n_terms=c.n_terms)
    rep = sk.lockstep_check(c, means, a.cpu().numpy(), b_ref)
    assert rep["mismatches"] == 0 and rep["best_ok"], rep["mismatch_rows"]

    # sizes beyond the stated maximum are rejected before any GPU work
    assert call(a, None, None, n_docs=ivf.IVF_STATIC_MAX_DOCS + 1) == ivf.IVF_E_INVALID
    assert call(a, None, None, kk=ivf.IVF_STATIC_MAX_K + 1) == ivf.IVF_E_INVALID
    assert call(a, None, None, kk=n + 1) == ivf.IVF_E_INVALID


def test_static_assignment_at_the_size_limits_with_exact_ties():
    """N at IVF_STATIC_MAX_DOCS and K = 12,000 (near IVF_STATIC_MAX_K: four
    warps per block, about 196 KB of shared memory each) with every mean
    duplicated: every object that meets a posting entry ties exactly between
    cluster j and j + 6,000, so far more objects are flagged than the 4,096
    that get a candidate list -- the rest are re-scored against every cluster
    from the caller's FP64 means.  The result must be the lowest-id FP64
    argmax, equal to ivf_assign's, on three calls in a row, and the calls
    after the first (which does the one-time set-up) must not change the
    device's free memory."""
    import torch

    import __graft_entry__

    __graft_entry__.build()
    import oracle.spherical_kmeans as sk
    from paper_2002_09094_gb300 import datagen as dg
    from paper_2002_09094_gb300 import ivf

    lib = ivf.load_library()
    n = ivf.IVF_STATIC_MAX_DOCS
    c = dg.make_corpus(dg.CorpusSpec(n_docs=n, n_terms=8000, length_kind="poisson", length_mean=40.0,
                                     length_lo=3, length_hi=200, zipf_s=1.1, seed=37))
    half = 6000
    k = 2 * half
    assert k <= ivf.IVF_STATIC_MAX_K
    ids = dg.init_doc_ids(c.n_docs, half, 37)
    rows = list(ids) + list(ids)
    lens = [c.row_ptr[d + 1] - c.row_ptr[d] for d in rows]
    ptr = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    term = np.concatenate([c.term[c.row_ptr[d]:c.row_ptr[d + 1]] for d in rows])
    val = np.concatenate([c.val[c.row_ptr[d]:c.row_ptr[d + 1]] for d in rows])
    with ivf.IVF(c.row_ptr, c.term, c.val, c.n_terms, k) as m:
        m.set_means(ptr, term, val)
        st = m.assign()
        a_ref, b_ref = m.get_assign(), m.get_best()
        tp, cid, w = m.get_inverted_file()
        mp, mt, mv = m.get_means()
    assert st["n_flagged"] > 4096  # the exact ties, more than the candidate slots

    # the oracle: lowest id among the FP64 maxima; exact ties keep the lower copy
    means = sk.Means(ptr=mp, term=mt.astype(np.int64), val=mv, n_terms=c.n_terms)
    rho = sk.similarities(c, means)
    a_o, best_o, _ = sk.assign_from_similarities(rho)
    distinct = rho[:, :half]
    top2 = np.partition(distinct, half - 2, axis=1)[:, half - 2:]
    clear = (top2[:, 1] - top2[:, 0]) >= 1e-6
    assert np.all(a_o < half) and int(np.count_nonzero(clear)) > 4096

    def dev(x):
        return torch.from_numpy(np.ascontiguousarray(x)).cuda()

    rp, tm, vl = dev(c.row_ptr), dev(c.term), dev(c.val)
    d_tp, d_cid, d_w = dev(tp), dev(cid), dev(w)
    d_mp, d_mt, d_mv = dev(mp), dev(mt), dev(mv)
    stream = torch.cuda.current_stream().cuda_stream
    free_after_first = None
    a = torch.empty((n,), dtype=torch.int32, device="cuda")
    b = torch.empty((n,), dtype=torch.float32, device="cuda")
    for call_no in range(3):
        a.fill_(-1)
        b.fill_(float("nan"))
        torch.cuda.synchronize()
        if call_no == 1:
            free_after_first = torch.cuda.mem_get_info()[0]
        st_call = lib.ivf_assign_static(n, rp.data_ptr(), tm.data_ptr(), vl.data_ptr(), c.n_terms, k,
                                        d_tp.data_ptr(), d_cid.data_ptr(), d_w.data_ptr(), d_mp.data_ptr(),
                                        d_mt.data_ptr(), d_mv.data_ptr(), a.data_ptr(), b.data_ptr(), None, stream)
        assert st_call == ivf.IVF_OK
        torch.cuda.synchronize()
        if call_no >= 1:
            assert torch.cuda.mem_get_info()[0] == free_after_first
        got = a.cpu().numpy()
        assert np.array_equal(got, a_ref)
        assert np.array_equal(got[clear], a_o[clear]) and np.all(got < half)
        assert np.allclose(b.cpu().numpy(), best_o, rtol=0, atol=BEST_TOL)
