"""ivf_assign_static: the assignment step for callers that cannot allocate (GPU).

Some callers cannot allocate device memory where they run the assignment:
their device memory belongs to their own pool or framework allocator, or their
loop must not pay for (or synchronise the device on) a cudaMalloc after
start-up.  ivf_assign_static serves them: every buffer is the caller's, and
the step's scratch sits in a fixed static device array inside the library.
This test calls it through the C ABI and checks its output against
ivf_assign on the same means, on two calls in a row (the second call starts
from whatever the first left in the shared scratch array).  The file is named
to be collected last.
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

    # sizes beyond the stated maximum are rejected before any GPU work
    assert call(a, None, None, n_docs=ivf.IVF_STATIC_MAX_DOCS + 1) == ivf.IVF_E_INVALID
    assert call(a, None, None, kk=ivf.IVF_STATIC_MAX_K + 1) == ivf.IVF_E_INVALID
    assert call(a, None, None, kk=n + 1) == ivf.IVF_E_INVALID
