"""Data-parallel IVF over object shards: the host protocol on CPU (gloo,
world size 2) and the library's shard entry points on one GPU.

CPU: each rank runs paper_2002_09094_gb300.sharded.ShardedIVF over its
contiguous shard with a backend built from the FP64 oracle (this file only),
so the sharding, the variable-length all-gather and the rank-order merge are
what is tested.  The means every rank ends with must be bit-identical across
ranks and equal the single-process oracle's trajectory (Lloyd, Algorithm 2)
to 1e-12, with identical assignments.

GPU: two contexts hold the two shards of one object set (run one after the
other on one GPU; nothing waits on the other), their member sums are joined
in shard order and both finish the update from them: the two get identical
means, equal to one context's ivf_update to 1e-12, and one shard alone gives
ivf_update's means bit for bit.
"""
import math
import os
import socket
import sys

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class OracleShard:
    """A rank's backend on CPU: assignment and member sums of its shard from
    the FP64 oracle; the merged update written out here in FP64, adding equal
    (cluster, term) sums in the order given (rank order)."""

    def __init__(self, corpus, means):
        self.c = corpus
        self.means = means
        self.prev = None
        self.a = None

    def assign(self):
        import oracle.spherical_kmeans as sk

        a, _, _ = sk.assign_from_similarities(sk.similarities(self.c, self.means))
        changed = len(a) if self.prev is None else int(np.count_nonzero(a != self.prev))
        self.prev = self.a = a
        return {"n_changed": changed}

    def get_assign(self):
        return self.a

    def get_partial_sums(self):
        import oracle.spherical_kmeans as sk

        s = sk.cluster_sums(self.c, self.a, self.means.k).tocoo()
        order = np.lexsort((s.col, s.row))
        return s.row[order].astype(np.int32), s.col[order].astype(np.int32), s.data[order].astype(np.float64)

    def update_from_partials(self, cl, tm, sm):
        import oracle.spherical_kmeans as sk

        k = self.means.k
        sums = {}
        for j, t, v in zip(cl.tolist(), tm.tolist(), sm.tolist()):  # in the order given
            sums[(j, t)] = sums.get((j, t), 0.0) + v
        ptr, terms, vals = [0], [], []
        for j in range(k):
            row = sorted((t, v) for (jj, t), v in sums.items() if jj == j and v != 0.0)
            nrm = math.sqrt(sum(v * v for _, v in row))
            if nrm > 0.0:
                terms += [t for t, _ in row]
                vals += [v / nrm for _, v in row]
            else:  # empty cluster: keeps its previous mean
                pt, pv = self.means.row(j)
                terms += pt.tolist()
                vals += pv.tolist()
            ptr.append(len(terms))
        self.means = sk.Means(ptr=np.array(ptr, np.int64), term=np.array(terms, np.int64),
                              val=np.array(vals, np.float64), n_terms=self.means.n_terms)


def _corpus():
    from paper_2002_09094_gb300 import datagen as dg

    return dg.make_corpus(dg.CorpusSpec(n_docs=301, n_terms=120, length_kind="poisson", length_mean=9.0,
                                        length_lo=2, length_hi=30, zipf_s=1.0, seed=61))


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle.spherical_kmeans as sk
    from paper_2002_09094_gb300 import datagen as dg
    from paper_2002_09094_gb300 import sharded

    c = _corpus()
    lo, hi = sharded.shard_bounds(c.n_docs, world, rank)
    rp, tm, vl = sharded.shard_rows(c.row_ptr, c.term, c.val, lo, hi)
    shard = dg.Corpus(row_ptr=rp, term=tm, val=vl, n_terms=c.n_terms)
    ids = dg.init_doc_ids(c.n_docs, 9, 61)
    mp_, mt_, mv_ = sharded.mean_rows(c.row_ptr, c.term, c.val, ids)
    means0 = sk.means_from_rows(mp_, mt_, mv_.astype(np.float64), c.n_terms)
    run = sharded.ShardedIVF(OracleShard(shard, means0), dist, device="cpu")
    iters, conv = run.iterate(4)
    m = run.m.means
    out[rank] = {"lo": lo, "hi": hi, "iters": iters, "assign": run.m.a.tolist(), "ptr": m.ptr.tolist(),
                 "term": m.term.tolist(), "val": m.val.tobytes(), "lens": run.exchanged}
    dist.destroy_process_group()


def test_sharded_protocol_gloo_world_size_two():
    sys.path.insert(0, ROOT)
    import oracle.spherical_kmeans as sk
    from paper_2002_09094_gb300 import datagen as dg
    from paper_2002_09094_gb300 import sharded

    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    r0, r1 = res[0], res[1]
    # the shards tile the object range; both ranks saw both ranks' sums
    assert (r0["lo"], r0["hi"], r1["lo"], r1["hi"]) == (0, 150, 150, 301)
    assert r0["lens"] == r1["lens"] and all(len(x) == 2 and min(x) > 0 for x in r0["lens"])
    # the same bits on both ranks
    assert r0["ptr"] == r1["ptr"] and r0["term"] == r1["term"] and r0["val"] == r1["val"]
    # the single-process Lloyd trajectory from the same initial means
    c = _corpus()
    ids = dg.init_doc_ids(c.n_docs, 9, 61)
    mp_, mt_, mv_ = sharded.mean_rows(c.row_ptr, c.term, c.val, ids)
    its = sk.iterate(c, sk.means_from_rows(mp_, mt_, mv_.astype(np.float64), c.n_terms), max_iter=4)
    assert r0["iters"] == len(its)
    last = its[-1]
    assert r0["assign"] + r1["assign"] == last.assign.tolist()
    assert r0["ptr"] == last.means_after.ptr.tolist() and r0["term"] == last.means_after.term.tolist()
    vals = np.frombuffer(r0["val"], dtype=np.float64)
    assert np.max(np.abs(vals - last.means_after.val)) <= 1e-12


def test_shard_helpers():
    sys.path.insert(0, ROOT)
    from paper_2002_09094_gb300 import sharded

    assert [sharded.shard_bounds(10, 3, r) for r in range(3)] == [(0, 3), (3, 6), (6, 10)]
    with pytest.raises(ValueError):
        sharded.shard_bounds(10, 3, 3)
    rp = np.array([0, 2, 2, 5, 6], np.int64)
    tm = np.arange(6, dtype=np.int32)
    vl = np.arange(6, dtype=np.float32)
    p, t, v = sharded.shard_rows(rp, tm, vl, 1, 3)
    assert p.tolist() == [0, 0, 3] and t.tolist() == [2, 3, 4]
    p, t, v = sharded.mean_rows(rp, tm, vl, [3, 0])
    assert p.tolist() == [0, 1, 3] and t.tolist() == [5, 0, 1]


@pytest.mark.gpu
def test_shard_member_sums_reproduce_the_update_on_gpu():
    import __graft_entry__

    __graft_entry__.build()
    import oracle.spherical_kmeans as sk
    from paper_2002_09094_gb300 import datagen as dg
    from paper_2002_09094_gb300 import ivf
    from paper_2002_09094_gb300 import sharded

    c = dg.make_corpus(dg.CorpusSpec(n_docs=20000, n_terms=6000, length_kind="lognormal", length_mean=40.0,
                                     length_lo=3, length_hi=300, zipf_s=1.05, seed=63))
    k = 700
    ids = dg.init_doc_ids(c.n_docs, k, 63)
    rows = sharded.mean_rows(c.row_ptr, c.term, c.val, ids)
    with ivf.IVF(c.row_ptr, c.term, c.val, c.n_terms, k) as one:
        one.set_means(*rows)
        one.assign()
        a_one = one.get_assign()
        full = one.get_partial_sums()
        one.update()
        means_one = one.get_means()
        # one shard = the whole set: the update from its own sums is ivf_update's, bit for bit
        one.set_means(*rows)
        one.assign()
        one.update_from_partials(*full)
        same = one.get_means()
    for x, y in zip(same, means_one):
        assert np.array_equal(np.asarray(x).view(np.uint8), np.asarray(y).view(np.uint8))
    ctxs, parts = [], []
    try:
        for r in range(2):
            lo, hi = sharded.shard_bounds(c.n_docs, 2, r)
            rp, tm, vl = sharded.shard_rows(c.row_ptr, c.term, c.val, lo, hi)
            m = ivf.IVF(rp, tm, vl, c.n_terms, k)
            ctxs.append(m)
            m.set_means(*rows)
            m.assign()
            parts.append(m.get_partial_sums())
        joined = [np.concatenate([p[q] for p in parts]) for q in range(3)]
        assert np.array_equal(np.concatenate([m.get_assign() for m in ctxs]), a_one)
        got = []
        for m in ctxs:
            m.update_from_partials(*joined)
            got.append(m.get_means())
        for x, y in zip(got[0], got[1]):
            assert np.array_equal(np.asarray(x).view(np.uint8), np.asarray(y).view(np.uint8))
        assert np.array_equal(got[0][0], means_one[0]) and np.array_equal(got[0][1], means_one[1])
        assert np.max(np.abs(got[0][2] - means_one[2])) <= 1e-12
        # and the oracle's update of the same assignment
        new, _, _ = sk.update(c, a_one, sk.means_from_rows(rows[0], rows[1], rows[2].astype(np.float64),
                                                           c.n_terms))
        assert np.array_equal(got[0][0], new.ptr) and np.max(np.abs(got[0][2] - new.val)) <= 1e-12
        # the next assignment on the shards equals the one-context one
        with ivf.IVF(c.row_ptr, c.term, c.val, c.n_terms, k) as one:
            one.set_means(*rows)
            one.iterate(1)
            one.assign()
            a2 = one.get_assign()
        for m in ctxs:
            m.assign()
        assert np.array_equal(np.concatenate([m.get_assign() for m in ctxs]), a2)
        # ids outside the problem are rejected before any change
        with pytest.raises(ivf.IvfError):
            ctxs[0].update_from_partials(np.array([k], np.int32), np.array([0], np.int32), np.array([1.0]))
    finally:
        for m in ctxs:
            m.close()
