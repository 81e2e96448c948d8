"""Data-parallel IVF spherical k-means over object shards, one rank per GPU.

The objects are independent in the assignment step (Section 2.4: each
object's argmax needs only the means), so every rank holds a contiguous
shard of the objects and a full copy of the means, and assigns its shard
with no exchange.  The update step (Algorithm 3's member sums) splits the
same way:

    s_j = sum over ranks r of s_j^(r),   s_j^(r) = sum_{i in C_j, i in shard r} x_i

Each rank computes its s_j^(r) (``get_partial_sums``), the ranks all-gather
those sparse lists, and every rank finishes the same update from the lists
concatenated in rank order (``update_from_partials``: equal (cluster, term)
pairs added in FP64 in that order, normalisation, inverted-file rebuild), so
every rank ends the iteration with bit-identical means.  The convergence test
adds the ranks' changed counts.  This module only shards, exchanges and
orders; every sum and normalisation runs in the per-rank backend (the C-ABI
library on a GPU).
"""
from __future__ import annotations

import numpy as np


def shard_bounds(n_docs: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous object range [lo, hi) of a rank: sizes differ by at most one."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    lo = n_docs * rank // world
    hi = n_docs * (rank + 1) // world
    return lo, hi


def shard_rows(row_ptr, term, val, lo: int, hi: int):
    """The CSR rows of objects [lo, hi) as their own CSR (row_ptr rebased to 0)."""
    rp = np.asarray(row_ptr, dtype=np.int64)
    a, b = int(rp[lo]), int(rp[hi])
    return (rp[lo:hi + 1] - a).astype(np.int64), np.asarray(term)[a:b], np.asarray(val)[a:b]


def mean_rows(row_ptr, term, val, doc_ids):
    """Cluster-major rows of the given objects (the initial means x_{d_j}),
    gathered unchanged; the library normalises them."""
    rp = np.asarray(row_ptr, dtype=np.int64)
    ids = np.asarray(doc_ids, dtype=np.int64)
    lens = rp[ids + 1] - rp[ids]
    ptr = np.zeros(len(ids) + 1, dtype=np.int64)
    np.cumsum(lens, out=ptr[1:])
    idx = np.concatenate([np.arange(rp[d], rp[d + 1]) for d in ids]) if len(ids) else np.zeros(0, np.int64)
    return ptr, np.asarray(term)[idx].astype(np.int32), np.asarray(val)[idx].astype(np.float32)


def all_gather_concat(arrays, dist, group=None, device="cpu"):
    """All-gather variable-length 1-D arrays (one tuple per rank, same dtypes)
    and concatenate each position in rank order.  Lengths are exchanged
    first, every rank pads to the longest, and the padding is dropped."""
    import torch

    n = len(arrays[0])
    sizes = torch.tensor([n], dtype=torch.int64, device=device)
    world = dist.get_world_size(group)
    all_sizes = [torch.zeros(1, dtype=torch.int64, device=device) for _ in range(world)]
    dist.all_gather(all_sizes, sizes, group=group)
    lens = [int(s.item()) for s in all_sizes]
    cap = max(lens) if lens else 0
    out = []
    for a in arrays:
        t = torch.as_tensor(np.ascontiguousarray(a)).to(device)
        buf = torch.zeros(max(cap, 1), dtype=t.dtype, device=device)
        buf[:n] = t
        parts = [torch.zeros_like(buf) for _ in range(world)]
        dist.all_gather(parts, buf, group=group)
        out.append(torch.cat([p[:ln] for p, ln in zip(parts, lens)]).cpu().numpy())
    return out, lens


class ShardedIVF:
    """One rank of a data-parallel run.

    backend: the rank's clustering context over its shard (an ``ivf.IVF``,
    or any object with ``assign() -> stats dict``, ``get_partial_sums()``,
    ``update_from_partials(cluster, term, sums)`` and ``get_assign()``);
    dist: ``torch.distributed`` with an initialised process group;
    device: where the exchange buffers live ("cuda" for NCCL, "cpu" for gloo).
    """

    def __init__(self, backend, dist, group=None, device="cpu"):
        self.m = backend
        self.dist = dist
        self.group = group
        self.device = device
        self.exchanged = []  # per iteration: member sums sent by each rank

    def iterate(self, max_iter: int):
        """Assign + exchange + update until no object changes anywhere (from
        the second iteration on) or max_iter.  Returns (iterations, converged)."""
        import torch

        for r in range(1, max_iter + 1):
            st = self.m.assign()
            cl, tm, sm = self.m.get_partial_sums()
            (gcl, gtm, gsm), lens = all_gather_concat((cl, tm, sm), self.dist, self.group, self.device)
            self.exchanged.append(lens)
            self.m.update_from_partials(gcl, gtm, gsm)
            changed = torch.tensor([int(st["n_changed"])], dtype=torch.int64, device=self.device)
            self.dist.all_reduce(changed, group=self.group)
            if r >= 2 and int(changed.item()) == 0:
                return r, True
        return max_iter, False
