"""Algorithm 3 (IVF) written out step by step in FP64, for small inputs.

Test infrastructure only.  Plain Python loops in the paper's order and
notation, used to pin the paper's claim (Section 3, and the Lloyd-type
property noted in Section 2.1) that IVF keeps the solution of the standard
Lloyd iteration from the same initial state, and to count multiplications
(Eq. 15).

Inverted file of the means (Section 3): for every term s a list
xi_s = ((c_(s,q), u_(s,q)))_{q=1..(nc)_s} in ascending cluster id, because
the update step appends cluster j's tuples while j runs upward.

Readings (shared with spherical_kmeans): R1/R2 for the argmax (lowest id
among all maxima, so an all-zero rho goes to cluster 0, where the printed
loop starting from rho_max = 0 would leave the object unassigned); R3 for an
empty cluster (its previous tuples are re-emitted under empty_policy 0,
nothing under 1; the printed division by |C_j| = 0 would give NaN).
"""
from __future__ import annotations

import math


def inverted_file_from_means(means) -> list:
    """xi[s] = [(c, u), ...] ascending in c, from cluster-major means."""
    xi = [[] for _ in range(means.n_terms)]
    for j in range(means.k):
        for t, u in zip(*means.row(j)):
            xi[int(t)].append((j, float(u)))
    return xi


def assignment_step(corpus, xi, k: int):
    """Assignment step of Algorithm 3: the triple loop, then the argmax.

    Returns (assign, best, rho_rows, multiplications).
    """
    assign, best, rho_rows = [], [], []
    mults = 0
    for i in range(corpus.n_docs):
        rho = [0.0] * k                                       # rho <- 0
        a0, a1 = int(corpus.row_ptr[i]), int(corpus.row_ptr[i + 1])
        for h in range(a0, a1):                                # s <- t_(i,h) in S_i
            s = int(corpus.term[h])
            v = float(corpus.val[h])
            for c, u in xi[s]:                                 # (c, u) in xi_s
                rho[c] = rho[c] + v * u                        # rho_c += v * u
                mults += 1
        rho_max, a = rho[0], 0                                 # j = 1..k, strict '>' (R1, R2)
        for j in range(1, k):
            if rho[j] > rho_max:
                rho_max, a = rho[j], j
        assign.append(a)
        best.append(rho_max)
        rho_rows.append(rho)
    return assign, best, rho_rows, mults


def update_step(corpus, assign, k: int, n_terms: int, prev_xi=None, empty_policy: int = 0):
    """Update step of Algorithm 3: per cluster a full w, / |C_j|, emit w_p / ||w||.

    Clusters are visited in ascending j so every list ends up ascending in c.
    """
    members = [[] for _ in range(k)]
    for i, a in enumerate(assign):
        members[a].append(i)
    xi = [[] for _ in range(n_terms)]
    prev_rows = None
    if prev_xi is not None:
        prev_rows = [[] for _ in range(k)]
        for p in range(n_terms):
            for c, u in prev_xi[p]:
                prev_rows[c].append((p, u))
    for j in range(k):
        w = [0.0] * n_terms
        for i in members[j]:
            for h in range(int(corpus.row_ptr[i]), int(corpus.row_ptr[i + 1])):
                s = int(corpus.term[h])
                w[s] = w[s] + float(corpus.val[h])
        size = len(members[j])
        if size > 0:
            w = [wp / size for wp in w]
        norm = math.sqrt(sum(wp * wp for wp in w))
        if size == 0 or norm == 0.0:                           # R3
            if empty_policy == 0 and prev_rows is not None:
                for p, u in prev_rows[j]:
                    xi[p].append((j, u))
            continue
        for p in range(n_terms):
            if w[p] != 0.0:                                    # R4: emit only w_p != 0
                xi[p].append((j, w[p] / norm))
    return xi


def iterate(corpus, xi0, k: int, max_iter: int, empty_policy: int = 0):
    """Algorithm 3 for r = 1..max_iter; returns [(assign, best, xi_after), ...]."""
    out = []
    xi = xi0
    prev = None
    for r in range(1, max_iter + 1):
        a, best, _, _ = assignment_step(corpus, xi, k)
        xi = update_step(corpus, a, k, corpus.n_terms, prev_xi=xi, empty_policy=empty_policy)
        out.append((a, best, xi))
        if r >= 2 and prev == a:
            break
        prev = a
    return out
