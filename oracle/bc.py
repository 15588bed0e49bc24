"""Betweenness-centrality oracle (test infrastructure only): Brandes' algorithm
for a batch of sources on an unweighted graph, in plain Python and float64.

Only the tests, the smoke check and the benchmark's CPU-baseline leg may use
this module; it shares no code with the CUDA path.

The batched approximate BC of Section 3.2 sums, over the chosen sources s,
the dependency delta_s(v) = sum over t of sigma_st(v) / sigma_st (Eq. 1
restricted to the sources): a breadth-first search from s counts the shortest
paths sigma_s(v) level by level, and a sweep from the deepest level back
accumulates delta_s(v) = sum over children w of sigma_s(v)/sigma_s(w) *
(1 + delta_s(w)).  ``levels`` also returns, per BFS level, the number of
(vertex, source) pairs discovered, which the batched algorithm's frontiers
hold.
"""
from __future__ import annotations

from collections import deque

import numpy as np


def _neighbours(A):
    cp = np.asarray(A.colptr, dtype=np.int64)
    rows = np.asarray(A.rowidx, dtype=np.int64)
    return [rows[cp[v]:cp[v + 1]] for v in range(int(A.ncols))]


def brandes(A, sources):
    """BC scores (float64, length n) summed over ``sources`` and the frontier
    size of every BFS level summed over the sources.  A is a square CSC
    pattern (values ignored); column v lists the neighbours of v."""
    n = int(A.ncols)
    nb = _neighbours(A)
    bc = np.zeros(n, dtype=np.float64)
    level_sizes = []
    for s in sources:
        s = int(s)
        sigma = np.zeros(n, dtype=np.float64)
        dist = np.full(n, -1, dtype=np.int64)
        sigma[s] = 1.0
        dist[s] = 0
        order = []
        q = deque([s])
        while q:
            v = q.popleft()
            order.append(v)
            for w in nb[v]:
                w = int(w)
                if dist[w] < 0:
                    dist[w] = dist[v] + 1
                    q.append(w)
                if dist[w] == dist[v] + 1:
                    sigma[w] += sigma[v]
        depth = int(dist.max())
        for d in range(depth + 1):
            cnt = int(np.count_nonzero(dist == d))
            if d < len(level_sizes):
                level_sizes[d] += cnt
            else:
                level_sizes.append(cnt)
        delta = np.zeros(n, dtype=np.float64)
        for w in reversed(order):
            for v in nb[w]:
                v = int(v)
                if dist[v] == dist[w] - 1:
                    delta[v] += sigma[v] / sigma[w] * (1.0 + delta[w])
            if w != s:
                bc[w] += delta[w]
    return bc, level_sizes
