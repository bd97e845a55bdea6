"""Exact, deliberately naive reference computations used to pin the oracle.

Written from the definitions (modularity Eq. 1; the core-community rule
Eq. 2), in pure Python integers / Fractions, independent of ``oracle/``.
"""
from fractions import Fraction

import numpy as np


def edges_of(row_ptr, col, w):
    """Undirected edge list {(u, v): weight} with u <= v from a symmetric CSR."""
    rp = np.asarray(row_ptr)
    c = np.asarray(col)
    out = {}
    for u in range(len(rp) - 1):
        for e in range(rp[u], rp[u + 1]):
            v = int(c[e])
            if v >= u:
                out[(u, v)] = 1 if w is None else int(np.asarray(w)[e])
    return out


def modularity_fraction(n, edges, labels, gamma=Fraction(1)):
    """mod(zeta, G) = sum_C omega(C)/omega(E) - gamma vol(C)^2 / (4 omega(E)^2);
    gamma = 1 is modularity (Eq. 1), other values the resolution-scaled
    objective that the gamma parameter of Section III-B optimises.

    vol(u): sum of incident non-loop edge weights plus twice the loop weight.
    omega(C): weight of edges with both ends in C, a loop counted once."""
    W = sum(edges.values())
    if W == 0:
        return Fraction(0)
    vol = [0] * n
    for (u, v), wt in edges.items():
        if u == v:
            vol[u] += 2 * wt
        else:
            vol[u] += wt
            vol[v] += wt
    comm = {}
    for u in range(n):
        comm.setdefault(int(labels[u]), []).append(u)
    q = Fraction(0)
    for c, members in comm.items():
        ms = set(members)
        inner = sum(wt for (u, v), wt in edges.items() if u in ms and v in ms)
        vc = sum(vol[u] for u in members)
        q += Fraction(inner, W) - gamma * Fraction(vc * vc, 4 * W * W)
    return q


def set_partitions(n):
    """All set partitions of range(n) as restricted-growth label arrays."""
    if n == 0:
        return np.zeros((1, 0), np.int32)
    out = [[0]]
    for i in range(1, n):
        nxt = []
        for p in out:
            m = max(p)
            for c in range(m + 2):
                nxt.append(p + [c])
        out = nxt
    return np.array(out, dtype=np.int32)


def max_modularity_bruteforce(n, edges):
    """Max modularity over all set partitions (vectorised over partitions)."""
    P = set_partitions(n)
    W = sum(edges.values())
    vol = np.zeros(n, np.int64)
    inner2 = np.zeros(len(P), np.int64)   # sum_C 2 omega(C)
    for (u, v), wt in edges.items():
        if u == v:
            vol[u] += 2 * wt
            inner2 += 2 * wt
        else:
            vol[u] += wt
            vol[v] += wt
            inner2 += 2 * wt * (P[:, u] == P[:, v])
    sq = np.zeros(len(P), np.int64)
    for c in range(n):
        vc = (P == c).astype(np.int64) @ vol
        sq += vc * vc
    num = 2 * W * inner2 - sq                 # over 4 W^2
    best = int(np.argmax(num))
    return Fraction(int(num[best]), 4 * W * W), P[best]
