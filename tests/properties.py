"""Properties of results that hold at any size, checked with numpy.

At the benchmark sizes (R-MAT scale 22 and up) the oracle is too slow to
run, so the GPU results there are checked against properties that determine
or constrain them, written from the definitions:

* the schedule colouring is first-fit Jones-Plassmann: every vertex has the
  smallest colour not used by its higher-priority neighbours (hub-hub edges,
  both ends above 4096 neighbours, excluded; self-loops ignored).  Checking
  this at every vertex determines the colouring completely.
* modularity (Eq. 1) of a labelling, as an exact integer fraction;
* a converged PLMR result has no vertex with a positive-gain move (the last
  move phase at the finest level ends on a sweep in which no vertex wants
  to move, and nothing moved during it).

Each checker is pinned on small graphs against the oracle's results and
against planted mistakes (tests/test_properties_cpu.py).  Nothing here
imports the oracle or the CUDA library.
"""
import numpy as np

HUB_RELAX = 4096   # hubs: more than this many neighbours, self-loop not counted


def fmix32(h):
    """MurmurHash3's 32-bit finaliser on a uint32 array."""
    h = np.asarray(h, dtype=np.uint32).copy()
    h ^= h >> np.uint32(16)
    h *= np.uint32(0x85EBCA6B)
    h ^= h >> np.uint32(13)
    h *= np.uint32(0xC2B2AE35)
    h ^= h >> np.uint32(16)
    return h


def priority_keys(n, seed):
    """(fmix32(v ^ s), v) as one uint64 per vertex, s = fmix32(seed_lo ^ seed_hi);
    a larger key is a higher priority."""
    s = fmix32(np.uint32((seed & 0xFFFFFFFF) ^ (seed >> 32)))
    v = np.arange(n, dtype=np.uint32)
    return (fmix32(v ^ s).astype(np.uint64) << np.uint64(32)) | v.astype(np.uint64)


def _entries(row_ptr, col):
    rp = np.asarray(row_ptr, dtype=np.int64)
    c = np.asarray(col, dtype=np.int64)
    n = len(rp) - 1
    src = np.repeat(np.arange(n, dtype=np.int64), np.diff(rp))
    return n, rp, src, c


def check_first_fit_colouring(row_ptr, col, colour, seed):
    """Raises AssertionError unless `colour` is the first-fit Jones-Plassmann
    colouring of the graph (without hub-hub edges) under the seed's priority."""
    n, rp, src, c = _entries(row_ptr, col)
    colour = np.asarray(colour, dtype=np.int64)
    assert colour.shape == (n,)
    if n == 0:
        return
    assert colour.min() >= 0
    deg = np.diff(rp) - np.bincount(src[src == c], minlength=n)   # neighbours, self-loop not counted
    hub = deg > HUB_RELAX
    keep = (src != c) & ~(hub[src] & hub[c])
    u, x = src[keep], c[keep]
    key = priority_keys(n, seed)
    higher = key[x] > key[u]
    u, x = u[higher], x[higher]          # x constrains u
    cu, cx = colour[u], colour[x]
    bad = np.flatnonzero(cu == cx)
    assert bad.size == 0, f"vertex {u[bad[0]]} shares colour {cu[bad[0]]} with higher-priority neighbour {x[bad[0]]}"
    # every colour below colour(u) is taken by some constraint of u
    below = cx < cu
    K = int(colour.max()) + 1
    pairs = np.unique(u[below] * K + cx[below])
    distinct = np.bincount(pairs // K, minlength=n)
    wrong = np.flatnonzero(distinct != colour)
    assert wrong.size == 0, (f"vertex {wrong[0]} has colour {colour[wrong[0]]} but only {distinct[wrong[0]]} "
                             "smaller colours among its higher-priority neighbours")


def _weights(w, m):
    return np.ones(m, dtype=np.int64) if w is None else np.asarray(w, dtype=np.int64)


def _int_sums(index, values, length):
    """Per-index sums of non-negative integers, exact: float64 sums are exact
    while every partial sum stays below 2^53."""
    values = np.asarray(values, dtype=np.int64)
    assert values.size == 0 or (values.min() >= 0 and int(values.sum()) < 2 ** 53)
    return np.rint(np.bincount(index, weights=values.astype(np.float64), minlength=length)).astype(np.int64)


def volumes(row_ptr, col, w):
    """vol(u) = sum of non-loop incident weights + 2 * loop weight; and W."""
    n, rp, src, c = _entries(row_ptr, col)
    wt = _weights(w, len(c))
    loop = src == c
    vol = _int_sums(src, wt * np.where(loop, 2, 1), n)
    W = (int(wt[~loop].sum()) // 2) + int(wt[loop].sum())
    return vol, W


def modularity_exact(row_ptr, col, w, labels, fraction=False):
    """Eq. 1 as (2W * S_in - S_vol2) / (4 W^2) with exact integers:
    S_in = 2 * sum_C omega(C), S_vol2 = sum_C vol(C)^2.  With fraction=True
    returns (value, numerator, denominator), the last two as Python ints."""
    n, rp, src, c = _entries(row_ptr, col)
    wt = _weights(w, len(c))
    lab = np.asarray(labels, dtype=np.int64)
    vol, W = volumes(row_ptr, col, w)
    if W == 0:
        return (0.0, 0, 0) if fraction else 0.0
    loop = src == c
    same = lab[src] == lab[c]
    s_in = int(wt[same & ~loop].sum()) + 2 * int(wt[loop].sum())
    vc = _int_sums(lab, vol, int(lab.max()) + 1 if n else 0)
    s_vol2 = sum(int(v) * int(v) for v in vc[vc != 0])
    N, D = 2 * W * s_in - s_vol2, 4 * W * W
    return (N / D, N, D) if fraction else N / D


def check_dense_labels(labels):
    """Labels are 0..k-1, every one used."""
    lab = np.asarray(labels, dtype=np.int64)
    if lab.size == 0:
        return 0
    k = int(lab.max()) + 1
    assert lab.min() == 0
    used = np.bincount(lab, minlength=k)
    assert np.all(used > 0), f"label {int(np.flatnonzero(used == 0)[0])} unused"
    return k


def positive_gain_moves(row_ptr, col, w, labels, sample):
    """Vertices of `sample` that have a move u: C -> D (D a neighbour's
    community, D != C) with gain
        2W (omega(u,D) - omega(u,C\\u)) - vol(u) (vol(D) - vol(C\\u)) > 0,
    computed exactly; returns a list of (u, D, gain)."""
    rp = np.asarray(row_ptr, dtype=np.int64)
    c = np.asarray(col, dtype=np.int64)
    wt = _weights(w, len(c))
    lab = np.asarray(labels, dtype=np.int64)
    vol, W = volumes(row_ptr, col, w)
    vc = _int_sums(lab, vol, int(lab.max()) + 1 if lab.size else 0)
    out = []
    for u in np.asarray(sample, dtype=np.int64):
        u = int(u)
        nb = c[rp[u]:rp[u + 1]]
        ws = wt[rp[u]:rp[u + 1]]
        keep = nb != u
        nb, ws = nb[keep], ws[keep]
        C = int(lab[u])
        vu = int(vol[u])
        omega = {}
        for x, wx in zip(lab[nb].tolist(), ws.tolist()):
            omega[x] = omega.get(x, 0) + wx
        wC = omega.get(C, 0)
        volC = int(vc[C]) - vu
        for D, wD in omega.items():
            if D == C:
                continue
            g = 2 * W * (wD - wC) - vu * (int(vc[D]) - volC)
            if g > 0:
                out.append((u, D, g))
    return out
