"""Seeded synthetic graph generators (inputs only: no community-detection arithmetic).

Both the oracle and the CUDA path take their graphs from here.  Every random
number is drawn from a counter-based splitmix64 stream (Steele, Lea & Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014): value i of
stream (seed, s) is mix(key + (i+1)*GAMMA) with key = mix(mix(seed) ^ s), so any
element can be drawn independently and in any order.  The generators run on
whatever torch device they are given (CPU in tests, CUDA for large workloads);
outputs are deterministic per device.  R-MAT and the vertex permutations use
integer arithmetic only and so are identical on every device; the planted
partition and Chung-Lu samplers use float64 logarithms / quantiles, whose last
bits may differ between CPU and GPU libm, so those graphs are only guaranteed
identical on the same device type.

Families (stand-ins for the paper's test graphs, Section V-B, Table II):
  * planted partition G(n, p_in, p_out) (the paper's ``G_n_pin_pout``),
    sampled per block pair with geometric skipping (Batagelj & Brandes 2005);
  * R-MAT (Chakrabarti, Zhan & Faloutsos 2004) with a seeded vertex
    permutation, as in Graph500 Kronecker graphs (``kron_g500-simple-logn*``);
  * Chung-Lu power-law graphs with deterministic truncated-Pareto expected
    degrees.

All graphs come out as symmetric CSR: ``row_ptr`` int64[n+1], ``col`` int32
sorted ascending per row without duplicates, ``w`` int32 (or None for unit
weights).  Self-loops are dropped.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Optional

import torch

MASK64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15


def _s64(x: int) -> int:
    """Python int in [0, 2^64) -> the int64 with the same bit pattern."""
    x &= MASK64
    return x - (1 << 64) if x >= (1 << 63) else x


def _mix_int(z: int) -> int:
    z &= MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def stream_key(seed: int, stream: int) -> int:
    return _mix_int(_mix_int(seed) ^ (stream & MASK64))


def _srl(x: torch.Tensor, k: int) -> torch.Tensor:
    """Logical right shift of int64 lanes."""
    return (x >> k) & ((1 << (64 - k)) - 1)


def _mix(z: torch.Tensor) -> torch.Tensor:
    z = (z ^ _srl(z, 30)) * _s64(0xBF58476D1CE4E5B9)
    z = (z ^ _srl(z, 27)) * _s64(0x94D049BB133111EB)
    return z ^ _srl(z, 31)


def rand_u64(seed: int, stream: int, idx: torch.Tensor) -> torch.Tensor:
    """Raw 64-bit draws (as int64 bit patterns) for counters ``idx`` (int64)."""
    key = stream_key(seed, stream)
    return _mix(idx * _s64(GAMMA) + _s64(key + GAMMA))


def rand_u53(seed: int, stream: int, idx: torch.Tensor) -> torch.Tensor:
    """Top 53 bits of each draw, as int64 in [0, 2^53)."""
    return _srl(rand_u64(seed, stream, idx), 11)


def rand_unit(seed: int, stream: int, idx: torch.Tensor) -> torch.Tensor:
    """Uniform float64 in [0, 1)."""
    return rand_u53(seed, stream, idx).to(torch.float64) * (1.0 / (1 << 53))


@dataclass
class Graph:
    n: int
    row_ptr: torch.Tensor          # int64 [n+1]
    col: torch.Tensor              # int32 [nnz]
    w: Optional[torch.Tensor]      # int32 [nnz] or None (unit weights)
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.col.numel())

    @property
    def m(self) -> int:
        """Undirected, loop-free edge count (the edges/s numerator)."""
        return self.nnz // 2

    def to(self, device) -> "Graph":
        return Graph(self.n, self.row_ptr.to(device), self.col.to(device),
                     None if self.w is None else self.w.to(device), self.name)

    def numpy(self):
        return (self.row_ptr.cpu().numpy(), self.col.cpu().numpy(),
                None if self.w is None else self.w.cpu().numpy())


def csr_from_undirected(n: int, a: torch.Tensor, b: torch.Tensor,
                        w: Optional[torch.Tensor], name: str = "") -> Graph:
    """Build a symmetric CSR from undirected edges {a_i, b_i} (a_i != b_i).

    Duplicate pairs are merged keeping the first weight in key order (callers
    pass unique pairs, or weights that depend only on the pair)."""
    dev = a.device
    lo = torch.minimum(a, b).to(torch.int64)
    hi = torch.maximum(a, b).to(torch.int64)
    keep = lo != hi
    lo, hi = lo[keep], hi[keep]
    if w is not None:
        w = w[keep]
    key = lo * n + hi
    if w is None:
        key = torch.unique(key)
    else:
        key, perm = torch.sort(key, stable=True)
        first = torch.ones_like(key, dtype=torch.bool)
        if key.numel() > 1:
            first[1:] = key[1:] != key[:-1]
        key = key[first]
        w = w[perm][first]
    lo = key // n
    hi = key % n
    src = torch.cat([lo, hi])
    dst = torch.cat([hi, lo])
    ww = None if w is None else torch.cat([w, w]).to(torch.int32)
    key2 = src * n + dst
    key2, perm = torch.sort(key2)
    src = key2 // n
    dst = key2 % n
    if ww is not None:
        ww = ww[perm]
    counts = torch.bincount(src, minlength=n)
    row_ptr = torch.zeros(n + 1, dtype=torch.int64, device=dev)
    row_ptr[1:] = torch.cumsum(counts, 0)
    return Graph(n, row_ptr, dst.to(torch.int32), ww, name)


def permutation(n: int, seed: int, stream: int, device) -> torch.Tensor:
    """Seeded random permutation of [0, n): sort of (draw, index) pairs."""
    idx = torch.arange(n, dtype=torch.int64, device=device)
    r = rand_u53(seed, stream, idx)
    # keys are distinct with overwhelming probability; stable sort breaks ties by index
    _, perm = torch.sort(r, stable=True)
    return perm


# ---------------------------------------------------------------------------
# R-MAT
# ---------------------------------------------------------------------------

def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19,
         c: float = 0.19, seed: int = 1, device="cpu", weighted: bool = False,
         chunk: int = 1 << 26) -> Graph:
    """R-MAT graph: 2^scale vertices, edge_factor * 2^scale generated edges.

    Each edge descends ``scale`` levels; at every level one 53-bit draw picks
    the quadrant with probabilities (a, b, c, 1-a-b-c) using integer
    thresholds.  A seeded permutation relabels the vertices; then the edges are
    symmetrised, de-duplicated and loops dropped.  Unit weights unless
    ``weighted`` (then 1..100, a function of the unordered pair)."""
    n = 1 << scale
    m_gen = edge_factor << scale
    ta = int(a * (1 << 53))
    tab = int((a + b) * (1 << 53))
    tabc = int((a + b + c) * (1 << 53))
    perm = permutation(n, seed, 0x5EED0000, device)
    keys = []
    for s in range(0, m_gen, chunk):
        e = min(m_gen, s + chunk)
        idx = torch.arange(s, e, dtype=torch.int64, device=device)
        src = torch.zeros_like(idx)
        dst = torch.zeros_like(idx)
        for lvl in range(scale):
            r = rand_u53(seed, lvl, idx)
            bs = (r >= tab).to(torch.int64)
            bd = ((r >= ta) & (r < tab)) | (r >= tabc)
            bit = 1 << (scale - 1 - lvl)
            src |= bs * bit
            dst |= bd.to(torch.int64) * bit
        src = perm[src]
        dst = perm[dst]
        keep = src != dst
        lo = torch.minimum(src[keep], dst[keep])
        hi = torch.maximum(src[keep], dst[keep])
        keys.append(torch.unique(lo * n + hi))
        del src, dst, idx, lo, hi
    key = torch.unique(torch.cat(keys))
    del keys
    lo, hi = key // n, key % n
    w = None
    if weighted:
        w = (_srl(rand_u64(seed, 0x3E16, key), 11) % 100 + 1).to(torch.int32)
    return csr_from_undirected(n, lo, hi, w, name=f"rmat{scale}_ef{edge_factor}")


# ---------------------------------------------------------------------------
# Planted partition
# ---------------------------------------------------------------------------

def _block_sizes(n: int, k: int):
    base, rem = divmod(n, k)
    return [base + (1 if i < rem else 0) for i in range(k)]


def planted_partition(n: int, k: int, p_in: float, p_out: float, seed: int = 1,
                      device="cpu", sizes=None) -> Graph:
    """G(n, p_in, p_out) with k equal blocks (remainder spread over the first
    blocks).  Every unordered vertex pair is an edge independently with p_in
    inside a block and p_out across; each block pair's candidate pairs are
    visited with geometric skipping.  Unit weights, no loops."""
    sizes = sizes or _block_sizes(n, k)
    starts = [0]
    for s in sizes[:-1]:
        starts.append(starts[-1] + s)
    us, vs = [], []
    pair_id = 0
    for i in range(len(sizes)):
        for j in range(i, len(sizes)):
            p = p_in if i == j else p_out
            si, sj = sizes[i], sizes[j]
            npairs = si * (si - 1) // 2 if i == j else si * sj
            pid = pair_id
            pair_id += 1
            if npairs == 0 or p <= 0.0:
                continue
            pos = _skip_sample(npairs, p, seed, pid, device)
            if pos.numel() == 0:
                continue
            if i == j:
                # strictly-lower-triangle index -> (r, c), r > c
                r = torch.floor((1.0 + torch.sqrt(1.0 + 8.0 * pos.to(torch.float64))) / 2.0).to(torch.int64)
                r = torch.where(r * (r - 1) // 2 > pos, r - 1, r)
                r = torch.where((r + 1) * r // 2 <= pos, r + 1, r)
                c = pos - r * (r - 1) // 2
                us.append(starts[i] + r)
                vs.append(starts[i] + c)
            else:
                us.append(starts[i] + pos // sj)
                vs.append(starts[j] + pos % sj)
    if us:
        a = torch.cat(us)
        b = torch.cat(vs)
    else:
        a = torch.zeros(0, dtype=torch.int64, device=device)
        b = torch.zeros(0, dtype=torch.int64, device=device)
    return csr_from_undirected(n, a, b, None, name=f"pp_n{n}_k{len(sizes)}")


def _tri_rc(pos: torch.Tensor):
    """Strictly-lower-triangle index -> (r, c) with r > c >= 0."""
    r = torch.floor((1.0 + torch.sqrt(1.0 + 8.0 * pos.to(torch.float64))) / 2.0).to(torch.int64)
    r = torch.where(r * (r - 1) // 2 > pos, r - 1, r)
    r = torch.where((r + 1) * r // 2 <= pos, r + 1, r)
    return r, pos - r * (r - 1) // 2


def planted_partition_fast(n: int, k: int, p_in: float, p_out: float, seed: int = 1,
                           device="cpu") -> Graph:
    """G(n, p_in, p_out) with k equal blocks (remainder spread over the first
    blocks), sampled in two passes instead of one per block pair: the
    intra-block pairs of all blocks, laid end to end, with probability p_in,
    and every unordered pair with probability p_out, keeping only pairs whose
    ends lie in different blocks.  Each pair is still an edge independently
    with p_in inside a block and p_out across (same distribution as
    ``planted_partition``, different random stream), with a few large
    operations per graph, so big batches generate quickly on a GPU."""
    sizes = _block_sizes(n, k)
    sz = torch.tensor(sizes, dtype=torch.int64, device=device)
    starts = torch.cumsum(sz, 0) - sz
    tri = sz * (sz - 1) // 2
    tri_end = torch.cumsum(tri, 0)
    us, vs = [], []
    total_in = int(tri_end[-1]) if k > 0 else 0
    if total_in > 0 and p_in > 0.0:
        pos = _skip_sample(total_in, p_in, seed, 0x0F00001, device)
        blk = torch.searchsorted(tri_end, pos, right=True)
        r, c = _tri_rc(pos - (tri_end[blk] - tri[blk]))
        us.append(starts[blk] + r)
        vs.append(starts[blk] + c)
    if n > 1 and p_out > 0.0:
        pos = _skip_sample(n * (n - 1) // 2, p_out, seed, 0x0F00002, device)
        r, c = _tri_rc(pos)
        ends = starts + sz
        cross = torch.searchsorted(ends, r, right=True) != torch.searchsorted(ends, c, right=True)
        us.append(r[cross])
        vs.append(c[cross])
    if us:
        a, b = torch.cat(us), torch.cat(vs)
    else:
        a = b = torch.zeros(0, dtype=torch.int64, device=device)
    return csr_from_undirected(n, a, b, None, name=f"ppf_n{n}_k{k}")


def _skip_sample(npairs: int, p: float, seed: int, stream: int, device) -> torch.Tensor:
    """Sorted positions in [0, npairs) kept with probability p (geometric gaps)."""
    if p >= 1.0:
        return torch.arange(npairs, dtype=torch.int64, device=device)
    lq = math.log1p(-p)
    out = []
    drawn = 0
    last = -1
    while True:
        exp = (npairs - last - 1) * p
        cnt = int(exp + 8.0 * math.sqrt(exp + 1.0) + 64)
        idx = torch.arange(drawn, drawn + cnt, dtype=torch.int64, device=device)
        u = rand_unit(seed, 0x70000000 + stream, idx)
        gap = torch.floor(torch.log1p(-u) / lq).to(torch.int64) + 1
        pos = last + torch.cumsum(gap, 0)
        drawn += cnt
        inside = pos < npairs
        out.append(pos[inside])
        if not bool(inside[-1]):
            break
        last = int(pos[-1])
    return torch.cat(out)


# ---------------------------------------------------------------------------
# Chung-Lu power law
# ---------------------------------------------------------------------------

def chung_lu(n: int, gamma: float = 2.1, dmin: float = 4.0, dmax: float = 1e5,
             seed: int = 1, device="cpu", wmax: int = 100, chunk: int = 1 << 26) -> Graph:
    """Chung-Lu graph with expected degrees from a truncated Pareto law.

    Expected degree of (pre-permutation) vertex i is the ((i+0.5)/n)-quantile
    of the density ~ x^-gamma on [dmin, dmax].  sum(w)/2 endpoint pairs are
    drawn, each endpoint independently with probability proportional to its
    expected degree (inverse CDF on the cumulative degrees); vertex ids are
    permuted by a seed; duplicates and loops are dropped.  Integer weights are
    uniform in 1..wmax, a function of the unordered pair (so symmetric)."""
    q = (torch.arange(n, dtype=torch.float64, device=device) + 0.5) / n
    e = 1.0 - gamma
    lo_, hi_ = dmin ** e, dmax ** e
    wdeg = (lo_ - q * (lo_ - hi_)) ** (1.0 / e)
    cdf = torch.cumsum(wdeg, 0)
    total = float(cdf[-1])
    m_gen = int(total / 2)
    perm = permutation(n, seed, 0xC1C1, device)
    keys = []
    for s in range(0, m_gen, chunk):
        cnt = min(m_gen, s + chunk) - s
        idx = torch.arange(s, s + cnt, dtype=torch.int64, device=device)
        ua = rand_unit(seed, 0xC2, idx) * total
        ub = rand_unit(seed, 0xC3, idx) * total
        ia = torch.searchsorted(cdf, ua, right=True).clamp_(max=n - 1)
        ib = torch.searchsorted(cdf, ub, right=True).clamp_(max=n - 1)
        a, b = perm[ia], perm[ib]
        keep = a != b
        lo = torch.minimum(a[keep], b[keep])
        hi = torch.maximum(a[keep], b[keep])
        keys.append(torch.unique(lo * n + hi))
        del ua, ub, ia, ib, a, b, lo, hi, idx
    key = torch.unique(torch.cat(keys))
    del keys
    w = (_srl(rand_u64(seed, 0xC4, key), 11) % wmax + 1).to(torch.int32)
    return csr_from_undirected(n, key // n, key % n, w, name=f"chunglu_n{n}")


# ---------------------------------------------------------------------------
# Small hand-made graphs for tests
# ---------------------------------------------------------------------------

def from_edge_list(n: int, edges, weights=None, self_loops=None) -> Graph:
    """Symmetric CSR from a Python list of undirected edges (u, v); optional
    int weights; optional {u: weight} self-loops (stored once in row u)."""
    rows = [dict() for _ in range(n)]
    for i, (u, v) in enumerate(edges):
        wt = 1 if weights is None else int(weights[i])
        assert u != v
        rows[u][v] = rows[u].get(v, 0) + wt
        rows[v][u] = rows[v].get(u, 0) + wt
    for u, wt in (self_loops or {}).items():
        rows[u][u] = rows[u].get(u, 0) + int(wt)
    row_ptr = [0]
    col, w = [], []
    for u in range(n):
        for v in sorted(rows[u]):
            col.append(v)
            w.append(rows[u][v])
        row_ptr.append(len(col))
    unit = weights is None and not self_loops and all(x == 1 for x in w)
    return Graph(n, torch.tensor(row_ptr, dtype=torch.int64),
                 torch.tensor(col, dtype=torch.int32),
                 None if unit else torch.tensor(w, dtype=torch.int32), "edgelist")


def random_graph(n: int, m: int, seed: int, weighted: bool = True,
                 loops: int = 0, wmax: int = 9) -> Graph:
    """Small random multigraph-free graph for pins: m pairs drawn uniformly,
    merged, plus ``loops`` random self-loops.  Host-side, pure Python."""
    idx = torch.arange(4 * m + 2 * loops + 4, dtype=torch.int64)
    r = rand_u53(seed, 0xAB, idx).tolist()
    edges, ws = [], []
    seen = set()
    for i in range(m):
        u, v = r[4 * i] % n, r[4 * i + 1] % n
        if u == v or (min(u, v), max(u, v)) in seen:
            continue
        seen.add((min(u, v), max(u, v)))
        edges.append((u, v))
        ws.append(1 + r[4 * i + 2] % wmax if weighted else 1)
    sl = {}
    for j in range(loops):
        u = r[4 * m + 2 * j] % n
        sl[u] = 1 + r[4 * m + 2 * j + 1] % wmax
    return from_edge_list(n, edges, ws if weighted else None, sl)


def cliques(k: int, s: int, ring: bool = False) -> Graph:
    """k disjoint cliques K_s (vertex block i*s..i*s+s-1); with ``ring``,
    clique i's last vertex is joined to clique i+1's first vertex (mod k)."""
    edges = []
    for i in range(k):
        b = i * s
        for x in range(s):
            for y in range(x + 1, s):
                edges.append((b + x, b + y))
        if ring and k > 1:
            edges.append((b + s - 1, ((i + 1) % k) * s))
    return from_edge_list(k * s, edges)


# ---------------------------------------------------------------------------
# Workload recipes
# ---------------------------------------------------------------------------

def planted_partition_config1(device="cpu") -> Graph:
    """n=10,000, 20 blocks of 500, p_in=0.02, p_out=0.0005, seed 1."""
    return planted_partition(10_000, 20, 0.02, 0.0005, seed=1, device=device)


def batch_planted_specs(count: int = 512, seed0: int = 1000, nmin: int = 1_000,
                        nmax: int = 1_000_000, avg_deg: float = 16.0, ratio: float = 20.0):
    """Per-graph (n, k, p_in, p_out, seed) for the batched workload:
    n log-uniform in [nmin, nmax], k uniform in [8, 64], p_in/p_out = ratio,
    expected average degree ``avg_deg``."""
    specs = []
    for j in range(count):
        sd = seed0 + j
        r = rand_u53(sd, 0xBA7C, torch.arange(2, dtype=torch.int64)).tolist()
        u = r[0] / float(1 << 53)
        n = int(round(math.exp(math.log(nmin) + u * (math.log(nmax) - math.log(nmin)))))
        k = 8 + r[1] % 57
        s = n / k
        p_out = avg_deg / (ratio * (s - 1) + (n - s))
        p_in = min(1.0, ratio * p_out)
        specs.append((n, k, p_in, p_out, sd))
    return specs
