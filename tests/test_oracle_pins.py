"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: closed forms
of Eq. (1), an independent exact (Fraction) modularity, networkx, brute force
over all partitions, invariants of coarsening (Section III-B), of the move rule
(Algorithm 2), of PLP (Algorithm 1) and of the core-community rule (Eq. 2).
"""
from fractions import Fraction
import itertools

import numpy as np
import pytest

from paper_1304_4453_gb300 import synth
from tests import exact

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def csr(g):
    return g.numpy()


# ---------------------------------------------------------------------------
# Modularity (Eq. 1)
# ---------------------------------------------------------------------------

def test_modularity_all_in_one_is_zero(oracle_mod):
    g = synth.random_graph(30, 80, seed=3, loops=4)
    rp, c, w = csr(g)
    q, N, D = oracle_mod.modularity(rp, c, w, np.zeros(g.n, np.int32))
    assert N == 0 and q == 0.0


@pytest.mark.parametrize("k,s", [(1, 3), (2, 5), (4, 4), (7, 3)])
def test_modularity_disjoint_cliques(oracle_mod, k, s):
    g = synth.cliques(k, s)
    rp, c, w = csr(g)
    lab = (np.arange(g.n) // s).astype(np.int32)
    q, N, D = oracle_mod.modularity(rp, c, w, lab)
    assert Fraction(N, D) == 1 - Fraction(1, k)


def test_modularity_singletons(oracle_mod):
    g = synth.random_graph(25, 60, seed=5, loops=5)
    rp, c, w = csr(g)
    ed = exact.edges_of(rp, c, w)
    W = sum(ed.values())
    vol = [0] * g.n
    for (u, v), wt in ed.items():
        vol[u] += wt if u != v else 2 * wt
        if u != v:
            vol[v] += wt
    loops = sum(wt for (u, v), wt in ed.items() if u == v)
    # a singleton keeps only its loop inside: sum_u s(u)/W - vol(u)^2/(4W^2)
    expect = Fraction(loops, W) - Fraction(sum(x * x for x in vol), 4 * W * W)
    q, N, D = oracle_mod.modularity(rp, c, w, np.arange(g.n, dtype=np.int32))
    assert Fraction(N, D) == expect


@pytest.mark.parametrize("r,s", [(3, 4), (5, 5), (8, 3)])
def test_modularity_ring_of_cliques(oracle_mod, r, s):
    g = synth.cliques(r, s, ring=True)
    rp, c, w = csr(g)
    lab = (np.arange(g.n) // s).astype(np.int32)
    q, N, D = oracle_mod.modularity(rp, c, w, lab)
    W = r * (s * (s - 1) // 2 + 1)
    per = Fraction(s * (s - 1) // 2, W) - Fraction((s * (s - 1) + 2) ** 2, 4 * W * W)
    assert Fraction(N, D) == r * per
    assert q == float(Fraction(N, D))


@pytest.mark.parametrize("seed", range(6))
def test_modularity_matches_exact_and_networkx(oracle_mod, seed):
    nx = pytest.importorskip("networkx")
    g = synth.random_graph(40, 120, seed=seed, loops=6)
    rp, c, w = csr(g)
    lab = np.asarray(synth.rand_u53(seed, 9, __import__("torch").arange(g.n)) % 6, np.int32)
    q, N, D = oracle_mod.modularity(rp, c, w, lab)
    ed = exact.edges_of(rp, c, w)
    assert Fraction(N, D) == exact.modularity_fraction(g.n, ed, lab)
    G = nx.Graph()
    G.add_nodes_from(range(g.n))
    for (u, v), wt in ed.items():
        G.add_edge(u, v, weight=wt)
    comms = [set(np.flatnonzero(lab == k).tolist()) for k in np.unique(lab)]
    assert abs(nx.community.modularity(G, comms, weight="weight") - q) < 1e-12


def test_modularity_edgeless_is_zero(oracle_mod):
    g = synth.from_edge_list(5, [])
    rp, c, w = csr(g)
    q, N, D = oracle_mod.modularity(rp, c, w, np.zeros(5, np.int32))
    assert q == 0.0


# ---------------------------------------------------------------------------
# Gain (Section III-B, Delta mod) == exact modularity difference
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(4))
def test_gain_equals_modularity_difference(oracle_mod, seed):
    g = synth.random_graph(14, 40, seed=100 + seed, loops=3)
    rp, c, w = csr(g)
    ed = exact.edges_of(rp, c, w)
    W = sum(ed.values())
    import torch
    lab = np.asarray(synth.rand_u53(seed, 1, torch.arange(g.n)) % 5, np.int32)
    before = exact.modularity_fraction(g.n, ed, lab)
    for u in range(g.n):
        for D in range(5):
            if D == lab[u]:
                continue
            after_lab = lab.copy()
            after_lab[u] = D
            after = exact.modularity_fraction(g.n, ed, after_lab)
            gnum = oracle_mod.gain(rp, c, w, lab, u, D)
            assert Fraction(gnum, 2 * W * W) == after - before, (u, D)


# ---------------------------------------------------------------------------
# Colouring (schedule)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("seed", [1, 2, 77])
def test_colouring_is_proper_and_first_fit(oracle_mod, seed):
    g = synth.rmat(10, seed=seed)
    rp, c, w = csr(g)
    k, col = oracle_mod.color(rp, c, w, seed)
    assert col.min() >= 0 and col.max() == k - 1
    for u in range(g.n):
        nb = c[rp[u]:rp[u + 1]]
        nb = nb[nb != u]
        assert not np.any(col[nb] == col[u])
        # first fit: every smaller colour appears among the neighbours
        assert set(range(col[u])) <= set(col[nb].tolist())
    k2, col2 = oracle_mod.color(rp, c, w, seed)
    assert np.array_equal(col, col2)


def _greedy_in_priority_order(rp, c, seed):
    """Sequential greedy colouring: vertices in descending priority
    (fmix32(v ^ fmix32(seed_lo ^ seed_hi)), v), each taking the smallest
    colour not used by its already coloured neighbours."""
    def fmix(h):
        h &= 0xFFFFFFFF
        h ^= h >> 16; h = (h * 0x85EBCA6B) & 0xFFFFFFFF
        h ^= h >> 13; h = (h * 0xC2B2AE35) & 0xFFFFFFFF
        return h ^ (h >> 16)
    n = len(rp) - 1
    s = fmix((seed & 0xFFFFFFFF) ^ (seed >> 32))
    nbrs = [[int(x) for x in c[rp[u]:rp[u + 1]] if x != u] for u in range(n)]
    order = sorted(range(n), key=lambda v: (fmix(v ^ s), v), reverse=True)
    col = [-1] * n
    for v in order:
        used = {col[x] for x in nbrs[v] if col[x] >= 0}
        k = 0
        while k in used:
            k += 1
        col[v] = k
    return col


@pytest.mark.parametrize("seed", [1, 5, 2**40 + 3])
def test_colouring_equals_greedy_in_priority_order(oracle_mod, seed):
    """Jones-Plassmann first-fit colours a vertex only after all of its
    higher-priority neighbours, and never after a lower-priority one, so it
    equals sequential greedy colouring in descending priority order."""
    for g in (synth.rmat(9, seed=3), synth.random_graph(200, 900, seed=seed % 97, loops=4)):
        rp, c, w = csr(g)
        want = _greedy_in_priority_order(rp, c, seed)
        k, col = oracle_mod.color(rp, c, w, seed)
        assert col.tolist() == want
        kj, colj = oracle_mod.color_jp(rp, c, w, seed)
        assert colj.tolist() == want and kj == k


@pytest.mark.parametrize("seed", [1, 3])
def test_colouring_one_pass_equals_rounds(oracle_mod, seed):
    """The schedule's one-pass colouring equals the Jones-Plassmann rounds
    on graphs with hubs (hub-hub edges skipped by both) and with loops."""
    for g in (synth.rmat(12, seed=seed), _hub_core_graph(nh=4, leaves=4100, seed=seed),
              synth.chung_lu(3000, seed=seed)):
        rp, c, w = csr(g)
        k, col = oracle_mod.color(rp, c, w, seed)
        kj, colj = oracle_mod.color_jp(rp, c, w, seed)
        assert k == kj and np.array_equal(col, colj)


def _hub_core_graph(nh=5, leaves=4200, seed=1):
    """nh mutually adjacent hubs (degree > 4096), each with `leaves` private
    leaves grouped in 5-cliques, plus random leaf-leaf edges across hubs."""
    rng = np.random.default_rng(seed)
    n = nh + nh * leaves
    edges = [(a, b) for a in range(nh) for b in range(a + 1, nh)]
    for h in range(nh):
        base = nh + h * leaves
        for i in range(leaves):
            edges.append((h, base + i))
        for q in range(0, leaves - 4, 5):
            grp = range(base + q, base + q + 5)
            edges += [(x, y) for x in grp for y in grp if x < y]
    for _ in range(3 * leaves):
        x, y = rng.integers(nh, n, size=2)
        if x != y:
            edges.append((int(min(x, y)), int(max(x, y))))
    return synth.from_edge_list(n, sorted(set(edges)))


def test_colouring_ignores_only_hub_hub_edges(oracle_mod):
    """Vertices with more than 4096 neighbours (hubs) do not constrain each
    other's colours; every other edge is properly coloured, and the result is
    sequential greedy colouring in priority order on the graph without its
    hub-hub edges."""
    g = _hub_core_graph()
    rp, c, w = csr(g)
    deg = np.diff(rp)
    hub = deg > 4096
    assert hub.sum() == 5
    for seed, colour in ((1, oracle_mod.color), (7, oracle_mod.color), (7, oracle_mod.color_jp)):
        k, col = colour(rp, c, w, seed)
        same_hub_pair = 0
        for u in range(g.n):
            nb = c[rp[u]:rp[u + 1]]
            for v in nb:
                if col[u] == col[v]:
                    assert hub[u] and hub[v], (u, v)
                    same_hub_pair += 1
        assert same_hub_pair > 0   # the hub clique shares colours
        keep = ~(hub[np.repeat(np.arange(g.n), deg)] & hub[c])
        c2 = c[keep]
        rp2 = np.zeros(g.n + 1, np.int64)
        rp2[1:] = np.cumsum(np.bincount(np.repeat(np.arange(g.n), deg)[keep], minlength=g.n))
        assert col.tolist() == _greedy_in_priority_order(rp2, c2, seed)


def test_hub_core_late_sweeps_never_lower_modularity(oracle_mod):
    """With adjacent hubs in one class, the re-check passes over a hub whose
    current or target community a hub moved earlier in the class left or
    entered, so late sweeps still never lower the exact modularity and the
    phase converges."""
    g = _hub_core_graph(nh=4, leaves=4100, seed=3)
    rp, c, w = csr(g)
    ed = exact.edges_of(rp, c, w)
    full, st = oracle_mod.move_phase(rp, c, w, 2)
    assert st["converged"] == 1
    prev = None
    for sweeps in range(4, st["sweeps"] + 1):
        z, _ = oracle_mod.move_phase(rp, c, w, 2, max_sweeps=sweeps)
        q = exact.modularity_fraction(g.n, ed, z)
        if prev is not None:
            assert q >= prev, sweeps
        prev = q
    assert np.array_equal(z, full)


def test_colouring_isolated_and_complete(oracle_mod):
    g = synth.from_edge_list(4, [], self_loops={1: 3})
    rp, c, w = csr(g)
    k, col = oracle_mod.color(rp, c, w, 1)
    assert k == 1 and np.all(col == 0)
    g = synth.cliques(1, 7)
    rp, c, w = csr(g)
    k, col = oracle_mod.color(rp, c, w, 1)
    assert k == 7 and sorted(col.tolist()) == list(range(7))


# ---------------------------------------------------------------------------
# Coarsening (Section III-B): invariants
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(4))
def test_coarsen_invariants(oracle_mod, seed):
    import torch
    g = synth.random_graph(60, 200, seed=200 + seed, loops=8)
    rp, c, w = csr(g)
    lab = np.asarray(synth.rand_u53(seed, 2, torch.arange(g.n)) % 17, np.int32)
    crp, cc, cw, pi = oracle_mod.coarsen(rp, c, w, lab)
    ed = exact.edges_of(rp, c, w)
    ced = exact.edges_of(crp, cc, cw)
    W = sum(ed.values())
    assert sum(ced.values()) == W                       # W' = W
    nc = len(crp) - 1
    assert nc == len(np.unique(lab))
    # pi is the dense rank of the label
    ranks = {l: i for i, l in enumerate(sorted(set(lab.tolist())))}
    assert all(pi[u] == ranks[lab[u]] for u in range(g.n))
    # symmetric, rows sorted strictly ascending
    for u in range(nc):
        row = cc[crp[u]:crp[u + 1]]
        assert np.all(np.diff(row) > 0)
        for e in range(crp[u], crp[u + 1]):
            v = cc[e]
            j = np.searchsorted(cc[crp[v]:crp[v + 1]], u)
            assert cc[crp[v] + j] == u and cw[crp[v] + j] == cw[e]
    # vol'(pi(C)) = vol(C) and mod(zeta, G) == mod(singletons, G') exactly
    def vols(n, edd):
        v = [0] * n
        for (a, b), wt in edd.items():
            v[a] += wt if a != b else 2 * wt
            if a != b:
                v[b] += wt
        return v
    vf, vc = vols(g.n, ed), vols(nc, ced)
    for C in range(nc):
        assert vc[C] == sum(vf[u] for u in range(g.n) if pi[u] == C)
    q1, N1, D1 = oracle_mod.modularity(rp, c, w, lab)
    q2, N2, D2 = oracle_mod.modularity(crp, cc, cw, np.arange(nc, dtype=np.int32))
    assert (N1, D1) == (N2, D2) and q1 == q2


# ---------------------------------------------------------------------------
# Move phase (Algorithm 2) and PLM / PLMR (Algorithms 3, 4)
# ---------------------------------------------------------------------------

def _no_positive_move(rp, c, w, lab):
    """Brute force: no vertex gains modularity by joining a neighbour's community."""
    n = len(rp) - 1
    ed = exact.edges_of(rp, c, w)
    base = exact.modularity_fraction(n, ed, lab)
    for u in range(n):
        for v in c[rp[u]:rp[u + 1]]:
            if v == u or lab[v] == lab[u]:
                continue
            t = lab.copy()
            t[u] = lab[v]
            if exact.modularity_fraction(n, ed, t) > base:
                return False
    return True


@pytest.mark.parametrize("seed", range(3))
def test_plmr_converged_has_no_positive_move(oracle_mod, seed):
    g = synth.random_graph(40, 110, seed=300 + seed, loops=3)
    rp, c, w = csr(g)
    r = oracle_mod.plm(rp, c, w, refine=True, seed=seed + 1)
    assert r.stats["converged"] == 1
    assert _no_positive_move(rp, c, w, r.labels)


def test_move_phase_converged_has_no_positive_move(oracle_mod):
    g = synth.rmat(8, seed=4)
    rp, c, w = csr(g)
    z, st = oracle_mod.move_phase(rp, c, w, 1)
    assert st["converged"] == 1
    assert _no_positive_move(rp, c, w, z)


@pytest.mark.parametrize("gname", ["rmat10", "rand_loops", "pp"])
def test_late_sweeps_never_lower_modularity(oracle_mod, gname):
    """From the re-check sweep (the 5th) on, every applied move has a
    positive gain against the volumes already updated, so modularity (exact
    fractions) never decreases from one sweep to the next, and the phase
    converges."""
    g = {"rmat10": lambda: synth.rmat(10, seed=8),
         "rand_loops": lambda: synth.random_graph(120, 500, seed=9, loops=10),
         "pp": lambda: synth.planted_partition(400, 8, 0.08, 0.01, seed=4)}[gname]()
    rp, c, w = csr(g)
    ed = exact.edges_of(rp, c, w)
    full, st = oracle_mod.move_phase(rp, c, w, 1)
    assert st["converged"] == 1
    prev = None
    for sweeps in range(4, st["sweeps"] + 1):
        z, _ = oracle_mod.move_phase(rp, c, w, 1, max_sweeps=sweeps)
        q = exact.modularity_fraction(g.n, ed, z)
        if prev is not None:
            assert q >= prev, sweeps
        prev = q
    assert np.array_equal(z, full)


def _sequential_louvain_complete(n, wmat, order):
    """Textbook sequential local moving on a complete graph (every colour class
    is one vertex), with every gain taken as an exact modularity difference,
    ties to the smallest community id, until no vertex moves."""
    edges = {(u, v): int(wmat[u][v]) for u in range(n) for v in range(u + 1, n)}
    lab = list(range(n))
    while True:
        moved = 0
        for u in order:
            base = exact.modularity_fraction(n, edges, lab)
            best, bestd = None, Fraction(0)
            for D in sorted(set(lab[v] for v in range(n) if v != u) - {lab[u]}):
                t = list(lab)
                t[u] = D
                d = exact.modularity_fraction(n, edges, t) - base
                if best is None or d > bestd:
                    best, bestd = D, d
            if best is not None and bestd > 0:
                lab[u] = best
                moved += 1
        if moved == 0:
            return lab


@pytest.mark.parametrize("seed,wmax", [(0, 20), (1, 20), (2, 20), (3, 1), (4, 2), (5, 2)])
def test_move_phase_on_complete_graph_is_sequential_louvain(oracle_mod, seed, wmax):
    """wmax 1 or 2 makes equal gains common, pinning the smallest-id tie rule."""
    import torch
    n = 9
    r = synth.rand_u53(seed, 77, torch.arange(n * n)).tolist()
    wm = [[0] * n for _ in range(n)]
    edges, ws = [], []
    for u in range(n):
        for v in range(u + 1, n):
            wm[u][v] = wm[v][u] = 1 + r[u * n + v] % wmax
            edges.append((u, v))
            ws.append(wm[u][v])
    g = synth.from_edge_list(n, edges, ws)
    rp, c, w = csr(g)
    k, col = oracle_mod.color(rp, c, w, 1)
    assert k == n                                   # one vertex per class
    order = list(np.argsort(col))
    z, st = oracle_mod.move_phase(rp, c, w, 1)
    assert st["converged"] == 1 and st["sweeps"] < 16   # damping never engaged
    assert list(z) == _sequential_louvain_complete(n, wm, order)


def _partition_ok(lab):
    k = lab.max() + 1 if len(lab) else 0
    return lab.min(initial=0) >= 0 and sorted(set(lab.tolist())) == list(range(k))


@pytest.mark.parametrize("refine", [False, True])
def test_plm_is_compact_partition_and_deterministic(oracle_mod, refine):
    g = synth.rmat(11, seed=3)
    rp, c, w = csr(g)
    r1 = oracle_mod.plm(rp, c, w, refine=refine)
    r2 = oracle_mod.plm(rp, c, w, refine=refine)
    r3 = oracle_mod.plm(rp, c, w, refine=refine, rev=True)   # class order reversed
    assert _partition_ok(r1.labels)
    assert np.array_equal(r1.labels, r2.labels) and np.array_equal(r1.labels, r3.labels)
    ed = exact.edges_of(rp, c, w)
    assert r1.modularity == float(exact.modularity_fraction(g.n, ed, r1.labels))


@pytest.mark.parametrize("seed", range(5))
def test_bruteforce_upper_bound(oracle_mod, seed):
    g = synth.random_graph(9, 16, seed=400 + seed, loops=2)
    rp, c, w = csr(g)
    ed = exact.edges_of(rp, c, w)
    best, _ = exact.max_modularity_bruteforce(g.n, ed)
    for res in (oracle_mod.plm(rp, c, w), oracle_mod.plm(rp, c, w, refine=True),
                oracle_mod.epp(rp, c, w, b=3)):
        assert Fraction(res.modularity) <= best + Fraction(1, 10**12)


@pytest.mark.parametrize("inst", ["two_k5", "cliques"])
def test_bruteforce_optimum_reached(oracle_mod, inst):
    if inst == "two_k5":
        edges = [(a, b) for a in range(5) for b in range(a + 1, 5)]
        edges += [(a + 5, b + 5) for a, b in edges] + [(4, 5)]
        g = synth.from_edge_list(10, edges)
    else:
        g = synth.cliques(3, 3)
    rp, c, w = csr(g)
    ed = exact.edges_of(rp, c, w)
    best, _ = exact.max_modularity_bruteforce(g.n, ed)
    for res in (oracle_mod.plm(rp, c, w), oracle_mod.plm(rp, c, w, refine=True),
                oracle_mod.epp(rp, c, w, b=2)):
        assert Fraction(res.modularity) == best or abs(res.modularity - float(best)) < 1e-15


def test_plm_degenerate(oracle_mod):
    g = synth.from_edge_list(6, [], self_loops={2: 5})
    rp, c, w = csr(g)
    r = oracle_mod.plm(rp, c, w)
    assert list(r.labels) == list(range(6))
    g = synth.from_edge_list(1, [])
    r = oracle_mod.plm(*csr(g))
    assert list(r.labels) == [0] and r.modularity == 0.0


# ---------------------------------------------------------------------------
# PLP (Algorithm 1)
# ---------------------------------------------------------------------------

def test_plp_disjoint_cliques_one_label_each(oracle_mod):
    g = synth.cliques(6, 5)
    rp, c, w = csr(g)
    r = oracle_mod.plp(rp, c, w, theta=0)
    lab = r.labels
    for i in range(6):
        assert len(set(lab[i * 5:(i + 1) * 5].tolist())) == 1
    assert len(set(lab.tolist())) == 6


@pytest.mark.parametrize("seed", range(3))
def test_plp_active_set_is_result_neutral(oracle_mod, seed):
    g = synth.rmat(11, seed=10 + seed)
    rp, c, w = csr(g)
    a = oracle_mod.plp(rp, c, w, seed=seed, use_active=True)
    b = oracle_mod.plp(rp, c, w, seed=seed, use_active=False)
    assert np.array_equal(a.labels, b.labels)
    assert a.stats["iters"] == b.stats["iters"] and a.stats["moves"] == b.stats["moves"]
    assert a.stats["decisions"] <= b.stats["decisions"]


@pytest.mark.parametrize("seed", range(3))
def test_plp_final_state_is_dominant(oracle_mod, seed):
    g = synth.random_graph(60, 180, seed=500 + seed, loops=5)
    rp, c, w = csr(g)
    r = oracle_mod.plp(rp, c, w, seed=seed, theta=0)
    assert r.stats["converged"] == 1
    lab = r.labels
    for v in range(g.n):
        tot = {}
        for e in range(rp[v], rp[v + 1]):
            if c[e] != v:
                tot[lab[c[e]]] = tot.get(lab[c[e]], 0) + (1 if w is None else int(w[e]))
        if tot:
            assert max(tot.values()) <= tot.get(lab[v], 0)
    # class order inside a colour class does not matter
    r2 = oracle_mod.plp(rp, c, w, seed=seed, theta=0, rev=True)
    assert np.array_equal(lab, r2.labels) and _partition_ok(lab)


# ---------------------------------------------------------------------------
# EPP (Algorithm 5) and the core communities (Eq. 2)
# ---------------------------------------------------------------------------

def test_epp_core_satisfies_eq2(oracle_mod):
    g = synth.planted_partition(300, 6, 0.1, 0.01, seed=3)
    rp, c, w = csr(g)
    r, base, core = oracle_mod.epp(rp, c, w, b=4, want_parts=True)
    assert _partition_ok(core) and _partition_ok(r.labels)
    for u, v in itertools.combinations(range(0, 300, 3), 2):
        same_all = all(base[i][u] == base[i][v] for i in range(4))
        assert same_all == (core[u] == core[v])
    # the final labelling is a union of core communities
    for k in np.unique(core):
        assert len(set(r.labels[core == k].tolist())) == 1


def test_combine_identical_bases_is_the_base(oracle_mod):
    g = synth.rmat(9, seed=2)
    rp, c, w = csr(g)
    z = oracle_mod.plp(rp, c, w).labels
    k, core = oracle_mod.combine([z, z, z])
    assert np.array_equal(core, z) and k == z.max() + 1


def test_combine_small_exhaustive(oracle_mod):
    import torch
    L = [np.asarray(synth.rand_u53(s, 3, torch.arange(40)) % 4, np.int32) for s in range(3)]
    k, core = oracle_mod.combine(L)
    keys = sorted(set(zip(*[l.tolist() for l in L])))
    expect = [keys.index(t) for t in zip(*[l.tolist() for l in L])]
    assert core.tolist() == expect and k == len(keys)
