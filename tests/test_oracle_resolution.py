"""Pins of the resolution parameter gamma of Section III-B in the oracle:
gamma scales the volume term of the move gain; 0 yields one community per
connected component, 1 is modularity, 2W yields singletons.  gamma is a
rational p/q so that the gain stays an exact integer."""
from fractions import Fraction

import numpy as np
import pytest
import torch
from scipy.sparse import csr_matrix
from scipy.sparse.csgraph import connected_components

from paper_1304_4453_gb300 import synth
from tests import exact


def _canon(lab):
    """Labels renamed by first occurrence, to compare partitions."""
    seen = {}
    return [seen.setdefault(int(x), len(seen)) for x in lab]


def _components(rp, c, n):
    a = csr_matrix((np.ones(len(c)), np.asarray(c), np.asarray(rp)), shape=(n, n))
    return connected_components(a, directed=False)[1]


def _several_components():
    """Disjoint cliques, a weighted random graph with loops, a path and
    isolated vertices, in one graph."""
    parts = [synth.cliques(3, 5), synth.random_graph(30, 60, seed=4, loops=3),
             synth.from_edge_list(6, [(i, i + 1) for i in range(5)]), synth.from_edge_list(3, [])]
    edges, ws, loops, base = [], [], {}, 0
    for g in parts:
        rp, c, w = g.numpy()
        for u in range(g.n):
            for e in range(rp[u], rp[u + 1]):
                v = int(c[e])
                wt = 1 if w is None else int(w[e])
                if v == u:
                    loops[base + u] = wt
                elif u < v:
                    edges.append((base + u, base + v))
                    ws.append(wt)
        base += g.n
    return synth.from_edge_list(base, edges, ws, loops)


@pytest.mark.parametrize("seed", range(3))
@pytest.mark.parametrize("res", [(0, 1), (1, 2), (3, 1), (5, 7)])
def test_gain_equals_generalised_modularity_difference(oracle_mod, seed, res):
    g = synth.random_graph(14, 40, seed=200 + seed, loops=3)
    rp, c, w = g.numpy()
    ed = exact.edges_of(rp, c, w)
    W = sum(ed.values())
    p, q = res
    gamma = Fraction(p, q)
    lab = np.asarray(synth.rand_u53(seed, 2, torch.arange(g.n)) % 5, np.int32)
    before = exact.modularity_fraction(g.n, ed, lab, gamma)
    for u in range(g.n):
        for D in range(5):
            if D == lab[u]:
                continue
            after_lab = lab.copy()
            after_lab[u] = D
            after = exact.modularity_fraction(g.n, ed, after_lab, gamma)
            gnum = oracle_mod.gain(rp, c, w, lab, u, D, resolution=res)
            assert Fraction(gnum, 2 * W * W * q) == after - before, (u, D)


@pytest.mark.parametrize("refine", [False, True])
def test_gamma_one_is_modularity(oracle_mod, refine):
    for g in (synth.rmat(10, seed=2), synth.random_graph(300, 1500, seed=6, loops=10)):
        rp, c, w = g.numpy()
        base = oracle_mod.plm(rp, c, w, refine=refine, seed=1)
        for res in ((1, 1), (2, 2), (7, 7)):
            r = oracle_mod.plm(rp, c, w, refine=refine, seed=1, resolution=res)
            assert np.array_equal(r.labels, base.labels) and r.modularity == base.modularity
            assert r.stats == base.stats


@pytest.mark.parametrize("refine", [False, True])
def test_gamma_zero_gives_connected_components(oracle_mod, refine):
    for g in (_several_components(), synth.rmat(9, seed=5)):
        rp, c, w = g.numpy()
        r = oracle_mod.plm(rp, c, w, refine=refine, seed=3, resolution=(0, 1))
        assert _canon(r.labels) == _canon(_components(rp, c, g.n))


def test_gamma_2w_gives_singletons(oracle_mod):
    for g in (_several_components(), synth.rmat(9, seed=5), synth.cliques(4, 6, ring=True)):
        rp, c, w = g.numpy()
        W = sum(exact.edges_of(rp, c, w).values())
        for res in ((2 * W, 1), (4 * W + 1, 2)):
            r = oracle_mod.plm(rp, c, w, refine=True, seed=1, resolution=res)
            assert list(r.labels) == list(range(g.n))
            assert r.stats["moves"] == 0


def test_invalid_resolution(oracle_mod):
    rp, c, w = synth.cliques(2, 3).numpy()
    for res in ((-1, 1), (1, 0)):
        with pytest.raises(ValueError):
            oracle_mod.plm(rp, c, w, resolution=res)
        with pytest.raises(ValueError):
            oracle_mod.gain(rp, c, w, np.zeros(6, np.int32), 0, 1, resolution=res)
        with pytest.raises(ValueError):
            oracle_mod.positive_moves(rp, c, w, np.zeros(6, np.int32), resolution=res)


def _heavy():
    """A weighted graph with 2W near 2^41, so that (2W)^2 is near 2^82."""
    base = synth.random_graph(40, 300, seed=9, loops=4, wmax=50)
    w = (base.w.to(torch.int64) * 20_000_000 + 3).clamp(max=2**31 - 1).to(torch.int32)
    return synth.Graph(base.n, base.row_ptr, base.col, w, "heavy")


def test_resolution_outside_128_bits_rejected(oracle_mod):
    """Both gain products are bounded by max(p, q) (2W)^2; a resolution whose
    bound reaches 2^126 could overflow the 128-bit gain and is rejected, one
    just inside is accepted (also after reduction by the gcd)."""
    g = _heavy()
    rp, c, w = g.numpy()
    W = sum(exact.edges_of(rp, c, w).values())
    w2 = (2 * W) ** 2
    inside = (2**126 - 1) // w2
    assert 2**40 < inside < 2**62
    for res in ((inside + 1, 1), (1, inside + 1), (2 * (inside + 1), 2)):
        with pytest.raises(ValueError):
            oracle_mod.plm(rp, c, w, resolution=res)
        with pytest.raises(ValueError):
            oracle_mod.gain(rp, c, w, np.zeros(g.n, np.int32), 0, 1, resolution=res)
    oracle_mod.plm(rp, c, w, resolution=(inside, 1))
    oracle_mod.plm(rp, c, w, resolution=(3 * inside, 3))     # reduces to (inside, 1)


@pytest.mark.parametrize("refine", [False, True])
def test_resolution_reduced_by_gcd_changes_nothing(oracle_mod, refine):
    g = synth.random_graph(300, 1500, seed=6, loops=10)
    rp, c, w = g.numpy()
    for p, q in ((3, 2), (5, 7), (1, 3)):
        a = oracle_mod.plm(rp, c, w, refine=refine, seed=2, resolution=(p, q))
        b = oracle_mod.plm(rp, c, w, refine=refine, seed=2, resolution=(6 * p, 6 * q))
        assert np.array_equal(a.labels, b.labels) and a.stats == b.stats


@pytest.mark.parametrize("res", [(1, 2), (3, 1), (5, 7)])
def test_converged_plmr_has_no_positive_gamma_move(oracle_mod, res):
    """After a converged PLMR run (the last move phase works on the input
    graph), no vertex has a move with positive gamma-gain (Algorithm 2's
    stopping rule), for gamma != 1."""
    elsewhere = 0
    for g in (synth.rmat(10, seed=2), synth.random_graph(300, 1500, seed=6, loops=10),
              synth.chung_lu(2000, seed=4)):
        rp, c, w = g.numpy()
        r = oracle_mod.plm(rp, c, w, refine=True, seed=1, resolution=res)
        assert r.stats["converged"] == 1
        assert oracle_mod.positive_moves(rp, c, w, r.labels, resolution=res) == 0
        # the check sees gamma: judged at the inverse gamma, some vertex
        # wants to move (on graphs that end with several communities)
        elsewhere += oracle_mod.positive_moves(rp, c, w, r.labels, resolution=(res[1], res[0]))
    assert elsewhere > 0
