"""Pins of the oracle's generic EPP(b, Base, Final) with iterated ensembles
(Section III-D; the hierarchy of core graphs of the scheme EPP adapts,
Section II).  The rounds are rebuilt here from the oracle's separate
primitives (base runs with their stated seeds, the Eq. 2 combination,
coarsening, the final PLM, prolongation), so a wrong seed, acceptance rule or
prolongation in the combined routine fails."""
import numpy as np
import pytest

from paper_1304_4453_gb300 import synth
from tests import exact


def _compact(z):
    _, inv = np.unique(z, return_inverse=True)
    return inv.astype(np.int32)


def _bases(O, rp, c, w, b, base, seed0):
    out = []
    for i in range(b):
        sd = seed0 + i
        if base == O.BASE_PLP:
            out.append(O.plp(rp, c, w, seed=sd).labels)
        else:
            out.append(O.plm(rp, c, w, refine=base == O.BASE_PLMR, seed=sd).labels)
    return out


def _by_hand(O, g, b, base, final_refine, rounds, seed):
    """EPP(b, Base, Final) with iterated rounds from the primitives."""
    rp, c, w = g.numpy()
    graphs = [(rp, c, w)]
    pis = []
    prev = 0.0
    for r in range(rounds):
        rp_r, c_r, w_r = graphs[-1]
        n_r = len(rp_r) - 1
        labs = _bases(O, rp_r, c_r, w_r, b, base, seed + r * b)
        k, core = O.combine(labs) if n_r else (0, np.zeros(0, np.int32))
        q = O.modularity(rp_r, c_r, w_r, core)[0]
        if r > 0 and (k == n_r or q <= prev):
            break
        prev = q
        crp, cc, cw, pi = O.coarsen(rp_r, c_r, w_r, core)
        graphs.append((crp, cc, cw))
        pis.append(pi)
    rp_f, c_f, w_f = graphs[-1]
    z = O.plm(rp_f, c_f, w_f, refine=final_refine, seed=seed).labels
    for pi in reversed(pis):
        z = z[pi]
    return _compact(z), len(pis)


CASES = [("rmat11", lambda: synth.rmat(11, seed=3)),
         ("weighted", lambda: synth.random_graph(300, 1500, seed=7, loops=20, wmax=50)),
         ("pp", lambda: synth.planted_partition(1500, 6, 0.03, 0.002, seed=4))]


@pytest.mark.parametrize("name,make", CASES)
@pytest.mark.parametrize("base", [0, 1, 2])
@pytest.mark.parametrize("rounds", [1, 2, 3])
def test_generic_epp_equals_its_rounds_by_hand(oracle_mod, name, make, base, rounds):
    g = make()
    rp, c, w = g.numpy()
    for b, final_refine in ((3, True), (2, False)):
        r = oracle_mod.epp_general(rp, c, w, b=b, base=base, final_refine=final_refine, rounds=rounds, seed=5)
        want, taken = _by_hand(oracle_mod, g, b, base, final_refine, rounds, 5)
        assert np.array_equal(r.labels, want)
        assert r.stats["levels"] == taken
        assert r.modularity == oracle_mod.modularity(rp, c, w, want)[0]


def test_one_round_of_plp_bases_is_epp(oracle_mod):
    for _, make in CASES:
        g = make()
        a = oracle_mod.epp(*g.numpy(), b=4, final_refine=True, seed=2)
        e = oracle_mod.epp_general(*g.numpy(), b=4, base=oracle_mod.BASE_PLP, final_refine=True, rounds=1, seed=2)
        assert np.array_equal(a.labels, e.labels) and a.modularity == e.modularity


@pytest.mark.parametrize("base", [1, 2])
def test_disjoint_cliques_stop_after_one_round(oracle_mod, base):
    """PLM bases find every clique; the core graph is then isolated
    vertices with loops, a second ensemble cannot merge anything, and the
    result is the clique partition with modularity 1 - 1/k."""
    k, s = 6, 7
    g = synth.cliques(k, s)
    rp, c, w = g.numpy()
    r = oracle_mod.epp_general(rp, c, w, b=3, base=base, rounds=4, seed=1)
    assert r.stats["levels"] == 1
    assert sorted(np.bincount(r.labels).tolist()) == [s] * k
    ed = exact.edges_of(rp, c, w)
    from fractions import Fraction
    assert exact.modularity_fraction(g.n, ed, r.labels) == 1 - Fraction(1, k)


def test_taken_rounds_raise_modularity_and_extra_rounds_change_nothing(oracle_mod):
    """Every taken round's core has strictly higher modularity than the one
    before (the stop rule), so allowing more rounds than were taken changes
    nothing."""
    g = synth.rmat(12, seed=3)
    rp, c, w = g.numpy()
    r = oracle_mod.epp_general(rp, c, w, b=3, base=oracle_mod.BASE_PLMR, rounds=8, seed=1)
    L = r.stats["levels"]
    assert 1 <= L < 8
    same = oracle_mod.epp_general(rp, c, w, b=3, base=oracle_mod.BASE_PLMR, rounds=L, seed=1)
    assert np.array_equal(r.labels, same.labels)


def test_generic_epp_below_bruteforce_optimum(oracle_mod):
    for seed in range(3):
        g = synth.random_graph(9, 14, seed=60 + seed, loops=2)
        rp, c, w = g.numpy()
        best, _ = exact.max_modularity_bruteforce(g.n, exact.edges_of(rp, c, w))
        for base in (0, 1, 2):
            r = oracle_mod.epp_general(rp, c, w, b=2, base=base, rounds=2, seed=seed)
            ed = exact.edges_of(rp, c, w)
            assert exact.modularity_fraction(g.n, ed, r.labels) <= best


def test_invalid_arguments(oracle_mod):
    rp, c, w = synth.cliques(2, 3).numpy()
    for kw in ({"b": 0}, {"base": 3}, {"rounds": 0}, {"rounds": 65}):
        with pytest.raises(ValueError):
            oracle_mod.epp_general(rp, c, w, **kw)
