"""Pins of the full-size property checkers (tests/properties.py) on graphs the
oracle handles: each checker accepts the oracle's results and rejects planted
mistakes, so that at full size, where the oracle is too slow, a GPU result
that passes them is pinned to the same definitions."""
import numpy as np
import pytest

from paper_1304_4453_gb300 import synth

from . import properties as P
from .test_oracle_pins import _hub_core_graph


def _graphs():
    return {
        "rmat12": synth.rmat(12, seed=3),
        "loops_w": synth.random_graph(400, 2500, seed=5, loops=25, wmax=40),
        "pp": synth.planted_partition(1500, 6, 0.04, 0.003, seed=4),
        "hub_core": _hub_core_graph(nh=5, leaves=4200, seed=2),
    }


GRAPHS = _graphs()


@pytest.mark.parametrize("name", sorted(GRAPHS))
@pytest.mark.parametrize("seed", [1, 9, 2**40 + 3])
def test_first_fit_checker_accepts_the_oracle_colouring(oracle_mod, name, seed):
    rp, c, w = GRAPHS[name].numpy()
    k, col = oracle_mod.color(rp, c, w, seed)
    P.check_first_fit_colouring(rp, c, col, seed)
    assert k == int(col.max()) + 1


@pytest.mark.parametrize("name", ["rmat12", "hub_core"])
def test_first_fit_checker_rejects_mistakes(oracle_mod, name):
    rp, c, w = GRAPHS[name].numpy()
    seed = 1
    k, col = oracle_mod.color(rp, c, w, seed)
    rng = np.random.default_rng(0)
    deg = np.diff(rp)
    # a colour one too high (not the smallest free one)
    for v in rng.choice(np.flatnonzero(deg > 0), 5, replace=False):
        bad = col.copy()
        bad[v] += 1
        with pytest.raises(AssertionError):
            P.check_first_fit_colouring(rp, c, bad, seed)
    # a vertex given the colour of a neighbour
    v = int(np.flatnonzero(deg > 1)[0])
    bad = col.copy()
    bad[v] = col[c[rp[v]]] if c[rp[v]] != v else col[c[rp[v] + 1]]
    if bad[v] != col[v]:
        with pytest.raises(AssertionError):
            P.check_first_fit_colouring(rp, c, bad, seed)
    # another seed's priorities
    with pytest.raises(AssertionError):
        P.check_first_fit_colouring(rp, c, col, seed + 1)


def test_first_fit_checker_rejects_a_strict_hub_colouring(oracle_mod):
    """On the hub core, hub-hub edges are ignored: the colouring that also
    separates adjacent hubs is a different one, and the checker tells them
    apart."""
    g = GRAPHS["hub_core"]
    rp, c, w = g.numpy()
    k, col = oracle_mod.color(rp, c, w, 1)
    hubs = np.flatnonzero(np.diff(rp) > P.HUB_RELAX)
    assert len(hubs) == 5 and len(set(col[hubs].tolist())) < 5   # some hubs share a colour
    bad = col.copy()
    bad[hubs] = np.arange(len(hubs)) + col.max() + 1               # distinct colours for the hubs
    with pytest.raises(AssertionError):
        P.check_first_fit_colouring(rp, c, bad, 1)


@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_exact_modularity_matches_the_oracle(oracle_mod, name):
    rp, c, w = GRAPHS[name].numpy()
    n = len(rp) - 1
    rng = np.random.default_rng(7)
    for k in (1, 5, n):
        lab = rng.integers(0, k, n).astype(np.int32)
        assert abs(P.modularity_exact(rp, c, w, lab) - oracle_mod.modularity(rp, c, w, lab)[0]) <= 1e-12
    assert P.modularity_exact(rp, c, w, np.zeros(n, np.int32)) == 0.0


@pytest.mark.parametrize("name", ["rmat12", "loops_w", "pp"])
def test_converged_plmr_has_no_positive_gain(oracle_mod, name):
    rp, c, w = GRAPHS[name].numpy()
    n = len(rp) - 1
    r = oracle_mod.plm(rp, c, w, refine=True, seed=1)
    assert r.stats["converged"] == 1
    assert P.check_dense_labels(r.labels) == r.stats["ncomm"]
    assert P.positive_gain_moves(rp, c, w, r.labels, np.arange(n)) == []
    assert abs(P.modularity_exact(rp, c, w, r.labels) - r.modularity) <= 1e-12


@pytest.mark.parametrize("name", ["rmat12", "loops_w", "pp"])
def test_positive_gain_checker_agrees_with_the_oracle(oracle_mod, name):
    """Vertices with a positive-gain move, on labellings far from converged:
    the checker finds exactly as many as the oracle's count."""
    rp, c, w = GRAPHS[name].numpy()
    n = len(rp) - 1
    rng = np.random.default_rng(3)
    for lab in (np.arange(n, dtype=np.int32), rng.integers(0, 7, n).astype(np.int32)):
        moves = P.positive_gain_moves(rp, c, w, lab, np.arange(n))
        assert len({u for u, _, _ in moves}) == oracle_mod.positive_moves(rp, c, w, lab) > 0
        for u, D, g in moves[:20]:
            assert g == oracle_mod.gain(rp, c, w, lab, u, D) > 0


def test_dense_label_checker():
    assert P.check_dense_labels(np.array([0, 1, 1, 2])) == 3
    with pytest.raises(AssertionError):
        P.check_dense_labels(np.array([0, 2, 2]))
    with pytest.raises(AssertionError):
        P.check_dense_labels(np.array([1, 1]))
