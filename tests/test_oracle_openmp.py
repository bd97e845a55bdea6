"""The oracle's OpenMP build (decisions of a colour class spread over threads)
gives exactly the sequential build's results: labels, modularity and every
schedule counter.  Vertices of a class decide independently on labels and
volumes fixed before the class (Section III-B's parallel loop), so the
thread count must not matter.  The golden records of the full-size workloads
are written with the OpenMP build, so this equality is what lets them stand
for the sequential oracle."""
import numpy as np
import pytest

from paper_1304_4453_gb300 import synth
from tests.test_oracle_pins import _hub_core_graph


def _graphs():
    return {
        "rmat14": synth.rmat(14, seed=5),
        "chunglu_w": synth.chung_lu(20000, seed=3),
        "hub_core": _hub_core_graph(nh=4, leaves=4100, seed=3),
        "pp": synth.planted_partition(4000, 10, 0.02, 0.001, seed=2),
    }


GRAPHS = _graphs()


@pytest.mark.parametrize("name", sorted(GRAPHS))
@pytest.mark.parametrize("threads", [4])
def test_openmp_plm_plmr_equal_sequential(oracle_mod, name, threads):
    g = GRAPHS[name]
    rp, c, w = g.numpy()
    assert oracle_mod.threads_used(threads) == threads
    for refine in (False, True):
        a = oracle_mod.plm(rp, c, w, refine=refine, seed=2)
        b = oracle_mod.plm(rp, c, w, refine=refine, seed=2, threads=threads)
        assert np.array_equal(a.labels, b.labels)
        assert a.modularity == b.modularity and a.stats == b.stats
    a = oracle_mod.plm(rp, c, w, refine=True, seed=2, resolution=(3, 2))
    b = oracle_mod.plm(rp, c, w, refine=True, seed=2, resolution=(3, 2), threads=threads)
    assert np.array_equal(a.labels, b.labels) and a.stats == b.stats


@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_openmp_plp_epp_equal_sequential(oracle_mod, name):
    g = GRAPHS[name]
    rp, c, w = g.numpy()
    a = oracle_mod.plp(rp, c, w, seed=4)
    b = oracle_mod.plp(rp, c, w, seed=4, threads=5)
    assert np.array_equal(a.labels, b.labels) and a.stats == b.stats
    a = oracle_mod.epp(rp, c, w, b=3, final_refine=True, seed=2)
    b = oracle_mod.epp(rp, c, w, b=3, final_refine=True, seed=2, threads=5)
    assert np.array_equal(a.labels, b.labels) and a.stats == b.stats


def test_openmp_build_really_runs_threads(oracle_mod):
    """The parallel build reports the thread count it was given; the
    sequential build always one."""
    assert oracle_mod.threads_used(1) == 1
    assert oracle_mod.threads_used(4) == 4
