"""The low-memory mode (cd_opts.scratch_budget; the GPU analogue of the
paper's memory-lean PLM*, Section III-B): coarsening processes ranges of
coarse rows so that its scratch stays within the budget.  Results must equal
the default mode's bit for bit (and so the oracle's), while the library
pool's high-water mark of use drops."""
import numpy as np
import pytest
import torch

from paper_1304_4453_gb300 import cd, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1304_4453_gb300 import build
    build.build()
    cd.lib()


@pytest.fixture(scope="module")
def O():
    from oracle import oracle
    oracle.build()
    return oracle


@pytest.mark.parametrize("budget", [1, 4096, 1 << 20])
def test_low_memory_results_equal_default(O, budget):
    """Budgets from one entry per pass (every coarse row its own pass) up to
    1 MiB; PLM, PLMR, EPP and the generic EPP give the default results."""
    for g in (synth.rmat(13, seed=2), synth.random_graph(400, 3000, seed=5, loops=30, wmax=40),
              synth.chung_lu(20000, seed=3)):
        G = cd.Graph.from_synth(g, device="cuda")
        for fn in (lambda **k: G.plm(seed=3, **k), lambda **k: G.plm(refine=True, seed=3, **k),
                   lambda **k: G.epp(b=3, seed=3, **k),
                   lambda **k: G.epp_general(b=2, base=cd.CD_BASE_PLM, rounds=2, seed=3, **k)):
            a = fn()
            b = fn(scratch_budget=budget)
            assert torch.equal(a.labels, b.labels) and a.modularity == b.modularity
            assert a.stats["sweeps"] == b.stats["sweeps"] and a.stats["ncomm"] == b.stats["ncomm"]
        o = O.plm(*g.numpy(), refine=True, seed=3)
        assert np.array_equal(G.plm(refine=True, seed=3, scratch_budget=budget).labels.cpu().numpy(), o.labels)


def test_low_memory_lowers_the_pool_high_water_mark():
    """At R-MAT scale 20 a run's device memory above the input graph is the
    coarsening scratch of level 0 (32 bytes per inter-community entry while
    sorting), the schedules the levels keep, and the coarse level-1 graph with
    its working buffers.  A 64 MB budget removes the first two (measured on a
    GB300: 1.47 GB -> 0.83 GB above the graph); the test asks for a third of
    the peak to go."""
    g = synth.rmat(20, seed=1, device="cuda")
    G = cd.Graph(g.row_ptr, g.col, g.w)
    del g
    torch.cuda.synchronize()
    G.plm(seed=1)
    used0, _, _ = cd.cd_memory_stats(reset_high=True)
    a = G.plm(seed=1)
    _, high_default, _ = cd.cd_memory_stats(reset_high=True)
    b = G.plm(seed=1, scratch_budget=64 << 20)
    _, high_low, _ = cd.cd_memory_stats(reset_high=True)
    assert torch.equal(a.labels, b.labels)
    assert high_low - used0 < (2 / 3) * (high_default - used0), (used0, high_default, high_low)


def test_negative_budget_rejected():
    G = cd.Graph.from_synth(synth.rmat(8, seed=1), device="cuda")
    with pytest.raises(cd.CDError) as e:
        G.plm(scratch_budget=-1)
    assert e.value.status == cd.CD_EINVAL
