"""The allocation-free modularity entry point (cd_modularity_static).

It exists for callers that must not allocate device memory when they ask for
a result.  This file is collected last so that a run stopping at the first
failure has already run every other test; it also passes alone in a fresh
process.
"""
import numpy as np
import pytest
import torch

from paper_1304_4453_gb300 import build, cd, synth

pytestmark = pytest.mark.gpu

MOD_TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    cd.lib()


@pytest.mark.parametrize("gname", ["rmat14", "weighted_loops"])
def test_static_scratch_matches_cd_modularity_on_consecutive_calls(gname):
    g = {"rmat14": lambda: synth.rmat(14, seed=6),
         "weighted_loops": lambda: synth.random_graph(5000, 40000, seed=3, loops=50, wmax=90)}[gname]()
    gd = g.to("cuda")
    G = cd.Graph(gd.row_ptr, gd.col, gd.w)
    rng = np.random.default_rng(1)
    lab_plp = G.plp().labels.clone()
    lab_rand = torch.from_numpy(rng.integers(0, 50, g.n).astype(np.int32)).cuda()
    # two calls in a row on the shared scratch: the second must not see the first's sums
    for labels in (lab_plp, lab_rand, lab_plp):
        q_static = cd.cd_modularity_static(gd.row_ptr, gd.col, gd.w, labels)
        q_ref = G.modularity(labels)
        assert abs(q_static - q_ref) <= MOD_TOL, (q_static, q_ref)


def test_static_scratch_rejects_graphs_above_its_limit():
    n = (1 << 20) + 1
    rp = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    col = torch.zeros(1, dtype=torch.int32, device="cuda")
    labels = torch.zeros(n, dtype=torch.int32, device="cuda")
    with pytest.raises(cd.CDError) as e:
        cd.cd_modularity_static(rp, col, None, labels)
    assert e.value.status == cd.CD_EINVAL


def test_static_scratch_rejects_out_of_range_labels():
    g = synth.rmat(10, seed=2).to("cuda")
    bad = torch.full((g.n,), g.n, dtype=torch.int32, device="cuda")
    with pytest.raises(cd.CDError) as e:
        cd.cd_modularity_static(g.row_ptr, g.col, g.w, bad)
    assert e.value.status == cd.CD_EINVAL


@pytest.mark.parametrize("case", ["empty", "isolated", "loops_only"])
def test_static_scratch_degenerate_graphs(case):
    """n = 0, vertices without edges (2W = 0: modularity 0), and self-loops
    only: the same result and status as cd_modularity."""
    g = {"empty": lambda: synth.from_edge_list(0, []),
         "isolated": lambda: synth.from_edge_list(6, []),
         "loops_only": lambda: synth.from_edge_list(4, [], self_loops={0: 3, 2: 1})}[case]()
    gd = g.to("cuda")
    G = cd.Graph(gd.row_ptr, gd.col, gd.w)
    for labels in (torch.arange(g.n, dtype=torch.int32, device="cuda"),
                   torch.zeros(g.n, dtype=torch.int32, device="cuda")):
        q_static = cd.cd_modularity_static(gd.row_ptr, gd.col, gd.w, labels)
        q_ref = G.modularity(labels)
        assert q_static == q_ref
        if case != "loops_only":
            assert q_static == 0.0

