"""GPU parity of EPP(b, Base, Final) with iterated ensembles
(cd_epp_general; Section III-D): PLP, PLM or PLMR bases, PLM or PLMR final,
one or several ensemble rounds.  Labels, modularity, the number of
communities and the number of core graphs taken equal the oracle's."""
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


GRAPHS = {
    "pp_small": synth.planted_partition(2000, 8, 0.03, 0.002, seed=2),
    "rmat12": synth.rmat(12, seed=3),
    "chunglu_w": synth.chung_lu(20000, seed=3),
    "rand_w_loops": synth.random_graph(300, 1500, seed=7, loops=20, wmax=50),
}


@pytest.mark.parametrize("name", sorted(GRAPHS))
@pytest.mark.parametrize("base", [cd.CD_BASE_PLP, cd.CD_BASE_PLM, cd.CD_BASE_PLMR])
@pytest.mark.parametrize("rounds", [1, 3])
def test_epp_general_bit_exact(O, name, base, rounds):
    g = GRAPHS[name]
    G = cd.Graph.from_synth(g, device="cuda")
    for b, final_refine in ((3, True), (1, False)):
        r = G.epp_general(b=b, base=base, final_refine=final_refine, rounds=rounds, seed=4)
        o = O.epp_general(*g.numpy(), b=b, base=base, final_refine=final_refine, rounds=rounds, seed=4)
        assert np.array_equal(r.labels.cpu().numpy(), o.labels), (b, final_refine)
        assert r.modularity == o.modularity
        assert r.stats["ncomm"] == o.stats["ncomm"] and r.stats["levels"] == o.stats["levels"]


def test_epp_general_plp_single_round_is_epp():
    g = GRAPHS["chunglu_w"]
    G = cd.Graph.from_synth(g, device="cuda")
    a = G.epp(b=4, final_refine=True, seed=2)
    e = G.epp_general(b=4, base=cd.CD_BASE_PLP, final_refine=True, rounds=1, seed=2)
    assert torch.equal(a.labels, e.labels) and a.modularity == e.modularity


def test_epp_general_degenerate_and_invalid(O):
    for g in (synth.from_edge_list(0, []), synth.from_edge_list(5, []), synth.cliques(4, 5)):
        G = cd.Graph.from_synth(g, device="cuda")
        r = G.epp_general(b=2, base=cd.CD_BASE_PLM, rounds=3)
        o = O.epp_general(*g.numpy(), b=2, base=O.BASE_PLM, rounds=3)
        assert np.array_equal(r.labels.cpu().numpy(), o.labels) and r.modularity == o.modularity
    G = cd.Graph.from_synth(GRAPHS["rmat12"], device="cuda")
    for kw in ({"b": 0}, {"base": 3}, {"rounds": 0}, {"rounds": 65}):
        with pytest.raises(cd.CDError) as e:
            G.epp_general(**kw)
        assert e.value.status == cd.CD_EINVAL
