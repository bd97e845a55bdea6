"""GPU parity of the resolution gamma = p/q (Section III-B): PLM, PLMR and
EPP's final phase maximise sum_C omega(C)/W - gamma vol(C)^2 / (4W^2) with the
exact integer gain 2W q (omega(u,D) - omega(u,C\\u)) - p vol(u) (vol(D) -
vol(C\\u)).  Labels, modularity (always the standard one) and the schedule
counters must equal the oracle's for every gamma, on the 64-bit and the
128-bit gain paths, including a graph that gamma alone moves to 128 bits."""
import numpy as np
import pytest
import torch

from paper_1304_4453_gb300 import cd, synth

pytestmark = pytest.mark.gpu

MOD_TOL = 1e-12
GAMMAS = [(0, 1), (1, 2), (1, 1), (3, 1), (5, 7)]
KEYS = ["levels", "sweeps", "moves", "entries", "candidates", "decisions", "converged", "ncomm"]


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
    "rmat14_hubs": synth.rmat(14, seed=5),
    "rand_w_loops": synth.random_graph(300, 1500, seed=7, loops=20, wmax=50),
    "chunglu_w": synth.chung_lu(20000, seed=3),
}


def _check(r, o):
    assert np.array_equal(r.labels.cpu().numpy(), o.labels)
    assert abs(r.modularity - o.modularity) <= MOD_TOL and r.modularity == o.modularity
    for k in KEYS:
        assert r.stats[k] == o.stats[k], (k, r.stats[k], o.stats[k])


@pytest.mark.parametrize("name", sorted(GRAPHS))
@pytest.mark.parametrize("res", GAMMAS)
def test_plm_plmr_resolution_bit_exact(O, name, res):
    g = GRAPHS[name]
    G = cd.Graph.from_synth(g, device="cuda")
    for refine in (False, True):
        r = G.plm(refine=refine, seed=3, resolution=res)
        o = O.plm(*g.numpy(), refine=refine, seed=3, resolution=res)
        _check(r, o)


def test_resolution_default_and_reduced_forms(O):
    """(0, 0) means 1 / 1; 6/4 decides like 3/2."""
    g = GRAPHS["rmat12"]
    G = cd.Graph.from_synth(g, device="cuda")
    a = G.plm(refine=True, resolution=(0, 0))
    b = G.plm(refine=True)
    assert torch.equal(a.labels, b.labels) and all(a.stats[k] == b.stats[k] for k in KEYS)
    c = G.plm(refine=True, resolution=(6, 4))
    d = G.plm(refine=True, resolution=(3, 2))
    assert torch.equal(c.labels, d.labels) and all(c.stats[k] == d.stats[k] for k in KEYS)
    _check(d, O.plm(*g.numpy(), refine=True, resolution=(3, 2)))


def _heavy(scale_w):
    base = synth.random_graph(400, 2500, seed=21, loops=10, wmax=50)
    w = (base.w.to(torch.int64) * scale_w + 7).clamp(max=2**31 - 1).to(torch.int32)
    return synth.Graph(base.n, base.row_ptr, base.col, w, "heavy")


@pytest.mark.parametrize("res", [(3, 1), (1, 3), (64, 1), (1, 64)])
def test_resolution_on_128_bit_paths(O, res):
    """2W >= 2^31 (128 bits for any gamma), and 2W < 2^31 where a large p or
    q alone pushes max(p, q) (2W)^2 past 2^63."""
    for g in (_heavy(3_000_000), _heavy(10_000)):
        G = cd.Graph.from_synth(g, device="cuda")
        for refine in (False, True):
            _check(G.plm(refine=refine, seed=2, resolution=res),
                   O.plm(*g.numpy(), refine=refine, seed=2, resolution=res))
    g = _heavy(10_000)
    assert 2 * cd.Graph.from_synth(g, device="cuda").W < 2**31
    W2 = (2 * cd.Graph.from_synth(g, device="cuda").W) ** 2
    assert 64 * W2 >= 2**63 > W2


@pytest.mark.parametrize("res", [(1, 2), (3, 1)])
def test_epp_final_phase_resolution(O, res):
    for name in ("pp_small", "chunglu_w"):
        g = GRAPHS[name]
        G = cd.Graph.from_synth(g, device="cuda")
        r = G.epp(b=3, final_refine=True, seed=2, resolution=res)
        o = O.epp(*g.numpy(), b=3, final_refine=True, seed=2, resolution=res)
        assert np.array_equal(r.labels.cpu().numpy(), o.labels)
        assert r.modularity == o.modularity


def test_invalid_resolution_rejected():
    g = GRAPHS["rmat12"]
    G = cd.Graph.from_synth(g, device="cuda")
    for res in ((-1, 1), (1, 0)):
        with pytest.raises(cd.CDError) as e:
            G.plm(resolution=res)
        assert e.value.status == cd.CD_EINVAL
    # max(p, q) (2W)^2 >= 2^126 could overflow the 128-bit gain
    H = cd.Graph.from_synth(_heavy(3_000_000), device="cuda")
    assert (2**62) * (2 * H.W) ** 2 >= 2**126
    for res in ((2**62, 1), (1, 2**62)):
        with pytest.raises(cd.CDError) as e:
            H.plm(refine=True, resolution=res)
        assert e.value.status == cd.CD_EINVAL
    # the library still works afterwards
    assert G.plm().stats["converged"] == 1 and H.plm().stats["converged"] == 1
