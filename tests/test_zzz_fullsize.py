"""Full-size checks on the benchmark workload: R-MAT scale 22, edge factor 16,
abcd = (0.57, 0.19, 0.19, 0.05), seed 1 (4,194,304 vertices, about 128M CSR
entries), generated on the device and run through the C ABI in the
configuration bench.py times (PLM, seed 1, default launch shape).

The oracle is too slow at this size, so the GPU results are checked against
properties that hold at any size (tests/properties.py, each pinned against
the oracle and planted mistakes on small graphs):

* the level-0 colouring is first-fit in priority order at every vertex,
  which determines it completely;
* PLM labels are dense, identical on a repeat run, and their modularity is
  the exact Eq. 1 value;
* a converged PLMR result has no positive-gain move, checked on a sample
  of vertices and on the 200 vertices of highest degree (the hub paths).

This file is collected last: it holds the largest graph of the suite.
"""
import numpy as np
import pytest
import torch

from paper_1304_4453_gb300 import cd, synth

from . import properties as P

pytestmark = pytest.mark.gpu

MOD_TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1304_4453_gb300 import build
    build.build()
    cd.lib()


@pytest.fixture(scope="module")
def rmat22():
    g = synth.rmat(22, 16, 0.57, 0.19, 0.19, seed=1, device="cuda")
    G = cd.Graph(g.row_ptr, g.col, g.w)
    host = (g.row_ptr.cpu().numpy(), g.col.cpu().numpy(), None)
    del g
    yield G, host
    G.close()


def test_rmat22_colouring_is_first_fit_in_priority_order(rmat22):
    G, (rp, c, w) = rmat22
    assert G.n == 1 << 22 and len(c) > 100_000_000
    out = torch.empty(G.n, dtype=torch.int32, device="cuda")
    for seed in (1, 7):
        k = cd.cd_color(G.h, out, seed)
        col = out.cpu().numpy()
        assert k == int(col.max()) + 1
        P.check_first_fit_colouring(rp, c, col, seed)


def test_rmat22_plm_bench_configuration(rmat22):
    G, (rp, c, w) = rmat22
    r1 = G.plm(refine=False, seed=1)
    r2 = G.plm(refine=False, seed=1)
    assert r1.stats["converged"] == 1
    lab = r1.labels.cpu().numpy()
    assert np.array_equal(lab, r2.labels.cpu().numpy())
    assert P.check_dense_labels(lab) == r1.stats["ncomm"]
    q = P.modularity_exact(rp, c, w, lab)
    assert abs(r1.modularity - q) <= MOD_TOL
    assert abs(G.modularity(r1.labels) - q) <= MOD_TOL
    assert q > 0


def test_rmat22_plmr_has_no_positive_gain_move(rmat22):
    G, (rp, c, w) = rmat22
    r = G.plm(refine=True, seed=1)
    if r.stats["converged"] != 1:
        pytest.skip("a move phase reached the sweep cap; the property needs a converged run")
    lab = r.labels.cpu().numpy()
    P.check_dense_labels(lab)
    assert abs(r.modularity - P.modularity_exact(rp, c, w, lab)) <= MOD_TOL
    rng = np.random.default_rng(11)
    deg = np.diff(rp)
    sample = np.union1d(rng.choice(G.n, 3000, replace=False), np.argsort(deg)[-200:])
    assert P.positive_gain_moves(rp, c, w, lab, sample) == []
