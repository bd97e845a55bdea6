"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Labels, colourings and coarse graphs must be bit-identical; modularity must
agree within 1e-12 (both sides evaluate the same exact integer fraction, so
in practice the doubles are equal).  The schedule counters (sweeps, moves,
adjacency entries scanned, candidates evaluated, decisions) must match too,
which pins the GPU to the oracle's colour-class schedule step by step.
"""
import numpy as np
import pytest
import torch

from paper_1304_4453_gb300 import cd, synth

pytestmark = pytest.mark.gpu

MOD_TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1304_4453_gb300 import build
    build.build()
    cd.lib()
    torch.cuda.init()


@pytest.fixture(scope="module")
def O():
    from oracle import oracle
    oracle.build()
    return oracle


def gpu_graph(g):
    return cd.Graph.from_synth(g, device="cuda")


def graphs_small():
    out = {
        "pp_small": synth.planted_partition(2000, 8, 0.03, 0.002, seed=2),
        "rmat12": synth.rmat(12, seed=3),
        "rmat14_hubs": synth.rmat(14, seed=5),
        "rand_w_loops": synth.random_graph(300, 1500, seed=7, loops=20, wmax=50),
        "chunglu_w": synth.chung_lu(20000, seed=3),
        "cliques_ring": synth.cliques(12, 6, ring=True),
    }
    return out


GRAPHS = graphs_small()
NAMES = sorted(GRAPHS)


def _np_labels(t):
    return t.detach().cpu().numpy()


# ---------------------------------------------------------------------------
# Building blocks
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name", NAMES)
def test_colouring_bit_exact(O, name):
    g = GRAPHS[name]
    G = gpu_graph(g)
    out = torch.empty(g.n, dtype=torch.int32, device="cuda")
    for seed in (1, 9):
        k = cd.cd_color(G.h, out, seed)
        k2, col = O.color(*g.numpy(), seed)
        assert k == k2
        assert np.array_equal(_np_labels(out), col)


@pytest.mark.parametrize("name", NAMES)
def test_modularity_bit_exact(O, name):
    g = GRAPHS[name]
    G = gpu_graph(g)
    rng = np.random.default_rng(5)
    for k in (1, 7, g.n):
        lab = rng.integers(0, k, g.n).astype(np.int32)
        q_gpu = G.modularity(torch.from_numpy(lab).cuda())
        q_host = G.modularity(lab)
        q_or = O.modularity(*g.numpy(), lab)[0]
        assert q_gpu == q_host
        assert abs(q_gpu - q_or) <= MOD_TOL and q_gpu == q_or


@pytest.mark.parametrize("name", NAMES)
def test_coarsen_bit_exact(O, name):
    g = GRAPHS[name]
    G = gpu_graph(g)
    rng = np.random.default_rng(11)
    lab = rng.integers(0, max(1, g.n // 7), g.n).astype(np.int32)
    ch = cd.cd_coarsen(G.h, lab)
    try:
        rp, col, w = cd.cd_graph_export(ch)
    finally:
        cd.cd_graph_destroy(ch)
    orp, ocol, ow, pi = O.coarsen(*g.numpy(), lab)
    assert np.array_equal(rp, orp)
    assert np.array_equal(col, ocol)
    assert np.array_equal(w, ow)


def test_export_roundtrip_with_loops(O):
    g = GRAPHS["rand_w_loops"]
    G = gpu_graph(g)
    rp, col, w = cd.cd_graph_export(G.h)
    grp, gcol, gw = g.numpy()
    assert np.array_equal(rp, grp) and np.array_equal(col, gcol) and np.array_equal(w, gw)


# ---------------------------------------------------------------------------
# PLM / PLMR / PLP / EPP
# ---------------------------------------------------------------------------

def _same_stats(gs, os_, keys):
    for k in keys:
        assert gs[k] == os_[k], (k, gs[k], os_[k])


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("refine", [False, True])
def test_plm_bit_exact(O, name, refine):
    g = GRAPHS[name]
    G = gpu_graph(g)
    r = G.plm(refine=refine, seed=3)
    o = O.plm(*g.numpy(), refine=refine, seed=3)
    assert np.array_equal(_np_labels(r.labels), o.labels)
    assert abs(r.modularity - o.modularity) <= MOD_TOL
    _same_stats(r.stats, o.stats, ["levels", "sweeps", "moves", "entries", "candidates",
                                   "decisions", "converged", "ncomm"])
    assert r.stats["colors0"] == o.stats["colors0"]


@pytest.mark.parametrize("name", NAMES)
def test_plp_bit_exact(O, name):
    g = GRAPHS[name]
    G = gpu_graph(g)
    for seed in (1, 4):
        r = G.plp(seed=seed)
        o = O.plp(*g.numpy(), seed=seed)
        assert np.array_equal(_np_labels(r.labels), o.labels)
        assert abs(r.modularity - o.modularity) <= MOD_TOL
        _same_stats(r.stats, o.stats, ["iters", "moves", "entries", "candidates", "decisions", "ncomm"])


@pytest.mark.parametrize("name", ["pp_small", "rmat12", "chunglu_w", "rand_w_loops"])
@pytest.mark.parametrize("final_refine", [False, True])
def test_epp_bit_exact(O, name, final_refine):
    g = GRAPHS[name]
    G = gpu_graph(g)
    r = G.epp(b=4, final_refine=final_refine, seed=2)
    o = O.epp(*g.numpy(), b=4, final_refine=final_refine, seed=2)
    assert np.array_equal(_np_labels(r.labels), o.labels)
    assert abs(r.modularity - o.modularity) <= MOD_TOL


def test_config1_planted_partition(O):
    """The n=10,000 planted-partition workload: PLP, then PLM, both exact."""
    g = synth.planted_partition_config1()
    G = gpu_graph(g)
    for fn, ofn in ((G.plp, O.plp), (G.plm, O.plm)):
        r = fn()
        o = ofn(*g.numpy())
        assert np.array_equal(_np_labels(r.labels), o.labels)
        assert abs(r.modularity - o.modularity) <= MOD_TOL


def test_int128_gain_path(O):
    """2W >= 2^31 takes the 128-bit gain and int64 coarse weights."""
    base = synth.random_graph(400, 2500, seed=21, loops=10, wmax=50)
    w = (base.w.to(torch.int64) * 3_000_000 + 7).clamp(max=2**31 - 1).to(torch.int32)
    g = synth.Graph(base.n, base.row_ptr, base.col, w, "heavy")
    G = gpu_graph(g)
    assert 2 * G.W >= 2**31
    for refine in (False, True):
        r = G.plm(refine=refine)
        o = O.plm(*g.numpy(), refine=refine)
        assert np.array_equal(_np_labels(r.labels), o.labels)
        assert r.modularity == o.modularity
    r = G.plp()
    o = O.plp(*g.numpy())
    assert np.array_equal(_np_labels(r.labels), o.labels)


def test_star_hub_path(O):
    """A star whose centre has degree 100,000 exercises the multi-block hub kernels."""
    n = 100_001
    leaves = list(range(1, n))
    edges = [(0, v) for v in leaves] + [(v, v + 1) for v in range(1, n - 1, 2)]
    g = synth.from_edge_list(n, edges)
    G = gpu_graph(g)
    for refine in (False, True):
        r = G.plm(refine=refine)
        o = O.plm(*g.numpy(), refine=refine)
        assert np.array_equal(_np_labels(r.labels), o.labels)
    r = G.plp()
    o = O.plp(*g.numpy())
    assert np.array_equal(_np_labels(r.labels), o.labels)


@pytest.mark.parametrize("case", ["empty", "one", "edgeless", "loops_only", "isolated_mix", "complete", "two_k5"])
def test_degenerate_graphs(O, case):
    if case == "empty":
        g = synth.from_edge_list(0, [])
    elif case == "one":
        g = synth.from_edge_list(1, [])
    elif case == "edgeless":
        g = synth.from_edge_list(7, [])
    elif case == "loops_only":
        g = synth.from_edge_list(4, [], self_loops={0: 3, 2: 1})
    elif case == "isolated_mix":
        g = synth.from_edge_list(10, [(1, 2), (2, 3), (1, 3), (6, 7)], self_loops={9: 2})
    elif case == "complete":
        g = synth.cliques(1, 40)
    else:
        edges = [(a, b) for a in range(5) for b in range(a + 1, 5)]
        edges += [(a + 5, b + 5) for a, b in edges] + [(4, 5)]
        g = synth.from_edge_list(10, edges)
    G = gpu_graph(g)
    for fn, ofn in ((lambda: G.plm(), lambda: O.plm(*g.numpy())),
                    (lambda: G.plm(refine=True), lambda: O.plm(*g.numpy(), refine=True)),
                    (lambda: G.plp(), lambda: O.plp(*g.numpy())),
                    (lambda: G.epp(b=3), lambda: O.epp(*g.numpy(), b=3))):
        r, o = fn(), ofn()
        assert np.array_equal(_np_labels(r.labels), o.labels)
        assert r.modularity == o.modularity


def test_host_and_device_buffers_agree():
    g = GRAPHS["rmat12"]
    G = gpu_graph(g)
    dev = G.plm()
    host = np.zeros(g.n, np.int32)
    mod, st, status = cd.cd_plm(G.h, host)
    assert np.array_equal(host, _np_labels(dev.labels)) and mod == dev.modularity
    Gh = cd.Graph(*g.numpy())          # host-side CSR input
    r = Gh.plm()
    assert np.array_equal(_np_labels(r.labels), host)


def test_repeat_runs_identical():
    g = GRAPHS["rmat14_hubs"]
    G = gpu_graph(g)
    a = G.plm(refine=True)
    la = _np_labels(a.labels).copy()
    b = G.plm(refine=True)
    assert np.array_equal(la, _np_labels(b.labels)) and a.modularity == b.modularity


def test_invalid_csr_rejected():
    g = synth.rmat(8, seed=1)
    rp, col, w = g.numpy()
    bad = col.copy()
    bad[3] = 10**6
    with pytest.raises(cd.CDError) as e:
        cd.Graph(rp, bad)
    assert e.value.status == cd.CD_EINVAL
    asym = synth.random_graph(30, 60, seed=2)
    rp2, c2, w2 = asym.numpy()
    w3 = w2.copy()
    w3[0] += 1
    with pytest.raises(cd.CDError) as e:
        cd.Graph(rp2, c2, w3)
    assert e.value.status == cd.CD_EINVAL
    with pytest.raises(cd.CDError) as e:
        cd.Graph(rp2, c2, -np.abs(w2))
    assert e.value.status == cd.CD_EINVAL
    G = gpu_graph(g)
    with pytest.raises(cd.CDError):
        G.modularity(np.full(g.n, g.n, np.int32))


def test_allocation_failure_is_reported_and_recoverable():
    g = GRAPHS["rmat12"]
    G = gpu_graph(g)
    ref = _np_labels(G.plm().labels).copy()
    for k in (1, 5, 40):
        cd.cd_debug_fail_alloc(k)
        try:
            G.plm()
        except cd.CDError as e:
            assert e.status == cd.CD_ENOMEM
        finally:
            cd.cd_debug_fail_alloc(0)
    assert np.array_equal(_np_labels(G.plm().labels), ref)


def test_sweep_cap_returns_notconv_with_valid_labels(O):
    g = GRAPHS["rmat12"]
    G = gpu_graph(g)
    r = G.plm(max_sweeps=2)
    o = O.plm(*g.numpy(), max_sweeps=2)
    assert r.status == cd.CD_ENOTCONV and o.stats["converged"] == 0
    assert np.array_equal(_np_labels(r.labels), o.labels)


@pytest.mark.parametrize("nh,leaves,seed", [(5, 4200, 1), (4, 4100, 3), (8, 4500, 5)])
def test_adjacent_hubs_share_classes(O, nh, leaves, seed):
    """Mutually adjacent hubs (more than 4096 neighbours) share colour classes:
    their label writes are deferred to the end of the class and the re-check
    passes over a hub whose communities a hub moved earlier in the class
    touched.  Everything must still match the oracle exactly, for PLM, PLMR,
    PLP and EPP."""
    from tests.test_oracle_pins import _hub_core_graph
    g = _hub_core_graph(nh=nh, leaves=leaves, seed=seed)
    G = gpu_graph(g)
    for seed_ in (1, 2):
        k, col = cd.cd_color(G.h, torch.empty(g.n, dtype=torch.int32, device="cuda"), seed_), None
        k2, col2 = O.color(*g.numpy(), seed_)
        assert k == k2
        for refine in (False, True):
            r = G.plm(refine=refine, seed=seed_)
            o = O.plm(*g.numpy(), refine=refine, seed=seed_)
            assert np.array_equal(_np_labels(r.labels), o.labels)
            assert abs(r.modularity - o.modularity) <= MOD_TOL
            _same_stats(r.stats, o.stats, ["levels", "sweeps", "moves", "entries", "candidates", "decisions", "ncomm"])
        r = G.plp(seed=seed_)
        o = O.plp(*g.numpy(), seed=seed_)
        assert np.array_equal(_np_labels(r.labels), o.labels)
        _same_stats(r.stats, o.stats, ["iters", "moves", "entries", "candidates", "decisions", "ncomm"])
    r = G.epp(b=3, seed=4)
    o = O.epp(*g.numpy(), b=3, seed=4)
    assert np.array_equal(_np_labels(r.labels), o.labels)


@pytest.mark.parametrize("name", ["rmat14_hubs", "rand_w_loops", "chunglu_w"])
def test_borrowed_csr_gives_identical_results(O, name):
    """CD_BORROW: the handle reads the caller's device arrays in place (with
    self-loops it keeps only a loop-free copy); every result equals the
    copying handle's and the oracle's."""
    g = GRAPHS[name].to("cuda")
    rp, col = g.row_ptr.contiguous(), g.col.contiguous()
    w = None if g.w is None else g.w.contiguous()
    B = cd.Graph(rp, col, w, borrow=True)
    C = cd.Graph(rp.clone(), col.clone(), None if w is None else w.clone())
    assert (B.n, B.m, B.W) == (C.n, C.m, C.W)
    for fn in (lambda G: G.plm(seed=2), lambda G: G.plm(refine=True, seed=2), lambda G: G.plp(seed=2),
               lambda G: G.epp(b=3, seed=2)):
        rb, rc = fn(B), fn(C)
        assert torch.equal(rb.labels, rc.labels) and rb.modularity == rc.modularity
    o = O.plm(*GRAPHS[name].numpy(), refine=True, seed=2)
    assert np.array_equal(B.plm(refine=True, seed=2).labels.cpu().numpy(), o.labels)
    lab = B.plm(seed=2).labels
    assert B.modularity(lab) == C.modularity(lab)
    rpx, colx, wx = cd.cd_graph_export(B.h)
    rpy, coly, wy = cd.cd_graph_export(C.h)
    assert np.array_equal(rpx, rpy) and np.array_equal(colx, coly) and np.array_equal(wx, wy)
    B.close()
    C.close()


def test_borrow_rejects_host_arrays():
    g = GRAPHS["rmat12"]
    with pytest.raises(cd.CDError) as e:
        cd.Graph(g.row_ptr, g.col, g.w, borrow=True)
    assert e.value.status == cd.CD_EINVAL


@pytest.mark.parametrize("name", NAMES)
def test_forced_128_bit_gains_change_nothing(O, name):
    """int_path 128 runs the 128-bit gain path on graphs whose gains fit 64
    bits: the decisions, and so every result, are the same."""
    g = GRAPHS[name]
    G = gpu_graph(g)
    for refine in (False, True):
        r = G.plm(refine=refine, seed=3, int_path=128)
        o = O.plm(*g.numpy(), refine=refine, seed=3)
        assert np.array_equal(_np_labels(r.labels), o.labels)
        _same_stats(r.stats, o.stats, ["levels", "sweeps", "moves", "entries", "candidates", "decisions"])


def test_int_path_64_rejected_where_inexact():
    base = synth.random_graph(400, 2500, seed=21, loops=10, wmax=50)
    w = (base.w.to(torch.int64) * 3_000_000 + 7).clamp(max=2**31 - 1).to(torch.int32)
    G = gpu_graph(synth.Graph(base.n, base.row_ptr, base.col, w, "heavy"))
    with pytest.raises(cd.CDError) as e:
        G.plm(int_path=64)
    assert e.value.status == cd.CD_EINVAL
    H = gpu_graph(GRAPHS["rmat12"])
    assert H.plm(int_path=64).stats["converged"] == 1
    with pytest.raises(cd.CDError):
        H.plm(int_path=32)
