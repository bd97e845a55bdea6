"""Batched and served runs: every graph's result in a batch equals its
single-graph result (labels, modularity and the schedule counters), which
the parity tests tie to the oracle; a batch and every result served in the
server's mix are also compared with the oracle directly.
"""
import numpy as np
import pytest
import torch

from paper_1304_4453_gb300 import cd, synth

pytestmark = pytest.mark.gpu

STAT_KEYS = ["levels", "sweeps", "moves", "iters", "entries", "candidates", "decisions",
             "converged", "ncomm", "colors0"]


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


def _mixed_graphs():
    """Uneven sizes, weighted and unit, degenerate cases, a hub."""
    gs = [synth.planted_partition(n, k, 16 * 20 / (20 * (n // k - 1) + n - n // k),
                                  16 / (20 * (n // k - 1) + n - n // k), seed=100 + i)
          for i, (n, k) in enumerate([(1000, 8), (3000, 12), (20000, 40), (500, 10), (60000, 16)])]
    gs += [synth.rmat(12, seed=3), synth.rmat(14, seed=5), synth.chung_lu(20000, seed=3),
           synth.random_graph(300, 1500, seed=7, loops=20, wmax=50), synth.cliques(12, 6, ring=True),
           synth.from_edge_list(0, []), synth.from_edge_list(7, []),
           synth.from_edge_list(4, [], self_loops={0: 3, 2: 1})]
    n = 20_001
    gs.append(synth.from_edge_list(n, [(0, v) for v in range(1, n)] + [(v, v + 1) for v in range(1, n - 1, 2)]))
    return gs


GRAPHS = _mixed_graphs()


def _single(G, algo, refine, ensemble, **kw):
    if algo == cd.CD_ALGO_PLM:
        return G.plm(refine=refine, **kw)
    if algo == cd.CD_ALGO_PLP:
        return G.plp(**kw)
    return G.epp(b=ensemble, final_refine=refine, **kw)


def _same(r, s):
    assert torch.equal(r.labels.cpu(), s.labels.cpu())
    assert r.modularity == s.modularity
    for k in STAT_KEYS:
        assert r.stats[k] == s.stats[k], (k, r.stats[k], s.stats[k])


@pytest.mark.parametrize("algo,refine,ensemble", [(cd.CD_ALGO_PLM, False, 1), (cd.CD_ALGO_PLM, True, 1),
                                                  (cd.CD_ALGO_PLP, False, 1), (cd.CD_ALGO_EPP, True, 3)])
def test_batch_equals_single(algo, refine, ensemble):
    Gs = [cd.Graph.from_synth(g, device="cuda") for g in GRAPHS]
    batch = cd.run_batch(Gs, algo, refine, ensemble, seed=4)
    for G, r in zip(Gs, batch):
        _same(r, _single(G, algo, refine, ensemble, seed=4))


def test_batch_matches_oracle(O):
    picks = [GRAPHS[1], GRAPHS[5], GRAPHS[8]]
    Gs = [cd.Graph.from_synth(g, device="cuda") for g in picks]
    for refine in (False, True):
        res = cd.run_batch(Gs, cd.CD_ALGO_PLM, refine, seed=2)
        for g, r in zip(picks, res):
            o = O.plm(*g.numpy(), refine=refine, seed=2)
            assert np.array_equal(r.labels.cpu().numpy(), o.labels)
            assert abs(r.modularity - o.modularity) <= 1e-12
            for k in ["levels", "sweeps", "moves", "entries", "candidates", "decisions", "ncomm"]:
                assert r.stats[k] == o.stats[k], k


@pytest.mark.parametrize("quantum,team_min", [(1, 1), (1 << 12, 3), (1 << 30, 8), (1 << 16, 64)])
def test_launch_shape_changes_nothing(quantum, team_min):
    """Team sizes and tiers differ with the shape options; results must not."""
    Gs = [cd.Graph.from_synth(g, device="cuda") for g in GRAPHS[:9]]
    ref = cd.run_batch(Gs, cd.CD_ALGO_PLM, True, seed=6)
    res = cd.run_batch(Gs, cd.CD_ALGO_PLM, True, seed=6, team_quantum=quantum, team_min=team_min)
    for a, b in zip(ref, res):
        _same(a, b)
    G = Gs[2]
    e1 = G.epp(b=4, seed=3)
    e2 = G.epp(b=4, seed=3, team_quantum=quantum, team_min=team_min)
    _same(e1, e2)


def test_batch_many_small_graphs():
    """Many jobs on many host threads over several levels each (the stream
    a job's buffers are freed on must order after the job's own work)."""
    rng = np.random.default_rng(11)
    specs = []
    for j in range(96):
        n = int(np.exp(rng.uniform(np.log(200), np.log(50000))))
        k = int(rng.integers(4, 17))
        s = n // k
        p_out = 16 / (20 * (s - 1) + n - s)
        specs.append(synth.planted_partition(n, k, min(1.0, 20 * p_out), p_out, seed=1000 + j))
    Gs = [cd.Graph.from_synth(g, device="cuda") for g in specs]
    for refine in (False, True):
        res = cd.run_batch(Gs, cd.CD_ALGO_PLM, refine, seed=1)
        for G, r in zip(Gs, res):
            _same(r, G.plm(refine=refine, seed=1))


def test_batch_repeated_handle_and_host_labels():
    g = GRAPHS[5]
    G = cd.Graph.from_synth(g, device="cuda")
    outs = [np.zeros(g.n, np.int32) for _ in range(3)]
    mods, sts, status = cd.cd_run_batch([G.h] * 3, cd.make_task(cd.CD_ALGO_PLM), outs)
    s = G.plm()
    for o, m in zip(outs, mods):
        assert np.array_equal(o, s.labels.cpu().numpy()) and m == s.modularity


def test_batch_mixed_gain_widths():
    """A graph with 2W >= 2^31 (128-bit gains) next to ordinary graphs."""
    base = synth.random_graph(400, 2500, seed=21, loops=10, wmax=50)
    w = (base.w.to(torch.int64) * 3_000_000 + 7).clamp(max=2**31 - 1).to(torch.int32)
    heavy = synth.Graph(base.n, base.row_ptr, base.col, w, "heavy")
    Gs = [cd.Graph.from_synth(g, device="cuda") for g in (heavy, GRAPHS[0], GRAPHS[8])]
    res = cd.run_batch(Gs, cd.CD_ALGO_PLM, True, seed=5)
    for G, r in zip(Gs, res):
        _same(r, G.plm(refine=True, seed=5))


def test_batch_invalid_arguments():
    G = cd.Graph.from_synth(GRAPHS[0], device="cuda")
    out = torch.empty(G.n, dtype=torch.int32, device="cuda")
    with pytest.raises(cd.CDError) as e:
        cd.cd_run_batch([G.h], cd.make_task(7), [out])
    assert e.value.status == cd.CD_EINVAL
    with pytest.raises(cd.CDError) as e:
        cd.cd_run_batch([G.h], cd.make_task(cd.CD_ALGO_EPP, ensemble=0), [out])
    assert e.value.status == cd.CD_EINVAL
    mods, sts, status = cd.cd_run_batch([], cd.make_task(cd.CD_ALGO_PLM), [])
    assert mods == [] and status == cd.CD_OK


# ---------------------------------------------------------------------------
# Server
# ---------------------------------------------------------------------------

def _oracle_run(O, g, algo, refine, ensemble, seed):
    if algo == cd.CD_ALGO_PLM:
        return O.plm(*g.numpy(), refine=refine, seed=seed)
    if algo == cd.CD_ALGO_PLP:
        return O.plp(*g.numpy(), seed=seed)
    return O.epp(*g.numpy(), b=ensemble, final_refine=refine, seed=seed)


ORACLE_KEYS = {cd.CD_ALGO_PLM: ["levels", "sweeps", "moves", "entries", "candidates", "decisions",
                                "converged", "ncomm"],
               cd.CD_ALGO_PLP: ["iters", "moves", "entries", "candidates", "decisions", "ncomm"],
               cd.CD_ALGO_EPP: ["ncomm"]}


def test_server_results_match_oracle(O):
    """Every served result, computed in the server's mix of concurrently
    admitted runs, equals the oracle's result for that graph and task:
    labels bit for bit, modularity, and the schedule counters."""
    Gs = [cd.Graph.from_synth(g, device="cuda") for g in GRAPHS]
    tasks = [(cd.CD_ALGO_PLM, False, 1), (cd.CD_ALGO_PLM, True, 1), (cd.CD_ALGO_PLP, False, 1),
             (cd.CD_ALGO_EPP, True, 2)]
    S = cd.Server(max_slots=8)
    try:
        tickets = []
        for i, (g, G) in enumerate(zip(GRAPHS, Gs)):
            for t in tasks[i % 2::2]:
                tickets.append((g, G, t, S.submit(G, *t, seed=7)))
        for g, G, t, tk in tickets:
            out = torch.empty(max(G.n, 1), dtype=torch.int32, device="cuda")[:G.n]
            status, mod, lat, st = S.poll(tk, out, timeout_ms=-1)
            assert lat >= 0
            o = _oracle_run(O, g, *t, seed=7)
            assert np.array_equal(out.cpu().numpy(), o.labels), t
            assert abs(mod - o.modularity) <= 1e-12 and mod == o.modularity
            for k in ORACLE_KEYS[t[0]]:
                assert st[k] == o.stats[k], (t, k, st[k], o.stats[k])
        assert S.info() == (0, 0, 0)
    finally:
        S.close()


def test_server_one_slot_and_host_labels():
    Gs = [cd.Graph.from_synth(g, device="cuda") for g in GRAPHS[:6]]
    S = cd.Server(max_slots=1)
    try:
        tks = [S.submit(G, cd.CD_ALGO_PLM) for G in Gs]
        for G, tk in zip(Gs, tks):
            out = np.zeros(G.n, np.int32)
            status, mod, lat, st = S.poll(tk, out, timeout_ms=-1)
            assert np.array_equal(out, G.plm().labels.cpu().numpy())
    finally:
        S.close()


def test_server_admission_limits():
    G = cd.Graph.from_synth(GRAPHS[4], device="cuda")
    S = cd.Server(device_mem_budget=1 << 20, max_slots=1, max_queue=1)
    try:
        with pytest.raises(cd.CDError) as e:
            S.submit(G, cd.CD_ALGO_PLM)
        assert e.value.status == cd.CD_EINVAL
        with pytest.raises(cd.CDError) as e:
            S.poll(12345)
        assert e.value.status == cd.CD_EINVAL
    finally:
        S.close()
    S = cd.Server(max_slots=1, max_queue=1)
    try:
        tks, busy = [], 0
        for _ in range(40):
            try:
                tks.append(S.submit(G, cd.CD_ALGO_PLM, refine=True))
            except cd.CDError as err:
                assert err.status == cd.CD_EBUSY
                busy += 1
        assert busy > 0
        ref = G.plm(refine=True)
        for tk in tks:
            out = torch.empty(G.n, dtype=torch.int32, device="cuda")
            S.poll(tk, out, timeout_ms=-1)
            assert torch.equal(out, ref.labels)
    finally:
        S.close()


def test_server_lanes_small_runs_pass_large_ones(O):
    """Runs above 2^21 entries + vertices go to the large lane, the rest to
    the small lane; both lanes give single-run results, and a small run
    submitted right after a large one does not wait for the large one's
    phases (it finishes first)."""
    big_g = synth.rmat(20, seed=4)
    small_g = [GRAPHS[i] for i in (0, 1, 3, 5, 9)]
    big = cd.Graph.from_synth(big_g, device="cuda")
    smalls = [cd.Graph.from_synth(g, device="cuda") for g in small_g]
    assert big.m * 2 + big.n > 1 << 21 and all(G.m * 2 + G.n <= 1 << 21 for G in smalls)
    ref_big = big.plm(seed=5)
    S = cd.Server(max_slots=8)
    try:
        t_big = S.submit(big, cd.CD_ALGO_PLM, seed=5)
        t_small = [S.submit(G, cd.CD_ALGO_PLM, seed=5) for G in smalls]
        lat_small = []
        for g, G, tk in zip(small_g, smalls, t_small):
            out = torch.empty(max(G.n, 1), dtype=torch.int32, device="cuda")[:G.n]
            status, mod, lat, st = S.poll(tk, out, timeout_ms=-1)
            assert np.array_equal(out.cpu().numpy(), O.plm(*g.numpy(), seed=5).labels)
            lat_small.append(lat)
        out = torch.empty(big.n, dtype=torch.int32, device="cuda")
        status, mod, lat_big, st = S.poll(t_big, out, timeout_ms=-1)
        assert torch.equal(out, ref_big.labels) and mod == ref_big.modularity
        assert max(lat_small) < lat_big, (lat_small, lat_big)
    finally:
        S.close()


def test_server_destroy_with_pending_runs():
    Gs = [cd.Graph.from_synth(g, device="cuda") for g in GRAPHS[:5]]
    S = cd.Server(max_slots=2)
    for G in Gs:
        S.submit(G, cd.CD_ALGO_EPP, ensemble=2)
    S.close()
    # the device is still usable
    r = Gs[0].plm()
    assert r.stats["converged"] == 1


# ---------------------------------------------------------------------------
# Degree-bin limits and the autotuner (speed-only options)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("bins", [(4, 4, 4, 4, 4), (1, 2, 3, 4, 5), (2, 8, 32, 256, 1024), (4, 16, 128, 1024, 4096),
                                  (3, 12, 64, 512, 2048), (4, 16, 16, 16, 4096), (4, 16, 128, 1024, 1024)])
def test_bin_limits_change_nothing(O, bins):
    """Moving vertices between the lane-group, block, global-table block and
    hub roles leaves every result and counter unchanged (the (4,4,4,4,4) case
    sends every vertex above degree 4 down the multi-block hub path, the last
    one every vertex of degree 17..4096 to the global-table block role)."""
    for g in (GRAPHS[0], GRAPHS[5], GRAPHS[7], GRAPHS[8], GRAPHS[9]):
        G = cd.Graph.from_synth(g, device="cuda")
        for refine in (False, True):
            _same(G.plm(refine=refine, seed=2, bin_max=bins), G.plm(refine=refine, seed=2))
        _same(G.plp(seed=2, bin_max=bins), G.plp(seed=2))
    g = GRAPHS[5]
    r = cd.Graph.from_synth(g, device="cuda").plm(refine=True, seed=2, bin_max=bins)
    o = O.plm(*g.numpy(), refine=True, seed=2)
    assert np.array_equal(r.labels.cpu().numpy(), o.labels)


def test_bin_limits_validated():
    G = cd.Graph.from_synth(GRAPHS[0], device="cuda")
    for bad in [(5, 16, 128, 1024), (4, 3, 128, 1024), (4, 16, 129, 1024), (4, 16, 128, 2048),
                (-1, 16, 128, 1024), (4, 16, 128, 1024, 8192), (4, 16, 128, 1024, 512)]:
        with pytest.raises(cd.CDError) as e:
            G.plm(bin_max=bad)
        assert e.value.status == cd.CD_EINVAL


def test_tuner_returns_a_shape_with_identical_results():
    Gs = [cd.Graph.from_synth(g, device="cuda") for g in GRAPHS[:6]]
    task = cd.make_task(cd.CD_ALGO_PLM, refine=True)
    best, ms = cd.cd_tune([G.h for G in Gs], task, cd.default_opts(seed=3), max_trials=6)
    assert ms > 0 and best.seed == 3 and best.team_min >= 1 and best.team_quantum >= 1
    kw = dict(seed=3, team_quantum=best.team_quantum, team_min=best.team_min, bin_max=list(best.bin_max))
    for a, b in zip(cd.run_batch(Gs, cd.CD_ALGO_PLM, True, **kw), cd.run_batch(Gs, cd.CD_ALGO_PLM, True, seed=3)):
        _same(a, b)
    best1, _ = cd.cd_tune([Gs[1].h], cd.make_task(cd.CD_ALGO_PLP), None, max_trials=3)
    assert 0 not in list(best1.bin_max)
