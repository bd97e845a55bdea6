"""Full-size parity on the benchmark workloads, bit for bit against the oracle.

The oracle's results on these graphs are stored in tests/golden/fullsize.json,
written by tests/golden/make_golden.py, which calls only oracle/ and the
seeded generators.  Each test regenerates the graph, checks its fingerprint
against the record (so a generator that drew a different graph fails
loudly), runs the library through the C ABI in the configuration bench.py
times (default options and launch shape), and compares:

* colourings: the number of colours and the SHA-256 of the colour array;
* PLM, PLMR and PLP (Algorithms 1-4): the SHA-256 of the labels, the
  modularity double (Eq. 1; both sides divide the same exact integers), and
  the schedule counters (levels, sweeps, moves, adjacency entries scanned,
  candidates, decisions, communities, convergence).

Workloads: R-MAT scale 22, edge factor 16, abcd = (0.57, 0.19, 0.19, 0.05),
seed 1 (4,194,304 vertices, 128M CSR entries), and Chung-Lu n = 16M,
exponent 2.1, degrees 4..1e5, weights 1..100, seed 1, whose 2W >= 2^31
takes the 128-bit gain path.  Properties that hold at any size
(tests/properties.py, pinned in tests/test_properties_cpu.py) are checked
as well.  R-MAT scale 26 (about 2.1 billion CSR entries), where a borrowed
device CSR (CD_BORROW) spares the graph's second copy, is checked against the
copying handle and the properties.

This file is collected late (only the allocation-free entry point's test comes
after it): it holds the largest graphs of the suite.
"""
import hashlib
import json
import os

import numpy as np
import pytest
import torch

from paper_1304_4453_gb300 import cd, synth

from . import properties as P

pytestmark = pytest.mark.gpu

MOD_TOL = 1e-12
GOLDEN = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "fullsize.json")))
STAT_KEYS = ["levels", "sweeps", "moves", "entries", "candidates", "decisions", "ncomm", "converged",
             "colors0"]
PLP_KEYS = ["iters", "moves", "entries", "candidates", "decisions", "ncomm", "converged"]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1304_4453_gb300 import build
    build.build()
    cd.lib()


def _sha(a) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def _fingerprint(rp, c, w):
    h = hashlib.sha256()
    for a in (rp.astype(np.int64), c.astype(np.int32)) + (() if w is None else (w.astype(np.int32),)):
        h.update(np.ascontiguousarray(a).tobytes())
    return {"n": int(len(rp) - 1), "nnz": int(len(c)), "weighted": w is not None, "sha256": h.hexdigest()}


def _check_run(r, rec, keys):
    assert r.stats["converged"] == rec["stats"]["converged"]
    assert _sha(r.labels.cpu().numpy().astype(np.int32)) == rec["labels_sha256"]
    assert abs(r.modularity - rec["modularity"]) <= MOD_TOL
    assert r.modularity == rec["modularity"]
    for k in keys:
        assert r.stats[k] == rec["stats"][k], (k, r.stats[k], rec["stats"][k])


@pytest.fixture(scope="module")
def rmat22():
    rec = GOLDEN["rmat22"]
    g = synth.rmat(22, 16, 0.57, 0.19, 0.19, seed=1, device="cuda")
    host = (g.row_ptr.cpu().numpy(), g.col.cpu().numpy(), None)
    assert _fingerprint(*host) == rec["graph"], "the generator drew another R-MAT 22 graph"
    G = cd.Graph(g.row_ptr, g.col, g.w)
    del g
    yield G, host, rec
    G.close()


@pytest.mark.parametrize("seed", [1, 7])
def test_rmat22_colouring_equals_oracle(rmat22, seed):
    G, (rp, c, w), rec = rmat22
    out = torch.empty(G.n, dtype=torch.int32, device="cuda")
    k = cd.cd_color(G.h, out, seed)
    want = rec[f"colour_seed{seed}"]
    assert k == want["colors"]
    col = out.cpu().numpy()
    assert _sha(col) == want["colour_sha256"]
    if seed == 7:   # the property checker agrees with the record as well
        P.check_first_fit_colouring(rp, c, col, seed)


def test_rmat22_plm_equals_oracle(rmat22):
    G, (rp, c, w), rec = rmat22
    r1 = G.plm(refine=False, seed=1)
    _check_run(r1, rec["plm"], STAT_KEYS)
    lab = r1.labels.cpu().numpy()
    assert P.check_dense_labels(lab) == r1.stats["ncomm"]
    q, N, D = P.modularity_exact(rp, c, w, lab, fraction=True)
    assert (str(N), str(D)) == (rec["plm"]["mod_num"], rec["plm"]["mod_den"])
    assert abs(G.modularity(r1.labels) - q) <= MOD_TOL
    r2 = G.plm(refine=False, seed=1)
    assert torch.equal(r1.labels, r2.labels)


def test_rmat22_plmr_equals_oracle(rmat22):
    G, (rp, c, w), rec = rmat22
    r = G.plm(refine=True, seed=1)
    _check_run(r, rec["plmr"], STAT_KEYS)
    assert r.stats["converged"] == 1
    lab = r.labels.cpu().numpy()
    rng = np.random.default_rng(11)
    deg = np.diff(rp)
    sample = np.union1d(rng.choice(G.n, 3000, replace=False), np.argsort(deg)[-200:])
    assert P.positive_gain_moves(rp, c, w, lab, sample) == []


def test_rmat22_plp_equals_oracle(rmat22):
    G, _, rec = rmat22
    r = G.plp(seed=1)
    _check_run(r, rec["plp"], PLP_KEYS)


@pytest.fixture(scope="module")
def chunglu16m():
    rec = GOLDEN.get("chunglu16m")
    if rec is None:
        pytest.fail("no golden record for Chung-Lu 16M (run tests/golden/make_golden.py --only chunglu16m)")
    g = synth.chung_lu(16_000_000, seed=1, device="cpu")
    host = g.numpy()
    assert _fingerprint(*host) == rec["graph"], \
        "the Chung-Lu generator drew another graph on this platform (float64 quantiles)"
    G = cd.Graph(g.row_ptr.cuda(), g.col.cuda(), g.w.cuda())
    del g
    yield G, rec
    G.close()


def test_chunglu16m_plmr_equals_oracle(chunglu16m):
    G, rec = chunglu16m
    assert 2 * G.W >= 2**31          # the 128-bit gain path
    r = G.plm(refine=True, seed=1)
    _check_run(r, rec["plmr"], STAT_KEYS)


def test_rmat26_borrowed_equals_copied():
    """R-MAT scale 26, edge factor 16 (67M vertices, 2.1 billion CSR entries,
    64-bit row offsets): PLM on a handle that borrows the device CSR, run in
    the low-memory mode (8 GiB of coarsening scratch), and on a copying
    handle in the default mode give identical labels and modularity, and the
    labels are a dense partition carrying their exact modularity."""
    g = synth.rmat(26, 16, 0.57, 0.19, 0.19, seed=1, device="cuda")
    assert g.n == 1 << 26 and g.nnz > 2_000_000_000
    torch.cuda.synchronize()
    torch.cuda.empty_cache()   # the generator's scratch goes back before the library allocates
    B = cd.Graph(g.row_ptr, g.col, g.w, borrow=True)
    rb = B.plm(refine=False, seed=1, scratch_budget=8 << 30)   # and the low-memory mode
    lab_b = rb.labels.cpu()
    B.close()
    C = cd.Graph(g.row_ptr, g.col, g.w)
    rc = C.plm(refine=False, seed=1)
    assert torch.equal(lab_b, rc.labels.cpu()) and rb.modularity == rc.modularity
    assert rb.stats["converged"] == 1
    assert P.check_dense_labels(lab_b.numpy()) == rb.stats["ncomm"]
    assert abs(C.modularity(rc.labels) - rb.modularity) <= MOD_TOL
    C.close()

