"""Input generators: structure and distribution of the batched-workload
planted-partition sampler (CPU only)."""
import math

import numpy as np
import torch

from paper_1304_4453_gb300 import synth


def _blocks(n, k):
    return np.repeat(np.arange(k), synth._block_sizes(n, k))


def _check_csr(g):
    rp, col, w = g.numpy()
    assert rp[0] == 0 and rp[-1] == col.size and np.all(np.diff(rp) >= 0)
    src = np.repeat(np.arange(g.n), np.diff(rp))
    assert np.all(src != col)
    for u in range(min(g.n, 500)):
        row = col[rp[u]:rp[u + 1]]
        assert np.all(np.diff(row) > 0)
    fwd = set(zip(src.tolist(), col.tolist()))
    assert all((v, u) in fwd for u, v in fwd)
    return src, col


def test_planted_partition_fast_structure_and_determinism():
    g1 = synth.planted_partition_fast(3001, 7, 0.05, 0.002, seed=9)
    g2 = synth.planted_partition_fast(3001, 7, 0.05, 0.002, seed=9)
    assert torch.equal(g1.row_ptr, g2.row_ptr) and torch.equal(g1.col, g2.col)
    _check_csr(g1)
    g3 = synth.planted_partition_fast(3001, 7, 0.05, 0.002, seed=10)
    assert not torch.equal(g1.col, g3.col)


def test_planted_partition_fast_edge_counts():
    """Intra- and inter-block edge counts are binomial with the right means."""
    n, k, p_in, p_out = 4000, 9, 0.02, 0.001
    sizes = synth._block_sizes(n, k)
    pairs_in = sum(s * (s - 1) // 2 for s in sizes)
    pairs_out = n * (n - 1) // 2 - pairs_in
    bl = _blocks(n, k)
    for seed in (1, 2, 3):
        g = synth.planted_partition_fast(n, k, p_in, p_out, seed=seed)
        src, col = _check_csr(g)
        intra = int((bl[src] == bl[col]).sum()) // 2
        inter = g.m - intra
        for cnt, N, p in ((intra, pairs_in, p_in), (inter, pairs_out, p_out)):
            sd = math.sqrt(N * p * (1 - p))
            assert abs(cnt - N * p) < 5 * sd, (cnt, N * p, sd)


def test_planted_partition_fast_pairs_uniform():
    """Every pair of a block (and across blocks) is equally likely: over many
    seeds, each of the 15 pairs of a 6-vertex graph with 2 blocks of 3 appears
    with frequency p_in or p_out."""
    n, k, p_in, p_out = 6, 2, 0.6, 0.25
    bl = _blocks(n, k)
    hits = np.zeros((n, n))
    trials = 4000
    for s in range(trials):
        g = synth.planted_partition_fast(n, k, p_in, p_out, seed=s)
        rp, col, _ = g.numpy()
        src = np.repeat(np.arange(n), np.diff(rp))
        hits[src, col] += 1
    for u in range(n):
        for v in range(u + 1, n):
            p = p_in if bl[u] == bl[v] else p_out
            sd = math.sqrt(trials * p * (1 - p))
            assert abs(hits[u, v] - trials * p) < 5 * sd, (u, v, hits[u, v], trials * p)


def test_planted_partition_fast_degenerate():
    assert synth.planted_partition_fast(1, 1, 0.5, 0.5).m == 0
    assert synth.planted_partition_fast(10, 2, 0.0, 0.0).m == 0
    full = synth.planted_partition_fast(12, 3, 1.0, 1.0)
    assert full.m == 12 * 11 // 2
