"""Write the oracle's results on the full-size workloads to fullsize.json.

Only the oracle (``oracle/``, its OpenMP build, whose results equal the
sequential build's: tests/test_oracle_openmp.py) and the seeded generators
are called; no value comes from the CUDA library.  The GPU tests in
tests/test_zy_fullsize.py compare the library's results on the same graphs
with these records, bit for bit.

Each record holds what a GPU run must reproduce exactly:
* the graph's fingerprint (n, nnz, SHA-256 of the CSR arrays), so that a
  generator that drew another graph on another platform fails loudly;
* for a colouring: the number of colours and the SHA-256 of the colour array;
* for PLM / PLMR (Algorithms 2-4) and PLP (Algorithm 1): the SHA-256 of the
  compacted labels (int32, little endian), the exact modularity fraction
  N / D of Eq. 1 over 4W^2, the double the oracle returns, and the schedule
  counters (levels, sweeps, moves, adjacency entries scanned, candidates,
  decisions, communities, convergence).

Usage: python tests/golden/make_golden.py [--threads T] [--only NAME ...]
(R-MAT scale 22 takes a few minutes on 8 cores; Chung-Lu n = 16M about half
an hour.)
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle  # noqa: E402
from paper_1304_4453_gb300 import synth  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "fullsize.json")

STAT_KEYS = ["levels", "sweeps", "moves", "entries", "candidates", "decisions", "ncomm",
             "converged", "colors0", "iters"]


def sha(a) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def fingerprint(rp, c, w) -> dict:
    h = hashlib.sha256()
    for a in (rp.astype(np.int64), c.astype(np.int32)) + (() if w is None else (w.astype(np.int32),)):
        h.update(np.ascontiguousarray(a).tobytes())
    return {"n": int(len(rp) - 1), "nnz": int(len(c)), "weighted": w is not None, "sha256": h.hexdigest()}


def run_record(kind, rp, c, w, threads, **kw) -> dict:
    t = time.time()
    if kind == "plp":
        r = oracle.plp(rp, c, w, threads=threads, **kw)
    else:
        r = oracle.plm(rp, c, w, refine=(kind == "plmr"), threads=threads, **kw)
    dt = time.time() - t
    mod, N, D = oracle.modularity(rp, c, w, r.labels)
    assert mod == r.modularity
    return {"labels_sha256": sha(r.labels.astype(np.int32)), "modularity": r.modularity,
            "mod_num": str(N), "mod_den": str(D),
            "stats": {k: r.stats[k] for k in STAT_KEYS}, "oracle_s": round(dt, 1), "threads": threads}


def colour_record(rp, c, w, seed) -> dict:
    k, col = oracle.color(rp, c, w, seed)
    return {"seed": seed, "colors": int(k), "colour_sha256": sha(col.astype(np.int32))}


WORKLOADS = {
    # R-MAT scale 22, edge factor 16, seed 1: the benchmark's graph
    "rmat22": (lambda: synth.rmat(22, 16, 0.57, 0.19, 0.19, seed=1),
               [("colour", {"seed": 1}), ("colour", {"seed": 7}),
                ("plm", {"seed": 1}), ("plmr", {"seed": 1}), ("plp", {"seed": 1})]),
    # Chung-Lu n = 16M, exponent 2.1, degrees 4..1e5, weights 1..100: the
    # PLMR workload with 2W >= 2^31 (128-bit gains)
    "chunglu16m": (lambda: synth.chung_lu(16_000_000, seed=1),
                   [("plmr", {"seed": 1})]),
}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=0, help="0: all cores (OpenMP build); 1: sequential")
    ap.add_argument("--only", nargs="*", default=None)
    a = ap.parse_args()
    oracle.build()
    out = json.load(open(OUT)) if os.path.exists(OUT) else {}
    out["_about"] = ("Oracle results on the full-size workloads, written by tests/golden/make_golden.py "
                     "(oracle/ and the seeded generators only). Labels, colourings and counters follow "
                     "Algorithms 1-4 under the colour-class schedule; modularity is Eq. 1 as the exact "
                     "fraction mod_num / mod_den.")
    for name, (make, runs) in WORKLOADS.items():
        if a.only and name not in a.only:
            continue
        t = time.time()
        g = make()
        rp, c, w = g.numpy()
        rec = {"graph": fingerprint(rp, c, w), "m": int(g.m), "gen_s": round(time.time() - t, 1)}
        print(name, rec["graph"], flush=True)
        for kind, kw in runs:
            key = kind if kind != "colour" else f"colour_seed{kw['seed']}"
            if kind == "colour":
                rec[key] = colour_record(rp, c, w, kw["seed"])
            else:
                rec[key] = dict(run_record(kind, rp, c, w, a.threads, **kw), seed=kw["seed"])
            print(" ", key, rec[key], flush=True)
        out[name] = rec
        with open(OUT, "w") as f:
            json.dump(out, f, indent=1, sort_keys=True)
            f.write("\n")


if __name__ == "__main__":
    main()
