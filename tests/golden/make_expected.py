"""Writes tests/golden/expected_counts.json from the CPU oracle.

Every stored value here comes from ``oracle`` (never from the CUDA path),
on graphs made by the seeded generators. Each record also stores a SHA-256
digest of the generated arrays, so a test can tell a changed input apart
from a changed count.

    python tests/golden/make_expected.py            # all workloads
    python tests/golden/make_expected.py --quick    # skip the 20M-edge graph
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

import oracle  # noqa: E402
from paper_2308_07932_gb300 import synth  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "expected_counts.json")


def digest(g) -> str:
    h = hashlib.sha256()
    for a in (g.rowptr, g.col, g.sign):
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


def sample_vertices(g, seed: int, n_random: int = 24, n_top: int = 4) -> np.ndarray:
    """Per-vertex check points: the highest-degree vertices of each side plus
    seeded random vertices of each side (gid = u, or nU + v)."""
    rng = np.random.default_rng(seed)
    degU = np.diff(g.rowptr)
    degV = np.bincount(g.col, minlength=g.nV)
    top_u = np.argsort(-degU, kind="stable")[:n_top]
    top_v = g.nU + np.argsort(-degV, kind="stable")[:n_top]
    ru = rng.choice(g.nU, size=min(n_random, g.nU), replace=False)
    rv = g.nU + rng.choice(g.nV, size=min(n_random, g.nV), replace=False)
    return np.unique(np.concatenate([top_u, top_v, ru, rv])).astype(np.int64)


WORKLOADS = {
    "uniform_2000x1000_e20000_p0.7": (synth.uniform_2k_1k, True),
    "vote_500x50000_p0.4_b2": (synth.vote_500_50k, True),
    "chunglu_m200000_s41": (lambda: synth.chung_lu_scaled(41, 200_000), True),
    "chunglu_m2000000_s43": (lambda: synth.chung_lu_scaled(43, 2_000_000), True),
    "chunglu_2Mx500k_e20M_a2.1_p0.8": (synth.chung_lu_2m, True),
}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--quick", action="store_true")
    ap.add_argument("--threads", type=int, default=oracle.default_threads())
    args = ap.parse_args()
    out = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            out = json.load(f)
    for name, (make, with_pv) in WORKLOADS.items():
        if args.quick and name.startswith("chunglu_2M"):
            continue
        t0 = time.time()
        g = make()
        bal, tot = oracle.count(g, threads=args.threads)
        rec = {"nU": g.nU, "nV": g.nV, "nE": g.nE, "sha256": digest(g),
               "balanced": bal, "total": tot}
        if with_pv:
            ids = sample_vertices(g, seed=len(name))
            rec["per_vertex_gids"] = ids.tolist()
            rec["per_vertex"] = oracle.per_vertex(g, ids, threads=args.threads).tolist()
        out[name] = rec
        print(f"{name}: balanced={bal} total={tot} ({time.time() - t0:.1f}s)", flush=True)
    out["_about"] = ("Counts from the CPU oracle (oracle/, Defs. 1-2; per-vertex by "
                     "Algorithm 3) on the seeded synthetic graphs of "
                     "paper_2308_07932_gb300.synth; written by tests/golden/make_expected.py.")
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main()
