"""Write the FP64 oracle's results at the full workload sizes that are too
slow to recompute inside a test run (a few minutes each on one core):

* the 512x512x300 CT pair (FFD spacing 5, 16x16x8 spatial-bin intervals,
  128 bins), FP32 and BF16 storage;
* the 32-pair PET/CT-shaped batch (BF16 storage, spacing 8, bins on the FFD
  grid, 32 bins).

For each case: D, the gradient norm, the largest gradient magnitude and 64
seeded gradient entries, at seeded coefficients.  Inputs come from ``synth``
and every value from ``oracle`` only.  The file records a hash of the
generator and oracle sources; the GPU test refuses a stale file.

    python tests/golden/make_full_size.py [--jobs 8]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
OUT = os.path.join(HERE, "full_size_oracle.json")
SOURCES = ["synth/__init__.py", "oracle/__init__.py", "oracle/srwcr_oracle.c"]
N_SAMPLES = 64


def source_hash() -> str:
    h = hashlib.sha256()
    for f in SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def cases():
    """(name, kind, argument, storage, coefficient seed, sigma)."""
    out = [("c5_f32", "c5", None, "f32", 5005, 2.0), ("c5_bf16", "c5", None, "bf16", 5005, 2.0)]
    out += [(f"c4_pair{p:02d}", "c4", p, "bf16", 7000 + p, 2.0) for p in range(32)]
    return out


def pair_of(kind, arg):
    import synth
    if kind == "c5":
        return synth.make_pair("c5_ct_512x512x300")
    return synth.batch_specs(32)[arg]


def run_case(case):
    import numpy as np
    import oracle
    import synth
    name, kind, arg, storage, seed, sigma = case
    t = time.time()
    pair = pair_of(kind, arg)
    prob = pair.prob
    c = synth.coefficients(prob, seed, sigma)
    geo = oracle.Geometry.from_problem(prob)
    A, M = oracle.prepare(pair.fixed, pair.moving, prob.n_bins, storage)
    st = oracle.value(geo, A, M, c)
    g = oracle.gradient(geo, A, M, c, st).ravel()
    idx = np.random.default_rng(seed).choice(prob.n_params, N_SAMPLES, replace=False)
    return name, {"kind": kind, "pair": arg, "storage": storage, "coef_seed": seed,
                  "coef_sigma": sigma, "dims": list(prob.dims), "D": float(st.D),
                  "n_degenerate": int(st.n_degenerate), "gnorm": float(np.linalg.norm(g)),
                  "gmax": float(np.abs(g).max()), "idx": [int(i) for i in idx],
                  "g_idx": [float(v) for v in g[idx]], "seconds": time.time() - t}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=os.cpu_count() or 1)
    args = ap.parse_args()
    import oracle
    oracle.build()
    todo = sorted(cases(), key=lambda cs: cs[1] != "c5")  # long cases first
    with mp.get_context("spawn").Pool(args.jobs) as pool:
        res = dict(pool.imap_unordered(run_case, todo))
    out = {"source_hash": source_hash(), "n_samples": N_SAMPLES,
           "cases": {k: res[k] for k in sorted(res)}}
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
