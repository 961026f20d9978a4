"""Writes c1_rounding_sensitivity.json: how far two FP64 runs of the oracle
drift apart over the Burgers DEIM horizon (N = 16384, r = 32, n_s = 96,
z = 5, 20 000 online steps) when they differ only by rounding.

Run (a) is the oracle as it stands; run (b) takes every np.linalg.svd call
through LAPACK's gesvd driver instead of gesdd (the same backward-stable SVD
with different rounding). Where (b)'s sample set differs from (a)'s after an
event (near ties of the QDEIM pivots or feature scores), (b) adopts (a)'s set,
so the two differ by rounding only. Every 100 events the record keeps the
relative L2 difference of the lifted states, its maximum so far and the
number of adopted cells. The GPU parity test bounds its own difference from
the oracle by a multiple of this curve.

This script calls only ``oracle`` and ``synth`` (and scipy's LAPACK).
Run from the repository root (about an hour on one core):

    python tests/golden/make_c1_sensitivity.py
"""
import json
import os
import sys
import time

import numpy as np
import scipy.linalg as sla

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import synth                    # noqa: E402
from oracle import rom as orom  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
EVERY = 100


def gesvd(a, full_matrices=True, compute_uv=True, hermitian=False):
    if not compute_uv:
        return sla.svd(a, compute_uv=False, lapack_driver="gesvd")
    return sla.svd(a, full_matrices=full_matrices, lapack_driver="gesvd")


def main():
    cfg = synth.config_burgers_hyper(precision=0)
    q0 = synth.initial_state(cfg)
    gesdd = np.linalg.svd
    t0 = time.perf_counter()
    ra = orom.AdaptiveROM(cfg, q0)
    np.linalg.svd = gesvd
    rb = orom.AdaptiveROM(cfg, q0)
    np.linalg.svd = gesdd
    adopted = 0
    if sorted(rb.P) != sorted(ra.P):
        adopted += len(set(rb.P) ^ set(ra.P))
        rb.P = list(ra.P)
        rb.M = orom.sampled_pinv(rb.Phi, rb.P)
    worst = 0.0
    rec = {"step": [], "diff": [], "worst": [], "adopted": []}
    n_ev = cfg.n_online // cfg.z
    for k in range(n_ev):
        for _ in range(cfg.z):
            ra.step()
        np.linalg.svd = gesvd
        for _ in range(cfg.z):
            rb.step()
        np.linalg.svd = gesdd
        if sorted(rb.P) != sorted(ra.P):
            adopted += len(set(rb.P) ^ set(ra.P))
            rb.P = list(ra.P)
            rb.M = orom.sampled_pinv(rb.Phi, rb.P)
        qa = ra.lifted()
        e = float(np.linalg.norm(rb.lifted() - qa) / np.linalg.norm(qa))
        worst = max(worst, e)
        if (k + 1) % EVERY == 0 or k + 1 == n_ev:
            rec["step"].append(int(ra.n))
            rec["diff"].append(e)
            rec["worst"].append(worst)
            rec["adopted"].append(adopted)
            print(f"{ra.n} {e:.2e} worst {worst:.2e} adopted {adopted} "
                  f"{time.perf_counter() - t0:.0f} s", flush=True)
    out = {"config": cfg.to_dict(), "every_events": EVERY, "events": n_ev, **rec,
           "oracle_seconds": round(time.perf_counter() - t0, 1),
           "generator": "tests/golden/make_c1_sensitivity.py (oracle only)"}
    with open(os.path.join(HERE, "c1_rounding_sensitivity.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
