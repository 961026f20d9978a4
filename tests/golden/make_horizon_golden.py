"""Writes horizon_<case>.npz: the FP64 oracle's reduced trajectories over the
full horizons of the configured workloads, for the GPU parity tests.

Cases (Algorithm 1, online loop from n = w_init):

* ``c2``  Sod shock tube, 8192 cells, r = 40, z = 10, lambda = 0.01, to t = 0.2
          or to the step whose reduced Newton solve has no root (stored as
          ``fail_step``, the time level of that step; -1 if none);
* ``c3``  twelve instances of the 256-instance Burgers batch (the smallest
          and largest N, the highest r, and nine more spread over N), 2000
          online steps each.

Every ``stride`` online steps (and after the last one) a record keeps q~ (the
lifted state after the step's adaptation event, if it has one) at a fixed
subsample of about 512 entries, its L2 norm and its products with
``synth.probe_vectors`` (seed 77). Each case also keeps ``rank_margin``, the
closest call of the oracle's rank decisions over the run (the minimum of
|log(x / tau)| over the quantities x that the rank tolerance tau is compared
with), which says whether a rounding-level change could flip a rank.
The numerical-rank tolerance is the FP64 form's, 1e-10, unless ``--tau`` says
otherwise. This script calls only ``oracle`` and ``synth``. Run from the
repository root (c2 ~ 8 min, c3 ~ 5 min on 5 processes):

    python tests/golden/make_horizon_golden.py c2|c3 [--tau T]
"""
import argparse
import json
import os
import sys
import time
from concurrent.futures import ProcessPoolExecutor

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import synth                    # noqa: E402
from oracle import rom as orom  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
STRIDE = 500


def subsample(n, count=512):
    return np.arange(0, n, max(1, n // count), dtype=np.int64)


def run_case(cfg, n_steps, tau, stride=STRIDE):
    """Records of one trajectory (dict of arrays)."""
    orom.RANK_TOL = tau
    q0 = synth.initial_state(cfg)
    m = orom.AdaptiveROM(cfg, q0)
    sub = subsample(cfg.n)
    W = synth.probe_vectors(cfg.n)
    steps, qs, norms, probes, ranks = [], [], [], [], []
    fail_step = -1
    for k in range(n_steps):
        try:
            m.step()
        except orom.NewtonNoConvergence:
            # the reduced Newton solve has no root any more (the state left the
            # physical range); the records end at the last completed step
            fail_step = m.n
            if not steps or steps[-1] != m.n:     # the last completed step
                q = m.lifted()
                steps.append(m.n)
                qs.append(q[sub])
                norms.append(float(np.linalg.norm(q)))
                probes.append(W.T @ q)
                ranks.append(orom.numerical_rank(m.Phi))
            break
        if (k + 1) % stride == 0 or k + 1 == n_steps:
            q = m.lifted()
            steps.append(m.n)
            qs.append(q[sub])
            norms.append(float(np.linalg.norm(q)))
            probes.append(W.T @ q)
            ranks.append(orom.numerical_rank(m.Phi))
    out = dict(steps=np.array(steps), sub=sub, q_sub=np.array(qs), norm=np.array(norms),
               probe=np.array(probes), rank=np.array(ranks), min_gap=np.array(m.min_gap),
               rank_margin=np.array(m.min_rank_margin), fail_step=np.array(fail_step))
    return out


def batch_picks(cfgs, count=12):
    """Smallest N, largest N, highest r, then instances spread over N."""
    ns = np.array([c.n_cells for c in cfgs])
    rs = np.array([c.r for c in cfgs])
    picks = [int(np.argmin(ns)), int(np.argmax(ns)), int(np.argmax(rs))]
    order = np.argsort(ns)
    for q in np.linspace(0.05, 0.95, count):
        i = int(order[int(q * (len(order) - 1))])
        if i not in picks and len(picks) < count:
            picks.append(i)
    return sorted(picks)


def _batch_one(args):
    i, tau = args
    cfg = synth.config_batch(256)[i]
    return i, run_case(cfg, 2000, tau)


def meta(cfg, tau, seconds):
    return json.dumps({"config": cfg.to_dict(), "rank_tol": tau, "stride": STRIDE,
                       "oracle_seconds": round(seconds, 1),
                       "generator": "tests/golden/make_horizon_golden.py (oracle only)"})


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["c2", "c3"])
    ap.add_argument("--tau", type=float, default=1e-10)
    ap.add_argument("--procs", type=int, default=4)
    args = ap.parse_args()
    t0 = time.perf_counter()
    suffix = "" if args.tau == 1e-10 else f"_tau{args.tau:g}"
    path = os.path.join(HERE, f"horizon_{args.case}{suffix}.npz")
    if args.case == "c2":
        cfg = synth.config_sod()
        rec = run_case(cfg, cfg.n_online, args.tau)
        np.savez_compressed(path, meta=meta(cfg, args.tau, time.perf_counter() - t0), **rec)
    else:
        cfgs = synth.config_batch(256)
        picks = batch_picks(cfgs)
        out = {}
        with ProcessPoolExecutor(args.procs) as ex:
            for i, rec in ex.map(_batch_one, [(i, args.tau) for i in picks]):
                for key, v in rec.items():
                    out[f"i{i}_{key}"] = v
        np.savez_compressed(path, picks=np.array(picks),
                            meta=json.dumps({"rank_tol": args.tau, "stride": STRIDE,
                                             "oracle_seconds": round(time.perf_counter() - t0, 1),
                                             "instances": picks, "steps": 2000,
                                             "generator": "tests/golden/make_horizon_golden.py "
                                                          "(oracle only)"}), **out)
    print(f"wrote {path} in {time.perf_counter() - t0:.0f} s")


if __name__ == "__main__":
    main()
