"""Full-horizon parity: the GPU path over the whole online horizon of the
configured workloads against stored FP64 oracle trajectories
(tests/golden/horizon_*.npz, written by tests/golden/make_horizon_golden.py,
which calls only the oracle).

Each record holds q~ after a step (every 500 steps and the last) at a fixed
subsample of about 512 entries, its L2 norm and its products with seeded
probe vectors. The GPU state is compared on all three: relative L2 of the
subsample, relative difference of the norm and of the probe products.

* Burgers DEIM, N = 16384, r = 32, n_s = 96, z = 5, all 20 000 steps (FP64):
  1e-10 at every record, and the same sample set at every one of the 4000
  events (compared through the sum and the sum of squares of the indices).
* 256-instance batch, 2000 steps: twelve instances (smallest and largest N,
  highest r, nine more) against the oracle run at the batch's rank tolerance
  (1e-5) within 1e-5, and against the FP64 form's (1e-10) within the distance
  between the two oracles plus 1e-5.
"""
import json
import os

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2605_28684_gb300 as pkg
    from paper_2605_28684_gb300 import build
    build.build()
    return pkg


def load(name):
    path = os.path.join(GOLDEN, name)
    if not os.path.exists(path):
        pytest.skip(f"{name} not generated")
    return np.load(path)


def record_errors(q, rec, j, W):
    """(subsample relative L2, norm relative, probe relative) of q against record j."""
    sub = rec["sub"]
    e_sub = np.linalg.norm(q[sub] - rec["q_sub"][j]) / np.linalg.norm(rec["q_sub"][j])
    e_norm = abs(np.linalg.norm(q) - rec["norm"][j]) / rec["norm"][j]
    pr = W.T @ q
    e_probe = np.max(np.abs(pr - rec["probe"][j])) / np.max(np.abs(rec["probe"][j]))
    return e_sub, e_norm, e_probe


def test_burgers_deim_full_horizon(g):
    rec = load("horizon_c1.npz")
    meta = json.loads(str(rec["meta"]))
    cfg = synth.config_burgers_hyper(precision=0)
    assert cfg.matches(meta["config"])
    q0 = synth.initial_state(cfg)
    W = synth.probe_vectors(cfg.n)
    gpu = g.AdaptiveROM(cfg, q0)
    steps = list(rec["steps"])
    fp = {int(s): (int(a), int(b)) for s, a, b in zip(rec["fp_step"], rec["fp_sum"], rec["fp_sumsq"])}
    worst = 0.0
    mismatched = []
    n = cfg.w_init
    j = 0
    for _ in range(cfg.n_online // cfg.z):
        gpu.step(cfg.z)
        n += cfg.z
        P = np.asarray(gpu.samples(), dtype=np.int64)
        if (int(P.sum()), int((P * P).sum())) != fp[n]:
            mismatched.append(n)
        if j < len(steps) and n == steps[j]:
            e = record_errors(gpu.q_tilde(), rec, j, W)
            worst = max(worst, *e)
            j += 1
    gpu.close()
    print(f"Burgers DEIM full horizon: worst error {worst:.2e} over {j} records; "
          f"{len(mismatched)} of {len(fp)} events with a different sample set")
    assert j == len(steps)
    assert not mismatched, mismatched[:10]
    assert worst <= 1e-10, worst


def test_batch_full_horizon_instances(g):
    rec10 = load("horizon_c3.npz")
    rec5 = load("horizon_c3_tau1e-05.npz")
    picks = [int(i) for i in rec10["picks"]]
    assert picks == [int(i) for i in rec5["picks"]]
    cfgs = synth.config_batch(256)
    q0s = [synth.initial_state(c) for c in cfgs]
    b = g.Batch(cfgs, q0s)
    steps = [int(s) for s in rec10[f"i{picks[0]}_steps"]]
    W = {i: synth.probe_vectors(cfgs[i].n) for i in picks}
    worst5 = {i: 0.0 for i in picks}
    worst10 = {i: 0.0 for i in picks}
    gap = {i: 0.0 for i in picks}
    done = cfgs[0].w_init
    for j, s in enumerate(steps):
        b.step(s - done)
        done = s
        for i in picks:
            r5 = {k: rec5[f"i{i}_{k}"] for k in ("sub", "q_sub", "norm", "probe")}
            r10 = {k: rec10[f"i{i}_{k}"] for k in ("sub", "q_sub", "norm", "probe")}
            q = b.q_tilde(i)
            worst5[i] = max(worst5[i], *record_errors(q, r5, j, W[i]))
            worst10[i] = max(worst10[i], *record_errors(q, r10, j, W[i]))
            gap[i] = max(gap[i], np.linalg.norm(r5["q_sub"][j] - r10["q_sub"][j])
                         / np.linalg.norm(r10["q_sub"][j]))
    b.close()
    for i in picks:
        print(f"instance {i} (N={cfgs[i].n_cells}, r={cfgs[i].r}, z={cfgs[i].z}): vs oracle tau 1e-5 "
              f"{worst5[i]:.2e}; vs FP64 oracle {worst10[i]:.2e} (oracle gap {gap[i]:.2e})")
    assert all(worst5[i] <= 1e-5 for i in picks), worst5
    assert all(worst10[i] <= gap[i] + 1e-5 for i in picks), (worst10, gap)


def test_sod_full_horizon(g):
    """Sod, 8192 cells, r = 40, z = 10: the oracle's FP64 Galerkin ROM reaches
    t = 0.2 only if its reduced Newton solves keep a root; the stored record
    says where it first has none (fail_step, -1 if never). The GPU follows
    the oracle at every record up to there (1e-9 relative) and then has no
    root at the same step either."""
    rec = load("horizon_c2.npz")
    cfg = synth.config_sod()
    q0 = synth.initial_state(cfg)
    W = synth.probe_vectors(cfg.n)
    fail = int(rec["fail_step"])
    gpu = g.AdaptiveROM(cfg, q0)
    n = cfg.w_init
    worst = 0.0
    for j, s in enumerate(int(x) for x in rec["steps"]):
        gpu.step(s - n)
        n = s
        worst = max(worst, *record_errors(gpu.q_tilde(), rec, j, W))
    print(f"Sod full horizon: worst error {worst:.2e} over {len(rec['steps'])} records, "
          f"oracle without a reduced root at time level {fail}")
    assert worst <= 1e-9, worst
    if fail >= 0:
        assert n == fail
        with pytest.raises(g.RomError) as ei:
            gpu.step(1)
        assert ei.value.code in (4, 5), ei.value.code     # no convergence / non-finite
    gpu.close()
