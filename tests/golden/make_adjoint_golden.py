"""Writes adjoint_burgers_n65536_r64.json: the terminal-misfit gradient of the
adaptive Burgers ROM at the gradient workload's full size (N = 65536, r = 64,
nu = 5e-3, z = 10, lambda = 0.1, w_init = 100, 1000 online steps), by the
FP64 oracle only, in forward mode and as the checkpointed reverse sweep
(checkpoints every 50 steps).

With ``--fd`` it also stores central differences of the forward oracle
(h = 1e-4 relative, Newton converged to 1e-14) as an independent check.

The oracle needs minutes at this size, so the values are stored for the GPU
tests to compare against. Run from the repository root:

    python tests/golden/make_adjoint_golden.py [--fd]
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import synth                      # noqa: E402
from oracle import adjoint as adj  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "adjoint_burgers_n65536_r64.json")


def central_differences(cfg, n_steps, target, rel=1e-4):
    out = {}
    tight = adj.at(cfg, newton_tol=1e-14, newton_max=40)
    for name, key in (("nu", "nu"), ("A", "amplitude")):
        base = getattr(cfg, key)
        h = rel * base
        Jp, _ = adj.misfit(adj.at(tight, **{key: base + h}), n_steps, target)
        Jm, _ = adj.misfit(adj.at(tight, **{key: base - h}), n_steps, target)
        out[name] = (Jp - Jm) / (2.0 * h)
    return out


def main():
    with_fd = "--fd" in sys.argv[1:]
    cfg = synth.config_adjoint()
    n_steps = cfg.n_online
    target = synth.burgers_target(cfg.n_cells, cfg.seed + 1)
    t0 = time.time()
    J, g_fwd = adj.tangent_gradient(cfg, n_steps, target)
    t1 = time.time()
    J2, g_rev = adj.adjoint_gradient(cfg, n_steps, target, ckpt_every=50)
    t2 = time.time()
    if J2 != J:
        raise RuntimeError("forward and reverse passes disagree on J")
    rel = {k: abs(g_rev[k] - g_fwd[k]) / abs(g_fwd[k]) for k in g_fwd}
    fd = central_differences(cfg, n_steps, target) if with_fd else None
    t3 = time.time()
    out = dict(
        workload="burgers_n65536_r64_z10_adjoint",
        config=cfg.to_dict(),
        n_steps=n_steps,
        target="synth.burgers_target(n_cells, seed + 1)",
        loss="J = 1/2 ||q~(last online step) - target||^2",
        J=J,
        grad_forward_mode={k: float(v) for k, v in g_fwd.items()},
        grad_reverse_sweep={k: float(v) for k, v in g_rev.items()},
        forward_vs_reverse_rel=rel,
        ckpt_every=50,
        central_differences=None if fd is None else {
            "h_rel": 1e-4, "newton_tol": 1e-14, "value": {k: float(v) for k, v in fd.items()},
            "forward_mode_vs_fd_rel": {k: abs(g_fwd[k] - fd[k]) / abs(fd[k]) for k in fd}},
        seconds={"forward_mode": round(t1 - t0, 1), "reverse_sweep": round(t2 - t1, 1),
                 "central_differences": round(t3 - t2, 1) if with_fd else None},
        numpy=np.__version__,
    )
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
        f.write("\n")
    print(json.dumps(out, indent=1, sort_keys=True))


if __name__ == "__main__":
    main()
