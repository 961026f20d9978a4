"""Sampling points of the hyper-reduced model (Eq. qdeim_qr, Eq. fgs_selection)
on inputs built to reach every branch of the feature-guided selection.

The feature-guided candidates are selected on the GPU by an exact radix
selection on the bit patterns of the scores: (y_{i+1} - y_i)^2 for Burgers,
(p_{i+1} - p_i)^2 of the cell pressures for the Euler system. Both sides
compute each score with the same IEEE operations in the same order (no fused
multiply-adds), so the scores are bit-identical and the feature-guided part
of the sample set must equal the oracle's greedy choice (largest score first,
ties to the lowest index, QDEIM points skipped) exactly. The QDEIM part is checked against the
GPU's own exported basis (greedy residual norms, to rounding level).
"""
import numpy as np
import pytest

import synth
from oracle import rom as orom

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2605_28684_gb300 as pkg
    from paper_2605_28684_gb300 import build
    build.build()
    return pkg


def _check_samples(gpu, cfg):
    from test_gpu_parity import greedy_residuals
    P = [int(i) for i in gpu.samples()]
    assert len(P) == cfg.n_s and len(set(P)) == cfg.n_s
    st = gpu.state()
    k = gpu.info()["rank"]
    kq = min(k, cfg.n_s)
    res = greedy_residuals(st["phi"][:, :kq], P[:kq])
    for j, p in enumerate(P[:kq]):
        norms = res[j]
        norms[P[:j]] = -1.0
        assert norms[p] >= (1 - 1e-10) * norms.max(), ("QDEIM pivot", j, p)
    expect = orom.fgs_extend(st["y_corr"], P[:kq], cfg.n_s - kq, cfg.problem, cfg.gamma)
    assert P[kq:] == expect
    return P, kq


def _snapshot(kind, n, seed):
    x = (np.arange(n) + 0.5) / n
    rng = np.random.default_rng(seed)
    if kind == "steps":          # three jumps: every other score is exactly zero
        y = np.where(x < 0.25, 1.0, np.where(x < 0.6, 1.7, 1.3))
    elif kind == "plateaus":     # many cells share each of a few exact scores
        y = np.floor(8 * x) * 0.125 + np.where(np.arange(n) % 2 == 0, 0.0, 0.25)
    else:                        # continuous values
        y = 1.0 + 0.5 * np.sin(2 * np.pi * x) + 0.01 * rng.standard_normal(n)
    return y


@pytest.mark.parametrize("n_cells,kind", [(4096, "steps"), (4096, "plateaus"), (16384, "smooth"),
                                          (100, "smooth"), (100, "steps")])
def test_feature_points_against_oracle_rule(g, n_cells, kind):
    cfg = synth.config_burgers_hyper()
    cfg.n_cells = n_cells
    if n_cells < 1000:           # fewer cells than n_s + r: every cell is a candidate
        cfg.r, cfg.n_s = 8, 96
    q0 = synth.initial_state(cfg)
    gpu = g.AdaptiveROM(cfg, q0)
    _check_samples(gpu, cfg)     # the sampling of the offline stage
    gpu.update_basis(_snapshot(kind, n_cells, 11))
    P, kq = _check_samples(gpu, cfg)
    gpu.step(2 * cfg.z)          # two more adaptation cycles on the model's own snapshots
    _check_samples(gpu, cfg)
    gpu.close()


def _euler_snapshot(kind, n, seed, gamma=1.4):
    """Conserved (rho, m, E) rows from primitives."""
    x = (np.arange(n) + 0.5) / n
    rng = np.random.default_rng(seed)
    rho = 1.0 + 0.2 * np.sin(2 * np.pi * x)
    u = 0.1 + 0.05 * np.cos(2 * np.pi * x)
    if kind == "levels":        # seven equal pressure jumps; all other cells near zero
        p = 1.0 + np.floor(8 * x) * 0.125
    else:                        # continuous values
        p = 1.0 + 0.5 * np.sin(2 * np.pi * x) + 0.01 * rng.standard_normal(n)
    return np.concatenate([rho, rho * u, p / (gamma - 1.0) + 0.5 * rho * u * u])


@pytest.mark.parametrize("n_cells,kind", [(512, "levels"), (512, "smooth"), (16384, "levels")])
def test_pressure_feature_points_against_oracle_rule(g, n_cells, kind):
    """Euler system in the explicit form, r = 20 QDEIM points and 20
    pressure-feature points: the sample sets of the offline stage, of two
    adaptation cycles on the model's own snapshots, and of an update on a
    built snapshot (16384 cells: 49152 keys, read from global memory)."""
    cfg = synth.config_sod(n_cells)
    cfg.time_scheme, cfg.r, cfg.n_s = 1, 20, 40
    q0 = synth.initial_state(cfg)
    gpu = g.AdaptiveROM(cfg, q0)
    _check_samples(gpu, cfg)
    gpu.step(2 * cfg.z)
    _check_samples(gpu, cfg)
    gpu.update_basis(_euler_snapshot(kind, n_cells, 5, cfg.gamma))
    _check_samples(gpu, cfg)
    gpu.close()
