"""Sampling points of the hyper-reduced model (Eq. qdeim_qr, Eq. fgs_selection)
on inputs built to reach every branch of the feature-guided selection.

The feature-guided candidates are selected on the GPU by an exact radix
selection on the bit patterns of the scores (y_{i+1} - y_i)^2. Both sides
compute each score with one IEEE subtraction and one multiplication, so the
scores are bit-identical and the feature-guided part of the sample set must
equal the oracle's greedy choice (largest score first, ties to the lowest
index, QDEIM points skipped) exactly. The QDEIM part is checked against the
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
    expect = orom.fgs_extend(st["y_corr"], P[:kq], cfg.n_s - kq)
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
