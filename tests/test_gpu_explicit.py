"""GPU parity of the explicit form (App. D, the RDE solver's scheme): fine
FOM steps of the training window and Galerkin / DEIM-Galerkin reduced steps
by the four-stage, third-order SSP Runge-Kutta scheme, with the coarse
correction still a backward-Euler step over z dt (Eq.
coarse_fom_backward_euler), against the oracle's whole trajectories."""
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


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def run_pair(g, cfg, n_steps, adopt=False):
    """(error after the offline stage, worst error at the events, adopted
    sampled cells) of the GPU trajectory against the oracle's."""
    from test_gpu_parity import adopt_if_near_tie
    q0 = synth.initial_state(cfg)
    ref = orom.AdaptiveROM(cfg, q0)
    gpu = g.AdaptiveROM(cfg, q0)
    adopted = adopt_if_near_tie(ref, gpu) if adopt else 0
    e0 = rel(gpu.state()["q_tilde"], ref.lifted())
    worst = 0.0
    for _ in range(n_steps // cfg.z):
        for _ in range(cfg.z):
            ref.step()
        gpu.step(cfg.z)
        if adopt:
            adopted += adopt_if_near_tie(ref, gpu)
        worst = max(worst, rel(gpu.q_tilde(), ref.lifted()))
    assert gpu.info()["rank"] == orom.numerical_rank(ref.Phi)
    gpu.close()
    return e0, worst, adopted


def test_explicit_burgers_galerkin_trajectory(g):
    """Burgers N = 512, r = 10, z = 10, 1000 explicit online steps."""
    cfg = synth.config_burgers_small()
    cfg.time_scheme = 1
    e0, worst, _ = run_pair(g, cfg, 1000)
    print(f"explicit Burgers Galerkin: offline {e0:.1e}, worst {worst:.2e}")
    assert e0 <= 1e-12
    assert worst <= 1e-10, worst


@pytest.mark.parametrize("n_cells", [512, 1024])
def test_explicit_burgers_deim_fgs_trajectory(g, n_cells):
    """DEIM-Galerkin with r = 10 QDEIM points and 10 feature-guided points
    (n_s = 2 r, the mix of the paper's RDE ROM), 500 explicit steps. The
    explicit diffusion limit bounds N at dt = 1e-4, nu = 0.01: 4 nu dt N^2 is
    1.0 and 4.2 here, inside the scheme's real stability interval [-5.15, 0]."""
    cfg = synth.config_burgers_small()
    cfg.n_cells = n_cells
    cfg.time_scheme = 1
    cfg.n_s = 20
    e0, worst, adopted = run_pair(g, cfg, 500, adopt=True)
    print(f"explicit Burgers DEIM N={n_cells}: offline {e0:.1e}, worst {worst:.2e}, adopted {adopted}")
    assert e0 <= 1e-12
    assert worst <= 1e-10, worst


def test_explicit_sod_galerkin_trajectory(g):
    """Sod, 1024 cells, r = 40, z = 10, the CFL-0.4 step (within the
    scheme's strong-stability limit), 200 explicit online steps."""
    cfg = synth.config_sod(1024)
    cfg.time_scheme = 1
    e0, worst, _ = run_pair(g, cfg, 200)
    print(f"explicit Sod Galerkin: offline {e0:.1e}, worst {worst:.2e}")
    assert e0 <= 1e-11
    assert worst <= 1e-10, worst


@pytest.mark.parametrize("n_cells", [512, 2048])
def test_explicit_sod_deim_fgs_trajectory(g, n_cells):
    """The Galerkin-FGS form of the paper's RDE ROM on Sod: DEIM-Galerkin
    with r = 20 QDEIM points and 20 points of largest squared pressure
    difference (n_s = 2 r), 200 explicit steps at the CFL-0.4 step. (At other
    sizes this hyper-reduced explicit model can lose stability, e.g. r = 10,
    n_s = 20; the sizes here stay bounded in the oracle.)"""
    cfg = synth.config_sod(n_cells)
    cfg.time_scheme = 1
    cfg.r, cfg.n_s = 20, 40
    e0, worst, adopted = run_pair(g, cfg, 200, adopt=True)
    print(f"explicit Sod DEIM-FGS N={n_cells}: offline {e0:.1e}, worst {worst:.2e}, adopted {adopted}")
    assert e0 <= 1e-11
    assert worst <= 1e-10, worst
