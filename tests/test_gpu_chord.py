"""Convergence of the reduced backward-Euler solve (Eq. be_residual_rom_section).

The GPU iterates with a chord Jacobian: I - dt Phi^T D J_f D^-1 Phi formed in
FP32 at the first iteration of a step and applied through its FP32 inverse,
against the FP64 residual that fixes the root. The oracle takes Newton steps
with the exact FP64 Jacobian. Both stop at max|delta| <= 1e-12 (1 + max|a|).
A chord iteration converges linearly, Newton quadratically, so the GPU may need
more iterations; these tests bound the difference to one iteration per step,
at the gradient workload's size (N = 65536, r = 64, nu = 5e-3; measured 4
against 3 on every step) and at small viscosity (nu = 1e-3), where the reduced
Jacobian is least dominated by its identity.

The lifted states are compared too (every tenth step, after the event's state
transfer) at the FP64 parity tolerance 1e-10.
"""
import numpy as np
import pytest

import synth

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


def _configs():
    big = synth.config_adjoint()                      # N = 65536, r = 64, nu = 5e-3, z = 10
    small_nu = synth.RomConfig(problem=synth.BURGERS, n_cells=4096, r=16, n_s=0, w_init=100, z=10,
                               dt=1e-4, nu=1e-3, lam=0.1, n_online=100, seed=7)
    return [(big, 30), (small_nu, 100)]


@pytest.mark.parametrize("case", [0, 1])
def test_chord_iterations_against_fp64_newton(g, case):
    from oracle import rom as orom
    cfg, steps = _configs()[case]
    q0 = synth.initial_state(cfg)
    ref = orom.AdaptiveROM(cfg, q0)
    gpu = g.AdaptiveROM(cfg, q0)
    it_gpu, it_ref = [], []
    worst = 0.0
    for n in range(steps):
        ref.step()
        gpu.step(1)
        it_gpu.append(gpu.info()["rom_newton_iters"])
        it_ref.append(ref.newton_iters[-1])
        if (n + 1) % 10 == 0:
            q, q_or = gpu.q_tilde(), ref.lifted()      # both after the event's state transfer
            worst = max(worst, float(np.linalg.norm(q - q_or) / np.linalg.norm(q_or)))
    gpu.close()
    it_gpu, it_ref = np.array(it_gpu), np.array(it_ref)
    print(f"\nN={cfg.n_cells} r={cfg.r} nu={cfg.nu}: iterations per step GPU chord "
          f"mean {it_gpu.mean():.2f} max {it_gpu.max()}, oracle Newton mean {it_ref.mean():.2f} "
          f"max {it_ref.max()}; trajectory difference {worst:.2e}")
    assert np.max(it_gpu - it_ref) <= 1
    assert worst < 1e-10
