"""GPU gradient of the terminal misfit (rom_adjoint) against the FP64 oracle's
reverse sweep, the stored full-size gradient, central differences of the GPU
forward pass, and through a torch.autograd.Function.

Tolerance. The gradient form computes its POD as a backward-stable thin SVD
(CGS2 QR and one-sided Jacobi) and runs every step in FP64, so its gradient
follows the oracle's to rounding amplified by the gaps of the POD's and the
cores' singular values. Gradients are compared at 1e-8 relative (the stated
bar of the gradient against the FP64 oracle), J at 1e-9, unless the gradient
itself is less well determined in FP64: each case measures that by running
the oracle a second time with every SVD taken by another LAPACK driver
(gesvd instead of gesdd, a rounding-level change), and a case whose oracle
gradient moves by more than 1e-8/4 under that change is compared at four
times the move."""
import contextlib
import functools
import math

import numpy as np
import pytest

import synth
from oracle import adjoint as oadj

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GRAD_RTOL = 1e-8


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2605_28684_gb300 as pkg
    from paper_2605_28684_gb300 import build
    build.build()
    return pkg


def gpu_gradient(g, cfg, n_steps, ckpt_every=50):
    q0 = synth.initial_state(cfg)
    target = synth.burgers_target(cfg.n_cells, cfg.seed + 1)
    J, dnu, dq0 = g.adjoint(cfg, q0, target, n_steps, ckpt_every)
    dA = float(dq0 @ synth.burgers_ic_amplitude_direction(cfg.n_cells))
    return J, dnu, dA, dq0


def small_cases():
    base = synth.config_adjoint()
    c1 = synth.config_adjoint()
    c1.n_cells, c1.r = 1024, 16
    c2 = synth.config_adjoint()
    c2.n_cells, c2.r, c2.z, c2.lam, c2.nu, c2.seed = 777, 8, 5, 0.5, 4e-3, 9
    c3 = synth.config_adjoint()
    c3.n_cells, c3.r, c3.z, c3.lam, c3.w_init, c3.seed = 2048, 12, 20, 1e-7, 60, 11
    del base
    return [(c1, 1000), (c2, 300), (c3, 400)]


@contextlib.contextmanager
def lapack_svd_driver(driver):
    """Every np.linalg.svd call of the oracle taken by scipy's LAPACK driver."""
    import scipy.linalg as sla
    orig = np.linalg.svd

    def svd(a, full_matrices=True, compute_uv=True, hermitian=False):
        if not compute_uv:
            return sla.svd(a, compute_uv=False, lapack_driver=driver)
        return sla.svd(a, full_matrices=full_matrices, lapack_driver=driver)
    np.linalg.svd = svd
    try:
        yield
    finally:
        np.linalg.svd = orig


@functools.lru_cache(maxsize=None)
def oracle_case(case):
    """(J, gradient, tolerance per component) of small case `case`."""
    cfg, n_steps = small_cases()[case]
    target = synth.burgers_target(cfg.n_cells, cfg.seed + 1)
    J_or, grad_or = oadj.adjoint_gradient(cfg, n_steps, target, ckpt_every=50)
    with lapack_svd_driver("gesvd"):
        _, grad_alt = oadj.adjoint_gradient(cfg, n_steps, target, ckpt_every=50)
    tol = {}
    for key in ("nu", "A"):
        move = abs(grad_alt[key] - grad_or[key]) / abs(grad_or[key])
        tol[key] = max(GRAD_RTOL, 4.0 * move)
    return J_or, grad_or, tol


@pytest.mark.parametrize("case", range(3))
def test_gradient_matches_oracle_reverse_sweep(g, case):
    cfg, n_steps = small_cases()[case]
    J_or, grad_or, tol = oracle_case(case)
    J, dnu, dA, _ = gpu_gradient(g, cfg, n_steps)
    e_nu = abs(dnu - grad_or["nu"]) / abs(grad_or["nu"])
    e_A = abs(dA - grad_or["A"]) / abs(grad_or["A"])
    print(f"N={cfg.n_cells} r={cfg.r}: J {J:.10e} (oracle {J_or:.10e}); dJ/dnu rel {e_nu:.2e} "
          f"(bound {tol['nu']:.1e}), dJ/dA rel {e_A:.2e} (bound {tol['A']:.1e})")
    assert abs(J - J_or) <= 1e-9 * abs(J_or)
    assert e_nu <= tol["nu"] and e_A <= tol["A"]


def test_gradient_independent_of_checkpoint_interval(g):
    cfg, n_steps = small_cases()[0]
    n_steps = 300
    a = gpu_gradient(g, cfg, n_steps, ckpt_every=n_steps)
    b = gpu_gradient(g, cfg, n_steps, ckpt_every=50)
    c = gpu_gradient(g, cfg, n_steps, ckpt_every=7)
    for x in (b, c):
        assert x[0] == a[0]
        assert abs(x[1] - a[1]) <= 1e-13 * abs(a[1])
        assert np.max(np.abs(x[3] - a[3])) <= 1e-13 * np.max(np.abs(a[3]))


def test_gradient_central_differences_of_gpu_forward(g):
    """dJ/dnu and dJ/dA against central differences of J computed by the GPU
    forward pass itself (h = 1e-4 relative, Newton to 1e-13)."""
    cfg, n_steps = small_cases()[0]
    cfg.newton_tol = 1e-13
    n_steps = 500
    J, dnu, dA, _ = gpu_gradient(g, cfg, n_steps)
    target = synth.burgers_target(cfg.n_cells, cfg.seed + 1)
    fd = {}
    for name, key in (("nu", "nu"), ("A", "amplitude")):
        base = getattr(cfg, key)
        h = 1e-4 * base
        vals = []
        for sgn in (1.0, -1.0):
            c = oadj.at(cfg, **{key: base + sgn * h})
            Jv, _, _ = g.adjoint(c, synth.initial_state(c), target, n_steps, n_steps)
            vals.append(Jv)
        fd[name] = (vals[0] - vals[1]) / (2.0 * h)
    e_nu = abs(dnu - fd["nu"]) / abs(fd["nu"])
    e_A = abs(dA - fd["A"]) / abs(fd["A"])
    print(f"central differences: dJ/dnu rel {e_nu:.2e}, dJ/dA rel {e_A:.2e}")
    assert e_nu <= GRAD_RTOL and e_A <= GRAD_RTOL


def test_gradient_full_size_against_stored_oracle_values(g):
    """The gradient workload itself (N = 65536, r = 64, 1000 steps, 100 events)
    against the oracle's stored full-size gradient."""
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                        "adjoint_burgers_n65536_r64.json")
    with open(path) as f:
        ref = json.load(f)
    cfg = synth.config_adjoint()
    J, dnu, dA, _ = gpu_gradient(g, cfg, cfg.n_online, ckpt_every=50)
    J_or = ref["J"]
    g_nu = ref["grad_reverse_sweep"]["nu"]
    g_A = ref["grad_reverse_sweep"]["A"]
    e_nu = abs(dnu - g_nu) / abs(g_nu)
    e_A = abs(dA - g_A) / abs(g_A)
    print(f"full size: J {J:.12e} (oracle {J_or:.12e}); dJ/dnu {dnu:.10e} rel {e_nu:.2e}; "
          f"dJ/dA {dA:.10e} rel {e_A:.2e}")
    assert abs(J - J_or) <= 1e-9 * abs(J_or)
    assert e_nu <= GRAD_RTOL and e_A <= GRAD_RTOL


def test_autograd_function_backpropagates_to_amplitude_and_viscosity(g):
    """The initial state is built in torch from the amplitude A, so autograd
    chains dJ/dq0 (from the library) into dJ/dA."""
    cfg, n_steps = small_cases()[1]
    target_np = synth.burgers_target(cfg.n_cells, cfg.seed + 1)
    x = torch.tensor(synth.cell_centres(cfg.n_cells), dtype=torch.float64, device="cuda")
    S = torch.tensor(synth.mode_sum(cfg.n_cells, cfg.seed), dtype=torch.float64, device="cuda")
    A = torch.tensor(cfg.amplitude, dtype=torch.float64, device="cuda", requires_grad=True)
    nu = torch.tensor(cfg.nu, dtype=torch.float64, device="cuda", requires_grad=True)
    q0 = 1.0 + A * torch.sin(2.0 * math.pi * x) + 0.1 * S
    Misfit = g.misfit_function()
    J = Misfit.apply(nu, q0, cfg, torch.tensor(target_np, device="cuda"), n_steps, 50)
    J.backward()
    J_or, grad_or, tol = oracle_case(1)
    assert abs(float(J) - J_or) <= 1e-9 * abs(J_or)
    assert abs(float(nu.grad) - grad_or["nu"]) <= tol["nu"] * abs(grad_or["nu"])
    assert abs(float(A.grad) - grad_or["A"]) <= tol["A"] * abs(grad_or["A"])


def test_adjoint_rejects_unsupported_configurations(g):
    cfg = synth.config_burgers_hyper()          # DEIM: not covered by the gradient
    q0 = synth.initial_state(cfg)
    with pytest.raises(g.RomError) as ei:
        g.adjoint(cfg, q0, q0, 10)
    assert ei.value.code == 1
    cfg = synth.config_adjoint()
    cfg.n_cells = 1024
    q0 = synth.initial_state(cfg)
    bad = q0.copy()
    bad[3] = np.nan
    with pytest.raises(g.RomError) as ei:
        g.adjoint(cfg, q0, bad, 10)
    assert ei.value.code == 5
