"""Pins of the oracle's explicit form (App. D: the RDE solver's four-stage,
third-order SSP Runge-Kutta scheme; the Galerkin ROM advanced by the same
scheme): the scheme's stability polynomial and order, the full-basis limit
of the explicit Galerkin and DEIM-Galerkin steps, and an adaptive run that
tracks the explicit FOM (no GPU)."""
import numpy as np
import pytest

import synth
from oracle import fv, rom


@pytest.mark.parametrize("z", [-0.3, -1.7, -4.0, 0.25 + 1.1j, -2.0 + 2.0j])
def test_ssprk43_stability_polynomial(z):
    """On dq/dt = lam q one step multiplies q by (1 + z/2)(2/3 + (1 + z/2)^3 / 3)
    (the stages written out), which expands to the third-order Taylor
    polynomial of exp(z) plus z^4/48."""
    lam = complex(z)
    q0 = np.array([1.0 + 0.0j, 0.5 - 0.25j])
    q1 = fv.ssprk43_step(q0, 1.0, lambda q: lam * q)
    R = 1 + z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 48
    assert np.allclose(q1, R * q0, rtol=1e-14, atol=0)


def test_ssprk43_is_third_order_on_a_nonlinear_problem():
    """dq/dt = q^2, q(0) = 1 has q(t) = 1 / (1 - t): halving h divides the
    error at t = 0.5 by about 8."""
    errs = []
    for n in (20, 40, 80, 160):
        h = 0.5 / n
        q = np.array([1.0])
        for _ in range(n):
            q = fv.ssprk43_step(q, h, lambda u: u * u)
        errs.append(abs(q[0] - 2.0))
    ratios = [errs[i] / errs[i + 1] for i in range(3)]
    assert all(7.0 < x < 9.0 for x in ratios), ratios


def full_basis(cfg, q):
    """An orthonormal basis of the whole state space and the preprocessing of
    a short FOM trajectory."""
    rng = np.random.default_rng(3)
    Q = rom.fom_trajectory(q, 3, cfg)
    q_ref, d, _ = rom.preprocess(Q, q, cfg.n_var)
    Phi = np.linalg.qr(rng.standard_normal((cfg.n, cfg.n)))[0]
    return Phi, q_ref, d


@pytest.mark.parametrize("problem", [0, 1])
def test_explicit_galerkin_with_full_basis_is_the_fom_step(problem):
    """With r = N the explicit Galerkin ROM is a change of variables of the
    FOM, which the Runge-Kutta stages commute with."""
    if problem == 0:
        cfg = synth.config_burgers_small()
        cfg.n_cells = 64
    else:
        cfg = synth.config_sod()
        cfg.n_cells, cfg.n_var = 48, 3
    cfg.time_scheme = 1
    q = synth.initial_state(cfg)
    Phi, q_ref, d = full_basis(cfg, q)
    a = Phi.T @ (d * (q - q_ref))
    a1, _ = rom.explicit_galerkin_step(a, Phi, q_ref, d, cfg)
    q_rom = rom.lift(a1, Phi, q_ref, d)
    q_fom = fv.explicit_step(q, cfg.dt, cfg.problem, cfg.nu, cfg.gamma)
    assert np.linalg.norm(q_rom - q_fom) <= 1e-12 * np.linalg.norm(q_fom)


@pytest.mark.parametrize("problem,order", [(0, "natural"), (0, "shuffled"), (1, "natural"), (1, "shuffled")])
def test_explicit_hyper_step_with_every_row_sampled_is_galerkin(problem, order):
    """With every row sampled (in any order) and Phi orthonormal,
    (P^T Phi)^+ P^T = Phi^T, so the DEIM-Galerkin right-hand side is the
    Galerkin one (Burgers, and the Euler system's 3N rows)."""
    if problem == 0:
        cfg = synth.config_burgers_small()
        cfg.n_cells = 96
    else:
        cfg = synth.config_sod()
        cfg.n_cells, cfg.n_var = 32, 3
    cfg.time_scheme = 1
    q = synth.initial_state(cfg)
    Phi, q_ref, d = full_basis(cfg, q)
    Phi = Phi[:, :12]
    a = Phi.T @ (d * (q - q_ref))
    P = list(range(cfg.n))
    if order == "shuffled":
        P = [int(i) for i in np.random.default_rng(7).permutation(cfg.n)]
    M = rom.sampled_pinv(Phi, P)
    a_g, _ = rom.explicit_galerkin_step(a, Phi, q_ref, d, cfg)
    a_h, _ = rom.explicit_galerkin_step(a, Phi, q_ref, d, cfg, P, M)
    assert np.max(np.abs(a_h - a_g)) <= 1e-12 * np.max(np.abs(a_g))


def test_explicit_adaptive_rom_tracks_the_explicit_fom():
    """Burgers N = 512, r = 10, z = 10, DEIM with QDEIM + feature-guided
    points (n_s = 20), everything explicit except the coarse correction
    (backward Euler over z dt, Eq. coarse_fom_backward_euler): the adaptive
    ROM stays within 1e-3 of the explicit FOM over 500 steps, and the explicit
    and implicit FOMs agree to first order in dt."""
    cfg = synth.config_burgers_small()
    cfg.time_scheme = 1
    cfg.n_s = 20
    q0 = synth.initial_state(cfg)
    m = rom.AdaptiveROM(cfg, q0)
    steps, traj = m.run(500, record_every=100)
    q = q0.copy()
    q_be = q0.copy()
    errs = []
    j = 0
    for n in range(1, steps[-1] + 1):
        q = fv.explicit_step(q, cfg.dt, cfg.problem, cfg.nu)
        if n in steps:
            errs.append(np.linalg.norm(traj[:, j] - q) / np.linalg.norm(q))
            j += 1
    for _ in range(cfg.w_init + 500):
        q_be = fv.be_step(q_be, cfg.dt, cfg.problem, cfg.nu)
    assert max(errs) < 1e-3, errs
    assert np.linalg.norm(q_be - q) / np.linalg.norm(q) < 1e-2


def test_sod_galerkin_fgs_tracks_the_fom_better_than_galerkin():
    """Sod, 512 cells, the Galerkin-FGS form (r = 20 QDEIM points and 20
    points of largest squared pressure difference, n_s = 2 r as in the
    paper's RDE ROM), 200 explicit steps: the hyper-reduced adaptive ROM
    stays bounded and ends closer to the explicit FOM than the plain
    Galerkin adaptive ROM of the same rank on the same training window
    (measured 2.1e-2 against 5.1e-2)."""
    cfg = synth.config_sod(512)
    cfg.time_scheme, cfg.r, cfg.n_s = 1, 20, 40
    q0 = synth.initial_state(cfg)
    fgs = rom.AdaptiveROM(cfg, q0)
    gal_cfg = synth.config_sod(512)
    gal_cfg.time_scheme, gal_cfg.r = 1, 20
    gal = rom.AdaptiveROM(gal_cfg, q0, Q_train=fgs.Q_train)
    q = fgs.Q_train[:, -1].copy()
    for _ in range(200):
        fgs.step()
        gal.step()
        q = fv.explicit_step(q, cfg.dt, cfg.problem, cfg.nu, cfg.gamma)
    e_fgs = rom.relative_error(fgs.lifted(), q)
    e_gal = rom.relative_error(gal.lifted(), q)
    assert np.isfinite(e_fgs) and e_fgs < 0.03, e_fgs
    assert e_fgs < 0.6 * e_gal, (e_fgs, e_gal)
