"""The seeded input recipe (no GPU): each generator produces what its
docstring states, so that every test and the bench run on the stated
workloads."""
import math

import numpy as np

import synth


def fourier_coefficients(u):
    """(b_k, c_k) with u = b_0 + sum_k b_k cos(2 pi k x) + c_k sin(2 pi k x) on
    the cell centres (exact for band-limited u)."""
    n = u.shape[0]
    x = synth.cell_centres(n)
    k = np.arange(n // 2)
    C = np.cos(2 * np.pi * np.outer(x, k))
    S = np.sin(2 * np.pi * np.outer(x, k))
    return 2.0 * (C.T @ u) / n, 2.0 * (S.T @ u) / n


def test_cell_centres():
    x = synth.cell_centres(4)
    assert np.array_equal(x, [0.125, 0.375, 0.625, 0.875])


def test_burgers_ic_is_the_stated_fourier_series():
    """u0 = 1 + A sin(2 pi x) + 0.1 sum_{k<=8} (a_k/k^2) sin(2 pi k x + theta_k)."""
    n, seed, A = 128, 9, 0.37
    a, theta = synth.fourier_modes(seed)
    u = synth.burgers_ic(n, seed, A)
    b, c = fourier_coefficients(u)
    assert math.isclose(b[0] / 2.0, 1.0, rel_tol=0, abs_tol=1e-12)
    for k in range(1, 9):
        amp = 0.1 * a[k - 1] / k**2
        # sin(2 pi k x + th) = sin th cos(2 pi k x) + cos th sin(2 pi k x)
        assert abs(b[k] - amp * np.sin(theta[k - 1])) <= 1e-12
        assert abs(c[k] - amp * np.cos(theta[k - 1]) - (A if k == 1 else 0.0)) <= 1e-12
    assert np.max(np.abs(b[9:])) <= 1e-12 and np.max(np.abs(c[9:])) <= 1e-12


def test_burgers_ic_amplitude_direction_and_positivity():
    n = 256
    d = synth.burgers_ic(n, 4, 0.6) - synth.burgers_ic(n, 4, 0.5)
    assert np.allclose(d, 0.1 * synth.burgers_ic_amplitude_direction(n), atol=1e-14)
    # the workloads' states are positive, so the Godunov flux takes its upwind
    # branch everywhere and the misfit is smooth in nu and A
    for seed in range(6):
        assert synth.burgers_ic(65536, seed).min() > 0.2


def test_burgers_target_is_a_shifted_sine_plus_modes():
    n, seed = 64, 5
    t = synth.burgers_target(n, seed)
    x = synth.cell_centres(n)
    assert np.allclose(t - 0.1 * synth.mode_sum(n, seed), 1.0 + 0.5 * np.sin(2 * np.pi * (x - 0.05)),
                       atol=1e-14)


def test_fourier_modes_are_seeded_and_ordered():
    a1, t1 = synth.fourier_modes(3)
    a2, t2 = synth.fourier_modes(3)
    assert np.array_equal(a1, a2) and np.array_equal(t1, t2)
    rng = np.random.default_rng(3)
    assert np.array_equal(a1, rng.standard_normal(8))
    assert np.array_equal(t1, rng.uniform(0.0, 2 * np.pi, 8))


def test_sod_initial_state():
    n, seed, g = 1000, 2, 1.4
    rho, u, p = synth.sod_primitive_ic(n, seed)
    left = synth.cell_centres(n) < 0.5
    assert np.all(u == 0.0)
    for arr, lv, rv in ((rho, 1.0, 0.125), (p, 1.0, 0.1)):
        rel = arr / np.where(left, lv, rv) - 1.0
        assert 0.005 < np.std(rel) < 0.015 and np.max(np.abs(rel)) < 0.06
    U = synth.sod_conserved_ic(n, seed, g)
    assert np.array_equal(U[:n], rho) and np.all(U[n:2 * n] == 0.0)
    assert np.allclose(U[2 * n:], p / (g - 1.0), rtol=1e-15)
    rho0, _, p0 = synth.sod_primitive_ic(n, None)
    assert np.array_equal(rho0, np.where(left, 1.0, 0.125)) and np.array_equal(p0, np.where(left, 1.0, 0.1))


def test_sod_time_step_reaches_t_end_within_cfl():
    for n in (256, 8192):
        dt, steps = synth.sod_dt(n, 2)
        assert math.isclose(dt * steps, 0.2, rel_tol=1e-14)
        rho, u, p = synth.sod_primitive_ic(n, 2)
        smax = float(np.max(np.abs(u) + np.sqrt(1.4 * p / rho)))
        assert dt * smax * n <= 0.4 * (1 + 1e-12)
        assert (steps - 1) * (0.4 / (smax * n)) < 0.2
    cfg = synth.config_sod()
    assert cfg.w_init + cfg.n_online == synth.sod_dt(8192, 2)[1]


def test_batch_recipe():
    cfgs = synth.config_batch(256)
    assert len(cfgs) == 256 and len({c.seed for c in cfgs}) == 256
    ns = np.array([c.n_cells for c in cfgs])
    assert ns.min() >= 2048 and ns.max() <= 65536
    # log-uniform: each of four equal bins of ln N holds about a quarter
    edges = np.linspace(np.log(2048), np.log(65536), 5)
    counts = np.histogram(np.log(ns), bins=edges)[0]
    assert counts.min() >= 40
    assert all(8 <= c.r <= 48 for c in cfgs) and len({c.r for c in cfgs}) >= 30
    assert {c.z for c in cfgs} == {5, 10, 20}
    assert all(c.lam == synth.LAMBDA_BY_Z[c.z] for c in cfgs)
    assert all(1e-3 <= c.nu <= 1e-2 for c in cfgs)
    assert all(c.precision == 1 and c.n_s == 0 and c.w_init == 100 and c.dt == 1e-4 for c in cfgs)
    # an instance's draw depends only on its seed
    assert synth.config_batch(3)[2].to_dict() == cfgs[2].to_dict()


def test_named_workloads():
    c = synth.config_burgers_small()
    assert (c.n_cells, c.r, c.z, c.lam, c.n_online, c.nu) == (512, 10, 10, 0.1, 2000, 0.01)
    c = synth.config_burgers_hyper(1)
    assert (c.n_cells, c.r, c.n_s, c.z, c.lam, c.n_online, c.precision) == (16384, 32, 96, 5, 0.5, 20000, 1)
    c = synth.config_adjoint()
    assert (c.n_cells, c.r, c.nu, c.z, c.lam, c.n_online, c.n_s) == (65536, 64, 5e-3, 10, 0.1, 1000, 0)
    c = synth.config_sod()
    assert (c.n_cells, c.n_var, c.r, c.z, c.n) == (8192, 3, 40, 10, 24576)


def test_random_orthonormal():
    Q = synth.random_orthonormal(50, 7, 1)
    assert np.allclose(Q.T @ Q, np.eye(7), atol=1e-14)
    assert np.array_equal(Q, synth.random_orthonormal(50, 7, 1))
