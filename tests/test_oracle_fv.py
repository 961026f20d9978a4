"""Pins of the oracle's full-order operators against closed forms, invariants,
finite differences and hand expansion (no GPU)."""
import math

import numpy as np
import pytest

import synth
from oracle import fv, riemann


def fd_jacobian(fun, q, eps=1e-7):
    J = np.zeros((q.size, q.size))
    for k in range(q.size):
        e = np.zeros(q.size)
        e[k] = eps
        J[:, k] = (fun(q + e) - fun(q - e)) / (2 * eps)
    return J


# ---------------------------------------------------------------- Burgers ---

def test_burgers_constant_state_is_steady():
    for c in (-1.3, 0.0, 0.7):
        assert np.all(fv.burgers_f(np.full(16, c), 0.01) == 0.0)


def test_burgers_hand_expansion_n4():
    """N=4, u>0: upwind flux u_{i-1}^2/2 - u_i^2/2 over dx plus the centred
    second difference, written out cell by cell."""
    u = np.array([1.0, 1.5, 0.75, 1.25])
    nu = 0.03
    n, dx = 4, 0.25
    exp = np.empty(4)
    for i in range(4):
        um, up = u[(i - 1) % n], u[(i + 1) % n]
        exp[i] = -(0.5 * u[i] ** 2 - 0.5 * um**2) / dx + nu * (up - 2 * u[i] + um) / dx**2
    assert np.allclose(fv.burgers_f(u, nu), exp, rtol=1e-15, atol=1e-13)


def test_godunov_flux_cases():
    # right-moving, left-moving, transonic rarefaction (flux 0), shock (max of both)
    assert fv.godunov_flux(2.0, 1.0) == 2.0
    assert fv.godunov_flux(-1.0, -3.0) == 4.5
    assert fv.godunov_flux(-1.0, 2.0) == 0.0
    assert fv.godunov_flux(1.0, -3.0) == 4.5
    assert fv.godunov_flux(3.0, -1.0) == 4.5


def test_burgers_mass_conservation():
    u = synth.burgers_ic(256, 5)
    f = fv.burgers_f(u, 0.01)
    assert abs(f.sum()) <= 1e-12 * np.abs(f).sum()
    J = fv.burgers_jac(u, 0.01).toarray()
    # columns of J_f sum to zero: d(sum f)/du_j = 0
    assert np.max(np.abs(J.sum(axis=0))) <= 1e-9 * np.max(np.abs(J))


@pytest.mark.parametrize("seed", [0, 3])
def test_burgers_jacobian_matches_finite_differences(seed):
    u = synth.burgers_ic(32, seed)
    u[5] = -0.4     # exercise both flux branches
    u[6] = -0.9
    J = fv.burgers_jac(u, 0.02).toarray()
    Jfd = fd_jacobian(lambda v: fv.burgers_f(v, 0.02), u)
    assert np.max(np.abs(J - Jfd)) <= 1e-7 * np.max(np.abs(J))


def test_be_step_conserves_mass_and_solves_residual():
    u0 = synth.burgers_ic(128, 1)
    h = 5e-4
    u1, iters = fv.be_step(u0, h, 0, 0.01, return_iters=True)
    assert iters <= 6
    r = u1 - u0 - h * fv.burgers_f(u1, 0.01)
    assert np.max(np.abs(r)) <= 1e-12
    assert abs(u1.sum() - u0.sum()) <= 1e-12 * abs(u0.sum())


def _burgers_fom(u, dt, steps, nu):
    for _ in range(steps):
        u = fv.be_step(u, dt, 0, nu)
    return u


def test_burgers_linearised_closed_form_first_order():
    """u = 1 + eps sin(2 pi x): to first order in eps the solution is
    1 + eps exp(-4 pi^2 nu t) sin(2 pi (x - t)). The scheme is first order in
    dx and dt, so halving both must roughly halve the error."""
    eps, nu, T = 1e-4, 0.02, 0.1
    errs = []
    for n in (64, 128, 256):
        x = synth.cell_centres(n)
        steps = n // 2
        dt = T / steps
        u = _burgers_fom(1.0 + eps * np.sin(2 * np.pi * x), dt, steps, nu)
        exact = 1.0 + eps * math.exp(-4 * math.pi**2 * nu * T) * np.sin(2 * np.pi * (x - T))
        errs.append(np.max(np.abs(u - exact)) / eps)
    assert errs[0] / errs[1] > 1.7 and errs[1] / errs[2] > 1.7
    assert errs[2] < 0.05


def cole_hopf(x, t, nu, amp=0.5, m=4096):
    """Exact u(x,t) for u0 = 1 + amp sin(2 pi x), nu > 0, periodic: Galilean
    shift w = u - 1 in the frame xi = x - t, w = -2 nu phi_xi / phi with
    phi solving the heat equation from phi0 = exp(-amp (1 - cos 2 pi xi)/(4 pi nu))."""
    xi = np.arange(m) / m
    phi0 = np.exp(-amp * (1 - np.cos(2 * np.pi * xi)) / (4 * np.pi * nu))
    k = np.fft.fftfreq(m, d=1.0 / m)
    ph = np.fft.fft(phi0) * np.exp(-nu * (2 * np.pi * k) ** 2 * t)
    # evaluate phi and phi_xi at xi = x - t by the Fourier series
    shift = np.exp(2j * np.pi * np.outer(x - t, k))
    phi = (shift @ ph).real / m
    dphi = (shift @ (2j * np.pi * k * ph)).real / m
    return 1.0 - 2 * nu * dphi / phi


def test_burgers_cole_hopf_convergence():
    nu, T = 0.05, 0.1
    errs = []
    for n in (64, 128, 256):
        x = synth.cell_centres(n)
        steps = n // 2
        u = _burgers_fom(1.0 + 0.5 * np.sin(2 * np.pi * x), T / steps, steps, nu)
        errs.append(np.max(np.abs(u - cole_hopf(x, T, nu))))
    assert errs[0] / errs[1] > 1.6 and errs[1] / errs[2] > 1.6
    assert errs[2] < 0.02


# ------------------------------------------------------------------ Euler ---

def test_euler_constant_state_is_steady():
    n = 16
    U = np.concatenate([np.full(n, 0.8), np.full(n, 0.3), np.full(n, 2.5)])
    assert np.max(np.abs(fv.euler_f(U, 1.4))) <= 1e-13


def test_euler_jacobian_matches_finite_differences():
    n = 16
    rho, _, p = synth.sod_primitive_ic(n, 3)
    u = 0.3 * np.sin(np.arange(n) + 0.5)          # avoid the kink of |u| at u = 0
    U = np.concatenate([rho, rho * u, p / 0.4 + 0.5 * rho * u * u])
    J = fv.euler_jac(U, 1.4).toarray()
    Jfd = fd_jacobian(lambda v: fv.euler_f(v, 1.4), U)
    assert np.max(np.abs(J - Jfd)) <= 1e-7 * np.max(np.abs(J))


def test_euler_conserves_mass_and_energy():
    n = 128
    U = synth.sod_conserved_ic(n, None)
    h = 0.4 / n / 1.2
    U1 = U
    for _ in range(10):
        U1 = fv.be_step(U1, h, 1, gamma=1.4)
    for v in (0, 2):
        s0, s1 = U[v * n:(v + 1) * n].sum(), U1[v * n:(v + 1) * n].sum()
        assert abs(s1 - s0) <= 1e-12 * abs(s0)


def test_riemann_star_state_textbook_sod():
    """Standard Sod problem: p* = 0.30313, u* = 0.92745 (textbook values)."""
    ps, us = riemann.star_state((1.0, 0.0, 1.0), (0.125, 0.0, 0.1))
    assert abs(ps - 0.30313) < 5e-6 and abs(us - 0.92745) < 5e-6


def test_riemann_rankine_hugoniot_and_isentrope():
    g = 1.4
    left, right = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)
    ps, us = riemann.star_state(left, right, g)
    # shock speed from the sampled jump: mass flux is continuous across it
    xi = np.linspace(1.5, 2.0, 20001)
    rho, u, p = riemann.sample(left, right, xi, g)
    k = int(np.argmax(rho < 0.2))
    S = 0.5 * (xi[k - 1] + xi[k])
    rho_s = rho[k - 1]
    assert abs(rho_s * (us - S) - 0.125 * (0.0 - S)) < 2e-4
    # rarefaction fan: p / rho^gamma constant
    xi = np.linspace(-1.1, -0.1, 50)
    rho, u, p = riemann.sample(left, right, xi, g)
    fan = (xi > -math.sqrt(g)) & (xi < us - math.sqrt(g * ps / rho.max()))
    ent = p / rho**g
    assert np.max(np.abs(ent - 1.0)) < 1e-12


def test_sod_fom_converges_to_exact_riemann_solution():
    """BE + Rusanov (first order, diffusive): the L1 error of rho against the
    exact solution at t = 0.1 decreases with resolution."""
    g, T = 1.4, 0.1
    errs = []
    for n in (100, 200, 400):
        U = synth.sod_conserved_ic(n, None)
        steps = int(math.ceil(T / (0.4 / n / math.sqrt(g))))
        h = T / steps
        for _ in range(steps):
            U = fv.be_step(U, h, 1, gamma=g)
        x = synth.cell_centres(n)
        rho_ex, _, _ = riemann.sample((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), (x - 0.5) / T, g)
        errs.append(np.mean(np.abs(U[:n] - rho_ex)))
    assert errs[0] > errs[1] > errs[2]
    assert errs[0] / errs[2] > 1.8
    assert errs[2] < 0.03
