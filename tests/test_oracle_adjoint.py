"""Pins of the gradient oracle (terminal misfit of the adaptive Burgers ROM
with respect to the viscosity and the initial-condition amplitude; no GPU).

What fixes the gradient independently of the oracle's own formulas:

* central finite differences of the forward oracle (``rom.AdaptiveROM``) with
  Newton converged to 1e-14, for the whole chain and for every piece (the
  BE root, the thin and square SVD, the iSVD update along a curve of
  orthonormal bases);
* the closed-form eigenvalues of the periodic second difference for df/dnu;
* dot-product identities <wbar, T v> = <T^T wbar, v> between the tangent and
  adjoint of every piece and of every online step, on random vectors;
* equality of the reverse sweep with forward mode, and its independence of the
  checkpoint interval (bit for bit).
"""
import json
import os

import numpy as np
import pytest

import synth
from oracle import adjoint as adj
from oracle import fv, rom


def cfg_small(n=64, r=3, w=20, z=5, lam=0.5, nu=5e-3):
    return synth.RomConfig(problem=synth.BURGERS, n_cells=n, r=r, n_s=0, w_init=w, z=z, dt=1e-4,
                           nu=nu, lam=lam, newton_tol=1e-14, newton_max=40, seed=4)


def central_fd(cfg, n_steps, target, name, rel):
    key = "nu" if name == "nu" else "amplitude"
    base = getattr(cfg, key)
    h = rel * base
    Jp, _ = adj.misfit(adj.at(cfg, **{key: base + h}), n_steps, target)
    Jm, _ = adj.misfit(adj.at(cfg, **{key: base - h}), n_steps, target)
    return (Jp - Jm) / (2.0 * h)


def stiefel_curve(Phi, dPhi):
    """An orthonormal basis curve through Phi with velocity dPhi (polar factor
    of Phi + t dPhi; dPhi tangent at Phi)."""
    def at(t):
        U, _, Vt = np.linalg.svd(Phi + t * dPhi, full_matrices=False)
        return U @ Vt
    return at


def random_stiefel_tangent(Phi, rng):
    S = rng.standard_normal(Phi.shape)
    A = Phi.T @ S
    return Phi @ (0.5 * (A - A.T)) + (S - Phi @ (Phi.T @ S))


# ------------------------------------------------------------- FOM pieces ---

@pytest.mark.parametrize("k", [1, 3, 17])
def test_f_nu_is_the_periodic_second_difference(k):
    """df/dnu on a Fourier mode: -(2 N sin(pi k / N))^2 times the mode."""
    n = 64
    x = synth.cell_centres(n)
    u = np.sin(2 * np.pi * k * x)
    lam_k = -(2 * n * np.sin(np.pi * k / n)) ** 2
    assert np.allclose(adj.burgers_f_nu(u), lam_k * u, rtol=0, atol=1e-9 * abs(lam_k))
    # and f is affine in nu with that slope
    v = 1.0 + 0.3 * u
    assert np.allclose(fv.burgers_f(v, 0.02) - fv.burgers_f(v, 0.01), 0.01 * adj.burgers_f_nu(v),
                       rtol=1e-10, atol=1e-10)


def test_be_root_derivatives_match_finite_differences():
    n, h, nu = 96, 5e-4, 5e-3
    rng = np.random.default_rng(0)
    y0 = synth.burgers_ic(n, 7)
    dy0 = rng.standard_normal(n)
    y1 = fv.be_step(y0, h, 0, nu, 1.4, 1e-15, 40)
    for dnu in (0.0, 1.0):
        dir_y = dy0 if dnu == 0.0 else np.zeros(n)
        tan = adj.be_tangent(y1, dir_y, h, nu, dnu)
        e = 1e-3 * nu if dnu else 1e-6          # steps in nu and in y
        yp = fv.be_step(y0 + e * dir_y, h, 0, nu + e * dnu, 1.4, 1e-15, 40)
        ym = fv.be_step(y0 - e * dir_y, h, 0, nu - e * dnu, 1.4, 1e-15, 40)
        fd = (yp - ym) / (2 * e)
        assert np.max(np.abs(fd - tan)) <= 1e-7 * np.max(np.abs(tan)), dnu
    ybar = rng.standard_normal(n)
    w, nubar = adj.be_adjoint(y1, ybar, h, nu)
    for dnu, dir_y in ((0.0, dy0), (1.0, np.zeros(n))):
        lhs = ybar @ adj.be_tangent(y1, dir_y, h, nu, dnu)
        assert abs(lhs - (w @ dir_y + nubar * dnu)) <= 1e-12 * max(1.0, abs(lhs))


# ------------------------------------------------------------------- SVD ---

def _aligned(U_ref, U):
    return U * np.sign(np.sum(U * U_ref, axis=0))[None, :]


@pytest.mark.parametrize("shape,cols", [((30, 8), 5), ((30, 8), 8), ((7, 7), 6), ((7, 7), 7)])
def test_svd_derivative_matches_finite_differences(shape, cols):
    rng = np.random.default_rng(1)
    X = rng.standard_normal(shape) * (1.6 ** -np.arange(shape[1]))[None, :]
    dX = rng.standard_normal(shape)
    U, s, Vt = np.linalg.svd(X, full_matrices=False)
    dU, ds = adj.svd_tangent(U, s, Vt, dX, cols)
    e = 1e-6
    Up, sp_, _ = np.linalg.svd(X + e * dX, full_matrices=False)
    Um, sm, _ = np.linalg.svd(X - e * dX, full_matrices=False)
    fdU = (_aligned(U[:, :cols], Up[:, :cols]) - _aligned(U[:, :cols], Um[:, :cols])) / (2 * e)
    assert np.max(np.abs(fdU - dU)) <= 1e-7 * np.max(np.abs(dU))
    assert np.max(np.abs((sp_[:cols] - sm[:cols]) / (2 * e) - ds)) <= 1e-7 * np.max(np.abs(ds))


@pytest.mark.parametrize("shape,cols", [((30, 8), 5), ((7, 7), 6), ((9, 9), 9)])
def test_svd_adjoint_dot_product(shape, cols):
    rng = np.random.default_rng(2)
    X = rng.standard_normal(shape)
    U, s, Vt = np.linalg.svd(X, full_matrices=False)
    dX = rng.standard_normal(shape)
    dU, ds = adj.svd_tangent(U, s, Vt, dX, cols)
    Ubar, sbar = rng.standard_normal(dU.shape), rng.standard_normal(cols)
    Xbar = adj.svd_adjoint(U, s, Vt, Ubar, sbar, cols)
    lhs = np.sum(Ubar * dU) + sbar @ ds
    assert abs(lhs - np.sum(Xbar * dX)) <= 1e-12 * max(1.0, abs(lhs))


# ------------------------------------------------------------------ iSVD ---

def _isvd_case(empty=False, null_cols=0, seed=3):
    n, r = 40, 5
    rng = np.random.default_rng(seed)
    Phi = synth.random_orthonormal(n, r, seed)
    sig = np.array([5.0, 3.0, 2.0, 1.0, 0.5])
    if null_cols:
        Phi[:, r - null_cols:] = 0.0
        sig[r - null_cols:] = 0.0
    yhat = rng.standard_normal(n)
    if empty:
        yhat = Phi @ rng.standard_normal(r)
    return Phi, sig, yhat, rng


@pytest.mark.parametrize("lam", [1.0, 0.5, 0.1])
def test_isvd_derivative_matches_finite_differences(lam):
    """Along a curve of orthonormal bases, singular values and snapshot."""
    Phi, sig, yhat, rng = _isvd_case()
    r = Phi.shape[1]
    dPhi = random_stiefel_tangent(Phi, rng)
    dsig, dy = rng.standard_normal(r), rng.standard_normal(Phi.shape[0])
    iv = adj._isvd(Phi, sig, yhat, lam, r)
    assert np.array_equal(iv.Phi_new, rom.isvd_update(Phi, sig, yhat, lam, r)[0])
    dPn, dsn = adj._isvd_tangent(iv, dPhi, dsig, dy, lam)
    curve = stiefel_curve(Phi, dPhi)
    e = 1e-6
    Pp, spp = rom.isvd_update(curve(e), sig + e * dsig, yhat + e * dy, lam, r)
    Pm, smm = rom.isvd_update(curve(-e), sig - e * dsig, yhat - e * dy, lam, r)
    assert np.max(np.abs((Pp - Pm) / (2 * e) - dPn)) <= 1e-7 * np.max(np.abs(dPn))
    assert np.max(np.abs((spp - smm) / (2 * e) - dsn)) <= 1e-7 * np.max(np.abs(dsn))


@pytest.mark.parametrize("empty,null_cols", [(False, 0), (True, 0), (False, 2)])
def test_isvd_adjoint_dot_product(empty, null_cols):
    Phi, sig, yhat, rng = _isvd_case(empty, null_cols)
    r = Phi.shape[1]
    live = r - null_cols
    dPhi = np.zeros_like(Phi)
    dPhi[:, :live] = random_stiefel_tangent(Phi[:, :live], rng)
    dsig = np.r_[rng.standard_normal(live), np.zeros(null_cols)]
    dy = rng.standard_normal(Phi.shape[0])
    iv = adj._isvd(Phi, sig, yhat, 0.5, r)
    assert iv.empty == empty
    dPn, dsn = adj._isvd_tangent(iv, dPhi, dsig, dy, 0.5)
    Pb, sb = rng.standard_normal(dPn.shape), rng.standard_normal(dsn.shape)
    Phib, sigb, yb = adj._isvd_adjoint(iv, Pb, sb, 0.5)
    lhs = np.sum(Pb * dPn) + sb @ dsn
    rhs = np.sum(Phib * dPhi) + sigb @ dsig + yb @ dy
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


# ------------------------------------------------------- online steps ---

def _recorded_run(cfg, n_steps):
    q0 = synth.initial_state(cfg)
    off = adj._offline(cfg, q0)
    st = adj._State(off.Phi.copy(), off.sigma.copy(), off.a.copy(), off.y_corr.copy(), cfg.w_init)
    return off, [adj._online_step(cfg, st, off.q_ref, off.d) for _ in range(n_steps)]


def test_step_adjoint_dot_product_at_every_step():
    """Each online step (with and without an event, with null basis columns)."""
    cfg = cfg_small(n=96, r=6, w=20, z=5, lam=0.5)
    off, recs = _recorded_run(cfg, 30)
    rng = np.random.default_rng(4)
    n, r = cfg.n_cells, cfg.r
    seen_null = False
    for rec in recs:
        live = rom.numerical_rank(rec.Phi)
        seen_null |= live < r
        dPhi = np.zeros_like(rec.Phi)
        dPhi[:, :live] = random_stiefel_tangent(rec.Phi[:, :live], rng)
        T = dict(Phi=dPhi, sigma=np.r_[rng.standard_normal(live), np.zeros(r - live)],
                 a=np.r_[rng.standard_normal(live), np.zeros(r - live)], y=rng.standard_normal(n))
        T0 = {k: v.copy() for k, v in T.items()}
        dq_ref, dd, dnu = rng.standard_normal(n), rng.standard_normal(), rng.standard_normal()
        dqt = adj._step_tangent(cfg, rec, off.q_ref, off.d, T, dq_ref, dd, dnu)
        B = {k: rng.standard_normal(np.shape(v)) for k, v in T.items()}
        qtb = rng.standard_normal(n)
        lhs = sum(np.sum(B[k] * T[k]) for k in B) + qtb @ dqt
        Ab = {k: v.copy() for k, v in B.items()}
        Ab.update(q_ref=np.zeros(n), d=0.0, nu=0.0)
        adj._step_adjoint(cfg, rec, off.q_ref, off.d, Ab, qtb)
        rhs = (sum(np.sum(Ab[k] * T0[k]) for k in ("Phi", "sigma", "a", "y"))
               + Ab["q_ref"] @ dq_ref + Ab["d"] * dd + Ab["nu"] * dnu)
        assert abs(lhs - rhs) <= 1e-11 * max(1.0, abs(lhs)), rec.event is not None
    assert seen_null


def test_offline_adjoint_dot_product():
    cfg = cfg_small(n=96, r=6, w=20)
    off, _ = _recorded_run(cfg, 0)
    rng = np.random.default_rng(5)
    n = cfg.n_cells
    dq0, dnu = rng.standard_normal(n), rng.standard_normal()
    dPhi, dsig, da, dy, dq_ref, dd = adj._offline_tangent(cfg, off, dq0, dnu)
    B = dict(Phi=rng.standard_normal(dPhi.shape), sigma=rng.standard_normal(dsig.shape),
             a=rng.standard_normal(cfg.r), y=rng.standard_normal(n), q_ref=rng.standard_normal(n),
             d=float(rng.standard_normal()), nu=float(rng.standard_normal()))
    lhs = (np.sum(B["Phi"] * dPhi) + B["sigma"] @ dsig + B["a"] @ da + B["y"] @ dy
           + B["q_ref"] @ dq_ref + B["d"] * dd + B["nu"] * dnu)
    q0b, nub = adj._offline_adjoint(cfg, off, {k: np.copy(v) if np.ndim(v) else v
                                              for k, v in B.items()})
    # the POD derivative sums terms of size |q0bar| ~ 1e5 to a result ~ 1e6:
    # rounding leaves ~1e-11 of it; a wrong term leaves O(1)
    assert abs(lhs - (q0b @ dq0 + nub * dnu)) <= 1e-9 * abs(lhs)


def test_basis_tangent_stays_tangent_over_many_events():
    """With lambda = 0.1 an unprojected basis derivative gains a normal part
    about ten times larger at every update; the projected one keeps
    Phi^T dPhi antisymmetric to rounding over 20 events."""
    cfg = cfg_small(n=128, r=3, w=30, z=10, lam=0.1)
    off, recs = _recorded_run(cfg, 200)
    dPhi, dsig, da, dy, dq_ref, dd = adj._offline_tangent(cfg, off, np.zeros(cfg.n_cells), 1.0)
    T = dict(Phi=dPhi, sigma=dsig, a=da, y=dy)
    for rec in recs:
        adj._step_tangent(cfg, rec, off.q_ref, off.d, T, dq_ref, dd, 1.0)
    Phi = recs[-1].event.isvd.Phi_new
    A = Phi.T @ T["Phi"]
    assert np.linalg.norm(A + A.T) <= 1e-13 * np.linalg.norm(T["Phi"])


# --------------------------------------------------------- whole chain ---

CHAIN_CASES = [
    # n, r, w_init, z, lambda, online steps
    (64, 3, 20, 5, 0.5, 40),
    (128, 10, 30, 10, 0.1, 100),     # null basis columns, the gradient workload's z and lambda
    (256, 8, 40, 20, 1e-7, 200),
]


@pytest.mark.parametrize("case", CHAIN_CASES)
def test_gradient_matches_central_differences(case):
    """Forward mode against central differences (h = 1e-4 relative) of the
    forward oracle, both parameters."""
    n, r, w, z, lam, steps = case
    cfg = cfg_small(n, r, w, z, lam)
    target = synth.burgers_target(n, cfg.seed + 1)
    J, g = adj.tangent_gradient(cfg, steps, target)
    J_rom, _ = adj.misfit(cfg, steps, target)
    assert J == J_rom                       # the recorded primal is the oracle's own
    for name in ("nu", "A"):
        fd = central_fd(cfg, steps, target, name, 1e-4)
        assert abs(g[name] - fd) <= 1e-6 * abs(fd), (name, g[name], fd)


@pytest.mark.parametrize("case", CHAIN_CASES)
def test_reverse_sweep_equals_forward_mode(case):
    n, r, w, z, lam, steps = case
    cfg = cfg_small(n, r, w, z, lam)
    target = synth.burgers_target(n, cfg.seed + 1)
    J, g = adj.tangent_gradient(cfg, steps, target)
    J2, g2 = adj.adjoint_gradient(cfg, steps, target, ckpt_every=7)
    assert J2 == J
    for name in ("nu", "A"):
        assert abs(g2[name] - g[name]) <= 1e-9 * abs(g[name]), (name, g[name], g2[name])


def test_checkpoint_interval_does_not_change_the_gradient():
    """Recomputing segments from checkpoints repeats the same arithmetic."""
    cfg = cfg_small(n=96, r=4, w=20, z=5, lam=0.5)
    target = synth.burgers_target(96, cfg.seed + 1)
    ref = adj.adjoint_gradient(cfg, 33, target, ckpt_every=1000)
    for every in (1, 5, 10, 33):
        assert adj.adjoint_gradient(cfg, 33, target, ckpt_every=every) == ref


def test_gradient_of_a_single_step():
    """One online step, no event: forward and reverse agree with central
    differences of the smallest chain (training FOM, POD, one Galerkin step)."""
    cfg = cfg_small(n=64, r=3, w=12, z=5, lam=0.5)
    target = synth.burgers_target(64, cfg.seed + 1)
    J, g = adj.tangent_gradient(cfg, 1, target)
    _, g2 = adj.adjoint_gradient(cfg, 1, target)
    for name in ("nu", "A"):
        fd = central_fd(cfg, 1, target, name, 1e-4)
        assert abs(g[name] - fd) <= 1e-7 * abs(fd)
        assert abs(g2[name] - g[name]) <= 1e-12 * abs(g[name])


def test_rejects_configurations_it_does_not_cover():
    cfg = cfg_small()
    cfg.n_s = 9
    with pytest.raises(ValueError):
        adj.tangent_gradient(cfg, 1, np.zeros(cfg.n_cells))
    with pytest.raises(ValueError):
        adj.adjoint_gradient(cfg_small(), 1, np.zeros(64), ckpt_every=0)


# ------------------------------------------------- stored full-size values ---

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                      "adjoint_burgers_n65536_r64.json")


def test_stored_full_size_gradient_is_current_and_consistent():
    """The stored gradient of the full-size workload (written by
    tests/golden/make_adjoint_golden.py from the oracle alone) belongs to the
    current workload definition, and its two routes and its central
    differences agree."""
    with open(GOLDEN) as f:
        gold = json.load(f)
    cfg = synth.config_adjoint()
    assert cfg.matches(gold["config"])
    assert gold["n_steps"] == cfg.n_online
    for name in ("nu", "A"):
        fwd, rev = gold["grad_forward_mode"][name], gold["grad_reverse_sweep"][name]
        assert abs(fwd - rev) <= 1e-8 * abs(fwd)        # measured 2e-9 and 9e-11
        fd = gold["central_differences"]["value"][name]
        assert abs(fwd - fd) <= 1e-6 * abs(fd)          # measured 1.3e-8 and 1e-9
    assert gold["J"] > 0.0
