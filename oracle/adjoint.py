"""Gradient of the adaptive ROM's terminal misfit (oracle).

Test infrastructure only; see the package docstring.

The paper states no adjoint. This module differentiates the method exactly as
``oracle.rom`` and ``oracle.fv`` state it for periodic Burgers (Sec. 5.1):
training FOM (Eq. fom_lmm with backward Euler), preprocessing (Sec. 3.1),
POD, the backward-Euler Galerkin steps (Eq. galerkin_continuous_rom), the
coarse FOM steps and iSVD updates of the adaptation events (Algorithm 1,
Algorithm 2) and the state transfers. The loss is

    J = 1/2 || q~^{n_T} - q_target ||^2,

q~^{n_T} the lifted ROM state returned by the last online step, i.e. computed
before that step's adaptation event, if it has one. The parameters are
the viscosity nu and the amplitude A of the initial condition
u0 = 1 + A sin(2 pi x) + 0.1 S(x), so dq0/dA = sin(2 pi x) and q_ref = q0
moves with A.

Two routes to (dJ/dnu, dJ/dA):

* ``tangent_gradient``   forward mode: every primal quantity carries its
  derivative along one parameter direction, pushed through each step by the
  chain rule. This is the plain definition of the derivative written out, one
  pass per parameter.
* ``adjoint_gradient``   reverse mode: one forward pass that keeps checkpoints
  of the full ROM state every ``ckpt_every`` online steps, then a reverse sweep
  over the segments (each recomputed from its checkpoint) that carries the
  adjoint of every state quantity back to the parameters. This is the
  computation a GPU backward pass performs.

Readings (the paper is silent on all of this):

* Discrete decisions are held fixed: the Godunov branch, the sign convention of
  singular vectors, the numerical rank (directions at or below the rank
  tolerance keep a zero derivative), and an empty iSVD residual.
* Every Newton root (training FOM, coarse FOM, reduced step) is differentiated
  by the implicit function theorem at the computed root, not through the
  iterates: for g(x, theta) = 0, dx = -g_x^{-1} g_theta dtheta.
* SVD derivatives take the textbook formulas for distinct singular values:
  with P = U^T dX V, ds_i = P_ii and U^T dU = F o (P S + S P^T),
  F_ij = 1 / (s_j^2 - s_i^2) (i != j), plus (I - U U^T) dX v_j / s_j for a thin
  SVD. Pairs of vanishing singular values contribute nothing (their left
  vectors meet only zero basis columns).
* The iSVD projection p = Phi^T yhat, q = yhat - Phi p is differentiated in
  its exact-arithmetic form; CGS2 computes the same quantities to rounding.
* Every basis derivative is projected onto the tangent space of orthonormal
  bases (``stiefel_project``) where it is formed: exact in exact arithmetic,
  and needed in floating point (see that function).

Only n_var = 1 (Burgers) and plain Galerkin (n_s = 0) are covered, which is
the configuration of the gradient workload (Burgers N = 65536, r = 64).
"""
from __future__ import annotations

import copy

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fv, rom


# ----------------------------------------------------------------------------
# derivatives of the FOM operator
# ----------------------------------------------------------------------------

def burgers_f_nu(u):
    """df/dnu of the Burgers operator: the centred second difference."""
    n = u.shape[0]
    return (np.roll(u, -1) - 2.0 * u + np.roll(u, 1)) * float(n * n)


def _be_matrix(y, h, nu):
    """I - h J_f(y), the backward-Euler Newton matrix at the root y."""
    n = y.shape[0]
    return (sp.identity(n, format="csr") - h * fv.burgers_jac(y, nu)).tocsc()


def be_tangent(y_new, dy_prev, h, nu, dnu):
    """Derivative of the BE root y_new of y - y_prev - h f(y; nu) = 0:
    (I - h J_f) dy = dy_prev + h f_nu dnu."""
    rhs = dy_prev + h * burgers_f_nu(y_new) * dnu
    return spla.spsolve(_be_matrix(y_new, h, nu), rhs)


def be_adjoint(y_new, ybar, h, nu):
    """Adjoint of ``be_tangent``: w = (I - h J_f)^-T ybar gives
    (ybar_prev, nubar) = (w, h w . f_nu)."""
    w = spla.spsolve(_be_matrix(y_new, h, nu).T.tocsc(), ybar)
    return w, h * float(w @ burgers_f_nu(y_new))


# ----------------------------------------------------------------------------
# SVD derivatives
# ----------------------------------------------------------------------------

def _gap_matrix(s):
    """F_ij = 1 / (s_j^2 - s_i^2) off the diagonal; zero on it and wherever
    both singular values vanish."""
    s2 = s * s
    diff = s2[None, :] - s2[:, None]
    F = np.zeros_like(diff)
    nz = diff != 0.0
    F[nz] = 1.0 / diff[nz]
    np.fill_diagonal(F, 0.0)
    return F


def svd_tangent(U, s, Vt, dX, cols):
    """(dU[:, :cols], ds[:cols]) of X = U diag(s) V^T (thin, X has at least as
    many rows as columns), for the leading ``cols`` singular triplets, all with
    s_j > 0."""
    V = Vt.T
    P = U.T @ dX @ V
    F = _gap_matrix(s)
    Om = F[:, :cols] * (P[:, :cols] * s[None, :cols] + s[:, None] * P[:cols, :].T)
    dU = U @ Om
    if U.shape[0] > U.shape[1]:
        W = dX @ V[:, :cols]
        dU = dU + (W - U @ (U.T @ W)) / s[None, :cols]
    return dU, np.diag(P)[:cols].copy()


def svd_adjoint(U, s, Vt, Ubar, sbar, cols):
    """Adjoint of ``svd_tangent``: Xbar with <Xbar, dX> = <Ubar, dU> + <sbar, ds>
    for every dX."""
    V = Vt.T
    F = _gap_matrix(s)
    # dU = U Om + (I - U U^T) dX V_c S_c^-1, Om_ic = F_ic (P_ic s_c + s_i P_ci)
    G = F[:, :cols] * (U.T @ Ubar)                      # d<Ubar, U Om> / d Om
    Pbar = np.zeros((s.shape[0], s.shape[0]))
    Pbar[:, :cols] += G * s[None, :cols]
    Pbar[:cols, :] += (G * s[:, None]).T
    Pbar[np.arange(cols), np.arange(cols)] += sbar
    Xbar = U @ Pbar @ V.T
    if U.shape[0] > U.shape[1]:
        R = Ubar / s[None, :cols]
        R = R - U @ (U.T @ R)
        Xbar = Xbar + R @ V[:, :cols].T
    return Xbar


def stiefel_project(Phi, dPhi):
    """dPhi - Phi sym(Phi^T dPhi): the part of dPhi tangent to the set of
    matrices with orthonormal columns at Phi. The exact derivative of an
    orthonormal basis has no other part, so this changes nothing in exact
    arithmetic; in floating point it removes the rounding-level normal part,
    which the iSVD derivative otherwise amplifies by about 1/lambda per update.
    The projection is self-adjoint, so the reverse sweep applies it too."""
    A = Phi.T @ dPhi
    return dPhi - Phi @ (0.5 * (A + A.T))


def _sign_flips(U_raw, U_signed):
    """+-1 per column: the flips that ``rom.sign_normalise`` applied."""
    out = np.ones(U_raw.shape[1])
    for j in range(U_raw.shape[1]):
        if np.any(U_raw[:, j] != U_signed[:, j]):
            out[j] = -1.0
    return out


def _live_count(s):
    """How many leading columns ``rom.drop_null_directions`` keeps (s is sorted
    in descending order, so the kept columns are a prefix)."""
    if s.shape[0] == 0 or not s[0] > 0:
        return 0
    return int(np.count_nonzero(s > rom.RANK_TOL * s[0]))


# ----------------------------------------------------------------------------
# primal forward pass with the intermediates each derivative needs
# ----------------------------------------------------------------------------

class _Record:
    """Intermediates of one piece of the forward pass."""

    def __init__(self, **kw):
        self.__dict__.update(kw)


def _offline(cfg, q0):
    """Offline stage of Algorithm 1 with its intermediates, equal to what
    ``rom.AdaptiveROM.__init__`` computes."""
    Q = rom.fom_trajectory(q0, cfg.w_init, cfg)
    q_ref, d, Xhat = rom.preprocess(Q, q0, cfg.n_var)
    U, s, Vt = np.linalg.svd(Xhat, full_matrices=False)
    Uk = U[:, :cfg.r]
    Us = rom.sign_normalise(Uk)
    Phi, sigma = rom.drop_null_directions(Us, s[:cfg.r].copy())
    q_last = Q[:, -1]
    a = Phi.T @ (d * (q_last - q_ref))
    y_corr = fv.be_step(q_last, cfg.z * cfg.dt, 0, cfg.nu, cfg.gamma,
                        cfg.newton_tol, cfg.newton_max)
    return _Record(Q=Q, q0=q0, q_ref=q_ref, d=float(d[0]), Xhat=Xhat, U=U, s=s, Vt=Vt,
                   flips=_sign_flips(Uk, Us), live=_live_count(s[:cfg.r]),
                   Phi=Phi, sigma=sigma, a=a, y_corr=y_corr)


def _isvd(Phi, sigma, yhat, lam, r):
    """The iSVD update of ``rom.isvd_update`` with its intermediates."""
    k = Phi.shape[1]
    p, q = rom.project_cgs2(Phi, yhat)
    rho = float(np.linalg.norm(q))
    scale = max(float(np.linalg.norm(yhat)), float(sigma[0]) if k else 0.0)
    empty = rho <= rom.RANK_TOL * scale
    qhat = np.zeros_like(q) if empty else q / rho
    if empty:
        rho = 0.0
    K = np.zeros((k + 1, k + 1))
    K[:k, :k] = lam * np.diag(sigma)
    K[:k, k] = p
    K[k, k] = rho
    Ub, sb, Vbt = np.linalg.svd(K)
    B = np.hstack([Phi, qhat[:, None]])
    Phit = B @ Ub
    keep = min(r, k + 1)
    Ps = rom.sign_normalise(Phit[:, :keep])
    Phi_new, s_new = rom.drop_null_directions(Ps, sb[:keep])
    return _Record(Phi=Phi, sigma=sigma, yhat=yhat, p=p, q=q, rho=rho, empty=empty,
                   qhat=qhat, Ub=Ub, sb=sb, Vbt=Vbt, B=B, keep=keep,
                   flips=_sign_flips(Phit[:, :keep], Ps), live=_live_count(sb[:keep]),
                   Phi_new=Phi_new, sigma_new=s_new)


def _is_event(cfg, n):
    return (n + 1 - cfg.w_init) % cfg.z == 0


class _State:
    """The online state (Phi, sigma, a, y_corr, n) of Algorithm 1."""

    def __init__(self, Phi, sigma, a, y_corr, n):
        self.Phi, self.sigma, self.a, self.y_corr, self.n = Phi, sigma, a, y_corr, n

    def copy(self):
        return _State(self.Phi.copy(), self.sigma.copy(), self.a.copy(), self.y_corr.copy(),
                      self.n)


def _online_step(cfg, st, q_ref, d):
    """One online iteration (reduced step, and the event if one is due) on
    ``st`` in place; returns the record of the step."""
    dv = np.full(q_ref.shape[0], d)
    a_prev = st.a
    a_new, _ = rom.galerkin_step(a_prev, st.Phi, q_ref, dv, cfg)
    qt = rom.lift(a_new, st.Phi, q_ref, dv)
    rec = _Record(Phi=st.Phi, a_prev=a_prev, a_new=a_new, qt=qt, event=None)
    st.a = a_new
    if _is_event(cfg, st.n):
        y_prev = st.y_corr
        y_new = fv.be_step(y_prev, cfg.z * cfg.dt, 0, cfg.nu, cfg.gamma,
                           cfg.newton_tol, cfg.newton_max)
        yhat = dv * (y_new - q_ref)
        iv = _isvd(st.Phi, st.sigma, yhat, cfg.lam, cfg.r)
        a_tr = iv.Phi_new.T @ (dv * (qt - q_ref))
        rec.event = _Record(y_prev=y_prev, y_new=y_new, isvd=iv)
        st.Phi, st.sigma, st.a, st.y_corr = iv.Phi_new, iv.sigma_new, a_tr, y_new
    st.n += 1
    return rec


def _check_cfg(cfg):
    if cfg.problem != 0 or cfg.n_var != 1 or cfg.n_s != 0 or getattr(cfg, "time_scheme", 0) != 0:
        raise ValueError("the gradient oracle covers plain backward-Euler Galerkin Burgers ROMs only")


def misfit(cfg, n_steps, target):
    """J and the final lifted state, by ``rom.AdaptiveROM`` itself."""
    import synth
    m = rom.AdaptiveROM(cfg, synth.initial_state(cfg))
    qt = None
    for _ in range(n_steps):
        qt = m.step()
    return 0.5 * float(np.sum((qt - target) ** 2)), qt


# ----------------------------------------------------------------------------
# forward mode
# ----------------------------------------------------------------------------

def _offline_tangent(cfg, off, dq0, dnu):
    """Tangents (dPhi, dsigma, da, dy_corr, dq_ref, dd) of the offline stage."""
    h = cfg.dt
    dQ = np.empty_like(off.Q)
    dq = dq0
    for k in range(off.Q.shape[1]):
        dq = be_tangent(off.Q[:, k], dq, h, cfg.nu, dnu)
        dQ[:, k] = dq
    dq_ref = dq0
    Xc = off.Q - off.q_ref[:, None]
    dXc = dQ - dq_ref[:, None]
    dd = -(off.d * off.d) * float(np.mean(2.0 * Xc * dXc))
    dXhat = dd * Xc + off.d * dXc
    nl = off.live
    dU, ds = svd_tangent(off.U, off.s, off.Vt, dXhat, nl)
    dPhi = np.zeros_like(off.Phi)
    dPhi[:, :nl] = stiefel_project(off.Phi[:, :nl], dU * off.flips[None, :nl])
    dsig = np.zeros_like(off.sigma)
    dsig[:nl] = ds
    q_last, dq_last = off.Q[:, -1], dQ[:, -1]
    e = q_last - off.q_ref
    da = dPhi.T @ (off.d * e) + off.Phi.T @ (dd * e + off.d * (dq_last - dq_ref))
    dy = be_tangent(off.y_corr, dq_last, cfg.z * h, cfg.nu, dnu)
    return dPhi, dsig, da, dy, dq_ref, dd


def _step_tangent(cfg, rec, q_ref, d, T, dq_ref, dd, dnu):
    """Pushes the tangent T = dict(Phi, sigma, a, y) through one online step;
    returns the tangent of the lifted state q~."""
    Phi, a_new = rec.Phi, rec.a_new
    dPhi = T["Phi"]
    f = fv.burgers_f(rec.qt, cfg.nu)
    Jf = fv.burgers_jac(rec.qt, cfg.nu)
    Pa = Phi @ a_new
    dqt_p = dq_ref + (dPhi @ a_new) / d - Pa * (dd / (d * d))
    rhs = T["a"] + cfg.dt * (dPhi.T @ (d * f) + Phi.T @ (dd * f)
                             + Phi.T @ (d * (Jf @ dqt_p + burgers_f_nu(rec.qt) * dnu)))
    dv = np.full(q_ref.shape[0], d)
    Jr = rom.galerkin_jacobian(a_new, Phi, q_ref, dv, cfg)
    da = np.linalg.solve(Jr, rhs)
    dqt = dqt_p + (Phi @ da) / d
    T["a"] = da
    ev = rec.event
    if ev is not None:
        dy = be_tangent(ev.y_new, T["y"], cfg.z * cfg.dt, cfg.nu, dnu)
        dyhat = dd * (ev.y_new - q_ref) + d * (dy - dq_ref)
        iv = ev.isvd
        dPhi_new, dsig_new = _isvd_tangent(iv, dPhi, T["sigma"], dyhat, cfg.lam)
        e = rec.qt - q_ref
        T["a"] = dPhi_new.T @ (d * e) + iv.Phi_new.T @ (dd * e + d * (dqt - dq_ref))
        T["Phi"], T["sigma"], T["y"] = dPhi_new, dsig_new, dy
    return dqt


def _isvd_tangent(iv, dPhi, dsig, dyhat, lam):
    """(dPhi_new, dsigma_new) of one iSVD update."""
    Phi, yhat = iv.Phi, iv.yhat
    k = Phi.shape[1]
    dp = dPhi.T @ yhat + Phi.T @ dyhat
    if iv.empty:
        dqhat = np.zeros_like(yhat)
        drho = 0.0
    else:
        dq = dyhat - dPhi @ iv.p - Phi @ dp
        drho = float(iv.qhat @ dq)
        dqhat = (dq - iv.qhat * drho) / iv.rho
    dK = np.zeros((k + 1, k + 1))
    dK[:k, :k] = lam * np.diag(dsig)
    dK[:k, k] = dp
    dK[k, k] = drho
    nl = iv.live
    dUb, dsb = svd_tangent(iv.Ub, iv.sb, iv.Vbt, dK, nl)
    dB = np.hstack([dPhi, dqhat[:, None]])
    dPhi_new = np.zeros((Phi.shape[0], iv.keep))
    dPhi_new[:, :nl] = stiefel_project(iv.Phi_new[:, :nl],
                                       (dB @ iv.Ub[:, :nl] + iv.B @ dUb) * iv.flips[None, :nl])
    dsig_new = np.zeros(iv.keep)
    dsig_new[:nl] = dsb
    return dPhi_new, dsig_new


def tangent_gradient(cfg, n_steps, target, directions=("nu", "A")):
    """(J, {name: dJ/dname}) by forward mode, one tangent pass per parameter.

    ``cfg.amplitude`` and ``cfg.nu`` are the point of differentiation.
    """
    import synth
    _check_cfg(cfg)
    q0 = synth.initial_state(cfg)
    off = _offline(cfg, q0)
    st = _State(off.Phi.copy(), off.sigma.copy(), off.a.copy(), off.y_corr.copy(), cfg.w_init)
    recs = [_online_step(cfg, st, off.q_ref, off.d) for _ in range(n_steps)]
    qT = recs[-1].qt
    J = 0.5 * float(np.sum((qT - target) ** 2))
    out = {}
    for name in directions:
        if name == "nu":
            dq0, dnu = np.zeros_like(q0), 1.0
        elif name == "A":
            dq0, dnu = synth.burgers_ic_amplitude_direction(cfg.n_cells), 0.0
        else:
            raise ValueError(name)
        dPhi, dsig, da, dy, dq_ref, dd = _offline_tangent(cfg, off, dq0, dnu)
        T = dict(Phi=dPhi, sigma=dsig, a=da, y=dy)
        dqt = None
        for rec in recs:
            dqt = _step_tangent(cfg, rec, off.q_ref, off.d, T, dq_ref, dd, dnu)
        out[name] = float((qT - target) @ dqt)
    return J, out


# ----------------------------------------------------------------------------
# reverse mode
# ----------------------------------------------------------------------------

def _isvd_adjoint(iv, Phi_new_bar, sig_new_bar, lam):
    """Adjoint of ``_isvd_tangent``: (Phibar, sigbar, yhatbar)."""
    Phi, yhat = iv.Phi, iv.yhat
    k = Phi.shape[1]
    nl = iv.live
    Pbar = stiefel_project(iv.Phi_new[:, :nl], Phi_new_bar[:, :nl]) * iv.flips[None, :nl]
    # dPhit = dB Ub_c + B dUb
    Bbar = Pbar @ iv.Ub[:, :nl].T
    Ubbar = iv.B.T @ Pbar
    Kbar = svd_adjoint(iv.Ub, iv.sb, iv.Vbt, Ubbar, sig_new_bar[:nl], nl)
    Phibar = Bbar[:, :k].copy()
    qhatbar = Bbar[:, k]
    sigbar = lam * np.diag(Kbar[:k, :k]).copy()
    pbar = Kbar[:k, k].copy()
    rhobar = Kbar[k, k]
    yhatbar = np.zeros_like(yhat)
    if not iv.empty:
        # dqhat = (dq - qhat drho)/rho, drho = qhat . dq
        qbar = qhatbar / iv.rho
        rhobar_tot = rhobar - float(iv.qhat @ qhatbar) / iv.rho
        qbar = qbar + iv.qhat * rhobar_tot
        # dq = dyhat - dPhi p - Phi dp
        yhatbar += qbar
        Phibar -= np.outer(qbar, iv.p)
        pbar = pbar - Phi.T @ qbar
    # dp = dPhi^T yhat + Phi^T dyhat
    Phibar += np.outer(yhat, pbar)
    yhatbar += Phi @ pbar
    return Phibar, sigbar, yhatbar


def _step_adjoint(cfg, rec, q_ref, d, Abar, qtbar):
    """Adjoint of ``_step_tangent``. ``Abar`` holds the adjoints of the state
    after the step (Phi, sigma, a, y) and of (q_ref, d, nu); ``qtbar`` is the
    adjoint arriving at this step's lifted state from the loss. Updates Abar
    to the adjoints of the state before the step."""
    Phi, a_new = rec.Phi, rec.a_new
    ev = rec.event
    qtbar = qtbar.copy()
    if ev is not None:
        iv = ev.isvd
        e = rec.qt - q_ref
        abar = Abar["a"]
        # a_tr = Phi_new^T (d e)
        Phinew_bar = Abar["Phi"] + np.outer(d * e, abar)
        we = iv.Phi_new @ abar
        Abar["d"] += float(we @ e)
        qtbar += d * we
        Abar["q_ref"] -= d * we
        Phibar, sigbar, yhatbar = _isvd_adjoint(iv, Phinew_bar, Abar["sigma"], cfg.lam)
        # yhat = d (y_new - q_ref)
        ybar_new = Abar["y"] + d * yhatbar
        Abar["d"] += float(yhatbar @ (ev.y_new - q_ref))
        Abar["q_ref"] -= d * yhatbar
        ybar_prev, nubar = be_adjoint(ev.y_new, ybar_new, cfg.z * cfg.dt, cfg.nu)
        Abar["nu"] += nubar
        Abar["Phi"], Abar["sigma"], Abar["y"] = Phibar, sigbar, ybar_prev
        Abar["a"] = np.zeros_like(abar)
    # dqt = dqt_p + Phi da / d, da = Jr^-1 rhs
    f = fv.burgers_f(rec.qt, cfg.nu)
    Jf = fv.burgers_jac(rec.qt, cfg.nu)
    dv = np.full(q_ref.shape[0], d)
    Jr = rom.galerkin_jacobian(a_new, Phi, q_ref, dv, cfg)
    dabar = Abar["a"] + Phi.T @ qtbar / d
    w = np.linalg.solve(Jr.T, dabar)                 # rhs adjoint
    Abar["a"] = w.copy()                             # rhs = da_prev + ...
    # rhs += dt [dPhi^T (d f) + Phi^T (dd f) + Phi^T (d (Jf dqt_p + f_nu dnu))]
    Abar["Phi"] += cfg.dt * np.outer(d * f, w)
    Pw = Phi @ w
    Abar["d"] += cfg.dt * float(Pw @ f)
    g = cfg.dt * d * Pw                               # adjoint of (Jf dqt_p + f_nu dnu)
    Abar["nu"] += float(g @ burgers_f_nu(rec.qt))
    dqtp_bar = qtbar + Jf.T @ g
    # dqt_p = dq_ref + dPhi a / d - Phi a dd / d^2 (plus the Phi da / d term above)
    Abar["q_ref"] += dqtp_bar
    Abar["Phi"] += np.outer(dqtp_bar / d, a_new)
    Abar["d"] -= float(dqtp_bar @ (Phi @ a_new)) / (d * d)


def _offline_adjoint(cfg, off, Abar):
    """Adjoint of ``_offline_tangent``: (q0bar, nubar) from the adjoints of the
    online state at its start and of (q_ref, d, nu)."""
    h = cfg.dt
    nubar = Abar["nu"]
    q_last = off.Q[:, -1]
    e = q_last - off.q_ref
    # y_corr = BE(q_last, z h)
    qlast_bar, nb = be_adjoint(off.y_corr, Abar["y"], cfg.z * h, cfg.nu)
    nubar += nb
    # a = Phi^T (d e)
    abar = Abar["a"]
    Phibar = Abar["Phi"] + np.outer(off.d * e, abar)
    we = off.Phi @ abar
    dbar = Abar["d"] + float(we @ e)
    qlast_bar = qlast_bar + off.d * we
    qref_bar = Abar["q_ref"] - off.d * we
    # Phi, sigma from the SVD of Xhat
    nl = off.live
    Ubar = stiefel_project(off.Phi[:, :nl], Phibar[:, :nl]) * off.flips[None, :nl]
    Xhat_bar = svd_adjoint(off.U, off.s, off.Vt, Ubar, Abar["sigma"][:nl], nl)
    # Xhat = d Xc, d = 1/mean(Xc^2)
    Xc = off.Q - off.q_ref[:, None]
    dbar += float(np.sum(Xhat_bar * Xc))
    Xc_bar = off.d * Xhat_bar - (off.d * off.d) * dbar * (2.0 / Xc.size) * Xc
    Qbar = Xc_bar.copy()
    Qbar[:, -1] += qlast_bar
    qref_bar = qref_bar - Xc_bar.sum(axis=1)
    # training FOM, reversed
    qbar = np.zeros_like(off.q0)
    for k in range(off.Q.shape[1] - 1, -1, -1):
        w, nb = be_adjoint(off.Q[:, k], qbar + Qbar[:, k], h, cfg.nu)
        nubar += nb
        qbar = w
    q0bar = qbar + qref_bar
    return q0bar, nubar


def adjoint_gradient(cfg, n_steps, target, ckpt_every=50):
    """(J, {"nu": dJ/dnu, "A": dJ/dA}) by reverse mode with checkpoints.

    The forward pass keeps the online state every ``ckpt_every`` steps and
    nothing else; the reverse sweep recomputes each segment from its
    checkpoint, then runs the adjoint of its steps backwards. Memory: the
    offline intermediates, n_steps / ckpt_every states and one segment's
    records.
    """
    import synth
    _check_cfg(cfg)
    if ckpt_every < 1:
        raise ValueError("ckpt_every must be positive")
    q0 = synth.initial_state(cfg)
    off = _offline(cfg, q0)
    st = _State(off.Phi.copy(), off.sigma.copy(), off.a.copy(), off.y_corr.copy(), cfg.w_init)
    ckpts = []
    qT = None
    for m in range(n_steps):
        if m % ckpt_every == 0:
            ckpts.append(st.copy())
        qT = _online_step(cfg, st, off.q_ref, off.d).qt
    J = 0.5 * float(np.sum((qT - target) ** 2))
    Abar = dict(Phi=np.zeros_like(off.Phi), sigma=np.zeros_like(off.sigma),
                a=np.zeros_like(off.a), y=np.zeros_like(off.y_corr),
                q_ref=np.zeros_like(off.q_ref), d=0.0, nu=0.0)
    for c in range(len(ckpts) - 1, -1, -1):
        st = ckpts[c].copy()
        m0 = c * ckpt_every
        m1 = min(n_steps, m0 + ckpt_every)
        recs = [_online_step(cfg, st, off.q_ref, off.d) for _ in range(m0, m1)]
        for m in range(m1 - 1, m0 - 1, -1):
            qtbar = (qT - target) if m == n_steps - 1 else np.zeros_like(qT)
            _step_adjoint(cfg, recs[m - m0], off.q_ref, off.d, Abar, qtbar)
    q0bar, nubar = _offline_adjoint(cfg, off, Abar)
    dA = float(q0bar @ synth.burgers_ic_amplitude_direction(cfg.n_cells))
    return J, {"nu": nubar, "A": dA}


def at(cfg, **kw):
    """A copy of ``cfg`` with some fields replaced (the point of evaluation)."""
    c = copy.copy(cfg)
    for k, v in kw.items():
        setattr(c, k, v)
    return c
