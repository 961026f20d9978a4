"""Full-order finite-volume operators and the backward-Euler Newton step (oracle).

Test infrastructure only; see the package docstring.

* Burgers: conservative form ``u_t + (u^2/2)_x = nu u_xx`` on the periodic unit
  interval. Convective flux at the interface i+1/2 is the Godunov flux of
  ``u^2/2``, ``F(uL, uR) = max(max(uL,0)^2/2, min(uR,0)^2/2)``, which reduces to
  the paper's first-order upwind flux ``uL^2/2`` when u > 0 (Sec. 5.1 problem
  setup); the diffusion term is the centred second difference. Jacobian entries
  take the derivative of the selected branch of the max (tie -> left branch).
* Euler (App. B, Eqs. sod_flux_appendix ... sod_sound_speed_appendix):
  conserved (rho, m, E), ideal gas, local Lax-Friedrichs (Rusanov) flux with
  ``s = max(|u_i|+c_i, |u_{i+1}|+c_{i+1})``, zero-gradient ghost cells. Density
  and pressure are floored at 1e-10 when primitives are recovered. The
  Jacobian is that of the discrete residual, with the derivative of the
  selected branch of the max in s (tie -> left state).
* Backward Euler (Eq. be_residual_rom_section / Eq. coarse_fom_backward_euler):
  ``q - q_prev - h f(q) = 0`` solved by Newton from ``q_prev`` with
  ``(I - h J_f) delta = -r``; stop once ``max|delta| <= tol (1 + max|q|)``.
* Explicit steps (App. D, the RDE solver): the four-stage, third-order
  strong-stability-preserving Runge-Kutta scheme. The paper names the scheme
  without its coefficients; this is the one with SSP coefficient 2 (Spiteri
  and Ruuth, SIAM J. Numer. Anal. 40, 2002): three half steps of forward
  Euler, an average with the start value, and a last half step.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

RHO_FLOOR = 1e-10
P_FLOOR = 1e-10


class NewtonNoConvergence(RuntimeError):
    pass


# ----------------------------------------------------------------------------
# Burgers
# ----------------------------------------------------------------------------

def godunov_flux(uL, uR):
    """Godunov flux of u^2/2 at an interface with left/right states uL, uR."""
    left = 0.5 * np.maximum(uL, 0.0) ** 2
    right = 0.5 * np.minimum(uR, 0.0) ** 2
    return np.maximum(left, right)


def godunov_flux_derivs(uL, uR):
    """(dF/duL, dF/duR) of the Godunov flux: derivative of the selected branch."""
    left = 0.5 * np.maximum(uL, 0.0) ** 2
    right = 0.5 * np.minimum(uR, 0.0) ** 2
    take_left = left >= right
    dL = np.where(take_left, np.maximum(uL, 0.0), 0.0)
    dR = np.where(take_left, 0.0, np.minimum(uR, 0.0))
    return dL, dR


def burgers_f(u, nu):
    """Semi-discrete Burgers operator f(u) on N periodic cells of width 1/N."""
    n = u.shape[0]
    dx = 1.0 / n
    u_right = np.roll(u, -1)          # u_{i+1}
    u_left = np.roll(u, 1)            # u_{i-1}
    F = godunov_flux(u, u_right)      # F[i] = F_{i+1/2}
    F_left = np.roll(F, 1)            # F_{i-1/2}
    conv = -(F - F_left) / dx
    diff = nu * (u_right - 2.0 * u + u_left) / dx**2
    return conv + diff


def burgers_jac(u, nu):
    """Sparse J_f = df/du of the Burgers operator (periodic tridiagonal)."""
    n = u.shape[0]
    dx = 1.0 / n
    u_right = np.roll(u, -1)
    dL, dR = godunov_flux_derivs(u, u_right)   # derivatives of F_{i+1/2}
    dL_left = np.roll(dL, 1)                   # dF_{i-1/2}/du_{i-1}
    dR_left = np.roll(dR, 1)                   # dF_{i-1/2}/du_i
    d = nu / dx**2
    diag = -dL / dx + dR_left / dx - 2.0 * d   # d f_i / d u_i
    upper = -dR / dx + d                       # d f_i / d u_{i+1}
    lower = dL_left / dx + d                   # d f_i / d u_{i-1}
    rows = np.arange(n)
    I = np.concatenate([rows, rows, rows])
    J = np.concatenate([rows, (rows + 1) % n, (rows - 1) % n])
    V = np.concatenate([diag, upper, lower])
    return sp.csr_matrix(sp.coo_matrix((V, (I, J)), shape=(n, n)))


# ----------------------------------------------------------------------------
# Euler (Sod), variable-blocked state [rho, m, E]
# ----------------------------------------------------------------------------

def euler_primitives(U, gamma):
    n = U.shape[0] // 3
    rho = np.maximum(U[:n], RHO_FLOOR)
    m = U[n:2 * n]
    E = U[2 * n:]
    u = m / rho
    p = np.maximum((gamma - 1.0) * (E - 0.5 * rho * u * u), P_FLOOR)
    return rho, m, E, u, p


def euler_physical_flux(rho, m, E, u, p):
    return np.stack([m, m * u + p, u * (E + p)])


def euler_f(U, gamma):
    """Semi-discrete Euler operator  -(F_{i+1/2} - F_{i-1/2}) / dx  (App. B)."""
    n = U.shape[0] // 3
    dx = 1.0 / n
    rho, m, E, u, p = euler_primitives(U, gamma)
    c = np.sqrt(gamma * p / rho)
    # ghost cells: copies of the end states
    idx = np.concatenate([[0], np.arange(n), [n - 1]])
    rho_g, m_g, E_g, u_g, p_g, c_g = rho[idx], m[idx], E[idx], u[idx], p[idx], c[idx]
    Ug = np.stack([U[:n][idx], m_g, E_g])        # raw conserved values of the cells
    Fg = euler_physical_flux(rho_g, m_g, E_g, u_g, p_g)
    speed = np.abs(u_g) + c_g
    s = np.maximum(speed[:-1], speed[1:])         # n+1 interfaces
    Fhat = 0.5 * (Fg[:, :-1] + Fg[:, 1:]) - 0.5 * s * (Ug[:, 1:] - Ug[:, :-1])
    rhs = -(Fhat[:, 1:] - Fhat[:, :-1]) / dx
    return rhs.reshape(-1)


def _euler_cell_derivs(U, gamma):
    """Per-cell derivatives of the physical flux (3x3) and of |u|+c (3,) w.r.t.
    the conserved variables, with the floors' derivatives taken as zero when a
    floor is active."""
    n = U.shape[0] // 3
    rho_raw = U[:n]
    rho = np.maximum(rho_raw, RHO_FLOOR)
    drho = (rho_raw > RHO_FLOOR).astype(float)    # d rho_used / d rho_raw
    m = U[n:2 * n]
    E = U[2 * n:]
    u = m / rho
    p_raw = (gamma - 1.0) * (E - 0.5 * rho * u * u)
    p = np.maximum(p_raw, P_FLOOR)
    pact = (p_raw > P_FLOOR).astype(float)
    g1 = gamma - 1.0
    # derivatives of u and p w.r.t. (rho_raw, m, E)
    du = np.stack([-m / rho**2 * drho, 1.0 / rho, np.zeros(n)])
    # p_raw = g1 (E - m^2/(2 rho))
    dp = pact * np.stack([g1 * 0.5 * m * m / rho**2 * drho, -g1 * m / rho, g1 * np.ones(n)])
    # physical flux F = [m, m u + p, u (E + p)]
    dF = np.zeros((3, 3, n))
    dF[0] = np.stack([np.zeros(n), np.ones(n), np.zeros(n)])
    dF[1] = m * du + dp + np.stack([np.zeros(n), u, np.zeros(n)])
    dF[2] = du * (E + p) + u * (dp + np.stack([np.zeros(n), np.zeros(n), np.ones(n)]))
    c = np.sqrt(gamma * p / rho)
    # c = sqrt(gamma p / rho): dc = c/2 (dp/p - drho_used/rho)
    drho_used = np.stack([drho, np.zeros(n), np.zeros(n)])
    dc = 0.5 * c * (dp / p - drho_used / rho)
    sgn = np.where(u >= 0.0, 1.0, -1.0)
    dspeed = sgn * du + dc
    F = euler_physical_flux(rho, m, E, u, p)
    return F, dF, np.abs(u) + c, dspeed


def euler_jac(U, gamma):
    """Sparse J_f of the Euler operator (3x3-block tridiagonal in cell index,
    variable-blocked ordering)."""
    n = U.shape[0] // 3
    dx = 1.0 / n
    F, dF, speed, dspeed = _euler_cell_derivs(U, gamma)
    Uc = np.stack([U[:n], U[n:2 * n], U[2 * n:]])
    # Interfaces k = 0..n, between ghost-extended cells L=k-1, R=k (clamped).
    L = np.clip(np.arange(n + 1) - 1, 0, n - 1)
    R = np.clip(np.arange(n + 1), 0, n - 1)
    take_left = speed[L] >= speed[R]
    s = np.where(take_left, speed[L], speed[R])
    dUdiff = Uc[:, R] - Uc[:, L]                       # (3, n+1)
    eye = np.eye(3)[:, :, None]
    # dFhat_k / dU_L and dU_R (3x3 each); same cell on both sides at the ends
    # is handled by summing the two contributions into that cell.
    ds_dL = np.where(take_left, 1.0, 0.0)[None, :] * dspeed[:, L]   # (3, n+1)
    ds_dR = np.where(take_left, 0.0, 1.0)[None, :] * dspeed[:, R]
    dFh_dL = 0.5 * dF[:, :, L] + 0.5 * s * eye - 0.5 * dUdiff[:, None, :] * ds_dL[None, :, :]
    dFh_dR = 0.5 * dF[:, :, R] - 0.5 * s * eye - 0.5 * dUdiff[:, None, :] * ds_dR[None, :, :]
    # f_i = -(Fhat_{i+1} - Fhat_i)/dx: interface i+1 joins cells (L, R) = (i, i+1)
    # and interface i joins (i-1, i); at the ends both sides are the same cell
    # and COO assembly sums the duplicate entries.
    i = np.arange(n)
    parts = [
        (L[i + 1], -dFh_dL[:, :, i + 1] / dx),
        (R[i + 1], -dFh_dR[:, :, i + 1] / dx),
        (L[i], dFh_dL[:, :, i] / dx),
        (R[i], dFh_dR[:, :, i] / dx),
    ]
    rows, cols, vals = [], [], []
    for cell, blk in parts:
        for a in range(3):
            for b in range(3):
                rows.append(a * n + i)
                cols.append(b * n + cell)
                vals.append(blk[a, b])
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = np.concatenate(vals)
    return sp.csr_matrix(sp.coo_matrix((vals, (rows, cols)), shape=(3 * n, 3 * n)))


# ----------------------------------------------------------------------------
# generic interface
# ----------------------------------------------------------------------------

def fom_f(q, problem, nu=0.0, gamma=1.4):
    if problem == 0:
        return burgers_f(q, nu)
    return euler_f(q, gamma)


def fom_jac(q, problem, nu=0.0, gamma=1.4):
    if problem == 0:
        return burgers_jac(q, nu)
    return euler_jac(q, gamma)


def be_step(q_prev, h, problem, nu=0.0, gamma=1.4, tol=1e-12, max_iter=20,
            return_iters=False):
    """One backward-Euler step ``q - q_prev - h f(q) = 0`` by Newton from q_prev.

    The linear system ``(I - h J_f) delta = -r`` is solved by sparse LU
    (SciPy); stop when ``max|delta| <= tol (1 + max|q|)`` after the update.
    """
    q = q_prev.copy()
    n = q.shape[0]
    I = sp.identity(n, format="csr")
    for it in range(1, max_iter + 1):
        r = q - q_prev - h * fom_f(q, problem, nu, gamma)
        Jr = (I - h * fom_jac(q, problem, nu, gamma)).tocsc()
        delta = spla.spsolve(Jr, -r)
        q = q + delta
        if np.max(np.abs(delta)) <= tol * (1.0 + np.max(np.abs(q))):
            return (q, it) if return_iters else q
    raise NewtonNoConvergence(f"BE Newton did not converge in {max_iter} iterations")


def ssprk43_step(q, h, rhs):
    """One step of the four-stage, third-order SSP Runge-Kutta scheme for
    dq/dt = rhs(q): q1 = q + h/2 rhs(q), q2 = q1 + h/2 rhs(q1),
    q3 = 2/3 q + 1/3 (q2 + h/2 rhs(q2)), q_new = q3 + h/2 rhs(q3).
    On dq/dt = lam q it multiplies q by 1 + z + z^2/2 + z^3/6 + z^4/48, z = h lam."""
    q1 = q + 0.5 * h * rhs(q)
    q2 = q1 + 0.5 * h * rhs(q1)
    q3 = (2.0 / 3.0) * q + (1.0 / 3.0) * (q2 + 0.5 * h * rhs(q2))
    return q3 + 0.5 * h * rhs(q3)


def explicit_step(q_prev, h, problem, nu=0.0, gamma=1.4):
    """One SSPRK(4,3) step of the FOM dq/dt = f(q)."""
    return ssprk43_step(q_prev, h, lambda u: fom_f(u, problem, nu, gamma))
