"""History-aware adaptive ROM: plain FP64 restatement of Algorithms 1 and 2 (oracle).

Test infrastructure only; see the package docstring. Each function follows one
passage of the paper:

* ``preprocess``     Sec. 3.1, Eqs. scaling_matrix_local_block and
                     variable_normalization: q_ref = initial solution,
                     D_v = 1/phi_v with phi_v the time-space mean of the squared
                     centred training field (read literally as a mean square).
* ``pod``            Sec. 3.1 / Algorithm 1 (POD step): leading r left singular
                     vectors and values of D (Q_train - q_ref 1^T).
* ``galerkin_step``  Eq. galerkin_continuous_rom discretised by backward Euler
                     (Eq. be_residual_rom_section), solved by Newton with the
                     exact reduced Jacobian I - dt Phi^T D J_f D^-1 Phi.
* ``hyper_step``     Eq. deim_galerkin_rom (DEIM with U = Phi) discretised the
                     same way: a - a^n - dt (P^T Phi)^+ P^T D f(q~(a)) = 0.
* ``lspg_step``      Eq. lspg_minimization with the test basis of Eq.
                     lspg_test_basis_be, by Gauss-Newton.
* ``hyper_lspg_step`` Eq. hyperreduced_lspg / hyperreduced_lspg_stationarity.
* ``qdeim``          Eq. qdeim_qr: first pivots of a column-pivoted QR of Phi^T.
* ``fgs_extend``     Eq. fgs_selection with the feature map Theta(y) = y
                     (Burgers) or the cell pressures (Euler, Sec. 5.3): the
                     rows with the largest squared forward difference of the
                     feature of the correction snapshot, skipping rows
                     already chosen.
* ``isvd_update``    Algorithm 2 / Eqs. isvd_residual ... isvd_truncation.
* ``windowed_svd_update``, ``direct_update``  the comparison rules of App. A
                     (Eqs. wsvd_window_matrix, wsvd_update; direct_optimization,
                     direct_update) on the window of correction snapshots.
* ``onestep_update``, ``oja_update``, ``grouse_update``  the instantaneous
                     comparison rules of App. A (Eqs. onestep_update,
                     oja_update, grouse_projection, grouse_update) on the
                     current correction snapshot.
* ``AdaptiveROM``    Algorithm 1.

Readings where the paper is silent: see the module-level constants and the
docstrings (Newton stopping rule, rank-deficient iSVD residual, sign
convention of singular vectors, oversampling rule for n_s > r).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from . import fv

RANK_TOL = 1e-10      # numerical-rank tolerance relative to the largest singular value
PHI_FLOOR = 1e-300    # preprocessing: guard for a variable with no variation


class NewtonNoConvergence(RuntimeError):
    pass


# ----------------------------------------------------------------------------
# offline pieces
# ----------------------------------------------------------------------------

def fine_fom_step(q, cfg):
    """One fine FOM step: backward Euler (Eq. fom_lmm with the BE
    coefficients, Eq. fom_discrete_solve), or SSPRK(4,3) for the explicit
    form (time_scheme 1, the RDE solver of App. D)."""
    if getattr(cfg, "time_scheme", 0) == 1:
        return fv.explicit_step(q, cfg.dt, cfg.problem, cfg.nu, cfg.gamma)
    return fv.be_step(q, cfg.dt, cfg.problem, cfg.nu, cfg.gamma, cfg.newton_tol, cfg.newton_max)


def fom_trajectory(q0, n_steps, cfg):
    """Fine FOM states q^1..q^n_steps as columns."""
    out = np.empty((q0.shape[0], n_steps))
    q = q0
    for k in range(n_steps):
        q = fine_fom_step(q, cfg)
        out[:, k] = q
    return out


def preprocess(Q_train, q0, n_var):
    """(q_ref, diag(D), D (Q_train - q_ref 1^T)).

    q_ref is the initial solution. For each variable v the characteristic
    magnitude phi_v is the mean over snapshots and cells of the squared centred
    field, and every cell block of D carries 1/phi_v.
    """
    q_ref = q0.copy()
    Xc = Q_train - q_ref[:, None]
    n_cells = q0.shape[0] // n_var
    dvals = np.empty(n_var)
    for v in range(n_var):
        blk = Xc[v * n_cells:(v + 1) * n_cells, :]
        phi = float(np.mean(blk * blk))
        if phi < PHI_FLOOR:
            phi = 1.0
        dvals[v] = 1.0 / phi
    d = np.repeat(dvals, n_cells)
    return q_ref, d, d[:, None] * Xc


def sign_normalise(U):
    """Flip each column so that its largest-magnitude entry is positive
    (tie -> lowest index). Singular vectors are unique only up to sign."""
    U = U.copy()
    for j in range(U.shape[1]):
        i = int(np.argmax(np.abs(U[:, j])))
        if U[i, j] < 0:
            U[:, j] = -U[:, j]
    return U


def pod(Xhat, r):
    """Leading r left singular vectors and singular values (LAPACK thin SVD)."""
    U, s, _ = np.linalg.svd(Xhat, full_matrices=False)
    U = sign_normalise(U[:, :r])
    s = s[:r].copy()
    return drop_null_directions(U, s)


def drop_null_directions(U, s):
    """Zero the columns (and singular values) with s_j <= RANK_TOL * s_1: such
    directions carry no information above rounding. A zero column is inert in
    every reduced operator (its coordinate keeps its value, zero)."""
    U = U.copy()
    s = s.copy()
    if s.shape[0] and s[0] > 0:
        null = s <= RANK_TOL * s[0]
        U[:, null] = 0.0
        s[null] = 0.0
    return U, s


# ----------------------------------------------------------------------------
# reduced steps
# ----------------------------------------------------------------------------

def lift(a, Phi, q_ref, d):
    """q~ = q_ref + D^-1 Phi a (Eq. trial_approximation)."""
    return q_ref + (Phi @ a) / d


def galerkin_residual(a, a_prev, Phi, q_ref, d, cfg):
    qt = lift(a, Phi, q_ref, d)
    f = fv.fom_f(qt, cfg.problem, cfg.nu, cfg.gamma)
    return a - a_prev - cfg.dt * (Phi.T @ (d * f))


def galerkin_jacobian(a, Phi, q_ref, d, cfg):
    qt = lift(a, Phi, q_ref, d)
    Jf = fv.fom_jac(qt, cfg.problem, cfg.nu, cfg.gamma)
    JfPhi = Jf @ (Phi / d[:, None])
    return np.eye(Phi.shape[1]) - cfg.dt * (Phi.T @ (d[:, None] * JfPhi))


def hyper_residual(a, a_prev, Phi, q_ref, d, P, M, cfg):
    """a - a^n - dt (P^T Phi)^+ P^T D f(q~(a)). f is evaluated on the full
    lifted state and then sampled, which is slow but obviously equal to
    evaluating it on the sample mesh."""
    qt = lift(a, Phi, q_ref, d)
    f = fv.fom_f(qt, cfg.problem, cfg.nu, cfg.gamma)
    return a - a_prev - cfg.dt * (M @ (d * f)[P])


def hyper_jacobian(a, Phi, q_ref, d, P, M, cfg):
    qt = lift(a, Phi, q_ref, d)
    Jf = fv.fom_jac(qt, cfg.problem, cfg.nu, cfg.gamma)
    JfPhi = Jf @ (Phi / d[:, None])
    return np.eye(Phi.shape[1]) - cfg.dt * (M @ (d[:, None] * JfPhi)[P, :])


def _newton(a_prev, resid, jac, tol, max_iter):
    """Newton from a_prev; stop once max|delta| <= tol (1 + max|a|)."""
    a = a_prev.copy()
    for it in range(1, max_iter + 1):
        g = resid(a)
        J = jac(a)
        delta = np.linalg.solve(J, -g)
        a = a + delta
        if np.max(np.abs(delta)) <= tol * (1.0 + np.max(np.abs(a))):
            return a, it
    raise NewtonNoConvergence(f"reduced Newton did not converge in {max_iter} iterations")


def galerkin_rhs(a, Phi, q_ref, d, cfg):
    """da/dt = Phi^T D f(q~(a)) (Eq. galerkin_continuous_rom)."""
    return Phi.T @ (d * fv.fom_f(lift(a, Phi, q_ref, d), cfg.problem, cfg.nu, cfg.gamma))


def hyper_rhs(a, Phi, q_ref, d, P, M, cfg):
    """da/dt = (P^T Phi)^+ P^T D f(q~(a)) (Eq. deim_galerkin_rom, continuous in
    time); f on the full lifted state, then sampled."""
    f = fv.fom_f(lift(a, Phi, q_ref, d), cfg.problem, cfg.nu, cfg.gamma)
    return M @ (d * f)[P]


def explicit_galerkin_step(a_prev, Phi, q_ref, d, cfg, P=None, M=None):
    """One SSPRK(4,3) step of the Galerkin ROM (hyper-reduced when P is given);
    returns (a_new, 0): no iterations."""
    if P is None:
        rhs = lambda a: galerkin_rhs(a, Phi, q_ref, d, cfg)      # noqa: E731
    else:
        rhs = lambda a: hyper_rhs(a, Phi, q_ref, d, P, M, cfg)   # noqa: E731
    return fv.ssprk43_step(a_prev, cfg.dt, rhs), 0


def galerkin_step(a_prev, Phi, q_ref, d, cfg):
    """One backward-Euler Galerkin ROM step (plain projection)."""
    return _newton(a_prev,
                   lambda a: galerkin_residual(a, a_prev, Phi, q_ref, d, cfg),
                   lambda a: galerkin_jacobian(a, Phi, q_ref, d, cfg),
                   cfg.newton_tol, cfg.newton_max)


def hyper_step(a_prev, Phi, q_ref, d, P, M, cfg):
    """One backward-Euler DEIM-Galerkin ROM step (U = Phi, sample set P)."""
    return _newton(a_prev,
                   lambda a: hyper_residual(a, a_prev, Phi, q_ref, d, P, M, cfg),
                   lambda a: hyper_jacobian(a, Phi, q_ref, d, P, M, cfg),
                   cfg.newton_tol, cfg.newton_max)


# ----------------------------------------------------------------------------
# least-squares Petrov-Galerkin steps (Sec. 3.1, Sec. 3.2)
# ----------------------------------------------------------------------------

def lspg_residual(a, a_prev, Phi, q_ref, d, cfg):
    """D r(q~(a)) with the backward-Euler residual r(q) = q - q^{n-1} - dt f(q)
    (Eq. be_residual_rom_section); the previous state is the lifted reduced
    state q~(a_prev) in the current basis."""
    qt = lift(a, Phi, q_ref, d)
    qp = lift(a_prev, Phi, q_ref, d)
    return d * (qt - qp - cfg.dt * fv.fom_f(qt, cfg.problem, cfg.nu, cfg.gamma))


def lspg_test_basis(a, Phi, q_ref, d, cfg):
    """Psi = (I - dt D J_f(q~) D^-1) Phi (Eq. lspg_test_basis_be)."""
    qt = lift(a, Phi, q_ref, d)
    Jf = fv.fom_jac(qt, cfg.problem, cfg.nu, cfg.gamma)
    return Phi - cfg.dt * (d[:, None] * (Jf @ (Phi / d[:, None])))


def _gauss_newton(a_prev, resid, jac, tol, max_iter):
    """Gauss-Newton for min |resid(a)|^2 from a_prev: each step is the least
    squares solution of jac(a) delta = -resid(a) (minimum norm, so null basis
    columns keep a zero step); stop once max|delta| <= tol (1 + max|a|)."""
    a = a_prev.copy()
    for it in range(1, max_iter + 1):
        delta = np.linalg.lstsq(jac(a), -resid(a), rcond=None)[0]
        a = a + delta
        if np.max(np.abs(delta)) <= tol * (1.0 + np.max(np.abs(a))):
            return a, it
    raise NewtonNoConvergence(f"Gauss-Newton did not converge in {max_iter} iterations")


def lspg_step(a_prev, Phi, q_ref, d, cfg):
    """One LSPG step: Eq. lspg_minimization, a = argmin |D r(q~(a))|, by
    Gauss-Newton with the Jacobian d(D r)/da = Psi; its fixed point satisfies
    Eq. lspg_stationarity, Psi^T D r = 0."""
    return _gauss_newton(a_prev,
                         lambda a: lspg_residual(a, a_prev, Phi, q_ref, d, cfg),
                         lambda a: lspg_test_basis(a, Phi, q_ref, d, cfg),
                         cfg.newton_tol, cfg.newton_max)


def hyper_lspg_step(a_prev, Phi, q_ref, d, P, M, cfg):
    """One hyper-reduced LSPG step (Eq. hyperreduced_lspg): minimise
    |Phi M P^T D r| = |M P^T D r| (Phi orthonormal, M = (P^T Phi)^+) by
    Gauss-Newton with the Jacobian M P^T Psi; the fixed point satisfies Eq.
    hyperreduced_lspg_stationarity."""
    def resid(a):
        return M @ lspg_residual(a, a_prev, Phi, q_ref, d, cfg)[P]

    def jac(a):
        return M @ lspg_test_basis(a, Phi, q_ref, d, cfg)[P, :]

    return _gauss_newton(a_prev, resid, jac, cfg.newton_tol, cfg.newton_max)


# ----------------------------------------------------------------------------
# sampling
# ----------------------------------------------------------------------------

def numerical_rank(Phi):
    """Number of non-zero (non-null) basis columns."""
    return int(np.count_nonzero(np.any(Phi != 0.0, axis=0)))


def qdeim(Phi, m):
    """First min(m, rank) pivots of the column-pivoted QR of Phi^T (Eq. qdeim_qr).
    Beyond the rank of Phi the pivoted QR has nothing left to pivot on."""
    _, piv = sla.qr(Phi.T, mode="r", pivoting=True)
    return [int(i) for i in piv[:min(m, numerical_rank(Phi))]]


def fgs_scores(y, problem=0, gamma=1.4):
    """Score of every row of the state for Eq. fgs_selection: the squared
    forward difference of the feature, i.e. its squared gradient up to the
    constant 1/dx^2.

    * Burgers: Theta(y) = y, periodic: (y_{i+1} - y_i)^2.
    * Euler: Theta(y) = the cell pressures p_i (Sec. 5.3 uses pressure as the
      feature; p recovered as in App. B, floors included). The right end has
      the zero-gradient ghost cell of the finite-volume scheme, so the last
      cell scores 0. The sample set is a set of rows of the 3N state, so each
      of a cell's three rows (rho, m, E) carries the cell's score."""
    if problem == 0:
        return (np.roll(y, -1) - y) ** 2
    p = fv.euler_primitives(y, gamma)[4]
    dp = np.append(p[1:], p[-1]) - p
    return np.tile(dp * dp, 3)


def fgs_extend(y, chosen, count, problem=0, gamma=1.4):
    """Greedy feature-guided points: largest scores first (tie -> lowest index),
    skipping rows already in ``chosen``."""
    g = fgs_scores(y, problem, gamma)
    order = np.lexsort((np.arange(g.shape[0]), -g))
    taken = set(chosen)
    out = []
    for i in order:
        if len(out) == count:
            break
        if int(i) not in taken:
            out.append(int(i))
            taken.add(int(i))
    return out


def sample_points(Phi, y_corr, n_s, problem=0, gamma=1.4):
    """QDEIM points (up to r) extended to n_s by feature-guided points."""
    P = qdeim(Phi, n_s)
    if n_s > len(P):
        P = P + fgs_extend(y_corr, P, n_s - len(P), problem, gamma)
    return P


def sampled_pinv(Phi, P):
    """(P^T Phi)^+ by SVD-based pseudo-inverse (NumPy pinv)."""
    return np.linalg.pinv(Phi[P, :])


# ----------------------------------------------------------------------------
# iSVD (Algorithm 2)
# ----------------------------------------------------------------------------

def project_cgs2(Phi, y):
    """Least-squares coordinates p = Phi^+ y and residual q = y - Phi p for an
    orthonormal Phi, by classical Gram-Schmidt applied twice: the second pass
    removes the component that rounding leaves in span(Phi) when ||q|| is much
    smaller than ||y|| (Eq. isvd_residual)."""
    p1 = Phi.T @ y
    q1 = y - Phi @ p1
    p2 = Phi.T @ q1
    q = q1 - Phi @ p2
    return p1 + p2, q


def isvd_update(Phi, sigma, yhat, lam, r, return_core=False):
    """Rank-one incremental SVD with forgetting factor, truncated to rank r.

    p solves min ||yhat - Phi p|| (least squares, by ``project_cgs2``);
    q = yhat - Phi p; the core
    K = [[lam Sigma, p], [0, ||q||]] is decomposed by a dense SVD, the augmented
    basis [Phi, q/||q||] is rotated by its left singular vectors and the
    leading r directions are kept. If ||q|| <= RANK_TOL * max(||yhat||, sigma_1)
    the new direction is empty: q/||q|| is replaced by 0 and K's corner by 0.
    """
    k = Phi.shape[1]
    p, q = project_cgs2(Phi, yhat)
    rho = float(np.linalg.norm(q))
    scale = max(float(np.linalg.norm(yhat)), float(sigma[0]) if k else 0.0)
    if rho <= RANK_TOL * scale:
        qhat = np.zeros_like(q)
        rho = 0.0
    else:
        qhat = q / rho
    K = np.zeros((k + 1, k + 1))
    K[:k, :k] = lam * np.diag(sigma)
    K[:k, k] = p
    K[k, k] = rho
    Ub, sb, _ = np.linalg.svd(K)
    Phit = np.hstack([Phi, qhat[:, None]]) @ Ub
    keep = min(r, k + 1)
    Phi_new, s_new = drop_null_directions(sign_normalise(Phit[:, :keep]), sb[:keep])
    if return_core:
        return Phi_new, s_new, K, Ub, sb
    return Phi_new, s_new


def rank_decision_margin(Phi, sigma, yhat, lam, r):
    """Diagnostic, not part of the method: how close the two rank decisions of
    one ``isvd_update`` come to the tolerance, as min |log(x / RANK_TOL)| over
    x = ||q|| / max(||yhat||, sigma_1) (is the new direction empty?) and
    x = s_j / s_1 of the kept core singular values (is direction j null?).
    A small margin means that a rounding-level change can flip the rank."""
    k = Phi.shape[1]
    p, q = project_cgs2(Phi, yhat)
    rho = float(np.linalg.norm(q))
    scale = max(float(np.linalg.norm(yhat)), float(sigma[0]) if k else 0.0)
    out = np.inf
    if scale > 0 and rho > 0:
        out = abs(np.log(rho / (RANK_TOL * scale)))
    K = np.zeros((k + 1, k + 1))
    K[:k, :k] = lam * np.diag(sigma)
    K[:k, k] = p
    K[k, k] = rho if rho > RANK_TOL * scale else 0.0
    sb = np.linalg.svd(K, compute_uv=False)[:min(r, k + 1)]
    if sb.shape[0] and sb[0] > 0:
        pos = sb[sb > 0]
        if pos.shape[0]:
            out = min(out, float(np.min(np.abs(np.log(pos / (RANK_TOL * sb[0]))))))
    return out


# ----------------------------------------------------------------------------
# comparison update rules (App. A): windowed SVD and the Direct method
# ----------------------------------------------------------------------------

def windowed_svd_update(Y, r):
    """Eqs. wsvd_window_matrix and wsvd_update: the leading r left singular
    vectors (and values) of the window of preprocessed correction snapshots
    Y (N x w), by the thin SVD, with the same numerical-rank truncation and
    sign convention as the POD."""
    U, s, _ = np.linalg.svd(Y, full_matrices=False)
    keep = min(r, U.shape[1])
    Phi = np.zeros((Y.shape[0], r))
    sig = np.zeros(r)
    P, sk = drop_null_directions(sign_normalise(U[:, :keep]), s[:keep])
    Phi[:, :keep], sig[:keep] = P, sk
    return Phi, sig


def direct_update(Phi, Y, r):
    """Eqs. direct_optimization and direct_update: Phi_new = Y (Phi^+ Y)^+ for
    the window Y (N x w), the pseudo-inverses cut at the numerical-rank
    tolerance. Reading: the update fixes a subspace, and the ROM's projections
    assume an orthonormal basis, so the returned basis is an orthonormal basis
    of span(Y (Phi^+ Y)^+) (its dominant left singular vectors, sign convention
    as the POD's); its 'singular values' are those of Phi^+ Y, which set its
    rank."""
    C = np.linalg.pinv(Phi, rcond=RANK_TOL) @ Y
    sC = np.linalg.svd(C, compute_uv=False)
    rank = int(np.count_nonzero(sC > RANK_TOL * sC[0])) if sC.size and sC[0] > 0 else 0
    X = Y @ np.linalg.pinv(C, rcond=RANK_TOL)
    U, _, _ = np.linalg.svd(X, full_matrices=False)
    k = min(rank, r)
    Phi_new = np.zeros((Y.shape[0], r))
    Phi_new[:, :k] = sign_normalise(U[:, :k])
    sig = np.zeros(r)
    sig[:k] = sC[:k]
    return Phi_new, sig


# ----------------------------------------------------------------------------
# instantaneous comparison rules (App. A): one-step, Oja, GROUSE
# ----------------------------------------------------------------------------
#
# Each acts on the live (non-null) columns of the basis and keeps the rank;
# null columns stay zero. orth(.) is read as the orthonormal factor of the
# thin QR factorisation: the online loop only uses the subspace (the
# Galerkin step and the state transfer are invariant under Phi -> Phi Q), so
# any orthonormal basis of the same span serves.

def _orth(X):
    Q, _ = np.linalg.qr(X)
    return Q


def _live(Phi):
    return Phi[:, :numerical_rank(Phi)]


def _with_nulls(Phi, P):
    out = np.zeros_like(Phi)
    out[:, :P.shape[1]] = P
    return out


def onestep_update(Phi, yhat, a):
    """Eq. onestep_update: Phi_new = orth(Phi + (yhat - Phi a) a^T / |a|^2) with
    a the reduced state before the update; after the rank-one correction
    (before orth) Phi a equals yhat, so yhat lies in the new span."""
    P = _live(Phi)
    k = P.shape[1]
    ak = np.asarray(a[:k], dtype=np.float64)
    nn = float(ak @ ak)
    if k == 0 or nn == 0.0:
        return Phi.copy()
    X = P + np.outer(yhat - P @ ak, ak) / nn
    return _with_nulls(Phi, _orth(X))


def oja_update(Phi, yhat, eta):
    """Eq. oja_update: Phi_new = orth(Phi + eta yhat (yhat^T Phi))."""
    P = _live(Phi)
    if P.shape[1] == 0:
        return Phi.copy()
    X = P + eta * np.outer(yhat, yhat @ P)
    return _with_nulls(Phi, _orth(X))


def grouse_update(Phi, yhat, eta):
    """Eqs. grouse_projection and grouse_update: w the least-squares
    coefficients of yhat in span(Phi) and r = yhat - Phi w (classical
    Gram-Schmidt twice, which keeps r orthogonal to Phi to rounding relative to
    |r|, so that the update stays orthonormal when yhat is nearly in the span),
    p = Phi w,
    alpha = eta |p| |r|, and the rank-one geodesic step
    Phi + ((cos alpha - 1) p/|p| + sin alpha r/|r|) w^T/|w| (orthonormal by
    construction; no update when p, r or w vanishes)."""
    P = _live(Phi)
    if P.shape[1] == 0:
        return Phi.copy()
    w, rv = project_cgs2(P, yhat)       # least squares for orthonormal P, residual by CGS2
    pv = P @ w
    npn, nr, nw = float(np.linalg.norm(pv)), float(np.linalg.norm(rv)), float(np.linalg.norm(w))
    if npn == 0.0 or nr == 0.0 or nw == 0.0:
        return Phi.copy()
    alpha = eta * npn * nr
    X = P + np.outer((np.cos(alpha) - 1.0) * pv / npn + np.sin(alpha) * rv / nr, w / nw)
    return _with_nulls(Phi, X)


INSTANT_RULES = (3, 4, 5)   # one-step, Oja, GROUSE


# ----------------------------------------------------------------------------
# Algorithm 1
# ----------------------------------------------------------------------------

class AdaptiveROM:
    """History-aware adaptive ROM (Algorithm 1) with the iSVD update.

    Offline stage: w_init fine FOM steps, preprocessing, POD, initial
    reduced state, first coarse correction state, initial sampling points.
    Online loop: one reduced BE step per call of ``step``; every z
    steps an adaptation event advances the coarse FOM by z*dt, updates the
    basis by iSVD, refreshes the sampling points and transfers the state.
    """

    def __init__(self, cfg, q0, Q_train=None):
        self.cfg = cfg
        self.q0 = np.asarray(q0, dtype=np.float64).copy()
        if Q_train is None:
            Q_train = fom_trajectory(self.q0, cfg.w_init, cfg)
        self.Q_train = Q_train
        self.q_ref, self.d, Xhat = preprocess(Q_train, self.q0, cfg.n_var)
        self.Phi, self.sigma = pod(Xhat, cfg.r)
        q_last = Q_train[:, -1]
        self.a = self.Phi.T @ (self.d * (q_last - self.q_ref))
        self.y_corr = self.coarse_step(q_last)
        self.P = None
        self.M = None
        if cfg.n_s > 0:
            self._refresh_sampling()
        self.n = cfg.w_init
        self.events = 0
        self.newton_iters = []
        self.min_gap = np.inf
        # diagnostic: the closest call of the rank decisions (the POD's and
        # those of every event)
        s_pod = np.linalg.svd(Xhat, compute_uv=False)[:cfg.r]
        pos = s_pod[s_pod > 0]
        self.min_rank_margin = (float(np.min(np.abs(np.log(pos / (RANK_TOL * s_pod[0])))))
                                if pos.shape[0] else np.inf)
        # the correction-snapshot window of the comparison update rules,
        # initialised with the last w training snapshots (App. A)
        self.rule = getattr(cfg, "update_rule", 0)
        self.window = None
        if self.rule in (1, 2):
            w = cfg.window
            cols = [self.d * (Q_train[:, j] - self.q_ref) for j in range(Q_train.shape[1] - w,
                                                                         Q_train.shape[1])]
            self.window = np.stack(cols, axis=1)

    # -- pieces --------------------------------------------------------------
    def coarse_step(self, y):
        c = self.cfg
        return fv.be_step(y, c.z * c.dt, c.problem, c.nu, c.gamma, c.newton_tol, c.newton_max)

    def _refresh_sampling(self):
        self.P = sample_points(self.Phi, self.y_corr, self.cfg.n_s, self.cfg.problem, self.cfg.gamma)
        self.M = sampled_pinv(self.Phi, self.P)

    def rom_step(self, a_prev):
        c = self.cfg
        if getattr(c, "time_scheme", 0) == 1:       # explicit Galerkin (App. D form)
            if c.n_s > 0:
                return explicit_galerkin_step(a_prev, self.Phi, self.q_ref, self.d, c, self.P, self.M)
            return explicit_galerkin_step(a_prev, self.Phi, self.q_ref, self.d, c)
        if getattr(c, "projection", 0) == 1:        # LSPG
            if c.n_s > 0:
                return hyper_lspg_step(a_prev, self.Phi, self.q_ref, self.d, self.P, self.M, c)
            return lspg_step(a_prev, self.Phi, self.q_ref, self.d, c)
        if c.n_s > 0:
            return hyper_step(a_prev, self.Phi, self.q_ref, self.d, self.P, self.M, c)
        return galerkin_step(a_prev, self.Phi, self.q_ref, self.d, c)

    def lifted(self):
        return lift(self.a, self.Phi, self.q_ref, self.d)

    def is_event(self, n):
        return (n + 1 - self.cfg.w_init) % self.cfg.z == 0

    def adapt(self, q_tilde):
        """The adaptation event of Algorithm 1 for the reconstructed state q_tilde."""
        c = self.cfg
        if self.rule in INSTANT_RULES:
            self._adapt_instant(q_tilde)
            return
        self.y_corr = self.coarse_step(self.y_corr)
        yhat = self.d * (self.y_corr - self.q_ref)
        if self.rule in (1, 2):
            # drop the oldest snapshot, append the new one
            self.window = np.concatenate([self.window[:, 1:], yhat[:, None]], axis=1)
            if self.rule == 1:
                Phi_new, sigma_new = windowed_svd_update(self.window, c.r)
            else:
                Phi_new, sigma_new = direct_update(self.Phi, self.window, c.r)
        else:
            self.min_rank_margin = min(self.min_rank_margin,
                                       rank_decision_margin(self.Phi, self.sigma, yhat, c.lam, c.r))
            Phi_new, sigma_new, _, _, s_all = isvd_update(self.Phi, self.sigma, yhat, c.lam, c.r,
                                                          return_core=True)
            if s_all.shape[0] > c.r and s_all[0] > 0:
                self.min_gap = min(self.min_gap, (s_all[c.r - 1] - s_all[c.r]) / s_all[0])
        self.Phi, self.sigma = Phi_new, sigma_new
        if c.n_s > 0:
            self._refresh_sampling()
        self.a = self.Phi.T @ (self.d * (q_tilde - self.q_ref))
        self.events += 1

    def _adapt_instant(self, q_tilde):
        """Event of the instantaneous rules (App. A, and the note to Algorithm
        1 that they take the coarse-FOM step at the end of the loop): the basis
        update uses the correction snapshot already held, which approximates
        the state at the current time level; the state is transferred; then
        the coarse FOM advances that snapshot by z dt for the next event."""
        c = self.cfg
        yhat = self.d * (self.y_corr - self.q_ref)
        if self.rule == 3:
            self.Phi = onestep_update(self.Phi, yhat, self.a)
        elif self.rule == 4:
            self.Phi = oja_update(self.Phi, yhat, getattr(c, "learning_rate", 0.0))
        else:
            self.Phi = grouse_update(self.Phi, yhat, getattr(c, "learning_rate", 0.0))
        if c.n_s > 0:
            self._refresh_sampling()
        self.a = self.Phi.T @ (self.d * (q_tilde - self.q_ref))
        self.y_corr = self.coarse_step(self.y_corr)
        self.events += 1

    # -- driver --------------------------------------------------------------
    def step(self):
        """One iteration of the online loop; returns q~^{n+1} (before transfer)."""
        a_new, iters = self.rom_step(self.a)
        self.newton_iters.append(iters)
        self.a = a_new
        q_tilde = self.lifted()
        if self.is_event(self.n):
            self.adapt(q_tilde)
        self.n += 1
        return q_tilde

    def run(self, n_steps, record_every=1):
        """Run n_steps online steps; returns (steps, trajectory columns)."""
        steps, traj = [], []
        for k in range(n_steps):
            qt = self.step()
            if (k + 1) % record_every == 0 or k + 1 == n_steps:
                steps.append(self.n)
                traj.append(qt)
        return np.array(steps), np.stack(traj, axis=1)

    # -- state import / export ---------------------------------------------------
    def get_state(self):
        return dict(Phi=self.Phi.copy(), sigma=self.sigma.copy(), a=self.a.copy(),
                    y_corr=self.y_corr.copy(), n=self.n,
                    P=None if self.P is None else list(self.P))

    def set_state(self, Phi, sigma, a, y_corr, n, P=None):
        self.Phi = np.array(Phi, dtype=np.float64)
        self.sigma = np.array(sigma, dtype=np.float64)
        self.a = np.array(a, dtype=np.float64)
        self.y_corr = np.array(y_corr, dtype=np.float64)
        self.n = int(n)
        if self.cfg.n_s > 0:
            if P is None:
                self._refresh_sampling()
            else:
                self.P = list(P)
                self.M = sampled_pinv(self.Phi, self.P)


def relative_error(q_tilde, q_fom):
    """epsilon^n = ||q~ - q|| / ||q|| (Eq. relative_error)."""
    return float(np.linalg.norm(q_tilde - q_fom) / np.linalg.norm(q_fom))
