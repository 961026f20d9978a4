"""Pins of the oracle's reduced-order pieces: iSVD against batch SVD and the
covariance recursion, Galerkin/DEIM steps against the FOM in the full-basis
limit, QDEIM against brute-force greedy pivoting, and Algorithm 1's schedule
and qualitative behaviour (no GPU)."""
import copy

import numpy as np
import pytest

import synth
from oracle import fv, rom


def principal_angle_sin(A, B):
    """Largest sine of the principal angles between span(A) and span(B)."""
    Qa, _ = np.linalg.qr(A)
    Qb, _ = np.linalg.qr(B)
    return float(np.linalg.norm(Qb - Qa @ (Qa.T @ Qb), 2))


def low_rank_stream(n, rank, count, seed, decay=0.5):
    rng = np.random.default_rng(seed)
    B = np.linalg.qr(rng.standard_normal((n, rank)))[0]
    C = rng.standard_normal((rank, count)) * (decay ** np.arange(rank))[:, None]
    return B @ C


# ------------------------------------------------------------------ iSVD ---

@pytest.mark.parametrize("lam", [1.0, 0.5, 0.1])
def test_isvd_equals_batch_svd_of_weighted_history(lam):
    """Columns from a rank-5 matrix, r = 5: after every update the iSVD
    singular values equal those of the exponentially weighted snapshot matrix
    [lam^(k-1) y_1, ..., y_k] and the subspaces coincide (Eqs.
    weighted_snapshot_matrix, isvd_augmented_history)."""
    n, r, count = 60, 5, 25
    Y = low_rank_stream(n, r, count, seed=11)
    Phi, s = rom.pod(Y[:, :r], r)
    for k in range(r, count):
        Phi, s = rom.isvd_update(Phi, s, Y[:, k], lam, r)
        # the POD batch (first r columns) enters with one common weight
        w = lam ** np.minimum(np.arange(k, -1, -1), k - r + 1).astype(float)
        W = Y[:, :k + 1] * w[None, :]
        U, sb, _ = np.linalg.svd(W, full_matrices=False)
        nz = sb[:r] > rom.RANK_TOL * sb[0]
        assert np.allclose(s[nz], sb[:r][nz], rtol=1e-10, atol=1e-12 * sb[0])
        assert principal_angle_sin(Phi[:, nz], U[:, :r][:, nz]) < 1e-8


def test_isvd_rank_growing_equals_batch_svd():
    """lam = 1 and no truncation (target rank above the data count): the
    stream reproduces the thin SVD of the concatenated matrix exactly."""
    n, count = 40, 12
    rng = np.random.default_rng(3)
    Y = rng.standard_normal((n, count))
    Phi, s = rom.pod(Y[:, :1], 1)
    for k in range(1, count):
        Phi, s = rom.isvd_update(Phi, s, Y[:, k], 1.0, count)
    U, sb, _ = np.linalg.svd(Y, full_matrices=False)
    assert np.allclose(s, sb, rtol=1e-12)
    # columns equal up to sign
    sg = np.sign(np.sum(Phi * U, axis=0))
    assert np.max(np.abs(Phi * sg - U)) < 1e-9


def test_isvd_covariance_recursion():
    """Rank <= r: Phi Sigma^2 Phi^T tracks C_{k+1} = lam^2 C_k + y y^T."""
    n, r, lam = 30, 4, 0.7
    Y = low_rank_stream(n, r, 15, seed=5)
    Phi, s = rom.pod(Y[:, :r], r)
    C = Y[:, :r] @ Y[:, :r].T
    for k in range(r, 15):
        C = lam**2 * C + np.outer(Y[:, k], Y[:, k])
        Phi, s = rom.isvd_update(Phi, s, Y[:, k], lam, r)
        assert np.max(np.abs(Phi @ np.diag(s**2) @ Phi.T - C)) < 1e-10 * np.max(np.abs(C))


def test_isvd_keeps_orthonormality_over_many_updates():
    n, r = 48, 6
    rng = np.random.default_rng(9)
    Phi, s = rom.pod(rng.standard_normal((n, r)), r)
    for k in range(10000):
        Phi, s = rom.isvd_update(Phi, s, rng.standard_normal(n), 0.9, r)
    assert np.max(np.abs(Phi.T @ Phi - np.eye(r))) <= 1e-13


def test_isvd_transfer_identity():
    """Phi_new^T Phi_old a == U(1:r,1:r)^T a when q/||q|| is orthogonal to Phi."""
    n, r = 50, 5
    rng = np.random.default_rng(2)
    Phi, s = rom.pod(rng.standard_normal((n, r)), r)
    a = rng.standard_normal(r)
    y = rng.standard_normal(n)
    # iSVD without the sign normalisation, to compare with the raw U
    p, q = rom.project_cgs2(Phi, y)
    rho = np.linalg.norm(q)
    K = np.zeros((r + 1, r + 1))
    K[:r, :r] = 0.5 * np.diag(s)
    K[:r, r] = p
    K[r, r] = rho
    U, _, _ = np.linalg.svd(K)
    Phi_new = np.hstack([Phi, (q / rho)[:, None]]) @ U[:, :r]
    assert np.allclose(Phi_new.T @ (Phi @ a), U[:r, :r].T @ a, atol=1e-13)


def test_isvd_brute_force_tiny():
    """N = 4, r = 2: the update is the rank-2 truncation of the explicit
    4 x 3 matrix [lam Phi Sigma, y] (the factorisation of Eq. isvd_factorization)."""
    rng = np.random.default_rng(1)
    Phi, s = rom.pod(rng.standard_normal((4, 2)), 2)
    y = rng.standard_normal(4)
    lam = 0.3
    Phi2, s2 = rom.isvd_update(Phi, s, y, lam, 2)
    M = np.hstack([lam * Phi * s[None, :], y[:, None]])
    U, sb, _ = np.linalg.svd(M, full_matrices=False)
    assert np.allclose(s2, sb[:2], rtol=1e-13)
    assert principal_angle_sin(Phi2, U[:, :2]) < 1e-12


def test_isvd_empty_residual_keeps_span():
    n, r = 20, 3
    rng = np.random.default_rng(4)
    Phi, s = rom.pod(rng.standard_normal((n, r)), r)
    y = Phi @ rng.standard_normal(r)          # y in span(Phi): q = 0
    Phi2, s2 = rom.isvd_update(Phi, s, y, 0.5, r)
    assert principal_angle_sin(Phi2, Phi) < 1e-12
    assert np.max(np.abs(Phi2.T @ Phi2 - np.eye(r))) < 1e-13


def test_rank_truncation_zeroes_null_directions():
    n = 30
    rng = np.random.default_rng(6)
    X = rng.standard_normal((n, 2)) @ rng.standard_normal((2, 8))   # rank 2
    Phi, s = rom.pod(X, 5)
    assert np.count_nonzero(s) == 2
    assert np.all(Phi[:, 2:] == 0.0)
    assert rom.numerical_rank(Phi) == 2


# ------------------------------------------------------------ preprocess ---

def test_preprocess_hand_worked_three_variables():
    """Sec. 3.1, Eqs. scaling_matrix_local_block and variable_normalization,
    worked by hand on 2 cells, 3 variables (blocked [rho0 rho1 m0 m1 E0 E1]),
    2 snapshots. Centred on q_ref = q0, the blocks are
        rho: [1, 0], [0, 2]   squares 1 0 0 4   mean 5/4  -> D = 0.8
        m:   [1, 0], [0, 3]   squares 1 0 0 9   mean 10/4 -> D = 0.4
        E:   [0, 2], [2, 0]   squares 0 4 4 0   mean 2    -> D = 0.5
    The literals fail each plausible misreading: a mean over cells only
    (rho 0.4), the RMS instead of the mean square (rho 0.894, E 0.707),
    centring on the time mean instead of q_ref (rho 1.6), one mean over all
    variables (0.522 each) and an interleaved layout."""
    q0 = np.array([1.0, 2.0, 0.0, 0.0, 3.0, 4.0])
    Q = np.array([[2.0, 1.0],
                  [2.0, 4.0],
                  [1.0, 0.0],
                  [0.0, 3.0],
                  [3.0, 5.0],
                  [6.0, 4.0]])
    q_ref, d, Xhat = rom.preprocess(Q, q0, 3)
    assert np.array_equal(q_ref, q0)
    assert np.allclose(d, [0.8, 0.8, 0.4, 0.4, 0.5, 0.5], rtol=1e-15, atol=0)
    expected = np.array([[0.8, 0.0],
                         [0.0, 1.6],
                         [0.4, 0.0],
                         [0.0, 1.2],
                         [0.0, 1.0],
                         [1.0, 0.0]])
    assert np.allclose(Xhat, expected, rtol=1e-15, atol=1e-15)


def test_preprocess_constant_variable_is_left_unscaled():
    """A variable that never leaves q_ref has phi_v = 0; the guard takes
    D_v = 1 so that the block stays zero instead of becoming NaN."""
    q0 = np.array([1.0, 2.0, 5.0, 5.0])
    Q = np.array([[3.0, 1.0],
                  [2.0, 4.0],
                  [5.0, 5.0],
                  [5.0, 5.0]])
    _, d, Xhat = rom.preprocess(Q, q0, 2)
    # variable 0: centred [2, 0], [0, 2] -> mean square 2 -> D = 0.5; variable 1: no variation
    assert np.array_equal(d, [0.5, 0.5, 1.0, 1.0])
    assert np.array_equal(Xhat[2:], np.zeros((2, 2)))


def test_burgers_trajectory_invariant_under_scalar_scaling():
    """For a single variable D is a scalar; q~ does not depend on it."""
    cfg = synth.config_burgers_small()
    cfg.n_cells, cfg.n_online, cfg.w_init, cfg.r = 64, 40, 20, 4
    q0 = synth.initial_state(cfg)
    A = rom.AdaptiveROM(cfg, q0)
    B = rom.AdaptiveROM(cfg, q0, A.Q_train)
    B.d = B.d * 7.0
    B.sigma = B.sigma * 7.0
    B.a = B.a * 7.0
    for _ in range(cfg.n_online):
        qa, qb = A.step(), B.step()
        assert np.max(np.abs(qa - qb)) <= 1e-12 * np.max(np.abs(qa))


# ------------------------------------------------------------- ROM steps ---

def _full_basis_setup(n=24, seed=0):
    cfg = synth.config_burgers_small()
    cfg.n_cells = n
    rng = np.random.default_rng(seed)
    Phi = np.linalg.qr(rng.standard_normal((n, n)))[0]
    q_ref = synth.burgers_ic(n, seed)
    d = np.full(n, 3.0)
    return cfg, Phi, q_ref, d


def test_galerkin_full_basis_equals_fom_step():
    """r = N: the BE Galerkin ROM step is the FOM BE step."""
    cfg, Phi, q_ref, d = _full_basis_setup()
    q_prev = synth.burgers_ic(cfg.n_cells, 9)
    a_prev = Phi.T @ (d * (q_prev - q_ref))
    a, _ = rom.galerkin_step(a_prev, Phi, q_ref, d, cfg)
    q_fom = fv.be_step(q_prev, cfg.dt, 0, cfg.nu)
    assert np.max(np.abs(rom.lift(a, Phi, q_ref, d) - q_fom)) < 1e-12


def test_hyper_full_sampling_equals_fom_step():
    """r = n_s = N: DEIM with every cell sampled is the FOM BE step."""
    cfg, Phi, q_ref, d = _full_basis_setup(seed=1)
    P = list(np.random.default_rng(2).permutation(cfg.n_cells))
    M = rom.sampled_pinv(Phi, P)
    q_prev = synth.burgers_ic(cfg.n_cells, 4)
    a_prev = Phi.T @ (d * (q_prev - q_ref))
    a, _ = rom.hyper_step(a_prev, Phi, q_ref, d, P, M, cfg)
    q_fom = fv.be_step(q_prev, cfg.dt, 0, cfg.nu)
    assert np.max(np.abs(rom.lift(a, Phi, q_ref, d) - q_fom)) < 1e-11


def test_galerkin_jacobian_matches_finite_differences():
    cfg, _, q_ref, d = _full_basis_setup(n=32)
    Phi = synth.random_orthonormal(32, 5, 3)
    a0 = np.random.default_rng(5).standard_normal(5) * 0.1
    J = rom.galerkin_jacobian(a0, Phi, q_ref, d, cfg)
    g = lambda a: rom.galerkin_residual(a, a0, Phi, q_ref, d, cfg)
    Jfd = np.stack([(g(a0 + e) - g(a0 - e)) / 2e-7 for e in np.eye(5) * 1e-7], axis=1)
    assert np.max(np.abs(J - Jfd)) < 1e-7


# -------------------------------------------------------------- sampling ---

def brute_greedy_pivots(Phi, m):
    """Column-pivoted Gram-Schmidt on the rows of Phi (= columns of Phi^T):
    repeatedly take the row with the largest remaining norm and remove its
    direction from every row."""
    R = Phi.copy()
    out = []
    for _ in range(m):
        norms = np.sum(R * R, axis=1)
        norms[out] = -1.0
        i = int(np.argmax(norms))
        out.append(i)
        v = R[i] / np.linalg.norm(R[i])
        R = R - np.outer(R @ v, v)
    return out


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_qdeim_matches_brute_force_greedy(seed):
    Phi = synth.random_orthonormal(200, 8, seed)
    assert rom.qdeim(Phi, 8) == brute_greedy_pivots(Phi, 8)
    P = rom.qdeim(Phi, 8)
    M = rom.sampled_pinv(Phi, P)
    assert np.allclose(M @ Phi[P, :], np.eye(8), atol=1e-12)


def test_fgs_greedy_order_and_ties():
    y = np.array([0.0, 1.0, 1.0, 3.0, 3.0, 2.0, 0.0, 0.0])
    # forward differences: 1, 0, 2, 0, -1, -2, 0, 0 -> squares 1,0,4,0,1,4,0,0
    assert rom.fgs_extend(y, [], 4) == [2, 5, 0, 4]
    assert rom.fgs_extend(y, [5], 2) == [2, 0]


def test_sample_points_oversample_to_ns():
    Phi = synth.random_orthonormal(100, 4, 1)
    y = np.sin(np.linspace(0, 6, 100))
    P = rom.sample_points(Phi, y, 12)
    assert len(P) == 12 and len(set(P)) == 12
    assert P[:4] == rom.qdeim(Phi, 12)


# ------------------------------------------------------------ Algorithm 1 ---

def small_cfg(n_online=200):
    cfg = synth.config_burgers_small()
    cfg.n_cells, cfg.n_online = 128, n_online
    return cfg


def test_event_schedule():
    cfg = small_cfg(95)
    m = rom.AdaptiveROM(cfg, synth.initial_state(cfg))
    m.run(cfg.n_online, record_every=1000)
    assert m.events == cfg.n_online // cfg.z
    assert m.n == cfg.w_init + cfg.n_online


def test_adaptive_rom_beats_correction_signal_and_static_rom():
    """Qualitative claims of Sec. 5.1: the adaptive ROM stays close to the
    fine FOM, closer than the coarse correction signal that informs it, and
    far closer than the static ROM."""
    cfg = small_cfg(600)
    q0 = synth.initial_state(cfg)
    # the correction snapshot runs z steps ahead of the ROM
    Q = rom.fom_trajectory(q0, cfg.w_init + cfg.n_online + cfg.z, cfg)
    A = rom.AdaptiveROM(cfg, q0, Q[:, :cfg.w_init])
    S = rom.AdaptiveROM(cfg, q0, Q[:, :cfg.w_init])
    S.is_event = lambda n: False
    for _ in range(cfg.n_online):
        qa, qs = A.step(), S.step()
    q_true = Q[:, A.n - 1]
    e_rom = rom.relative_error(qa, q_true)
    e_sig = rom.relative_error(A.y_corr, Q[:, A.n - 1 + cfg.z])
    e_static = rom.relative_error(qs, q_true)
    assert e_rom < 1e-3
    assert e_rom < e_sig
    assert e_static > 10 * e_rom


def test_trajectory_insensitive_to_rounding_with_rank_tolerance():
    """With the numerical-rank tolerance, perturbing every correction snapshot
    at the rounding level (1e-16 relative) moves the trajectory by far less
    than the 1e-10 parity tolerance."""
    cfg = small_cfg(300)
    q0 = synth.initial_state(cfg)
    A = rom.AdaptiveROM(cfg, q0)
    B = rom.AdaptiveROM(cfg, q0, A.Q_train)
    rng = np.random.default_rng(7)
    orig = rom.project_cgs2
    worst = 0.0
    try:
        for _ in range(cfg.n_online):
            qa = A.step()
            rom.project_cgs2 = lambda P, y: orig(P, y * (1 + 1e-16 * rng.standard_normal(y.shape)))
            qb = B.step()
            rom.project_cgs2 = orig
            worst = max(worst, np.linalg.norm(qa - qb) / np.linalg.norm(qa))
    finally:
        rom.project_cgs2 = orig
    assert worst < 1e-11


@pytest.mark.parametrize("lam", [1.0, 0.5])
def test_basis_path_equals_batch_svd_of_weighted_snapshots(lam):
    """The correction states follow the coarse FOM alone (Algorithm 1), so
    while no direction is truncated the basis after k events spans the leading
    directions of the weighted matrix
    [lam^k Xhat, lam^(k-1) yhat_2, ..., yhat_(k+1)], yhat_j = D (y_j - q_ref),
    y_j = j coarse BE steps from the last training state (the offline stage
    makes y_1; event j advances to y_(j+1) and feeds it; Eqs.
    weighted_snapshot_matrix, isvd_augmented_history), and the singular values
    are that matrix's."""
    cfg = small_cfg(40)
    cfg.n_cells, cfg.w_init, cfg.z, cfg.lam, cfg.r = 96, 12, 5, lam, 40
    q0 = synth.initial_state(cfg)
    m = rom.AdaptiveROM(cfg, q0)
    q_ref, d, Xhat = rom.preprocess(m.Q_train, q0, 1)
    y = m.Q_train[:, -1]
    cols = []
    for _ in range(cfg.n_online):
        m.step()
    for _ in range(m.events + 1):          # y_1 .. y_(k+1)
        y = fv.be_step(y, cfg.z * cfg.dt, 0, cfg.nu, cfg.gamma, cfg.newton_tol, cfg.newton_max)
        cols.append(d * (y - q_ref))
    k = m.events
    assert k == 8
    W = np.hstack([lam ** k * Xhat] + [lam ** (k - j) * cols[j][:, None] for j in range(1, k + 1)])
    U, s, _ = np.linalg.svd(W, full_matrices=False)
    live = s > 1e-8 * s[0]                 # safely above the rank tolerance
    n_live = int(np.count_nonzero(live))
    assert n_live <= rom.numerical_rank(m.Phi) < cfg.r
    # measured: 4e-16 s_1 and 1e-8 (the last compared direction is 4x above the next)
    assert np.allclose(m.sigma[:n_live], s[:n_live], rtol=0, atol=1e-12 * s[0])
    assert principal_angle_sin(m.Phi[:, :n_live], U[:, :n_live]) < 1e-6


# ------------------------------------------------------------------- LSPG ---

def test_lspg_with_a_full_basis_is_the_fom_step():
    """r = N: the trial manifold is the whole space, the minimum of |D r| is
    zero and the LSPG step (Eq. lspg_minimization) is the backward-Euler FOM
    step (Eq. be_residual_rom_section), solved here by the FOM's own Newton
    with a sparse LU."""
    n = 48
    cfg = synth.config_burgers_small()
    cfg.n_cells, cfg.r, cfg.dt, cfg.nu = n, n, 1e-3, 0.01
    q_prev = synth.burgers_ic(n, 5)
    q_ref = synth.burgers_ic(n, 6)
    d = np.full(n, 2.5)
    Phi = synth.random_orthonormal(n, n, 3)
    a_prev = Phi.T @ (d * (q_prev - q_ref))
    a, _ = rom.lspg_step(a_prev, Phi, q_ref, d, cfg)
    q_fom = fv.be_step(q_prev, cfg.dt, 0, cfg.nu)
    assert np.max(np.abs(rom.lift(a, Phi, q_ref, d) - q_fom)) <= 1e-12 * np.max(np.abs(q_fom))


def test_lspg_step_of_a_nearly_linear_operator_is_the_least_squares_solution():
    """Near u = 0 the Burgers operator is the viscous term nu L (the flux is
    quadratic in u, here 1e-3 of the diffusion), so the LSPG step is the
    linear least-squares problem min |(I - dt nu L) Phi a - Phi a_prev|:
    Gauss-Newton must reach the solution the normal equations give directly
    (to the size of the neglected flux), which differs from the Galerkin
    solution Phi^T (I - dt nu L) Phi a = a_prev."""
    n, r = 64, 6
    cfg = synth.config_burgers_small()
    cfg.n_cells, cfg.r, cfg.dt, cfg.nu = n, r, 5e-4, 0.02
    Phi = synth.random_orthonormal(n, r, 8)
    q_ref = np.zeros(n)
    d = np.ones(n)
    a_prev = np.random.default_rng(2).standard_normal(r) * 1e-3
    L = (np.roll(np.eye(n), 1, axis=0) - 2 * np.eye(n) + np.roll(np.eye(n), -1, axis=0)) * n * n
    A = np.eye(n) - cfg.dt * cfg.nu * L
    a_ls = np.linalg.solve((A @ Phi).T @ (A @ Phi), (A @ Phi).T @ (Phi @ a_prev))
    a, _ = rom.lspg_step(a_prev, Phi, q_ref, d, cfg)
    assert np.max(np.abs(a - a_ls)) <= 1e-4 * np.max(np.abs(a_ls))
    a_g = np.linalg.solve(Phi.T @ A @ Phi, a_prev)
    assert np.max(np.abs(a_g - a_ls)) > 1e-3 * np.max(np.abs(a_ls))


def test_hyper_reduced_lspg_equals_deim_galerkin():
    """With the DEIM basis equal to the trial basis and P^T Phi of full column
    rank, (P^T Phi)^+ P^T Phi = I, so the hyper-reduced LSPG objective
    |(P^T Phi)^+ P^T D r| (Eq. hyperreduced_lspg) is the norm of the
    DEIM-Galerkin residual (Eq. deim_galerkin_rom) and its Gauss-Newton
    matrix is that residual's square Jacobian: the minimiser is the
    DEIM-Galerkin root."""
    cfg = synth.config_burgers_hyper()
    cfg.n_cells, cfg.r, cfg.n_s = 512, 8, 24
    q0 = synth.initial_state(cfg)
    m = rom.AdaptiveROM(cfg, q0)
    for _ in range(7):
        m.step()
    a_g, _ = rom.hyper_step(m.a, m.Phi, m.q_ref, m.d, m.P, m.M, cfg)
    a_l, _ = rom.hyper_lspg_step(m.a, m.Phi, m.q_ref, m.d, m.P, m.M, cfg)
    assert np.max(np.abs(a_l - a_g)) <= 1e-11 * np.max(np.abs(a_g))


def test_sod_lspg_qdeim_is_the_deim_galerkin_model():
    """The same identity on the Euler system at the Sod ROM's dimensions
    (Sec. 5.2: LSPG-QDEIM with r = n_s = w_init = 4, 256 cells): over the
    whole horizon to t = 0.2 the adaptive LSPG-QDEIM model and the adaptive
    DEIM-Galerkin model give the same states, every step converging."""
    out = {}
    for proj in (1, 0):
        cfg = synth.config_sod(256)
        cfg.r = cfg.n_s = cfg.w_init = 4
        cfg.projection = proj
        m = rom.AdaptiveROM(cfg, synth.initial_state(cfg))
        m.run(cfg.n_online, record_every=10 ** 6)
        out[proj] = m.lifted()
    assert np.all(np.isfinite(out[1]))
    assert np.max(np.abs(out[1] - out[0])) <= 1e-12 * np.max(np.abs(out[0]))


def test_lspg_and_galerkin_agree_as_dt_vanishes():
    """LSPG tests the residual with Psi = Phi - dt D J_f D^-1 Phi, Galerkin
    with Phi; the two steps from the same state differ at least at second
    order in dt (more here, where f is nearly in span(Phi) right after
    training): halving dt divides the difference by at least three."""
    cfg = synth.config_burgers_small()
    q0 = synth.initial_state(cfg)
    m = rom.AdaptiveROM(cfg, q0)
    diffs = []
    for dt in (4e-4, 2e-4, 1e-4):
        c = copy.copy(cfg)
        c.dt = dt
        a_g, _ = rom.galerkin_step(m.a, m.Phi, m.q_ref, m.d, c)
        a_l, _ = rom.lspg_step(m.a, m.Phi, m.q_ref, m.d, c)
        diffs.append(np.linalg.norm(a_g - a_l))
    assert diffs[0] / diffs[1] > 3.0 and diffs[1] / diffs[2] > 3.0, diffs
    assert diffs[2] > 0.0


def test_lspg_adaptive_rom_runs_and_tracks_the_fom():
    """Algorithm 1 with the LSPG step (plain projection): the ROM error
    against the fine FOM stays of the size the Galerkin ROM reaches."""
    cfg = synth.config_burgers_small()
    cfg.n_cells, cfg.n_online = 256, 300
    q0 = synth.initial_state(cfg)
    res = {}
    for proj in (0, 1):
        c = copy.copy(cfg)
        c.projection = proj
        m = rom.AdaptiveROM(c, q0)
        q = m.Q_train[:, -1]
        for _ in range(cfg.n_online):
            qt = m.step()
            q = fv.be_step(q, c.dt, 0, c.nu)
        res[proj] = rom.relative_error(qt, q)
    assert res[1] < 5 * res[0] + 1e-6, res


# ------------------------------------------------- comparison update rules ---

def test_windowed_svd_equals_the_rank_growing_isvd_of_the_window():
    """Eq. wsvd_update by LAPACK against the same window fed column by column
    through the iSVD with lambda = 1 and no truncation (Algorithm 2 in its
    rank-growing mode reproduces the thin SVD of the concatenated columns):
    same singular values and subspace."""
    rng = np.random.default_rng(12)
    n, w, r = 80, 12, 5
    Y = low_rank_stream(n, 9, w, seed=13) + 1e-3 * rng.standard_normal((n, w))
    Phi_w, s_w = rom.windowed_svd_update(Y, r)
    Phi, s = rom.pod(Y[:, :1], 1)
    for j in range(1, w):
        Phi, s = rom.isvd_update(Phi, s, Y[:, j], 1.0, w)
    assert np.allclose(s_w, s[:r], rtol=1e-10)
    assert principal_angle_sin(Phi_w, Phi[:, :r]) < 1e-8


def test_direct_update_minimises_its_objective_and_keeps_a_fitted_span():
    """Eq. direct_optimization: X = Y (Phi^+ Y)^+ minimises |X Phi^+ Y - Y|_F,
    so random perturbations of X never lower it; and a window inside
    span(Phi) of full rank r leaves that span unchanged."""
    rng = np.random.default_rng(21)
    n, w, r = 60, 8, 4
    Phi = synth.random_orthonormal(n, r, 22)
    Y = rng.standard_normal((n, w))
    C = Phi.T @ Y
    X = Y @ np.linalg.pinv(C)
    f0 = np.linalg.norm(X @ C - Y)
    for _ in range(20):
        Xp = X + 1e-3 * rng.standard_normal(X.shape)
        assert np.linalg.norm(Xp @ C - Y) >= f0
    Yin = Phi @ rng.standard_normal((r, w))
    Phi_new, s = rom.direct_update(Phi, Yin, r)
    assert np.count_nonzero(s) == r
    assert principal_angle_sin(Phi_new, Phi) < 1e-12
    assert np.max(np.abs(Phi_new.T @ Phi_new - np.eye(r))) < 1e-13


def test_window_of_the_comparison_rules_holds_the_last_snapshots():
    """App. A: the window starts as the last w training snapshots and at every
    event drops the oldest and appends the new preprocessed correction
    snapshot."""
    cfg = synth.config_burgers_small()
    cfg.n_cells, cfg.w_init, cfg.r, cfg.z = 128, 20, 4, 5
    cfg.update_rule, cfg.window = 2, 6
    q0 = synth.initial_state(cfg)
    m = rom.AdaptiveROM(cfg, q0)
    expect = [m.d * (m.Q_train[:, j] - m.q_ref) for j in range(14, 20)]
    assert np.array_equal(m.window, np.stack(expect, axis=1))
    snaps = []
    for _ in range(3 * cfg.z):
        m.step()
        if m.is_event(m.n - 1):
            snaps.append(m.d * (m.y_corr - m.q_ref))
    expect = expect[3:] + snaps
    assert np.array_equal(m.window, np.stack(expect, axis=1))


@pytest.mark.parametrize("rule", [1, 2])
def test_comparison_rules_track_the_fom(rule):
    """Algorithm 1 with the windowed-SVD and Direct updates stays close to the
    fine FOM over 300 steps (history-aware rules, App. A)."""
    cfg = synth.config_burgers_small()
    cfg.n_cells, cfg.n_online, cfg.r = 256, 300, 6
    cfg.update_rule, cfg.window = rule, 16
    q0 = synth.initial_state(cfg)
    m = rom.AdaptiveROM(cfg, q0)
    q = m.Q_train[:, -1]
    for _ in range(cfg.n_online):
        qt = m.step()
        q = fv.be_step(q, cfg.dt, 0, cfg.nu)
    assert rom.relative_error(qt, q) < 1e-2
