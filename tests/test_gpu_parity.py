"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs.

Tolerances. Operator, FOM step and per-step checks: relative 1e-12 .. 1e-10
(FP64 with the FP64 residual deciding every Newton root). Whole trajectories:
relative L2 1e-10 at every recorded step; the oracle's own sensitivity to
rounding-level perturbations stays below 1e-11 over these horizons (see
test_oracle_rom.test_trajectory_insensitive_to_rounding_with_rank_tolerance).
Singular values: absolute 1e-12 sigma_1. Basis columns are compared after
aligning signs (singular vectors are unique up to sign)."""
import numpy as np
import pytest

import synth
from oracle import fv, rom as orom

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


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def assert_basis_close(P_g, P_or, sigma, tol=1e-9, floor=1e-14):
    """Columns of two bases agree up to sign, each within the accuracy its
    singular-value gap allows (a singular vector is determined to about
    floor / gap, floor = eps * sigma_1 relative for a rounding-level
    perturbation)."""
    nz = sigma > 0
    Pa = align_columns(P_g[:, nz], P_or[:, nz])
    s = sigma[nz]
    gaps = np.abs(np.diff(np.concatenate([[np.inf], s, [0.0]])))
    gap = np.minimum(gaps[:-1], gaps[1:]) / sigma[0]
    for j in range(s.shape[0]):
        allowed = max(tol, floor / gap[j])
        assert np.max(np.abs(Pa[:, j] - P_or[:, nz][:, j])) <= allowed, (j, gap[j])


def align_columns(A, B):
    """Flip the columns of A to match the signs of B's."""
    s = np.sign(np.sum(A * B, axis=0))
    s[s == 0] = 1.0
    return A * s


# ------------------------------------------------------------------ FOM ---

@pytest.mark.parametrize("n", [512, 2053, 16384, 65536])
def test_fom_rhs_parity(g, n):
    q = synth.burgers_ic(n, 3)
    q[n // 3: n // 3 + 5] = -0.5          # both Godunov branches
    qd = torch.tensor(q, device="cuda", dtype=torch.float64)
    fd = torch.empty_like(qd)
    g.fom_rhs_dev(0, n, 0.01, 1.4, qd.data_ptr(), fd.data_ptr())
    f_or = fv.burgers_f(q, 0.01)
    assert np.max(np.abs(fd.cpu().numpy() - f_or)) <= 1e-13 * np.max(np.abs(f_or))


@pytest.mark.parametrize("n,h,nu", [(512, 1e-3, 0.01), (2053, 5e-4, 2e-3), (8192, 5e-4, 2e-3),
                                    (12000, 5e-4, 2e-3), (16384, 5e-4, 2e-3),
                                    (65536, 1e-3, 5e-3), (100, 1e-2, 0.01)])
def test_fom_be_step_parity(g, n, h, nu):
    q0 = synth.burgers_ic(n, 7)
    qp = torch.tensor(q0, device="cuda", dtype=torch.float64)
    qn = torch.empty_like(qp)
    iters = g.fom_step_dev(0, n, nu, 1.4, h, 1e-12, 20, qp.data_ptr(), qn.data_ptr())
    q_or = fv.be_step(q0, h, 0, nu)
    q_gpu = qn.cpu().numpy()
    assert 1 <= iters <= 20
    assert np.max(np.abs(q_gpu - q_or)) <= 1e-11 * np.max(np.abs(q_or))
    assert abs(q_gpu.sum() - q0.sum()) <= 1e-11 * abs(q0.sum())      # mass


def test_fom_nonconvergence_reported(g):
    n = 1024
    q0 = synth.burgers_ic(n, 1)
    qp = torch.tensor(q0, device="cuda", dtype=torch.float64)
    qn = torch.empty_like(qp)
    with pytest.raises(g.RomError) as ei:
        g.fom_step_dev(0, n, 0.01, 1.4, 1e-3, 1e-30, 1, qp.data_ptr(), qn.data_ptr())
    assert ei.value.code == 4


# ----------------------------------------------------------------- iSVD ---

def _isvd_case(n, r, k, seed, lam, in_span=False):
    rng = np.random.default_rng(seed)
    Phi = np.zeros((n, r))
    Phi[:, :k] = synth.random_orthonormal(n, k, seed)
    sigma = np.zeros(r)
    sigma[:k] = np.sort(rng.uniform(0.5, 3.0, k))[::-1] * 10.0 ** -np.arange(k)
    if in_span:
        y = Phi[:, :k] @ rng.standard_normal(k)
    else:
        y = Phi[:, :k] @ rng.standard_normal(k) + 0.1 * rng.standard_normal(n)
    return Phi, sigma, y


@pytest.mark.parametrize("n,r,k,lam,in_span", [
    (4096, 10, 10, 0.1, False), (4096, 10, 6, 0.5, False), (5000, 32, 32, 1.0, False),
    (20000, 64, 40, 0.01, False), (3000, 8, 8, 0.3, True), (2048, 16, 1, 0.0, False),
    (4099, 48, 48, 1e-7, False)])
def test_isvd_update_parity(g, n, r, k, lam, in_span):
    Phi, sigma, y = _isvd_case(n, r, k, seed=n + r + k, lam=lam, in_span=in_span)
    P_or, s_or = orom.isvd_update(Phi[:, :k], sigma[:k], y, lam, r)
    kk = P_or.shape[1]
    Pd = torch.tensor(Phi.T.copy(), device="cuda")          # column-major N x r
    sd = torch.tensor(sigma, device="cuda")
    yd = torch.tensor(y, device="cuda")
    g.isvd_update_dev(n, r, lam, 1e-10, Pd.data_ptr(), sd.data_ptr(), yd.data_ptr())
    P_g = Pd.cpu().numpy().T
    s_g = sd.cpu().numpy()
    s_full = np.zeros(r)
    s_full[:kk] = s_or
    assert np.max(np.abs(s_g - s_full)) <= 1e-12 * s_full[0]
    nz = s_full > 0
    P_full = np.zeros((n, r))
    P_full[:, :kk] = P_or
    assert np.all(P_g[:, ~nz] == 0.0)
    Pa = align_columns(P_g[:, nz], P_full[:, nz])
    # columns with a healthy relative gap are unique: compare them entry-wise
    gaps = np.abs(np.diff(np.concatenate([[np.inf], s_full[nz], [0.0]])))
    gap = np.minimum(gaps[:-1], gaps[1:]) / s_full[0]
    good = gap > 1e-6
    assert np.max(np.abs(Pa[:, good] - P_full[:, nz][:, good])) <= 1e-9
    assert np.max(np.abs(P_g[:, nz].T @ P_g[:, nz] - np.eye(int(nz.sum())))) <= 1e-13


# ------------------------------------------------------------- ROM runs ---

def test_burgers_small_config_full_trajectory(g):
    """Burgers N=512, r=10, z=10, lambda=0.1, 2000 online steps."""
    cfg = synth.config_burgers_small()
    q0 = synth.initial_state(cfg)
    ref = orom.AdaptiveROM(cfg, q0)
    gpu = g.AdaptiveROM(cfg, q0)
    st = gpu.state()
    assert st["step"] == cfg.w_init
    assert np.max(np.abs(st["sigma"] - ref.sigma)) <= 1e-12 * ref.sigma[0]
    assert rel(st["q_tilde"], ref.lifted()) <= 1e-12
    worst = 0.0
    for block in range(cfg.n_online // 100):
        for _ in range(100):
            q_or = ref.step()
        gpu.step(100)
        # the last step of each block of 100 is an event (z = 10): compare q~
        # after the transfer with the oracle's lifted state
        worst = max(worst, rel(gpu.q_tilde(), ref.lifted()))
    st = gpu.state()
    assert worst <= 1e-10, worst
    assert np.max(np.abs(st["sigma"] - ref.sigma)) <= 1e-10 * ref.sigma[0]
    assert gpu.info()["rank"] == orom.numerical_rank(ref.Phi)
    gpu.close()


def test_single_step_from_loaded_state(g):
    """Load the oracle's state after 337 steps, advance one step (no event) and
    then to the next event: the reduced step and the event agree to 1e-10."""
    cfg = synth.config_burgers_small()
    cfg.n_cells = 1024
    q0 = synth.initial_state(cfg)
    ref = orom.AdaptiveROM(cfg, q0)
    for _ in range(337):
        ref.step()
    gpu = g.AdaptiveROM(cfg, q0)
    s = ref.get_state()
    gpu.load_state(s["Phi"], ref.sigma, s["a"], s["y_corr"], s["n"])
    q_or = ref.step()
    gpu.step(1)
    assert rel(gpu.q_tilde(), q_or) <= 1e-12
    while not ref.is_event(ref.n):
        ref.step()
        gpu.step(1)
    ref.step()                 # event step
    gpu.step(1)
    st = gpu.state()
    assert rel(st["q_tilde"], ref.lifted()) <= 1e-11
    assert rel(st["y_corr"], ref.y_corr) <= 1e-12
    assert np.max(np.abs(st["sigma"] - ref.sigma)) <= 1e-11 * ref.sigma[0]
    gpu.close()


def test_update_basis_with_host_snapshot(g):
    cfg = synth.config_burgers_small()
    q0 = synth.initial_state(cfg)
    ref = orom.AdaptiveROM(cfg, q0)
    gpu = g.AdaptiveROM(cfg, q0)
    y = synth.burgers_ic(cfg.n_cells, 11) * 0.2 + ref.Q_train[:, -1] * 0.8
    # oracle: the event with y as the correction snapshot
    ref.coarse_step = lambda yy: y
    ref.adapt(ref.lifted())
    gpu.update_basis(y)
    st = gpu.state()
    assert rel(st["q_tilde"], ref.lifted()) <= 1e-12
    assert np.max(np.abs(st["sigma"] - ref.sigma)) <= 1e-12 * ref.sigma[0]
    assert_basis_close(st["phi"], ref.Phi, ref.sigma)
    gpu.close()


def test_checkpoint_resume_bit_exact(g):
    cfg = synth.config_burgers_small()
    q0 = synth.initial_state(cfg)
    a = g.AdaptiveROM(cfg, q0)
    b = g.AdaptiveROM(cfg, q0)
    a.step(123)
    st = a.state()
    b.load_state(st["phi"], st["sigma"], st["a"], st["y_corr"], st["step"])
    a.step(200)
    b.step(200)
    assert np.array_equal(a.q_tilde(), b.q_tilde())
    a.close()
    b.close()


def greedy_residuals(Phi, order):
    """Remaining squared row norms before each pick of a greedy pivot sequence."""
    R = Phi.copy()
    out = []
    for p in order:
        norms = np.sum(R * R, axis=1)
        out.append(norms.copy())
        v = R[p] / np.linalg.norm(R[p])
        R = R - np.outer(R @ v, v)
    return out


def adopt_if_near_tie(ref, gpu, rtol=1e-10):
    """Sampling decisions are argmax / top-m choices. The trailing basis
    directions (singular values near the rank tolerance) are determined only
    to about eps * sigma_1 / gap (~1e-7), and QDEIM weighs every column
    equally, so two correct implementations can pick different cells where
    the top candidates differ by less than that. Check that every GPU
    decision is valid for the GPU's own inputs (its exported basis and
    correction snapshot) to rounding level in FP64, then continue the oracle
    with the GPU's set. Returns the number of differing cells."""
    gpu_P = [int(i) for i in gpu.samples()]
    if sorted(gpu_P) == sorted(ref.P):
        return 0
    st = gpu.state()
    kq = min(gpu.info()["rank"], ref.cfg.n_s)
    res = greedy_residuals(st["phi"][:, :kq], gpu_P[:kq])
    for j, p in enumerate(gpu_P[:kq]):
        norms = res[j]
        norms[gpu_P[:j]] = -1.0
        assert norms[p] >= (1 - rtol) * norms.max(), ("QDEIM pivot", j, p)
    g = orom.fgs_scores(st["y_corr"], ref.cfg.problem, ref.cfg.gamma)
    g[gpu_P[:kq]] = -1.0
    m = ref.cfg.n_s - kq
    thr = np.sort(g)[::-1][m - 1]
    for p in gpu_P[kq:]:
        assert g[p] >= (1 - rtol) * thr, ("feature point", p, g[p], thr)
    ndiff = len(set(gpu_P) ^ set(ref.P))
    ref.P = gpu_P
    ref.M = orom.sampled_pinv(ref.Phi, ref.P)
    return ndiff


@pytest.mark.parametrize("n_cells,n_steps", [(2048, 400), (16384, 100)])
def test_hyper_reduced_trajectory(g, n_cells, n_steps):
    """DEIM-Galerkin (r=32, n_s=96, z=5, lambda=0.5): same sample sets at
    every event and the trajectory within 1e-10."""
    cfg = synth.config_burgers_hyper()
    cfg.n_cells = n_cells
    q0 = synth.initial_state(cfg)
    ref = orom.AdaptiveROM(cfg, q0)
    gpu = g.AdaptiveROM(cfg, q0)
    adopt_if_near_tie(ref, gpu)
    worst = 0.0
    for k in range(n_steps // cfg.z):
        for _ in range(cfg.z):
            ref.step()
        gpu.step(cfg.z)
        adopt_if_near_tie(ref, gpu)
        worst = max(worst, rel(gpu.q_tilde(), ref.lifted()))
    assert worst <= 1e-10, worst
    gpu.close()


def test_reduced_newton_nonconvergence_reported(g):
    cfg = synth.config_burgers_small()
    cfg.newton_max, cfg.newton_tol = 1, 1e-300
    q0 = synth.initial_state(cfg)
    with pytest.raises(g.RomError) as ei:
        gpu = g.AdaptiveROM(cfg, q0)          # FOM Newton cannot converge in 1 iteration
    assert ei.value.code == 4


@pytest.mark.parametrize("hyper,n_cells,n_steps", [(True, 2048, 400), (True, 16384, 100),
                                                   (False, 512, 2000)])
def test_mixed_precision_against_fp64_oracle(g, hyper, n_cells, n_steps):
    """Mixed form (FP32 basis, FP32 projections with FP32 accumulation, FP64
    core SVD and re-orthonormalisation) against two FP64 oracles:

    * parity: the oracle run with the mixed form's numerical-rank tolerance
      (1e-5, what FP32 projections resolve), relative L2 of q~ within 1e-5 at
      every event;
    * error against the FP64 form: the oracle with the FP64 form's tolerance
      (1e-10). The mixed form must lie within the distance that the rank
      tolerance alone puts between the two oracles, plus 1e-5; that distance
      (8.1e-4 at N = 512 over 2000 steps, 3.6e-5 and 4.4e-6 on the DEIM cases)
      is above the 1e-5 target, so the mixed form does not reach the FP64
      form's accuracy."""
    cfg = synth.config_burgers_hyper() if hyper else synth.config_burgers_small()
    cfg.n_cells = n_cells
    cfg.precision = 1
    q0 = synth.initial_state(cfg)
    saved = orom.RANK_TOL
    try:
        orom.RANK_TOL = 1e-5
        ref = orom.AdaptiveROM(cfg, q0)
        orom.RANK_TOL = 1e-10
        ref64 = orom.AdaptiveROM(cfg, q0)
        gpu = g.AdaptiveROM(cfg, q0)
        if hyper:
            orom.RANK_TOL = 1e-5
            adopt_if_near_tie(ref, gpu, rtol=1e-6)
        worst = worst64 = gap = 0.0
        for _ in range(n_steps // cfg.z):
            orom.RANK_TOL = 1e-5
            for _ in range(cfg.z):
                ref.step()
            orom.RANK_TOL = 1e-10
            for _ in range(cfg.z):
                ref64.step()
            gpu.step(cfg.z)
            orom.RANK_TOL = 1e-5
            if hyper:
                adopt_if_near_tie(ref, gpu, rtol=1e-6)
            qg = gpu.q_tilde()
            worst = max(worst, rel(qg, ref.lifted()))
            worst64 = max(worst64, rel(qg, ref64.lifted()))
            gap = max(gap, rel(ref.lifted(), ref64.lifted()))
    finally:
        orom.RANK_TOL = saved
    st = gpu.state()
    P = st["phi"][:, st["sigma"] > 0]
    assert np.max(np.abs(P.T @ P - np.eye(P.shape[1]))) <= 1e-6     # FP32 basis stays orthonormal
    assert gpu.info()["rank"] == orom.numerical_rank(ref.Phi)
    print(f"mixed form N={n_cells}: vs oracle (tau 1e-5) {worst:.2e}; vs FP64 oracle (tau 1e-10) "
          f"{worst64:.2e}; oracle tau gap {gap:.2e}")
    assert worst <= 1e-5, worst
    assert worst64 <= gap + 1e-5, (worst64, gap)
    gpu.close()


@pytest.mark.parametrize("n_cells", [256, 300, 777])
def test_offline_pod_matches_batch_svd(g, n_cells):
    """The offline stage (training FOM, scaling, POD grown one snapshot at a
    time by the iSVD) against the oracle's batch SVD of the whole training
    matrix: singular values and basis. N = 300 with this seed once let a
    rounding-level direction into the growing basis."""
    cfg = synth.RomConfig(problem=synth.BURGERS, n_cells=n_cells, r=8, n_s=0, w_init=100, z=5,
                          dt=1e-4, nu=4e-3, lam=0.5, seed=2000)
    q0 = synth.initial_state(cfg)
    ref = orom.AdaptiveROM(cfg, q0)
    gpu = g.AdaptiveROM(cfg, q0)
    st = gpu.state()
    k = orom.numerical_rank(ref.Phi)
    assert gpu.info()["rank"] == k
    assert np.max(np.abs(st["sigma"][:k] - ref.sigma[:k])) <= 1e-10 * ref.sigma[0]
    # the growing POD drops content below 1e-13 sigma_1 at each of the 100
    # updates (<= 1e-12 sigma_1 in all), so a singular vector is fixed to about
    # 1e-12 sigma_1 / gap, short of the batch SVD's rounding-level 1e-14 / gap
    assert_basis_close(st["phi"][:, :k], ref.Phi[:, :k], ref.sigma[:k], tol=1e-8, floor=1e-11)
    P = st["phi"][:, :k]
    assert np.max(np.abs(P.T @ P - np.eye(k))) <= 1e-12
    gpu.close()


# ------------------------------------------------------------------- LSPG ---

@pytest.mark.parametrize("n_cells,n_steps", [(512, 1000), (2053, 300)])
def test_lspg_trajectory_against_oracle(g, n_cells, n_steps):
    """Algorithm 1 with the LSPG step (Eq. lspg_minimization, test basis of Eq.
    lspg_test_basis_be; Gauss-Newton in FP64) against the oracle's
    Gauss-Newton: q~ within 1e-10 at every event, and different from the
    Galerkin trajectory."""
    cfg = synth.config_burgers_small()
    cfg.n_cells, cfg.projection = n_cells, 1
    q0 = synth.initial_state(cfg)
    ref = orom.AdaptiveROM(cfg, q0)
    gpu = g.AdaptiveROM(cfg, q0)
    worst = 0.0
    for _ in range(n_steps // cfg.z):
        for _ in range(cfg.z):
            ref.step()
        gpu.step(cfg.z)
        worst = max(worst, rel(gpu.q_tilde(), ref.lifted()))
    gal_cfg = synth.config_burgers_small()
    gal_cfg.n_cells = n_cells
    gal = g.AdaptiveROM(gal_cfg, q0)
    gal.step(n_steps)
    diff = rel(gal.q_tilde(), gpu.q_tilde())
    print(f"LSPG N={n_cells}: worst error {worst:.2e}; LSPG vs Galerkin {diff:.2e}; "
          f"Gauss-Newton iterations {gpu.info()['rom_newton_iters']}")
    assert worst <= 1e-10, worst
    assert diff > 1e-9
    gal.close()
    gpu.close()


def test_hyper_reduced_lspg_follows_the_oracle(g):
    """projection = LSPG with n_s > 0: the GPU runs the DEIM-Galerkin step,
    whose root minimises the hyper-reduced LSPG objective (Eq.
    hyperreduced_lspg_stationarity with the DEIM basis = Phi); the oracle runs
    the literal hyper-reduced Gauss-Newton. Same trajectory within 1e-10."""
    cfg = synth.config_burgers_hyper()
    cfg.n_cells, cfg.projection = 2048, 1
    q0 = synth.initial_state(cfg)
    ref = orom.AdaptiveROM(cfg, q0)
    gpu = g.AdaptiveROM(cfg, q0)
    adopt_if_near_tie(ref, gpu)
    worst = 0.0
    for _ in range(100 // cfg.z):
        for _ in range(cfg.z):
            ref.step()
        gpu.step(cfg.z)
        adopt_if_near_tie(ref, gpu)
        worst = max(worst, rel(gpu.q_tilde(), ref.lifted()))
    assert worst <= 1e-10, worst
    gpu.close()


# ------------------------------------------------- comparison update rules ---

@pytest.mark.parametrize("rule,window", [(1, 16), (2, 16), (2, 6)])
def test_comparison_update_rules_against_oracle(g, rule, window):
    """Algorithm 1 with the windowed-SVD (rule 1) and Direct (rule 2) updates
    of App. A on the window of correction snapshots, against the oracle: q~
    within 1e-9 at every event (the windowed SVD is rebuilt by the growing
    iSVD on the GPU, by LAPACK in the oracle; the Direct basis may differ by a
    rotation within its span, which q~ does not see), and the same rank."""
    cfg = synth.config_burgers_small()
    cfg.r, cfg.update_rule, cfg.window = 6, rule, window
    q0 = synth.initial_state(cfg)
    ref = orom.AdaptiveROM(cfg, q0)
    gpu = g.AdaptiveROM(cfg, q0)
    worst = 0.0
    for _ in range(400 // cfg.z):
        for _ in range(cfg.z):
            ref.step()
        gpu.step(cfg.z)
        worst = max(worst, rel(gpu.q_tilde(), ref.lifted()))
        assert gpu.info()["rank"] == orom.numerical_rank(ref.Phi)
    st = gpu.state()
    P = st["phi"][:, st["sigma"] > 0]
    assert np.max(np.abs(P.T @ P - np.eye(P.shape[1]))) <= 1e-12
    print(f"update rule {rule} (window {window}): worst error {worst:.2e}")
    assert worst <= 1e-9, worst
    gpu.close()


@pytest.mark.parametrize("rule,eta", [(3, 0.0), (4, 0.01), (4, 1.0)])
def test_instant_update_rules_against_oracle(g, rule, eta):
    """Algorithm 1 with the one-step (3) and Oja (4) rules of App. A (the
    learning rates of the paper's Burgers tuning table), which update the basis
    from the snapshot already held and advance the coarse FOM at the end of
    the event, against the oracle, from the oracle's offline state loaded into
    the GPU (these rules carry the offline basis forward, and the GPU's own
    POD, the rank-growing iSVD of the training window, differs from the
    oracle's thin SVD in its trailing kept column by about 3e-10 in 1 - cos):
    q~ within 1e-10 at every event over 400 steps, the same rank, an
    orthonormal basis and the same held snapshot."""
    cfg = synth.config_burgers_small()
    cfg.r, cfg.update_rule, cfg.learning_rate = 8, rule, eta
    q0 = synth.initial_state(cfg)
    ref = orom.AdaptiveROM(cfg, q0)
    gpu = g.AdaptiveROM(cfg, q0)
    s0 = ref.get_state()
    gpu.load_state(s0["Phi"], ref.sigma, s0["a"], s0["y_corr"], s0["n"])
    worst = 0.0
    for _ in range(400 // cfg.z):
        for _ in range(cfg.z):
            ref.step()
        gpu.step(cfg.z)
        worst = max(worst, rel(gpu.q_tilde(), ref.lifted()))
        assert gpu.info()["rank"] == orom.numerical_rank(ref.Phi)
    st = gpu.state()
    k = gpu.info()["rank"]
    P = st["phi"][:, :k]
    assert np.max(np.abs(P.T @ P - np.eye(k))) <= 1e-12
    assert rel(st["y_corr"], ref.y_corr) <= 1e-12
    print(f"update rule {rule} (eta {eta}): worst error {worst:.2e}")
    assert worst <= 1e-10, worst
    gpu.close()


@pytest.mark.parametrize("eta", [0.01, 1e-3])
def test_grouse_against_oracle_within_its_rounding_sensitivity(g, eta):
    """GROUSE (rule 5) turns the basis by alpha = eta |p| |r| towards r/|r|.
    On this workload |r| is about 7e-7 |yhat| at an event, so r/|r| is set by
    the rounding of the projection and the trajectory is sensitive at that
    level: two runs of the oracle that differ only in the summation order of
    the projection drift from 2e-13 after the first event to 1e-3 after five
    (measured at eta = 0.01). From the oracle's offline state loaded into the
    GPU, the GPU agrees with the oracle to 1e-11 after the first event and
    stays within 100 times the oracle pair's difference (plus 1e-11) at every
    event over 60 steps; the basis stays orthonormal (by construction)."""
    cfg = synth.config_burgers_small()
    cfg.r, cfg.update_rule, cfg.learning_rate = 8, 5, eta
    q0 = synth.initial_state(cfg)
    ref = orom.AdaptiveROM(cfg, q0)
    alt = orom.AdaptiveROM(cfg, q0, Q_train=ref.Q_train)
    orig = orom.project_cgs2

    def reversed_order(Phi, y):
        p, q = orig(np.ascontiguousarray(Phi[::-1]), np.ascontiguousarray(y[::-1]))
        return p, q[::-1].copy()

    gpu = g.AdaptiveROM(cfg, q0)
    s0 = ref.get_state()
    gpu.load_state(s0["Phi"], ref.sigma, s0["a"], s0["y_corr"], s0["n"])
    for ev in range(6):
        for _ in range(cfg.z):
            ref.step()
            orom.project_cgs2 = reversed_order
            try:
                alt.step()
            finally:
                orom.project_cgs2 = orig
        gpu.step(cfg.z)
        e_gpu = rel(gpu.q_tilde(), ref.lifted())
        e_pair = rel(alt.lifted(), ref.lifted())
        print(f"GROUSE eta {eta}, event {ev + 1}: GPU {e_gpu:.2e}, oracle pair {e_pair:.2e}")
        if ev == 0:
            assert e_gpu <= 1e-11
        assert e_gpu <= 100.0 * e_pair + 1e-11
    st = gpu.state()
    k = gpu.info()["rank"]
    P = st["phi"][:, :k]
    assert np.max(np.abs(P.T @ P - np.eye(k))) <= 1e-12
    gpu.close()
