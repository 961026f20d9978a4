"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module draws random numbers and lays out workload parameters only. It holds
none of the method's arithmetic (no flux, no projection, no SVD), so both the
CUDA path and the CPU oracle can take their inputs from here without sharing
any computation.

Workloads (the paper's problem families, Sec. 5.1 and 5.2 / App. B):

* Burgers on the periodic unit interval, cell centres ``x_i = (i + 1/2)/N``,
  initial condition ``u0 = 1 + A sin(2 pi x) + 0.1 S(x)`` with
  ``S(x) = sum_{k=1..8} (a_k / k^2) sin(2 pi k x + theta_k)``,
  ``a_k ~ N(0, 1)`` and ``theta_k ~ U[0, 2 pi)`` drawn from
  ``numpy.random.default_rng(seed)`` in that order.
* Sod shock tube (App. B) on [0, 1]: left (rho, u, p) = (1, 0, 1), right
  (0.125, 0, 0.1), with rho and p of every cell multiplied by ``1 + 0.01 xi``,
  ``xi ~ N(0, 1)`` (rho first, then p), u = 0. The state is variable-blocked:
  ``[rho_0..rho_{N-1}, m_0..m_{N-1}, E_0..E_{N-1}]``.
* A batch of independent Burgers ROMs with N log-uniform in [2048, 65536],
  r uniform in {8..48}, nu uniform in [1e-3, 1e-2], z in {5, 10, 20}.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, fields, asdict

import numpy as np

BURGERS = 0
EULER = 1

TWO_PI = 2.0 * math.pi


def cell_centres(n_cells: int) -> np.ndarray:
    """Cell centres of a uniform grid on [0, 1]."""
    return (np.arange(n_cells, dtype=np.float64) + 0.5) / n_cells


def fourier_modes(seed: int, n_modes: int = 8):
    """Amplitudes a_k ~ N(0,1) and phases theta_k ~ U[0, 2pi), k = 1..n_modes."""
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(n_modes)
    theta = rng.uniform(0.0, TWO_PI, n_modes)
    return a, theta


def mode_sum(n_cells: int, seed: int, n_modes: int = 8) -> np.ndarray:
    """S(x) = sum_k (a_k / k^2) sin(2 pi k x + theta_k) at the cell centres."""
    x = cell_centres(n_cells)
    a, theta = fourier_modes(seed, n_modes)
    s = np.zeros(n_cells)
    for k in range(1, n_modes + 1):
        s += (a[k - 1] / k**2) * np.sin(TWO_PI * k * x + theta[k - 1])
    return s


def burgers_ic(n_cells: int, seed: int, amplitude: float = 0.5) -> np.ndarray:
    """u0 = 1 + A sin(2 pi x) + 0.1 S(x) (the Burgers initial-condition family)."""
    x = cell_centres(n_cells)
    return 1.0 + amplitude * np.sin(TWO_PI * x) + 0.1 * mode_sum(n_cells, seed)


def gaussian_ic(n_cells: int, width: float = 0.1) -> np.ndarray:
    """u0 = exp(-((x - 1/2) / width)^2 / 2): the Gaussian pulse of the paper's
    Burgers experiments (Sec. 5.1, L = 1, width 0.1), at the cell centres."""
    x = cell_centres(n_cells)
    return np.exp(-0.5 * ((x - 0.5) / width) ** 2)


def burgers_ic_amplitude_direction(n_cells: int) -> np.ndarray:
    """d u0 / d A = sin(2 pi x): the direction of the amplitude parameter."""
    return np.sin(TWO_PI * cell_centres(n_cells))


def burgers_target(n_cells: int, seed: int) -> np.ndarray:
    """Seeded terminal target 1 + 0.5 sin(2 pi (x - 0.05)) + 0.1 S_seed(x)."""
    x = cell_centres(n_cells)
    return 1.0 + 0.5 * np.sin(TWO_PI * (x - 0.05)) + 0.1 * mode_sum(n_cells, seed)


def sod_primitive_ic(n_cells: int, seed: int | None, perturb: float = 0.01):
    """(rho, u, p) of the Sod problem, optionally with seeded 1% perturbations."""
    x = cell_centres(n_cells)
    left = x < 0.5
    rho = np.where(left, 1.0, 0.125)
    u = np.zeros(n_cells)
    p = np.where(left, 1.0, 0.1)
    if seed is not None and perturb != 0.0:
        rng = np.random.default_rng(seed)
        rho = rho * (1.0 + perturb * rng.standard_normal(n_cells))
        p = p * (1.0 + perturb * rng.standard_normal(n_cells))
    return rho, u, p


def sod_conserved_ic(n_cells: int, seed: int | None, gamma: float = 1.4,
                     perturb: float = 0.01) -> np.ndarray:
    """Variable-blocked conserved state [rho, m, E] of the (perturbed) Sod problem.

    The primitive-to-conserved map is the textbook one (App. B, the conserved
    initial state); it is input preparation, not part of the online path.
    """
    rho, u, p = sod_primitive_ic(n_cells, seed, perturb)
    m = rho * u
    E = p / (gamma - 1.0) + 0.5 * rho * u * u
    return np.concatenate([rho, m, E])


@dataclass
class RomConfig:
    """Hyper-parameters of one adaptive ROM (Algorithm 1 inputs + FOM setup)."""
    problem: int = BURGERS
    n_cells: int = 512
    n_var: int = 1
    r: int = 10
    n_s: int = 0              # 0: plain Galerkin; >0: hyper-reduced Galerkin
    w_init: int = 100
    z: int = 10
    dt: float = 1e-4
    nu: float = 0.01
    gamma: float = 1.4
    lam: float = 0.1
    newton_tol: float = 1e-12
    newton_max: int = 20
    n_online: int = 2000      # online steps after the training window
    precision: int = 0        # 0: FP64, 1: mixed FP32
    projection: int = 0       # 0: Galerkin, 1: least-squares Petrov-Galerkin
    ic: str = "fourier"       # "fourier": the seeded family; "gaussian": the paper's pulse
    update_rule: int = 0      # 0: iSVD (Algorithm 2); 1: windowed SVD; 2: Direct; 3: one-step;
                              # 4: Oja; 5: GROUSE (App. A)
    learning_rate: float = 0.0  # eta of rules 4 and 5
    window: int = 0           # snapshots in the window of rules 1 and 2
    time_scheme: int = 0      # 0: backward Euler; 1: SSPRK(4,3), explicit (Galerkin only)
    seed: int = 0
    amplitude: float = 0.5

    @property
    def n(self) -> int:
        return self.n_var * self.n_cells

    def to_dict(self):
        return asdict(self)

    def matches(self, stored: dict) -> bool:
        """True if a configuration stored with a record describes this one:
        every stored field is equal, and fields the record predates hold
        their defaults."""
        cur = self.to_dict()
        defaults = {f.name: f.default for f in fields(self)}
        return (all(cur.get(k) == v for k, v in stored.items())
                and all(cur[k] == defaults[k] for k in cur.keys() - stored.keys()))


LAMBDA_BY_Z = {5: 0.5, 10: 0.1, 20: 1e-7}


def config_burgers_small() -> RomConfig:
    """Burgers N=512, r=10, nu=0.01, dt=1e-4, w_init=100, z=10, lambda=0.1, 2000 steps."""
    return RomConfig(problem=BURGERS, n_cells=512, r=10, n_s=0, w_init=100, z=10,
                     dt=1e-4, nu=0.01, lam=0.1, n_online=2000, seed=0)


def config_burgers_hyper(precision: int = 0) -> RomConfig:
    """Burgers N=16384, r=32, n_s=96, nu=2e-3, z=5, lambda=0.5, 20000 steps."""
    return RomConfig(problem=BURGERS, n_cells=16384, r=32, n_s=96, w_init=100, z=5,
                     dt=1e-4, nu=2e-3, lam=0.5, n_online=20000, seed=1,
                     precision=precision)


def sod_dt(n_cells: int, seed: int, gamma: float = 1.4, cfl: float = 0.4,
           t_end: float = 0.2):
    """Fixed time step from CFL 0.4 on the perturbed initial state, snapped so
    that an integer number of steps reaches t_end. Returns (dt, n_steps)."""
    rho, u, p = sod_primitive_ic(n_cells, seed)
    c = np.sqrt(gamma * p / rho)
    dx = 1.0 / n_cells
    dt0 = cfl * dx / float(np.max(np.abs(u) + c))
    n_steps = int(math.ceil(t_end / dt0))
    return t_end / n_steps, n_steps


def config_sod(n_cells: int = 8192, seed: int = 2) -> RomConfig:
    """Sod, 3N state, r=40, z=10, lambda=0.01, fixed CFL-0.4 step to t=0.2;
    training window w_init = r = 40 (the method's default window)."""
    dt, n_steps = sod_dt(n_cells, seed)
    w_init = 40
    return RomConfig(problem=EULER, n_cells=n_cells, n_var=3, r=40, n_s=0,
                     w_init=w_init, z=10, dt=dt, nu=0.0, gamma=1.4, lam=0.01,
                     n_online=n_steps - w_init, seed=seed)


def config_batch(count: int = 256, seed0: int = 1000, n_online: int = 2000):
    """Independent Burgers ROM instances of uneven size (log-uniform N)."""
    out = []
    for i in range(count):
        rng = np.random.default_rng(seed0 + i)
        n = int(round(math.exp(rng.uniform(math.log(2048), math.log(65536)))))
        r = int(rng.integers(8, 49))
        nu = float(rng.uniform(1e-3, 1e-2))
        z = int(rng.choice([5, 10, 20]))
        out.append(RomConfig(problem=BURGERS, n_cells=n, r=r, n_s=0, w_init=100, z=z,
                             dt=1e-4, nu=nu, lam=LAMBDA_BY_Z[z], n_online=n_online,
                             seed=seed0 + i, precision=1))
    return out


PAPER_SWEEP_Z = (5, 10, 25, 50)
PAPER_SWEEP_LAMBDA = (1e-7, 0.1, 0.25, 0.5, 0.75, 1.0)


def config_paper_burgers_sweep(precision: int = 1):
    """The paper's Burgers setting (Sec. 5.1): Gaussian pulse, N = 1000 cells,
    nu = 0.01, dt = 1e-3, 500 steps in all (w_init = 4 training steps, 496
    online), r = w_init = 4, for every adaptation interval z in {5, 10, 25, 50}
    and forgetting factor lambda in {1e-7, 0.1, 0.25, 0.5, 0.75, 1} (the
    batched engine runs the mixed form, plain Galerkin)."""
    return [RomConfig(problem=BURGERS, n_cells=1000, r=4, n_s=0, w_init=4, z=z, dt=1e-3, nu=0.01,
                      lam=lam, n_online=496, ic="gaussian", precision=precision)
            for z in PAPER_SWEEP_Z for lam in PAPER_SWEEP_LAMBDA]


def config_adjoint() -> RomConfig:
    """Burgers N=65536, r=64, nu=5e-3, z=10, lambda=0.1, 1000 steps (terminal misfit)."""
    return RomConfig(problem=BURGERS, n_cells=65536, r=64, n_s=0, w_init=100, z=10,
                     dt=1e-4, nu=5e-3, lam=0.1, n_online=1000, seed=4)


def initial_state(cfg: RomConfig) -> np.ndarray:
    """The seeded initial state q0 of a configuration."""
    if cfg.problem == BURGERS and cfg.ic == "gaussian":
        return gaussian_ic(cfg.n_cells)
    if cfg.problem == BURGERS:
        return burgers_ic(cfg.n_cells, cfg.seed, cfg.amplitude)
    return sod_conserved_ic(cfg.n_cells, cfg.seed, cfg.gamma)


def random_orthonormal(n: int, r: int, seed: int) -> np.ndarray:
    """A seeded N x r matrix with orthonormal columns (QR of a Gaussian matrix),
    used only to make test inputs for the basis-update kernels."""
    rng = np.random.default_rng(seed)
    q, _ = np.linalg.qr(rng.standard_normal((n, r)))
    return q


def probe_vectors(n: int, count: int = 4, seed: int = 77) -> np.ndarray:
    """A seeded n x count Gaussian matrix. Stored trajectory records keep the
    products W^T q~ with these vectors next to a subsample of q~, so that a
    difference anywhere in a full-size state shows up in a few numbers."""
    return np.random.default_rng(seed).standard_normal((n, count))
