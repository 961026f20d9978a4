"""Pins of the oracle's feature-guided points for the Euler system (Eq.
fgs_selection with the pressure feature of Sec. 5.3): scores from states
built out of chosen primitive variables, where the pressure, and so the
expected score of every cell, is known in closed form."""
import numpy as np
import pytest

import synth
from oracle import rom

GAMMA = 1.4


def conserved(rho, u, p, gamma=GAMMA):
    """(rho, m, E) rows of the variable-blocked state from primitives."""
    rho, u, p = (np.asarray(x, dtype=np.float64) for x in (rho, u, p))
    return np.concatenate([rho, rho * u, p / (gamma - 1.0) + 0.5 * rho * u * u])


def test_pressure_scores_closed_form():
    """p_i = 1 + i^2/16 gives (p_{i+1} - p_i)^2 = ((2 i + 1)/16)^2; the last
    cell faces the zero-gradient ghost cell and scores 0; a cell's three rows
    share its score. Moving, non-uniform flow, so that the kinetic energy
    must be taken out correctly."""
    n = 12
    i = np.arange(n, dtype=np.float64)
    rho = 1.0 + 0.1 * i
    u = 0.3 * (-1.0) ** i
    p = 1.0 + i * i / 16.0
    g = rom.fgs_scores(conserved(rho, u, p), problem=1, gamma=GAMMA)
    cell = ((2.0 * i + 1.0) / 16.0) ** 2
    cell[-1] = 0.0
    assert g.shape == (3 * n,)
    for v in range(3):
        np.testing.assert_allclose(g[v * n:(v + 1) * n], cell, rtol=1e-12, atol=1e-15)


def test_pressure_feature_ignores_a_contact():
    """A density jump at constant pressure and velocity (a contact) has no
    pressure gradient: every score is at rounding level."""
    n = 40
    rho = np.where(np.arange(n) < n // 2, 1.0, 0.125)
    g = rom.fgs_scores(conserved(rho, np.full(n, 0.5), np.full(n, 0.7)), problem=1, gamma=GAMMA)
    assert np.max(g) <= 1e-28


@pytest.mark.parametrize("seed", [0, 1])
def test_pressure_scores_galilean_invariant(seed):
    """Pressure, and so every score, does not change when a uniform velocity
    is added to the flow."""
    rng = np.random.default_rng(seed)
    n = 64
    rho = rng.uniform(0.2, 2.0, n)
    u = rng.uniform(-1.0, 1.0, n)
    p = rng.uniform(0.1, 3.0, n)
    g0 = rom.fgs_scores(conserved(rho, u, p), problem=1, gamma=GAMMA)
    g1 = rom.fgs_scores(conserved(rho, u + 0.7, p), problem=1, gamma=GAMMA)
    np.testing.assert_allclose(g1, g0, rtol=1e-9, atol=1e-14)


def test_feature_points_take_whole_cells_in_score_order():
    """Two pressure jumps, the larger between cells 9 and 10 and the smaller
    between cells 25 and 26: the greedy points are the three rows of cell 9,
    then those of cell 25 (rows rho, m, E in index order); rows already chosen
    are skipped."""
    n = 32
    p = np.ones(n)
    p[10:] = 3.0
    p[26:] = 3.5
    y = conserved(np.full(n, 1.0), np.full(n, 0.2), p)
    assert rom.fgs_extend(y, [], 5, problem=1, gamma=GAMMA) == [9, n + 9, 2 * n + 9, 25, n + 25]
    assert rom.fgs_extend(y, [n + 9, 25], 3, problem=1, gamma=GAMMA) == [9, 2 * n + 9, n + 25]


def test_sod_initial_state_points_at_the_diaphragm():
    """The Sod initial state's only pressure jump is at the diaphragm: the
    feature points of highest score are the rows of the cell left of it."""
    cfg = synth.config_sod(256)
    q0 = synth.initial_state(cfg)
    nc = cfg.n_cells
    g = rom.fgs_scores(q0, problem=1, gamma=cfg.gamma)
    p = (cfg.gamma - 1.0) * (q0[2 * nc:] - 0.5 * q0[nc:2 * nc] ** 2 / q0[:nc])
    j = int(np.argmax(np.abs(np.diff(p))))
    assert rom.fgs_extend(q0, [], 3, problem=1, gamma=cfg.gamma) == [j, nc + j, 2 * nc + j]
    assert g[j] == pytest.approx((p[j + 1] - p[j]) ** 2, rel=1e-12)


def test_burgers_scores_unchanged_by_the_default():
    """The default (problem 0) is the Burgers feature Theta(y) = y."""
    y = np.array([0.0, 1.0, 1.0, 3.0, 3.0, 2.0, 0.0, 0.0])
    assert list(rom.fgs_scores(y)) == [1.0, 0.0, 4.0, 0.0, 1.0, 4.0, 0.0, 0.0]
