"""Pins of the oracle's instantaneous comparison rules (App. A): one-step
(Eq. onestep_update), Oja (Eq. oja_update) and GROUSE (Eqs.
grouse_projection, grouse_update), by properties the formulas fix and a hand
expansion, and of their place in the online loop (the update takes the
correction snapshot already held, then the coarse FOM advances)."""
import numpy as np
import pytest

import synth
from oracle import rom as orom


def _basis(n, k, r, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, k)))
    Phi = np.zeros((n, r))
    Phi[:, :k] = Q
    return Phi, rng


def _out_of_span(P, y):
    return float(np.linalg.norm(y - P @ (P.T @ y)) / np.linalg.norm(y))


def test_onestep_snapshot_enters_span_and_rank_is_kept():
    Phi, rng = _basis(200, 4, 6, 1)
    y = rng.standard_normal(200)
    a = np.concatenate([rng.standard_normal(4), np.zeros(2)])
    new = orom.onestep_update(Phi, y, a)
    P = new[:, :4]
    assert np.allclose(P.T @ P, np.eye(4), atol=1e-13)
    assert np.all(new[:, 4:] == 0.0)
    assert _out_of_span(P, y) <= 1e-12          # Phi a = yhat after the rank-one correction
    assert _out_of_span(Phi[:, :4], y) > 0.5    # it was not there before


def test_onestep_keeps_the_directions_orthogonal_to_the_state():
    Phi, rng = _basis(150, 5, 5, 2)
    y = rng.standard_normal(150)
    a = rng.standard_normal(5)
    new = orom.onestep_update(Phi, y, a)
    B = np.linalg.svd(a[None, :])[2][1:].T      # 5 x 4, orthogonal to a
    for x in B.T:
        v = Phi @ x
        assert _out_of_span(new, v) <= 1e-12


def test_oja_single_direction_hand_expansion():
    """r = 1, phi = e1, yhat = (1, 2, 0), eta = 0.5: phi + eta yhat (yhat . phi)
    = (1.5, 1, 0), normalised."""
    Phi = np.zeros((3, 1))
    Phi[0, 0] = 1.0
    new = orom.oja_update(Phi, np.array([1.0, 2.0, 0.0]), 0.5)
    expect = np.array([1.5, 1.0, 0.0]) / np.sqrt(3.25)
    assert np.allclose(np.abs(new[:, 0]), expect, atol=1e-15)


def test_oja_first_order_in_the_learning_rate():
    """d(Phi Phi^T) = eta [(I - P) y y^T P + P y y^T (I - P)] + O(eta^2), P = Phi Phi^T."""
    Phi, rng = _basis(60, 3, 3, 3)
    y = rng.standard_normal(60)
    P = Phi @ Phi.T
    lin = (np.eye(60) - P) @ np.outer(y, y) @ P
    lin = lin + lin.T
    errs = []
    for eta in (1e-4, 1e-5):
        new = orom.oja_update(Phi, y, eta)
        errs.append(np.linalg.norm(new @ new.T - P - eta * lin))
    assert errs[1] < errs[0] / 50               # the remainder is second order


def test_grouse_orthonormal_by_construction():
    Phi, rng = _basis(120, 6, 8, 4)
    y = rng.standard_normal(120)
    for eta in (1e-3, 0.1, 1.0):
        new = orom.grouse_update(Phi, y, eta)
        P = new[:, :6]
        assert np.abs(P.T @ P - np.eye(6)).max() <= 1e-13
        assert np.all(new[:, 6:] == 0.0)


def test_grouse_step_by_the_angle_reaches_the_snapshot():
    """With alpha equal to the angle between yhat and span(Phi) (eta = theta /
    (|p| |r|), theta = atan(|r| / |p|)) the geodesic step turns the subspace
    onto yhat."""
    Phi, rng = _basis(90, 4, 4, 5)
    y = rng.standard_normal(90)
    p = Phi @ (Phi.T @ y)
    r = y - p
    theta = np.arctan2(np.linalg.norm(r), np.linalg.norm(p))
    new = orom.grouse_update(Phi, y, theta / (np.linalg.norm(p) * np.linalg.norm(r)))
    assert _out_of_span(new, y) <= 1e-12
    half = orom.grouse_update(Phi, y, 0.5 * theta / (np.linalg.norm(p) * np.linalg.norm(r)))
    assert _out_of_span(half, y) > 0.1


@pytest.mark.parametrize("rule,eta", [(3, 0.0), (4, 0.01), (5, 0.01)])
def test_instant_rule_event_uses_the_held_snapshot(rule, eta):
    """At the first event the update takes yhat = D (y_corr - q_ref) of the
    snapshot computed at the end of the offline stage, then the coarse FOM
    advances that snapshot; the basis stays orthonormal over the run."""
    cfg = synth.config_burgers_small()
    cfg.n_cells, cfg.update_rule, cfg.learning_rate = 256, rule, eta
    q0 = synth.initial_state(cfg)
    m = orom.AdaptiveROM(cfg, q0)
    y_held = m.y_corr.copy()
    for _ in range(cfg.z - 1):
        m.step()
    phi_old, a_old = m.Phi.copy(), None
    a_new, _ = m.rom_step(m.a)
    a_old = a_new
    m.step()                                    # the event step
    yhat = m.d * (y_held - m.q_ref)
    if rule == 3:
        expect = orom.onestep_update(phi_old, yhat, a_old)
    elif rule == 4:
        expect = orom.oja_update(phi_old, yhat, eta)
    else:
        expect = orom.grouse_update(phi_old, yhat, eta)
    assert np.array_equal(m.Phi, expect)
    assert np.allclose(m.y_corr, m.coarse_step(y_held), rtol=0, atol=1e-14)
    for _ in range(3 * cfg.z):
        m.step()
    P = m.Phi[:, :orom.numerical_rank(m.Phi)]
    assert np.abs(P.T @ P - np.eye(P.shape[1])).max() <= 1e-12
