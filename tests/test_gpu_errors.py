"""Error paths of the C ABI on the GPU, made without faulting the GPU.

* ROM_ETIMEOUT: the bound of the grid barrier's wait is lowered to one clock
  cycle through the library's test hook, so the first CTA to reach a barrier
  gives up before the others arrive; the kernels record the timeout and
  return (every wait stays bounded), the call reports ROM_ETIMEOUT and the
  context is poisoned (ROM_ESTATE afterwards). The kernels used here index
  only by row and iteration counts, never by values another CTA computed, so
  the partial work a timed-out launch leaves behind stays in bounds.
* ROM_ENONFINITE: NaN / Inf in host inputs are refused on the host.
"""
import numpy as np
import pytest

import synth

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


def test_fom_step_wait_timeout_is_reported(g):
    n = 65536                                   # 64 chunks: many CTAs at every barrier
    q0 = synth.burgers_ic(n, 7)
    qp = torch.tensor(q0, device="cuda", dtype=torch.float64)
    qn = torch.empty_like(qp)
    g.debug_set_wait_limit(1)
    try:
        with pytest.raises(g.RomError) as ei:
            g.fom_step_dev(0, n, 5e-3, 1.4, 1e-3, 1e-12, 20, qp.data_ptr(), qn.data_ptr())
    finally:
        g.debug_set_wait_limit(0)
    assert ei.value.code == 6                   # ROM_ETIMEOUT
    # the device is still usable: the same step now converges
    it = g.fom_step_dev(0, n, 5e-3, 1.4, 1e-3, 1e-12, 20, qp.data_ptr(), qn.data_ptr())
    assert 1 <= it <= 20


def test_wait_timeout_poisons_the_context(g):
    cfg = synth.config_burgers_small()
    cfg.n_cells = 4096
    q0 = synth.initial_state(cfg)
    rom = g.AdaptiveROM(cfg, q0)
    rom.step(3)                                 # no event yet: only the Galerkin step kernel
    g.debug_set_wait_limit(1)
    try:
        with pytest.raises(g.RomError) as ei:
            rom.step(5)
    finally:
        g.debug_set_wait_limit(0)
    assert ei.value.code == 6                   # ROM_ETIMEOUT
    for call in (lambda: rom.step(1), lambda: rom.state(), lambda: rom.info()):
        with pytest.raises(g.RomError) as ei:
            call()
        assert ei.value.code == 7               # ROM_ESTATE
    rom.close()
    # a new context on the same device works
    rom2 = g.AdaptiveROM(cfg, q0)
    rom2.step(20)
    assert np.all(np.isfinite(rom2.q_tilde()))
    rom2.close()


def test_nonfinite_host_inputs_are_refused(g):
    cfg = synth.config_burgers_small()
    q0 = synth.initial_state(cfg)
    bad_q0 = q0.copy()
    bad_q0[7] = np.nan
    with pytest.raises(g.RomError) as ei:
        g.AdaptiveROM(cfg, bad_q0)
    assert ei.value.code == 5                   # ROM_ENONFINITE
    rom = g.AdaptiveROM(cfg, q0)
    rom.step(4)
    before = rom.state()
    y = before["y_corr"].copy()
    y[100] = np.inf
    with pytest.raises(g.RomError) as ei:
        rom.update_basis(y)
    assert ei.value.code == 5
    bad_phi = before["phi"].copy()
    bad_phi[3, 0] = np.nan
    with pytest.raises(g.RomError) as ei:
        rom.load_state(bad_phi, before["sigma"], before["a"], before["y_corr"], before["step"])
    assert ei.value.code == 5
    # refused inputs leave the context unchanged and usable
    after = rom.state()
    assert np.array_equal(after["q_tilde"], before["q_tilde"])
    rom.update_basis(before["y_corr"])
    rom.step(6)
    assert np.all(np.isfinite(rom.q_tilde()))
    rom.close()
