"""The C-ABI library loads and exports every function include/rom.h declares,
and rejects invalid arguments before touching the device (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2605_28684_gb300 import build, _lib
    build.build()
    return _lib.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "rom.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rom_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "rom_init" in names and "rom_isvd_update_dev" in names
    for name in names:
        assert hasattr(lib, name), name


def test_binding_lists_match_header():
    from paper_2605_28684_gb300 import _lib
    assert sorted(_lib.EXPORTED) == declared_functions()


def test_invalid_configs_rejected(lib):
    import paper_2605_28684_gb300 as g
    base = synth.config_burgers_small()
    q0 = synth.initial_state(base)
    bad = []
    for field, val in [("r", 0), ("r", 65), ("r", 200), ("z", 0), ("lam", 1.5), ("dt", 0.0),
                       ("n_s", 5), ("w_init", 0), ("n_var", 3), ("newton_tol", 0.0)]:
        c = synth.config_burgers_small()
        setattr(c, field, val)
        bad.append(c)
    for c in bad:
        cfg = g.make_config(c)
        ctx = ctypes.c_void_p()
        rc = lib.rom_init(ctypes.byref(cfg), q0.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                          None, ctypes.byref(ctx))
        assert rc == 1 and not ctx.value     # ROM_EINVAL, no context
    assert lib.rom_init(None, None, None, ctypes.byref(ctypes.c_void_p())) == 1
    assert lib.rom_step(None, 1) == 1
    assert lib.rom_state(None, None, None, None, None, None, None) == 1
    lib.rom_destroy(None)
    assert lib.rom_status_string(4) == b"Newton iteration did not converge"


def test_invalid_batches_rejected(lib):
    """The batched engine runs Burgers in the mixed form without hyper-reduction;
    anything else is refused before any device work."""
    import paper_2605_28684_gb300 as g
    good = synth.config_batch(2)
    q0s = [synth.initial_state(c) for c in good]
    D = ctypes.POINTER(ctypes.c_double)

    def init(cfgs, count=None):
        n = len(cfgs)
        arr = (g._lib.RomConfigC * n)(*[g.make_config(c) for c in cfgs])
        ptrs = (D * n)(*[q.ctypes.data_as(D) for q in q0s[:n]])
        out = ctypes.c_void_p()
        rc = lib.rom_batch_init(arr, ptrs, n if count is None else count, None, ctypes.byref(out))
        return rc, out.value

    for field, val in [("precision", 0), ("problem", 1), ("n_s", 4), ("r", 65), ("n_cells", 128),
                       ("z", 0)]:
        cfgs = synth.config_batch(2)
        setattr(cfgs[1], field, val)
        rc, out = init(cfgs)
        assert rc == 1 and not out, field
    rc, out = init(good, count=0)
    assert rc == 1 and not out
    assert lib.rom_batch_step(None, 1) == 1
    assert lib.rom_batch_state(None, 0, None, None, None, None, None, None) == 1
    assert lib.rom_batch_info(None, 0, None, None, None) == 1
    lib.rom_batch_destroy(None)
