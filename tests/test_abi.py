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
                       ("n_s", 5), ("w_init", 0), ("n_var", 3), ("newton_tol", 0.0),
                       # sizes the FOM partitioning cannot hold (128 chunks x 1024 rows)
                       ("n_cells", 4), ("n_cells", 128 * 1024 + 1),
                       # r beyond the training window, too many samples, no BF16 form
                       ("w_init", 5), ("n_s", 257), ("precision", 2),
                       ("nu", -1e-3), ("dt", float("nan")), ("newton_max", 0),
                       # unknown projection; LSPG is FP64 only
                       ("projection", 2)]:
        c = synth.config_burgers_small()
        setattr(c, field, val)
        bad.append(c)
    for field, val in [("n_cells", 128 * 256 + 1), ("n_s", 60), ("n_var", 1), ("projection", 1)]:
        c = synth.config_sod(256)
        setattr(c, field, val)
        bad.append(c)
    c = synth.config_burgers_small()
    c.projection, c.precision = 1, 1          # no mixed-precision LSPG form
    bad.append(c)
    # DEIM-Galerkin Euler: the explicit form only, and its nine mesh rows per
    # sample must fit shared memory (r = 40, n_s = 80 does not)
    c = synth.config_sod(256)
    c.r, c.n_s = 20, 40
    bad.append(c)
    c = synth.config_sod(256)
    c.time_scheme, c.n_s = 1, 80
    bad.append(c)
    # comparison update rules: unknown rule, window outside 1..min(w_init, 64), FP64 only
    for rule, window, prec in [(6, 8, 0), (1, 0, 0), (2, 101, 0), (1, 8, 1)]:
        c = synth.config_burgers_small()
        c.update_rule, c.window, c.precision = rule, window, prec
        bad.append(c)
    # instantaneous rules: FP64, plain Galerkin sampling (n_s = 0), backward
    # Euler, a finite non-negative learning rate
    for rule, field, val in [(3, "precision", 1), (4, "learning_rate", -1.0), (5, "learning_rate", float("nan")),
                             (5, "time_scheme", 1)]:
        c = synth.config_burgers_small()
        c.update_rule, c.learning_rate = rule, 0.01
        setattr(c, field, val)
        bad.append(c)
    c = synth.config_burgers_hyper()
    c.n_cells, c.update_rule = 2048, 4
    bad.append(c)
    # time schemes: unknown; the explicit form is Galerkin, FP64 and iSVD only
    for field, val in [("time_scheme", 2), ("projection", 1), ("precision", 1), ("update_rule", 1)]:
        c = synth.config_burgers_small()
        c.time_scheme, c.window = 1, 8
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
                       ("z", 0), ("projection", 1), ("time_scheme", 1)]:
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


def test_context_free_entry_points_reject_invalid_arguments(lib):
    """Every case below fails the argument check, which comes before any
    device call; the pointers are never dereferenced."""
    P = ctypes.c_void_p
    a, b = P(0x10000), P(0x20000)           # stand-ins for device buffers
    EINVAL = 1
    nan = float("nan")
    # f(q): null buffers, too few cells, unknown problem
    for args in [(0, 64, 0.01, 1.4, None, b), (0, 64, 0.01, 1.4, a, None), (0, 1, 0.01, 1.4, a, b),
                 (2, 64, 0.01, 1.4, a, b)]:
        assert lib.rom_fom_rhs_dev(*args, None) == EINVAL, args
    # one BE step (both variants): buffers, aliasing, sizes, step, Newton controls, problem
    step_cases = [
        dict(q_prev=None), dict(q=a), dict(n=1), dict(h=0.0), dict(h=nan), dict(newton_max=0),
        dict(tol=0.0), dict(problem=2), dict(n=1 << 40),
    ]
    base = dict(problem=0, n=512, nu=0.01, gamma=1.4, h=1e-3, tol=1e-12, newton_max=20, q_prev=a, q=b)
    for fn in (lib.rom_fom_step_dev, lib.rom_fom_step_noalloc_dev):
        for case in step_cases:
            c = dict(base, **case)
            rc = fn(c["problem"], c["n"], c["nu"], c["gamma"], c["h"], c["tol"], c["newton_max"],
                    c["q_prev"], c["q"], None, None)
            assert rc == EINVAL, (fn, case)
    for n in (4, 40000):                     # the Euler step's cell range
        assert lib.rom_fom_step_dev(1, n, 0.0, 1.4, 1e-4, 1e-12, 20, a, b, None, None) == EINVAL
    # the allocation-free step serves Burgers only
    assert lib.rom_fom_step_noalloc_dev(1, 512, 0.0, 1.4, 1e-4, 1e-12, 20, a, b, None, None) == EINVAL
    # rank-one update: sizes, rank range, buffers, forgetting factor
    for n, r, lam, phi in [(1, 1, 0.5, a), (64, 0, 0.5, a), (128, 65, 0.5, a), (16, 16, 0.5, a),
                           (64, 8, 0.5, None), (64, 8, 1.5, a), (64, 8, -0.1, a), (64, 8, nan, a)]:
        assert lib.rom_isvd_update_dev(n, r, lam, 1e-10, phi, b, b, None, None) == EINVAL, (n, r, lam)


def test_context_calls_reject_a_null_context(lib):
    D = ctypes.POINTER(ctypes.c_double)
    buf = (ctypes.c_double * 64)()
    i64 = (ctypes.c_int64 * 8)()
    i32 = (ctypes.c_int32 * 8)()
    dp = ctypes.cast(buf, D)
    EINVAL = 1
    assert lib.rom_step(None, -1) == EINVAL
    assert lib.rom_update_basis(None, None) == EINVAL
    assert lib.rom_load_state(None, dp, dp, dp, dp, 100) == EINVAL
    assert lib.rom_samples(None, i32) == EINVAL
    assert lib.rom_info(None, None, None, None) == EINVAL
    assert lib.rom_profile(None, 1) == EINVAL
    assert lib.rom_profile_read(None, dp, i64) == EINVAL
    assert lib.rom_batch_layout(None, None, None, None, None, None, None) == EINVAL
    assert lib.rom_batch_profile(None, 1) == EINVAL
    assert lib.rom_batch_work(None, None, None) == EINVAL
    assert lib.rom_batch_fom_work(None, None, None) == EINVAL
    assert lib.rom_batch_profile_read(None, dp, i64) == EINVAL
    for code in range(8):
        assert lib.rom_status_string(code)


def test_binding_checks_host_array_sizes_before_the_library():
    """The library copies N (or N x r) doubles from host arrays; the binding
    refuses arrays of other shapes before calling it (here on an object with
    no context, so nothing else could run)."""
    import paper_2605_28684_gb300 as g
    rom = g.AdaptiveROM.__new__(g.AdaptiveROM)
    rom.N, rom.r, rom._lib, rom._ctx = 12, 3, None, ctypes.c_void_p()
    with pytest.raises(ValueError):
        rom.update_basis(np.zeros(11))
    good = dict(phi=np.zeros((12, 3)), sigma=np.zeros(3), a=np.zeros(3), y_corr=np.zeros(12))
    for key, bad in [("phi", np.zeros((3, 12))), ("phi", np.zeros((12, 2))), ("sigma", np.zeros(4)),
                     ("a", np.zeros(2)), ("y_corr", np.zeros(13))]:
        args = dict(good, **{key: bad})
        with pytest.raises(ValueError):
            rom.load_state(args["phi"], args["sigma"], args["a"], args["y_corr"], 100)


def test_nonfinite_initial_state_refused_before_the_device(lib):
    """A NaN or Inf in the host initial state is refused on the host
    (ROM_ENONFINITE) before any device call, so no context is made."""
    import paper_2605_28684_gb300 as g
    cfg = synth.config_burgers_small()
    D = ctypes.POINTER(ctypes.c_double)
    for bad in (float("nan"), float("inf"), -float("inf")):
        q0 = synth.initial_state(cfg)
        q0[123] = bad
        c = g.make_config(cfg)
        ctx = ctypes.c_void_p()
        rc = lib.rom_init(ctypes.byref(c), q0.ctypes.data_as(D), None, ctypes.byref(ctx))
        assert rc == 5 and not ctx.value, bad       # ROM_ENONFINITE


def test_validation_accepts_the_euler_galerkin_fgs_form(lib):
    """Sod with feature-guided points in the explicit form passes the
    argument checks (without a device it then fails at the first device call,
    ROM_ECUDA); the same model in the backward-Euler form, or with a mesh too
    large for shared memory, is refused first (ROM_EINVAL)."""
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a device is present: rom_init would build the context")
    except ImportError:
        pass
    import paper_2605_28684_gb300 as g
    D = ctypes.POINTER(ctypes.c_double)
    for mod, expect in [(dict(time_scheme=1, r=20, n_s=40), 3), (dict(r=20, n_s=40), 1),
                        (dict(time_scheme=1, n_s=80), 1)]:
        c = synth.config_sod(256)
        for k, v in mod.items():
            setattr(c, k, v)
        q0 = synth.initial_state(c)
        cfg = g.make_config(c)
        ctx = ctypes.c_void_p()
        rc = lib.rom_init(ctypes.byref(cfg), q0.ctypes.data_as(D), None, ctypes.byref(ctx))
        assert rc == expect and not ctx.value, (mod, rc)
