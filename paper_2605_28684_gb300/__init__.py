"""GB300-native adaptive reduced-order model with incremental-SVD basis updates.

Python binding of librom (C ABI in include/rom.h). Every numerical step runs in
the library's CUDA kernels; this module only marshals arguments. It raises if
librom.so is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import RomError, ROM_OK  # noqa: F401

BURGERS, EULER = 0, 1
FP64, MIXED_FP32 = 0, 1

_DP = ctypes.POINTER(ctypes.c_double)


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_DP)


def make_config(cfg) -> _lib.RomConfigC:
    """Build the C configuration from any object with the rom_config fields
    (lambda is read from ``lam`` or ``lambda_``)."""
    c = _lib.RomConfigC()
    c.problem = int(cfg.problem)
    c.precision = int(getattr(cfg, "precision", 0))
    c.n_cells = int(cfg.n_cells)
    c.n_var = int(cfg.n_var)
    c.r = int(cfg.r)
    c.n_s = int(cfg.n_s)
    c.w_init = int(cfg.w_init)
    c.z = int(cfg.z)
    c.newton_max = int(getattr(cfg, "newton_max", 20))
    c.dt = float(cfg.dt)
    c.nu = float(cfg.nu)
    c.gamma = float(getattr(cfg, "gamma", 1.4))
    c.lambda_ = float(getattr(cfg, "lam", getattr(cfg, "lambda_", 0.1)))
    c.newton_tol = float(getattr(cfg, "newton_tol", 1e-12))
    c.rank_tol = float(getattr(cfg, "rank_tol", 0.0))     # <= 0: the precision's default
    c.projection = int(getattr(cfg, "projection", 0))
    c.update_rule = int(getattr(cfg, "update_rule", 0))
    c.window = int(getattr(cfg, "window", 0))
    c.time_scheme = int(getattr(cfg, "time_scheme", 0))
    c.learning_rate = float(getattr(cfg, "learning_rate", 0.0))
    return c


class AdaptiveROM:
    """One adaptive ROM held on the GPU (Algorithm 1 with the iSVD update)."""

    def __init__(self, cfg, q0, stream: int | None = None):
        self._lib = _lib.load()
        self.cfg = cfg
        self._c = make_config(cfg)
        self.N = int(cfg.n_cells) * int(cfg.n_var)
        self.r = int(cfg.r)
        q0 = np.ascontiguousarray(q0, dtype=np.float64)
        if q0.shape != (self.N,):
            raise ValueError(f"q0 must have {self.N} entries")
        self._ctx = ctypes.c_void_p()
        self._stream = ctypes.c_void_p(stream or 0)
        _lib.check(self._lib.rom_init(ctypes.byref(self._c), _dptr(q0), self._stream,
                                      ctypes.byref(self._ctx)), "rom_init")

    def step(self, n_steps: int = 1):
        _lib.check(self._lib.rom_step(self._ctx, int(n_steps)), "rom_step")

    def update_basis(self, y=None):
        if y is None:
            _lib.check(self._lib.rom_update_basis(self._ctx, None), "rom_update_basis")
        else:
            y = np.ascontiguousarray(y, dtype=np.float64)
            if y.shape != (self.N,):
                raise ValueError(f"y must have {self.N} entries")
            _lib.check(self._lib.rom_update_basis(self._ctx, _dptr(y)), "rom_update_basis")

    def state(self, q_tilde=True, phi=True, y_corr=True):
        qt = np.empty(self.N) if q_tilde else None
        a = np.empty(self.r)
        s = np.empty(self.r)
        ph = np.empty((self.r, self.N)) if phi else None
        yc = np.empty(self.N) if y_corr else None
        step = ctypes.c_int64()
        _lib.check(self._lib.rom_state(self._ctx, None if qt is None else _dptr(qt), _dptr(a),
                                       _dptr(s), None if ph is None else _dptr(ph),
                                       None if yc is None else _dptr(yc), ctypes.byref(step)),
                   "rom_state")
        return dict(q_tilde=qt, a=a, sigma=s, phi=None if ph is None else ph.T.copy(),
                    y_corr=yc, step=step.value)

    def q_tilde(self, out=None):
        qt = np.empty(self.N) if out is None else out
        if qt.dtype != np.float64 or qt.shape != (self.N,) or not qt.flags.c_contiguous:
            raise ValueError("out must be a contiguous float64 array of N entries")
        _lib.check(self._lib.rom_state(self._ctx, _dptr(qt), None, None, None, None, None),
                   "rom_state")
        return qt

    def load_state(self, phi, sigma, a, y_corr, step):
        """Phi (N x r), sigma (r), a (r), y_corr (N) and the step count, as
        ``state`` returns them; the library copies exactly these sizes."""
        ph = np.asarray(phi, dtype=np.float64)
        s = np.ascontiguousarray(sigma, dtype=np.float64)
        av = np.ascontiguousarray(a, dtype=np.float64)
        yc = np.ascontiguousarray(y_corr, dtype=np.float64)
        if ph.shape != (self.N, self.r) or s.shape != (self.r,) or av.shape != (self.r,) \
                or yc.shape != (self.N,):
            raise ValueError(f"expected phi ({self.N}, {self.r}), sigma and a ({self.r},), "
                             f"y_corr ({self.N},)")
        ph = np.ascontiguousarray(ph.T)                                  # column-major N x r
        _lib.check(self._lib.rom_load_state(self._ctx, _dptr(ph), _dptr(s), _dptr(av), _dptr(yc),
                                            int(step)), "rom_load_state")

    def samples(self):
        out = np.empty(int(self.cfg.n_s), dtype=np.int32)
        _lib.check(self._lib.rom_samples(self._ctx, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))),
                   "rom_samples")
        return out

    def info(self):
        v = [ctypes.c_int32() for _ in range(3)]
        _lib.check(self._lib.rom_info(self._ctx, *[ctypes.byref(x) for x in v]), "rom_info")
        return dict(rank=v[0].value, rom_newton_iters=v[1].value, fom_newton_iters=v[2].value)

    PHASES = ("reduced_steps", "coarse_fom", "isvd_update", "sampling", "feature_select")

    def profile(self, enable: bool):
        _lib.check(self._lib.rom_profile(self._ctx, 1 if enable else 0), "rom_profile")

    def profile_read(self):
        ms = (ctypes.c_double * len(self.PHASES))()
        cnt = (ctypes.c_int64 * len(self.PHASES))()
        _lib.check(self._lib.rom_profile_read(self._ctx, ms, cnt), "rom_profile_read")
        return {p: dict(ms=ms[i], launches=cnt[i]) for i, p in enumerate(self.PHASES)}

    def close(self):
        if getattr(self, "_ctx", None) is not None and self._ctx.value:
            self._lib.rom_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many independent Burgers ROMs advanced together on the GPU (mixed form)."""

    PHASES = ("reduced_steps", "coarse_fom", "isvd_update")

    def __init__(self, cfgs, q0s, stream: int | None = None):
        self._lib = _lib.load()
        self.cfgs = list(cfgs)
        n = len(self.cfgs)
        arr = (_lib.RomConfigC * n)()
        for i, c in enumerate(self.cfgs):
            arr[i] = make_config(c)
        self._q0 = [np.ascontiguousarray(q, dtype=np.float64) for q in q0s]
        for c, q in zip(self.cfgs, self._q0):
            if q.shape != (int(c.n_cells),):
                raise ValueError("each q0 must have n_cells entries")
        ptrs = (_DP * n)(*[_dptr(q) for q in self._q0])
        self._b = ctypes.c_void_p()
        _lib.check(self._lib.rom_batch_init(arr, ptrs, n, ctypes.c_void_p(stream or 0),
                                            ctypes.byref(self._b)), "rom_batch_init")
        self.count = n

    def step(self, n_steps: int = 1):
        _lib.check(self._lib.rom_batch_step(self._b, int(n_steps)), "rom_batch_step")

    def state(self, i: int, q_tilde=True, phi=False, y_corr=False):
        c = self.cfgs[i]
        N, r = int(c.n_cells), int(c.r)
        qt = np.empty(N) if q_tilde else None
        a = np.empty(r)
        s = np.empty(r)
        ph = np.empty((r, N)) if phi else None
        yc = np.empty(N) if y_corr else None
        step = ctypes.c_int64()
        _lib.check(self._lib.rom_batch_state(self._b, int(i), None if qt is None else _dptr(qt),
                                             _dptr(a), _dptr(s), None if ph is None else _dptr(ph),
                                             None if yc is None else _dptr(yc), ctypes.byref(step)),
                   "rom_batch_state")
        return dict(q_tilde=qt, a=a, sigma=s, phi=None if ph is None else ph.T.copy(),
                    y_corr=yc, step=step.value)

    def q_tilde(self, i: int):
        return self.state(i)["q_tilde"]

    def info(self, i: int):
        v = [ctypes.c_int32() for _ in range(3)]
        _lib.check(self._lib.rom_batch_info(self._b, int(i), *[ctypes.byref(x) for x in v]),
                   "rom_batch_info")
        return dict(rank=v[0].value, rom_newton_iters=v[1].value, fom_newton_iters=v[2].value)

    def layout(self):
        bb, rows = ctypes.c_int64(), ctypes.c_int64()
        tiles, tile_rows = ctypes.c_int32(), ctypes.c_int32()
        grid, graph = ctypes.c_int32(), ctypes.c_int32()
        _lib.check(self._lib.rom_batch_layout(self._b, ctypes.byref(bb), ctypes.byref(rows),
                                              ctypes.byref(tiles), ctypes.byref(tile_rows),
                                              ctypes.byref(grid), ctypes.byref(graph)),
                   "rom_batch_layout")
        return dict(basis_bytes=bb.value, rows=rows.value, tiles=tiles.value,
                    tile_rows=tile_rows.value, grid=grid.value, graph=graph.value)

    def profile(self, enable: bool):
        _lib.check(self._lib.rom_batch_profile(self._b, 1 if enable else 0), "rom_batch_profile")

    def profile_read(self):
        ms = (ctypes.c_double * 3)()
        cnt = (ctypes.c_int64 * 3)()
        _lib.check(self._lib.rom_batch_profile_read(self._b, ms, cnt), "rom_batch_profile_read")
        return {p: dict(ms=ms[i], launches=cnt[i]) for i, p in enumerate(self.PHASES)}

    def work(self):
        it, by = ctypes.c_int64(), ctypes.c_double()
        _lib.check(self._lib.rom_batch_work(self._b, ctypes.byref(it), ctypes.byref(by)),
                   "rom_batch_work")
        return dict(newton_iters=it.value, sweep_bytes=by.value)

    def fom_work(self):
        """Coarse FOM work since the last profile call: Newton iterations times
        n_cells over all instances and events, and their algorithmic bytes."""
        it, by = ctypes.c_int64(), ctypes.c_double()
        _lib.check(self._lib.rom_batch_fom_work(self._b, ctypes.byref(it), ctypes.byref(by)),
                   "rom_batch_fom_work")
        return dict(row_iterations=it.value, fom_bytes=by.value)

    def close(self):
        if getattr(self, "_b", None) is not None and self._b.value:
            self._lib.rom_batch_destroy(self._b)
            self._b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fom_rhs_dev(problem, n_cells, nu, gamma, q_ptr: int, f_ptr: int, stream: int = 0):
    lib = _lib.load()
    _lib.check(lib.rom_fom_rhs_dev(problem, n_cells, nu, gamma, ctypes.c_void_p(q_ptr),
                                   ctypes.c_void_p(f_ptr), ctypes.c_void_p(stream)), "rom_fom_rhs_dev")


def fom_step_dev(problem, n_cells, nu, gamma, h, tol, max_iter, q_prev_ptr: int, q_ptr: int,
                 stream: int = 0) -> int:
    lib = _lib.load()
    it = ctypes.c_int32()
    _lib.check(lib.rom_fom_step_dev(problem, n_cells, nu, gamma, h, tol, max_iter,
                                    ctypes.c_void_p(q_prev_ptr), ctypes.c_void_p(q_ptr),
                                    ctypes.byref(it), ctypes.c_void_p(stream)), "rom_fom_step_dev")
    return it.value


def isvd_update_dev(n, r, lam, rank_tol, phi_ptr: int, sigma_ptr: int, y_ptr: int,
                    stream: int = 0, want_ubar: bool = False):
    lib = _lib.load()
    ub = np.zeros((r + 1) * (r + 1)) if want_ubar else None
    _lib.check(lib.rom_isvd_update_dev(n, r, lam, rank_tol, ctypes.c_void_p(phi_ptr),
                                       ctypes.c_void_p(sigma_ptr), ctypes.c_void_p(y_ptr),
                                       None if ub is None else _dptr(ub), ctypes.c_void_p(stream)),
               "rom_isvd_update_dev")
    return None if ub is None else ub.reshape(r + 1, r + 1).T


def debug_set_wait_limit(cycles: int):
    """Bound of every device-side wait of the library's kernels, in SM clock
    cycles (a test hook; <= 0 restores the default of about 2 s)."""
    lib = _lib.load()
    _lib.check(lib.rom_debug_set_wait_limit(int(cycles)), "rom_debug_set_wait_limit")


def adjoint(cfg, q0, target, n_steps: int, ckpt_every: int = 50, stream: int | None = None,
            want_q_final: bool = False):
    """J = 1/2 |q~^{n_T} - target|^2 of the adaptive ROM and its gradient with
    respect to nu and the initial state q0 (rom_adjoint). Returns
    (J, dJ/dnu, dJ/dq0[, q~^{n_T}])."""
    lib = _lib.load()
    c = make_config(cfg)
    n = int(cfg.n_cells) * int(cfg.n_var)
    q0 = np.ascontiguousarray(q0, dtype=np.float64)
    target = np.ascontiguousarray(target, dtype=np.float64)
    if q0.shape != (n,) or target.shape != (n,):
        raise ValueError(f"q0 and target must have {n} entries")
    J, dnu = ctypes.c_double(), ctypes.c_double()
    dq0 = np.empty(n)
    qf = np.empty(n) if want_q_final else None
    _lib.check(lib.rom_adjoint(ctypes.byref(c), _dptr(q0), _dptr(target), int(n_steps),
                               int(ckpt_every), ctypes.c_void_p(stream or 0),
                               ctypes.byref(J), ctypes.byref(dnu), _dptr(dq0),
                               None if qf is None else _dptr(qf)), "rom_adjoint")
    if want_q_final:
        return J.value, dnu.value, dq0, qf
    return J.value, dnu.value, dq0


def misfit_function():
    """A torch.autograd.Function over rom_adjoint: ``apply(nu, q0, cfg,
    target, n_steps, ckpt_every)`` returns J as a 0-d float64 tensor and
    backpropagates dJ/dnu and dJ/dq0 (device tensors on q0's device). The
    forward and reverse passes both run in the library's kernels; torch only
    carries the results."""
    import torch

    class _Misfit(torch.autograd.Function):
        @staticmethod
        def forward(ctx, nu, q0, cfg, target, n_steps, ckpt_every):
            import copy
            c = copy.copy(cfg)
            c.nu = float(nu.detach().cpu())
            J, dnu, dq0 = adjoint(c, q0.detach().cpu().double().numpy(),
                                  target.detach().cpu().double().numpy(), n_steps, ckpt_every)
            ctx.save_for_backward(torch.tensor(dnu, dtype=torch.float64, device=nu.device),
                                  torch.from_numpy(dq0).to(q0.device))
            return torch.tensor(J, dtype=torch.float64, device=q0.device)

        @staticmethod
        def backward(ctx, gJ):
            dnu, dq0 = ctx.saved_tensors
            return gJ * dnu, gJ * dq0, None, None, None, None

    return _Misfit
