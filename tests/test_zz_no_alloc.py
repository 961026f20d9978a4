"""The allocation-free FOM step against the allocating one, through the C ABI.

rom_fom_step_noalloc_dev is for callers that must not allocate device memory
(a host that owns all device memory through its own pool, or a time-critical
loop that cannot pay for cudaMalloc/cudaFree). It keeps its scratch in one
fixed array inside the library, so it must give the same result as
rom_fom_step_dev on every call, including a second call right after the first
(the array still holds the previous call's contents). This file is collected
last so that a stop at the first failure has already run every other test."""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_noalloc_fom_step_matches_allocating_entry_point():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_28684_gb300 import build, _lib
    build.build()
    lib = _lib.load()
    n, nu, h = 16384, 2e-3, 5e-4
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    q = torch.tensor(synth.burgers_ic(n, 5), device="cuda", dtype=torch.float64)
    for call in range(2):
        ref = torch.empty_like(q)
        out = torch.full_like(q, float("nan"))
        it_ref, it_out = ctypes.c_int32(), ctypes.c_int32()
        rc = lib.rom_fom_step_dev(0, n, nu, 1.4, h, 1e-12, 20, ctypes.c_void_p(q.data_ptr()),
                                  ctypes.c_void_p(ref.data_ptr()), ctypes.byref(it_ref), stream)
        assert rc == 0
        rc = lib.rom_fom_step_noalloc_dev(0, n, nu, 1.4, h, 1e-12, 20,
                                          ctypes.c_void_p(q.data_ptr()),
                                          ctypes.c_void_p(out.data_ptr()), ctypes.byref(it_out),
                                          stream)
        assert rc == 0, call
        r, o = ref.cpu().numpy(), out.cpu().numpy()
        assert it_out.value == it_ref.value
        # same tolerance as the FOM parity tests
        assert np.max(np.abs(o - r)) <= 1e-11 * np.max(np.abs(r)), call
        q = out.clone()          # the second call advances from the first one's result
    # sizes beyond the fixed scratch are rejected
    big = 131072 + 1
    rc = lib.rom_fom_step_noalloc_dev(0, big, nu, 1.4, h, 1e-12, 20, ctypes.c_void_p(q.data_ptr()),
                                      ctypes.c_void_p(q.data_ptr() + 8), None, stream)
    assert rc == 1
