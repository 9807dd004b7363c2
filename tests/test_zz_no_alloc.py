"""wd_apply_f32_noalloc: the FP32 operator for callers that cannot allocate
device memory (a process whose device memory belongs to another allocator,
or code that must not synchronise the device).  It keeps its scratch in a
static device array; this file runs last so that a failure here stops a run
only after every other test has run.

Checked through the C ABI against wd_apply_f32, which allocates its scratch,
on two calls in a row, within the FP32 operator's tolerance (2e-6 relative)."""
import ctypes

import numpy as np
import pytest

from inputs import lattice as L

pytestmark = pytest.mark.gpu

TOL = 2e-6


def _call(lib, fn, h, x, y, nrhs, dagger):
    import torch
    rc = getattr(lib, fn)(h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                          nrhs, dagger, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return rc


@pytest.mark.parametrize("dims,nrhs", [((16, 16, 16, 16), 2), ((6, 4, 2, 8), 3)])
def test_noalloc_matches_allocating_entry_point(dims, nrhs):
    import torch
    import paper_0710_1988_gb300 as wdl
    lib = wdl.lib()
    U = L.gauge_field(dims, 0.5, 900)
    op = wdl.WilsonOperator(dims, torch.from_numpy(U).cuda(), 0.1362, 0.02)
    n = 12 * L.volume(dims)
    for call in range(2):  # two calls in a row, different inputs
        x = torch.from_numpy(L.gaussian_spinor(dims, 901 + call, nrhs=nrhs).ravel()).cuda()
        ref = torch.empty_like(x)
        got = torch.full_like(x, float("nan"))
        dagger = call % 2
        assert _call(lib, "wd_apply_f32", op._h, x, ref, nrhs, dagger) == 0
        assert _call(lib, "wd_apply_f32_noalloc", op._h, x, got, nrhs, dagger) == 0
        r = ref.cpu().numpy().reshape(nrhs, n)
        g = got.cpu().numpy().reshape(nrhs, n)
        assert np.all(np.isfinite(g))
        for q in range(nrhs):
            assert np.abs(g[q] - r[q]).max() <= TOL * np.abs(r[q]).max()
    op.close()


def test_noalloc_rejects_requests_beyond_the_scratch():
    import torch
    import paper_0710_1988_gb300 as wdl
    from paper_0710_1988_gb300 import _lib
    lib = wdl.lib()
    dims = (16, 16, 16, 16)                 # V (12 + 12 nrhs) float4 > 64 MiB for nrhs = 5
    op = wdl.WilsonOperator(dims, torch.from_numpy(L.unit_gauge_field(dims)).cuda(), 0.1)
    x = torch.zeros(5 * 12 * L.volume(dims), dtype=torch.complex128, device="cuda:0")
    y = torch.empty_like(x)
    assert _call(lib, "wd_apply_f32_noalloc", op._h, x, y, 5, 0) == _lib.WD_BAD_ARG
    assert "static scratch" in _lib.last_error()
    op.close()
