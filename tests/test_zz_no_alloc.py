"""lbm_residual_noalloc, the residual for callers that must not allocate device memory, against
lbm_residual of a context over the same two states, on two calls in a row.

Collected last on purpose (file name), so a run that stops at the first failure has run every
other test before this one; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1311_7239_gb300 import build, lbm

    build.build()
    return lbm


def _noalloc(lbm, ux, uy, uxp, uyp, r_ptr, stream):
    return lbm.lib().lbm_residual_noalloc(ux.data_ptr(), uy.data_ptr(), uxp.data_ptr(), uyp.data_ptr(), ux.numel(), r_ptr,
                                          stream)


def test_noalloc_residual_matches_context_residual_twice(lbm):
    import torch

    nx, ny = 72, 40
    lat = lbm.Lattice(nx=nx, ny=ny, bc_x=lbm.WALL, bc_y=lbm.WALL, nu=0.05, phi=0.5, K=2.0, p_rest=0.5,
                      u_wall=[(0, 0), (0, 0), (0, 0), (0.1, 0)])
    stream = ctypes.c_void_p(lat.cfg.stream)
    r_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    lat.step(30)
    _, ux_prev, uy_prev = lat.macros()
    for call in range(2):
        lat.step(1)
        want = lat.residual()  # context path: u(t) and u(t-1) gathered from its two buffers
        _, ux, uy = lat.macros()
        # device output
        rc = _noalloc(lbm, ux, uy, ux_prev, uy_prev, ctypes.c_void_p(r_dev.data_ptr()), stream)
        assert rc == lbm.OK, lbm.lib().lbm_last_error()
        got_dev = float(r_dev.cpu()[0])
        # host output
        r_host = ctypes.c_double(-1.0)
        rc = _noalloc(lbm, ux, uy, ux_prev, uy_prev, ctypes.cast(ctypes.byref(r_host), ctypes.c_void_p), stream)
        assert rc == lbm.OK, lbm.lib().lbm_last_error()
        assert want > 0
        assert abs(got_dev - want) <= 1e-3 * want, (call, got_dev, want)
        assert abs(r_host.value - want) <= 1e-3 * want, (call, r_host.value, want)
        ux_prev, uy_prev = ux, uy
    lat.close()


def test_noalloc_rejects_sizes_beyond_its_scratch(lbm):
    import torch

    a = torch.zeros(4, dtype=torch.float32, device="cuda")
    r = ctypes.c_double(0.0)
    L = lbm.lib()
    rc = L.lbm_residual_noalloc(a.data_ptr(), a.data_ptr(), a.data_ptr(), a.data_ptr(), (1 << 26) + 1,
                                ctypes.cast(ctypes.byref(r), ctypes.c_void_p), None)
    assert rc == lbm.EINVAL
    assert b"67108864" in L.lbm_last_error()
    rc = L.lbm_residual_noalloc(a.data_ptr(), a.data_ptr(), a.data_ptr(), a.data_ptr(), 0,
                                ctypes.cast(ctypes.byref(r), ctypes.c_void_p), None)
    assert rc == lbm.EINVAL
