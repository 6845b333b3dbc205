"""lbm_residual_noalloc, the residual for callers that must not allocate device memory (a
service with one memory pool sized at start-up, a framework that owns all device memory, a
real-time loop that cannot absorb the device-wide synchronisation of cudaMalloc/cudaFree):

* against lbm_residual of a context over the same two states, on two calls in a row;
* against the FP64 oracle's residual of the same seeded float32 fields, for one block, several
  blocks with a ragged last one, a ragged n of five million and the largest accepted n (2^26
  cells: all 4096 partial-sum slots of its fixed scratch array), each with two back-to-back calls
  on one stream whose second result must not depend on what the first left in the array.

Collected last on purpose (file name), so a run that stops at the first failure has run every
other test before this one; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from oracle import mrt_d2q8 as fl

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
        # both are FP64 sums of the same FP32 velocities (the same read-out of the populations)
        assert abs(got_dev - want) <= 1e-10 * want, (call, got_dev, want)
        assert abs(r_host.value - want) <= 1e-10 * want, (call, r_host.value, want)
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


def _fields(n, seed):
    """Seeded float32 velocity fields u(t), u(t-1) of n cells: a smooth-ish field and a small change."""
    rng = np.random.default_rng(seed)
    ux = rng.standard_normal(n, dtype=np.float32) * np.float32(0.05)
    uy = rng.standard_normal(n, dtype=np.float32) * np.float32(0.05)
    uxp = ux + rng.standard_normal(n, dtype=np.float32) * np.float32(1e-4)
    uyp = uy + rng.standard_normal(n, dtype=np.float32) * np.float32(1e-4)
    return ux, uy, uxp, uyp


def _oracle_residual(ux, uy, uxp, uyp, chunk=1 << 22):
    """The oracle's residual of the float32 fields promoted to FP64 (in chunks of the sums it forms,
    to bound host memory at 2^26 cells)."""
    if ux.size <= chunk:
        return fl.residual(*(a.astype(np.float64) for a in (ux, uy, uxp, uyp)))
    num = den = 0.0
    for k in range(0, ux.size, chunk):
        a, b, c, d = (v[k:k + chunk].astype(np.float64) for v in (ux, uy, uxp, uyp))
        r = fl.residual(a, b, c, d)
        dk = float(np.sum(a * a + b * b))
        num += r * r * dk
        den += dk
    return float(np.sqrt(num / den))


@pytest.mark.parametrize("n", [2880, 300 * 217, 5_000_003, 1 << 26], ids=["1-block", "4-blocks-ragged", "5M-ragged", "max-2^26"])
def test_noalloc_residual_matches_oracle_back_to_back(lbm, n):
    """Two calls in a row on one stream with different fields; the second result is read only after
    both calls are queued, so it must come from its own partial sums (each call writes every slot it
    reads).  FP64 sums on both sides: agreement to 1e-12 relative."""
    import torch

    s = torch.cuda.Stream()
    r_dev = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
    want, args = [], []
    for seed in (1, 2):
        host = _fields(n, seed + n % 97)
        want.append(_oracle_residual(*host))
        args.append([torch.from_numpy(a).cuda() for a in host])
    torch.cuda.synchronize()
    for call in range(2):
        rc = _noalloc(lbm, *args[call], ctypes.c_void_p(r_dev.data_ptr() + 8 * call), ctypes.c_void_p(s.cuda_stream))
        assert rc == lbm.OK, lbm.lib().lbm_last_error()
    s.synchronize()
    got = r_dev.cpu().numpy()
    for call in range(2):
        assert want[call] > 0
        assert abs(got[call] - want[call]) <= 1e-12 * want[call], (n, call, got[call], want[call])
    # the same through a host result (the call waits for its stream)
    r_host = ctypes.c_double(-1.0)
    rc = _noalloc(lbm, *args[0], ctypes.cast(ctypes.byref(r_host), ctypes.c_void_p), ctypes.c_void_p(s.cuda_stream))
    assert rc == lbm.OK and abs(r_host.value - want[0]) <= 1e-12 * want[0], (rc, r_host.value, want[0])
    del args
    torch.cuda.empty_cache()
