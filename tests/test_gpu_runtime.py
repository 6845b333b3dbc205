"""Runtime services around the step: checkpoint/resume is bitwise, and host-side allocation
faults come back as clean status codes."""
import os
import subprocess
import sys

import numpy as np
import pytest

from tests.cases import Case

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lbm():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1311_7239_gb300 import build, lbm

    build.build()
    return lbm


@pytest.mark.parametrize("thermal", [False, True])
def test_save_load_resumes_bitwise(lbm, tmp_path, thermal):
    if thermal:
        from tests.test_gpu_parity import _thermal_case

        case = _thermal_case(L=40)
    else:
        case = Case(70, 40, nu=0.05, phi=0.5, K=3.0, het=True, bc_x="wall", bc_y="wall", walls={"top": (0.08, 0.0)})
    path = str(tmp_path / "state.lbm")
    with case.lattice(lbm) as a:
        a.step(37)
        a.save(path)
        a.step(45)
        fa = a.get_populations()
        ra = a.residual()
    cfg = case.config(lbm)
    with lbm.Lattice(cfg) as b:  # fresh context, uniform medium until the load brings the saved one
        b.load(path)
        assert b.step_count() == 37
        b.step(45)
        fb = b.get_populations()
        rb = b.residual()
    if thermal:
        assert np.array_equal(fa[0].cpu().numpy(), fb[0].cpu().numpy()) and np.array_equal(fa[1].cpu().numpy(), fb[1].cpu().numpy())
    else:
        assert np.array_equal(fa.cpu().numpy(), fb.cpu().numpy())
    assert ra == rb


def test_load_rejects_mismatched_state(lbm, tmp_path):
    path = str(tmp_path / "state.lbm")
    with Case(30, 20).lattice(lbm) as a:
        a.save(path)
    with Case(31, 20).lattice(lbm) as b:
        with pytest.raises(lbm.LbmError) as e:
            b.load(path)
        assert e.value.code == lbm.EINVAL
    with Case(30, 20).lattice(lbm) as b:
        with pytest.raises(lbm.LbmError):
            b.load(str(tmp_path / "missing.lbm"))


@pytest.mark.parametrize("k", [1, 3, 5])
def test_injected_allocation_failure_is_enomem(lbm, k):
    code = (
        "import sys; sys.path.insert(0, %r)\n"
        "from paper_1311_7239_gb300 import lbm\n"
        "try:\n"
        "    lbm.Lattice(nx=64, ny=32)\n"
        "    print('created')\n"
        "except lbm.LbmError as e:\n"
        "    print('code', e.code)\n"
        "lat = lbm.Lattice(nx=64, ny=32); lat.step(3); lat.sync(); print('second ok')\n" % ROOT
    )
    r = subprocess.run([sys.executable, "-c", code], env=dict(os.environ, LBM_FAULT_ALLOC=str(k)), capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr
    assert "code -2" in r.stdout and "second ok" in r.stdout


def test_write_fields_round_trip(lbm, tmp_path):
    import numpy as np

    cfg = lbm.default_config(nx=20, ny=12, bc_x=lbm.WALL, bc_y=lbm.WALL, u_wall=[(0, 0), (0, 0), (0, 0), (0.05, 0)])
    with lbm.Lattice(cfg) as lat:
        lat.step(17)
        p, ux, uy = [t.cpu().numpy() for t in lat.macros()]
        lat.write_fields(tmp_path / "fields.npz")
    z = np.load(tmp_path / "fields.npz")
    assert int(z["step"]) == 17
    assert np.array_equal(z["p"], p) and np.array_equal(z["ux"], ux) and np.array_equal(z["uy"], uy)


@pytest.mark.parametrize("prec", [0, 1])
def test_bench_cavity_stays_bounded_for_50k_steps(lbm, prec):
    """The 4096^2 benchmark cavity (eps 0.4, Da 1e-3, Re 100, lid 0.1) for the 50k steps of its
    configuration: no non-finite velocity, speeds below the lid's, a small per-step change (the
    flow is still spinning up: its viscous time L^2 / nu is 4M steps)."""
    L = 4096
    cfg = lbm.default_config(nx=L, ny=L, bc_x=lbm.WALL, bc_y=lbm.WALL, nu=0.1 * L / 100, phi=0.4, K=1e-3 * L * L,
                             u_wall=[(0, 0), (0, 0), (0, 0), (0.1, 0)], precision=prec, p_rest=0.4, dev_scale_log2=10)
    with lbm.Lattice(cfg) as lat:
        lat.step(9999)
        lat.step(1)
        r1 = lat.residual()
        lat.step(39999)
        lat.step(1)
        r2 = lat.residual()
        _, ux, uy = lat.macros()
        umax = float((ux * ux + uy * uy).sqrt().max())
        lat.sync()
        assert lat.step_count() == 50000
    assert umax <= 0.1 and 0 < r1 < 1e-2 and 0 < r2 < 1e-2, (umax, r1, r2)


def test_probe_async_matches_probe_in_a_pipelined_loop(lbm):
    """lbm_probe_async into pinned host memory (two buffers, an event per step) gives, one step
    later, what lbm_probe gives after each step; the same into device memory."""
    import torch

    case = Case(64, 40, nu=0.05, phi=0.5, K=3.0, bc_x="wall", bc_y="wall", walls={"top": (0.1, 0.0)}, het=True)
    stream = torch.cuda.current_stream()
    with case.lattice(lbm) as a, case.lattice(lbm) as b:
        bufs = [torch.zeros(4, dtype=torch.float32).pin_memory() for _ in range(2)]
        evs = [torch.cuda.Event() for _ in range(2)]
        want, got = [], []
        for k in range(12):
            a.step(1)
            want.append(a.probe(31, 20).copy())
            b.step(1)
            b.probe_async(31, 20, bufs[k & 1])
            evs[k & 1].record(stream)
            if k:
                evs[(k - 1) & 1].synchronize()
                got.append(bufs[(k - 1) & 1].numpy().copy())
        evs[11 & 1].synchronize()
        got.append(bufs[11 & 1].numpy().copy())
        assert all(np.array_equal(g, w) for g, w in zip(got, want))
        dev = torch.zeros(4, dtype=torch.float32, device="cuda")
        b.probe_async(31, 20, dev)
        b.sync()
        assert np.array_equal(dev.cpu().numpy(), a.probe(31, 20))


def test_set_walls_from_pageable_pinned_and_device_memory(lbm):
    """A lid set with lbm_set_walls before stepping gives bitwise the run of a lattice created with
    that lid, whether the velocities come from pageable host memory (a copy), page-locked host
    memory (read by the device directly) or device memory."""
    import torch

    lid = Case(48, 32, nu=0.05, phi=0.5, K=3.0, bc_x="wall", bc_y="wall", walls={"top": (0.1, 0.0), "left": (0.0, 0.02)})
    still = Case(48, 32, nu=0.05, phi=0.5, K=3.0, bc_x="wall", bc_y="wall")
    w = np.zeros((4, 2), np.float32)
    w[3, 0], w[0, 1] = 0.1, 0.02
    sources = [w, torch.from_numpy(w).pin_memory(), torch.from_numpy(w).cuda()]
    # (the stored initial state depends on the walls through the moving-wall term of the links
    # that cross them, so both lattices are initialised after their walls are set)
    with lid.lattice(lbm) as ref:
        ref.init_equilibrium(1.0, 0.0, 0.0)
        ref.step(40)
        want = ref.get_populations().cpu().numpy()
    for src in sources:
        with still.lattice(lbm) as lat:
            lat.set_walls(src)
            lat.init_equilibrium(1.0, 0.0, 0.0)
            lat.step(40)
            got = lat.get_populations().cpu().numpy()
        assert np.array_equal(got, want), type(src)
    # and a change between steps takes effect from the next step: set before step 21 of 40
    with lid.lattice(lbm) as ref, lid.lattice(lbm) as lat:
        ref.init_equilibrium(1.0, 0.0, 0.0)
        lat.init_equilibrium(1.0, 0.0, 0.0)
        w2 = w.copy()
        w2[3, 0] = 0.05
        ref.step(20)
        ref.set_walls(w2)
        ref.step(20)
        lat.step(20)
        w2_pinned = torch.from_numpy(w2).pin_memory()  # read when the stream gets there: kept alive
        lat.set_walls(w2_pinned)
        lat.step(20)
        assert np.array_equal(lat.get_populations().cpu().numpy(), ref.get_populations().cpu().numpy())
