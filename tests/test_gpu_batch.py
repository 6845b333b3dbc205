"""Batched ensembles (lbm_batch_*): the persistent batched kernel gives bitwise the results of the
single-lattice kernel on every lattice, for every launch shape; the one-by-one mode and the
autotuner leave results unchanged; a small lattice of the batch matches the FP64 oracle.  Batches
with in-place streaming give bitwise the results of single in-place lattices."""
import numpy as np
import pytest

from oracle import mrt_d2q8 as fl
from paper_1311_7239_gb300 import workloads as ensemble
from tests.cases import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1311_7239_gb300 import build, lbm

    build.build()
    return lbm


def _singles(lbm, cfgs, media, steps):
    import torch

    out = []
    for cfg, (eps, K) in zip(cfgs, media):
        lat = lbm.Lattice(lbm.Config.from_buffer_copy(cfg))
        lat.set_medium(torch.tensor(eps, device="cuda"), torch.tensor(K, device="cuda"))
        lat.init_equilibrium(float(cfg.p_rest), 0.0, 0.0, phi_p_uniform=True)
        lat.step(steps)
        out.append(lat.get_populations().cpu().numpy())
        lat.close()
    return out


@pytest.mark.parametrize("prec", [0, 1])
def test_batch_equals_single_lattices_bitwise(lbm, prec):
    cfgs, media = ensemble.ensemble(lbm, n=7, seed=3, lo=8, hi=300, precision=prec)
    steps = 45
    want = _singles(lbm, cfgs, media, steps)
    # (threads per CTA, CTAs per SM, work items per CTA): persistent grids, one CTA per item, CTAs of
    # 2, 4 and 8 consecutive items
    for tiling in (lbm.TILING_FLAT, lbm.TILING_ROWS):
        for shape in [(128, 4, 1), (64, 8, 1), (256, 2, 1), (128, 32, 1), (128, 0, 1), (64, 0, 1), (128, 0, 2), (64, 0, 4),
                      (256, 0, 8)]:
            with ensemble.build(lbm, cfgs, media) as b:
                b.set_tiling(tiling)
                b.set_items_per_cta(shape[2])
                b.set_launch(*shape[:2])
                assert b.get_tiling() == tiling and b.get_items_per_cta() == shape[2]
                b.step(steps)  # a graph of 32 + 13 launches
                b.sync()
                for d in range(len(cfgs)):
                    got = b.get_populations(d).cpu().numpy()
                    assert np.array_equal(got, want[d]), (tiling, shape, d)
                assert b.info()["steps"] == steps


def test_step_each_and_tune_leave_results_unchanged(lbm):
    cfgs, media = ensemble.ensemble(lbm, n=5, seed=11, lo=16, hi=200)
    with ensemble.build(lbm, cfgs, media) as a, ensemble.build(lbm, cfgs, media) as b:
        nt, k, ms = a.tune(steps=3)
        assert nt in (64, 128, 256) and 0 <= k <= 16 and ms > 0
        assert a.get_launch() == (nt, k) and a.get_tiling() in (lbm.TILING_ROWS, lbm.TILING_FLAT)
        assert a.get_items_per_cta() in (1, 2, 4) and (k == 0 or a.get_items_per_cta() == 1)
        a.step(40)
        b.step_each(40)
        for d in range(len(cfgs)):
            assert np.array_equal(a.get_populations(d).cpu().numpy(), b.get_populations(d).cpu().numpy())


def test_batch_lattice_matches_oracle(lbm):
    cfgs, media = ensemble.ensemble(lbm, n=3, seed=5, lo=12, hi=40)
    steps = 300
    with ensemble.build(lbm, cfgs, media) as b:
        b.step(steps)
        res = [tuple(t.cpu().numpy() for t in b.macros(d)) for d in range(3)]
    for d, cfg in enumerate(cfgs):
        eps, K = media[d]
        kind_wall = cfg.bc_x == lbm.WALL
        flow = fl.Flow(nx=cfg.nx, ny=cfg.ny, phi=eps.astype(np.float64), K=K.astype(np.float64), nu=cfg.nu,
                       accel=np.array([cfg.ax, 0.0]), bc_x="wall" if kind_wall else "periodic", bc_y="wall",
                       u_top=(cfg.u_wall[3][0], 0.0))
        f = fl.run(fl.initial_state(flow, p0=cfg.p_rest / flow.phi), flow, steps)
        ux, uy, p = fl.macroscopic(f, flow)
        pg, uxg, uyg = res[d]
        assert rel_l2(np.stack([uxg, uyg]), np.stack([ux, uy])) <= 1e-5
        assert rel_l2(pg, p) <= 1e-5


def test_tuning_choice_is_cached_on_disk(lbm, tmp_path):
    cfgs, media = ensemble.ensemble(lbm, n=4, seed=2, lo=16, hi=96)
    path = str(tmp_path / "tune.json")
    with ensemble.build(lbm, cfgs, media) as b:
        nt, k, ms, hit = b.tune_cached(path, steps=2)
        assert not hit
    with ensemble.build(lbm, cfgs, media) as b:
        nt2, k2, ms2, hit2 = b.tune_cached(path, steps=2)
        assert hit2 and (nt2, k2) == (nt, k) and b.get_launch() == (nt, k)


def _inplace(lbm, cfgs):
    for c in cfgs:
        c.streaming = lbm.STREAM_INPLACE
    return cfgs


@pytest.mark.parametrize("prec", [0, 1])
def test_inplace_batch_equals_single_inplace_lattices_bitwise(lbm, prec):
    cfgs, media = ensemble.ensemble(lbm, n=7, seed=3, lo=8, hi=300, precision=prec)
    cfgs = _inplace(lbm, cfgs)
    steps = 45
    want = _singles(lbm, cfgs, media, steps)
    with ensemble.build(lbm, cfgs, media) as b:
        assert b.get_launch() == (128, 0)
        with pytest.raises(lbm.LbmError):
            b.set_launch(64, 0)
        b.step(steps)  # a graph of 32 + 13 launches (both parities)
        b.sync()
        for d in range(len(cfgs)):
            assert np.array_equal(b.get_populations(d).cpu().numpy(), want[d]), d


def test_inplace_batch_step_each_tune_and_memory(lbm):
    cfgs, media = ensemble.ensemble(lbm, n=5, seed=11, lo=16, hi=200)
    with ensemble.build(lbm, cfgs, media) as ab:
        bytes_ab = ab.info()["bytes"]
    cfgs = _inplace(lbm, cfgs)
    with ensemble.build(lbm, cfgs, media) as a, ensemble.build(lbm, cfgs, media) as b:
        nt, k, ms = a.tune(steps=3)
        assert (nt, k) == (128, 0) and ms > 0
        a.step(41)
        b.step_each(41)
        for d in range(len(cfgs)):
            assert np.array_equal(a.get_populations(d).cpu().numpy(), b.get_populations(d).cpu().numpy())
        assert a.info()["bytes"] < 0.75 * bytes_ab  # one population pool instead of two (media stay)
    mixed = list(cfgs)
    mixed[1].streaming = lbm.STREAM_AB
    with pytest.raises(lbm.LbmError):
        ensemble.build(lbm, mixed, media)
