"""The synthetic workloads' recipes (host logic, no GPU): the 512-lattice ensemble is deterministic,
its lattices stay inside the stated ranges, and each channel's body force gives the stated centre
speed of the mean medium, checked against a finite-difference solution of the 1-D Brinkman
equation (Eq. 23 without the Forchheimer term) rather than against the closed form it was set from."""
import math

import numpy as np
import pytest


@pytest.fixture(scope="module")
def lbm():
    from paper_1311_7239_gb300 import build, lbm

    build.build()
    return lbm


def _brinkman_centre_speed(H, nu, phi, K, a, n=4000):
    """u'' - (phi / K) u + phi a / nu = 0 on (0, H) with u = 0 at halfway walls 0 and H (nu_e = nu),
    second-order finite differences on n cells; returns u at y = H / 2."""
    h = H / n
    y = (np.arange(n - 1) + 1) * h
    main = np.full(n - 1, -2.0 / h**2 - phi / K)
    off = np.full(n - 2, 1.0 / h**2)
    A = np.diag(main) + np.diag(off, 1) + np.diag(off, -1)
    u = np.linalg.solve(A, np.full(n - 1, -phi * a / nu))
    return float(np.interp(H / 2, y, u))


def test_ensemble_domains_of_the_bench_form():
    from paper_1311_7239_gb300 import synth

    doms = list(synth.ensemble_domains(512, 42, 64, 1024))
    assert len(doms) == 512
    cells = sum(d["nx"] * d["ny"] for d in doms)
    assert abs(cells - 162e6) < 0.01 * 162e6                                # the 162 M cells of the bench form
    assert {d["kind"] for d in doms} == {"cavity", "channel"}
    assert all(64 <= d["nx"] <= 1024 and 64 <= d["ny"] <= 1024 for d in doms)
    assert all(10 <= d["Re"] <= 400 for d in doms)


def test_ensemble_configs_recipe(lbm):
    from paper_1311_7239_gb300 import synth, workloads

    cfgs, media = workloads.ensemble(lbm, n=24, seed=42, lo=64, hi=256)
    cfgs2, media2 = workloads.ensemble(lbm, n=24, seed=42, lo=64, hi=256)
    assert all(bytes(a) == bytes(b) for a, b in zip(cfgs, cfgs2))            # deterministic
    assert all(np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) for a, b in zip(media, media2))
    doms = list(synth.ensemble_domains(24, 42, 64, 256))
    for c, (eps, K), dom in zip(cfgs, media, doms):
        assert eps.shape == (c.ny, c.nx) and K.shape == (c.ny, c.nx)
        assert eps.min() >= 0.1 and eps.max() <= 0.9 and K.min() > 0
        assert abs(c.p_rest - float(eps.mean())) < 1e-6                      # rest state phi p = mean(eps)
        if c.bc_x == lbm.WALL:                                              # cavity: lid speed U
            speed = c.u_wall[3][0]
        else:                                                               # channel: the centre speed its force gives
            speed = _brinkman_centre_speed(c.ny, c.nu, c.phi, c.K, c.ax, n=800)
        # Re = U H / nu of the domain's draw, unless the viscosity floor (tau_v >= 0.56) holds nu up
        assert c.nu >= 0.02 - 1e-12 and (abs(c.nu - 0.02) < 1e-12 or abs(speed * c.ny / c.nu - dom["Re"]) < 0.02 * dom["Re"])
        assert speed / (math.sqrt(1 / 3) * math.sqrt(0.1)) <= 0.17          # |u| / (c_s sqrt(eps_min))


def test_ensemble_channel_force_gives_the_stated_centre_speed(lbm):
    from paper_1311_7239_gb300 import workloads

    cfgs, _ = workloads.ensemble(lbm, n=40, seed=7, lo=64, hi=256)
    channels = [c for c in cfgs if c.bc_x == lbm.PERIODIC]
    assert channels
    for c in channels[:6]:
        u_c = _brinkman_centre_speed(c.ny, c.nu, c.phi, c.K, c.ax)
        assert abs(u_c - 0.02) < 2e-4, (c.ny, u_c)
