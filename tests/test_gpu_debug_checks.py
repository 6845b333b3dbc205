"""The debug build of the library (-DLBM_DEBUG: every kernel checks its index invariants and sets
an error bit instead of leaving its buffers) runs small and ragged lattices of every boundary set-up
and storage precision, both streaming forms (A-B and in-place), the thermal step, ensembles in both
launch forms and the adjoint (pressure columns and wall nodes) without reporting a violation."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import itertools, sys
import numpy as np
import torch
from paper_1311_7239_gb300 import lbm, workloads
bcs = {"periodic": lbm.PERIODIC, "wall": lbm.WALL, "pressure": lbm.PRESSURE, "nee": lbm.NEE}
runs = 0
for (nx, ny), (bx, by), prec in itertools.product([(2, 3), (3, 2), (5, 7), (33, 17), (130, 9), (600, 5), (1100, 6)],
                                                  [("periodic", "wall"), ("wall", "wall"), ("pressure", "wall"), ("nee", "nee"),
                                                   ("periodic", "periodic"), ("wall", "periodic"), ("periodic", "nee"),
                                                   ("pressure", "nee"), ("nee", "wall")],
                                                  [0, 1, 2]):
    for thermal, streaming in itertools.product((0, 1), (0, 1)):
        kw = dict(nx=nx, ny=ny, bc_x=bcs[bx], bc_y=bcs[by], precision=prec, u_wall=[(0, 0.01), (0, 0), (0, 0), (0.05, 0)],
                  p_in=1.001, p_out=0.999, ax=1e-5, streaming=streaming)
        if thermal:
            kw.update(thermal=1, tau_T=0.8, g_beta=1e-4, T0=11.0, T_wall=[21.0, 1.0, None, None])
        try:
            lat = lbm.Lattice(lbm.default_config(**kw))
        except lbm.LbmError:
            continue  # a set-up the library rejects (too small for its boundaries)
        with lat:
            eps = torch.full((ny, nx), 0.5, device="cuda") + 0.1 * torch.rand(ny, nx, device="cuda")
            lat.set_medium(eps, torch.full((ny, nx), 5.0, device="cuda"))
            lat.init_equilibrium(0.5, 0.0, 0.0, phi_p_uniform=True)
            lat.step(37)
            pops = lat.get_populations()
            lat.set_populations(*(pops if thermal else (pops,)))
            lat.step(2)
            lat.macros()
            lat.residual()
            if thermal and bx in ("wall", "nee"):
                lat.nusselt(lbm.LEFT)
            lat.sync()
            runs += 1
cfgs, media = workloads.ensemble(lbm, n=9, seed=3, lo=8, hi=300)
with workloads.build(lbm, cfgs, media) as b:
    for tiling in (lbm.TILING_FLAT, lbm.TILING_ROWS):
        b.set_tiling(tiling)
        for shape in [(64, 0), (128, 0), (128, 2), (256, 1)]:
            b.set_launch(*shape)
            b.step(11)
            b.sync()
for prec in (0, 1):
    cfgs, media = workloads.ensemble(lbm, n=9, seed=3, lo=8, hi=300, precision=prec)
    for c in cfgs:
        c.streaming = lbm.STREAM_INPLACE
    with workloads.build(lbm, cfgs, media) as b:
        b.step(11)
        b.step_each(3)
        b.macros(4)
        b.sync()
cfg = lbm.default_config(nx=40, ny=17, bc_x=lbm.PRESSURE, bc_y=lbm.WALL, p_in=1.002, p_out=0.998, phi=0.4, K=4.0, p_rest=0.4)
with lbm.Lattice(cfg) as lat:
    lat.set_medium(torch.full((17, 40), 0.4, device="cuda") + 0.05 * torch.rand(17, 40, device="cuda"), None)
    lat.init_equilibrium(0.4, 0.0, 0.0, phi_p_uniform=True)
    lat.adjoint(20, "flux")
for bx, by in ((lbm.NEE, lbm.NEE), (lbm.PRESSURE, lbm.NEE), (lbm.PERIODIC, lbm.NEE), (lbm.NEE, lbm.WALL)):
    cfg = lbm.default_config(nx=37, ny=9, bc_x=bx, bc_y=by, p_in=1.002, p_out=0.998, u_wall=[(0, 0.01), (0, 0), (0, 0), (0.05, 0)])
    with lbm.Lattice(cfg) as lat:
        lat.init_equilibrium(1.0, 0.0, 0.0)
        lat.adjoint(12, "flux")
print("runs", runs)
'''


def test_debug_build_reports_no_index_violation():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1311_7239_gb300 import build

    path = build.build(debug=True)
    env = dict(os.environ, LBM_LIBRARY=path, PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", SCRIPT], env=env, capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "runs" in r.stdout
