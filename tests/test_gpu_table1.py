"""Natural convection in a square porous cavity (Sec. 3.4) run to steady state on the GPU and
compared with the average Nusselt numbers the paper prints in Table 1 (tests/golden/table1_nusselt.txt).

Set-up as Sec. 3.4: Pr = 1, J = sigma = gamma = 1, zeta3 = zeta4 = 1.1, T_h = 21, T_c = 1,
adiabatic top and bottom, Eq. 26 for tau_v and tau_T with Ma = 0.1 (the paper only bounds Ma by
0.3).  Walls are halfway bounce-back (anti-bounce-back for the temperature), so L = nx.  The
paper's "Present" column is matched within the spread it reports between its own result and
the two finite-element references (about 2-3 % at Ra = 1e5).
"""
import os

import numpy as np
import pytest

from oracle import thermal_d2q5 as th

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_nusselt.txt")


def _table():
    rows = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        da, ra, phi, present, ref4, ref7, grid = line.split()
        rows[(float(da), float(ra), float(phi))] = (float(present), float(ref4), None if ref7 == "-" else float(ref7), int(grid))
    return rows


@pytest.fixture(scope="module")
def lbm():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1311_7239_gb300 import build, lbm

    build.build()
    return lbm


def steady_nusselt(lbm, L, Da, Ra, phi, Ma=0.1, chunk=20000, max_steps=2_000_000, tol=2e-5):
    nu, tau_v, tau_T, gb = th.parameters_from_Ra(L, Ra, 1.0, Ma)
    cfg = lbm.default_config(nx=L, ny=L, bc_x=lbm.WALL, bc_y=lbm.WALL, nu=nu, phi=phi, K=Da * L * L, thermal=1,
                             tau_T=tau_T, g_beta=gb, T0=11.0, T_wall=[21.0, 1.0, None, None], p_rest=phi)
    with lbm.Lattice(cfg) as lat:
        prev = None
        steps = 0
        while steps < max_steps:
            lat.step(chunk)
            steps += chunk
            nu_l, nu_r = lat.nusselt(lbm.LEFT), lat.nusselt(lbm.RIGHT)
            if prev is not None and abs(nu_l - prev) <= tol * nu_l and abs(nu_l - nu_r) <= 1e-3 * nu_l:
                return nu_l, nu_r, steps
            prev = nu_l
    return nu_l, nu_r, steps


@pytest.mark.parametrize("Ra", [1e4, 1e5])
def test_table1_nusselt_da1e2_phi06(lbm, Ra):
    present, ref4, ref7, grid = _table()[(1e-2, Ra, 0.6)]
    nu_l, nu_r, steps = steady_nusselt(lbm, grid, 1e-2, Ra, 0.6)
    spread = max(abs(present - ref4), abs(present - ref7)) / present
    print(f"Ra={Ra:g}: Nu_left={nu_l:.4f} Nu_right={nu_r:.4f} after {steps} steps; Table 1 present {present} "
          f"(refs {ref4}, {ref7}); rel. diff {abs(nu_l - present) / present:.3%}")
    assert abs(nu_l - present) <= max(0.02, spread) * present
