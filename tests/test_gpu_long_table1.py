"""Table 1's Da = 1e-6, Ra = 1e9 rows (Sec. 3.4): natural convection in a porous cavity run to
steady state on the GPU against the printed average Nusselt numbers of the hot wall.

The paper's 250 grid would put tau_v of Eq. 26 at 0.5041 even at Ma = 0.3; an 800 grid at
Ma = 0.3 (the bound the paper states) gives tau_v = 0.5131.  The steady state is reached after
about 8 million steps (the hot-wall Nusselt number then changes by less than 1e-6 per 2 million
steps), several GPU-minutes per row, so these tests carry their own marker and are not part of
``-m gpu``:

    python -m pytest tests/test_gpu_long_table1.py -m gpu_long

Measured (GB300, halfway walls): Nu = 12.414 at eps = 0.6 on 800^2 (converged); 11.915 / 12.378 /
12.714 for eps = 0.4 / 0.6 / 0.9 on 1200^2 after 24 million steps.  Table 1 prints 11.476 / 11.878 /
12.142, so these rows are 3.8-4.7 % above the paper, outside the 2 % within which the other 24 rows
match; the grid changes the result by 0.3 % (800^2 to 1200^2).  The tests therefore check the
steady state and the hot/cold balance, and bound the deviation from Table 1 at 6 % as a regression
check: they do not count as a match.
"""
import pytest

from oracle import thermal_d2q5 as th
from tests.test_gpu_table1 import _table, lbm  # noqa: F401  (lbm: the module fixture)

pytestmark = pytest.mark.gpu_long


def _run(lbm, L, Da, Ra, phi, Ma, chunk, max_steps, tol):
    """Halfway walls, Eq. 26 parameters; chunks until the hot-wall Nusselt number changes by less than
    tol (relative) over a chunk.  Returns (Nu_left, Nu_right, steps, steady)."""
    nu, tau_v, tau_T, gb = th.parameters_from_Ra(L, Ra, 1.0, Ma)
    cfg = lbm.default_config(nx=L, ny=L, bc_x=lbm.WALL, bc_y=lbm.WALL, nu=nu, phi=phi, K=Da * L * L, thermal=1, tau_T=tau_T,
                             g_beta=gb, T0=11.0, T_wall=[21.0, 1.0, None, None], p_rest=phi)
    with lbm.Lattice(cfg) as lat:
        prev, steps = None, 0
        while steps < max_steps:
            lat.step(chunk)
            steps += chunk
            nu_l, nu_r = lat.nusselt(lbm.LEFT), lat.nusselt(lbm.RIGHT)
            if prev is not None and abs(nu_l - prev) <= tol * nu_l:
                return nu_l, nu_r, steps, True
            prev = nu_l
    return nu_l, nu_r, steps, False


@pytest.mark.parametrize("phi", [0.4, 0.6, 0.9])
def test_table1_nusselt_ra1e9_bounded(lbm, phi):  # noqa: F811
    Da, Ra, grid, Ma = 1e-6, 1e9, 800, 0.3
    present, ref4, ref7, _ = _table()[(Da, Ra, phi)]
    nu_l, nu_r, steps, steady = _run(lbm, grid, Da, Ra, phi, Ma, chunk=1_000_000, max_steps=16_000_000, tol=1e-5)
    print(f"{grid}^2 halfway walls, Ma={Ma}, Da={Da:g} Ra={Ra:g} phi={phi}: Nu_left={nu_l:.4f} Nu_right={nu_r:.4f} after {steps} "
          f"steps; Table 1 present {present} (refs {[r for r in (ref4, ref7) if r is not None]}); "
          f"rel. diff {(nu_l - present) / present:+.3%}")
    assert steady                                               # the steady-state test was met
    assert abs(nu_l - nu_r) <= 5e-3 * nu_l                      # heat in = heat out
    assert abs(nu_l - present) <= 0.06 * present               # regression bound, not a match (see above)
