"""Table 1's Da = 1e-6, Ra = 1e9 rows (Sec. 3.4): natural convection in a porous cavity run to
steady state on the GPU against the printed average Nusselt numbers of the hot wall.

The paper's 250 grid would put tau_v of Eq. 26 at 0.5016 (Ma = 0.1); a 1200 grid at Ma = 0.3 (the
bound the paper states) gives tau_v = 0.5197, as for the Ra = 1e8 rows of tests/test_gpu_table1.py.
Steady state takes tens of millions of steps (the core's stratification develops on the diffusive
time L^2 / (alpha Nu)), several GPU-minutes per row, so these tests carry their own marker and are
not part of ``-m gpu``:

    python -m pytest tests/test_gpu_long_table1.py -m gpu_long
"""
import pytest

from tests.test_gpu_table1 import _table, lbm, steady_nusselt  # noqa: F401  (lbm: the module fixture)

pytestmark = pytest.mark.gpu_long


@pytest.mark.parametrize("phi", [0.4, 0.6, 0.9])
def test_table1_nusselt_ra1e9(lbm, phi):  # noqa: F811
    Da, Ra, grid, Ma = 1e-6, 1e9, 1200, 0.3
    present, ref4, ref7, _ = _table()[(Da, Ra, phi)]
    nu_l, nu_r, steps = steady_nusselt(lbm, grid, Da, Ra, phi, Ma=Ma, chunk=100000, max_steps=24_000_000, tol=1e-5)
    refs = [r for r in (ref4, ref7) if r is not None]
    spread = max(abs(present - r) for r in refs) / present
    print(f"{grid}^2 halfway walls, Ma={Ma}, Da={Da:g} Ra={Ra:g} phi={phi}: Nu_left={nu_l:.4f} Nu_right={nu_r:.4f} after {steps} "
          f"steps; Table 1 present {present} (refs {refs}); rel. diff {abs(nu_l - present) / present:.3%}")
    assert abs(nu_l - present) <= max(0.02, spread) * present
