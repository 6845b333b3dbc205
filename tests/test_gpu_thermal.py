"""Parity of the coupled flow + temperature step (Appendix B, Eqs. B.2-B.7; Sec. 3.4) at the
natural-convection workload's size and tiling, in every storage precision and both streaming forms.

Two kinds of check:

* One step, cell by cell, on a 1100 x 7 lattice with isothermal sides and adiabatic top and
  bottom: a row is longer than one 512-cell work item, so items end inside rows and span row
  ends, as on every lattice wider than 512 cells (e.g. the 2048^2 natural-convection cavity).
* 32 steps (one replay of the 32-step CUDA graph that long runs replay) of the 2048^2
  natural-convection workload (eps = 0.6, Da = 1e-2, Ra = 1e5, Pr = 1, Ma = 0.1, T_h = 21,
  T_c = 1) from a seeded random pre-collision state, on sampled cells: after k steps a cell
  depends only on the cells within k of it (one link per step, Eq. 15 and Eq. B.2), so the FP64
  oracle computes each sampled cell on the (2k+1)^2 crop around it, with the real walls where the
  crop meets them.

With 16-bit storage the random inputs are drawn on the storage's grid (every stored value,
including the anti-bounce-back value parked for an isothermal wall, is exactly representable at the
storage scale), so the library starts from exactly the oracle's state.  One step is then within one
unit of the storage's rounding (one ulp at the stored magnitude) of the FP64 result, element by
element; after k steps within k such units of the largest stored magnitude.
"""
import numpy as np
import pytest

from oracle import mrt_d2q8 as fl
from oracle import thermal_d2q5 as th
from tests.cases import Case, to_gpu

pytestmark = pytest.mark.gpu

K_STEPS = 32
T0, TH, TC = 11.0, 21.0, 1.0
SIG_BITS = {1: 11, 2: 8}  # significant bits of FP16 and BF16
PREC_NAME = {0: "fp32", 1: "fp16", 2: "bf16"}


@pytest.fixture(scope="module")
def lbm():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1311_7239_gb300 import build, lbm

    build.build()
    return lbm


def ulp(v, bits):
    """Spacing of a floating-point format with `bits` significant bits at |v| (normal range)."""
    a = np.maximum(np.abs(np.asarray(v, dtype=np.float64)), 1e-30)
    return np.exp2(np.floor(np.log2(a)) - (bits - 1))


def thermal_state(flow, tp, p_rest, seed, prec):
    """Random pre-collision (f, g) in FP64.  With 16-bit storage (prec 1, 2) the deviations from the
    rest state are multiples of a grid step h with |value| < 2^bits h, so that they and the
    isothermal-wall values -g + 0.4 (T_w - T0) are exact in the storage format at any power-of-two
    scale (no overflow, no subnormals)."""
    rng = np.random.default_rng(seed)
    ny, nx = flow.ny, flow.nx
    p = 1.0 + 0.02 * rng.standard_normal((ny, nx))
    ux, uy = 0.02 * rng.standard_normal((2, ny, nx))
    T = np.clip(T0 + 4.0 * rng.standard_normal((ny, nx)), TC, TH)
    f = fl.equilibrium(p, ux, uy, flow.phi) + 0.002 * rng.standard_normal((8, ny, nx))
    g = th.equilibrium(T, ux, uy, tp) + 0.01 * rng.standard_normal((5, ny, nx))
    rest_f = 3.0 * fl.W[:, None, None] * p_rest
    rest_g = T0 / 5.0
    if prec == 0:
        return f.astype(np.float32).astype(np.float64), g.astype(np.float32).astype(np.float64)
    bits = SIG_BITS[prec]
    # flow deviations |d| < 1/8 on a grid of 2^-(bits+3); temperature |d| < 4 (wall values up to
    # |d| + 4 < 8) on a grid of 8 / 2^bits
    hf = 2.0 ** -(bits + 3)
    hg = 8.0 / 2.0**bits
    df = np.clip(np.round((f - rest_f) / hf), -(2**bits - 1), 2**bits - 1) * hf
    dg = np.clip(np.round((g - rest_g) / hg), -(2**bits - 1) // 2, (2**bits - 1) // 2) * hg
    assert np.abs(df).max() < 0.13 and np.abs(dg).max() + 4.0 < 8.0
    return rest_f + df, rest_g + dg


def _check_close(got, want, rest, prec, tol_fp32, what):
    """Element-wise: FP32 storage within tol_fp32; 16-bit within one unit of the storage's rounding
    at the element's own magnitude (plus 1e-6 for the FP32 arithmetic and the read-out)."""
    dgot, dwant = got - rest, want - rest
    err = np.abs(dgot - dwant)
    if prec == 0:
        bound = np.full_like(err, tol_fp32)
    else:
        bound = ulp(dwant, SIG_BITS[prec]) + 1e-6
    worst = np.unravel_index(np.argmax(err - bound), err.shape)
    assert (err <= bound).all(), (what, worst, float(err[worst]), float(bound[worst]), float(dwant[worst]))
    return float(err.max())


@pytest.mark.parametrize("streaming", [0, 1], ids=["ab", "inplace"])
@pytest.mark.parametrize("prec", [0, 1, 2], ids=["fp32", "fp16", "bf16"])
def test_thermal_one_step_rows_of_three_items(lbm, prec, streaming):
    """One coupled step from a random state on 1100 x 7 (275 four-cell groups per row, work items
    of 128 groups: items end inside rows and span row ends), halfway walls, isothermal sides at 21 and 1, adiabatic
    top and bottom, a buoyancy strong enough to change u by ~1e-3 per step, against the oracle's
    coupled step, element by element."""
    case = Case(1100, 7, nu=0.05, phi=0.6, K=3.0, bc_x="wall", bc_y="wall", precision=prec, streaming=streaming,
                thermal=dict(tau_T=0.8, g_beta=2e-4, T0=T0, T_left=TH, T_right=TC))
    flow, tp = case.flow(), case.thermal_params()
    cfg = case.config(lbm)
    f0, g0 = thermal_state(flow, tp, case.p_rest(), seed=31, prec=prec)
    with lbm.Lattice(cfg) as lat:
        lat.set_populations(to_gpu(f0), to_gpu(g0))
        lat.step(1)
        f1, g1 = [t.cpu().numpy().astype(np.float64) for t in lat.get_populations()]
        lat.sync()
    fo, go = th.coupled_step(f0, g0, flow, tp)
    rest_f = 3.0 * fl.W[:, None, None] * case.p_rest()
    ef = _check_close(f1, fo, rest_f, prec, 4e-6, "f")
    eg = _check_close(g1, go, T0 / 5.0, prec, 4e-5, "g")
    print(f"{PREC_NAME[prec]} {'in-place' if streaming else 'A-B'}: max |df| {ef:.2e}, max |dg| {eg:.2e}")


def _samples(n, n_random, seed):
    pts = [(0, 0), (n - 1, 0), (0, n - 1), (n - 1, n - 1),  # corners
           (0, n // 3), (n - 1, 2 * n // 3), (n // 2, 0), (n // 3, n - 1),  # hot, cold, adiabatic walls
           (1, n - 2), (n - 2, 1), (511, n // 2), (512, n // 2), (1023, 7), (1536, n - 2)]  # item edges
    rng = np.random.default_rng(seed)
    for _ in range(n_random):
        pts.append((int(rng.integers(0, n)), int(rng.integers(0, n))))
    return pts


_ORACLE = {}


def _oracle_samples(cfg, prec, f0, g0):
    """FP64 oracle values of the sampled cells after K_STEPS steps, each on its own crop (cached per
    precision: both streaming forms start from the same state)."""
    if prec in _ORACLE:
        return _ORACLE[prec]
    L = cfg.nx
    tp_kw = dict(tau_T=cfg.tau_T, g_beta=cfg.g_beta, T0=cfg.T0, sigma=cfg.sigma, zeta3=cfg.zeta3, zeta4=cfg.zeta4)
    out = {}
    for (x, y) in _samples(L, 50, seed=11):
        x0, x1 = max(0, x - K_STEPS), min(L - 1, x + K_STEPS)
        y0, y1 = max(0, y - K_STEPS), min(L - 1, y + K_STEPS)
        w, h = x1 - x0 + 1, y1 - y0 + 1
        flow = fl.Flow(nx=w, ny=h, phi=np.full((h, w), cfg.phi), K=np.full((h, w), cfg.K), nu=cfg.nu,
                       forchheimer=bool(cfg.forchheimer), bc_x="wall", bc_y="wall")
        tp = th.Thermal(T_left=TH if x0 == 0 else None, T_right=TC if x1 == L - 1 else None, **tp_kw)
        f = f0[:, y0:y1 + 1, x0:x1 + 1].copy()
        g = g0[:, y0:y1 + 1, x0:x1 + 1].copy()
        for _ in range(K_STEPS):
            f, g = th.coupled_step(f, g, flow, tp)
        out[(x, y)] = (f[:, y - y0, x - x0], g[:, y - y0, x - x0])
    _ORACLE[prec] = out
    return out


@pytest.mark.parametrize("streaming", [0, 1], ids=["ab", "inplace"])
@pytest.mark.parametrize("prec", [0, 1, 2], ids=["fp32", "fp16", "bf16"])
def test_natural_convection_2048_sampled_cells(lbm, prec, streaming):
    """The 2048^2 natural-convection workload, 32 steps through lbm_step from a random state, on 64
    sampled cells (corners, each wall, work-item edges, random interior) against oracle crops.
    Bounds, per step: FP32 16 ulp of the largest flow deviation and of the largest temperature
    value stored (deviation, or the anti-bounce-back value parked at an isothermal wall); FP16 /
    BF16 one unit of the storage's rounding at those magnitudes."""
    import torch

    from paper_1311_7239_gb300 import workloads

    cfg = workloads.natural_convection(lbm, L=2048, precision=prec)
    cfg.streaming = streaming
    L = cfg.nx
    flow = fl.Flow(nx=L, ny=L, phi=np.full((L, L), cfg.phi), K=np.full((L, L), cfg.K), nu=cfg.nu,
                   forchheimer=bool(cfg.forchheimer), bc_x="wall", bc_y="wall")
    tp = th.Thermal(tau_T=cfg.tau_T, g_beta=cfg.g_beta, T0=cfg.T0, T_left=TH, T_right=TC)
    f0, g0 = thermal_state(flow, tp, cfg.p_rest, seed=2048, prec=prec)
    with lbm.Lattice(cfg) as lat:
        lat.set_populations(torch.from_numpy(f0.astype(np.float32)).cuda(), torch.from_numpy(g0.astype(np.float32)).cuda())
        lat.step(K_STEPS)
        f1, g1 = [t.cpu().numpy() for t in lat.get_populations()]
        lat.sync()
    want = _oracle_samples(cfg, prec, f0, g0)
    rest_f = 3.0 * fl.W * cfg.p_rest
    amp_f = float(np.abs(f0 - rest_f[:, None, None]).max())
    amp_g = float(np.abs(g0 - T0 / 5.0).max()) + 0.4 * (TH - T0)  # values parked at the isothermal walls
    bits = SIG_BITS.get(prec, 24)
    units = 16 if prec == 0 else 1  # FP32: the collision's arithmetic; 16-bit: one rounding of the store
    tol_f, tol_g = K_STEPS * units * float(ulp(amp_f, bits)), K_STEPS * units * float(ulp(amp_g, bits))
    worst_f = worst_g = 0.0
    for (x, y), (fw, gw) in want.items():
        ef = float(np.abs((f1[:, y, x] - rest_f) - (fw - rest_f)).max())
        eg = float(np.abs((g1[:, y, x] - T0 / 5.0) - (gw - T0 / 5.0)).max())
        worst_f, worst_g = max(worst_f, ef), max(worst_g, eg)
        assert ef <= tol_f and eg <= tol_g, ((x, y), ef, tol_f, eg, tol_g)
    print(f"2048^2 natural convection {PREC_NAME[prec]} {'in-place' if streaming else 'A-B'}, {K_STEPS} steps: "
          f"max |df| {worst_f:.2e} (bound {tol_f:.1e}), max |dg| {worst_g:.2e} (bound {tol_g:.1e})")
