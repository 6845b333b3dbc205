"""GPU parity of the fused stream-collide path (through the C-ABI) against the FP64 oracle.

Bar (FP32 storage): one step from an arbitrary state matches the oracle element by element to
FP32 rounding (|df| <= 2e-6 absolute on populations of size ~0.1-1), and trajectories of
hundreds to thousands of steps match in relative L2 of u and p to <= 1e-5.
"""
import numpy as np
import pytest

from oracle import mrt_d2q8 as fl
from oracle import thermal_d2q5 as th
from tests.cases import Case, rel_l2, random_state, to_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1311_7239_gb300 import build, lbm

    build.build()
    return lbm


CAV = {"top": (0.1, 0.0)}
ONE_STEP_CASES = {
    "periodic-periodic-uniform": Case(16, 12, bc_x="periodic", bc_y="periodic", ax=2e-4, ay=-1e-4),
    "channel-lid-het": Case(33, 17, bc_x="periodic", bc_y="wall", walls={"top": (0.05, 0.0)}, het=True, ax=1e-4),
    "cavity-moving-walls-het": Case(37, 21, bc_x="wall", bc_y="wall", het=True,
                                    walls={"top": (0.1, 0.0), "bottom": (0.0, 0.01), "left": (0.0, 0.02), "right": (0.0, -0.03)}),
    "cavity-ragged-3-tiles": Case(1100, 6, bc_x="wall", bc_y="wall", walls=CAV, phi=0.7, K=5.0),
    "wall-x-periodic-y": Case(20, 9, bc_x="wall", bc_y="periodic", walls={"left": (0.0, 0.05)}, forch=False),
    "pressure-het": Case(41, 13, bc_x="pressure", bc_y="wall", het=True, p_in=1.01, p_out=0.99),
    "tiny-2x3": Case(2, 3, bc_x="periodic", bc_y="wall", walls=CAV),
    "tiny-3x2-walls": Case(3, 2, bc_x="wall", bc_y="wall", walls=CAV),
    "brinkman-no-forch": Case(64, 8, forch=False, phi=0.1, K=40.96, ax=1e-5),
    # wall nodes with non-equilibrium extrapolation (LBM_NEE)
    "nee-cavity-moving-walls-het": Case(37, 21, bc_x="nee", bc_y="nee", het=True,
                                        walls={"top": (0.1, 0.0), "bottom": (0.0, 0.01), "left": (0.0, 0.02), "right": (0.0, -0.03)}),
    "nee-channel-lid": Case(33, 17, bc_x="periodic", bc_y="nee", walls={"top": (0.05, 0.0)}, ax=1e-4),
    "nee-walls-pressure-het": Case(41, 13, bc_x="pressure", bc_y="nee", het=True, p_in=1.01, p_out=0.99),
    "nee-x-halfway-y": Case(20, 9, bc_x="nee", bc_y="wall", walls={"left": (0.0, 0.05), "top": (0.03, 0.0)}),
    "nee-ragged-3-tiles": Case(1100, 6, bc_x="nee", bc_y="nee", walls=CAV, phi=0.7, K=5.0),
    "nee-tiny-3x3": Case(3, 3, bc_x="nee", bc_y="nee", walls=CAV),
}


@pytest.mark.parametrize("name", list(ONE_STEP_CASES))
def test_one_step_matches_oracle_elementwise(lbm, name):
    case = ONE_STEP_CASES[name]
    flow = case.flow()
    f0 = random_state(flow, seed=11)
    with case.lattice(lbm) as lat:
        lat.set_populations(to_gpu(f0))
        back = lat.get_populations().cpu().numpy()
        # import/export of a pre-collision state is the identity (pressure columns recomputed)
        assert np.abs(back - f0).max() <= 2e-6
        lat.step(1)
        got = lat.get_populations().cpu().numpy()
        lat.sync()
    want = fl.step(f0, flow)
    err = np.abs(got - want).max()
    assert err <= 2e-6, f"{name}: max |df| = {err:.3e}"


def test_init_equilibrium_matches_oracle(lbm):
    for phip in (False, True):
        case = Case(50, 30, bc_x="wall", bc_y="wall", walls=CAV, het=True)
        flow = case.flow()
        p0 = 1.0 / flow.phi if phip else 1.0
        want = fl.initial_state(flow, p0=p0, u0=(0.01, -0.02))
        with case.lattice(lbm) as lat:
            lat.init_equilibrium(1.0, 0.01, -0.02, phi_p_uniform=phip)
            got = lat.get_populations().cpu().numpy()
        assert np.abs(got - want).max() <= 2e-6


def _trajectory(lbm, case, steps, phip_uniform=None):
    """Run both sides from the equilibrium initial state; phip_uniform = c starts from the rest
    state phi p = c (p = c / phi), else from p = 1."""
    flow = case.flow()
    f = fl.initial_state(flow, p0=1.0 if phip_uniform is None else phip_uniform / flow.phi)
    with case.lattice(lbm) as lat:
        if phip_uniform is not None:
            lat.init_equilibrium(phip_uniform, 0.0, 0.0, phi_p_uniform=True)
        lat.step(steps)
        p, ux, uy = [t.cpu().numpy() for t in lat.macros()]
        lat.sync()
    f = fl.run(f, flow, steps)
    uxo, uyo, po = fl.macroscopic(f, flow)
    e_u = rel_l2(np.stack([ux, uy]), np.stack([uxo, uyo]))
    e_p = rel_l2(p, po)
    return e_u, e_p


def test_poiseuille_64_trajectory(lbm, accuracy):
    """Porous Poiseuille channel: 64x64, eps = 0.1, Da = 0.01, nu = 0.1, Re = 10 body force (Sec. 3.1)."""
    H, phi, nu = 64, 0.1, 0.1
    K = 0.01 * H * H
    th_ = np.sqrt(phi / K)
    G = (10 * nu / H) * nu / (K * (1 - 1 / np.cosh(th_ * H / 2)))
    e_u, e_p = _trajectory(lbm, Case(H, H, nu=nu, phi=phi, K=K, forch=False, ax=G), 1500)
    accuracy.append({"case": "porous Poiseuille 64x64, eps 0.1, Da 0.01, Re 10", "precision": "fp32", "steps": 1500,
                     "rel_l2_u": e_u, "rel_l2_p": e_p, "bound": 1e-5})
    assert e_u <= 1e-5 and e_p <= 1e-5, (e_u, e_p)


def test_lid_cavity_trajectory(lbm, accuracy):
    """Lid-driven porous cavity (Sec. 3.3 set-up, halfway walls): eps = 0.4, Da = 1e-3, Re = 100."""
    L = 96
    e_u, e_p = _trajectory(lbm, Case(L, L, nu=0.1 * L / 100, phi=0.4, K=1e-3 * L * L, bc_x="wall", bc_y="wall", walls=CAV), 800)
    accuracy.append({"case": "lid-driven porous cavity 96x96, eps 0.4, Da 1e-3, Re 100", "precision": "fp32", "steps": 800,
                     "rel_l2_u": e_u, "rel_l2_p": e_p, "bound": 1e-5})
    assert e_u <= 1e-5 and e_p <= 1e-5, (e_u, e_p)


def test_heterogeneous_pressure_channel_trajectory(lbm, accuracy):
    case = Case(96, 48, nu=0.1, phi=0.3, K=1e-3 * 48 * 48, het=True, eps_sd=0.03, corr=12.0, bc_x="pressure", bc_y="wall",
                p_in=1.002, p_out=0.998)
    e_u, e_p = _trajectory(lbm, case, 600, phip_uniform=case.p_rest())
    accuracy.append({"case": "heterogeneous pressure-driven channel 96x48", "precision": "fp32", "steps": 600,
                     "rel_l2_u": e_u, "rel_l2_p": e_p, "bound": 1e-5})
    assert e_u <= 1e-5 and e_p <= 1e-5, (e_u, e_p)


def _thermal_case(L=48, prec=0, Ra=1e4):
    nu, tau_v, tau_T, gb = th.parameters_from_Ra(L, Ra, 1.0, 0.1)
    return Case(L, L, nu=nu, phi=0.6, K=1e-2 * L * L, bc_x="wall", bc_y="wall", precision=prec,
                thermal=dict(tau_T=tau_T, g_beta=gb, T0=11.0, T_left=21.0, T_right=1.0))


def test_natural_convection_trajectory_and_nusselt(lbm, accuracy):
    case = _thermal_case()
    flow, tp = case.flow(), case.thermal_params()
    f, g = fl.initial_state(flow), th.initial_state(flow, tp)
    steps = 600
    with case.lattice(lbm) as lat:
        lat.step(steps)
        p, ux, uy, T = [t.cpu().numpy() for t in lat.macros()]
        nu_l, nu_r = lat.nusselt(0), lat.nusselt(1)
    for _ in range(steps):
        f, g = th.coupled_step(f, g, flow, tp)
    uxo, uyo, po, To = th.coupled_macroscopic(f, g, flow, tp)
    e_u, e_T, e_p = rel_l2(np.stack([ux, uy]), np.stack([uxo, uyo])), rel_l2(T, To), rel_l2(p, po)
    accuracy.append({"case": "natural convection 48x48, Ra 1e4, eps 0.6, Da 1e-2", "precision": "fp32", "steps": steps,
                     "rel_l2_u": e_u, "rel_l2_T": e_T, "rel_l2_T_minus_T0": rel_l2(T - 11.0, To - 11.0), "rel_l2_p": e_p,
                     "bound": 1e-5})
    assert e_u <= 1e-5
    assert e_T <= 1e-6
    assert e_p <= 1e-5
    nu_o = th.nusselt_left_wall(To, 21.0, 21.0, 1.0, case.nx)
    assert abs(nu_l - nu_o) <= 1e-5 * abs(nu_o)
    # right wall: mirror of the same formula
    Tm = To[:, ::-1]
    nu_or = th.nusselt_left_wall(Tm, 1.0, 1.0, 21.0, case.nx)
    assert abs(nu_r - nu_or) <= 1e-5 * abs(nu_or)


def test_residual_matches_oracle(lbm):
    case = Case(40, 30, nu=0.05, phi=0.5, K=2.0, bc_x="wall", bc_y="wall", walls=CAV)
    flow = case.flow()
    f = fl.run(fl.initial_state(flow), flow, 59)
    u_prev = fl.macroscopic(f, flow)[:2]
    f = fl.step(f, flow)
    u_now = fl.macroscopic(f, flow)[:2]
    want = fl.residual(u_now[0], u_now[1], u_prev[0], u_prev[1])
    with case.lattice(lbm) as lat:
        lat.step(60)
        got = lat.residual()
    assert abs(got - want) <= 1e-3 * want, (got, want)


def test_errors_are_reported(lbm):
    import torch

    case = Case(16, 8)
    with case.lattice(lbm) as lat:
        with pytest.raises(lbm.LbmError) as e:
            lat.residual()  # no step taken yet
        assert e.value.code == lbm.ESTATE
        bad = torch.zeros(8, 16, dtype=torch.float32, device="cuda")
        with pytest.raises(lbm.LbmError) as e:
            lat.set_medium(bad, None)
        assert e.value.code == lbm.EINVAL
        f = torch.full((8, 8, 16), float("nan"), device="cuda")
        lat.set_populations(f)
        lat.step(2)
        with pytest.raises(lbm.LbmError) as e:
            lat.sync()
        assert e.value.code == lbm.EUNSTABLE


def test_host_pointers_round_trip(lbm):
    """Host (numpy) arrays in and out give the same result as device tensors."""
    case = Case(30, 20, bc_x="wall", bc_y="wall", walls=CAV, het=True)
    flow = case.flow()
    f0 = random_state(flow, seed=3).astype(np.float32)
    with case.lattice(lbm) as lat:
        lat.set_populations(f0)
        lat.step(3)
        out_h = np.empty((8, 20, 30), np.float32)
        lat.get_populations(f=out_h)
        out_d = lat.get_populations().cpu().numpy()
        p_h, ux_h, uy_h = (np.empty((20, 30), np.float32) for _ in range(3))
        lat.macros(p_h, ux_h, uy_h)
        p_d, ux_d, uy_d = (t.cpu().numpy() for t in lat.macros())
    assert np.array_equal(out_h, out_d)
    assert np.array_equal(ux_h, ux_d) and np.array_equal(p_h, p_d)


# BF16 keeps 8 significant bits: its measured errors against the FP64 oracle (6.6e-3 on the 96^2
# cavity, 1.0e-2 on 600 x 64, a few percent on the thermal transient) miss the 1e-3 that FP16 meets.
# The BF16 runs below are therefore not parity passes: they record the error with the 1e-3 target
# and meets_target = false, and assert only a regression bound (about 1.5x the measured error).
BF16_TARGET = 1e-3


def _cavity_storage_error(lbm, prec):
    L = 96
    case = Case(L, L, nu=0.1 * L / 100, phi=0.4, K=1e-3 * L * L, bc_x="wall", bc_y="wall", walls=CAV, precision=prec)
    return _trajectory(lbm, case, 800)


def test_reduced_precision_storage_error(lbm, accuracy):
    """FP16 storage of f - f_rest with FP32 arithmetic: relative L2 error of u and p vs the FP64
    oracle on the lid-driven cavity, within the 1e-3 target."""
    e_u, e_p = _cavity_storage_error(lbm, 1)
    print(f"fp16: rel-L2 u {e_u:.3e}, p {e_p:.3e}")
    accuracy.append({"case": "lid-driven porous cavity 96x96, eps 0.4, Da 1e-3, Re 100", "precision": "fp16",
                     "steps": 800, "rel_l2_u": e_u, "rel_l2_p": e_p, "bound": 1e-3})
    assert e_u <= 1e-3 and e_p <= 1e-3, (e_u, e_p)


def test_bf16_storage_error_bounded_target_missed(lbm, accuracy):
    """BF16 storage on the same cavity: not a parity pass (see BF16_TARGET); regression bound 1e-2."""
    e_u, e_p = _cavity_storage_error(lbm, 2)
    print(f"bf16: rel-L2 u {e_u:.3e}, p {e_p:.3e} (target {BF16_TARGET:g} not met)")
    accuracy.append({"case": "lid-driven porous cavity 96x96, eps 0.4, Da 1e-3, Re 100", "precision": "bf16",
                     "steps": 800, "rel_l2_u": e_u, "rel_l2_p": e_p, "target": BF16_TARGET, "regression_bound": 1e-2})
    assert e_u <= 1e-2 and e_p <= 1e-2, (e_u, e_p)


def _long_rows_error(lbm, prec):
    case = Case(600, 64, nu=0.1 * 64 / 100, phi=0.4, K=1e-3 * 64 * 64, bc_x="wall", bc_y="wall", walls=CAV, precision=prec)
    return _trajectory(lbm, case, 400)


def test_reduced_precision_long_rows(lbm, accuracy):
    """FP16 storage with rows longer than one work item: a 600 x 64 lid-driven cavity (two 512-cell
    items per row, the second ragged) against the oracle, within the 1e-3 target."""
    e_u, e_p = _long_rows_error(lbm, 1)
    print(f"fp16, 600x64: rel-L2 u {e_u:.3e}, p {e_p:.3e}")
    accuracy.append({"case": "lid-driven porous cavity 600x64, eps 0.4, Da 1e-3", "precision": "fp16",
                     "steps": 400, "rel_l2_u": e_u, "rel_l2_p": e_p, "bound": 1e-3})
    assert e_u <= 1e-3 and e_p <= 1e-3, (e_u, e_p)


def test_bf16_long_rows_error_bounded_target_missed(lbm, accuracy):
    """BF16 on the 600 x 64 cavity (1.0e-2 at 600 x 64, 9.6e-3 at 500 x 64): not a parity pass;
    regression bound 2e-2."""
    e_u, e_p = _long_rows_error(lbm, 2)
    print(f"bf16, 600x64: rel-L2 u {e_u:.3e}, p {e_p:.3e} (target {BF16_TARGET:g} not met)")
    accuracy.append({"case": "lid-driven porous cavity 600x64, eps 0.4, Da 1e-3", "precision": "bf16",
                     "steps": 400, "rel_l2_u": e_u, "rel_l2_p": e_p, "target": BF16_TARGET, "regression_bound": 2e-2})
    assert e_u <= 2e-2 and e_p <= 2e-2, (e_u, e_p)


@pytest.mark.parametrize("bc", ["periodic", "nee"])
@pytest.mark.parametrize("prec", [1, 2])
def test_reduced_precision_one_step_long_rows(lbm, prec, bc):
    """One step with 16-bit storage from a random state against the oracle, cell by cell, on a
    periodic 1100 x 7 channel with a moving top wall (three items per row, ragged), to the
    storage's rounding, twice (the imported state and the result): FP16 2^-11 of |d| <= 0.1 at
    scale 2^10, BF16 2^-8."""
    case = Case(1100, 7, bc_x=bc, bc_y="wall" if bc == "periodic" else "nee", walls={"top": (0.05, 0.0)}, ax=1e-4, precision=prec)
    flow = case.flow()
    f0 = random_state(flow, seed=3)
    with case.lattice(lbm) as lat:
        lat.set_populations(to_gpu(f0))
        lat.step(1)
        got = lat.get_populations().cpu().numpy()
        lat.sync()
    want = fl.step(f0, flow)  # the bound covers the rounding of the imported state and of the result
    tol = 1e-4 if prec == 1 else 8e-4
    assert np.abs(got - want).max() <= tol, np.abs(got - want).max()


def _thermal_storage_error(lbm, prec):
    case = _thermal_case(prec=prec)
    flow, tp = case.flow(), case.thermal_params()
    f, g = fl.initial_state(flow), th.initial_state(flow, tp)
    steps = 600
    with case.lattice(lbm) as lat:
        lat.step(steps)
        p, ux, uy, T = [t.cpu().numpy() for t in lat.macros()]
    for _ in range(steps):
        f, g = th.coupled_step(f, g, flow, tp)
    uxo, uyo, po, To = th.coupled_macroscopic(f, g, flow, tp)
    return steps, rel_l2(np.stack([ux, uy]), np.stack([uxo, uyo])), rel_l2(T - 11.0, To - 11.0)


def test_reduced_precision_thermal_error(lbm, accuracy):
    """Natural convection with FP16 storage, within the 1e-3 target for u and T - T0."""
    steps, e_u, e_T = _thermal_storage_error(lbm, 1)
    print(f"fp16: rel-L2 u {e_u:.3e}, T-T0 {e_T:.3e}")
    accuracy.append({"case": "natural convection 48x48, Ra 1e4, eps 0.6, Da 1e-2", "precision": "fp16",
                     "steps": steps, "rel_l2_u": e_u, "rel_l2_T_minus_T0": e_T, "bound": 1e-3})
    assert e_u <= 1e-3 and e_T <= 1e-3, (e_u, e_T)


def test_bf16_thermal_error_bounded_target_missed(lbm, accuracy):
    """Natural convection with BF16 storage: the 8-bit significand's rounding (2^-9 per stored
    value) accumulates over the slow thermal transient to a few percent; not a parity pass,
    regression bound 6e-2."""
    steps, e_u, e_T = _thermal_storage_error(lbm, 2)
    print(f"bf16: rel-L2 u {e_u:.3e}, T-T0 {e_T:.3e} (target {BF16_TARGET:g} not met)")
    accuracy.append({"case": "natural convection 48x48, Ra 1e4, eps 0.6, Da 1e-2", "precision": "bf16",
                     "steps": steps, "rel_l2_u": e_u, "rel_l2_T_minus_T0": e_T, "target": BF16_TARGET,
                     "regression_bound": 6e-2})
    assert e_u <= 6e-2 and e_T <= 6e-2, (e_u, e_T)


def test_graph_replay_equals_single_launches(lbm):
    """lbm_step(n) replays a captured graph of 32 steps; the result is bitwise that of n single steps."""
    case = Case(150, 70, nu=0.05, phi=0.5, K=3.0, bc_x="wall", bc_y="wall", walls=CAV, het=True)
    with case.lattice(lbm) as a, case.lattice(lbm) as b:
        a.step(101)   # three graph replays + 5 launches
        for _ in range(101):
            b.step(1)
        fa = a.get_populations().cpu().numpy()
        fb = b.get_populations().cpu().numpy()
        a.step(64)   # a graph starting from the other buffer
        b.step(64)
        ga = a.get_populations().cpu().numpy()
        gb = b.get_populations().cpu().numpy()
        assert a.step_count() == b.step_count() == 165
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)


def _jcase(nx, ny, J_lo, het_phi=True):
    """Partially porous channel with the viscosity ratio J_lo in the lower (porous) half."""
    lower = np.arange(ny)[:, None] < ny // 2
    case = Case(nx, ny, nu=0.16, phi=0.5, K=1e-3 * ny * ny, forch=False, walls={"top": (0.01, 0.0)}, het=het_phi)
    Jf = (np.where(lower, J_lo, 1.0) * np.ones((ny, nx))).astype(np.float32)
    return case, Jf


def test_viscosity_ratio_field_one_step_and_trajectory(lbm):
    """Per-cell J (region-dependent s_v of Sec. 3.2): one step from a random state element by
    element, and a 400-step trajectory, against the oracle with the same J field."""
    import torch

    case, Jf = _jcase(37, 22, 4.0)
    flow = case.flow()
    flow.J = Jf.astype(np.float64)
    f0 = random_state(flow, seed=5)
    with case.lattice(lbm) as lat:
        lat.set_viscosity_ratio(torch.tensor(Jf, device="cuda"))
        lat.set_populations(to_gpu(f0))
        lat.step(1)
        got = lat.get_populations().cpu().numpy()
    assert np.abs(got - fl.step(f0, flow)).max() <= 2e-6
    with case.lattice(lbm) as lat:
        lat.set_viscosity_ratio(Jf)  # host array
        lat.init_equilibrium(case.p_rest(), 0.0, 0.0, phi_p_uniform=True)
        lat.step(400)
        p, ux, uy = (t.cpu().numpy() for t in lat.macros())
        with pytest.raises(lbm.LbmError) as e:
            lat.set_viscosity_ratio(np.zeros_like(Jf))
        assert e.value.code == lbm.EINVAL
    f = fl.run(fl.initial_state(flow, p0=case.p_rest() / flow.phi), flow, 400)
    uxo, uyo, po = fl.macroscopic(f, flow)
    assert rel_l2(np.stack([ux, uy]), np.stack([uxo, uyo])) <= 1e-5
    assert rel_l2(p, po) <= 1e-5


def test_nee_lid_cavity_trajectory(lbm, accuracy):
    """The paper's lid-driven porous cavity (Sec. 3.3: eps = 0.1, Re = 10, nu = 0.256 on 128 x 128,
    Da = 1e-2) with its own wall treatment, extrapolated wall nodes on the four sides (H = 127)."""
    L, nu = 128, 0.256
    u0 = 10 * nu / (L - 1)
    case = Case(L, L, nu=nu, phi=0.1, K=1e-2 * (L - 1) ** 2, bc_x="nee", bc_y="nee", walls={"top": (u0, 0.0)})
    e_u, e_p = _trajectory(lbm, case, 600)
    accuracy.append({"case": "lid-driven porous cavity 128x128 with extrapolated wall nodes, eps 0.1, Da 1e-2, Re 10",
                     "precision": "fp32", "steps": 600, "rel_l2_u": e_u, "rel_l2_p": e_p, "bound": 1e-5})
    assert e_u <= 1e-5 and e_p <= 1e-5, (e_u, e_p)


def test_nee_poiseuille_steady_state_matches_eq24(lbm):
    """Porous Poiseuille between wall nodes (H = ny - 1) run to steady state on the GPU against the
    profile behind Eq. 24 (second-order scheme: 1.5e-3 at ny = 65 in the oracle)."""
    N, phi, nu = 65, 0.1, 0.3
    H = N - 1
    K = 0.01 * H * H
    th_ = np.sqrt(phi / K)
    u0 = nu / H
    G = u0 * nu / (K * (1 - 1 / np.cosh(th_ * H / 2)))
    cfg = lbm.default_config(nx=8, ny=N, bc_x=lbm.PERIODIC, bc_y=lbm.NEE, nu=nu, phi=phi, K=K, forchheimer=0, ax=G, p_rest=phi)
    lat = lbm.Lattice(cfg)
    try:
        for _ in range(400):
            lat.step(100)
            if lat.residual() < 1e-11:
                break
        ux = lat.macros()[1].cpu().numpy()[:, 0].astype(np.float64)
    finally:
        lat.close()
    y = np.arange(N, dtype=np.float64)
    exact = G * K / nu * (1 - np.cosh(th_ * (y - H / 2)) / np.cosh(th_ * H / 2))
    err = np.abs(ux - exact).max() / exact.max()
    assert err < 2e-3, err


def test_nee_rejections(lbm):
    with pytest.raises(lbm.LbmError) as e:
        lbm.Lattice(lbm.default_config(nx=8, ny=2, bc_y=lbm.NEE))
    assert e.value.code == lbm.EINVAL
    # three nodes across: a valid lattice, but both walls extrapolate from the same middle row, which
    # the adjoint does not take
    lat = lbm.Lattice(lbm.default_config(nx=8, ny=3, bc_y=lbm.NEE))
    try:
        lat.init_equilibrium(1.0, 0.0, 0.0)
        with pytest.raises(lbm.LbmError) as e:
            lat.adjoint(4, "flux")
        assert e.value.code == lbm.EINVAL
    finally:
        lat.close()


def _thermal_nee_case(L=48, prec=0, Ra=1e4):
    nu, tau_v, tau_T, gb = th.parameters_from_Ra(L - 1, Ra, 1.0, 0.1)
    return Case(L, L, nu=nu, phi=0.6, K=1e-2 * (L - 1) ** 2, bc_x="nee", bc_y="nee", precision=prec,
                thermal=dict(tau_T=tau_T, g_beta=gb, T0=11.0, T_left=21.0, T_right=1.0))


@pytest.mark.parametrize("prec,bound", [(0, 1e-5), (1, 1e-3)])
def test_natural_convection_wall_nodes_trajectory_and_nusselt(lbm, accuracy, prec, bound):
    """Natural convection with the paper's wall treatment for both equations (extrapolated wall
    nodes, isothermal sides, adiabatic top and bottom) against the coupled oracle step, and the
    wall-node Nusselt numbers of both sides."""
    case = _thermal_nee_case(prec=prec)
    flow, tp = case.flow(), case.thermal_params()
    f = fl.initial_state(flow)
    g = th.initial_state(flow, tp, f=f)
    steps = 600
    with case.lattice(lbm) as lat:
        lat.step(steps)
        p, ux, uy, T = [t.cpu().numpy() for t in lat.macros()]
        nu_l, nu_r = lat.nusselt(0), lat.nusselt(1)
    for _ in range(steps):
        f, g = th.coupled_step(f, g, flow, tp)
    uxo, uyo, po, To = th.coupled_macroscopic(f, g, flow, tp)
    e_u = rel_l2(np.stack([ux, uy]), np.stack([uxo, uyo]))
    e_T = rel_l2(T - 11.0, To - 11.0)
    accuracy.append({"case": "natural convection 48x48 with extrapolated wall nodes, Ra 1e4, eps 0.6, Da 1e-2",
                     "precision": {0: "fp32", 1: "fp16"}[prec], "steps": steps, "rel_l2_u": e_u, "rel_l2_T_minus_T0": e_T,
                     "bound": bound})
    assert e_u <= bound and e_T <= bound, (e_u, e_T)
    nl, nr = th.nusselt_wall_nodes(To, 0, 21.0, 1.0), th.nusselt_wall_nodes(To, 1, 21.0, 1.0)
    assert abs(nu_l - nl) <= 20 * bound * abs(nl) and abs(nu_r - nr) <= 20 * bound * abs(nr), (nu_l, nl, nu_r, nr)


@pytest.mark.parametrize("bc", ["wall", "nee"])
def test_thermal_one_step_matches_oracle_elementwise(lbm, bc):
    """One coupled step (flow + temperature, buoyancy) from a random state, cell by cell, with
    halfway walls or extrapolated wall nodes on all sides (isothermal sides, adiabatic top and
    bottom, moving lid)."""
    case = Case(23, 17, nu=0.05, phi=0.6, K=3.0, bc_x=bc, bc_y=bc, walls={"top": (0.04, 0.0)},
                thermal=dict(tau_T=0.8, g_beta=2e-4, T0=11.0, T_left=21.0, T_right=1.0))
    flow, tp = case.flow(), case.thermal_params()
    rng = np.random.default_rng(21)
    f0 = random_state(flow, seed=9)
    T = 11.0 + 5.0 * rng.standard_normal((flow.ny, flow.nx))
    g0 = th.equilibrium(T, *(0.03 * rng.standard_normal((2, flow.ny, flow.nx))), tp) + 0.01 * rng.standard_normal((5, flow.ny, flow.nx))
    if bc == "nee":
        f0, g0 = th.boundary_nodes(f0, g0, flow, tp)
    f0 = f0.astype(np.float32).astype(np.float64)
    g0 = g0.astype(np.float32).astype(np.float64)
    with case.lattice(lbm) as lat:
        lat.set_populations(to_gpu(f0), to_gpu(g0))
        lat.step(1)
        f1, g1 = [t.cpu().numpy() for t in lat.get_populations()]
        lat.sync()
    fo, go = th.coupled_step(f0, g0, flow, tp)
    ef, eg = np.abs(f1 - fo), np.abs(g1 - go)
    assert ef.max() <= 4e-6, (ef.max(), np.unravel_index(ef.argmax(), ef.shape))
    assert eg.max() <= 4e-5, (eg.max(), np.unravel_index(eg.argmax(), eg.shape))
