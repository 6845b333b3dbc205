"""In-place streaming (LBM_STREAM_INPLACE: one population buffer) through the C-ABI.

The in-place step computes what the A-B step computes (Eq. 15 followed by Eq. 14, and Eq. B.2 for
the temperature); only where the populations are kept changes.  So the bars are those of the A-B
form: one step from an arbitrary state matches the FP64 oracle cell by cell to FP32 rounding,
trajectories match in relative L2 to 1e-5 (FP32) and 1e-3 (FP16), and read-outs, residual,
checkpoints and the Nusselt number work on the in-place layout.  The steps alternate between two
layouts, so every multi-step check covers both parities.
"""
import dataclasses
import os
import tempfile

import numpy as np
import pytest

from oracle import mrt_d2q8 as fl
from oracle import thermal_d2q5 as th
from tests.cases import Case, rel_l2, random_state, to_gpu

pytestmark = pytest.mark.gpu

IP = 1
CAV = {"top": (0.1, 0.0)}


@pytest.fixture(scope="module")
def lbm():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1311_7239_gb300 import build, lbm

    build.build()
    return lbm


MULTI_STEP_CASES = {
    "periodic-periodic-uniform": Case(16, 12, bc_x="periodic", bc_y="periodic", ax=2e-4, ay=-1e-4, streaming=IP),
    "channel-lid-het": Case(33, 17, bc_x="periodic", bc_y="wall", walls={"top": (0.05, 0.0)}, het=True, ax=1e-4, streaming=IP),
    "cavity-moving-walls-het": Case(37, 21, bc_x="wall", bc_y="wall", het=True, streaming=IP,
                                    walls={"top": (0.1, 0.0), "bottom": (0.0, 0.01), "left": (0.0, 0.02), "right": (0.0, -0.03)}),
    "cavity-ragged-3-blocks": Case(1100, 6, bc_x="wall", bc_y="wall", walls=CAV, phi=0.7, K=5.0, streaming=IP),
    "wall-x-periodic-y": Case(20, 9, bc_x="wall", bc_y="periodic", walls={"left": (0.0, 0.05)}, forch=False, streaming=IP),
    "periodic-x-ragged": Case(131, 5, bc_x="periodic", bc_y="wall", walls=CAV, ax=1e-4, streaming=IP),
    "tiny-2x3": Case(2, 3, bc_x="periodic", bc_y="wall", walls=CAV, streaming=IP),
    "tiny-3x2-walls": Case(3, 2, bc_x="wall", bc_y="wall", walls=CAV, streaming=IP),
    "tiny-5x2-periodic": Case(5, 2, bc_x="periodic", bc_y="periodic", ax=1e-4, streaming=IP),
    # extrapolated sides: pressure columns and wall nodes (their states are computed before the step)
    "pressure-het": Case(41, 13, bc_x="pressure", bc_y="wall", het=True, p_in=1.01, p_out=0.99, streaming=IP),
    "nee-cavity-moving-walls-het": Case(37, 21, bc_x="nee", bc_y="nee", het=True, streaming=IP,
                                        walls={"top": (0.1, 0.0), "bottom": (0.0, 0.01), "left": (0.0, 0.02), "right": (0.0, -0.03)}),
    "nee-channel-lid": Case(33, 17, bc_x="periodic", bc_y="nee", walls={"top": (0.05, 0.0)}, ax=1e-4, streaming=IP),
    "nee-walls-pressure-het": Case(41, 13, bc_x="pressure", bc_y="nee", het=True, p_in=1.01, p_out=0.99, streaming=IP),
    "nee-x-halfway-y": Case(20, 9, bc_x="nee", bc_y="wall", walls={"left": (0.0, 0.05), "top": (0.03, 0.0)}, streaming=IP),
    "nee-x-periodic-y": Case(20, 9, bc_x="nee", bc_y="periodic", walls={"right": (0.0, -0.04)}, ay=1e-4, streaming=IP),
    "nee-ragged-3-blocks": Case(1100, 6, bc_x="nee", bc_y="nee", walls=CAV, phi=0.7, K=5.0, streaming=IP),
    "nee-tiny-3x3": Case(3, 3, bc_x="nee", bc_y="nee", walls=CAV, streaming=IP),
    "pressure-tiny-3x2": Case(3, 2, bc_x="pressure", bc_y="periodic", p_in=1.01, p_out=0.99, streaming=IP),
}


@pytest.mark.parametrize("name", list(MULTI_STEP_CASES))
def test_steps_match_oracle_elementwise(lbm, name):
    """Import of a random pre-collision state, then three single steps (parities 0, 1, 0), each
    against the oracle cell by cell."""
    case = MULTI_STEP_CASES[name]
    flow = case.flow()
    f = random_state(flow, seed=11)
    with case.lattice(lbm) as lat:
        lat.set_populations(to_gpu(f))
        back = lat.get_populations().cpu().numpy()
        assert np.abs(back - f).max() <= 2e-6  # import/export is the identity on the in-place layout
        for k in range(3):
            lat.step(1)
            got = lat.get_populations().cpu().numpy()
            f = fl.step(f, flow)
            err = np.abs(got - f).max()
            assert err <= 2e-6 * (k + 1), f"{name}, step {k + 1}: max |df| = {err:.3e}"
        lat.sync()


def test_init_equilibrium_matches_oracle(lbm):
    for phip in (False, True):
        case = Case(50, 30, bc_x="wall", bc_y="wall", walls=CAV, het=True, streaming=IP)
        flow = case.flow()
        p0 = 1.0 / flow.phi if phip else 1.0
        want = fl.initial_state(flow, p0=p0, u0=(0.01, -0.02))
        with case.lattice(lbm) as lat:
            lat.init_equilibrium(1.0, 0.01, -0.02, phi_p_uniform=phip)
            got = lat.get_populations().cpu().numpy()
        assert np.abs(got - want).max() <= 2e-6


def _trajectory(lbm, case, steps):
    flow = case.flow()
    f = fl.initial_state(flow)
    with case.lattice(lbm) as lat:
        lat.init_equilibrium(1.0, 0.0, 0.0)  # after the medium: p = 1 with the per-cell porosity
        lat.step(steps)
        p, ux, uy = [t.cpu().numpy() for t in lat.macros()]
        lat.sync()
    f = fl.run(f, flow, steps)
    uxo, uyo, po = fl.macroscopic(f, flow)
    return rel_l2(np.stack([ux, uy]), np.stack([uxo, uyo])), rel_l2(p, po)


def test_lid_cavity_trajectory(lbm, accuracy):
    L = 96
    case = Case(L, L, nu=0.1 * L / 100, phi=0.4, K=1e-3 * L * L, bc_x="wall", bc_y="wall", walls=CAV, streaming=IP)
    e_u, e_p = _trajectory(lbm, case, 800)
    accuracy.append({"case": "lid-driven porous cavity 96x96, eps 0.4, Da 1e-3, Re 100, in-place streaming", "precision": "fp32",
                     "steps": 800, "rel_l2_u": e_u, "rel_l2_p": e_p, "bound": 1e-5})
    assert e_u <= 1e-5 and e_p <= 1e-5, (e_u, e_p)


def test_heterogeneous_channel_trajectory(lbm, accuracy):
    case = Case(96, 48, nu=0.1, phi=0.3, K=1e-3 * 48 * 48, het=True, eps_sd=0.03, corr=12.0, bc_x="periodic", bc_y="wall",
                ax=2e-6, walls={"top": (0.02, 0.0)}, streaming=IP)
    e_u, e_p = _trajectory(lbm, case, 600)
    accuracy.append({"case": "heterogeneous body-forced channel 96x48 with a moving wall, in-place streaming", "precision": "fp32",
                     "steps": 600, "rel_l2_u": e_u, "rel_l2_p": e_p, "bound": 1e-5})
    assert e_u <= 1e-5 and e_p <= 1e-5, (e_u, e_p)


def _reduced_precision_cavity(lbm, prec):
    L = 96
    case = Case(L, L, nu=0.1 * L / 100, phi=0.4, K=1e-3 * L * L, bc_x="wall", bc_y="wall", walls=CAV, precision=prec, streaming=IP)
    return _trajectory(lbm, case, 800)


@pytest.mark.parametrize("prec,bound", [(0, 1e-5), (1, 1e-3)])
def test_nee_cavity_and_pressure_channel_trajectories(lbm, accuracy, prec, bound):
    """In-place streaming with extrapolated sides over many steps (both parities, graph replays):
    the lid-driven cavity with wall nodes on all sides and the pressure-driven heterogeneous
    channel with wall nodes above and below, against the oracle's trajectories."""
    L = 64
    cav = Case(L, L, nu=0.1 * L / 100, phi=0.4, K=1e-3 * L * L, bc_x="nee", bc_y="nee", walls=CAV, precision=prec, streaming=IP)
    ch = Case(96, 48, nu=0.1, phi=0.35, K=1e-3 * 48 * 48, het=True, eps_sd=0.03, corr=12.0, bc_x="pressure", bc_y="nee",
              p_in=1.002, p_out=0.998, precision=prec, streaming=IP)
    name = {0: "fp32", 1: "fp16"}[prec]
    for label, case, steps in (("lid-driven porous cavity 64x64 with extrapolated wall nodes, in-place streaming", cav, 500),
                               ("pressure-driven heterogeneous channel 96x48 with extrapolated wall nodes, in-place streaming", ch, 400)):
        e_u, e_p = _trajectory(lbm, case, steps)
        accuracy.append({"case": label, "precision": name, "steps": steps, "rel_l2_u": e_u, "rel_l2_p": e_p, "bound": bound})
        assert e_u <= bound and e_p <= bound, (label, e_u, e_p)


def test_reduced_precision_cavity(lbm, accuracy):
    """FP16 storage with in-place streaming, within the 1e-3 target."""
    e_u, e_p = _reduced_precision_cavity(lbm, 1)
    accuracy.append({"case": "lid-driven porous cavity 96x96, eps 0.4, Da 1e-3, Re 100, in-place streaming",
                     "precision": "fp16", "steps": 800, "rel_l2_u": e_u, "rel_l2_p": e_p, "bound": 1e-3})
    assert e_u <= 1e-3 and e_p <= 1e-3, (e_u, e_p)


def test_bf16_cavity_error_bounded_target_missed(lbm, accuracy):
    """BF16 storage with in-place streaming: its 8-bit significand misses the 1e-3 target (about
    6e-3 here, as with A-B streaming); not a parity pass, regression bound 1e-2."""
    e_u, e_p = _reduced_precision_cavity(lbm, 2)
    accuracy.append({"case": "lid-driven porous cavity 96x96, eps 0.4, Da 1e-3, Re 100, in-place streaming",
                     "precision": "bf16", "steps": 800, "rel_l2_u": e_u, "rel_l2_p": e_p, "target": 1e-3,
                     "regression_bound": 1e-2})
    assert e_u <= 1e-2 and e_p <= 1e-2, (e_u, e_p)


def _thermal_case(prec=0, L=48, Ra=1e4):
    nu, tau_v, tau_T, gb = th.parameters_from_Ra(L, Ra, 1.0, 0.1)
    return Case(L, L, nu=nu, phi=0.6, K=1e-2 * L * L, bc_x="wall", bc_y="wall", precision=prec, streaming=IP,
                thermal=dict(tau_T=tau_T, g_beta=gb, T0=11.0, T_left=21.0, T_right=1.0))


@pytest.mark.parametrize("prec,bound", [(0, 1e-5), (1, 1e-3)])
def test_natural_convection_trajectory_and_nusselt(lbm, accuracy, prec, bound):
    case = _thermal_case(prec)
    flow, tp = case.flow(), case.thermal_params()
    f, g = fl.initial_state(flow), th.initial_state(flow, tp)
    steps = 600
    with case.lattice(lbm) as lat:
        lat.step(steps)
        p, ux, uy, T = [t.cpu().numpy() for t in lat.macros()]
        nu_l = lat.nusselt(0)
    for _ in range(steps):
        f, g = th.coupled_step(f, g, flow, tp)
    uxo, uyo, po, To = th.coupled_macroscopic(f, g, flow, tp)
    e_u, e_T = rel_l2(np.stack([ux, uy]), np.stack([uxo, uyo])), rel_l2(T - 11.0, To - 11.0)
    accuracy.append({"case": "natural convection 48x48, Ra 1e4, eps 0.6, Da 1e-2, in-place streaming",
                     "precision": {0: "fp32", 1: "fp16"}[prec], "steps": steps, "rel_l2_u": e_u, "rel_l2_T_minus_T0": e_T,
                     "bound": bound})
    assert e_u <= bound and e_T <= bound, (e_u, e_T)
    nu_o = th.nusselt_left_wall(To, 21.0, 21.0, 1.0, case.nx)
    assert abs(nu_l - nu_o) <= 10 * bound * abs(nu_o), (nu_l, nu_o)


@pytest.mark.parametrize("bc", ["wall", "nee"])
def test_thermal_one_step_matches_oracle_elementwise(lbm, bc):
    """One and two coupled steps from a random state with isothermal and adiabatic walls (halfway,
    or extrapolated wall nodes) and a moving lid (the anti-bounce-back slots of both parities)."""
    case = Case(23, 17, nu=0.05, phi=0.6, K=3.0, bc_x=bc, bc_y=bc, walls={"top": (0.04, 0.0)}, streaming=IP,
                thermal=dict(tau_T=0.8, g_beta=2e-4, T0=11.0, T_left=21.0, T_right=1.0))
    flow, tp = case.flow(), case.thermal_params()
    rng = np.random.default_rng(21)
    f = random_state(flow, seed=9)
    T = 11.0 + 5.0 * rng.standard_normal((flow.ny, flow.nx))
    g = th.equilibrium(T, *(0.03 * rng.standard_normal((2, flow.ny, flow.nx))), tp) + 0.01 * rng.standard_normal((5, flow.ny, flow.nx))
    if bc == "nee":
        f, g = th.boundary_nodes(f, g, flow, tp)
    f = f.astype(np.float32).astype(np.float64)
    g = g.astype(np.float32).astype(np.float64)
    with case.lattice(lbm) as lat:
        lat.set_populations(to_gpu(f), to_gpu(g))
        for k in range(2):
            lat.step(1)
            f1, g1 = [t.cpu().numpy() for t in lat.get_populations()]
            f, g = th.coupled_step(f, g, flow, tp)
            assert np.abs(f1 - f).max() <= 4e-6 * (k + 1), np.abs(f1 - f).max()
            assert np.abs(g1 - g).max() <= 4e-5 * (k + 1), np.abs(g1 - g).max()
        lat.sync()


SIDES = {
    "halfway-walls": dict(bc_x="wall", bc_y="wall", walls=CAV),
    "nee-walls": dict(bc_x="nee", bc_y="nee", walls={"top": (0.1, 0.0), "left": (0.0, 0.02)}),
    "pressure-nee": dict(bc_x="pressure", bc_y="nee", p_in=1.002, p_out=0.998),
    "pressure-halfway": dict(bc_x="pressure", bc_y="wall", p_in=1.002, p_out=0.998, walls=CAV),
}


@pytest.mark.parametrize("sides", list(SIDES))
def test_same_result_as_ab_streaming(lbm, sides):
    """In-place and A-B forms of the same run (FP32, per-cell medium, moving walls, 101 steps: three
    graph replays and five single steps) agree to FP32 rounding; the probe and the residual too."""
    case = Case(150, 70, nu=0.05, phi=0.5, K=3.0, het=True, **SIDES[sides])
    with case.lattice(lbm) as a, dataclasses.replace(case, streaming=IP).lattice(lbm) as b:
        a.step(101)
        b.step(101)
        fa, fb = a.get_populations().cpu().numpy(), b.get_populations().cpu().numpy()
        ra, rb = a.residual(), b.residual()
        pa, pb = a.probe(75, 69), b.probe(75, 69)
    assert rel_l2(fb, fa) <= 1e-6, rel_l2(fb, fa)
    assert abs(ra - rb) <= 1e-3 * abs(ra), (ra, rb)  # u(t-1): the collision's sums vs the read-out's (rounding order)
    assert np.allclose(np.asarray(pa), np.asarray(pb), rtol=1e-5, atol=1e-7)
    print("in-place vs A-B after 101 steps: max |df| =", float(np.abs(fb - fa).max()), "bitwise:", bool(np.array_equal(fa, fb)))


def test_residual_matches_oracle(lbm):
    case = Case(40, 30, nu=0.05, phi=0.5, K=2.0, bc_x="wall", bc_y="wall", walls=CAV, streaming=IP)
    flow = case.flow()
    f = fl.run(fl.initial_state(flow), flow, 59)
    u_prev = fl.macroscopic(f, flow)[:2]
    f = fl.step(f, flow)
    u_now = fl.macroscopic(f, flow)[:2]
    want = fl.residual(u_now[0], u_now[1], u_prev[0], u_prev[1])
    with case.lattice(lbm) as lat:
        lat.step(20)
        lat.step(40)  # the last step of each call records the u(t-1) of the residual
        got = lat.residual()
    assert abs(got - want) <= 1e-3 * want, (got, want)


def test_graph_replay_equals_single_launches(lbm):
    case = Case(150, 70, nu=0.05, phi=0.5, K=3.0, bc_x="wall", bc_y="wall", walls=CAV, het=True, streaming=IP)
    with case.lattice(lbm) as a, case.lattice(lbm) as b:
        a.step(101)
        for _ in range(101):
            b.step(1)
        assert np.array_equal(a.get_populations().cpu().numpy(), b.get_populations().cpu().numpy())
        a.step(64)  # a graph starting from the other parity
        b.step(64)
        assert np.array_equal(a.get_populations().cpu().numpy(), b.get_populations().cpu().numpy())


def test_save_load_continues_bitwise(lbm):
    case = Case(70, 40, nu=0.05, phi=0.5, K=3.0, bc_x="wall", bc_y="wall", walls=CAV, streaming=IP,
                thermal=dict(tau_T=0.8, g_beta=2e-4, T0=11.0, T_left=21.0, T_right=1.0))
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "state.bin")
        with case.lattice(lbm) as a:
            a.step(37)  # odd: saved at parity 1
            a.save(path)
            r_a = a.residual()
            a.step(13)
            want = [t.cpu().numpy() for t in a.get_populations()]
        with case.lattice(lbm) as b:
            b.load(path)
            assert b.step_count() == 37
            assert b.residual() == r_a
            b.step(13)
            got = [t.cpu().numpy() for t in b.get_populations()]
        with dataclasses.replace(case, streaming=0).lattice(lbm) as c:
            with pytest.raises(lbm.LbmError):
                c.load(path)  # a state file of the other streaming form
    assert all(np.array_equal(x, y) for x, y in zip(got, want))


def test_memory_and_rejections(lbm):
    """One population buffer instead of two: a 1024^2 FP32 context saves one buffer (32 MiB) less the
    ghost rows/column and, unless LBM_OPT_NO_RESIDUAL_RECORD is set, the 8 B per cell u(t-1) record."""
    import torch

    n = 1024 * 1024
    one = 8 * n * 4
    base = Case(1024, 1024, bc_x="wall", bc_y="wall", walls=CAV)
    cfg_nr = dataclasses.replace(base, streaming=IP).config(lbm)
    cfg_nr.options = lbm.OPT_NO_RESIDUAL_RECORD
    with base.lattice(lbm) as a, dataclasses.replace(base, streaming=IP).lattice(lbm) as b, lbm.Lattice(cfg_nr) as c:
        ma, mb, mc = a.memory_bytes(), b.memory_bytes(), c.memory_bytes()
        c.step(5)
        with pytest.raises(lbm.LbmError) as e:
            c.residual()
        assert e.value.code == lbm.ESTATE
    assert ma - mc >= 0.99 * one, (ma, mc)
    assert ma - mb >= 0.99 * one - 8 * n, (ma, mb)
    # extrapolated sides: a single lattice takes them (with a few bytes per boundary node for their
    # states), an in-place batch does not
    for bx, by in (("nee", "wall"), ("wall", "nee"), ("pressure", "wall")):
        with Case(32, 16, bc_x=bx, bc_y=by, streaming=IP).lattice(lbm) as lat:
            lat.step(3)
        with pytest.raises(lbm.LbmError) as e:
            lbm.Batch([Case(32, 16, bc_x=bx, bc_y=by, streaming=IP).config(lbm)])
        assert e.value.code == lbm.EINVAL
    torch.cuda.synchronize()
