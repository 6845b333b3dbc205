"""GPU discrete adjoint (lbm_adjoint, through the C-ABI) against the FP64 oracle adjoint
(complex-step Jacobians) and against central finite differences of the FP64 oracle forward model.

Bar: the FP32 adjoint (FP64 gradient accumulation) agrees with both to 1e-4 relative to the
largest gradient component, and to 1e-4 relative element by element on every cell whose gradient
is at least FLOOR of the largest (below it the FP32 forward state's rounding, ~1e-6 of the largest
gradient, dominates a per-element relative error).
"""
import numpy as np
import pytest

from oracle import adjoint as adj
from oracle import mrt_d2q8 as fl
from tests.cases import Case, rel_l2

pytestmark = pytest.mark.gpu
FLOOR = 1e-2


def _per_element(g, g_ref, scale):
    """Largest relative error |g - g_ref| / |g_ref| over the cells with |g_ref| >= FLOOR * scale, and
    how many cells that is."""
    g, g_ref = np.asarray(g, dtype=np.float64), np.asarray(g_ref, dtype=np.float64)
    m = np.abs(g_ref) >= FLOOR * scale
    return (float((np.abs(g - g_ref)[m] / np.abs(g_ref[m])).max()) if m.any() else 0.0), int(m.sum())


@pytest.fixture(scope="module")
def lbm():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1311_7239_gb300 import build, lbm

    build.build()
    return lbm


def _run(lbm, case, T, kind, target, phip):
    flow = case.flow()
    with case.lattice(lbm) as lat:
        if phip is not None:
            lat.init_equilibrium(phip, 0.0, 0.0, phi_p_uniform=True)
        else:
            lat.init_equilibrium(1.0, 0.0, 0.0)
        tgt = None
        if target is not None:
            import torch

            tgt = tuple(torch.tensor(t, dtype=torch.float32, device="cuda") for t in target)
        L, gk, ge = lat.adjoint(T, kind, tgt)
        gk, ge = gk.cpu().numpy(), ge.cpu().numpy()
    Lo, gko, geo = adj.gradient(flow, T, kind, None if target is None else tuple(np.float64(t) for t in target),
                                p0=1.0 if phip is None else phip, phi_p_uniform=phip is not None)
    return flow, (L, gk, ge), (Lo, gko, geo)


CASES = {
    "pressure-channel-flux": (Case(64, 32, nu=0.1, phi=0.35, K=0.05 * 32 * 32, het=True, eps_sd=0.03, corr=8.0, bc_x="pressure",
                                   bc_y="wall", p_in=1.003, p_out=0.997), 60, "flux", True),
    "lid-cavity-misfit": (Case(24, 20, nu=0.06, phi=0.5, K=4.0, het=True, eps_sd=0.05, corr=4.0, bc_x="wall", bc_y="wall",
                               walls={"top": (0.08, 0.0)}), 40, "misfit", False),
    "forced-channel-flux": (Case(20, 16, nu=0.08, phi=0.4, K=6.0, het=True, eps_sd=0.05, corr=4.0, ax=3e-4), 30, "flux", False),
    # rows longer than one work item (150 cell pairs > 128 threads): the split-row tiling
    "long-row-pressure-channel": (Case(300, 8, nu=0.1, phi=0.35, K=0.05 * 8 * 8, het=True, eps_sd=0.03, corr=8.0, bc_x="pressure",
                                       bc_y="wall", p_in=1.001, p_out=0.999), 12, "flux", True),
    # extrapolated wall nodes (Sec. 3's wall treatment): on all four sides, where each inner corner
    # node is the nb of three wall nodes; on the y sides of pressure-driven and force-driven
    # channels; and on split rows
    "nee-lid-cavity-misfit": (Case(24, 20, nu=0.06, phi=0.5, K=4.0, het=True, eps_sd=0.05, corr=4.0, bc_x="nee", bc_y="nee",
                                   walls={"top": (0.08, 0.0)}), 40, "misfit", False),
    "nee-pressure-channel-flux": (Case(64, 32, nu=0.1, phi=0.35, K=0.05 * 32 * 32, het=True, eps_sd=0.03, corr=8.0,
                                       bc_x="pressure", bc_y="nee", p_in=1.003, p_out=0.997), 60, "flux", True),
    "nee-forced-channel-flux": (Case(20, 16, nu=0.08, phi=0.4, K=6.0, het=True, eps_sd=0.05, corr=4.0, ax=3e-4, bc_y="nee"), 30,
                                "flux", False),
    "nee-long-row-cavity-misfit": (Case(300, 8, nu=0.1, phi=0.5, K=4.0, het=True, eps_sd=0.05, corr=4.0, bc_x="nee", bc_y="nee",
                                        walls={"top": (0.05, 0.0), "left": (0.0, 0.02)}), 12, "misfit", False),
}


@pytest.mark.parametrize("name", list(CASES))
def test_adjoint_matches_oracle_adjoint(lbm, accuracy, name):
    case, T, kind, phip = CASES[name]
    rng = np.random.default_rng(7)
    target = None
    if kind == "misfit":
        target = (0.01 * rng.standard_normal((case.ny, case.nx)), 0.01 * rng.standard_normal((case.ny, case.nx)))
    flow, (L, gk, ge), (Lo, gko, geo) = _run(lbm, case, T, kind, target, case.p_rest() if phip else None)
    assert abs(L - Lo) <= 1e-5 * abs(Lo) + 1e-9, (L, Lo)
    sk, se = np.abs(gko).max(), np.abs(geo).max()
    assert sk > 0 and se > 0
    ek, nk = _per_element(gk, gko, sk)
    ee, ne = _per_element(ge, geo, se)
    accuracy.append({"case": f"adjoint {name}, T {T}", "precision": "fp32 (fp64 gradients)", "rel_loss": abs(L - Lo) / abs(Lo),
                     "max_rel_grad_logK": float(np.abs(gk - gko).max() / sk), "max_rel_grad_eps": float(np.abs(ge - geo).max() / se),
                     "max_elementwise_rel_grad_logK": ek, "max_elementwise_rel_grad_eps": ee, "elementwise_cells": [nk, ne],
                     "elementwise_floor": FLOOR, "bound": 1e-4})
    assert np.abs(gk - gko).max() <= 1e-4 * sk, (np.abs(gk - gko).max(), sk)
    assert np.abs(ge - geo).max() <= 1e-4 * se, (np.abs(ge - geo).max(), se)
    assert ek <= 1e-4 and ee <= 1e-4, (ek, nk, ee, ne)


def test_adjoint_matches_central_differences_at_64_cells(lbm, accuracy):
    """Config-4-like crop: pressure-driven heterogeneous channel, outlet flux, 64 random cells."""
    case, T, kind, _ = CASES["pressure-channel-flux"]
    phip = case.p_rest()
    flow, (L, gk, ge), _ = _run(lbm, case, T, kind, None, phip)
    rng = np.random.default_rng(64)
    cells = [(int(rng.integers(0, case.ny)), int(rng.integers(0, case.nx))) for _ in range(64)]
    sk, se = np.abs(gk).max(), np.abs(ge).max()

    def loss(phi, K):
        fl2 = fl.Flow(**{**flow.__dict__, "phi": phi, "K": K})
        lk = np.log(K)
        f = adj.initial_state(fl2, lk, phi, phip, (0.0, 0.0), True)
        for _ in range(T):
            f = adj.step(f, fl2, lk, phi)
        return adj.loss_value(f, fl2, "flux")

    worst = {"logK": 0.0, "phi": 0.0}
    worst_el = {"logK": 0.0, "phi": 0.0}
    for cell in cells:
        for which, h in (("logK", 1e-4), ("phi", 1e-5)):
            vals = []
            for s in (1, -1):
                phi, K = flow.phi.copy(), flow.K.copy()
                if which == "logK":
                    K[cell] *= np.exp(s * h)
                else:
                    phi[cell] += s * h
                vals.append(loss(phi, K))
            fd = (vals[0] - vals[1]) / (2 * h)
            g, sc = (gk[cell], sk) if which == "logK" else (ge[cell], se)
            worst[which] = max(worst[which], abs(g - fd) / sc)
            assert abs(g - fd) <= 1e-4 * sc, (cell, which, g, fd, sc)
            if abs(fd) >= FLOOR * sc:  # element by element where the gradient is not tiny
                worst_el[which] = max(worst_el[which], abs(g - fd) / abs(fd))
                assert abs(g - fd) <= 1e-4 * abs(fd), (cell, which, g, fd)
    accuracy.append({"case": f"adjoint vs central differences of the FP64 oracle, 64 cells, T {T}", "precision": "fp32 (fp64 gradients)",
                     "max_rel_grad_logK": worst["logK"], "max_rel_grad_eps": worst["phi"],
                     "max_elementwise_rel_grad_logK": worst_el["logK"], "max_elementwise_rel_grad_eps": worst_el["phi"],
                     "elementwise_floor": FLOOR, "bound": 1e-4})


def test_autograd_function(lbm):
    import torch

    from paper_1311_7239_gb300.lbm import PorousFlowLoss

    case, T, kind, _ = CASES["forced-channel-flux"]
    eps, K = case.medium()
    logk = torch.tensor(np.log(K), dtype=torch.float32, device="cuda", requires_grad=True)
    e = torch.tensor(eps, dtype=torch.float32, device="cuda", requires_grad=True)
    loss = PorousFlowLoss.apply(logk, e, case.config(lbm), T, "flux", None)
    (2.0 * loss).backward()
    flow = case.flow()
    Lo, gko, geo = adj.gradient(flow, T, "flux")
    assert abs(loss.item() - Lo) <= 1e-5 * abs(Lo)
    assert rel_l2(logk.grad.cpu().numpy(), 2 * gko) <= 1e-4
    assert rel_l2(e.grad.cpu().numpy(), 2 * geo) <= 1e-4


def test_workspace_is_reused_and_released(lbm):
    """Repeated adjoint calls (as in an optimisation loop) reuse the retained workspace and give
    bitwise the same result; a call with another T resizes it; release frees it."""
    case, T, kind, phip = CASES["pressure-channel-flux"]
    p0 = case.p_rest()
    with case.lattice(lbm) as lat:
        base = lat.memory_bytes()
        lat.init_equilibrium(p0, 0.0, 0.0, phi_p_uniform=True)
        L1, gk1, ge1 = lat.adjoint(T, kind)
        held = lat.memory_bytes()
        assert held > base
        lat.init_equilibrium(p0, 0.0, 0.0, phi_p_uniform=True)
        L2, gk2, ge2 = lat.adjoint(T, kind)
        assert lat.memory_bytes() == held
        assert L1 == L2 and bool((gk1 == gk2).all()) and bool((ge1 == ge2).all())
        lat.init_equilibrium(p0, 0.0, 0.0, phi_p_uniform=True)
        L3, gk3, ge3 = lat.adjoint(2 * T + 7, kind)
        Lo, gko, geo = adj.gradient(case.flow(), 2 * T + 7, kind, None, p0=p0, phi_p_uniform=True)
        assert abs(L3 - Lo) <= 1e-5 * abs(Lo)
        assert np.abs(gk3.cpu().numpy() - gko).max() <= 1e-4 * np.abs(gko).max()
        assert np.abs(ge3.cpu().numpy() - geo).max() <= 1e-4 * np.abs(geo).max()
        lat.release_workspace()
        assert lat.memory_bytes() == base


def test_adjoint_step_name_is_the_same_call(lbm):
    """lbm_adjoint_step (the interface description's name) returns what lbm_adjoint returns."""
    import torch

    case, T, kind, phip = CASES["forced-channel-flux"]
    with case.lattice(lbm) as lat:
        lat.init_equilibrium(1.0, 0.0, 0.0)
        L1, gk1, ge1 = lat.adjoint(T, kind)
        lat.init_equilibrium(1.0, 0.0, 0.0)
        gk2 = torch.zeros_like(gk1)
        ge2 = torch.zeros_like(ge1)
        L2 = torch.zeros(1, dtype=torch.float64, device="cuda")
        rc = lbm.lib().lbm_adjoint_step(lat._h, T, lbm.LOSS_OUTLET_FLUX, None, None, gk2.data_ptr(), ge2.data_ptr(), L2.data_ptr())
        assert rc == lbm.OK
        assert L1 == float(L2.item()) and bool((gk1 == gk2).all()) and bool((ge1 == ge2).all())


@pytest.mark.parametrize("name", ["lid-cavity-misfit", "nee-pressure-channel-flux"])
def test_inplace_context_adjoint_equals_ab_context(lbm, name):
    """An in-place context's adjoint runs the A-B sweep on workspace buffers: the loss and gradients
    are bitwise those of an A-B context, its state after the call is the A-B state after T steps
    (to one rounding), and stepping and the residual continue from there."""
    import dataclasses

    import torch

    case, T, kind, phip = CASES[name]
    rng = np.random.default_rng(7)
    target = None
    if kind == "misfit":
        target = tuple(torch.tensor(0.01 * rng.standard_normal((case.ny, case.nx)), dtype=torch.float32, device="cuda")
                       for _ in range(2))
    p0 = case.p_rest() if phip else 1.0
    with case.lattice(lbm) as a, dataclasses.replace(case, streaming=1).lattice(lbm) as b:
        for lat in (a, b):
            lat.init_equilibrium(p0, 0.0, 0.0, phi_p_uniform=bool(phip))
        La, gka, gea = a.adjoint(T, kind, target)
        Lb, gkb, geb = b.adjoint(T, kind, target)
        assert La == Lb and bool((gka == gkb).all()) and bool((gea == geb).all())
        # the state moves into the in-place layout as deviations; a link through a moving wall is
        # parked minus its wall term and read back plus it, within one rounding
        sa, sb = a.get_populations().cpu().numpy(), b.get_populations().cpu().numpy()
        assert np.abs(sa - sb).max() <= 1e-6, np.abs(sa - sb).max()
        a.step(7)
        b.step(7)
        fa, fb = a.get_populations().cpu().numpy(), b.get_populations().cpu().numpy()
        assert rel_l2(fb, fa) <= 1e-6
        assert abs(a.residual() - b.residual()) <= 1e-3 * abs(a.residual())
