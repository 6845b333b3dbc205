"""Pins of the oracle adjoint (oracle/adjoint.py): transpose identities of its pieces and the whole
gradient against central finite differences of the FP64 forward model."""
import numpy as np
import pytest

from oracle import adjoint as adj
from oracle import mrt_d2q8 as fl
from paper_1311_7239_gb300 import synth

rng = np.random.default_rng(4000)


def _flow(nx, ny, bc_x, bc_y, walls=None, forch=True, ax=0.0, p_in=1.0, p_out=1.0, seed=1):
    eps, K = synth.heterogeneous_medium(ny, nx, H=ny, seed=seed, da_mean=0.5 / ny**2 * 10, corr_len=3.0, eps_mean=0.5,
                                        eps_sd=0.08, eps_lo=0.2, eps_hi=0.9)
    w = walls or {}
    return fl.Flow(nx=nx, ny=ny, phi=eps, K=K, nu=0.08, forchheimer=forch, accel=np.array([ax, 0.0]), bc_x=bc_x, bc_y=bc_y,
                   u_top=w.get("top", (0.0, 0.0)), u_bottom=w.get("bottom", (0.0, 0.0)), u_left=w.get("left", (0.0, 0.0)),
                   u_right=w.get("right", (0.0, 0.0)), p_in=p_in, p_out=p_out)


CASES = {
    "cavity-lid-misfit": dict(nx=7, ny=6, bc_x="wall", bc_y="wall", walls={"top": (0.08, 0.0)}),
    "channel-force-flux": dict(nx=8, ny=5, bc_x="periodic", bc_y="wall", ax=2e-4),
    "pressure-flux": dict(nx=9, ny=5, bc_x="pressure", bc_y="wall", p_in=1.004, p_out=0.996),
    # extrapolated wall nodes (Sec. 3's wall treatment) on every side, on the y sides of a
    # force-driven channel, and with pressure columns
    "nee-cavity-lid-misfit": dict(nx=7, ny=6, bc_x="nee", bc_y="nee", walls={"top": (0.08, 0.0)}),
    "nee-channel-force-flux": dict(nx=8, ny=5, bc_x="periodic", bc_y="nee", ax=2e-4),
    "nee-pressure-flux": dict(nx=9, ny=5, bc_x="pressure", bc_y="nee", p_in=1.004, p_out=0.996),
    "nee-sides-force-misfit": dict(nx=6, ny=7, bc_x="nee", bc_y="wall", ax=2e-4, walls={"left": (0.0, 0.03)}),
}


@pytest.mark.parametrize("name", list(CASES))
def test_stream_transpose_dot_product(name):
    flow = _flow(**CASES[name])
    v = rng.standard_normal((8, flow.ny, flow.nx))
    lam = rng.standard_normal((8, flow.ny, flow.nx))
    Sv = fl.stream(v, flow) - fl.stream(np.zeros_like(v), flow)  # linear part
    assert abs(np.sum(lam * Sv) - np.sum(adj.stream_transpose(lam, flow) * v)) < 1e-12


def _fd(flow, T, kind, target, which, cell, h, phi_p_uniform):
    vals = []
    for s in (+1, -1):
        phi = flow.phi.copy()
        K = flow.K.copy()
        if which == "logK":
            K[cell] = np.exp(np.log(K[cell]) + s * h)
        else:
            phi[cell] += s * h
        fl2 = fl.Flow(**{**flow.__dict__, "phi": phi, "K": K})
        logK2 = np.log(K)
        f = adj.initial_state(fl2, logK2, phi, 1.0, (0.0, 0.0), phi_p_uniform)
        for _ in range(T):
            f = adj.step(f, fl2, logK2, phi)
        vals.append(adj.loss_value(f, fl2, kind, target))
    return (vals[0] - vals[1]) / (2 * h)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("phi_p_uniform", [False, True])
def test_gradient_matches_central_differences(name, phi_p_uniform):
    flow = _flow(**CASES[name])
    T = 12
    kind = "misfit" if "misfit" in name else "flux"
    target = (0.01 * rng.standard_normal((flow.ny, flow.nx)), 0.01 * rng.standard_normal((flow.ny, flow.nx)))
    L, glogk, gphi = adj.gradient(flow, T, kind, target, phi_p_uniform=phi_p_uniform)
    cells = [(0, 0), (flow.ny - 1, flow.nx - 1), (flow.ny // 2, 1), (1, flow.nx - 2), (flow.ny // 2, flow.nx // 2)]
    scale = max(np.abs(glogk).max(), np.abs(gphi).max())
    for cell in cells:
        fd_k = _fd(flow, T, kind, target, "logK", cell, 1e-5, phi_p_uniform)
        fd_p = _fd(flow, T, kind, target, "phi", cell, 1e-6, phi_p_uniform)
        assert abs(fd_k - glogk[cell]) <= 1e-6 * scale + 1e-5 * abs(fd_k), (cell, fd_k, glogk[cell])
        assert abs(fd_p - gphi[cell]) <= 1e-6 * scale + 1e-5 * abs(fd_p), (cell, fd_p, gphi[cell])
    assert scale > 0


def test_one_step_jacobian_transpose_dot_product():
    """<lam, J v> with J v by a complex step of the whole step, against <J^T lam, v> from the reverse pieces."""
    flow = _flow(**CASES["pressure-flux"])
    logK, phi = np.log(flow.K), flow.phi
    f = adj.initial_state(flow, logK, phi)
    for _ in range(5):
        f = adj.step(f, flow, logK, phi)
    v = rng.standard_normal(f.shape)
    v[:, :, [0, flow.nx - 1]] = 0.0  # the pressure columns of a state are a function of the rest
    lam = rng.standard_normal(f.shape)
    Jv = np.imag(adj.step(f + 1e-30j * v, flow, logK, phi)) / 1e-30
    fs = fl.stream(adj._collide(f, flow, logK, phi), flow)
    l1, _, _ = adj.pressure_vjp(fs, lam, flow, logK, phi)
    l2 = adj.stream_transpose(l1, flow)
    JTlam, _, _ = adj.collide_vjp(f, l2, flow, logK, phi)
    assert abs(np.sum(lam * Jv) - np.sum(JTlam * v)) < 1e-10 * np.abs(np.sum(lam * Jv))


@pytest.mark.parametrize("name", ["nee-cavity-lid-misfit", "nee-pressure-flux"])
def test_one_step_jacobian_transpose_dot_product_wall_nodes(name):
    """The same identity through the wall-node map W (and the pressure columns before it), whose
    corner nodes share their inner neighbour with the wall nodes beside them."""
    flow = _flow(**CASES[name])
    logK, phi = np.log(flow.K), flow.phi
    f = adj.initial_state(flow, logK, phi)
    for _ in range(5):
        f = adj.step(f, flow, logK, phi)
    v = rng.standard_normal(f.shape)
    lam = rng.standard_normal(f.shape)
    Jv = np.imag(adj.step(f + 1e-30j * v, flow, logK, phi)) / 1e-30
    fs = fl.stream(adj._collide(f, flow, logK, phi), flow)
    l1, _, _ = adj.boundary_vjp(fs, lam, flow, logK, phi)
    l2 = adj.stream_transpose(l1, flow)
    JTlam, _, _ = adj.collide_vjp(f, l2, flow, logK, phi)
    assert abs(np.sum(lam * Jv) - np.sum(JTlam * v)) < 1e-10 * np.abs(np.sum(lam * Jv))


def test_wall_vjp_against_single_cell_complex_steps():
    """wall_vjp perturbs all inner neighbours at once and scatters the result; here each entry of the
    VJP is recomputed by perturbing one cell's input (or theta) alone: d/dx <lam, W(fs)>.  With wall
    nodes on all four sides the inner corner node (1, 1) is the nb of three wall nodes (the corner
    (0, 0) and its neighbours (0, 1) and (1, 0)), so a scatter that dropped a shared contribution,
    or a wall node that kept its own adjoint, fails."""
    flow = _flow(**CASES["nee-cavity-lid-misfit"])
    logK, phi = np.log(flow.K), flow.phi
    fs = fl.stream(adj._collide(adj.initial_state(flow, logK, phi), flow, logK, phi), flow)
    lam = rng.standard_normal(fs.shape)
    got, glk, gph = adj.wall_vjp(fs, lam, flow, logK, phi)
    ny, nx = flow.ny, flow.nx
    for (y, x) in [(1, 1), (1, nx - 2), (ny - 2, 1), (ny - 2, nx - 2), (2, 1), (1, 3), (3, 3), (0, 0), (0, 2), (2, 0)]:
        for j in range(8):
            fc = fs.astype(np.complex128)
            fc[j, y, x] += 1e-30j
            want = np.sum(lam * np.imag(fl.wall_nodes(fc, flow)) / 1e-30)
            assert abs(got[j, y, x] - want) <= 1e-13 * (1 + abs(want)), ((y, x), j, got[j, y, x], want)
        for which, g in (("logK", glk), ("phi", gph)):
            lk = logK.astype(np.complex128)
            ph = phi.astype(np.complex128)
            (lk if which == "logK" else ph)[y, x] += 1e-30j
            want = np.sum(lam * np.imag(fl.wall_nodes(fs.astype(np.complex128), flow, phi=ph, K=np.exp(lk))) / 1e-30)
            assert abs(g[y, x] - want) <= 1e-13 * (1 + abs(want)), ((y, x), which, g[y, x], want)
