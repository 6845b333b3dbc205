"""Pins of the FP64 oracle's D2Q5 temperature step (Appendix B) and buoyancy coupling (Sec. 3.4)."""
import numpy as np
import pytest

from oracle import mrt_d2q8 as fl
from oracle import thermal_d2q5 as th

rng = np.random.default_rng(1311)


def _flow(nx, ny, **kw):
    return fl.Flow(nx=nx, ny=ny, phi=np.full((ny, nx), 0.6), K=np.full((ny, nx), 1e30), nu=0.1, **kw)


def test_N_is_eqB4_moment_polynomials_and_orthogonal():
    rows = np.array(
        [[1, ex, ey, 5 * (ex * ex + ey * ey) - 4, ex * ex - ey * ey] for ex, ey in th.E5], dtype=float
    ).T
    assert np.array_equal(rows, th.N)
    assert np.array_equal(th.N @ th.N.T, np.diag([5.0, 2, 2, 20, 4]))
    assert np.allclose(th.N @ th.N_INV, np.eye(5), atol=1e-15, rtol=0)


def test_rest_weights_are_one_fifth_at_varpi_zero():
    w = th.Thermal(tau_T=1.0, g_beta=0.0, T0=0.0).rest_weights()
    assert np.allclose(w, 0.2, atol=1e-16, rtol=0)


def test_collision_keeps_T_and_relaxes_flux_to_uT():
    p = th.Thermal(tau_T=0.7, g_beta=0.0, T0=1.0)
    g = rng.uniform(0.1, 1.0, (5, 4, 3))
    ux, uy = 0.05 * rng.standard_normal((2, 4, 3))
    gp = th.collide(g, ux, uy, p)
    T = g.sum(0)
    assert np.allclose(gp.sum(0), T, rtol=1e-14)
    jx = g[1] - g[3]
    jx_p = gp[1] - gp[3]
    assert np.allclose(jx_p, jx - (jx - ux * T) / 0.7, rtol=1e-13, atol=1e-15)


def test_total_temperature_conserved_with_adiabatic_walls():
    flow = _flow(7, 6, bc_x="wall", bc_y="wall")
    p = th.Thermal(tau_T=0.9, g_beta=0.0, T0=1.0)
    g = rng.uniform(0.1, 1.0, (5, 6, 7))
    total = g.sum()
    ux, uy = 0.05 * rng.standard_normal((2, 6, 7))
    for _ in range(20):
        g = th.stream(th.collide(g, ux, uy, p), flow, p)
    assert abs(g.sum() - total) < 1e-12 * total


def test_conduction_between_isothermal_walls_is_linear_and_nu_is_one():
    """u = 0, T_h at x = -1/2 and T_c at x = nx - 1/2 (halfway walls): T(x) = T_h - dT (x + 1/2)/nx."""
    nx, ny = 10, 3
    flow = _flow(nx, ny, bc_x="wall", bc_y="periodic")
    p = th.Thermal(tau_T=0.8, g_beta=0.0, T0=11.0, T_left=21.0, T_right=1.0)
    g = th.initial_state(flow, p)
    z = np.zeros((ny, nx))
    for _ in range(3000):
        g = th.stream(th.collide(g, z, z, p), flow, p)
    T = th.temperature(g)
    x = np.arange(nx) + 0.5
    assert np.allclose(T, 21.0 - 20.0 * x / nx, atol=1e-9)
    assert abs(th.nusselt_left_wall(T, 21.0, 21.0, 1.0, nx) - 1.0) < 1e-9


def test_advected_sine_mode_decays_and_moves_as_eqB1():
    """sigma dT/dt + u . grad T = alpha_e lap T with alpha_e = sigma c_sT^2 (tau_T - 1/2) (after Eq. B.7):
    a sine mode of wavenumber k moves at u/sigma and decays at alpha_e k^2 / sigma."""
    nx, ny = 64, 1
    flow = _flow(nx, ny, bc_x="periodic", bc_y="periodic")
    sig, tau = 1.0, 0.9
    p = th.Thermal(tau_T=tau, g_beta=0.0, T0=1.0, sigma=sig)
    k = 2 * np.pi / nx
    x = np.arange(nx)
    A = 0.1
    u = 0.02
    T_init = 1.0 + A * np.sin(k * x)[None, :]
    n0 = np.stack([T_init, u * T_init / sig, 0 * T_init, 0 * T_init, 0 * T_init])
    g = np.einsum("ik,kyx->iyx", th.N_INV, n0)
    ux = np.full((ny, nx), u)
    uy = np.zeros((ny, nx))
    steps = 400
    for _ in range(steps):
        g = th.stream(th.collide(g, ux, uy, p), flow, p)
    T = th.temperature(g)[0]
    alpha = sig * 0.4 * (tau - 0.5)
    exact = 1.0 + A * np.exp(-alpha * k * k * steps / sig) * np.sin(k * (x - u * steps / sig))
    assert np.abs(T - exact).max() < 2e-3 * A


def test_eq26_parameters_of_the_table1_case():
    nu, tau_v, tau_T, g_beta = th.parameters_from_Ra(L=2048, Ra=1e5, Pr=1.0, Ma=0.1)
    assert abs(tau_v - (0.5 + 0.1 * 2048 * np.sqrt(3) / np.sqrt(1e5))) < 1e-12
    # Pr = nu / alpha and Ra = g beta dT L^3 Pr / nu^2 (Sec. 3.4) hold for the returned values
    alpha = 1.0 * 0.4 * (tau_T - 0.5)
    assert abs(nu / alpha - 1.0) < 1e-12
    assert abs(g_beta * 20.0 * 2048**3 * 1.0 / nu**2 - 1e5) < 1e-6 * 1e5


def test_stably_stratified_rest_state_is_hydrostatic_with_upward_buoyancy():
    """A hot-over-cold linear T profile between isothermal top/bottom walls stays at rest, and its
    pressure is hydrostatic with the buoyancy a = g beta (T - T0) pointing up (+y, Sec. 3.4).

    At rest Eq. 2 reduces to grad(phi p) = rho0 phi a, so with uniform phi and rho0 = 1
    dp/dy = g beta (T - T0); T is linear in y, so p is quadratic and the difference of two adjacent
    cells equals g beta (T_mid - T0) exactly, T_mid the mean of the two cells' temperatures.
    A buoyancy pointing down (-y) reverses the sign of every difference."""
    nx, ny = 4, 16
    flow = fl.Flow(nx=nx, ny=ny, phi=np.full((ny, nx), 0.6), K=np.full((ny, nx), 0.01 * ny * ny), nu=0.1, bc_x="periodic", bc_y="wall")
    p = th.Thermal(tau_T=0.8, g_beta=1e-4, T0=11.0, T_bottom=1.0, T_top=21.0)
    # start from a pure-conduction state and let both fields relax
    f = fl.initial_state(flow)
    g = th.initial_state(flow, p)
    for _ in range(4000):
        f, g = th.coupled_step(f, g, flow, p)
    ux, uy, pr, T = th.coupled_macroscopic(f, g, flow, p)
    y = np.arange(ny) + 0.5
    assert np.allclose(T[:, 0], 1.0 + 20.0 * y / ny, atol=1e-8)
    assert np.abs(ux).max() < 1e-12 and np.abs(uy).max() < 1e-10
    dp = np.diff(pr, axis=0)
    expect = p.g_beta * (0.5 * (T[1:] + T[:-1]) - p.T0)
    assert np.abs(dp - expect).max() < 1e-10 * np.abs(expect).max()


def test_side_heated_cavity_rises_at_the_hot_wall():
    """Hot left wall, cold right wall, adiabatic bottom/top (the Table 1 cavity, Sec. 3.4) at
    Ra = 1e4, Da = 1e-2: warm fluid rises along the hot wall and sinks along the cold one, so the
    cavity turns clockwise (u_x > 0 under the top wall, u_x < 0 over the bottom wall).  Hot-wall
    Nusselt numbers cannot see the direction of a (a y-mirror leaves them unchanged); this does."""
    L = 24
    nu, _, tau_T, g_beta = th.parameters_from_Ra(L, 1e4, 1.0, 0.1)
    flow = fl.Flow(nx=L, ny=L, phi=np.full((L, L), 0.6), K=np.full((L, L), 1e-2 * L * L), nu=nu, bc_x="wall",
                   bc_y="wall")
    p = th.Thermal(tau_T=tau_T, g_beta=g_beta, T0=11.0, T_left=21.0, T_right=1.0)
    f = fl.initial_state(flow)
    g = th.initial_state(flow, p)
    for _ in range(1000):
        f, g = th.coupled_step(f, g, flow, p)
    ux, uy, _, T = th.coupled_macroscopic(f, g, flow, p)
    scale = np.sqrt(g_beta * 20.0 * L)  # the buoyancy velocity U of Eq. 26; the Darcy drag holds u near 0.016 U
    assert uy[:, 0].mean() > 0.005 * scale and uy[:, -1].mean() < -0.005 * scale
    assert ux[-1].mean() > 0.005 * scale and ux[0].mean() < -0.005 * scale
    # the hot wall side is the warmer half at mid height: the field is not mirrored either
    assert T[L // 2, : L // 2].mean() > T[L // 2, L // 2 :].mean()


def test_conduction_between_extrapolated_wall_nodes_is_linear_and_nu_is_one():
    """Isothermal wall nodes ('nee' x sides, the paper's extrapolation) at T_h and T_c, no flow
    (g beta = 0): the steady temperature is linear between the wall nodes (H = nx - 1) and both
    walls' Nusselt numbers are 1."""
    L = 17
    nu, tau_v, tau_T, gb = th.parameters_from_Ra(L - 1, 1e3, 1.0, 0.1)
    flow = fl.Flow(nx=L, ny=6, phi=np.full((6, L), 0.6), K=np.full((6, L), 1e-2 * (L - 1) ** 2), nu=nu, bc_x="nee",
                   bc_y="periodic")
    tp = th.Thermal(tau_T=tau_T, g_beta=0.0, T0=11.0, T_left=21.0, T_right=1.0)
    f = fl.initial_state(flow)
    g = th.initial_state(flow, tp, f=f)
    for _ in range(6000):
        f, g = th.coupled_step(f, g, flow, tp)
    T = th.coupled_macroscopic(f, g, flow, tp)[3]
    lin = 21.0 - 20.0 * np.arange(L) / (L - 1)
    assert np.abs(T - lin).max() < 1e-9
    assert abs(th.nusselt_wall_nodes(T, 0, 21.0, 1.0, corners_on_y_walls=False) - 1.0) < 1e-9
    assert abs(th.nusselt_wall_nodes(T, 1, 21.0, 1.0, corners_on_y_walls=False) - 1.0) < 1e-9


def test_adiabatic_extrapolated_wall_node_copies_the_neighbour_temperature():
    """An adiabatic 'nee' wall node takes T_b = T_nb exactly (g_eq(T_nb, u_w) + g_nb - g_eq(T_nb, u_nb)
    sums to T_nb); an isothermal one takes T_w."""
    nx, ny = 6, 5
    flow = fl.Flow(nx=nx, ny=ny, phi=np.full((ny, nx), 0.6), K=np.full((ny, nx), 4.0), nu=0.1, bc_x="nee", bc_y="nee",
                   u_top=(0.05, 0.0))
    tp = th.Thermal(tau_T=0.8, g_beta=1e-4, T0=11.0, T_left=21.0, T_right=1.0)
    rng = np.random.default_rng(4)
    f = fl.equilibrium(1.0 + 0.01 * rng.standard_normal((ny, nx)), *(0.02 * rng.standard_normal((2, ny, nx))), flow.phi)
    g = th.equilibrium(11.0 + rng.standard_normal((ny, nx)), *(0.02 * rng.standard_normal((2, ny, nx))), tp)
    g2 = th.boundary_nodes(f, g, flow, tp)[1]
    T, T2 = th.temperature(g), th.temperature(g2)
    assert np.allclose(T2[0, 1:-1], T[1, 1:-1]) and np.allclose(T2[-1, 1:-1], T[-2, 1:-1])  # adiabatic bottom/top
    assert np.allclose(T2[0, 0], T[1, 1]) and np.allclose(T2[-1, -1], T[-2, -2])  # corners: y walls, diagonal nb
    assert np.allclose(T2[1:-1, 0], 21.0) and np.allclose(T2[1:-1, -1], 1.0)  # isothermal sides
