"""FP64 oracle of the D2Q5 MRT temperature step and its buoyancy coupling (Appendix B, Sec. 3.4).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``); shares no code with the CUDA library.

Populations g have shape (5, ny, nx), index 0..4 = the paper's i = 0..4 (Eq. B.3).

Coupled step (the coupling order is not printed in the paper; this is the reading used):
    T = sum_i g_i (Eq. B.5, n_0)  ->  a = g beta (T - T0) j (Sec. 3.4)
    flow collision with that a (Eqs. 14-20)  ->  u(t)
    temperature collision with u(t) (Eq. B.2 with n_eq of Eq. B.6)
    both streams (Eq. 15 / Eq. B.2).
Thermal walls: a wall with a prescribed temperature T_w uses anti-bounce-back,
g_opp(i)(x, t+1) = -g_i+(x, t) + 2 w_i T_w, where w_i T is the u = 0 equilibrium of Eq. B.6
(w_i = 1/5 at varpi = 0); an adiabatic wall uses plain bounce-back.  On the wall nodes of 'nee'
sides (the paper's extrapolation, Sec. 3) g_b = g_eq(T_b, u_w) + g_nb - g_eq(T_nb, u_nb), with
T_b = T_w for a prescribed temperature and T_b = T_nb (zero normal gradient) for an adiabatic
wall, and u_nb the flow velocity at nb with the buoyancy of T_nb.
"""
from __future__ import annotations

from dataclasses import dataclass, replace

import numpy as np

from . import mrt_d2q8 as fl

# Eq. B.3: D2Q5 velocities
E5 = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1]], dtype=np.int64)
OPP5 = np.array([int(np.nonzero((E5 == -E5[i]).all(axis=1))[0][0]) for i in range(5)], dtype=np.int64)

# Eq. B.4: transformation matrix
N = np.array(
    [
        [1, 1, 1, 1, 1],
        [0, 1, 0, -1, 0],
        [0, 0, 1, 0, -1],
        [-4, 1, 1, 1, 1],
        [0, 1, -1, 1, -1],
    ],
    dtype=np.float64,
)
N_INV = np.linalg.inv(N)


@dataclass
class Thermal:
    """Temperature-field parameters (Appendix B, Sec. 3.4).

    tau_T: relaxation time of the first moments (zeta1 = zeta2 = 1/tau_T, Eq. B.7).
    zeta3, zeta4: remaining rates (1.1 in Sec. 3.4); sigma: thermal capacity ratio; varpi: Eq. B.6.
    g_beta: g * beta of the Boussinesq body force a = g beta (T - T0) j; T0: reference temperature.
    T_left/T_right/T_bottom/T_top: wall temperature, or None for an adiabatic wall.
    """

    tau_T: float
    g_beta: float
    T0: float
    sigma: float = 1.0
    zeta3: float = 1.1
    zeta4: float = 1.1
    varpi: float = 0.0
    T_left: float | None = None
    T_right: float | None = None
    T_bottom: float | None = None
    T_top: float | None = None

    def rates(self):
        """Theta = diag(1, zeta1, zeta2, zeta3, zeta4), Eq. B.7."""
        z = 1.0 / self.tau_T
        return np.array([1.0, z, z, self.zeta3, self.zeta4])

    def rest_weights(self):
        """w_i with g_eq,i(T, u = 0) = w_i T: N^-1 applied to n_eq(T = 1, u = 0) of Eq. B.6."""
        return N_INV @ np.array([1.0, 0.0, 0.0, self.varpi, 0.0])


def equilibrium_moments(T, ux, uy, th: Thermal):
    """Eq. B.6: n_eq = (T, u_x T / sigma, u_y T / sigma, varpi T, 0)."""
    return np.stack([T, ux * T / th.sigma, uy * T / th.sigma, th.varpi * T, 0.0 * T])


def temperature(g):
    """T = n_0 = sum_i g_i (Eq. B.5 and the sentence after it)."""
    return g.sum(axis=0)


def collide(g, ux, uy, th: Thermal):
    """g+ = N^-1 [n - Theta (n - n_eq)] (Eq. B.2 in moment space)."""
    n = np.einsum("ki,i...->k...", N, g)
    n_eq = equilibrium_moments(n[0], ux, uy, th)
    theta = th.rates().reshape((5,) + (1,) * (g.ndim - 1))
    return np.einsum("ik,k...->i...", N_INV, n - theta * (n - n_eq))


def stream(g_plus, flow: fl.Flow, th: Thermal):
    """g_i(x + e_i, t+1) = g_i+(x, t); links through a wall: anti-bounce-back (wall temperature
    given) or bounce-back (adiabatic).  At a corner the bottom/top wall owns the link (the D2Q5
    links are axis-aligned, so no link crosses two walls)."""
    ny, nx = flow.ny, flow.nx
    ys, xs = np.mgrid[0:ny, 0:nx]
    w = th.rest_weights()
    out = np.zeros_like(g_plus)
    out[0] = g_plus[0]
    for i in range(1, 5):
        tx = xs + E5[i, 0]
        ty = ys + E5[i, 1]
        if flow.bc_x in ("periodic", "nee"):  # 'nee' wall nodes are overwritten by wall_nodes
            tx = tx % nx
        if flow.bc_y in ("periodic", "nee"):
            ty = ty % ny
        inside = (tx >= 0) & (tx < nx) & (ty >= 0) & (ty < ny)
        out[i, ty[inside], tx[inside]] = g_plus[i, ys[inside], xs[inside]]
        for mask, Tw in (
            (tx < 0, th.T_left),
            (tx >= nx, th.T_right),
            (ty < 0, th.T_bottom),
            (ty >= ny, th.T_top),
        ):
            if not mask.any():
                continue
            src = g_plus[i, ys[mask], xs[mask]]
            if Tw is None:
                out[OPP5[i], ys[mask], xs[mask]] = src
            else:
                out[OPP5[i], ys[mask], xs[mask]] = -src + 2.0 * w[i] * Tw
    return out


def equilibrium(T, ux, uy, th: Thermal):
    """g_eq = N^-1 n_eq (Eq. B.6)."""
    return np.einsum("ik,k...->i...", N_INV, equilibrium_moments(T, ux, uy, th))


def _buoyant(flow: fl.Flow, th: Thermal, T):
    """The flow problem with a = a0 + g beta (T - T0) j as a field (Sec. 3.4)."""
    ax0, ay0 = fl._accel(flow, T)
    return replace(flow, accel=np.stack([ax0 + 0.0 * T, ay0 + th.g_beta * (T - th.T0)]))


def boundary_nodes(f, g, flow: fl.Flow, th: Thermal):
    """Wall nodes of 'nee' sides for both equations after streaming (flow: fl.wall_nodes with the
    buoyancy of the streamed temperature; temperature: see the module docstring)."""
    if "nee" not in (flow.bc_x, flow.bc_y):
        return fl.boundary_nodes(f, flow), g
    bflow = _buoyant(flow, th, temperature(g))
    yb, xb, yn, xn, side = fl.wall_node_list(bflow)
    fn, gn = f[:, yn, xn], g[:, yn, xn]
    ax, ay = fl._accel(bflow, f[0])
    ux, uy = fl.velocity(fn, flow.phi[yn, xn], flow.K[yn, xn], flow.nu, flow.rho0, flow.forchheimer, ax[yn, xn], ay[yn, xn])
    Tn = temperature(gn)
    Tw = [th.T_left, th.T_right, th.T_bottom, th.T_top]
    Tb = np.array([Tn[k] if Tw[side[k]] is None else Tw[side[k]] for k in range(side.size)])
    uw = np.array([flow.u_left, flow.u_right, flow.u_bottom, flow.u_top], dtype=np.float64)[side]
    g_out = g.copy()
    g_out[:, yb, xb] = equilibrium(Tb, uw[:, 0], uw[:, 1], th) + gn - equilibrium(Tn, ux, uy, th)
    return fl.boundary_nodes(f, bflow), g_out


def initial_state(flow: fl.Flow, th: Thermal, T_init=None, f=None):
    """g at equilibrium (Eq. B.6) with u = 0 and T = T_init (default T0); with 'nee' sides its wall
    nodes follow the extrapolation from the flow state f (default: the flow's initial state)."""
    T = np.full((flow.ny, flow.nx), th.T0 if T_init is None else float(T_init))
    z = np.zeros_like(T)
    g = equilibrium(T, z, z, th)
    if "nee" in (flow.bc_x, flow.bc_y):
        g = boundary_nodes(fl.initial_state(flow) if f is None else f, g, flow, th)[1]
    return g


def coupled_step(f, g, flow: fl.Flow, th: Thermal):
    """One step of the flow (Eq. 6) and temperature (Eq. B.2) equations with buoyancy."""
    T = temperature(g)
    bflow = _buoyant(flow, th, T)
    ax, ay = fl._accel(bflow, T)
    f_plus, ux, uy, _ = fl.collide(f, flow, ax=ax, ay=ay)
    g_plus = collide(g, ux, uy, th)
    return boundary_nodes(fl.stream(f_plus, flow), stream(g_plus, flow, th), flow, th)


def coupled_macroscopic(f, g, flow: fl.Flow, th: Thermal):
    """(ux, uy, p, T) of a pre-collision state, u with the buoyancy of that state's T."""
    T = temperature(g)
    ax0, ay0 = fl._accel(flow, T)
    ux, uy, p = fl.macroscopic(f, flow, ax=ax0 + 0.0 * T, ay=ay0 + th.g_beta * (T - th.T0))
    return ux, uy, p, T


def nusselt_left_wall(T, T_wall, T_hot, T_cold, width):
    """Average Nusselt number of the x = 0 wall (Table 1's quantity).

    Nu = (L / dT) * mean_y(-dT/dx at the wall), L = width (wall-to-wall distance), dT = T_hot - T_cold.
    The wall lies at x = -1/2; dT/dx there is the derivative of the parabola through
    (wall, T_wall), (x=0, T[:,0]), (x=1, T[:,1]).
    """
    s = np.array([0.0, 0.5, 1.5])  # distances from the wall
    # coefficients c of dT/ds(0) = c . (T_wall, T0, T1): derivative of the Lagrange basis at s = 0
    c = np.zeros(3)
    for k in range(3):
        others = [s[j] for j in range(3) if j != k]
        denom = np.prod([s[k] - o for o in others])
        # d/ds prod_{j != k} (s - s_j) at s = 0
        c[k] = (-(others[0]) - (others[1])) / denom
    dTdx = c[0] * T_wall + c[1] * T[:, 0] + c[2] * T[:, 1]
    return float(-np.mean(dTdx) * width / (T_hot - T_cold))


def nusselt_wall_nodes(T, side, T_hot, T_cold, corners_on_y_walls=True):
    """Average Nusselt number of the x = 0 (side 0) or x = nx-1 (side 1) wall when the walls lie
    on the outermost nodes: Nu = (L / dT) * mean_y(-+ dT/dx at the wall node), L = nx - 1, with the
    second-order one-sided difference dT/dx ~ (-3 T_0 + 4 T_1 - T_2) / 2 (mirrored for side 1).
    When the bottom/top walls are wall nodes too they own the corner nodes, whose rows are left out."""
    if corners_on_y_walls:
        T = T[1:-1]
    Tn = T if side == 0 else T[:, ::-1]
    dTds = (-3.0 * Tn[:, 0] + 4.0 * Tn[:, 1] - Tn[:, 2]) / 2.0
    L = T.shape[1] - 1
    # s runs into the fluid: -dT/dx = -dT/ds at the left wall, +dT/ds at the right one
    return float((-1.0 if side == 0 else 1.0) * np.mean(dTds) * L / (T_hot - T_cold))


def parameters_from_Ra(L, Ra, Pr, Ma, J=1.0, sigma=1.0, gamma=1.0, varpi=0.0, dT=20.0):
    """Eq. 26 and the definitions of Sec. 3.4 (c = delta_t = 1).

    Returns (nu, tau_v, tau_T, g_beta): tau_v = 1/2 + Ma J L sqrt(3 Pr) / sqrt(Ra),
    tau_T = 1/2 + gamma c_s^2 (tau_v - 1/2) / (J sigma c_sT^2 Pr), c_sT^2 = (4 + varpi)/10,
    upsilon_e = c_s^2 (tau_v - 1/2) = J upsilon, and U = Ma / sqrt(3) = sqrt(g beta dT L).
    """
    tau_v = 0.5 + Ma * J * L * np.sqrt(3.0 * Pr) / np.sqrt(Ra)
    c_sT2 = (4.0 + varpi) / 10.0
    tau_T = 0.5 + gamma * fl.C_S2 * (tau_v - 0.5) / (J * sigma * c_sT2 * Pr)
    nu = fl.C_S2 * (tau_v - 0.5) / J
    U = Ma / np.sqrt(3.0)
    g_beta = U * U / (dT * L)
    return nu, tau_v, tau_T, g_beta
