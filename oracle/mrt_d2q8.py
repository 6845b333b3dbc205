"""FP64 oracle of the porous D2Q8 MRT-LB flow step (Liu & He, arXiv 1311.7239, Sec. 2.2 and Sec. 3).

TEST INFRASTRUCTURE ONLY: imported by tests, ``__graft_entry__.smoke()`` and the CPU legs of
``bench.py``; never by the product path.  It shares no code with the CUDA library.

Everything here is numpy on arrays of shape (8, ny, nx) for populations (index 0..7 holds the
paper's i = 1..8) and (ny, nx) for fields; row y = 0 is the bottom wall side, y = ny-1 the top.
Every function also accepts complex128 inputs so that ``oracle.adjoint`` can take complex-step
derivatives through it; for that reason magnitudes are written as sqrt(x^2 + y^2), never abs().

One time step follows the paper's order (Eq. 6 split as Eqs. 14-15):
    f(x, t)  --m = M f (Eq. 8)-->  u (Eqs. 17-19), p (Eq. 20), F (Eq. 3), S (Eq. 16), m_eq (Eqs. 11-12)
             --collide (Eq. 14)-->  m+  --f+ = M^-1 m+ (Eq. 15)-->  stream (Eq. 15)  -->  f(x, t+1)

Readings of the paper used here, where it is silent or ambiguous:
  * The third and fifth equilibrium moments j_x, j_y of Eq. 11 are rho0*u_x, rho0*u_y (the
    incompressible approximation J ~ rho0 u stated after Eq. 12, confirmed by Eq. A.3, whose
    first-order j_x is -rho0 F_x / 2).
  * In Eq. 20, s0(u) = omega0 * (-1.5 |u|^2 / phi) = -2|u|^2/(3 phi) (the general s_i(u) given
    after Eq. 20 at i = 0); the printed extra rho0 is dropped, which is moot at rho0 = 1.
  * Walls are halfway bounce-back (the wall lies half a link outside the outermost fluid cell)
    with the moving-wall term 2 omega_i rho0 (e_i . u_w) / c_s^2; the linear term of Eq. 22 has no
    phi, so neither has this term.  At a corner the y-side wall (bottom or top) owns the link.
  * Pressure inlet/outlet columns use non-equilibrium extrapolation (the scheme the paper cites
    for its boundaries, Sec. 3): f_b = f_eq(p_b, u_nb; phi_b) + f_nb - f_eq(p_nb, u_nb; phi_nb),
    with f_eq = M^-1 m_eq and nb the adjacent interior column, applied after streaming.
  * The same extrapolation on wall nodes ('nee' sides, the paper's own wall treatment, Sec. 3):
    the wall lies on the outermost nodes (channel height H = ny - 1), and a wall node takes
    f_b = f_eq(p_nb, u_w; phi_b) + f_nb - f_eq(p_nb, u_nb; phi_nb), nb being the node one step
    inward along the wall normal (the diagonal one at a corner where the other side is not
    periodic), p extrapolated with zero normal gradient.  Bottom/top walls own the corners.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# ---------------------------------------------------------------------------------------------
# Lattice (Eq. 7) and weights (the omega_i listed after Eq. 20), c = 1, c_s^2 = 1/3 (Sec. 2.2)
# ---------------------------------------------------------------------------------------------
C_S2 = 1.0 / 3.0
E = np.array([[1, 0], [0, 1], [-1, 0], [0, -1], [1, 1], [-1, 1], [-1, -1], [1, -1]], dtype=np.int64)
W = np.array([1 / 9] * 4 + [1 / 36] * 4, dtype=np.float64)
W0 = 4.0 / 9.0
# opposite direction of each i (e_opp = -e_i), found by search rather than typed
OPP = np.array([int(np.nonzero((E == -E[i]).all(axis=1))[0][0]) for i in range(8)], dtype=np.int64)

# Transformation matrix, Eq. 10 (rows: p, e, j_x, q_x, j_y, q_y, p_xx, p_xy; Eq. 9)
M = np.array(
    [
        [1, 1, 1, 1, 1, 1, 1, 1],
        [-1, -1, -1, -1, 1, 1, 1, 1],
        [1, 0, -1, 0, 1, -1, -1, 1],
        [-2, 0, 2, 0, 1, -1, -1, 1],
        [0, 1, 0, -1, 1, 1, -1, -1],
        [0, -2, 0, 2, 1, 1, -1, -1],
        [1, -1, 1, -1, 0, 0, 0, 0],
        [0, 0, 0, 0, 1, -1, 1, -1],
    ],
    dtype=np.float64,
)
# Eq. 8: f = M^-1 m.  Obtained numerically (LU inverse), not from the closed form.
M_INV = np.linalg.inv(M)

# Equilibrium-moment constants chosen after Eq. 12
ALPHA2, C1, C2, GAMMA1, GAMMA2, GAMMA3 = -1.0, -2.0, -2.0, 2.0 / 3.0, 0.0, 2.0 / 3.0


# ---------------------------------------------------------------------------------------------
# Problem description
# ---------------------------------------------------------------------------------------------
@dataclass
class Flow:
    """One porous-flow problem on an nx x ny lattice (all quantities in lattice units).

    phi, K: porosity and permeability per cell, arrays (ny, nx) (Eq. 3).
    nu: fluid kinematic viscosity upsilon (Eq. 3); J = upsilon_e / upsilon (Eq. 5).
    accel: external acceleration a (Eq. 3), shape (2,) or (2, ny, nx).
    rates: optional full diagonal of Lambda (Eq. 13); default (1, s_e, 1, s_q, 1, s_q, s_v, s_v)
           with s_v = 1/tau_v and upsilon_e = c_s^2 (tau_v - 1/2) (Eq. 21).
    forchheimer: F_phi from Ergun's relation (Eq. 4) if True, else F_phi = 0 (Brinkman limit).
    bc_x: 'periodic' | 'wall' | 'pressure' | 'nee';  bc_y: 'periodic' | 'wall' | 'nee'
          ('wall': halfway bounce-back; 'nee': wall nodes with non-equilibrium extrapolation).
    u_left/u_right/u_bottom/u_top: wall velocities (2,) of the four sides (moving lid = u_top).
    p_in/p_out: pressures of the x = 0 and x = nx-1 columns when bc_x == 'pressure'.
    """

    nx: int
    ny: int
    phi: np.ndarray
    K: np.ndarray
    nu: float
    J: float = 1.0
    rho0: float = 1.0
    s_e: float = 1.1
    s_q: float = 1.2
    rates: np.ndarray | None = None
    forchheimer: bool = True
    accel: np.ndarray = field(default_factory=lambda: np.zeros(2))
    bc_x: str = "periodic"
    bc_y: str = "wall"
    u_left: tuple = (0.0, 0.0)
    u_right: tuple = (0.0, 0.0)
    u_bottom: tuple = (0.0, 0.0)
    u_top: tuple = (0.0, 0.0)
    p_in: float = 1.0
    p_out: float = 1.0

    def tau_v(self):
        """Eq. 21 with upsilon_e = J * upsilon (Eq. 5): tau_v = upsilon_e / c_s^2 + 1/2.

        J may be a field (ny, nx): the region-dependent s_v = 1/[1/2 + J upsilon / c_s^2] of Sec. 3.2."""
        return np.asarray(self.J) * self.nu / C_S2 + 0.5

    def relaxation(self) -> np.ndarray:
        """Diagonal of Lambda, Eq. 13, with the values of Sec. 3 (s1 = s3 = s5 = 1); shape (8,), or
        (8, ny, nx) when J is a field."""
        if self.rates is not None:
            return np.asarray(self.rates, dtype=np.float64)
        s_v = 1.0 / self.tau_v()
        one = np.ones_like(s_v)
        return np.stack([one, self.s_e * one, one, self.s_q * one, one, self.s_q * one, s_v, s_v])


def ergun_F(phi):
    """Geometric function F_phi = 1.75 / sqrt(150 phi^3), Eq. 4."""
    return 1.75 / np.sqrt(150.0 * phi**3)


def _norm2(x, y):
    """sqrt(x^2 + y^2), defined as exactly 0 where the real parts of x and y are both 0.

    At a zero vector the magnitude has no derivative; the value 0 there makes the complex-step
    derivative of |v| zero at v = 0 (the one-sided limit used by the adjoint).
    """
    s = x * x + y * y
    zero = (np.real(x) == 0) & (np.real(y) == 0)
    s = np.where(zero, 1.0, s)
    return np.where(zero, 0.0, np.sqrt(s))


def _accel(flow: Flow, like):
    a = np.asarray(flow.accel)
    if a.ndim == 1:
        ax = np.full(like.shape, a[0], dtype=np.result_type(like, a))
        ay = np.full(like.shape, a[1], dtype=np.result_type(like, a))
        return ax, ay
    return a[0], a[1]


# ---------------------------------------------------------------------------------------------
# Macroscopic quantities, Eqs. 17-20
# ---------------------------------------------------------------------------------------------
def velocity(f, phi, K, nu, rho0, forchheimer, ax, ay):
    """Eqs. 18-19: u = v / (l0 + sqrt(l0^2 + l1 |v|)), the explicit solution of Eq. 17 with F of Eq. 3."""
    sum_ex_f = np.einsum("i,i...->...", E[:, 0].astype(np.float64), f)
    sum_ey_f = np.einsum("i,i...->...", E[:, 1].astype(np.float64), f)
    vx = sum_ex_f / rho0 + 0.5 * phi * ax
    vy = sum_ey_f / rho0 + 0.5 * phi * ay
    F_phi = ergun_F(phi) if forchheimer else 0.0 * phi
    l0 = 0.5 * (1.0 + phi * 0.5 * nu / K)
    l1 = phi * 0.5 * F_phi / np.sqrt(K)
    denom = l0 + np.sqrt(l0 * l0 + l1 * _norm2(vx, vy))
    return vx / denom, vy / denom


def pressure(f, ux, uy, phi, rho0):
    """Eq. 20: p = c_s^2 / (phi (1 - omega0)) [sum_i f_i + rho0 s0(u)], s0(u) = omega0 (-1.5 |u|^2 / phi)."""
    s0 = W0 * (-1.5 * (ux * ux + uy * uy) / phi)
    return C_S2 / (phi * (1.0 - W0)) * (f.sum(axis=0) + rho0 * s0)


def body_force(ux, uy, phi, K, nu, forchheimer, ax, ay):
    """Total body force, Eq. 3: F = -(phi nu / K) u - (phi F_phi / sqrt K) |u| u + phi a."""
    F_phi = ergun_F(phi) if forchheimer else 0.0 * phi
    umag = _norm2(ux, uy)
    Fx = -phi * nu / K * ux - phi * F_phi / np.sqrt(K) * umag * ux + phi * ax
    Fy = -phi * nu / K * uy - phi * F_phi / np.sqrt(K) * umag * uy + phi * ay
    return Fx, Fy


def equilibrium_moments(p, ux, uy, phi, rho0):
    """Eqs. 11-12 with alpha2 = -1, c1 = c2 = -2, gamma2 = 0, gamma1 = gamma3 = 2/3."""
    usq = ux * ux + uy * uy
    return np.stack(
        [
            5.0 / 3.0 * phi * p + 2.0 / 3.0 * rho0 * usq / phi,
            ALPHA2 * phi * p + 0.75 * GAMMA2 * rho0 * usq / phi,
            rho0 * ux,
            0.5 * C1 * rho0 * ux,
            rho0 * uy,
            0.5 * C2 * rho0 * uy,
            1.5 * GAMMA1 * rho0 * (ux * ux - uy * uy) / phi,
            1.5 * GAMMA3 * rho0 * ux * uy / phi,
        ]
    )


def forcing_moments(ux, uy, Fx, Fy, phi, rho0):
    """Moment-space forcing term S, Eq. 16."""
    zero = 0.0 * ux
    return rho0 * np.stack(
        [
            zero,
            4.0 * (ux * Fx + uy * Fy) / (5.0 * phi),
            Fx,
            -Fx,
            Fy,
            -Fy,
            2.0 * (ux * Fx - uy * Fy) / phi,
            (ux * Fy + uy * Fx) / phi,
        ]
    )


def equilibrium(p, ux, uy, phi, rho0=1.0):
    """Equilibrium populations f_eq = M^-1 m_eq (Eqs. 8, 11)."""
    return np.einsum("ik,k...->i...", M_INV, equilibrium_moments(p, ux, uy, phi, rho0))


def macroscopic(f, flow: Flow, phi=None, K=None, ax=None, ay=None):
    """(ux, uy, p) of pre-collision populations f (Eqs. 17-20)."""
    phi = flow.phi if phi is None else phi
    K = flow.K if K is None else K
    if ax is None:
        ax, ay = _accel(flow, f[0])
    ux, uy = velocity(f, phi, K, flow.nu, flow.rho0, flow.forchheimer, ax, ay)
    return ux, uy, pressure(f, ux, uy, phi, flow.rho0)


# ---------------------------------------------------------------------------------------------
# Collision, Eq. 14 (moment space), and back-transform, Eq. 15
# ---------------------------------------------------------------------------------------------
def collide(f, flow: Flow, phi=None, K=None, ax=None, ay=None):
    """Post-collision populations f+ = M^-1 [m - Lambda (m - m_eq) + (I - Lambda/2) S].

    Returns (f_plus, ux, uy, p).  phi, K, ax, ay default to the flow's fields; the adjoint passes
    perturbed copies.
    """
    phi = flow.phi if phi is None else phi
    K = flow.K if K is None else K
    if ax is None:
        ax, ay = _accel(flow, f[0])
    rho0 = flow.rho0
    m = np.einsum("ki,i...->k...", M, f)
    ux, uy = velocity(f, phi, K, flow.nu, rho0, flow.forchheimer, ax, ay)
    p = pressure(f, ux, uy, phi, rho0)
    Fx, Fy = body_force(ux, uy, phi, K, flow.nu, flow.forchheimer, ax, ay)
    m_eq = equilibrium_moments(p, ux, uy, phi, rho0)
    S = forcing_moments(ux, uy, Fx, Fy, phi, rho0)
    lam = flow.relaxation()
    if lam.ndim == 1:
        lam = lam.reshape((8,) + (1,) * (f.ndim - 1))
    m_plus = m - lam * (m - m_eq) + (1.0 - lam / 2.0) * S
    return np.einsum("ik,k...->i...", M_INV, m_plus), ux, uy, p


# ---------------------------------------------------------------------------------------------
# Streaming, Eq. 15, with the wall rules
# ---------------------------------------------------------------------------------------------
def _wall_velocity(flow: Flow, tx, ty):
    """Velocity of the wall crossed by a link that ends at (tx, ty) outside the lattice.

    The bottom/top wall owns links that leave through y (corners included); otherwise the
    left/right wall.
    """
    uw = np.zeros(tx.shape + (2,))
    side = [
        (ty < 0, flow.u_bottom),
        (ty >= flow.ny, flow.u_top),
    ]
    xside = [(tx < 0, flow.u_left), (tx >= flow.nx, flow.u_right)]
    in_y = (ty >= 0) & (ty < flow.ny)
    for mask, u in xside:
        uw[mask & in_y] = u
    for mask, u in side:
        uw[mask] = u
    return uw


def stream(f_plus, flow: Flow):
    """f_i(x + e_i, t+1) = f_i+(x, t) (Eq. 15); a link that leaves the fluid bounces back halfway:
    f_opp(i)(x, t+1) = f_i+(x, t) - 2 omega_i rho0 (e_i . u_w) / c_s^2.

    'pressure' and 'nee' sides stream periodically here; ``pressure_columns`` and ``wall_nodes``
    then overwrite their boundary nodes.
    """
    ny, nx = flow.ny, flow.nx
    ys, xs = np.mgrid[0:ny, 0:nx]
    out = np.zeros_like(f_plus)
    for i in range(8):
        tx = xs + E[i, 0]
        ty = ys + E[i, 1]
        if flow.bc_x in ("periodic", "pressure", "nee"):
            tx = tx % nx
        if flow.bc_y in ("periodic", "nee"):
            ty = ty % ny
        inside = (tx >= 0) & (tx < nx) & (ty >= 0) & (ty < ny)
        out[i, ty[inside], tx[inside]] = f_plus[i, ys[inside], xs[inside]]
        leave = ~inside
        if leave.any():
            uw = _wall_velocity(flow, tx[leave], ty[leave])
            e_dot_uw = E[i, 0] * uw[:, 0] + E[i, 1] * uw[:, 1]
            out[OPP[i], ys[leave], xs[leave]] = (
                f_plus[i, ys[leave], xs[leave]] - 2.0 * W[i] * flow.rho0 * e_dot_uw / C_S2
            )
    return out


def pressure_columns(f, flow: Flow, phi=None, K=None):
    """Non-equilibrium extrapolation for the pressure inlet (x = 0, p_in) and outlet (x = nx-1, p_out).

    f_b = f_eq(p_b, u_nb; phi_b) + [f_nb - f_eq(p_nb, u_nb; phi_nb)], f_eq = M^-1 m_eq (Eq. 11),
    u_nb and p_nb from Eqs. 17-20 at the adjacent interior column.  Returns a new array.
    """
    phi = flow.phi if phi is None else phi
    K = flow.K if K is None else K
    ax, ay = _accel(flow, f[0])
    out = f.astype(np.result_type(f, phi, K), copy=True)
    for xb, xn, pb in ((0, 1, flow.p_in), (flow.nx - 1, flow.nx - 2, flow.p_out)):
        fn = f[:, :, xn]
        ux, uy = velocity(fn, phi[:, xn], K[:, xn], flow.nu, flow.rho0, flow.forchheimer, ax[:, xn], ay[:, xn])
        pn = pressure(fn, ux, uy, phi[:, xn], flow.rho0)
        out[:, :, xb] = (
            equilibrium(pb + 0.0 * pn, ux, uy, phi[:, xb], flow.rho0)
            + fn
            - equilibrium(pn, ux, uy, phi[:, xn], flow.rho0)
        )
    return out


def wall_node_list(flow: Flow):
    """Wall nodes of the 'nee' sides as index arrays (y, x, y_nb, x_nb, side), side 0..3 =
    left, right, bottom, top; bottom/top walls own the corners, whose nb is the diagonal node
    when the x sides are not periodic."""
    ny, nx = flow.ny, flow.nx
    nodes = []
    if flow.bc_x == "nee":
        for y in range(ny):
            if flow.bc_y == "nee" and y in (0, ny - 1):
                continue
            nodes.append((y, 0, y, 1, 0))
            nodes.append((y, nx - 1, y, nx - 2, 1))
    if flow.bc_y == "nee":
        for x in range(nx):
            xn = x
            if flow.bc_x != "periodic" and x in (0, nx - 1):
                xn = 1 if x == 0 else nx - 2
            nodes.append((0, x, 1, xn, 2))
            nodes.append((ny - 1, x, ny - 2, xn, 3))
    return tuple(np.array([n[k] for n in nodes], dtype=np.int64) for k in range(5))


def wall_nodes(f, flow: Flow, phi=None, K=None):
    """Non-equilibrium extrapolation on the wall nodes of 'nee' sides (Sec. 3's wall treatment).

    f_b = f_eq(p_nb, u_w; phi_b) + [f_nb - f_eq(p_nb, u_nb; phi_nb)] with u_nb, p_nb from Eqs. 17-20
    at nb, the node one step inward along the wall normal; bottom/top walls own the corners, whose
    nb is the diagonal node when the x sides are not periodic.  Returns a new array.
    """
    phi = flow.phi if phi is None else phi
    K = flow.K if K is None else K
    ax, ay = _accel(flow, f[0])
    out = f.astype(np.result_type(f, phi, K), copy=True)
    yb, xb, yn, xn, side = wall_node_list(flow)
    if yb.size == 0:
        return out
    uw = np.array([flow.u_left, flow.u_right, flow.u_bottom, flow.u_top], dtype=np.float64)[side]
    fn = f[:, yn, xn]
    ux, uy = velocity(fn, phi[yn, xn], K[yn, xn], flow.nu, flow.rho0, flow.forchheimer, ax[yn, xn], ay[yn, xn])
    pn = pressure(fn, ux, uy, phi[yn, xn], flow.rho0)
    out[:, yb, xb] = (
        equilibrium(pn, uw[:, 0], uw[:, 1], phi[yb, xb], flow.rho0)
        + fn
        - equilibrium(pn, ux, uy, phi[yn, xn], flow.rho0)
    )
    return out


def boundary_nodes(f, flow: Flow):
    """The extrapolated boundary nodes after streaming: pressure columns, then wall nodes."""
    if flow.bc_x == "pressure":
        f = pressure_columns(f, flow)
    if "nee" in (flow.bc_x, flow.bc_y):
        f = wall_nodes(f, flow)
    return f


# ---------------------------------------------------------------------------------------------
# Time stepping
# ---------------------------------------------------------------------------------------------
def initial_state(flow: Flow, p0=1.0, u0=(0.0, 0.0)):
    """Moments at equilibrium with u = u0 and p = p0 (the initial condition of Sec. 3.1).

    p0 may be a scalar or an (ny, nx) field; p0 = c / phi gives a uniform phi p, the rest state
    of a medium whose porosity varies (the pressure term of Eq. 2 is grad(phi p))."""
    ux = np.full((flow.ny, flow.nx), float(u0[0]))
    uy = np.full((flow.ny, flow.nx), float(u0[1]))
    p = np.broadcast_to(np.asarray(p0, dtype=np.float64), (flow.ny, flow.nx))
    f = equilibrium(p, ux, uy, flow.phi, flow.rho0)
    # the initial state, like every later one, satisfies the boundary-node rules
    return boundary_nodes(f, flow)


def step(f, flow: Flow):
    """One time step of Eq. 6: collide (Eq. 14) then stream (Eq. 15), then the boundary nodes."""
    f_plus = collide(f, flow)[0]
    return boundary_nodes(stream(f_plus, flow), flow)


def run(f, flow: Flow, steps: int):
    for _ in range(steps):
        f = step(f, flow)
    return f


def residual(ux_new, uy_new, ux_old, uy_old):
    """Relative velocity change ||u^t - u^(t-1)||_2 / ||u^t||_2 over all cells."""
    num = np.sum((ux_new - ux_old) ** 2 + (uy_new - uy_old) ** 2)
    den = np.sum(ux_new**2 + uy_new**2)
    return float(np.sqrt(num / den)) if den > 0 else 0.0
