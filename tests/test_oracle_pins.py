"""Pins of the FP64 oracle's flow step against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: printed matrices (Eq. A.4),
closed forms (Eq. 22, Eqs. 23-24 and their Couette variant), exact invariants of Eq. 14, the
BGK and free-fluid reductions stated after Eq. 22, and brute force by an independently written
scalar evaluator of Eq. 6 (tests/literal_eq6.py).
"""
from fractions import Fraction
import os

import numpy as np
import pytest

from oracle import mrt_d2q8 as fl
from tests import literal_eq6 as lit

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
rng = np.random.default_rng(20131128)


def _uniform_flow(nx, ny, phi, K, nu, **kw):
    return fl.Flow(nx=nx, ny=ny, phi=np.full((ny, nx), phi), K=np.full((ny, nx), K), nu=nu, **kw)


def _random_state(flow, amp=0.05):
    """Equilibrium at random p, u plus a random non-equilibrium part."""
    ny, nx = flow.ny, flow.nx
    p = 1.0 + 0.1 * rng.standard_normal((ny, nx))
    ux = 0.05 * rng.standard_normal((ny, nx))
    uy = 0.05 * rng.standard_normal((ny, nx))
    f = fl.equilibrium(p, ux, uy, flow.phi)
    return f + amp * 0.1 * rng.standard_normal(f.shape)


# --------------------------------------------------------------------------- lattice / matrices
def test_velocities_follow_eq7():
    assert [tuple(e) for e in fl.E] == lit.EV
    for i in range(8):
        assert tuple(fl.E[fl.OPP[i]]) == (-fl.E[i][0], -fl.E[i][1])


def test_M_rows_orthogonal_with_expected_norms():
    G = fl.M @ fl.M.T
    assert np.array_equal(G, np.diag([8.0, 8, 6, 12, 6, 12, 4, 4]))
    assert np.allclose(fl.M @ fl.M_INV, np.eye(8), atol=1e-15, rtol=0)


def test_M_is_the_moment_polynomials_of_eq9_and_inverse_is_exact():
    assert np.array_equal(fl.M, np.array(lit.MF))
    exact = np.array([[float(v) for v in r] for r in lit.MINV])
    assert np.allclose(fl.M_INV, exact, atol=1e-16, rtol=0)


def _read_A4():
    rows = []
    with open(os.path.join(GOLDEN, "eqA4_Cx_Cy.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#") or line.startswith("C_"):
                continue
            rows.append([float(Fraction(t)) for t in line.split()])
    A = np.array(rows)
    return A[:8], A[8:]


def test_Cx_Cy_match_printed_eqA4():
    Cx, Cy = _read_A4()
    assert np.allclose(fl.M @ np.diag(fl.E[:, 0].astype(float)) @ fl.M_INV, Cx, atol=1e-15, rtol=0)
    assert np.allclose(fl.M @ np.diag(fl.E[:, 1].astype(float)) @ fl.M_INV, Cy, atol=1e-15, rtol=0)


# --------------------------------------------------------------------------- equilibrium, Eq. 22
def test_equilibrium_moments_equal_eq22_distribution():
    n = 200
    p = 1 + 0.3 * rng.standard_normal(n)
    ux, uy = 0.1 * rng.standard_normal((2, n))
    phi = rng.uniform(0.1, 1.0, n)
    rho0 = 1.0
    cs2 = 1.0 / 3.0
    feq22 = np.empty((8, n))
    for i, (ex, ey) in enumerate(lit.EV):
        eu = ex * ux + ey * uy
        w = float(lit.WEIGHTS[i])
        feq22[i] = rho0 * w * (phi * p / (rho0 * cs2) + eu / cs2 + eu**2 / (2 * phi * cs2**2) - (ux**2 + uy**2) / (2 * phi * cs2))
    assert np.allclose(fl.equilibrium(p, ux, uy, phi, rho0), feq22, atol=1e-15, rtol=1e-14)


# --------------------------------------------------------------------------- collision invariants
def _het_flow(nx=6, ny=5, forch=True, accel=True):
    phi = rng.uniform(0.2, 0.9, (ny, nx))
    K = np.exp(rng.uniform(np.log(1e-2), np.log(10.0), (ny, nx)))
    a = np.stack([1e-3 * rng.standard_normal((ny, nx)), 1e-3 * rng.standard_normal((ny, nx))]) if accel else np.zeros(2)
    return fl.Flow(nx=nx, ny=ny, phi=phi, K=K, nu=0.07, forchheimer=forch, accel=a)


def test_collision_conserves_mass_and_adds_force_to_momentum():
    flow = _het_flow()
    f = _random_state(flow)
    fp, ux, uy, p = fl.collide(f, flow)
    assert np.allclose(fp.sum(0), f.sum(0), atol=1e-15, rtol=1e-14)
    Fx, Fy = fl.body_force(ux, uy, flow.phi, flow.K, flow.nu, True, flow.accel[0], flow.accel[1])
    ex, ey = fl.E[:, 0].astype(float), fl.E[:, 1].astype(float)
    jx0, jy0 = np.einsum("i,iyx->yx", ex, f), np.einsum("i,iyx->yx", ey, f)
    jx1, jy1 = np.einsum("i,iyx->yx", ex, fp), np.einsum("i,iyx->yx", ey, fp)
    assert np.allclose(jx1, jx0 + flow.rho0 * Fx, atol=1e-15, rtol=1e-12)
    assert np.allclose(jy1, jy0 + flow.rho0 * Fy, atol=1e-15, rtol=1e-12)
    assert np.abs(Fx).max() > 1e-5  # the check is not vacuous


def test_conserved_moment_rates_do_not_change_the_result():
    flow = _het_flow()
    f = _random_state(flow)
    base = fl.collide(f, flow)[0]
    lam = flow.relaxation().copy()
    lam[[0, 2, 4]] = [0.3, 1.7, 0.6]
    flow.rates = lam
    other = fl.collide(f, flow)[0]
    assert np.allclose(base, other, atol=1e-15, rtol=1e-13)


def test_explicit_velocity_solves_implicit_eq17():
    flow = _het_flow()
    f = _random_state(flow, amp=0.5)
    ux, uy, _ = fl.macroscopic(f, flow)
    Fx, Fy = fl.body_force(ux, uy, flow.phi, flow.K, flow.nu, True, flow.accel[0], flow.accel[1])
    jx = np.einsum("i,iyx->yx", fl.E[:, 0].astype(float), f)
    jy = np.einsum("i,iyx->yx", fl.E[:, 1].astype(float), f)
    assert np.allclose(flow.rho0 * ux, jx + 0.5 * flow.rho0 * Fx, atol=1e-16, rtol=1e-13)
    assert np.allclose(flow.rho0 * uy, jy + 0.5 * flow.rho0 * Fy, atol=1e-16, rtol=1e-13)


def test_single_rate_reduces_to_bgk_with_eq22():
    """Lambda = I/tau, no drag and no force: f+ = f - (f - f_eq^(22)) / tau (statement after Eq. 21)."""
    tau = 0.83
    flow = _uniform_flow(5, 4, 0.7, 1e300, 0.1, forchheimer=False, rates=np.full(8, 1 / tau))
    f = _random_state(flow)
    fp = fl.collide(f, flow)[0]
    ex, ey = fl.E[:, 0].astype(float), fl.E[:, 1].astype(float)
    ux = np.einsum("i,iyx->yx", ex, f)
    uy = np.einsum("i,iyx->yx", ey, f)
    phi = flow.phi
    # Eq. 20 with the s0 reading, then Eq. 22
    p = 3.0 / (5.0 * phi) * (f.sum(0) - 2.0 / 3.0 * (ux**2 + uy**2) / phi)
    feq = np.empty_like(f)
    for i in range(8):
        eu = ex[i] * ux + ey[i] * uy
        w = float(lit.WEIGHTS[i])
        feq[i] = w * (3 * phi * p + 3 * eu + 4.5 * eu**2 / phi - 1.5 * (ux**2 + uy**2) / phi)
    assert np.allclose(fp, f - (f - feq) / tau, atol=1e-15, rtol=1e-13)


# --------------------------------------------------------------------------- brute force, Eq. 6
@pytest.mark.parametrize(
    "bc_x,bc_y,walls",
    [
        ("periodic", "periodic", None),
        ("periodic", "wall", {"bottom": (0.0, 0.0), "top": (0.08, 0.0), "left": (0, 0), "right": (0, 0)}),
        ("wall", "wall", {"bottom": (0.0, 0.01), "top": (0.1, 0.0), "left": (0.0, 0.02), "right": (0.0, -0.03)}),
        ("wall", "periodic", {"bottom": (0, 0), "top": (0, 0), "left": (0.0, 0.05), "right": (0.0, 0.0)}),
    ],
)
def test_brute_force_8x8_matches_literal_eq6(bc_x, bc_y, walls):
    nx = ny = 8
    walls = walls or {"bottom": (0, 0), "top": (0, 0), "left": (0, 0), "right": (0, 0)}
    flow = _het_flow(nx, ny)
    flow.bc_x, flow.bc_y = bc_x, bc_y
    flow.u_bottom, flow.u_top, flow.u_left, flow.u_right = walls["bottom"], walls["top"], walls["left"], walls["right"]
    f = _random_state(flow)
    fo = f.copy()
    fl_nested = [[list(f[:, y, x]) for x in range(nx)] for y in range(ny)]
    rates = list(flow.relaxation())
    for _ in range(3):
        fo = fl.step(fo, flow)
        fl_nested = lit.step(
            fl_nested, nx, ny, flow.phi, flow.K, flow.nu, flow.accel[0], flow.accel[1], rates, True, bc_x, bc_y, walls
        )
    ref = np.array(fl_nested).transpose(2, 0, 1)
    assert np.allclose(fo, ref, atol=1e-14, rtol=1e-12)


# --------------------------------------------------------------------------- analytic flows
def _steady(flow, f, max_steps, tol=1e-13, every=200):
    prev = fl.macroscopic(f, flow)[0]
    for k in range(0, max_steps, every):
        f = fl.run(f, flow, every)
        ux = fl.macroscopic(f, flow)[0]
        if np.abs(ux - prev).max() <= tol * np.abs(ux).max():
            break
        prev = ux
    return f


def test_free_fluid_poiseuille_is_exact_parabola_at_magic_rates():
    """phi -> 1, K -> inf, F_phi = 0: the incompressible MRT limit (statement after Eq. 22).
    With (1/s_v - 1/2)(1/s_q - 1/2) = 3/16, halfway bounce-back places the wall exactly, so the
    discrete steady state is the parabola u = G y'(H - y') / (2 nu) to rounding."""
    H, nu, G = 12, 0.2, 1e-5
    tau = 3 * nu + 0.5
    s_q = 1.0 / (0.5 + (3.0 / 16.0) / (tau - 0.5))
    flow = _uniform_flow(2, H, 1.0, 1e300, nu, forchheimer=False, accel=np.array([G, 0.0]), s_q=s_q)
    f = _steady(flow, fl.initial_state(flow), 20000)
    ux, uy, _ = fl.macroscopic(f, flow)
    y = np.arange(H) + 0.5
    exact = G * y * (H - y) / (2 * nu)
    assert np.abs(ux[:, 0] - exact).max() < 1e-10 * exact.max()
    assert np.abs(uy).max() < 1e-14


def _brinkman_poiseuille(y, H, G, phi, K, nu, J=1.0):
    """Eq. 23 with F_phi = 0 solved in closed form (the cosh profile behind Eq. 24), y = distance from the wall."""
    th = np.sqrt(phi * nu / (K * J * nu))
    return G * K / nu * (1 - np.cosh(th * (y - H / 2)) / np.cosh(th * H / 2))


def test_porous_poiseuille_brinkman_cosh_profile():
    """phi = 0.1, Da = 0.01, F_phi = 0 (Sec. 3.1 setup with halfway walls): Eq. 24's profile."""
    H, phi, nu = 32, 0.1, 0.3
    K = 0.01 * H * H
    Re = 1.0
    th = np.sqrt(phi / K)
    u0 = Re * nu / H
    G = u0 * nu / (K * (1 - 1 / np.cosh(th * H / 2)))  # Eq. 24 solved for a_x
    flow = _uniform_flow(2, H, phi, K, nu, forchheimer=False, accel=np.array([G, 0.0]))
    f = _steady(flow, fl.initial_state(flow), 40000, tol=1e-11)
    ux = fl.macroscopic(f, flow)[0][:, 0]
    y = np.arange(H) + 0.5
    exact = _brinkman_poiseuille(y, H, G, phi, K, nu)
    assert abs(exact.max() - u0) < 1e-3 * u0  # Eq. 24 gives the centre-line speed
    err = np.abs(ux - exact).max() / exact.max()
    assert err < 2e-3, err


def test_porous_poiseuille_with_ergun_drag_matches_bvp():
    """Eq. 23 including the Forchheimer term, solved by a 1-D boundary-value solver."""
    from scipy.integrate import solve_bvp

    H, phi, nu = 24, 0.4, 0.2
    K = 0.01 * H * H
    G = 3e-3
    Fphi = 1.75 / np.sqrt(150 * phi**3)
    flow = _uniform_flow(2, H, phi, K, nu, forchheimer=True, accel=np.array([G, 0.0]))
    f = _steady(flow, fl.initial_state(flow), 40000, tol=1e-11)
    ux = fl.macroscopic(f, flow)[0][:, 0]

    def rhs(y, s):  # (nu_e/phi) u'' = nu/K u + F/sqrt(K) u^2 - a
        return np.vstack([s[1], phi / nu * (nu / K * s[0] + Fphi / np.sqrt(K) * s[0] ** 2 - G)])

    ys = np.linspace(0, H, 401)
    sol = solve_bvp(rhs, lambda a, b: np.array([a[0], b[0]]), ys, np.zeros((2, ys.size)), tol=1e-10, max_nodes=100000)
    assert sol.success
    exact = sol.sol(np.arange(H) + 0.5)[0]
    # the nonlinear term matters here: the Brinkman-only profile differs by much more
    brink = _brinkman_poiseuille(np.arange(H) + 0.5, H, G, phi, K, nu)
    assert np.abs(brink - exact).max() > 0.05 * exact.max()
    assert np.abs(ux - exact).max() < 3e-3 * exact.max()


def test_porous_couette_sinh_profile_pins_moving_wall():
    """Couette flow (Sec. 3.2): a = 0, top wall at u0, F_phi = 0: u = u0 sinh(th y)/sinh(th H)."""
    H, phi, nu, u0 = 24, 0.1, 0.25, 0.01
    K = 0.01 * H * H
    flow = _uniform_flow(2, H, phi, K, nu, forchheimer=False, u_top=(u0, 0.0))
    f = _steady(flow, fl.initial_state(flow), 40000, tol=1e-11)
    ux = fl.macroscopic(f, flow)[0][:, 0]
    th = np.sqrt(phi / K)
    y = np.arange(H) + 0.5
    exact = u0 * np.sinh(th * y) / np.sinh(th * H)
    assert np.abs(ux - exact).max() < 2e-3 * u0


def test_partially_porous_couette_heterogeneous_phi():
    """Sec. 3.2 partially filled channel at J = 1, F_phi = 0: lower half phi = 0.1 (porous), upper
    half phi = 1 with K -> inf.  With u, u' continuous at y = H/2 (uniform upsilon_e), the porous
    part is d0 sinh(th y)/sinh(th H/2) and the free part the line d0 + s (y - H/2), s = d0 th coth(th H/2)."""
    H, nu, u0 = 32, 0.16, 0.01
    K = 1e-3 * H * H
    phi = np.where(np.arange(H)[:, None] < H // 2, 0.1, 1.0) * np.ones((H, 2))
    Kf = np.where(np.arange(H)[:, None] < H // 2, K, 1e30) * np.ones((H, 2))
    flow = fl.Flow(nx=2, ny=H, phi=phi, K=Kf, nu=nu, forchheimer=False, u_top=(u0, 0.0))
    # start from the rest state phi p = 1 (uniform p over a porosity jump is not a rest state)
    f = _steady(flow, fl.initial_state(flow, p0=1.0 / phi), 60000, tol=1e-11)
    ux = fl.macroscopic(f, flow)[0][:, 0]
    th = np.sqrt(0.1 / K)
    d0 = u0 / (1 + th * (H / 2) / np.tanh(th * H / 2))
    s = d0 * th / np.tanh(th * H / 2)
    y = np.arange(H) + 0.5
    exact = np.where(y < H / 2, d0 * np.sinh(th * y) / np.sinh(th * H / 2), d0 + s * (y - H / 2))
    assert np.abs(ux - exact).max() < 1e-2 * u0


def test_pressure_driven_channel_with_nee_columns():
    """Pressure inlet/outlet by non-equilibrium extrapolation: in a uniform porous channel the
    steady flow equals the body-force case with phi a_x = -d(phi p)/dx, i.e. a_x = (p_in - p_out)/(nx - 1)."""
    nx, H, phi, nu = 16, 16, 0.5, 0.2
    K = 0.01 * H * H
    dp = 2e-3
    flow = _uniform_flow(nx, H, phi, K, nu, forchheimer=False, bc_x="pressure", p_in=1.0 + dp / 2, p_out=1.0 - dp / 2)
    f = _steady(flow, fl.initial_state(flow), 40000, tol=1e-11)
    ux, uy, p = fl.macroscopic(f, flow)
    G = dp / (nx - 1)
    exact = _brinkman_poiseuille(np.arange(H) + 0.5, H, G, phi, K, nu)
    mid = ux[:, nx // 2]
    assert np.abs(mid - exact).max() < 1e-2 * exact.max()
    # pressure falls linearly between the two prescribed columns
    pc = p[H // 2]
    assert abs(pc[0] - flow.p_in) < 1e-4 * dp + 1e-12
    assert np.allclose(np.diff(pc), -G, rtol=2e-2)


@pytest.mark.parametrize("J", [1.0, 4.0])
def test_partially_porous_couette_with_viscosity_ratio(J):
    """Sec. 3.2 with J = upsilon_e / upsilon in the porous half (s_v per region, J = 1 in the free
    half), F_phi = 0.  From Eq. 23 and continuity of u and of the shear stress upsilon_e u' at
    y = H/2: porous part d0 sinh(th y)/sinh(th H/2), th = sqrt(phi/(K J)); free part
    d0 + s (y - H/2) with s = J d0 th coth(th H/2), and u(H) = u0."""
    H, nu, u0 = 32, 0.16, 0.01
    K = 1e-3 * H * H
    lower = np.arange(H)[:, None] < H // 2
    phi = np.where(lower, 0.1, 1.0) * np.ones((H, 2))
    Kf = np.where(lower, K, 1e30) * np.ones((H, 2))
    Jf = np.where(lower, J, 1.0) * np.ones((H, 2))
    flow = fl.Flow(nx=2, ny=H, phi=phi, K=Kf, nu=nu, J=Jf, forchheimer=False, u_top=(u0, 0.0))
    f = _steady(flow, fl.initial_state(flow, p0=1.0 / phi), 80000, tol=1e-11)
    ux = fl.macroscopic(f, flow)[0][:, 0]
    th = np.sqrt(0.1 / (K * J))
    d0 = u0 / (1 + J * th * (H / 2) / np.tanh(th * H / 2))
    s = J * d0 * th / np.tanh(th * H / 2)
    y = np.arange(H) + 0.5
    exact = np.where(y < H / 2, d0 * np.sinh(th * y) / np.sinh(th * H / 2), d0 + s * (y - H / 2))
    assert np.abs(ux - exact).max() < 1.5e-2 * u0, np.abs(ux - exact).max() / u0


# ---------------------------------------------------------------------------------------------
# Wall nodes with non-equilibrium extrapolation (the paper's own wall treatment, Sec. 3): walls on
# the outermost nodes, channel height H = ny - 1.  The scheme is second-order accurate, so the
# error against the closed forms of Eq. 23 falls ~4x when the grid is refined 2x.
# ---------------------------------------------------------------------------------------------
def _nee_poiseuille_error(N, phi=0.1, nu=0.3):
    H = N - 1
    K = 0.01 * H * H
    th = np.sqrt(phi / K)
    u0 = nu / H  # Re = 1
    G = u0 * nu / (K * (1 - 1 / np.cosh(th * H / 2)))  # Eq. 24 solved for a_x
    flow = _uniform_flow(2, N, phi, K, nu, forchheimer=False, accel=np.array([G, 0.0]), bc_y="nee")
    f = _steady(flow, fl.initial_state(flow), 40000, tol=1e-12)
    ux = fl.macroscopic(f, flow)[0][:, 0]
    exact = _brinkman_poiseuille(np.arange(N, dtype=np.float64), H, G, phi, K, nu)
    return np.abs(ux - exact).max() / exact.max()


def test_nee_walls_porous_poiseuille_second_order():
    e17, e33 = _nee_poiseuille_error(17), _nee_poiseuille_error(33)
    assert e33 < 7e-3, e33
    assert e17 / e33 > 3.3, (e17, e33)


def test_nee_walls_porous_couette_moving_node():
    """Top wall node moving at u0, a = 0, F_phi = 0: u = u0 sinh(th y) / sinh(th H) with y the
    distance from the bottom wall node; the moving node itself carries u0."""
    N, phi, nu, u0 = 25, 0.1, 0.25, 0.01
    H = N - 1
    K = 0.01 * H * H
    th = np.sqrt(phi / K)
    flow = _uniform_flow(2, N, phi, K, nu, forchheimer=False, bc_y="nee", u_top=(u0, 0.0))
    f = _steady(flow, fl.initial_state(flow), 40000, tol=1e-12)
    ux, uy = fl.macroscopic(f, flow)[:2]
    exact = u0 * np.sinh(th * np.arange(N)) / np.sinh(th * H)
    assert np.abs(ux[:, 0] - exact).max() < 5e-3 * u0
    assert abs(ux[-1, 0] - u0) < 1e-3 * u0
    assert np.abs(uy).max() < 1e-4 * u0  # extrapolated walls do not conserve mass exactly


def test_nee_wall_node_is_equilibrium_at_wall_velocity_for_equilibrium_neighbour():
    """If the inner neighbour is at equilibrium, the extrapolated wall node is the equilibrium at
    the neighbour's pressure and the wall's velocity (the non-equilibrium part vanishes).  K -> inf
    and F_phi = 0, so that Eqs. 18-20 recover the neighbour's (p, u) exactly."""
    flow = _uniform_flow(5, 4, 0.6, 1e30, 0.1, forchheimer=False, bc_x="nee", bc_y="nee", u_top=(0.07, 0.0),
                         u_left=(0.0, 0.02))
    p = 1.0 + 0.02 * rng.standard_normal((4, 5))
    ux, uy = 0.03 * rng.standard_normal((2, 4, 5))
    f = fl.equilibrium(p, ux, uy, flow.phi)
    g = fl.wall_nodes(f, flow)
    # top node (x = 2, y = 3) from (2, 2); left node (0, 1) from (1, 1); corner (0, 3) from (1, 2)
    for (y, x), (yn, xn), uw in (((3, 2), (2, 2), (0.07, 0.0)), ((1, 0), (1, 1), (0.0, 0.02)), ((3, 0), (2, 1), (0.07, 0.0))):
        want = fl.equilibrium(p[yn, xn], uw[0], uw[1], 0.6)
        assert np.allclose(g[:, y, x], want, atol=1e-13), (y, x)
    # interior untouched
    assert np.array_equal(g[:, 1:3, 1:4], f[:, 1:3, 1:4])


def test_residual_hand_example_and_invariants():
    """The steady-state residual ||u(t) - u(t-1)||_2 / ||u(t)||_2 on a two-cell example worked by
    hand: u(t) = ((1, 2), (2, 0)), u(t-1) = ((1, 2), (1, 1)) differ by (0, 0) and (1, -1), so the
    numerator is sqrt(2) and the denominator sqrt(1 + 4 + 4 + 0) = 3."""
    ux_new, uy_new = np.array([1.0, 2.0]), np.array([2.0, 0.0])
    ux_old, uy_old = np.array([1.0, 1.0]), np.array([2.0, 1.0])
    assert abs(fl.residual(ux_new, uy_new, ux_old, uy_old) - np.sqrt(2.0) / 3.0) < 1e-15
    # invariants: zero for an unchanged field, unchanged by a common scale, zero for a zero field
    rng = np.random.default_rng(1)
    a, b, c, d = rng.standard_normal((4, 5, 7))
    assert fl.residual(a, b, a, b) == 0.0
    assert abs(fl.residual(3 * a, 3 * b, 3 * c, 3 * d) - fl.residual(a, b, c, d)) < 1e-14
    assert fl.residual(0 * a, 0 * b, c, d) == 0.0
