"""Parity at the benchmark's full sizes and launch configuration, on sampled outputs.

The 4096^2 lid-driven porous cavity that bench.py times (eps = 0.4, Da = 1e-3, Re = 100, lid 0.1,
halfway walls) starts from a seeded random pre-collision state and advances k = 32 steps through
lbm_step, i.e. one replay of the 32-step CUDA graph that the benchmark replays.  After k steps a
cell depends only on the cells within k of it (one link per step, Eq. 15), so the FP64 oracle
computes each sampled cell on the (2k+1)^2 crop around it: where the crop meets the lattice's walls
they are the real walls; its other edges are k cells from the centre and cannot reach it in k
steps.  The samples cover the four corners (two under the moving lid), the four walls and the
interior.  The in-place streaming form is checked the same way.

The same property checks the 512-lattice ensemble in the launch form its benchmark uses, and the
full-size adjoint (2048 x 1024 channel, T = 4000) is checked through a property that holds at any
size: its gradient's projection on a uniform change of log K (and of eps) equals the central
difference of the loss computed by the forward path.  The porous Poiseuille configuration (64 x 64,
eps = 0.1, Da = 0.01, Re = 10) runs to its steady state as specified (residual below 1e-10 or
20000 steps) against Eq. 24's profile and, with the Ergun drag, a 1-D solve of Eq. 23.
"""
import numpy as np
import pytest

from oracle import mrt_d2q8 as fl
from tests.cases import random_state

pytestmark = pytest.mark.gpu

L = 4096
K_STEPS = 32
LID = 0.1


@pytest.fixture(scope="module")
def lbm():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1311_7239_gb300 import build, lbm

    build.build()
    return lbm


def _samples(nx, ny, n_random, seed):
    pts = [(0, 0), (nx - 1, 0), (0, ny - 1), (nx - 1, ny - 1),  # corners (top two under the lid)
           (nx // 3, 0), (nx // 2, ny - 1), (0, ny // 3), (nx - 1, 2 * ny // 3),  # walls and lid
           (1, ny - 2), (nx - 2, ny - 2), (5, ny - 1), (nx - 6, 1)]  # next to corners
    rng = np.random.default_rng(seed)
    for _ in range(n_random):
        pts.append((int(rng.integers(0, nx)), int(rng.integers(0, ny))))
    return pts


def _crop_flow(x, y, nx, ny, k, phi, K, nu, lid):
    """Oracle set-up of the crop around (x, y): walls on both axes (the real ones where the crop
    reaches the lattice edge, with their velocities), uniform medium."""
    x0, x1 = max(0, x - k), min(nx - 1, x + k)
    y0, y1 = max(0, y - k), min(ny - 1, y + k)
    flow = fl.Flow(nx=x1 - x0 + 1, ny=y1 - y0 + 1, phi=phi, K=K, nu=nu, bc_x="wall", bc_y="wall",
                   u_top=(lid, 0.0) if y1 == ny - 1 else (0.0, 0.0))
    return flow, (x0, x1, y0, y1)


def _sampled_parity(lbm, precision, tol, streaming=0):
    import torch

    nu, phi, K = LID * L / 100.0, 0.4, 1e-3 * L * L
    full = fl.Flow(nx=L, ny=L, phi=phi, K=K, nu=nu, bc_x="wall", bc_y="wall", u_top=(LID, 0.0))
    f0 = random_state(full, seed=2024, amp=0.02, u_amp=0.03).astype(np.float32)
    cfg = lbm.default_config(nx=L, ny=L, bc_x=lbm.WALL, bc_y=lbm.WALL, nu=nu, phi=phi, K=K,
                             u_wall=[(0, 0), (0, 0), (0, 0), (LID, 0)], precision=precision, p_rest=phi, dev_scale_log2=10,
                             streaming=streaming)
    lat = lbm.Lattice(cfg)
    try:
        lat.set_populations(torch.from_numpy(f0).cuda())
        lat.step(K_STEPS)
        got = lat.get_populations().cpu().numpy()
        lat.sync()
    finally:
        lat.close()
    worst = 0.0
    for (x, y) in _samples(L, L, 52, seed=7):
        flow, (x0, x1, y0, y1) = _crop_flow(x, y, L, L, K_STEPS, phi, K, nu, LID)
        f = f0[:, y0:y1 + 1, x0:x1 + 1].astype(np.float64)
        f = fl.run(f, flow, K_STEPS)
        want = f[:, y - y0, x - x0]
        err = float(np.abs(got[:, y, x] - want).max())
        worst = max(worst, err)
        assert err <= tol, ((x, y), err)
    return worst


def test_bench_cavity_4096_fp32_sampled_cells(lbm):
    worst = _sampled_parity(lbm, 0, 2e-5)
    print(f"4096^2 FP32, {K_STEPS} steps: max |df| over 64 sampled cells = {worst:.2e}")


def test_bench_cavity_4096_fp16_sampled_cells(lbm):
    """FP16 deviation storage (the packed two-cell collision): each step rounds the stored deviation
    (|s d| ~ 50 at s = 2^10: a unit of 2^-5 / 2^10 = 3e-5), so the bound is k such units."""
    worst = _sampled_parity(lbm, 1, K_STEPS * 3.1e-5)
    print(f"4096^2 FP16, {K_STEPS} steps: max |df| over 64 sampled cells = {worst:.2e}")


def test_bench_cavity_4096_bf16_sampled_cells(lbm):
    """BF16 deviation storage (unscaled, 8-bit significand): a unit of 2^-8 |d|, |d| <= 0.1."""
    worst = _sampled_parity(lbm, 2, K_STEPS * 4e-4)
    print(f"4096^2 BF16, {K_STEPS} steps: max |df| over 64 sampled cells = {worst:.2e}")


def test_bench_cavity_4096_inplace_fp32_sampled_cells(lbm):
    """The same with in-place streaming (one population buffer, 32 steps: both parities)."""
    worst = _sampled_parity(lbm, 0, 2e-5, streaming=1)
    print(f"4096^2 FP32 in-place, {K_STEPS} steps: max |df| over 64 sampled cells = {worst:.2e}")


def test_bench_cavity_4096_inplace_fp16_sampled_cells(lbm):
    worst = _sampled_parity(lbm, 1, K_STEPS * 3.1e-5, streaming=1)
    print(f"4096^2 FP16 in-place, {K_STEPS} steps: max |df| over 64 sampled cells = {worst:.2e}")


def test_ensemble_512_in_bench_launch_form(lbm):
    """The 512-lattice ensemble of the benchmark, in the launch form its tuner picks (one CTA per
    work item): after 32 steps from the rest state, sampled cells of eight lattices (largest,
    smallest, channels and cavities) match the oracle on crops of their own medium."""
    from paper_1311_7239_gb300 import workloads

    cfgs, media = workloads.ensemble(lbm, n=512, seed=42)
    b = workloads.build(lbm, cfgs, media)
    try:
        b.set_launch(64, 0)
        b.step(K_STEPS)
        b.sync()
        cells = [c.nx * c.ny for c in cfgs]
        kinds = [c.bc_x for c in cfgs]
        pick = {int(np.argmax(cells)), int(np.argmin(cells))}
        pick |= set([d for d in range(len(cfgs)) if kinds[d] == lbm.PERIODIC][:3])
        pick |= set([d for d in range(len(cfgs)) if kinds[d] == lbm.WALL][:3])
        for d in sorted(pick):
            cfg = cfgs[d]
            got = b.get_populations(d).cpu().numpy()
            eps, K = (m.astype(np.float64) for m in media[d])
            nx, ny = cfg.nx, cfg.ny
            periodic = cfg.bc_x == lbm.PERIODIC
            p_rest = float(cfg.p_rest)
            full_init = fl.initial_state(fl.Flow(nx=nx, ny=ny, phi=eps, K=K, nu=cfg.nu), p0=p_rest / eps)
            for (x, y) in _samples(nx, ny, 8, seed=d):
                k = K_STEPS
                x0, x1 = (0, nx - 1) if periodic else (max(0, x - k), min(nx - 1, x + k))
                y0, y1 = max(0, y - k), min(ny - 1, y + k)
                flow = fl.Flow(nx=x1 - x0 + 1, ny=y1 - y0 + 1, phi=eps[y0:y1 + 1, x0:x1 + 1], K=K[y0:y1 + 1, x0:x1 + 1],
                               nu=cfg.nu, accel=np.array([cfg.ax, 0.0]), bc_x="periodic" if periodic else "wall", bc_y="wall",
                               u_top=(cfg.u_wall[3][0], 0.0) if y1 == ny - 1 else (0.0, 0.0))
                f = fl.run(full_init[:, y0:y1 + 1, x0:x1 + 1].copy(), flow, k)
                err = float(np.abs(got[:, y, x] - f[:, y - y0, x - x0]).max())
                assert err <= 2e-5, (d, (x, y), err)
    finally:
        b.close()


def test_adjoint_2048x1024_T4000_directional_derivative(lbm):
    """Full-size adjoint (the benchmark's channel, T = 4000): <dL/dlogK, 1> and <dL/deps, 1> equal
    the central differences of the loss under a uniform shift of log K (h = 1e-2) and of eps
    (h = 1e-4), both computed by the forward path; the bound 2e-3 covers FP32 roundoff of the loss
    over 4000 steps and the O(h^2) truncation.  A uniform eps shift moves phi p of the pressure
    columns against the interior's rest state phi p = mean(eps), and the pressure waves that this
    starts dominate the outlet flux at T = 4000 (dL/d eps ~ 1e3 L), so its step is small."""
    import torch

    from paper_1311_7239_gb300 import workloads

    T = 4000
    cfg, eps, logk = workloads.adjoint_channel(lbm)
    lat = lbm.Lattice(cfg)
    try:
        def loss(e, lk):
            lat.set_medium_log(torch.tensor(e, device="cuda"), torch.tensor(lk, device="cuda"))
            lat.init_equilibrium(float(cfg.p_rest), 0.0, 0.0, phi_p_uniform=True)
            lat.step(T)
            ux = lat.macros()[1]
            return float(ux[:, -1].double().sum())

        lat.set_medium_log(torch.tensor(eps, device="cuda"), torch.tensor(logk, device="cuda"))
        lat.init_equilibrium(float(cfg.p_rest), 0.0, 0.0, phi_p_uniform=True)
        L0, gk, ge = lat.adjoint(T, "flux")
        assert abs(L0 - loss(eps, logk)) <= 1e-6 * abs(L0)
        h = 1e-2
        fd_k = (loss(eps, logk + h) - loss(eps, logk - h)) / (2 * h)
        h = 1e-4
        fd_e = (loss(eps + h, logk) - loss(eps - h, logk)) / (2 * h)
        fd_e2 = (loss(eps + 2 * h, logk) - loss(eps - 2 * h, logk)) / (4 * h)
        ad_k, ad_e = float(gk.sum()), float(ge.sum())
        print(f"adjoint 2048x1024 T={T}: <g_logK,1> {ad_k:.6e} vs FD {fd_k:.6e}; <g_eps,1> {ad_e:.6e} vs FD {fd_e:.6e} "
              f"(FD at 2h: {fd_e2:.6e})")
        assert abs(ad_k - fd_k) <= 2e-3 * abs(fd_k), (ad_k, fd_k)
        assert abs(ad_e - fd_e) <= 2e-3 * abs(fd_e), (ad_e, fd_e)
    finally:
        lat.close()


def _poiseuille_64(lbm, forch):
    """Configuration 1 on the GPU: run until the residual (checked every 100 steps) is below 1e-10
    or 20000 steps; returns (u_x(y) at x = 0, G, K, nu, phi, steps, residual)."""
    H, phi, nu, Re = 64, 0.1, 0.1, 10.0
    K = 0.01 * H * H
    th_ = np.sqrt(phi / K)
    u0 = Re * nu / H
    G = u0 * nu / (K * (1 - 1 / np.cosh(th_ * H / 2)))  # Eq. 24 solved for a_x (F_phi = 0)
    cfg = lbm.default_config(nx=H, ny=H, bc_x=lbm.PERIODIC, bc_y=lbm.WALL, nu=nu, phi=phi, K=K, forchheimer=int(forch), ax=G,
                             p_rest=phi)
    lat = lbm.Lattice(cfg)
    try:
        steps, r = 0, 1.0
        while steps < 20000:
            lat.step(99)
            lat.step(1)
            steps += 100
            r = lat.residual()
            if r < 1e-10:
                break
        ux = lat.macros()[1].cpu().numpy()
    finally:
        lat.close()
    assert np.abs(ux - ux[:, :1]).max() <= 1e-6 * np.abs(ux).max()  # uniform along the channel
    return ux[:, 0].astype(np.float64), G, K, nu, phi, steps, r


def test_config1_poiseuille_steady_state_brinkman_profile(lbm):
    ux, G, K, nu, phi, steps, r = _poiseuille_64(lbm, forch=False)
    H = ux.size
    y = np.arange(H) + 0.5
    th_ = np.sqrt(phi / K)
    exact = G * K / nu * (1 - np.cosh(th_ * (y - H / 2)) / np.cosh(th_ * H / 2))
    err = np.abs(ux - exact).max() / exact.max()
    print(f"config 1 (F_phi = 0): {steps} steps, residual {r:.2e}, max error vs Eq. 24 profile {err:.2e}")
    assert err < 2e-3, err


def test_config1_poiseuille_steady_state_ergun_bvp(lbm):
    from scipy.integrate import solve_bvp

    ux, G, K, nu, phi, steps, r = _poiseuille_64(lbm, forch=True)
    H = ux.size
    Fphi = 1.75 / np.sqrt(150 * phi**3)

    def rhs(y, s):  # (nu_e / phi) u'' = nu / K u + F_phi / sqrt(K) u^2 - a   (Eq. 23)
        return np.vstack([s[1], phi / nu * (nu / K * s[0] + Fphi / np.sqrt(K) * s[0] ** 2 - G)])

    ys = np.linspace(0, H, 801)
    sol = solve_bvp(rhs, lambda a, b: np.array([a[0], b[0]]), ys, np.zeros((2, ys.size)), tol=1e-10, max_nodes=200000)
    assert sol.success
    exact = sol.sol(np.arange(H) + 0.5)[0]
    err = np.abs(ux - exact).max() / exact.max()
    print(f"config 1 (Ergun F_phi = {Fphi:.3f}): {steps} steps, residual {r:.2e}, max error vs Eq. 23 solve {err:.2e}")
    assert err < 3e-3, err
