"""FP64 oracle of the discrete adjoint of the porous D2Q8 MRT-LB flow step: the gradient of a scalar
loss of the final state with respect to the per-cell log-permeability and porosity.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``); shares no code with the CUDA library.

The forward map is the oracle's own step (Eq. 6 as collision Eq. 14 + streaming Eq. 15, then the
boundary nodes), f(t+1) = B(S(C(f(t); theta)); theta), from f(0) = B(f_eq(p0, u0; phi)) (the
initial condition of Sec. 3.1), where B = W o N: N the pressure columns, then W the wall nodes of
the sides with non-equilibrium extrapolation (Sec. 3's wall treatment).  The reverse sweep stores
every state and applies, per step,
  lambda <- J_W^T lambda,  lambda <- J_N^T lambda,  lambda <- S^T lambda,  lambda <- J_C^T lambda,
accumulating dL/dtheta from the theta-dependence of W, N and C and, at the end, of f(0).

Independent route: every Jacobian of a nonlinear per-cell map (the collision C, the pressure
columns N, the wall nodes W, the initial equilibrium, the loss) is taken by the complex-step derivative
Im F(x + i h e_k) / h with h = 1e-30, which is exact to rounding and needs no hand derivation.
Only the streaming map S is linear; its transpose is written out as the reversed link table.
At |v| = 0 the magnitude has no derivative; the oracle's |v| is defined to have zero derivative
there (see ``mrt_d2q8._norm2``), the one-sided limit of the smooth part of Eq. 18.

Losses: 'flux' Q = sum_y u_x(nx-1, y) of the final state (the outlet flux of a channel), and
'misfit' 1/2 sum |u - u*|^2 over all cells.
"""
from __future__ import annotations

import numpy as np

from . import mrt_d2q8 as fl

H = 1e-30


def _theta_fields(flow: fl.Flow, logK=None, phi=None):
    logK = np.log(flow.K) if logK is None else logK
    phi = flow.phi if phi is None else phi
    return logK, phi


def stream_transpose(lam, flow: fl.Flow):
    """Transpose of the linear part of ``mrt_d2q8.stream``: the streaming map sends f+_i(x) to
    f_i(x + e_i) or, through a wall, to f_opp(i)(x); its transpose gathers the adjoint back."""
    ny, nx = flow.ny, flow.nx
    ys, xs = np.mgrid[0:ny, 0:nx]
    out = np.zeros_like(lam)
    for i in range(8):
        tx = xs + fl.E[i, 0]
        ty = ys + fl.E[i, 1]
        if flow.bc_x in ("periodic", "pressure", "nee"):
            tx = tx % nx
        if flow.bc_y in ("periodic", "nee"):
            ty = ty % ny
        inside = (tx >= 0) & (tx < nx) & (ty >= 0) & (ty < ny)
        out[i][inside] = lam[i, ty[inside], tx[inside]]
        leave = ~inside
        out[i][leave] = lam[fl.OPP[i]][leave]
    return out


def _collide(f, flow, logK, phi):
    return fl.collide(f, flow, phi=phi, K=np.exp(logK))[0]


def collide_vjp(f, lam, flow: fl.Flow, logK, phi):
    """(J_C^T lam, dC/dlogK^T lam, dC/dphi^T lam) per cell, by complex steps (10 evaluations: one
    per population, one per parameter; cells are independent, so each evaluation perturbs the
    same component of every cell at once)."""
    out = np.zeros_like(f)
    for j in range(8):
        fc = f.astype(np.complex128)
        fc[j] += 1j * H
        col = np.imag(_collide(fc, flow, logK, phi)) / H  # d C_i / d f_j, per cell
        out[j] = np.sum(col * lam, axis=0)
    dlogk = np.sum(np.imag(_collide(f.astype(np.complex128), flow, logK + 1j * H, phi)) / H * lam, axis=0)
    dphi = np.sum(np.imag(_collide(f.astype(np.complex128), flow, logK, phi + 1j * H)) / H * lam, axis=0)
    return out, dlogk, dphi


def _pressure(f, flow, logK, phi):
    return fl.pressure_columns(f, flow, phi=phi, K=np.exp(logK))


def pressure_vjp(fs, lam, flow: fl.Flow, logK, phi):
    """VJP of the pressure-column map N(fs): columns 0 and nx-1 are overwritten by a function of
    the adjacent columns and of theta there and at the boundary column."""
    nx = flow.nx
    out = lam.copy()
    out[:, :, 0] = 0.0
    out[:, :, nx - 1] = 0.0
    bmask = np.zeros((flow.ny, nx), dtype=bool)
    bmask[:, [0, nx - 1]] = True
    nmask = np.zeros((flow.ny, nx), dtype=bool)
    nmask[:, [1, nx - 2]] = True
    lam_b = np.where(bmask[None], lam, 0.0)
    for j in range(8):  # d N_b / d fs_j(nb)
        fc = fs.astype(np.complex128)
        fc[j] = fc[j] + 1j * H * nmask
        dN = np.imag(_pressure(fc, flow, logK, phi)) / H
        out[j] += np.where(nmask, _shift_to_neighbour(np.sum(dN * lam_b, axis=0), nx), 0.0)
    glogk = np.zeros((flow.ny, nx))
    gphi = np.zeros((flow.ny, nx))
    for mask in (bmask, nmask):
        for which in ("logK", "phi"):
            lk = logK + (1j * H * mask if which == "logK" else 0)
            ph = phi + (1j * H * mask if which == "phi" else 0)
            dN = np.imag(_pressure(fs.astype(np.complex128), flow, lk, ph)) / H
            contrib = np.sum(dN * lam_b, axis=0)  # sits in the boundary columns
            if mask is nmask:
                contrib = _shift_to_neighbour(contrib, nx)
            (glogk if which == "logK" else gphi)[mask] += contrib[mask]
    return out, glogk, gphi


def _walls(f, flow, logK, phi):
    return fl.wall_nodes(f, flow, phi=phi, K=np.exp(logK))


def wall_vjp(fs, lam, flow: fl.Flow, logK, phi):
    """VJP of the wall-node map W(fs): each wall node b is overwritten by a function of the state at
    its inner neighbour nb and of phi at b and theta at nb.  Several wall nodes may share one nb
    (a corner and its two neighbours along the walls), so the contributions are summed into nb."""
    yb, xb, yn, xn, _ = fl.wall_node_list(flow)
    out = lam.copy()
    glogk = np.zeros((flow.ny, flow.nx))
    gphi = np.zeros((flow.ny, flow.nx))
    if yb.size == 0:
        return out, glogk, gphi
    bmask = np.zeros((flow.ny, flow.nx), dtype=bool)
    bmask[yb, xb] = True
    nmask = np.zeros((flow.ny, flow.nx), dtype=bool)
    nmask[yn, xn] = True
    # W reads the input at nb only: a node that is both a wall node and some wall node's nb would
    # make the per-mask attribution below ambiguous (lattices of fewer than three nodes across)
    assert not (bmask & nmask).any()
    out[:, yb, xb] = 0.0
    lam_b = np.where(bmask[None], lam, 0.0)
    for j in range(8):  # d W_b / d fs_j(nb(b)), summed into nb
        fc = fs.astype(np.complex128)
        fc[j] = fc[j] + 1j * H * nmask
        dW = np.imag(_walls(fc, flow, logK, phi)) / H
        np.add.at(out[j], (yn, xn), np.sum(dW * lam_b, axis=0)[yb, xb])
    for mask in (bmask, nmask):
        for which in ("logK", "phi"):
            lk = logK + (1j * H * mask if which == "logK" else 0)
            ph = phi + (1j * H * mask if which == "phi" else 0)
            dW = np.imag(_walls(fs.astype(np.complex128), flow, lk, ph)) / H
            contrib = np.sum(dW * lam_b, axis=0)[yb, xb]  # d/dtheta at b or at nb(b), held by b
            where = (yb, xb) if mask is bmask else (yn, xn)
            np.add.at(glogk if which == "logK" else gphi, where, contrib)
    return out, glogk, gphi


def _shift_to_neighbour(a, nx):
    """Move values of columns 0 and nx-1 onto columns 1 and nx-2 (where the derivative belongs)."""
    out = np.zeros_like(a)
    out[:, 1] += a[:, 0]
    out[:, nx - 2] += a[:, nx - 1]
    return out


def _cell_velocity(f, flow, logK, phi):
    K = np.exp(logK)
    ax, ay = fl._accel(flow, f[0])
    return fl.velocity(f, phi, K, flow.nu, flow.rho0, flow.forchheimer, ax, ay)


def loss_value(f, flow: fl.Flow, kind="flux", target=None, logK=None, phi=None):
    logK, phi = _theta_fields(flow, logK, phi)
    ux, uy = _cell_velocity(f, flow, logK, phi)
    if kind == "flux":
        return np.sum(ux[:, flow.nx - 1])
    tx, ty = target
    return 0.5 * np.sum((ux - tx) ** 2 + (uy - ty) ** 2)


def loss_grad(f, flow: fl.Flow, kind, target, logK, phi):
    """(dL/df, dL/dlogK, dL/dphi) of a loss that is a sum of per-cell terms (complex steps)."""
    g = np.zeros_like(f)
    for j in range(8):
        fc = f.astype(np.complex128)
        fc[j] += 1j * H
        g[j] = _per_cell_loss_imag(fc, flow, kind, target, logK, phi) / H
    glogk = _per_cell_loss_imag(f.astype(np.complex128), flow, kind, target, logK + 1j * H, phi) / H
    gphi = _per_cell_loss_imag(f.astype(np.complex128), flow, kind, target, logK, phi + 1j * H) / H
    return g, glogk, gphi


def _per_cell_loss_imag(fc, flow, kind, target, logK, phi):
    ux, uy = _cell_velocity(fc, flow, logK, phi)
    if kind == "flux":
        out = np.zeros(ux.shape)
        out[:, flow.nx - 1] = np.imag(ux[:, flow.nx - 1])
        return out
    tx, ty = target
    return np.imag(0.5 * ((ux - tx) ** 2 + (uy - ty) ** 2))


def _has_walls(flow):
    return "nee" in (flow.bc_x, flow.bc_y)


def _equilibrium_state(flow: fl.Flow, phi, p0, u0, phi_p_uniform):
    """f_eq(p0, u0; phi) of every cell (Eq. 22), before the boundary nodes."""
    ny, nx = flow.ny, flow.nx
    p = (p0 / phi) if phi_p_uniform else p0 + 0.0 * phi
    ux = np.full((ny, nx), float(u0[0])) + 0.0 * phi
    uy = np.full((ny, nx), float(u0[1])) + 0.0 * phi
    return fl.equilibrium(p, ux, uy, phi, flow.rho0)


def _boundary(f, flow, logK, phi):
    """B = W o N: the pressure columns, then the wall nodes."""
    if flow.bc_x == "pressure":
        f = _pressure(f, flow, logK, phi)
    if _has_walls(flow):
        f = _walls(f, flow, logK, phi)
    return f


def boundary_vjp(fs, lam, flow, logK, phi):
    """(J_B^T lam, dB/dlogK^T lam, dB/dphi^T lam) at B's input fs: W's VJP at N(fs), then N's."""
    glogk = np.zeros((flow.ny, flow.nx))
    gphi = np.zeros((flow.ny, flow.nx))
    if _has_walls(flow):
        fN = _pressure(fs, flow, logK, phi) if flow.bc_x == "pressure" else fs
        lam, a, b = wall_vjp(fN, lam, flow, logK, phi)
        glogk += a
        gphi += b
    if flow.bc_x == "pressure":
        lam, a, b = pressure_vjp(fs, lam, flow, logK, phi)
        glogk += a
        gphi += b
    return lam, glogk, gphi


def initial_state(flow: fl.Flow, logK, phi, p0=1.0, u0=(0.0, 0.0), phi_p_uniform=False):
    """f(0) of Sec. 3.1 as a function of theta (equilibrium, then the boundary nodes)."""
    return _boundary(_equilibrium_state(flow, phi, p0, u0, phi_p_uniform), flow, logK, phi)


def step(f, flow, logK, phi):
    return _boundary(fl.stream(_collide(f, flow, logK, phi), flow), flow, logK, phi)


def gradient(flow: fl.Flow, T: int, kind="flux", target=None, p0=1.0, u0=(0.0, 0.0), phi_p_uniform=False):
    """(L, dL/dlogK, dL/dphi) after T steps from the equilibrium initial state."""
    logK, phi = _theta_fields(flow)
    f0 = initial_state(flow, logK, phi, p0, u0, phi_p_uniform)
    states = [f0]
    for _ in range(T):
        states.append(step(states[-1], flow, logK, phi))
    L = float(np.real(loss_value(states[-1], flow, kind, target, logK, phi)))
    lam, glogk, gphi = loss_grad(states[-1], flow, kind, target, logK, phi)
    for t in range(T - 1, -1, -1):
        f = states[t]
        fs = fl.stream(_collide(f, flow, logK, phi), flow)
        lam, a, b = boundary_vjp(fs, lam, flow, logK, phi)
        glogk += a
        gphi += b
        lam = stream_transpose(lam, flow)
        lam, a, b = collide_vjp(f, lam, flow, logK, phi)
        glogk += a
        gphi += b
    # the initial state f(0) = B(f_eq(theta)): the boundary nodes couple each boundary cell to its
    # inner neighbour, then the equilibrium of a cell depends on that cell's phi only (Eq. 22)
    f_eq = _equilibrium_state(flow, phi, p0, u0, phi_p_uniform)
    lam, a, b = boundary_vjp(f_eq, lam, flow, logK, phi)
    glogk += a
    gphi += b
    d0 = np.imag(_equilibrium_state(flow, phi + 1j * H, p0, u0, phi_p_uniform)) / H
    gphi += np.sum(d0 * lam, axis=0)
    return L, glogk, gphi
