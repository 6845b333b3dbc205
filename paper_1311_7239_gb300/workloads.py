"""Synthetic workloads shaped like the paper's test flows (Sec. 3): configurations and media.

Batched ensemble of independent porous cavities and channels (``ensemble``, ``build``):

Each lattice draws its size, kind and Reynolds number from ``synth.ensemble_domains`` and its
porosity / permeability field from ``synth.heterogeneous_medium`` (log K Gaussian with mean
log(Da H^2), eps = clip(0.3 + 0.1 N, 0.1, 0.9), correlation length 32 cells).  Lattice parameters:
  cavity  -- halfway walls, top wall moving at U = 0.03, nu = max(U H / Re, 0.02);
  channel -- periodic in x, walls in y, body force a_x chosen so that the Darcy-Brinkman centre
             speed of the mean medium (the closed form behind Eq. 24 with F_phi = 0) is U = 0.02,
             nu = max(U H / Re, 0.02).
The floor on nu keeps tau_v >= 0.56 and the speeds keep |u| / (c_s sqrt(eps)) <= 0.17 where the
porosity is lowest (eps >= 0.1): the equilibrium of Eq. 11 carries |u|^2 / eps.  With a lid at
U = 0.05 (0.27 over eps = 0.1) FP32 stays bounded but FP16 and BF16 deviation storage diverge at
the lid within a few thousand steps.
All lattices start from the rest state phi p = mean(eps) (uniform phi p over a varying porosity).

Pressure-driven heterogeneous channel for the adjoint (``adjoint_channel``): log K Gaussian with
mean log(1e-3 H^2), sigma 1, correlation length 32; eps = clip(0.3 + 0.1 N, 0.1, 0.9); the four
columns next to the inlet and the outlet hold the mean medium, so that the prescribed pressure
columns meet a uniform porosity; nu = 0.1; p_in - p_out from the Darcy estimate of a mean speed
of 0.01 (phi u = -K grad(phi p) / (rho0 nu), Eq. 2 without inertia and viscous terms).

Natural convection in a square porous cavity (``natural_convection``, Sec. 3.4): Pr = 1,
J = sigma = gamma = 1, zeta3 = zeta4 = 1.1, T_h = 21 (left), T_c = 1 (right), adiabatic top and
bottom, tau_v and tau_T from Eq. 26 with Ma = 0.1 and c_sT^2 = 2/5; g beta from
U = Ma / sqrt(3) = sqrt(g beta dT L).
"""
from __future__ import annotations

import math

import numpy as np

from . import synth


def ensemble(lbm, n=512, seed=42, lo=64, hi=1024, precision=0, da=1e-3):
    """(configs, media) for ``lbm.Batch``: media[d] = (eps, K) float32 arrays [ny, nx]."""
    cfgs, media = [], []
    for dom in synth.ensemble_domains(n, seed, lo, hi):
        nx, ny, Re = dom["nx"], dom["ny"], dom["Re"]
        eps, K = synth.heterogeneous_medium(ny, nx, H=ny, seed=dom["seed"], da_mean=da, corr_len=32.0)
        eps = eps.astype(np.float32)
        K = K.astype(np.float32)
        phi_m = float(eps.mean())
        K_m = float(np.exp(np.log(K.astype(np.float64)).mean()))
        if dom["kind"] == "cavity":
            U = 0.03
            nu = max(U * ny / Re, 0.02)
            kw = dict(bc_x=lbm.WALL, bc_y=lbm.WALL, u_wall=[(0, 0), (0, 0), (0, 0), (U, 0)])
        else:
            U = 0.02
            nu = max(U * ny / Re, 0.02)
            th = math.sqrt(phi_m / K_m)
            x = min(th * ny / 2, 300.0)
            G = U * nu / (K_m * (1.0 - 1.0 / math.cosh(x)))
            kw = dict(bc_x=lbm.PERIODIC, bc_y=lbm.WALL, ax=G)
        cfg = lbm.default_config(nx=nx, ny=ny, nu=nu, phi=phi_m, K=K_m, precision=precision, p_rest=phi_m, **kw)
        cfgs.append(cfg)
        media.append((eps, K))
    return cfgs, media


def build(lbm, cfgs, media):
    """A ``lbm.Batch`` with every medium set and the rest state phi p = mean(eps) per lattice."""
    b = lbm.Batch(cfgs)
    for d, (eps, K) in enumerate(media):
        b.set_medium(d, np.ascontiguousarray(eps), np.ascontiguousarray(K))
        b.init_equilibrium(d, float(cfgs[d].p_rest), 0.0, 0.0, phi_p_uniform=True)
    return b


def adjoint_channel(lbm, nx=2048, ny=1024, seed=1234, u_mean=0.01, nu=0.1, precision=0):
    """(config, eps, logK) of the pressure-driven heterogeneous channel (float32 [ny, nx] fields)."""
    eps, K = synth.heterogeneous_medium(ny, nx, H=ny, seed=seed, da_mean=1e-3, sigma_logk=1.0, corr_len=32.0, eps_mean=0.3,
                                        eps_sd=0.1, eps_lo=0.1, eps_hi=0.9)
    logk = np.log(K)
    for cols in (slice(0, 4), slice(nx - 4, nx)):
        eps[:, cols] = eps.mean()
        logk[:, cols] = logk.mean()
    phi_m = float(eps.mean())
    K_m = float(np.exp(logk.mean()))
    dphip = u_mean * phi_m * nu * (nx - 1) / K_m
    dp = dphip / phi_m
    cfg = lbm.default_config(nx=nx, ny=ny, nu=nu, phi=phi_m, K=K_m, bc_x=lbm.PRESSURE, bc_y=lbm.WALL, p_in=1.0 + dp / 2,
                             p_out=1.0 - dp / 2, p_rest=phi_m, precision=precision)
    return cfg, eps.astype(np.float32), logk.astype(np.float32)


def natural_convection(lbm, L=2048, Ra=1e5, Pr=1.0, phi=0.6, Da=1e-2, Ma=0.1, precision=0):
    tau_v = 0.5 + Ma * L * math.sqrt(3.0 * Pr) / math.sqrt(Ra)
    tau_T = 0.5 + (1.0 / 3.0) * (tau_v - 0.5) / (0.4 * Pr)
    nu = (tau_v - 0.5) / 3.0
    U = Ma / math.sqrt(3.0)
    g_beta = U * U / (20.0 * L)
    return lbm.default_config(nx=L, ny=L, bc_x=lbm.WALL, bc_y=lbm.WALL, nu=nu, phi=phi, K=Da * L * L, thermal=1, tau_T=tau_T,
                              g_beta=g_beta, T0=11.0, T_wall=[21.0, 1.0, None, None], p_rest=phi, precision=precision,
                              dev_scale_log2=8)
