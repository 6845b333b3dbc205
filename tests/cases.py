"""Paired problem set-ups: the same case as an oracle ``Flow`` (FP64, numpy) and as a liblbm
configuration, plus small helpers shared by the GPU parity tests."""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from oracle import mrt_d2q8 as fl
from oracle import thermal_d2q5 as th
from paper_1311_7239_gb300 import synth

_BC = {"periodic": 0, "wall": 1, "pressure": 2, "nee": 3}


@dataclass
class Case:
    nx: int
    ny: int
    nu: float = 0.1
    phi: float = 0.4
    K: float = 10.0
    het: bool = False           # per-cell random medium
    eps_sd: float = 0.1         # porosity spread of the random medium
    corr: float = 0.0           # correlation length of the random medium (0: ny / 8)
    forch: bool = True
    ax: float = 0.0
    ay: float = 0.0
    bc_x: str = "periodic"
    bc_y: str = "wall"
    walls: dict = field(default_factory=dict)  # side -> (ux, uy)
    p_in: float = 1.0
    p_out: float = 1.0
    precision: int = 0
    seed: int = 5
    thermal: dict | None = None  # keys of oracle.thermal_d2q5.Thermal
    streaming: int = 0           # 0: A-B buffers, 1: in-place (one buffer)

    def medium(self):
        if not self.het:
            return np.full((self.ny, self.nx), self.phi), np.full((self.ny, self.nx), self.K)
        eps, K = synth.heterogeneous_medium(self.ny, self.nx, H=self.ny, seed=self.seed, da_mean=self.K / self.ny**2,
                                            corr_len=self.corr or max(2.0, self.ny / 8), eps_mean=self.phi, eps_sd=self.eps_sd, eps_lo=0.1,
                                            eps_hi=0.95)
        # the GPU stores float32 fields: give the oracle the same values
        return eps.astype(np.float32).astype(np.float64), K.astype(np.float32).astype(np.float64)

    def flow(self) -> fl.Flow:
        eps, K = self.medium()
        w = {s: tuple(self.walls.get(s, (0.0, 0.0))) for s in ("left", "right", "bottom", "top")}
        return fl.Flow(nx=self.nx, ny=self.ny, phi=eps, K=K, nu=self.nu, forchheimer=self.forch,
                       accel=np.array([self.ax, self.ay]), bc_x=self.bc_x, bc_y=self.bc_y,
                       u_left=w["left"], u_right=w["right"], u_bottom=w["bottom"], u_top=w["top"],
                       p_in=self.p_in, p_out=self.p_out)

    def thermal_params(self):
        return th.Thermal(**self.thermal) if self.thermal else None

    def p_rest(self):
        eps, _ = self.medium()
        return float(np.mean(eps))

    def config(self, lbm):
        w = [self.walls.get(s, (0.0, 0.0)) for s in ("left", "right", "bottom", "top")]
        kw = dict(nx=self.nx, ny=self.ny, nu=self.nu, phi=self.phi, K=self.K, forchheimer=int(self.forch), ax=self.ax,
                  ay=self.ay, bc_x=_BC[self.bc_x], bc_y=_BC[self.bc_y], u_wall=w, p_in=self.p_in, p_out=self.p_out,
                  precision=self.precision, p_rest=self.p_rest(), streaming=self.streaming)
        if self.thermal:
            t = self.thermal
            kw.update(thermal=1, tau_T=t["tau_T"], g_beta=t["g_beta"], T0=t["T0"],
                      T_wall=[t.get("T_left"), t.get("T_right"), t.get("T_bottom"), t.get("T_top")])
        return lbm.default_config(**kw)

    def lattice(self, lbm):
        import torch

        lat = lbm.Lattice(self.config(lbm))
        if self.het:
            eps, K = self.medium()
            lat.set_medium(torch.tensor(eps, dtype=torch.float32, device="cuda"),
                           torch.tensor(K, dtype=torch.float32, device="cuda"))
        return lat


def to_gpu(a):
    import torch

    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.sqrt((b * b).sum())
    return float(np.sqrt(((a - b) ** 2).sum()) / den) if den > 0 else float(np.sqrt((a * a).sum()))


def random_state(flow: fl.Flow, seed: int, amp: float = 0.02, u_amp: float = 0.05):
    rng = np.random.default_rng(seed)
    p = 1.0 + 0.05 * rng.standard_normal((flow.ny, flow.nx))
    ux = u_amp * rng.standard_normal((flow.ny, flow.nx))
    uy = u_amp * rng.standard_normal((flow.ny, flow.nx))
    f = fl.equilibrium(p, ux, uy, flow.phi) + amp * 0.1 * rng.standard_normal((8, flow.ny, flow.nx))
    f = f.astype(np.float32).astype(np.float64)
    if flow.bc_x == "pressure" or "nee" in (flow.bc_x, flow.bc_y):
        f = fl.boundary_nodes(f, flow).astype(np.float32).astype(np.float64)
    return f
