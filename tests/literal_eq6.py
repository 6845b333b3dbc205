"""A second, deliberately different FP64 evaluator of the flow step, for brute-force checks of the
oracle on tiny lattices.

Pure-Python scalar loops, one cell at a time.  Unlike ``oracle.mrt_d2q8`` it
  * builds e_i from the trigonometric form of Eq. 7,
  * builds M from the polynomial meaning of each moment of Eq. 9 (1, 2|e|^2 - 3, e_x,
    e_x (3|e|^2 - 5), e_y, e_y (3|e|^2 - 5), e_x^2 - e_y^2, e_x e_y) instead of the typed Eq. 10,
  * inverts M exactly with fractions (Gauss-Jordan),
  * applies Eq. 6 in velocity space in one go (f(x + e_i, t+1) = f_i + RHS_i), and
  * resolves every link through an explicit neighbour table.
"""
from __future__ import annotations

import math
from fractions import Fraction


def velocities():
    out = []
    for i in range(1, 9):
        if i <= 4:
            ang = (i - 1) * math.pi / 2
            out.append((round(math.cos(ang)), round(math.sin(ang))))
        else:
            ang = (2 * i - 9) * math.pi / 4
            out.append((round(math.sqrt(2) * math.cos(ang)), round(math.sqrt(2) * math.sin(ang))))
    return out


EV = velocities()
WEIGHTS = [Fraction(1, 9) if ex * ex + ey * ey == 1 else Fraction(1, 36) for ex, ey in EV]


def moment_rows():
    rows = []
    for poly in (
        lambda x, y: 1,
        lambda x, y: 2 * (x * x + y * y) - 3,
        lambda x, y: x,
        lambda x, y: x * (3 * (x * x + y * y) - 5),
        lambda x, y: y,
        lambda x, y: y * (3 * (x * x + y * y) - 5),
        lambda x, y: x * x - y * y,
        lambda x, y: x * y,
    ):
        rows.append([Fraction(poly(ex, ey)) for ex, ey in EV])
    return rows


def invert(A):
    n = len(A)
    aug = [list(A[r]) + [Fraction(int(r == c)) for c in range(n)] for r in range(n)]
    for c in range(n):
        piv = next(r for r in range(c, n) if aug[r][c] != 0)
        aug[c], aug[piv] = aug[piv], aug[c]
        pv = aug[c][c]
        aug[c] = [v / pv for v in aug[c]]
        for r in range(n):
            if r != c and aug[r][c] != 0:
                fac = aug[r][c]
                aug[r] = [a - fac * b for a, b in zip(aug[r], aug[c])]
    return [row[n:] for row in aug]


MROWS = moment_rows()
MINV = invert(MROWS)
MF = [[float(v) for v in r] for r in MROWS]
MINVF = [[float(v) for v in r] for r in MINV]


def opposite(i):
    ex, ey = EV[i]
    return EV.index((-ex, -ey))


def link_table(nx, ny, bc_x, bc_y, walls):
    """For every (x, y, i): ('move', tx, ty, i) or ('bounce', x, y, opp(i), u_wall)."""
    table = {}
    for y in range(ny):
        for x in range(nx):
            for i, (ex, ey) in enumerate(EV):
                tx, ty = x + ex, y + ey
                if bc_x == "periodic":
                    tx %= nx
                if bc_y == "periodic":
                    ty %= ny
                if 0 <= tx < nx and 0 <= ty < ny:
                    table[(x, y, i)] = ("move", tx, ty, i)
                else:
                    if ty < 0:
                        uw = walls["bottom"]
                    elif ty >= ny:
                        uw = walls["top"]
                    elif tx < 0:
                        uw = walls["left"]
                    else:
                        uw = walls["right"]
                    table[(x, y, i)] = ("bounce", x, y, opposite(i), uw)
    return table


def step(f, nx, ny, phi, K, nu, ax, ay, rates, forch, bc_x, bc_y, walls, rho0=1.0):
    """One step of Eq. 6 on f[y][x][i] (nested lists); returns the new nested list."""
    table = link_table(nx, ny, bc_x, bc_y, walls)
    new = [[[None] * 8 for _ in range(nx)] for _ in range(ny)]
    for y in range(ny):
        for x in range(nx):
            fc = f[y][x]
            ph, k = phi[y][x], K[y][x]
            m = [sum(MF[r][i] * fc[i] for i in range(8)) for r in range(8)]
            jx = sum(EV[i][0] * fc[i] for i in range(8))
            jy = sum(EV[i][1] * fc[i] for i in range(8))
            vx = jx / rho0 + 0.5 * ph * ax[y][x]
            vy = jy / rho0 + 0.5 * ph * ay[y][x]
            fphi = 1.75 / math.sqrt(150 * ph**3) if forch else 0.0
            l0 = 0.5 * (1 + 0.5 * ph * nu / k)
            l1 = 0.5 * ph * fphi / math.sqrt(k)
            den = l0 + math.sqrt(l0 * l0 + l1 * math.hypot(vx, vy))
            ux, uy = vx / den, vy / den
            u2 = ux * ux + uy * uy
            p = (1 / 3) / (ph * (5 / 9)) * (sum(fc) - (2 / 3) * rho0 * u2 / ph)
            umag = math.sqrt(u2)
            Fx = -ph * nu / k * ux - ph * fphi / math.sqrt(k) * umag * ux + ph * ax[y][x]
            Fy = -ph * nu / k * uy - ph * fphi / math.sqrt(k) * umag * uy + ph * ay[y][x]
            meq = [
                5 / 3 * ph * p + 2 / 3 * rho0 * u2 / ph,
                -ph * p,
                rho0 * ux,
                -rho0 * ux,
                rho0 * uy,
                -rho0 * uy,
                rho0 * (ux * ux - uy * uy) / ph,
                rho0 * ux * uy / ph,
            ]
            S = [
                0.0,
                rho0 * 4 * (ux * Fx + uy * Fy) / (5 * ph),
                rho0 * Fx,
                -rho0 * Fx,
                rho0 * Fy,
                -rho0 * Fy,
                rho0 * 2 * (ux * Fx - uy * Fy) / ph,
                rho0 * (ux * Fy + uy * Fx) / ph,
            ]
            rhs_m = [-rates[r] * (m[r] - meq[r]) + (1 - rates[r] / 2) * S[r] for r in range(8)]
            for i in range(8):
                post = fc[i] + sum(MINVF[i][r] * rhs_m[r] for r in range(8))
                kind = table[(x, y, i)]
                if kind[0] == "move":
                    _, tx, ty, ii = kind
                    new[ty][tx][ii] = post
                else:
                    _, bx, by, oi, uw = kind
                    ex, ey = EV[i]
                    new[by][bx][oi] = post - 2 * float(WEIGHTS[i]) * rho0 * (ex * uw[0] + ey * uw[1]) * 3
    return new
