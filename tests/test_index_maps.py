"""CPU checks of two device-side index maps, restated here from the kernels' rules (no GPU):

* the lane groups of the wall-node adjoint transpose (`k_adj_wall`): one group per inner neighbour
  nb, holding every wall node that extrapolates from it, must cover the oracle's wall-node list
  (`oracle.mrt_d2q8.wall_node_list`, node -> nb and wall) exactly once, with no nb in two groups
  and no nb that is itself a wall node, for every side combination from four nodes across;
* the boundary-node planes of the in-place pre-pass (`k_edge_ip`): the thread index k of a
  boundary node and the plane index the step reads it back from must agree, each boundary node
  written once.
"""
import numpy as np
import pytest

from oracle import mrt_d2q8 as fl

SIDES = [(bx, by) for bx in ("periodic", "wall", "pressure", "nee") for by in ("periodic", "wall", "nee")
         if "nee" in (bx, by) or bx == "pressure"]


def wall_groups(nx, ny, bcx, bcy):
    """(nb, [(y, x, wall)]) per lane group, in the kernel's order."""
    per = bcx == "periodic"
    gy = (nx if per else nx - 2) if bcy == "nee" else 0
    row0 = 2 if bcy == "nee" else 0
    gx = (ny - 4 if bcy == "nee" else ny) if bcx == "nee" else 0
    out = []
    for grp in range(2 * (gy + gx)):
        nodes = []
        if grp < 2 * gy:
            top = grp >= gy
            g = grp - (gy if top else 0)
            xt = g if per else g + 1
            yt = ny - 2 if top else 1
            yw, w = (ny - 1, 3) if top else (0, 2)
            nodes.append((yw, xt, w))
            if not per and xt == 1:
                nodes.append((yw, 0, w))
            if not per and xt == nx - 2:
                nodes.append((yw, nx - 1, w))
            if bcx == "nee" and xt == 1:
                nodes.append((yt, 0, 0))
            if bcx == "nee" and xt == nx - 2:
                nodes.append((yt, nx - 1, 1))
        else:
            g2 = grp - 2 * gy
            right = g2 >= gx
            yt = row0 + g2 - (gx if right else 0)
            xt = nx - 2 if right else 1
            nodes.append((yt, nx - 1 if right else 0, 1 if right else 0))
        out.append(((yt, xt), nodes))
    return out


@pytest.mark.parametrize("bcx,bcy", [s for s in SIDES if "nee" in s])
def test_wall_node_groups_cover_the_wall_node_list_once(bcx, bcy):
    for nx in range(4, 11):
        for ny in range(4, 11):
            flow = fl.Flow(nx=nx, ny=ny, phi=np.ones((ny, nx)), K=np.ones((ny, nx)), nu=0.1, bc_x=bcx, bc_y=bcy)
            want = sorted(zip(*[a.tolist() for a in fl.wall_node_list(flow)]))
            got, targets = [], set()
            for (yt, xt), nodes in wall_groups(nx, ny, bcx, bcy):
                assert (yt, xt) not in targets and 0 <= yt < ny and 0 <= xt < nx
                targets.add((yt, xt))
                assert len(nodes) <= 3
                got += [(y, x, yt, xt, w) for (y, x, w) in nodes]
            assert sorted(got) == want, (bcx, bcy, nx, ny)
            assert not ({(y, x) for (y, x, *_) in got} & targets)


def boundary_node(nx, ny, bcx, bcy, x, y):
    return (bcy == "nee" and y in (0, ny - 1)) or (bcx == "nee" and x in (0, nx - 1)) or (bcx == "pressure" and x in (0, nx - 1))


def edge_index(nx, ny, x, y):
    if y == 0:
        return x
    if y == ny - 1:
        return nx + x
    return 2 * nx + (y if x == 0 else ny + y)


@pytest.mark.parametrize("bcx,bcy", SIDES)
def test_boundary_node_planes_agree_with_the_pre_pass(bcx, bcy):
    for nx in range(3, 11):
        for ny in range(2 if bcy != "nee" else 3, 11):
            n = 2 * (nx + ny)
            written = {}
            for k in range(n):  # the pre-pass: thread k's cell, skipped where another thread has it
                if k < 2 * nx:
                    if k >= nx and ny == 1:
                        continue
                    y, x = (0, k) if k < nx else (ny - 1, k - nx)
                else:
                    r = k - 2 * nx
                    x, y = (0, r) if r < ny else (nx - 1, r - ny)
                    if y in (0, ny - 1):
                        continue
                if not boundary_node(nx, ny, bcx, bcy, x, y):
                    continue
                assert (x, y) not in written
                written[(x, y)] = k
                assert edge_index(nx, ny, x, y) == k
            cells = {(x, y) for y in range(ny) for x in range(nx) if boundary_node(nx, ny, bcx, bcy, x, y)}
            assert set(written) == cells, (bcx, bcy, nx, ny)
