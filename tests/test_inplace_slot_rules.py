"""The in-place streaming scheme (LBM_STREAM_INPLACE), checked on the CPU from its definition.

The scheme, as lbm.h and the device header define it: of each pair of opposite velocities the
member with e_x > 0, or e_x = 0 and e_y > 0, is positive; at parity par a cell c reads population
i from plane (par ? i : opp(i)), at c for a positive i and at c - e_i otherwise; a population that
would come from beyond a wall is read, plus the moving-wall term, from the slot where the cell
parked its own opposite population; the post-collision population j goes where cell c + e_j reads
j at the next parity.  Ghost rows -1 and ny are rows of the planes, the ghost column sits after the
last plane.  The interior threads address the same slots as aligned vectors of rows y, y + 1 and
one-cell-shifted vectors; the wall and last-column groups form a frame done cell by cell.

These tests restate those rules in Python and check what makes them correct: every slot lies in
the buffer, no slot is read or written by two cells of one step (so one buffer needs no second
copy and no ordering between threads), each cell writes exactly the slots it read, the interior
vector addressing equals the generic rule, and a trajectory of the scheme equals the pull of
Eq. 15 with halfway bounce-back (the A-B form) for D2Q8 with moving walls and D2Q5 with
anti-bounce-back at isothermal walls.  Pure Python on small lattices.
"""
import itertools
import random

import pytest

PERIODIC, WALL = 0, 1
EX = [1, 0, -1, 0, 1, -1, -1, 1]   # Eq. 7 velocities (0-based)
EY = [0, 1, 0, -1, 1, 1, -1, -1]
W8 = [1 / 9] * 4 + [1 / 36] * 4
EX5 = [0, 1, 0, -1, 0]
EY5 = [0, 0, 1, 0, -1]


def opp(i):
    return (i + 2) & 3 if i < 4 else 4 + ((i - 4 + 2) & 3)


def opp5(i):
    return 0 if i == 0 else 1 + ((i - 1 + 2) & 3)


def positive(i, ex, ey):
    return ex[i] > 0 or (ex[i] == 0 and ey[i] > 0)


class Layout:
    def __init__(self, nx, ny, bcx, bcy):
        self.nx, self.ny, self.bcx, self.bcy = nx, ny, bcx, bcy
        self.pitch = (nx + 127) // 128 * 128
        self.plane = self.pitch * (ny + 2)

    def wrap(self, v, n, periodic):
        return (v + n if v < 0 else (v - n if v >= n else v)) if periodic else v

    def slot(self, q, plane, cx, cy):
        assert 0 <= cx <= self.nx and -1 <= cy <= self.ny
        if cx >= self.nx:
            return q * self.plane - self.pitch + plane * (self.ny + 2) + (cy + 1)
        return plane * self.plane + cy * self.pitch + cx

    def off(self, q, ex, ey, op, cx, cy, i, par):
        if i != 0 and not positive(i, ex, ey):
            cx -= ex[i]
            cy -= ey[i]
        cx = self.wrap(cx, self.nx, self.bcx == PERIODIC)
        cy = self.wrap(cy, self.ny, self.bcy == PERIODIC)
        plane = 0 if (q == 5 and i == 0) else (i if par else op(i))
        return self.slot(q, plane, cx, cy)

    def wall_of(self, sx, sy):
        if sy < 0:
            return 2
        if sy >= self.ny:
            return 3
        return 0 if sx < 0 else 1

    def source(self, q, ex, ey, op, x, y, i, par):
        sx = self.wrap(x - ex[i], self.nx, self.bcx == PERIODIC)
        sy = self.wrap(y - ey[i], self.ny, self.bcy == PERIODIC)
        if 0 <= sx < self.nx and 0 <= sy < self.ny:
            return self.off(q, ex, ey, op, x, y, i, par), -1
        return self.off(q, ex, ey, op, sx, sy, op(i), par), self.wall_of(sx, sy)


SIZES = [(2, 2), (3, 5), (5, 3), (9, 7), (13, 6), (17, 9), (128, 3)]
BCS = list(itertools.product((PERIODIC, WALL), repeat=2))


@pytest.mark.parametrize("q", [8, 5])
@pytest.mark.parametrize("bcx,bcy", BCS)
def test_slots_in_buffer_and_no_slot_shared_within_a_step(q, bcx, bcy):
    ex, ey, op = (EX, EY, opp) if q == 8 else (EX5, EY5, opp5)
    for nx, ny in SIZES:
        L = Layout(nx, ny, bcx, bcy)
        end = q * L.plane - L.pitch + q * (ny + 2)
        for par in (0, 1):
            reader, writer = {}, {}
            own_reads = {}
            for y in range(ny):
                for x in range(nx):
                    reads = set()
                    for i in range(q):
                        o, _ = L.source(q, ex, ey, op, x, y, i, par)
                        assert -L.pitch <= o < end
                        assert o not in reader, "two cells read one slot"
                        reader[o] = (x, y)
                        reads.add(o)
                        o2 = L.off(q, ex, ey, op, x + ex[i], y + ey[i], i, 1 - par)
                        assert -L.pitch <= o2 < end
                        assert o2 not in writer, "two cells write one slot"
                        writer[o2] = (x, y)
                    own_reads[(x, y)] = reads
            for o, c in reader.items():
                if o in writer:
                    assert writer[o] == c, "a slot read by one cell and written by another"
            # a cell writes its normal read slots; its bounce-back reads are its own parked slots
            writes_of = {}
            for o, c in writer.items():
                writes_of.setdefault(c, set()).add(o)
            for c in writes_of:
                normal = {L.off(q, ex, ey, op, c[0], c[1], i, par) for i in range(q)}
                assert writes_of[c] == normal


def _interior_groups(nx, ny, bcx, bcy):
    for y in range(ny):
        for x0 in range(0, nx, 4):
            edge = (bcx == WALL and x0 == 0) or x0 + 4 >= nx or (bcy == WALL and (y == 0 or y == ny - 1))
            if not edge:
                yield x0, y


@pytest.mark.parametrize("bcx,bcy", BCS)
def test_interior_vector_addressing_equals_the_rule(bcx, bcy):
    """Slots of the interior threads: own cells (e1, e2, e5, e8), row y + 1 (e4), and cells x + 1 of
    rows y, y - 1, y + 1 (e3, e6, e7); population opp(i) is stored into the slot i came from."""
    row = {0: 0, 1: 0, 2: 0, 3: 1, 4: 0, 5: -1, 6: 1, 7: 0}
    shift = {0: 0, 1: 0, 2: 1, 3: 0, 4: 0, 5: 1, 6: 1, 7: 0}
    row5 = {0: 0, 1: 0, 2: 0, 3: 0, 4: 1}
    shift5 = {0: 0, 1: 0, 2: 0, 3: 1, 4: 0}
    for nx, ny in SIZES + [(40, 5)]:
        L = Layout(nx, ny, bcx, bcy)
        for par in (0, 1):
            for x0, y in _interior_groups(nx, ny, bcx, bcy):
                assert x0 + 4 <= nx - 1
                for c in range(4):
                    x = x0 + c
                    for i in range(8):
                        ry = (y + row[i]) % ny
                        vo = (i if par else opp(i)) * L.plane + ry * L.pitch + x + shift[i]
                        assert vo == L.source(8, EX, EY, opp, x, y, i, par)[0]
                        j = opp(i)
                        assert vo == L.off(8, EX, EY, opp, x + EX[j], y + EY[j], j, 1 - par)
                    for i in range(5):
                        ry = (y + row5[i]) % ny
                        pl = 0 if i == 0 else (i if par else opp5(i))
                        vo = pl * L.plane + ry * L.pitch + x + shift5[i]
                        assert vo == L.source(5, EX5, EY5, opp5, x, y, i, par)[0]
                        j = opp5(i)
                        assert vo == L.off(5, EX5, EY5, opp5, x + EX5[j], y + EY5[j], j, 1 - par)


def _frame(nx, ny, bcx, bcy):
    """The frame cells as the launch enumerates them (whole wall rows, then per row the cells
    x < L and x >= R)."""
    Lc = (min(nx, 4)) if bcx == WALL else 0
    x0e = 0 if nx <= 4 else (nx - 1) // 4 * 4
    R = max(x0e, Lc)
    E = Lc + (nx - R)
    wr = 2 if bcy == WALL else 0
    cells = []
    for k in range(wr * nx + (ny - wr) * E):
        if k < wr * nx:
            cells.append((k if k < nx else k - nx, 0 if k < nx else ny - 1))
        else:
            r, j = divmod(k - wr * nx, E)
            cells.append((j if j < Lc else R + (j - Lc), r + (1 if wr else 0)))
    return cells


@pytest.mark.parametrize("bcx,bcy", BCS)
def test_frame_and_interior_cover_every_cell_once(bcx, bcy):
    for nx, ny in itertools.product([2, 3, 4, 5, 7, 8, 9, 13, 130, 515], [2, 3, 7]):
        seen = {}
        for c in _frame(nx, ny, bcx, bcy):
            assert 0 <= c[0] < nx and 0 <= c[1] < ny and c not in seen
            seen[c] = 1
        for x0, y in _interior_groups(nx, ny, bcx, bcy):
            for c in range(4):
                assert (x0 + c, y) not in seen
                seen[(x0 + c, y)] = 1
        assert len(seen) == nx * ny


def _run(q, nx, ny, bcx, bcy, steps, seed):
    """The scheme against the pull with bounce-back, with an arbitrary per-cell update in place of
    the collision (the slot rules do not depend on what the collision computes)."""
    ex, ey, op = (EX, EY, opp) if q == 8 else (EX5, EY5, opp5)
    rng = random.Random(seed)
    L = Layout(nx, ny, bcx, bcy)
    uw = [(rng.uniform(-.1, .1), rng.uniform(-.1, .1)) for _ in range(4)]
    Tdir = [rng.random() < .5 for _ in range(4)]
    Tw = [rng.uniform(-1, 1) for _ in range(4)]

    def bounce(i, w, own):  # Eq. 15 at a wall: moving-wall bounce-back (D2Q8), anti-bounce-back (D2Q5)
        if q == 8:
            return own + 6 * W8[i] * (ex[i] * uw[w][0] + ey[i] * uw[w][1])
        return -own + 0.4 * Tw[w] if Tdir[w] else own

    def unbounce(i, w, v):
        if q == 8:
            return v - 6 * W8[i] * (ex[i] * uw[w][0] + ey[i] * uw[w][1])
        return 0.4 * Tw[w] - v if Tdir[w] else v

    def update(f, x, y, t):
        return [f[j] * (1 + 0.01 * j) + 0.001 * (x + 3 * y + 7 * j + t) - 0.0005 * f[op(j)] for j in range(q)]

    cells = [(x, y) for y in range(ny) for x in range(nx)]
    f0 = {c: [rng.uniform(-1, 1) for _ in range(q)] for c in cells}
    pre = dict(f0)
    for t in range(steps):  # A-B pull
        post = {c: update(pre[c], c[0], c[1], t) for c in cells}
        nxt = {}
        for (x, y) in cells:
            v = []
            for i in range(q):
                sx = L.wrap(x - ex[i], nx, bcx == PERIODIC)
                sy = L.wrap(y - ey[i], ny, bcy == PERIODIC)
                if 0 <= sx < nx and 0 <= sy < ny:
                    v.append(post[(sx, sy)][i])
                else:
                    v.append(bounce(i, L.wall_of(sx, sy), post[(x, y)][op(i)]))
            nxt[(x, y)] = v
        pre = nxt
    A, par = {}, 0
    for (x, y) in cells:  # the state written into the layout of parity 0
        for i in range(q):
            o, w = L.source(q, ex, ey, op, x, y, i, par)
            A[o] = f0[(x, y)][i] if w < 0 else unbounce(i, w, f0[(x, y)][i])

    def read(x, y):
        out = []
        for i in range(q):
            o, w = L.source(q, ex, ey, op, x, y, i, par)
            out.append(A[o] if w < 0 else bounce(i, w, A[o]))
        return out

    for t in range(steps):
        reads = {c: read(*c) for c in cells}
        for (x, y) in cells:
            post = update(reads[(x, y)], x, y, t)
            for j in range(q):
                A[L.off(q, ex, ey, op, x + ex[j], y + ey[j], j, 1 - par)] = post[j]
        par ^= 1
    return max(abs(a - b) for c in cells for a, b in zip(read(*c), pre[c]))


@pytest.mark.parametrize("q", [8, 5])
@pytest.mark.parametrize("bcx,bcy", BCS)
def test_trajectory_equals_the_pull_with_bounce_back(q, bcx, bcy):
    for nx, ny in [(2, 2), (5, 3), (9, 7), (13, 6)]:
        assert _run(q, nx, ny, bcx, bcy, steps=5, seed=nx * 31 + ny) < 1e-12


class _Mutated(Layout):
    """The rule with a planted mistake: the positive member of a pair read at c - e_i as well."""

    def off(self, q, ex, ey, op, cx, cy, i, par):
        if i != 0:
            cx -= ex[i]
            cy -= ey[i]
        cx = self.wrap(cx, self.nx, self.bcx == PERIODIC)
        cy = self.wrap(cy, self.ny, self.bcy == PERIODIC)
        cx = min(max(cx, 0), self.nx)
        cy = min(max(cy, -1), self.ny)
        return self.slot(q, i if par else op(i), cx, cy)


def _violations(L):
    reader, writer = {}, {}
    bad = 0
    for par in (0, 1):
        reader.clear()
        writer.clear()
        for y in range(L.ny):
            for x in range(L.nx):
                for i in range(8):
                    o, _ = L.source(8, EX, EY, opp, x, y, i, par)
                    bad += o in reader
                    reader[o] = (x, y)
                    o2 = L.off(8, EX, EY, opp, x + EX[i], y + EY[i], i, 1 - par)
                    bad += o2 in writer
                    writer[o2] = (x, y)
        bad += sum(1 for o, c in reader.items() if o in writer and writer[o] != c)
    return bad


def test_a_broken_rule_is_caught():
    """The race check above fails on the rule with a planted mistake and passes on the real one."""
    assert _violations(Layout(9, 7, WALL, PERIODIC)) == 0
    assert _violations(_Mutated(9, 7, WALL, PERIODIC)) > 0
