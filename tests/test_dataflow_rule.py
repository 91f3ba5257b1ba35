"""The covering argument of the dataflow step order (tiling variant 6), checked
by brute force on small lattices (CPU only).

A unit of work is a strip (128 columns x `rows` rows) or an east boundary
block (NN: 8 rows, CBC: its block size) of one lattice.  Step t reads the
buffer step t-1 wrote and writes the buffer step t-1 read, so unit U of step t
must wait for every unit V of step t-1 that wrote a node U reads (read after
write) or read a node U writes (write after read).  Here every unit's used
reads and its writes are derived from the stencils of the step: pull streaming,
bounce-back's own-node read, the network's 3 x 3 feature nodes with their pulls,
and the characteristic outflow's stencil.  The test checks that the flags the
kernels wait on cover all of them.  The waits below restate the device rule
(3 x 3 strips around a strip; for an east tile also the boundary blocks that
meet its rows +- 2; for a boundary block the east-tile strips and boundary
blocks that meet its rows +- 2).  Reads whose values the step discards (the
x-wrap of a non-periodic lattice's edge columns, rebuilt by its boundary
condition) are not dependencies.
"""
import itertools
import random

import pytest

TILE = 128


def wrap(v, n):
    return v % n


def rows_meeting(a, b, ny):
    """Rows of the wrapped segments covering a..b (the device's row_segments)."""
    if b - a + 1 >= ny:
        return set(range(ny))
    return {wrap(y, ny) for y in range(a, b + 1)}


class Lattice:
    def __init__(self, nx, ny, rows, ext, per, periodic, solid):
        self.nx, self.ny, self.rows, self.ext, self.per = nx, ny, rows, ext, per
        self.periodic = periodic
        self.solid = solid                       # set of solid (x, y)
        self.tiles = (nx + TILE - 1) // TILE
        self.nrow = (ny + rows - 1) // rows
        self.L = nx - 1

    # ---- units and ownership ----
    def strips(self):
        return [("s", r, c) for r in range(self.nrow) for c in range(self.tiles)]

    def ext_blocks(self):
        if not self.ext:
            return []
        return [("e", j) for j in range((self.ny + self.per - 1) // self.per)]

    def strip_nodes(self, r, c):
        return [(x, y) for y in range(r * self.rows, min((r + 1) * self.rows, self.ny))
                for x in range(c * TILE, min((c + 1) * TILE, self.nx))]

    def is_ext_node(self, x, y):
        return self.ext is not None and x == self.L and (x, y) not in self.solid

    def owner(self, x, y):
        if self.is_ext_node(x, y):
            return ("e", y // self.per)
        return ("s", y // self.rows, x // TILE)

    # ---- footprints (node granularity) ----
    def pull_sources(self, x, y):
        out = []
        for cx, cy in itertools.product((-1, 0, 1), repeat=2):
            sx, sy = x - cx, wrap(y - cy, self.ny)
            if 0 <= sx < self.nx:
                out.append((sx, sy))
            elif self.periodic:
                out.append((wrap(sx, self.nx), sy))
            # else: the pulled value is rebuilt by the inlet or outflow (discarded)
        return out

    def reads(self, unit):
        out = set()
        if unit[0] == "s":
            for x, y in self.strip_nodes(unit[1], unit[2]):
                if self.is_ext_node(x, y):
                    continue                     # rebuilt by a boundary block
                out.update(self.pull_sources(x, y))
                if (x, y) in self.solid:
                    out.add((x, y))              # momentum exchange: own slot
            return out
        j = unit[1]
        L = self.L
        for y in range(j * self.per, min((j + 1) * self.per, self.ny)):
            if (L, y) in self.solid:
                continue
            if self.ext == "nn":
                # features: post-stream populations of (L-1-col, y+dy) pulled
                # from their neighbours (reversed at solid nodes)
                for col, dy in itertools.product(range(3), (-1, 0, 1)):
                    fx = L - 1 - col
                    if fx < 0:
                        continue
                    fy = wrap(y + dy, self.ny)
                    for cx, cy in itertools.product((-1, 0, 1), repeat=2):
                        sx = fx - cx
                        if 0 <= sx < self.nx:
                            out.add((sx, wrap(fy - cy, self.ny)))
                out.update(s for s in self.pull_sources(L, y))
            else:
                # characteristic outflow: macros of (L, y), (L-1, y), (L-2, y),
                # (L, y +- 1) and the known pulls
                for dx, dy in ((0, 0), (1, 0), (2, 0), (0, -1), (0, 1), (1, -1), (1, 1)):
                    if L - dx >= 0:
                        out.add((L - dx, wrap(y + dy, self.ny)))
        return out

    def writes(self, unit):
        if unit[0] == "s":
            return {n for n in self.strip_nodes(unit[1], unit[2]) if not self.is_ext_node(*n)}
        j = unit[1]
        return {(self.L, y) for y in range(j * self.per, min((j + 1) * self.per, self.ny))
                if (self.L, y) not in self.solid}

    # ---- the kernels' waits ----
    def east_tiles(self):
        return range(max(0, self.L - 4) // TILE, self.L // TILE + 1)

    def waits(self, unit):
        w = set()
        if unit[0] == "s":
            r, c = unit[1], unit[2]
            for dr, dc in itertools.product((-1, 0, 1), repeat=2):
                w.add(("s", wrap(r + dr, self.nrow), wrap(c + dc, self.tiles)))
            if self.ext and (c * TILE + TILE - 1) >= self.L - 4:
                y0 = r * self.rows
                for y in rows_meeting(y0 - 2, min(y0 + self.rows, self.ny) + 1, self.ny):
                    w.add(("e", y // self.per))
            return w
        y0 = unit[1] * self.per
        for y in rows_meeting(y0 - 2, min(y0 + self.per, self.ny) + 1, self.ny):
            w.add(("e", y // self.per))
            for c in self.east_tiles():
                w.add(("s", y // self.rows, c))
        return w


def needed(lat):
    """Units of step t-1 each unit of step t depends on (RAW and WAR)."""
    units = lat.strips() + lat.ext_blocks()
    deps = {u: set() for u in units}
    for u in units:
        for n in lat.reads(u):
            deps[u].add(lat.owner(*n))           # u reads what owner(n) wrote
    for v in units:
        for n in lat.reads(v):
            deps[lat.owner(*n)].add(v)           # owner(n) overwrites what v read
    return deps


def check(lat):
    deps = needed(lat)
    for u, d in deps.items():
        missing = d - lat.waits(u)
        assert not missing, (lat.nx, lat.ny, lat.rows, lat.ext, lat.per, u, sorted(missing))


def random_solid(nx, ny, rng, frac):
    return {(x, y) for x in range(nx) for y in range(ny) if rng.random() < frac}


@pytest.mark.parametrize("seed", range(6))
def test_waits_cover_every_dependency(seed):
    rng = random.Random(seed)
    cases = 0
    while cases < 25:
        ext = rng.choice([None, "nn", "cbc"])
        periodic = ext is None and rng.random() < 0.5
        nx = rng.choice([1, 2, 3, 5, 127, 128, 129, 131, 132, 133, 200, 255, 256, 260, 390])
        ny = rng.randint(1, 30)
        rows = rng.randint(2, 9)
        per = rng.choice([8, 16]) if ext == "nn" else rng.choice([3, 5, 126, 158])
        if nx * ny > 6000:
            continue
        lat = Lattice(nx, ny, rows, ext, per, periodic, random_solid(nx, ny, rng, 0.1))
        check(lat)
        cases += 1


def test_waits_cover_tall_cbc_blocks():
    """Characteristic-outflow blocks of 158 rows (160 threads, one halo row on
    each side) over several strip rows."""
    for nx, ny, rows in [(131, 400, 40), (5, 333, 16), (260, 170, 24)]:
        check(Lattice(nx, ny, rows, "cbc", 158, False, set()))


def test_a_narrower_rule_misses_dependencies():
    """The check has teeth: waiting only for the strip itself, or dropping the
    boundary blocks' +- 2 rows, leaves dependencies uncovered."""
    lat = Lattice(200, 24, 4, "nn", 8, False, set())

    class OwnStrip(Lattice):
        def waits(self, unit):
            return {unit} if unit[0] == "s" else Lattice.waits(self, unit)

    class NoHalo(Lattice):
        def waits(self, unit):
            if unit[0] == "e":
                y0 = unit[1] * self.per
                return {("e", unit[1])} | {("s", y // self.rows, c)
                                           for y in range(y0, min(y0 + self.per, self.ny))
                                           for c in self.east_tiles()}
            return Lattice.waits(self, unit)

    for cls in (OwnStrip, NoHalo):
        bad = cls(lat.nx, lat.ny, lat.rows, lat.ext, lat.per, False, set())
        with pytest.raises(AssertionError):
            check(bad)
    check(lat)
