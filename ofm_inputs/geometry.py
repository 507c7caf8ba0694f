"""Synthetic geometries standing in for the paper's alkane and P3HT systems.

The paper's inputs (MD structures and charge-patching potentials, Sec. III and
Sec. IV) are not available.  Each workload here is a periodic real-space grid
with a potential V(r) that is a sum of Gaussian wells, plus a list of cuboid
fragment boxes (Sec. II: each fragment is a molecule embedded in a box).

Conventions shared by every consumer:
  * grid point (i, j, k) sits at r = h * (i, j, k); arrays are indexed
    V[k, j, i] (z, y, x) so that x is the fastest-varying index in memory;
  * a well is (x, y, z, D, w) and contributes -D * exp(-d^2 / (2 w^2)) with d
    the minimum-image distance, truncated where d > 8 w (exp(-32) ~ 1e-14);
  * a fragment box is off + [0, ext) taken modulo the grid in each dimension.

Everything random is drawn from numpy.random.default_rng(seed).
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

WELL_CUTOFF_WIDTHS = 8.0


@dataclass(frozen=True)
class Grid:
    n: tuple  # (nx, ny, nz)
    h: float

    @property
    def npoints(self) -> int:
        return int(self.n[0] * self.n[1] * self.n[2])

    @property
    def lengths(self) -> tuple:
        return tuple(self.h * ni for ni in self.n)


@dataclass(frozen=True)
class Fragment:
    off: tuple  # (x, y, z) grid offset of the box corner
    ext: tuple  # (ex, ey, ez) box extent in grid points
    n_states: int


@dataclass(frozen=True)
class WindowRule:
    """How the energy window of the final generalized eigenproblem is chosen.

    kind == "from_lowest": [E_1, E_1 + width] with E_1 the lowest eigenvalue.
    kind == "above_gap":   [E_{n_occ+1}, E_{n_occ+1} + width]  (1-based).
    kind == "around_gap":  [E_{n_occ} - width, E_{n_occ+1} + width].
    """
    kind: str
    width: float
    n_occ: int = 0


@dataclass
class Workload:
    name: str
    grid: Grid
    wells: np.ndarray          # (W, 5): x, y, z, depth D, width w  [bohr, Ha]
    frags: list                # list[Fragment]
    window: WindowRule
    precision: str             # precision the workload is specified in
    description: str = ""
    _V: np.ndarray = field(default=None, repr=False)

    @property
    def V(self) -> np.ndarray:
        if self._V is None:
            self._V = gaussian_potential(self.grid, self.wells)
        return self._V

    @property
    def basis_size(self) -> int:
        return int(sum(f.n_states for f in self.frags))

    def fragment_atoms(self) -> list:
        """The atoms of each fragment: the centres (bohr) of the wells that
        lie inside its box (periodic), one (k, 3) array per fragment.  This
        is what the distance cutoff between fragments is measured on."""
        return fragment_atoms(self.grid, self.frags, self.wells)


def fragment_atoms(grid: Grid, frags, wells) -> list:
    """Well centres inside each periodic box off + [0, ext) (grid points of
    spacing h), as one (k, 3) array per box."""
    xyz = np.asarray(wells, dtype=np.float64).reshape(-1, 5)[:, :3] if len(wells) else np.zeros((0, 3))
    out = []
    for f in frags:
        inside = np.ones(len(xyz), dtype=bool)
        for d in range(3):
            u = np.mod(xyz[:, d] / grid.h - f.off[d], grid.n[d])
            inside &= u < f.ext[d]
        out.append(xyz[inside].copy())
    return out


def gaussian_potential(grid: Grid, wells: np.ndarray,
                       cutoff: float = WELL_CUTOFF_WIDTHS) -> np.ndarray:
    """V[z, y, x] = -sum_i D_i exp(-d_min(r, R_i)^2 / (2 w_i^2)), float64."""
    nx, ny, nz = grid.n
    h = grid.h
    L = grid.lengths
    V = np.zeros((nz, ny, nx), dtype=np.float64)
    for (cx, cy, cz, D, w) in np.asarray(wells, dtype=np.float64):
        rad = cutoff * w
        axes = []
        for c, n, Ld in ((cx, nx, L[0]), (cy, ny, L[1]), (cz, nz, L[2])):
            r = int(math.ceil(rad / h))
            if 2 * r + 1 >= n:
                idx = np.arange(n)
                d = np.mod(idx * h - c + 0.5 * Ld, Ld) - 0.5 * Ld
            else:
                ci = int(math.floor(c / h))
                ii = np.arange(ci - r, ci + r + 2)
                d = ii * h - c
                idx = np.mod(ii, n)
            axes.append((idx, d))
        (ix, dx), (iy, dy), (iz, dz) = axes
        d2 = dz[:, None, None] ** 2 + dy[None, :, None] ** 2 + dx[None, None, :] ** 2
        val = np.where(d2 <= rad * rad, -D * np.exp(-d2 / (2.0 * w * w)), 0.0)
        V[np.ix_(iz, iy, ix)] += val
    return V


# --------------------------------------------------------------------------
# Workload definitions
# --------------------------------------------------------------------------

def _tiny(seed: int = 0) -> Workload:
    """32x12x12 grid, 8 jittered wells along x, 4 half-overlapping boxes."""
    grid = Grid((32, 12, 12), 0.5)
    rng = np.random.default_rng(seed)
    Lx, Ly, Lz = grid.lengths
    xs = (np.arange(8) + 0.5) * (Lx / 8.0)
    pos = np.stack([xs, np.full(8, Ly / 2), np.full(8, Lz / 2)], axis=1)
    pos = pos + rng.uniform(-0.3, 0.3, size=(8, 3))
    wells = np.concatenate([pos, np.ones((8, 1)), np.ones((8, 1))], axis=1)
    frags = [Fragment((8 * a, 0, 0), (16, 12, 12), 6) for a in range(4)]
    return Workload("tiny_32x12x12", grid, wells, frags,
                    WindowRule("from_lowest", 0.5), "f64",
                    "8 Gaussian wells (D=1 Ha, w=1 bohr), 4 boxes 16x12x12, 6 states")


def tiny_fragments_of(n_wells: int, seed: int = 0) -> Workload:
    """The tiny workload's grid and wells with fragments of n_wells
    consecutive wells (monomer-, dimer-, trimer-like for 1, 2, 3): one box per
    starting well (periodic), 4n + 4 points wide with 2 bohr of margin on each
    side, one state per well."""
    base = _tiny(seed)
    s = int(n_wells)
    frags = [Fragment(((4 * i - 2) % base.grid.n[0], 0, 0), (4 * s + 4, 12, 12), s) for i in range(8)]
    return Workload(f"tiny_{s}wells", base.grid, base.wells, frags,
                    WindowRule("from_lowest", 0.5), "f64",
                    f"tiny grid and wells, 8 boxes of {s} consecutive wells, {s} states each")


def _alkane_chain(seed: int = 0) -> Workload:
    """256x32x32 grid, zig-zag chain of 64 C-like and 128 H-like wells."""
    grid = Grid((256, 32, 32), 0.5)
    wells = []
    for k in range(64):
        s = 1.0 if k % 2 == 0 else -1.0
        xc, yc, zc = (k + 0.5) * 2.0, 8.0 + s * 0.6, 8.0
        wells.append((xc, yc, zc, 1.2, 0.9))
        for dz in (1.7, -1.7):
            wells.append((xc, yc + s * 1.2, zc + dz, 0.6, 0.6))
    wells = np.array(wells, dtype=np.float64)
    if seed:
        rng = np.random.default_rng(seed)
        wells[:, :3] += rng.uniform(-0.1, 0.1, size=(len(wells), 3))
    frags = [Fragment((8 * a, 0, 0), (16, 32, 32), 32) for a in range(31)]
    return Workload("alkane_chain_256x32x32", grid, wells, frags,
                    WindowRule("above_gap", 0.3, n_occ=len(wells)), "f32",
                    "64 C-like (1.2 Ha, 0.9 bohr) + 128 H-like (0.6 Ha, 0.6 bohr) wells; "
                    "31 boxes 16x32x32 at x stride 8, 32 states each")


def _self_avoiding_chains(rng, L, n_chains, n_per_chain, step, min_dist,
                          max_retries=100):
    """Random walks with uniform step directions; a step landing within
    min_dist (minimum image) of any placed well is redrawn, and after
    max_retries failures the chain restarts from a fresh random origin."""
    L = np.asarray(L, dtype=np.float64)
    cell = min_dist
    ncell = np.maximum((L // cell).astype(int), 1)
    csize = L / ncell
    buckets: dict = {}
    placed = []

    def key(p):
        return tuple((np.floor(np.mod(p, L) / csize).astype(int) % ncell).tolist())

    def clash(p):
        k = key(p)
        for ox in (-1, 0, 1):
            for oy in (-1, 0, 1):
                for oz in (-1, 0, 1):
                    kk = ((k[0] + ox) % ncell[0], (k[1] + oy) % ncell[1], (k[2] + oz) % ncell[2])
                    for q in buckets.get(kk, ()):
                        d = np.mod(p - q + 0.5 * L, L) - 0.5 * L
                        if d @ d < min_dist * min_dist:
                            return True
        return False

    def add(p):
        buckets.setdefault(key(p), []).append(p)

    chains = []
    for _ in range(n_chains):
        while True:
            chain = []
            p = rng.uniform(0, 1, size=3) * L
            if clash(p):
                continue
            chain.append(p)
            local: dict = {}
            ok = True
            # tentative wells are checked against placed chains and this chain
            while len(chain) < n_per_chain:
                for _try in range(max_retries):
                    v = rng.normal(size=3)
                    v /= np.linalg.norm(v)
                    q = np.mod(chain[-1] + step * v, L)
                    if clash(q):
                        continue
                    bad = False
                    for c in chain[:-1]:
                        d = np.mod(q - c + 0.5 * L, L) - 0.5 * L
                        if d @ d < min_dist * min_dist:
                            bad = True
                            break
                    if not bad:
                        chain.append(q)
                        break
                else:
                    ok = False
                    break
            if ok:
                break
        for p in chain:
            add(p)
            placed.append(p)
        chains.append(np.array(chain))
    return chains


def _box_around(points, grid: Grid, margin: float, lo: int, hi: int, mult: int = 8):
    """Cuboid of grid points around a set of (periodic) positions."""
    L = np.asarray(grid.lengths)
    c0 = points[0]
    rel = np.mod(points - c0 + 0.5 * L, L) - 0.5 * L
    mn, mx = rel.min(axis=0), rel.max(axis=0)
    centre = c0 + 0.5 * (mn + mx)
    off, ext = [], []
    for d in range(3):
        span = (mx[d] - mn[d] + 2 * margin) / grid.h
        e = int(math.ceil(span / mult) * mult)
        e = max(lo, min(hi, e))
        e = min(e, grid.n[d])
        o = int(round(centre[d] / grid.h - 0.5 * e)) % grid.n[d]
        off.append(o)
        ext.append(e)
    return tuple(off), tuple(ext)


def _box_overlap_fraction(grid: Grid, fa, fb) -> float:
    """Shared grid points of two periodic boxes over the smaller box's points."""
    cnt = 1
    for d in range(3):
        sa = set(((fa.off[d] + np.arange(fa.ext[d])) % grid.n[d]).tolist())
        sb = set(((fb.off[d] + np.arange(fb.ext[d])) % grid.n[d]).tolist())
        cnt *= len(sa & sb)
    return cnt / min(np.prod(fa.ext), np.prod(fb.ext))


def _amorphous_polymer(seed: int = 0) -> Workload:
    """128^3 grid, 800 wells on 8 self-avoiding chains, uneven boxes
    overlapping their chain neighbour by 30-60 %."""
    grid = Grid((128, 128, 128), 0.5)
    rng = np.random.default_rng(seed)
    chains = _self_avoiding_chains(rng, grid.lengths, 8, 100, 1.45, 1.2)
    wells, frags = [], []
    seg = 10
    for ch in chains:
        D = rng.uniform(0.6, 1.2, size=len(ch))
        w = rng.uniform(0.6, 1.0, size=len(ch))
        for p, d, ww in zip(ch, D, w):
            wells.append((p[0], p[1], p[2], d, ww))
        # consecutive segments of 10 wells; each next segment starts at the
        # first well whose box shares at most 60 % of the smaller box with
        # the previous fragment's box (boxes: bounding box + U(2, 7) bohr of
        # margin, edges multiples of 8 points in [16, 40])
        start, prev = 0, None
        while start + seg <= len(ch):
            margin = rng.uniform(2.0, 7.0)
            n_states = int(rng.integers(8, 65))
            s0 = start
            while True:
                off, ext = _box_around(ch[s0:s0 + seg], grid, margin, 16, 40)
                f = Fragment(off, ext, n_states)
                if prev is None or s0 + seg >= len(ch) or _box_overlap_fraction(grid, prev, f) <= 0.6:
                    break
                s0 += 1
            if prev is not None and s0 + seg > len(ch):
                break
            frags.append(f)
            prev = f
            start = s0 + 1
    return Workload("amorphous_polymer_128c", grid, np.array(wells), frags,
                    WindowRule("above_gap", 0.3, n_occ=len(wells)), "f32",
                    "800 wells on 8 self-avoiding chains (1.45 bohr steps), "
                    "boxes 16^3..40^3 overlapping their chain neighbour by at most 60 %, "
                    "states U{8..64}")


def _chains_scaled(seed: int = 0) -> Workload:
    """192^3 grid, 14 alkane-like chains (C backbone + 2 H per C), ~4000 boxes."""
    grid = Grid((192, 192, 192), 0.5)
    rng = np.random.default_rng(seed)
    backbones = _self_avoiding_chains(rng, grid.lengths, 14, 64, 2.0, 1.6)
    L = np.asarray(grid.lengths)
    wells, frags = [], []
    per_chain = int(round(4000 / 14))
    for bb in backbones:
        for k, p in enumerate(bb):
            wells.append((p[0], p[1], p[2], 1.2, 0.9))
            v = rng.normal(size=3)
            v /= np.linalg.norm(v)
            for s in (1.0, -1.0):
                q = np.mod(p + s * 1.7 * v, L)
                wells.append((q[0], q[1], q[2], 0.6, 0.6))
        # fragment centres at uniform arc length along the unwrapped backbone
        steps = np.mod(np.diff(bb, axis=0) + 0.5 * L, L) - 0.5 * L
        unwrapped = np.concatenate([bb[:1], bb[:1] + np.cumsum(steps, axis=0)])
        seglen = np.linalg.norm(steps, axis=1)
        arc = np.concatenate([[0.0], np.cumsum(seglen)])
        for t in np.linspace(0.0, arc[-1], per_chain):
            i = min(int(np.searchsorted(arc, t, side="right")) - 1, len(seglen) - 1)
            f = (t - arc[i]) / seglen[i]
            c = unwrapped[i] + f * steps[i]
            e = int(rng.choice([24, 28, 32]))
            off = tuple(int(round(c[d] / grid.h - 0.5 * e)) % grid.n[d] for d in range(3))
            frags.append(Fragment(off, (e, e, e), 48))
    return Workload("chains_scaled_192c", grid, np.array(wells), frags,
                    WindowRule("above_gap", 0.3, n_occ=len(wells)), "f32",
                    "14 chains x 64 C-like wells + 2 H-like each; ~4000 boxes "
                    "24^3..32^3 at uniform arc length, 48 states")


def lattice_workload(cells=(16, 8, 8), seed: int = 0, states: int = 96) -> Workload:
    """Boxes of 40^3 points on a periodic lattice of stride 24 (40 % overlap
    per dimension), one box per lattice cell, on a grid of 24 points per cell
    (spacing 0.5 bohr); wells on self-avoiding random-walk chains of 313
    wells (1.45 bohr steps), 64 chains per 16x8x8 cells (scaled with the
    volume, at least one), depth U(0.6, 1.2) Ha, width U(0.6, 1.0) bohr.
    cells=(16, 8, 8) is the large 384x192x192 workload; smaller lattices keep
    its box shape, overlap and state count."""
    cx, cy, cz = (int(c) for c in cells)
    grid = Grid((24 * cx, 24 * cy, 24 * cz), 0.5)
    rng = np.random.default_rng(seed)
    n_chains = max(1, int(round(64 * cx * cy * cz / 1024)))
    chains = _self_avoiding_chains(rng, grid.lengths, n_chains, 313, 1.45, 1.2)
    wells = []
    for ch in chains:
        D = rng.uniform(0.6, 1.2, size=len(ch))
        w = rng.uniform(0.6, 1.0, size=len(ch))
        for p, d, ww in zip(ch, D, w):
            wells.append((p[0], p[1], p[2], d, ww))
    frags = [Fragment((24 * i, 24 * j, 24 * k), (40, 40, 40), states)
             for k in range(cz) for j in range(cy) for i in range(cx)]
    name = ("large_lattice_384x192x192" if (cx, cy, cz) == (16, 8, 8)
            else f"lattice_{grid.n[0]}x{grid.n[1]}x{grid.n[2]}")
    return Workload(name, grid, np.array(wells), frags,
                    WindowRule("around_gap", 0.2, n_occ=len(wells)), "f32",
                    f"~{len(wells)} wells on {n_chains} self-avoiding chains; {len(frags)} boxes "
                    f"40^3 on a {cx}x{cy}x{cz} lattice of stride 24, {states} states")


def _large_lattice(seed: int = 0) -> Workload:
    """384x192x192 grid, ~20000 wells on 64 chains, 1024 boxes 40^3 stride 24."""
    return lattice_workload((16, 8, 8), seed)


def _lattice_4x4x4(seed: int = 0) -> Workload:
    """96^3 grid: 4x4x4 cells of the large lattice (64 boxes 40^3, stride 24,
    96 states), a few-GB case of the same kernels' shapes."""
    return lattice_workload((4, 4, 4), seed)


WORKLOADS = {
    "tiny": _tiny,
    "alkane": _alkane_chain,
    "polymer": _amorphous_polymer,
    "scaled": _chains_scaled,
    "large": _large_lattice,
    "lattice4": _lattice_4x4x4,
}


def make_workload(name: str, seed: int = 0) -> Workload:
    return WORKLOADS[name](seed)


def small_workload(grid_n=(16, 8, 8), h=0.5, frags=None, n_wells=4, depth=1.0,
                   width=1.0, seed=0, V_shift=0.0, zero_potential=False) -> Workload:
    """Small seeded case for unit tests: wells spread along x, random jitter."""
    grid = Grid(tuple(grid_n), h)
    rng = np.random.default_rng(seed)
    Lx, Ly, Lz = grid.lengths
    xs = (np.arange(n_wells) + 0.5) * (Lx / n_wells)
    pos = np.stack([xs, np.full(n_wells, Ly / 2), np.full(n_wells, Lz / 2)], axis=1)
    pos = pos + rng.uniform(-0.3, 0.3, size=(n_wells, 3))
    wells = np.concatenate([pos, np.full((n_wells, 1), depth),
                            np.full((n_wells, 1), width)], axis=1)
    if frags is None:
        nx, ny, nz = grid.n
        frags = [Fragment((0, 0, 0), (nx // 2, ny, nz), 4),
                 Fragment((nx // 4, 0, 0), (nx // 2, ny, nz), 4),
                 Fragment((nx // 2, 0, 0), (nx // 2, ny, nz), 4)]
    wl = Workload(f"small_{grid_n[0]}x{grid_n[1]}x{grid_n[2]}", grid, wells, list(frags),
                  WindowRule("from_lowest", 0.5), "f64", "unit-test case")
    V = np.zeros(grid.n[::-1]) if zero_potential else gaussian_potential(grid, wells)
    wl._V = V + V_shift
    return wl


def random_states(grid: Grid, frag: Fragment, seed: int, dtype=np.float64) -> np.ndarray:
    """Seeded random fragment states: (P_a, n_a) column-major-by-state array,
    point order x fastest within the box.  Used where the assembly is tested
    on arbitrary (non-eigen) states."""
    rng = np.random.default_rng(seed)
    P = int(frag.ext[0] * frag.ext[1] * frag.ext[2])
    return rng.standard_normal((P, frag.n_states)).astype(dtype) / math.sqrt(P)
