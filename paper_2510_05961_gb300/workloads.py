"""Seeded synthetic workloads shaped like the MSM benchmarks of arXiv 2510.05961.

This module only draws positions, charges and cells (numpy ``default_rng``); it
holds none of the method's arithmetic (no grids, levels, kernels or stencils),
so the CUDA path and the FP64 oracle can both take their inputs from it.

The paper's own benchmark structures (PACKMOL packings, Sec. 4.2) are not
available, so every workload here is a stand-in with the shape and statistics
of the corresponding experiment: uniform random positions in cubic boxes,
charge-neutral charge sets, a rigid-water box and a rock-salt supercell.

Positions and charges are returned as float32 (the precision the GPU path
reads); the oracle promotes exactly these values to float64.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Workload:
    """One MSM problem: atoms, an orthorhombic cell and the method settings."""

    name: str
    pos: np.ndarray              # (n, 3) float32, Cartesian, Angstrom-like units
    q: np.ndarray                # (n,) float32
    cell: tuple                  # (Lx, Ly, Lz) box edge lengths
    pbc: tuple                   # (px, py, pz) 0 = open, 1 = periodic
    h: float                     # target level-1 grid spacing
    a: float                     # level-zero cutoff r_cut^(0)
    p: int                       # B-spline order
    levels: int = 0              # 0 = planner's rule
    grid_override: tuple = (0, 0, 0)
    qi_mode: int = 0             # 0 = minimal quasi-interpolation, 1 = exact interpolation
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])


def _neutral_pm1(rng, n):
    """n charges, half +1 and half -1 (one extra +1 if n is odd), shuffled."""
    q = np.ones(n, dtype=np.float64)
    q[: n // 2] = -1.0
    rng.shuffle(q)
    return q


def open_cluster(n=1000, side=30.0, seed=1000, h=2.5, a=10.0, p=4, levels=3):
    """Open cluster: n charges uniform in a cube, +1/-1 with zero net charge."""
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0.0, side, size=(n, 3))
    q = _neutral_pm1(rng, n)
    return Workload("open_cluster_n%d" % n, pos.astype(np.float32), q.astype(np.float32),
                    (side, side, side), (0, 0, 0), h, a, p, levels)


def random_box(n, density=0.1, seed=None, h=2.0, a=8.0, p=4, pbc=(1, 1, 1)):
    """Periodic cube at fixed density, uniform positions, +/-1 charges, neutral.

    This is the linear-scaling sweep: n = 1000 * 2**k, density 0.1 per A^3.
    """
    if seed is None:
        seed = 3000 + int(round(math.log2(max(n, 1) / 1000.0))) if n >= 1000 else 3000 + n
    rng = np.random.default_rng(seed)
    L = (n / density) ** (1.0 / 3.0)
    pos = rng.uniform(0.0, L, size=(n, 3))
    q = _neutral_pm1(rng, n)
    return Workload("random_box_n%d" % n, pos.astype(np.float32), q.astype(np.float32),
                    (L, L, L), tuple(pbc), h, a, p)


def _random_rotations(rng, m):
    """m uniformly random rotation matrices (random unit quaternions)."""
    u1, u2, u3 = rng.uniform(size=(3, m))
    qw = np.sqrt(1 - u1) * np.sin(2 * np.pi * u2)
    qx = np.sqrt(1 - u1) * np.cos(2 * np.pi * u2)
    qy = np.sqrt(u1) * np.sin(2 * np.pi * u3)
    qz = np.sqrt(u1) * np.cos(2 * np.pi * u3)
    R = np.empty((m, 3, 3))
    R[:, 0, 0] = 1 - 2 * (qy * qy + qz * qz)
    R[:, 0, 1] = 2 * (qx * qy - qz * qw)
    R[:, 0, 2] = 2 * (qx * qz + qy * qw)
    R[:, 1, 0] = 2 * (qx * qy + qz * qw)
    R[:, 1, 1] = 1 - 2 * (qx * qx + qz * qz)
    R[:, 1, 2] = 2 * (qy * qz - qx * qw)
    R[:, 2, 0] = 2 * (qx * qz - qy * qw)
    R[:, 2, 1] = 2 * (qy * qz + qx * qw)
    R[:, 2, 2] = 1 - 2 * (qx * qx + qy * qy)
    return R


def water_box(nmol=4096, L=49.6, seed=2000, min_oo=2.5, h=1.5, a=9.0, p=6):
    """Rigid 3-site water molecules in a periodic cube.

    O sites by random sequential addition with a minimum periodic O-O distance,
    random orientations, O-H 0.9572, H-O-H 104.52 deg, q_O = -0.834, q_H = +0.417.
    """
    rng = np.random.default_rng(seed)
    nc = max(1, int(L // min_oo))
    ce = L / nc
    cells = {}
    O = np.empty((nmol, 3))
    k = 0
    tries = 0
    while k < nmol:
        tries += 1
        if tries > 200 * nmol:
            raise RuntimeError("water_box: random sequential addition did not converge")
        x = rng.uniform(0.0, L, size=3)
        c = tuple((x // ce).astype(int) % nc)
        ok = True
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    key = ((c[0] + dx) % nc, (c[1] + dy) % nc, (c[2] + dz) % nc)
                    for j in cells.get(key, ()):
                        d = O[j] - x
                        d -= L * np.round(d / L)
                        if d @ d < min_oo * min_oo:
                            ok = False
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if not ok:
                break
        if ok:
            O[k] = x
            cells.setdefault(c, []).append(k)
            k += 1
    roh = 0.9572
    half = math.radians(104.52) / 2.0
    h1 = np.array([roh * math.sin(half), 0.0, roh * math.cos(half)])
    h2 = np.array([-roh * math.sin(half), 0.0, roh * math.cos(half)])
    R = _random_rotations(rng, nmol)
    H1 = O + R @ h1
    H2 = O + R @ h2
    pos = np.empty((3 * nmol, 3))
    pos[0::3] = O
    pos[1::3] = H1
    pos[2::3] = H2
    q = np.empty(3 * nmol)
    q[0::3] = -0.834
    q[1::3] = 0.417
    q[2::3] = 0.417
    return Workload("water_box_%dmol" % nmol, pos.astype(np.float32), q.astype(np.float32),
                    (L, L, L), (1, 1, 1), h, a, p)


def rocksalt(ncell=32, a0=5.64, sigma=0.1, qsigma=0.1, seed=4000, h=2.0, a=8.0, p=4):
    """Rock-salt supercell with Gaussian displacements and perturbed charges.

    Charges are +/-(1 + qsigma * N(0,1)), shifted to zero net charge.
    """
    rng = np.random.default_rng(seed)
    basis_p = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]])
    basis_m = np.array([[.5, 0, 0], [0, .5, 0], [0, 0, .5], [.5, .5, .5]])
    g = np.arange(ncell)
    cells = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 1, 3)
    frac = np.concatenate([(cells + basis_p).reshape(-1, 3), (cells + basis_m).reshape(-1, 3)])
    sign = np.concatenate([np.ones(4 * ncell ** 3), -np.ones(4 * ncell ** 3)])
    pos = frac * a0 + rng.normal(0.0, sigma, size=frac.shape)
    q = sign * (1.0 + qsigma * rng.normal(size=sign.shape))
    q -= q.mean()
    L = ncell * a0
    return Workload("rocksalt_%dcubed" % ncell, pos.astype(np.float32), q.astype(np.float32),
                    (L, L, L), (1, 1, 1), h, a, p)


def nacl_crystal(ncell=1, a0=1.0):
    """Ideal rock-salt crystal (conventional cell replicated ncell^3 times), +/-1 charges.

    Returns (pos float64, q float64, L). Used for the Madelung constant.
    """
    basis_p = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]])
    basis_m = np.array([[.5, 0, 0], [0, .5, 0], [0, 0, .5], [.5, .5, .5]])
    g = np.arange(ncell)
    cells = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 1, 3)
    frac = np.concatenate([(cells + basis_p).reshape(-1, 3), (cells + basis_m).reshape(-1, 3)])
    q = np.concatenate([np.ones(4 * ncell ** 3), -np.ones(4 * ncell ** 3)])
    return frac * a0, q, ncell * a0


def batch_systems(nsys=512, seed=5000, nmin=20, nmax=4000, density=0.08, h=2.0, a=8.0, p=4):
    """Many independent systems of uneven size and mixed periodicity.

    Sizes log-uniform in [nmin, nmax]; system s is open (s % 3 == 0), a slab
    periodic in x and y (s % 3 == 1) or fully periodic (s % 3 == 2). Cube side
    (n / density)^(1/3); charges N(0, 0.5) shifted to zero sum.
    """
    rng = np.random.default_rng(seed)
    out = []
    for s in range(nsys):
        n = int(math.floor(math.exp(rng.uniform(math.log(nmin), math.log(nmax)))))
        side = (n / density) ** (1.0 / 3.0)
        pos = rng.uniform(0.0, side, size=(n, 3))
        q = rng.normal(0.0, 0.5, size=n)
        q -= q.mean()
        kind = s % 3
        pbc = (0, 0, 0) if kind == 0 else ((1, 1, 0) if kind == 1 else (1, 1, 1))
        out.append(Workload("batch_%d" % s, pos.astype(np.float32), q.astype(np.float32),
                            (side, side, side), pbc, h, a, p))
    return out


def redraw(w, seed, qsigma=0.5):
    """Same system shape (cell, periodicity, settings, atom count), new inputs:
    positions uniform in the cell, charges N(0, qsigma) shifted to zero sum.
    A plan made for w serves the redrawn system too."""
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0.0, 1.0, size=(w.n, 3)) * np.asarray(w.cell, np.float64)
    q = rng.normal(0.0, qsigma, size=w.n)
    q -= q.mean()
    return Workload(w.name + "_redrawn", pos.astype(np.float32), q.astype(np.float32), w.cell, w.pbc, w.h, w.a,
                    w.p, w.levels, w.grid_override, w.qi_mode)


def lattice_on_grid(ncell=4, a0=4.0, pbc=(1, 1, 1), seed=6000, qsigma=0.1, h=2.0, a=8.0, p=4):
    """Undisplaced rock-salt lattice whose sites fall exactly on level-1 grid
    points and binning-cell faces (with h = a0 / 2 and a power-of-two grid),
    charges +/-(1 + qsigma N(0,1)) shifted to zero sum. Along an open axis the
    crystal gets one more layer of sites, so that its sites lie exactly on both
    faces of the cell (s = 0 and s = 1, i.e. x = 0 and x = L)."""
    rng = np.random.default_rng(seed)
    m = 2 * ncell
    g = np.arange(m)
    idx = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    cell = [ncell * a0] * 3
    extra = []
    # open axes: add the layer at the far face (index m) along each open axis
    for d in range(3):
        if not pbc[d]:
            layer = idx[idx[:, d] == 0].copy()
            layer[:, d] = m
            extra.append(layer)
    if extra:
        idx = np.unique(np.concatenate([idx] + extra), axis=0)
    pos = idx * (0.5 * a0)
    sign = np.where(idx.sum(1) % 2 == 0, 1.0, -1.0)
    q = sign * (1.0 + qsigma * rng.normal(size=len(sign)))
    q -= q.mean()
    return Workload("lattice_on_grid_%d" % ncell, pos.astype(np.float32), q.astype(np.float32), tuple(cell),
                    tuple(pbc), h, a, p)


def sheet(n=400, side=24.0, thickness=2.0, periodic=True, seed=7000, h=0.8, a=8.0, p=8):
    """A two-dimensional arrangement: n charges in the plane z = 0 of a cell
    side x side x thickness (periodic in x, y and open along z, a slab of zero
    thickness; or open along all axes), jittered square lattice (no two charges
    closer than 0.4 of the spacing), charges +/-1 alternating on the lattice,
    neutral for even n."""
    rng = np.random.default_rng(seed)
    m = int(math.ceil(math.sqrt(n)))
    sp = side / m
    idx = np.stack(np.meshgrid(np.arange(m), np.arange(m), indexing="ij"), axis=-1).reshape(-1, 2)[:n]
    pos = np.zeros((n, 3))
    pos[:, :2] = (idx + 0.5 + rng.uniform(-0.3, 0.3, size=(n, 2))) * sp
    q = np.where(idx.sum(1) % 2 == 0, 1.0, -1.0)
    q -= q.mean()
    return Workload("sheet_%d" % n, pos.astype(np.float32), q.astype(np.float32), (side, side, thickness),
                    (1, 1, 0) if periodic else (0, 0, 0), h, a, p)


def chain(n=200, length=80.0, width=2.0, periodic=True, seed=7100, h=0.8, a=8.0, p=8):
    """A one-dimensional arrangement: n charges on the line x = y = 0 of a cell
    width x width x length (periodic along z and open across, a wire of zero
    width; or open along all axes), jittered lattice along z, charges +/-1
    alternating, neutral for even n."""
    rng = np.random.default_rng(seed)
    sp = length / n
    pos = np.zeros((n, 3))
    pos[:, 2] = (np.arange(n) + 0.5 + rng.uniform(-0.3, 0.3, size=n)) * sp
    q = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    q -= q.mean()
    return Workload("chain_%d" % n, pos.astype(np.float32), q.astype(np.float32), (width, width, length),
                    (0, 0, 1) if periodic else (0, 0, 0), h, a, p)


def scaling_sizes(kmax=14):
    """The sweep sizes n = 1000 * 2**k, k = 0 .. kmax."""
    return [1000 * 2 ** k for k in range(kmax + 1)]
