"""Seeded synthetic inputs: electrode geometries and parameter sets.

This module holds no arithmetic of the method itself (no stencil, flux,
collision or charge rule).  It builds node-id arrays (0 = fluid, e >= 1 =
electrode e) and the physical parameters of the nanocapacitor workloads, and
is shared by the CUDA path's tests and benchmark and by the oracle's tests.

Arrays are indexed ``[z, y, x]``; flattened, node ``r = x + nx*(y + ny*z)``.

Workloads (lattice units, k_B T = e = 1):

* parallel plates (Sec. "Parallel plate capacitor"): electrode 1 is the layer
  z = 0, electrode 2 the layer z = nz-1, fluid in between, periodic in x, y;
  the interface-to-interface gap is L = nz - 2.
* coaxial cylinders (Sec. "Cylindrical (coaxial) capacitor", Fig. 7): axis at
  ((nx-1)/2, (ny-1)/2) along z; nodes with radius < R1 are electrode 1, nodes
  with radius > R2 electrode 2, fluid between; periodic in all directions.
* porous electrode: seed-placed spheres joined to a backing plate at z = 0
  (electrode 1) facing a counter plate at z = nz-1 (electrode 2).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

SEED = 4732


def bulk_density(debye_length: float, bjerrum: float) -> float:
    """1:1 salt concentration for a Debye length (Eq. lambda with z = +-1):
    lambda_D = (8 pi l_B rho_s)^(-1/2)."""
    return 1.0 / (8.0 * math.pi * bjerrum * debye_length ** 2)


def plates(nx: int, ny: int, nz: int) -> np.ndarray:
    ids = np.zeros((nz, ny, nx), dtype=np.uint8)
    ids[0] = 1
    ids[nz - 1] = 2
    return ids


def coax(nx: int, ny: int, nz: int, r1: float, r2: float) -> np.ndarray:
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    cx, cy = (nx - 1) / 2.0, (ny - 1) / 2.0
    rad = np.sqrt((x - cx) ** 2 + (y - cy) ** 2)
    plane = np.zeros((ny, nx), dtype=np.uint8)
    plane[rad < r1] = 1
    plane[rad > r2] = 2
    return np.repeat(plane[None], nz, axis=0)


def porous(nx: int, ny: int, nz: int, n_spheres: int, rmin: float, rmax: float,
           zmax: float, seed: int = SEED) -> np.ndarray:
    """Spheres with radii U[rmin, rmax] and centres uniform in
    [0,nx) x [0,ny) x [0,zmax), periodic images in x and y, joined to a
    backing plate at z = 0 (electrode 1); counter plate at z = nz-1."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ids = plates(nx, ny, nz)
    zz, yy, xx = np.mgrid[0:nz, 0:ny, 0:nx].astype(np.float32)
    cen = rng.uniform([0, 0, 0], [nx, ny, zmax], size=(n_spheres, 3))
    rad = rng.uniform(rmin, rmax, size=n_spheres)
    solid = np.zeros((nz, ny, nx), dtype=bool)
    for (cx, cy, cz), r in zip(cen, rad):
        dx = np.abs(xx - cx); dx = np.minimum(dx, nx - dx)
        dy = np.abs(yy - cy); dy = np.minimum(dy, ny - dy)
        solid |= dx * dx + dy * dy + (zz - cz) ** 2 <= r * r
    solid[nz - 2:] = False  # keep the counter plate separated by fluid
    solid[nz - 3] = False
    ids[solid & (ids == 0)] = 1
    return ids


def random_blobs(nx: int, ny: int, nz: int, n_elec: int, fill: float, seed: int) -> np.ndarray:
    """Random solid clusters of ``n_elec`` electrodes for parity tests (all
    directions periodic)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ids = np.zeros((nz, ny, nx), dtype=np.uint8)
    target = int(fill * ids.size)
    solid = 0
    while solid < target:
        c = rng.integers(0, [nz, ny, nx])
        r = rng.uniform(0.8, 2.5)
        e = rng.integers(1, n_elec + 1)
        # the ball touches only nodes within 2 of its centre (r < 2.5);
        # periodic distances as the minimum image
        win = [np.unique(np.arange(c[a] - 2, c[a] + 3) % n) for a, n in enumerate((nz, ny, nx))]
        dd = [((w - c[a] + n // 2) % n - n // 2) ** 2 for a, (w, n) in enumerate(zip(win, (nz, ny, nx)))]
        d2 = dd[0][:, None, None] + dd[1][None, :, None] + dd[2][None, None, :]
        sub = ids[np.ix_(*win)]
        hit = (d2 <= r * r) & (sub == 0)
        sub[hit] = e
        ids[np.ix_(*win)] = sub
        solid += int(hit.sum())
    return ids


@dataclass
class Workload:
    """One nanocapacitor lattice and its physical parameters."""
    name: str
    ids: np.ndarray
    n_elec: int
    periodic: tuple
    psi: tuple
    bjerrum: float
    debye: float
    tau: float = 1.0
    D: tuple = (0.05, 0.05)
    z: tuple = (1.0, -1.0)
    e_app: tuple = (0.0, 0.0, 0.0)
    flow: bool = True
    steps: int = 1
    extra: dict = field(default_factory=dict)

    @property
    def shape(self):
        nz, ny, nx = self.ids.shape
        return (nx, ny, nz)

    @property
    def nodes(self) -> int:
        return int(self.ids.size)

    @property
    def rho_bulk(self):
        rs = bulk_density(self.debye, self.bjerrum)
        return tuple(rs for _ in self.z)

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)


def plate_capacitor(nx=4, ny=4, nz=64, *, debye=8.0, bjerrum=4.8, psi=(0.1, 0.2),
                    steps=20000, **kw) -> Workload:
    """4x4x64 parallel-plate nanocapacitor, 1:1 salt, Debye length 8,
    voltage 0.1, fluid initially at rest (l_B = 4.8 as in Fig. 5)."""
    return Workload("plates_%dx%dx%d" % (nx, ny, nz), plates(nx, ny, nz), 2, (1, 1, 0), tuple(psi),
                    bjerrum, debye, steps=steps, **kw)


def coax_capacitor(nx=128, ny=128, nz=4, *, r1=10.0, r2=50.0, debye=5.0, bjerrum=1.2,
                   psi=(0.0, 0.1), steps=20000, **kw) -> Workload:
    """128x128x4 coaxial nanocapacitor, R1 = 10, R2 = 50, Debye length 5,
    l_B = 1.2 (as in Sec. "Potential profile" of the coaxial capacitor)."""
    return Workload("coax_%dx%dx%d" % (nx, ny, nz), coax(nx, ny, nz, r1, r2), 2, (1, 1, 1),
                    tuple(psi), bjerrum, debye, steps=steps,
                    extra={"r1": r1, "r2": r2}, **kw)


def eof_plates(nx=64, ny=64, nz=256, *, debye=16.0, bjerrum=1.44, voltage=0.2, ex=1e-3,
               steps=50000, **kw) -> Workload:
    """64x64x256 electro-osmosis between charged plates: voltage 0.2,
    tangential field 1e-3 along x, Debye length 16, tau = 1, l_B = 1.44."""
    return Workload("eof_%dx%dx%d" % (nx, ny, nz), plates(nx, ny, nz), 2, (1, 1, 0),
                    (0.0, voltage), bjerrum, debye, e_app=(ex, 0.0, 0.0), steps=steps, **kw)


def porous_electrode(nx=256, ny=256, nz=128, *, n_spheres=200, seed=SEED, debye=8.0,
                     bjerrum=1.44, voltage=0.1, steps=2000, **kw) -> Workload:
    """256x256x128 porous electrode of 200 seed-placed spheres of radius
    6-12 in z < 64 on a backing plate, facing a counter plate."""
    ids = porous(nx, ny, nz, n_spheres, 6.0, 12.0, min(64.0, nz / 2.0), seed)
    return Workload("porous_%dx%dx%d" % (nx, ny, nz), ids, 2, (1, 1, 0), (0.0, voltage),
                    bjerrum, debye, flow=False, steps=steps, **kw)


def batch_instances(count=256, seed=SEED):
    """Seed-generated sweep of parallel-plate and coaxial instances: gap
    L_z ~ U{32..512}, cross-section side ~ U{8..64}, Debye length
    log-uniform in [2, 32], voltage ~ U[-0.5, 0.5]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for k in range(count):
        side = int(rng.integers(8, 65))
        gap = int(rng.integers(32, 513))
        debye = float(math.exp(rng.uniform(math.log(2.0), math.log(32.0))))
        volt = float(rng.uniform(-0.5, 0.5))
        if k % 2 == 0:
            w = plate_capacitor(side, side, gap + 2, debye=debye, bjerrum=1.44, psi=(0.0, volt))
        else:
            r2 = side / 2.0 - 2.0
            r1 = max(1.0, r2 / 5.0)
            w = coax_capacitor(side, side, gap, r1=r1, r2=r2, debye=debye, bjerrum=1.44,
                               psi=(0.0, volt))
        out.append(w.with_(name="inst%03d_%s" % (k, w.name)))
    return out


def porous_crop(nx=32, ny=32, nz=16, *, seed=SEED, debye=8.0, bjerrum=1.44, voltage=0.1,
                steps=2000, **kw) -> Workload:
    """32x32x16 crop of the porous electrode made by the same generator
    (spheres on a backing plate, counter plate at z = nz-1), scaled to the
    box: 2 spheres of radius 3-5 in z < 8.  Used for the gradient checks."""
    ids = porous(nx, ny, nz, 2, 3.0, 5.0, min(8.0, nz / 2.0), seed)
    return Workload("porous_crop_%dx%dx%d" % (nx, ny, nz), ids, 2, (1, 1, 0), (0.0, voltage),
                    bjerrum, debye, flow=False, steps=steps, **kw)
