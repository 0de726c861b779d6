"""Seeded synthetic inputs: wavenumber fields, point sources and receivers.

This module holds none of the solver's arithmetic; it only builds the
velocity models and right-hand sides that both the CUDA path and its tests
consume.  Every generator is deterministic for a given seed.

Conventions: arrays are ``(ny, nx)`` with x fastest; row ``j = 0`` is the
surface (y = 0) and rows go down in depth, so node (i, j) sits at
x = i h, depth z = j h.
"""

import math

import numpy as np


class Model:
    """A grid, its spacing and the squared wavenumber k^2 = (2 pi f / c)^2."""

    def __init__(self, name, nx, ny, h, k2, velocity=None, freq=None,
                 physical=None):
        self.name, self.nx, self.ny, self.h = name, int(nx), int(ny), float(h)
        self.k2 = np.ascontiguousarray(k2, dtype=np.float64).reshape(ny, nx)
        self.velocity = velocity
        self.freq = freq
        # (nx, ny) of the physical domain when the grid was padded
        self.physical = physical or (self.nx, self.ny)

    @property
    def n(self):
        return self.nx * self.ny

    def kh_max(self):
        return float(np.sqrt(self.k2.max()) * self.h)


def constant_k(n, k):
    """Unit square, constant wavenumber k, n x n nodes, h = 1/(n-1)
    (the MP-2a / MP-2b model problems)."""
    h = 1.0 / (n - 1)
    return Model(f"mp2_n{n}_k{k:g}", n, n, h, np.full((n, n), float(k) ** 2))


def k2_from_velocity(c, freq):
    return (2.0 * math.pi * freq / np.asarray(c, np.float64)) ** 2


def wedge(freq, nx, ny):
    """Three-layer wedge on [0, 600] x [0, 1000] m (depth down).  The layer
    boundaries are straight dipping lines: 2000 m/s above
    z = 400 - x/3, 1500 m/s down to z = 750 - x/4, 3000 m/s below; a node on
    an interface takes the upper layer's velocity."""
    h = 600.0 / (nx - 1)
    if abs(1000.0 / (ny - 1) - h) > 1e-9 * h:
        raise ValueError("wedge grid must have equal spacing in x and z")
    x = np.arange(nx) * h
    z = np.arange(ny)[:, None] * h
    c = np.full((ny, nx), 3000.0)
    c[z <= 750.0 - x / 4.0] = 1500.0
    c[z <= 400.0 - x / 3.0] = 2000.0
    return Model(f"wedge_f{freq:g}_{nx}x{ny}", nx, ny, h,
                 k2_from_velocity(c, freq), velocity=c, freq=freq)


def layered_faulted(nx=2301, ny=751, h=4.0, freq=31.25, seed=0,
                    pad_to=(2305, 769), nlayers=10, vmin=1500.0, vmax=5500.0):
    """Seeded layered-and-faulted velocity model (stands in for a field
    model such as Marmousi, which is not available).

    ``nlayers`` layers from ``vmin`` at the top to ``vmax`` at the bottom;
    each interface is a linear dip of at most 10 degrees plus three random
    sinusoids of amplitude <= 60 m; two normal faults dipping 60 degrees
    shift the interfaces down by a throw of 50-150 m on their hanging wall.
    The grid is padded by edge replication to ``pad_to`` nodes so that it
    coarsens to a small coarsest level.
    """
    rng = np.random.default_rng(seed)
    Lx = (nx - 1) * h
    Lz = (ny - 1) * h
    x = np.arange(nx) * h
    z = np.arange(ny)[:, None] * h
    ninterf = nlayers - 1
    base = np.linspace(0.08 * Lz, 0.92 * Lz, ninterf)
    depth = np.empty((ninterf, nx))
    for l in range(ninterf):
        dip = math.tan(math.radians(rng.uniform(-10.0, 10.0)))
        d = base[l] + dip * (x - 0.5 * Lx) * 0.1
        for _ in range(3):
            amp = rng.uniform(0.0, 60.0)
            lam = rng.uniform(0.1 * Lx, 0.6 * Lx)
            ph = rng.uniform(0.0, 2 * math.pi)
            d = d + amp * np.sin(2 * math.pi * x / lam + ph)
        depth[l] = d
    faults = []
    for _ in range(2):
        x0 = rng.uniform(0.2 * Lx, 0.8 * Lx)
        throw = rng.uniform(50.0, 150.0)
        faults.append((x0, throw))
    cot60 = 1.0 / math.tan(math.radians(60.0))
    count = np.zeros((ny, nx), dtype=np.int64)
    shift = np.zeros((ny, nx))
    for (x0, throw) in faults:
        hanging = x[None, :] > (x0 + z * cot60)
        shift = shift + np.where(hanging, throw, 0.0)
    for l in range(ninterf):
        count += (z > depth[l][None, :] + shift).astype(np.int64)
    vel = np.linspace(vmin, vmax, nlayers)[count]
    px, py = pad_to if pad_to else (nx, ny)
    if px < nx or py < ny:
        raise ValueError("pad_to must not shrink the grid")
    vpad = np.pad(vel, ((0, py - ny), (0, px - nx)), mode="edge")
    return Model(f"layered_{nx}x{ny}_f{freq:g}", px, py, h,
                 k2_from_velocity(vpad, freq), velocity=vpad, freq=freq,
                 physical=(nx, ny))


def gaussian_anomalies(model, rel=0.05, nblobs=3, seed=1):
    """Velocity perturbed by +-rel Gaussian blobs (sigma 5-10% of the
    domain); returns the squared slowness m = 1/c^2 of the perturbed model."""
    rng = np.random.default_rng(seed)
    ny, nx, h = model.ny, model.nx, model.h
    c = np.sqrt((2 * math.pi * model.freq) ** 2 / model.k2)
    xx = np.arange(nx)[None, :] * h
    zz = np.arange(ny)[:, None] * h
    Lx, Lz = (nx - 1) * h, (ny - 1) * h
    pert = np.zeros((ny, nx))
    for b in range(nblobs):
        cx, cz = rng.uniform(0.2, 0.8) * Lx, rng.uniform(0.3, 0.8) * Lz
        sig = rng.uniform(0.05, 0.10) * max(Lx, Lz)
        sign = 1.0 if b % 2 == 0 else -1.0
        pert += sign * rel * np.exp(-((xx - cx) ** 2 + (zz - cz) ** 2)
                                    / (2 * sig * sig))
    return 1.0 / (c * (1.0 + pert)) ** 2


def point_sources(nx, ny, nodes):
    """Unit point sources, one right-hand side per (i, j) node:
    complex128 array (len(nodes), ny, nx)."""
    b = np.zeros((len(nodes), ny, nx), dtype=np.complex128)
    for s, (i, j) in enumerate(nodes):
        b[s, j, i] = 1.0
    return b


def centre_node(nx, ny):
    return ((nx - 1) // 2, (ny - 1) // 2)


def centre_cluster(nx, ny, count, spacing=None):
    """``count`` source nodes on a near-square lattice around the centre."""
    side = int(math.ceil(math.sqrt(count)))
    sp = spacing or max(1, min(nx, ny) // (4 * side))
    ci, cj = centre_node(nx, ny)
    nodes = []
    for s in range(count):
        a, b = s % side, s // side
        nodes.append((ci + (a - side // 2) * sp, cj + (b - side // 2) * sp))
    return nodes


def surface_line(nx, count, first=35, step=35, row=0):
    """``count`` sources on the surface row at i = first + step * s."""
    nodes = [(first + step * s, row) for s in range(count)]
    if nodes and nodes[-1][0] >= nx:
        raise ValueError("surface line runs off the grid")
    return nodes


def surface_receivers(nx, row=0):
    """Flat node indices of a receiver at every node of a row."""
    return (row * nx + np.arange(nx)).astype(np.int32)


def random_complex(shape, seed):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(shape)
            + 1j * rng.standard_normal(shape)).astype(np.complex128)
