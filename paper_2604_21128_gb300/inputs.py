"""Seeded synthetic inputs for the 2D QLA workloads.

This module holds only input generation: the refractive-index map n(x, y)
and the numbers that describe each workload (grid, spacing, steps, packet
parameters).  It contains none of the method's arithmetic; the packet field
itself is computed separately by the CUDA library (``qla_set_packet``) and by
the oracle.  Both the tests and the benchmark draw their inputs from here.

Medium recipe (Sec. V-B: an ellipse with a thin continuous boundary layer in
which n rises from the outside value to the inside value; also the inverse
"vacuum bubble" in a uniform dielectric):
    X, Y   = coordinates in the frame of the ellipse (rotated by ``angle``,
             counter-clockwise from +x), minimum image on the periodic box
    rho    = sqrt((X/a)^2 + (Y/b)^2)
    s      = (rho - 1) / |grad rho|      (approximate signed distance)
    n      = n_out + (n_in - n_out) * (1 - tanh(s / edge)) / 2
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

BATCH_SEED = 20261203


def _min_image(d, L):
    return (d + 0.5 * L) % L - 0.5 * L


def ellipse_medium(nx: int, ny: int, delta: float, a: float, b: float,
                   n_in: float, n_out: float, edge: float, angle: float = 0.0,
                   centre=None) -> np.ndarray:
    """Index map (ny, nx) float64 of a smooth ellipse; lengths in physical
    units (cells * delta).  ``centre`` defaults to the box centre.  Built in
    row blocks so large lattices need little temporary memory."""
    Lx, Ly = nx * delta, ny * delta
    xc, yc = (0.5 * Lx, 0.5 * Ly) if centre is None else centre
    ca, sa = math.cos(angle), math.sin(angle)
    dx = _min_image(np.arange(nx) * delta - xc, Lx)[None, :]
    out = np.empty((ny, nx))
    rows = max(1, (1 << 22) // max(nx, 1))
    for j0 in range(0, ny, rows):
        j1 = min(ny, j0 + rows)
        dy = _min_image(np.arange(j0, j1) * delta - yc, Ly)[:, None]
        X = dx * ca + dy * sa
        Y = -dx * sa + dy * ca
        rho = np.sqrt((X / a) ** 2 + (Y / b) ** 2)
        g = np.sqrt((X / a ** 2) ** 2 + (Y / b ** 2) ** 2)
        pos = rho > 0
        grad = np.where(pos, g / np.where(pos, rho, 1.0), 1.0)
        s = np.where(pos, (rho - 1.0) / grad, -min(a, b))
        out[j0:j1] = n_out + (n_in - n_out) * 0.5 * (1.0 - np.tanh(s / edge))
    return out


def slab_medium(nx: int, ny: int, delta: float, x1: float, x2: float,
                n1: float, n2: float, edge: float, axis: int = 0) -> np.ndarray:
    """Slab n2 between x1 and x2 (smooth tanh edges) in a background n1,
    varying along ``axis`` only (0 = x, 1 = y)."""
    if axis == 0:
        x = np.arange(nx) * delta
        prof = n1 + (n2 - n1) * 0.25 * (1 + np.tanh((x - x1) / edge)) * (1 + np.tanh((x2 - x) / edge))
        return np.ascontiguousarray(np.broadcast_to(prof[None, :], (ny, nx)))
    y = np.arange(ny) * delta
    prof = n1 + (n2 - n1) * 0.25 * (1 + np.tanh((y - x1) / edge)) * (1 + np.tanh((x2 - y) / edge))
    return np.ascontiguousarray(np.broadcast_to(prof[:, None], (ny, nx)))


@dataclasses.dataclass
class Packet:
    """Gaussian E_z packet: centre (x0, y0), propagation angle, wavenumber
    k0, envelope width (exp(-xi^2/width^2)), optional transverse width
    (0 = planar front), amplitude.  Physical units."""
    x0: float
    y0: float
    angle: float
    k0: float
    width: float
    transverse_width: float = 0.0
    amplitude: float = 1.0

    def as_dict(self):
        return dataclasses.asdict(self)


@dataclasses.dataclass
class Workload:
    name: str
    nx: int
    ny: int
    delta: float
    steps: int
    packet: Packet
    medium_args: dict
    energy_every: int = 0

    def medium(self) -> np.ndarray:
        return ellipse_medium(self.nx, self.ny, self.delta, **self.medium_args)

    @property
    def sites(self) -> int:
        return self.nx * self.ny


def _ellipse_x_extent(a, b, angle):
    return math.sqrt((a * math.cos(angle)) ** 2 + (b * math.sin(angle)) ** 2)


def ellipse_256() -> Workload:
    """256x256 periodic, unit spacing, 400 steps: dielectric ellipse (semi-axes
    40x20, n_in = 2, tanh edge 3) in vacuum; packet k0 = 0.3, width 20, moving
    +x, centred 80 cells left of the ellipse's left vertex."""
    nx = ny = 256
    xc, yc = nx / 2, ny / 2
    return Workload(
        "ellipse_256_fp64_400", nx, ny, 1.0, 400,
        Packet(x0=xc - 40 - 80, y0=yc, angle=0.0, k0=0.3, width=20.0),
        dict(a=40.0, b=20.0, n_in=2.0, n_out=1.0, edge=3.0, angle=0.0))


def ellipse_8192() -> Workload:
    """8192x8192, 20000 steps: ellipse n_in = 2 (semi-axes 1200x600, rotated
    30 degrees, tanh edge 8) in vacuum; packet k0 = 0.2, width 300, moving +x,
    starting three widths left of the ellipse; energy every 100 steps."""
    nx = ny = 8192
    xc, yc = nx / 2, ny / 2
    ang = math.radians(30.0)
    x0 = xc - _ellipse_x_extent(1200.0, 600.0, ang) - 3 * 300.0
    return Workload(
        "ellipse_8192_20000", nx, ny, 1.0, 20000,
        Packet(x0=x0, y0=yc, angle=0.0, k0=0.2, width=300.0),
        dict(a=1200.0, b=600.0, n_in=2.0, n_out=1.0, edge=8.0, angle=ang),
        energy_every=100)


def bubble_16384() -> Workload:
    """16384x16384, 20000 steps: elliptical vacuum bubble (n = 1, semi-axes
    2400x1200, tanh edge 8) in a uniform dielectric n = 2; packet k0 = 0.2,
    width 600, launched inside the dielectric three widths left of the bubble."""
    nx = ny = 16384
    xc, yc = nx / 2, ny / 2
    return Workload(
        "bubble_16384_20000", nx, ny, 1.0, 20000,
        Packet(x0=xc - 2400.0 - 3 * 600.0, y0=yc, angle=0.0, k0=0.2, width=600.0),
        dict(a=2400.0, b=1200.0, n_in=1.0, n_out=2.0, edge=8.0, angle=0.0),
        energy_every=100)


def scaled(w: Workload, nx: int, ny: int, steps: int) -> Workload:
    """Same geometry as ``w`` on a smaller nx x ny box: every length is
    scaled by nx / w.nx (edge clamped to at least 1.5 cells)."""
    f = nx / w.nx
    m = dict(w.medium_args)
    m["a"] *= f
    m["b"] *= f
    m["edge"] = max(1.5, m["edge"] * f)
    p = dataclasses.replace(w.packet, x0=w.packet.x0 * f, y0=w.packet.y0 * ny / w.ny,
                            k0=w.packet.k0 / f, width=w.packet.width * f,
                            transverse_width=w.packet.transverse_width * f)
    return Workload(f"{w.name}_scaled_{nx}x{ny}", nx, ny, w.delta, steps, p, m, w.energy_every)


def batch_instances(count: int = 256, seed: int = BATCH_SEED,
                    sides=(512, 768, 1024, 1536, 2048)):
    """Uneven square instances: side drawn from ``sides``; ellipse semi-axes
    5-25% of the side, orientation in [0, pi), n_in ~ U[1.5, 4] in vacuum;
    packet angle in [0, 2 pi), k0 in [0.1, 0.4], width side/16 and transverse
    width side/8 (a localised packet stays continuous on the periodic box),
    centred a quarter side from the box centre, against its direction."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        side = int(rng.choice(sides))
        a = float(rng.uniform(0.05, 0.25)) * side
        b = float(rng.uniform(0.05, 0.25)) * side
        ang = float(rng.uniform(0.0, math.pi))
        n_in = float(rng.uniform(1.5, 4.0))
        phi = float(rng.uniform(0.0, 2 * math.pi))
        k0 = float(rng.uniform(0.1, 0.4))
        c = side / 2
        p = Packet(x0=c - 0.25 * side * math.cos(phi), y0=c - 0.25 * side * math.sin(phi),
                   angle=phi, k0=k0, width=side / 16, transverse_width=side / 8)
        out.append(Workload(f"batch_{k}", side, side, 1.0, 2000, p,
                            dict(a=a, b=b, n_in=n_in, n_out=1.0, edge=3.0, angle=ang)))
    return out


def ellipsoid_medium3(nx: int, ny: int, nz: int, delta: float, a: float, b: float, c: float,
                      n_in: float, n_out: float, edge: float, centre=None) -> np.ndarray:
    """Index map (nz, ny, nx) of a smooth ellipsoid (semi-axes a, b, c along
    x, y, z, lengths in physical units): rho = |(X/a, Y/b, Z/c)|, signed
    distance s = (rho - 1)/|grad rho|, n = n_out + (n_in - n_out)(1 - tanh(s/edge))/2,
    built plane by plane along z."""
    cx, cy, cz = (nx * delta / 2, ny * delta / 2, nz * delta / 2) if centre is None else centre
    X = np.arange(nx)[None, :] * delta - cx
    Y = np.arange(ny)[:, None] * delta - cy
    out = np.empty((nz, ny, nx))
    for k in range(nz):
        Z = k * delta - cz
        rho = np.sqrt((X / a) ** 2 + (Y / b) ** 2 + (Z / c) ** 2)
        rs = np.maximum(rho, 1e-12)
        grad = np.sqrt((X / a ** 2) ** 2 + (Y / b ** 2) ** 2 + (Z / c ** 2) ** 2) / rs
        sdist = (rho - 1.0) / np.maximum(grad, 1e-12)
        out[k] = n_out + (n_in - n_out) * 0.5 * (1.0 - np.tanh(sdist / edge))
    return out


def cube_256():
    """3D workload: 256^3, delta = 1, a dielectric ellipsoid (semi-axes 60,
    40, 30 cells, n = 2, tanh edge 3) in vacuum at the box centre; a planar
    E_z packet (k0 = 0.3, width 16 cells) moving along +x from x = 40."""
    return dict(name="cube_256", n=256, delta=1.0,
                medium=dict(a=60.0, b=40.0, c=30.0, n_in=2.0, n_out=1.0, edge=3.0),
                packet=dict(x0=40.0, k0=0.3, width=16.0))


def random_state(nx: int, ny: int, seed: int, planes=6) -> np.ndarray:
    """Seeded N(0,1) amplitudes of shape (6, ny, nx); planes beyond ``planes``
    of the TE set are zero when planes == 3 (q2, q3, q4 live)."""
    rng = np.random.default_rng(seed)
    q = rng.standard_normal((6, ny, nx))
    if planes == 3:
        q[[0, 1, 5]] = 0.0
    return q


def random_medium(nx: int, ny: int, seed: int, lo=1.0, hi=3.0, smooth=2) -> np.ndarray:
    """Seeded smooth random index map in [lo, hi] (box-filtered noise)."""
    rng = np.random.default_rng(seed)
    r = rng.uniform(0.0, 1.0, (ny, nx))
    for _ in range(smooth):
        r = (r + np.roll(r, 1, 0) + np.roll(r, -1, 0) + np.roll(r, 1, 1) + np.roll(r, -1, 1)) / 5
    r = (r - r.min()) / max(r.max() - r.min(), 1e-12)
    return lo + (hi - lo) * r


def surrogate_instance(rng, size=256):
    """One seeded training lattice for the learned surrogate: the vacuum
    bubble of the 16384^2 workload scaled to ``size`` (semi-axes 37.5 x 18.75
    at 256, n = 1 inside a uniform n = 2, edge 1.5 cells) at a random
    orientation and offset, and a Gaussian E_z packet with random angle,
    k0 in [0.15, 0.35] rad/cell, width in [8, 16] cells and transverse width
    in [24, 64] cells (wavenumbers stay resolved on the coarse lattice, so
    they are drawn in cells rather than scaled).  Returns (medium kwargs for
    ellipse_medium, packet kwargs)."""
    f = size / 16384.0
    ang = float(rng.uniform(0.0, math.pi))
    c = size / 2 + rng.uniform(-0.1, 0.1, 2) * size
    med = dict(a=2400.0 * f, b=1200.0 * f, n_in=1.0, n_out=2.0, edge=max(1.5, 8.0 * f),
               angle=ang, centre=(float(c[0]), float(c[1])))
    phi = float(rng.uniform(0.0, 2 * math.pi))
    r = 0.3 * size
    pk = dict(x0=float(c[0] - r * math.cos(phi)), y0=float(c[1] - r * math.sin(phi)), angle=phi,
              k0=float(rng.uniform(0.15, 0.35)), width=float(rng.uniform(8.0, 16.0)),
              transverse_width=float(rng.uniform(24.0, 64.0)), amplitude=1.0)
    return med, pk
