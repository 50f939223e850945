"""Seeded synthetic inputs for the drop-on-film pressure Poisson workloads.

This module produces only *inputs*: phase volume fractions of a liquid drop
above a liquid film in a gas (the geometry of the paper's drop-film impact
study, §3.1), curvature bands, and counter-based pseudo-random face velocities
and normal weights.  It holds none of the solver's arithmetic: no density
mixing, no face coefficients, no divergence, no operator.  Both the CUDA path
and the CPU oracle consume what it returns.

Every generator is written with plain torch tensor ops so the same code runs
on the host (CPU tensors, used by the oracle side) and on a CUDA device (large
workloads), and gives bitwise identical results on both: it uses only integer
arithmetic and the correctly rounded float64 operations +, -, *, / and sqrt.
The one exception is :func:`normal_weights`, whose log/cos are not guaranteed
bitwise equal across devices; generate it once and copy it where needed.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used in counter mode:
``x_n = mix64(seed + (n + 1) * 0x9E3779B97F4A7C15)``, where ``mix64`` is the
published SplitMix64 output function.  With seed 0, ``x_0`` equals the first
output of the reference SplitMix64 stream started from state 0.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import torch

__all__ = [
    "GAMMA",
    "splitmix64",
    "uniform53",
    "Geometry",
    "scaled_geometry",
    "fractions_subcell",
    "fractions_ramp",
    "face_velocities",
    "normal_weights",
    "curvature_band",
]

GAMMA = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB


def _i64(x: int) -> int:
    """Reinterpret an unsigned 64-bit constant as a signed int64 value."""
    x &= (1 << 64) - 1
    return x - (1 << 64) if x >= (1 << 63) else x


def _srl(z: torch.Tensor, s: int) -> torch.Tensor:
    """Logical right shift of int64 bit patterns (torch's >> is arithmetic)."""
    return (z >> s) & ((1 << (64 - s)) - 1)


def splitmix64(seed: int, counter: torch.Tensor) -> torch.Tensor:
    """SplitMix64 in counter mode; returns the 64-bit outputs as int64 bit patterns.

    ``counter`` is an int64 tensor of non-negative stream positions.  All
    products wrap modulo 2**64 (two's complement), which is exactly the
    unsigned arithmetic of the published generator.
    """
    z = counter.to(torch.int64) + 1
    z = z * _i64(GAMMA) + _i64(seed)
    z = (z ^ _srl(z, 30)) * _i64(_M1)
    z = (z ^ _srl(z, 27)) * _i64(_M2)
    return z ^ _srl(z, 31)


def uniform53(seed: int, counter: torch.Tensor) -> torch.Tensor:
    """Uniform float64 in [0, 1): the top 53 bits of SplitMix64 times 2**-53 (exact)."""
    return _srl(splitmix64(seed, counter), 11).to(torch.float64) * (2.0 ** -53)


@dataclass(frozen=True)
class Geometry:
    """A spherical drop above a flat film, in cell units of an n^3 grid.

    ``center`` and ``radius`` are in cells (cell (i,j,k) spans [i, i+1) etc.),
    the film fills z < ``z_film`` cells.
    """

    n: int
    center: tuple
    radius: float
    z_film: float


def scaled_geometry(n: int) -> Geometry:
    """The drop/film layout of the 32^3 case scaled by n/32.

    At 32^3: drop radius 8 cells centred at (16, 16, 20), film z < 6.  Scaled:
    centre (n/2, n/2, 5n/8), radius n/4, film thickness 3n/16 (256^3 gives
    R = 64 at (128, 128, 160) and a 48-cell film; 1024^3 gives R = 256).
    """
    return Geometry(n=n, center=(n / 2, n / 2, 5 * n / 8), radius=n / 4, z_film=3 * n / 16)


def _axis(n: int, device) -> torch.Tensor:
    return torch.arange(n, device=device, dtype=torch.int64)


def fractions_subcell(geom: Geometry, sub: int = 4, device="cpu"):
    """Drop and film volume fractions by sub^3 point sampling per cell (exact integers).

    Sample points sit at offsets (a + 1/2)/sub inside each cell.  Positions are
    held as integers in units of 1/(2 sub) cells, so membership tests are exact:
    a point is in the drop when its squared distance to the centre is <= R^2,
    in the film when its z is < z_film.  Requires 2*sub*center, 2*sub*R and
    2*sub*z_film to be integers.  Returns (f_drop, f_film), float64 (nz,ny,nx),
    with the film clipped so the two fractions never sum above 1.
    """
    n = geom.n
    s2 = 2 * sub
    c = [s2 * x for x in geom.center]
    r = s2 * geom.radius
    zf = s2 * geom.z_film
    for v in (*c, r, zf):
        if abs(v - round(v)) > 0:
            raise ValueError("geometry not representable on the 1/(2 sub) lattice")
    c = [int(round(x)) for x in c]
    r2 = int(round(r)) ** 2
    zf = int(round(zf))
    ax = _axis(n, device)
    cnt_drop = torch.zeros((n, n, n), dtype=torch.int64, device=device)
    cnt_film = torch.zeros((n, n, n), dtype=torch.int64, device=device)
    for a in range(sub):
        pos = s2 * ax + 2 * a + 1  # sample coordinate along one axis
        dx2 = (pos - c[0]) ** 2
        for b in range(sub):
            posb = s2 * ax + 2 * b + 1
            dyb2 = (posb - c[1]) ** 2
            for cc in range(sub):
                posc = s2 * ax + 2 * cc + 1
                dzc2 = (posc - c[2]) ** 2
                d2 = dzc2.view(n, 1, 1) + dyb2.view(1, n, 1) + dx2.view(1, 1, n)
                cnt_drop += (d2 <= r2).to(torch.int64)
                cnt_film += (posc < zf).to(torch.int64).view(n, 1, 1)
    tot = sub ** 3
    f_drop = cnt_drop.to(torch.float64) / tot
    f_film = torch.minimum(cnt_film.to(torch.float64) / tot, 1.0 - f_drop)
    return f_drop, f_film


def fractions_ramp(geom: Geometry, width: float = 1.5, device="cpu", z_chunk: int = 64):
    """Drop and film fractions with interfaces smeared linearly over ``width`` cells.

    f = clamp(1/2 - d/width, 0, 1), d the signed distance in cells from the
    cell centre to the interface (sphere: |x - c| - R; film: z - z_film).
    Built from +, -, *, /, sqrt only, so host and device agree bitwise.
    Returns (f_drop, f_film) float64 (nz, ny, nx), film clipped to 1 - f_drop.
    """
    n = geom.n
    cx, cy, cz = (float(v) for v in geom.center)
    R = float(geom.radius)
    x = torch.arange(n, device=device, dtype=torch.float64) + 0.5
    dx2 = ((x - cx) ** 2).view(1, 1, n)
    dy2 = ((x - cy) ** 2).view(1, n, 1)
    f_drop = torch.empty((n, n, n), dtype=torch.float64, device=device)
    for z0 in range(0, n, z_chunk):
        z1 = min(n, z0 + z_chunk)
        dz2 = ((x[z0:z1] - cz) ** 2).view(-1, 1, 1)
        d = torch.sqrt((dz2 + dy2) + dx2) - R
        f_drop[z0:z1] = torch.clamp(0.5 - d / width, 0.0, 1.0)
    dfilm = x - float(geom.z_film)
    f_film_z = torch.clamp(0.5 - dfilm / width, 0.0, 1.0).view(n, 1, 1)
    f_film = torch.minimum(f_film_z.expand(n, n, n), 1.0 - f_drop)
    return f_drop, f_film


def face_velocities(n: int, seed: int = 0, device="cpu", z_chunk: int = None):
    """Random face velocities u ~ U[-1, 1] on interior faces, 0 on the walls.

    Shapes: ux (n, n, n+1), uy (n, n+1, n), uz (n+1, n, n) -- face index i of
    ux lies between cells i-1 and i.  One SplitMix64 stream per seed, read in
    C order of ux, then uy, then uz (wall entries consume a number too).
    ``z_chunk`` generates that many z-slices at a time (same values, bounded temporaries).
    """
    shapes = [(n, n, n + 1), (n, n + 1, n), (n + 1, n, n)]
    out = []
    base = 0
    for axis, shp in enumerate(shapes):
        cnt = 1
        for s in shp:
            cnt *= s
        slab = shp[1] * shp[2]
        u = torch.empty(shp, dtype=torch.float64, device=device)
        step = shp[0] if z_chunk is None else z_chunk
        for z0 in range(0, shp[0], step):
            z1 = min(shp[0], z0 + step)
            ctr = torch.arange(base + z0 * slab, base + z1 * slab, device=device, dtype=torch.int64)
            u[z0:z1] = (2.0 * uniform53(seed, ctr) - 1.0).view(z1 - z0, shp[1], shp[2])
            del ctr
        # walls: first and last face along the face-normal axis
        if axis == 0:
            u[:, :, 0] = 0.0
            u[:, :, -1] = 0.0
        elif axis == 1:
            u[:, 0, :] = 0.0
            u[:, -1, :] = 0.0
        else:
            u[0] = 0.0
            u[-1] = 0.0
        out.append(u)
        base += cnt
    return tuple(out)


def normal_weights(shape, seed: int = 1, device="cpu", chunk: int = None):
    """w ~ N(0, 1) by Box-Muller on consecutive SplitMix64 pairs (cos branch).

    Element m uses counters 2m (u1, mapped to (0, 1] as 1 - U) and 2m+1 (u2).
    ``chunk`` generates that many elements at a time (same values, bounded temporaries).
    """
    cnt = 1
    for s in shape:
        cnt *= s
    w = torch.empty(cnt, dtype=torch.float64, device=device)
    step = cnt if chunk is None else chunk
    for a in range(0, cnt, step):
        m = torch.arange(a, min(cnt, a + step), device=device, dtype=torch.int64)
        u1 = 1.0 - uniform53(seed, 2 * m)
        u2 = uniform53(seed, 2 * m + 1)
        w[a:a + m.numel()] = torch.sqrt(-2.0 * torch.log(u1)) * torch.cos((2.0 * math.pi) * u2)
    return w.view(*shape)


def curvature_band(f_drop: torch.Tensor, geom: Geometry) -> torch.Tensor:
    """Interface curvature of the drop: 2/R (R in domain units, h = 1/n) where 0 < f_drop < 1.

    The exact mean curvature of a sphere is 2/R; it is placed on the cells of
    the smeared interface band and is 0 elsewhere.
    """
    kappa = 2.0 / (geom.radius / geom.n)
    out = torch.zeros_like(f_drop)
    for z0 in range(0, f_drop.shape[0], 64):  # bounded temporaries at large n
        f = f_drop[z0:z0 + 64]
        out[z0:z0 + 64].masked_fill_((f > 0.0) & (f < 1.0), kappa)
    return out
