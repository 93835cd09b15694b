"""Seeded synthetic collage problems (inputs only: no rendering, loss or gradient arithmetic).

Both the CUDA path and the FP64 oracle read their inputs from here, so this module holds nothing
but a counter-style random generator and the construction of element outlines, containers and
initial transforms.  It mirrors the paper's problem statement (Sec. 3, "Collage Problem", Eq. 1):
items ``g_i`` given as closed paths of cubic Beziers (Sec. 3, "Vector Representation") or as
polygons / open polylines, a container ``C``, and per-item translate / rotate / scale.

Coordinates are the unit square with y pointing down (image rows).  Element outlines are given in
element-local coordinates around the local origin; the world position is ``R(theta)(s*v) + t``
(Eq. 2).  A problem is a plain dict of numpy arrays:

    kind      int32[n]     0 closed cubic Bezier path (3 control points per curve, closed),
                           1 closed polygon, 2 open polyline
    pt_off    int32[n+1]   CSR offsets into pts (in points)
    pts       float32[2*pt_off[n]]  interleaved x, y
    hw        float32[n]   stroke half-width of open polylines (unit coords, world units)
    params0   float32[4n]  (tx, ty, theta, s) per element
    ring_off  int32[r+1]   container rings (closed polygons, nonzero fill rule)
    ring_pts  float32[2*ring_off[r]]
    grid      int          finest grid side in pixels

The random stream is PCG32 (O'Neill 2014, PCG-XSH-RR 64/32, "pcg32_srandom_r" seeding) with the
seed ``1000*config + collage_index``.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "PCG32", "config_problem", "CONFIGS", "regular_polygon", "blob_controls",
    "convex_polygon", "polyline", "disk_container", "annulus_container",
    "star_container", "open_rect_container", "make_problem", "circle_controls", "fit_problem",
    "FIT_LOSS",
]

_MASK64 = (1 << 64) - 1
_MULT = 6364136223846793005


class PCG32:
    """PCG-XSH-RR with 64-bit state and 32-bit output (O'Neill 2014)."""

    def __init__(self, seed: int, seq: int = 54):
        self.state = 0
        self.inc = ((seq << 1) | 1) & _MASK64
        self.next_u32()
        self.state = (self.state + (seed & _MASK64)) & _MASK64
        self.next_u32()

    def next_u32(self) -> int:
        old = self.state
        self.state = (old * _MULT + self.inc) & _MASK64
        xorshifted = (((old >> 18) ^ old) >> 27) & 0xFFFFFFFF
        rot = old >> 59
        return ((xorshifted >> rot) | (xorshifted << ((-rot) & 31))) & 0xFFFFFFFF

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        """Uniform double in [lo, hi) from the top 24 bits of one draw."""
        return lo + (hi - lo) * ((self.next_u32() >> 8) * (1.0 / 16777216.0))

    def randint(self, lo: int, hi: int) -> int:
        """Integer uniform in [lo, hi] (inclusive), by rejection-free modulo of 32 bits."""
        return lo + self.next_u32() % (hi - lo + 1)


# ----------------------------------------------------------------------------------------------
# Element outlines (element-local coordinates around the origin)
# ----------------------------------------------------------------------------------------------

def regular_polygon(r: float, n: int) -> np.ndarray:
    a = 2.0 * np.pi * np.arange(n) / n
    return np.stack([r * np.cos(a), r * np.sin(a)], 1)


def blob_controls(rng: PCG32, scale: float, n_cubics: int = 8) -> np.ndarray:
    """Closed blob: 3*n_cubics control points at equal angles, radius U[0.6,1.0]*scale."""
    m = 3 * n_cubics
    pts = np.empty((m, 2))
    for k in range(m):
        rad = rng.uniform(0.6, 1.0) * scale
        a = 2.0 * np.pi * k / m
        pts[k] = (rad * math.cos(a), rad * math.sin(a))
    return pts


def circle_controls(r: float, n_cubics: int) -> np.ndarray:
    """Closed path of n_cubics curves close to a circle of radius r: anchors at equal angles,
    handles along the tangents with length (4/3) tan(pi / (2 n_cubics)) r."""
    h = 4.0 / 3.0 * math.tan(math.pi / (2 * n_cubics)) * r
    pts = []
    for k in range(n_cubics):
        a0, a1 = 2.0 * np.pi * k / n_cubics, 2.0 * np.pi * (k + 1) / n_cubics
        p0 = np.array([r * math.cos(a0), r * math.sin(a0)])
        p1 = np.array([r * math.cos(a1), r * math.sin(a1)])
        pts += [p0, p0 + h * np.array([-math.sin(a0), math.cos(a0)]),
                p1 - h * np.array([-math.sin(a1), math.cos(a1)])]
    return np.array(pts)


def convex_polygon(rng: PCG32, r: float, n_sides: int) -> np.ndarray:
    """Convex polygon: n sorted random angles on a circle of radius r."""
    ang = sorted(rng.uniform(0.0, 2.0 * np.pi) for _ in range(n_sides))
    return np.array([(r * math.cos(a), r * math.sin(a)) for a in ang])


def polyline(rng: PCG32, r: float, n_verts: int) -> np.ndarray:
    """Open zig-zag polyline spanning [-r, r] in x with y jitter of +-r/2."""
    xs = np.linspace(-r, r, n_verts)
    ys = np.array([r * rng.uniform(-0.5, 0.5) for _ in range(n_verts)])
    return np.stack([xs, ys], 1)


# ----------------------------------------------------------------------------------------------
# Containers (rings of the nonzero fill rule)
# ----------------------------------------------------------------------------------------------

def disk_container(cx=0.5, cy=0.5, r=0.45, n=256):
    return [regular_polygon(r, n) + (cx, cy)]


def annulus_container(cx=0.5, cy=0.5, r_in=0.2, r_out=0.48, n=256):
    outer = regular_polygon(r_out, n) + (cx, cy)
    inner = (regular_polygon(r_in, n) + (cx, cy))[::-1]  # reversed: a hole under nonzero
    return [outer, inner]


def star_container(rng: PCG32, cx=0.5, cy=0.5, r_in=0.25, r_out=0.45, points=12):
    phase = rng.uniform(0.0, 2.0 * np.pi)
    m = 2 * points
    v = []
    for k in range(m):
        rad = r_out if k % 2 == 0 else r_in
        a = phase + 2.0 * np.pi * k / m
        v.append((cx + rad * math.cos(a), cy + rad * math.sin(a)))
    return [np.array(v)]


def open_rect_container(x0=0.05, x1=0.95, y_top=-0.1, y1=0.95):
    """Rectangle whose top edge lies above the image, so the image shows no top wall."""
    return [np.array([(x0, y_top), (x1, y_top), (x1, y1), (x0, y1)])]


# ----------------------------------------------------------------------------------------------
# Placement inside a container, by closed-form sampling per container type
# ----------------------------------------------------------------------------------------------

def _sample_in_disk(rng, cx, cy, r):
    rad = r * math.sqrt(rng.uniform())
    a = rng.uniform(0.0, 2.0 * np.pi)
    return cx + rad * math.cos(a), cy + rad * math.sin(a)


def _sample_in_annulus(rng, cx, cy, r0, r1):
    rad = math.sqrt(rng.uniform(r0 * r0, r1 * r1))
    a = rng.uniform(0.0, 2.0 * np.pi)
    return cx + rad * math.cos(a), cy + rad * math.sin(a)


def make_problem(elements, container_rings, params0, grid):
    """Pack python lists into the flat problem dict described in the module docstring."""
    kinds, offs, pts, hws = [], [0], [], []
    for kind, p, hw in elements:
        p = np.asarray(p, dtype=np.float64)
        kinds.append(kind)
        offs.append(offs[-1] + len(p))
        pts.append(p.reshape(-1))
        hws.append(hw)
    roff = [0]
    rpts = []
    for ring in container_rings:
        ring = np.asarray(ring, dtype=np.float64)
        roff.append(roff[-1] + len(ring))
        rpts.append(ring.reshape(-1))
    return {
        "kind": np.asarray(kinds, np.int32),
        "pt_off": np.asarray(offs, np.int32),
        "pts": np.concatenate(pts).astype(np.float32) if pts else np.zeros(0, np.float32),
        "hw": np.asarray(hws, np.float32),
        "params0": np.asarray(params0, np.float32).reshape(-1),
        "ring_off": np.asarray(roff, np.int32),
        "ring_pts": np.concatenate(rpts).astype(np.float32),
        "grid": int(grid),
    }


def _mixed_element(rng, r):
    """60% blobs (8 cubics), 30% convex polygons (5-12 sides), 10% open polylines (4-10 verts)."""
    u = rng.uniform()
    if u < 0.6:
        return (0, blob_controls(rng, r), 0.0)
    if u < 0.9:
        return (1, convex_polygon(rng, r, rng.randint(5, 12)), 0.0)
    return (2, polyline(rng, r, rng.randint(4, 10)), 0.002)


def config_problem(config: int, collage_index: int = 0, n_elems: int | None = None,
                   grid: int | None = None):
    """Build one collage of the named workload (1..5); ``n_elems``/``grid`` shrink it for tests."""
    rng = PCG32(1000 * config + collage_index)
    els, params = [], []
    if config == 1:
        # 16 regular 32-gons, r ~ U[0.04,0.08], in a disk container of radius 0.45 on 128^2.
        n = 16 if n_elems is None else n_elems
        rings = disk_container()
        for _ in range(n):
            r = rng.uniform(0.04, 0.08)
            els.append((1, regular_polygon(r, 32), 0.0))
            x, y = _sample_in_disk(rng, 0.5, 0.5, 0.45 - r)
            params.append((x, y, 0.0, 1.0))
        g = 128
    elif config == 2:
        # 200 blobs (8 cubics, control radii U[0.6,1.0]*scale, scale U[0.02,0.06]) in a 12-point star on 512^2.
        n = 200 if n_elems is None else n_elems
        rings = star_container(rng)
        for _ in range(n):
            els.append((0, blob_controls(rng, rng.uniform(0.02, 0.06)), 0.0))
            x, y = _sample_in_disk(rng, 0.5, 0.5, 0.25)
            params.append((x, y, 0.0, 1.0))
        g = 512
    elif config == 3:
        # 1000 mixed elements, element radius U[0.006,0.018], annulus 0.2/0.48, pyramid up to 1024^2.
        n = 1000 if n_elems is None else n_elems
        rings = annulus_container()
        for _ in range(n):
            els.append(_mixed_element(rng, rng.uniform(0.006, 0.018)))
            x, y = _sample_in_annulus(rng, 0.5, 0.5, 0.2, 0.48)
            params.append((x, y, rng.uniform(0.0, 2.0 * np.pi), 1.0))
        g = 1024
    elif config == 4:
        # one collage of the batch: n ~ U[20,800], grid in {256,512,1024}, star or annulus,
        # 32-gon disks and blobs sized for ~50% expected fill of the container.
        n = rng.randint(20, 800) if n_elems is None else n_elems
        g = (256, 512, 1024)[rng.randint(0, 2)]
        if rng.uniform() < 0.5:
            rings = star_container(rng)
            area_c = 24 * 0.5 * 0.25 * 0.45 * math.sin(2 * np.pi / 24)  # 24 triangles
            sampler = lambda: _sample_in_disk(rng, 0.5, 0.5, 0.25)
        else:
            rings = annulus_container()
            area_c = np.pi * (0.48 ** 2 - 0.2 ** 2)
            sampler = lambda: _sample_in_annulus(rng, 0.5, 0.5, 0.2, 0.48)
        r_mean = math.sqrt(0.5 * area_c / (n * np.pi))
        for _ in range(n):
            r = r_mean * rng.uniform(0.7, 1.3)
            if rng.uniform() < 0.5:
                els.append((1, regular_polygon(r, 32), 0.0))
            else:
                els.append((0, blob_controls(rng, r / 0.8), 0.0))
            x, y = sampler()
            params.append((x, y, 0.0, 1.0))
    elif config == 5:
        # 5000 mixed elements, radius U[0.005,0.02], open-top rectangle on 2048^2.
        n = 5000 if n_elems is None else n_elems
        rings = open_rect_container()
        for _ in range(n):
            els.append(_mixed_element(rng, rng.uniform(0.005, 0.02)))
            params.append((rng.uniform(0.05, 0.95), rng.uniform(0.0, 0.95),
                           rng.uniform(0.0, 2.0 * np.pi), 1.0))
        g = 2048
    else:
        raise ValueError(f"unknown workload {config}")
    if grid is not None:
        g = grid
    return make_problem(els, rings, params, g)


def fit_problem(index: int = 0, n_cubics: int = 20, grid: int = 256, r0: float = 0.3):
    """Outline fitting (Sec. 3, Vector Representation): one closed path of n_cubics curves (the
    paper uses 20), initially a circle of radius r0 about the centre, fitted to a seeded 12-point
    star silhouette given as the container rings; the transform is the identity about the centre."""
    rng = PCG32(7000 + index)
    r_in, r_out = rng.uniform(0.18, 0.28), rng.uniform(0.36, 0.46)
    rings = star_container(rng, r_in=r_in, r_out=r_out)
    return make_problem([(0, circle_controls(r0, n_cubics), 0.0)], rings, [(0.5, 0.5, 0.0, 1.0)], grid)


# Fitting loss: L_c of Eq. 5 alone with the same weight inside and outside the silhouette.
FIT_LOSS = dict(alpha=1.0, beta=0.0, gamma=0.0, delta=0.0, w_in=1.0, w_out=1.0, pad_px=0.0)


# Loss weights and schedules of the five workloads (Eq. 8 weights 3e3 / 8e4 / 5e-4).
CONFIGS = {
    1: dict(name="disks16_disk_128", gamma=0.0, delta=0.0, pad_px=0.0,
            levels=[(128, 50)], lr=1e-2),
    2: dict(name="blobs200_star_512", gamma=5e-4, delta=0.0, pad_px=0.0,
            levels=[(512, 1)], lr=1e-2),
    3: dict(name="mixed1000_annulus_1024", gamma=5e-4, delta=0.0, pad_px=2.0,
            levels=[(128, 300), (256, 200), (512, 100), (1024, 50)], lr=1e-2),
    4: dict(name="batch64_mixed_grids", gamma=5e-4, delta=0.0, pad_px=0.0,
            levels=[(0, 50)], lr=1e-2),
    5: dict(name="open5000_rect_2048", gamma=5e-4, delta=1e3, pad_px=1.0,
            levels=[(2048, 20)], lr=1e-2),
}
