"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke
check.  This module holds no arithmetic of the method (no metaball field, no
lattice Boltzmann formula): it only draws random numbers and places shapes,
with every value rounded to float32 so that the FP64 oracle and the FP32 GPU
path read identical bits.

The paper's own workloads (XRCT avatars of natural cobbles, silicone-oil
settling tanks, the hand-made DKT shapes) are not available; these scenes
stand in for them with the shapes, sizes and counts of the five benchmark
configurations (metaball counts, centre spreads, k ranges, lattice sizes).
"""
from dataclasses import dataclass, field

import numpy as np


def f32(a):
    """Round to the nearest float32 and return as float64."""
    return np.asarray(np.asarray(a, dtype=np.float64).astype(np.float32), dtype=np.float64)


@dataclass
class ParticleSpec:
    centers: np.ndarray          # (n, 3) body frame, lattice units
    k: np.ndarray                # (n,) > 0
    density: float               # particle density (fluid rho0 = 1)
    skin: float                  # sphero-metaball skin radius R_s
    pos: np.ndarray              # (3,)
    quat: np.ndarray             # (4,) w, x, y, z (unit up to float32 rounding)
    vel: np.ndarray = field(default_factory=lambda: np.zeros(3))
    omega: np.ndarray = field(default_factory=lambda: np.zeros(3))
    nominal_radius: float = 0.0  # generator's size scale (placement only)


@dataclass
class Scene:
    name: str
    shape: tuple                 # (nx, ny, nz)
    tau: float
    gravity: tuple
    particles: list
    steps: int
    seed: int


def random_unit_quaternion(rng):
    """Uniform random rotation (Shoemake's method)."""
    u1, u2, u3 = rng.random(3)
    q = np.array([np.sqrt(u1) * np.cos(2 * np.pi * u3), np.sqrt(1 - u1) * np.sin(2 * np.pi * u2),
                  np.sqrt(1 - u1) * np.cos(2 * np.pi * u2), np.sqrt(u1) * np.sin(2 * np.pi * u3)])
    if q[0] < 0:
        q = -q
    return f32(q)


def uniform_in_ball(rng, n, radius):
    out = []
    while len(out) < n:
        p = rng.uniform(-radius, radius, 3)
        if p @ p <= radius * radius:
            out.append(p)
    return np.array(out)


def lattice_noise(shape, seed, q=19):
    """Standard-normal numbers of shape (q, nz, ny, nx) for perturbing populations."""
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    return rng.standard_normal((q, nz, ny, nx)).astype(np.float32)


def velocity_field_noise(shape, seed):
    """Smooth-ish random velocity components in [-1, 1], shape (3, nz, ny, nx)."""
    nx, ny, nz = shape
    rng = np.random.default_rng(seed + 7)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    out = np.empty((3, nz, ny, nx))
    for a in range(3):
        kx, ky, kz = rng.integers(1, 4, 3)
        ph = rng.uniform(0, 2 * np.pi, 3)
        out[a] = (np.sin(2 * np.pi * kx * x / nx + ph[0]) * np.cos(2 * np.pi * ky * y / ny + ph[1])
                  * np.sin(2 * np.pi * kz * z / nz + ph[2]))
    return out


# ---------------------------------------------------------------------------
# particle shapes
# ---------------------------------------------------------------------------
def blob_4(rng):
    """Four control points uniform in a ball of radius 6, k ~ U[4, 9]."""
    c = uniform_in_ball(rng, 4, 6.0)
    k = rng.uniform(4.0, 9.0, 4)
    return f32(c), f32(k), 8.0


def cobble(rng, n_range=(24, 40), semi=(12.0, 20.0), k_range=(9.0, 36.0)):
    """Cobblestone-like: n control points, Gaussian inside a random ellipsoid."""
    n = int(rng.integers(n_range[0], n_range[1] + 1))
    a = rng.uniform(semi[0], semi[1], 3)
    c = []
    while len(c) < n:
        p = rng.normal(0.0, a / 2.0)
        if ((p / a) ** 2).sum() <= 1.0:
            c.append(p)
    c = np.array(c)
    c -= c.mean(axis=0)
    k = np.exp(rng.uniform(np.log(k_range[0]), np.log(k_range[1]), n))
    return f32(c), f32(k), float(a.max())


def grain_prolate(rng, n=32, semi=(12.0, 6.0, 6.0), k_range=(9.0, 36.0)):
    """Elongated grain: n points in a 2:1 prolate ellipsoid along x."""
    a = np.array(semi)
    c = []
    while len(c) < n:
        p = rng.uniform(-a, a)
        if ((p / a) ** 2).sum() <= 1.0:
            c.append(p)
    c = np.array(c)
    c -= c.mean(axis=0)
    k = np.exp(rng.uniform(np.log(k_range[0]), np.log(k_range[1]), n)) * 0.25
    return f32(c), f32(k), float(a.max())


def clustered(rng, n, R):
    """n points uniform in a ball of 0.5 R; k_i ~ U[0.5, 1.5] scaled so that
    sum k = R^2 (far-field radius R)."""
    c = uniform_in_ball(rng, n, 0.5 * R)
    c -= c.mean(axis=0)
    u = rng.uniform(0.5, 1.5, n)
    k = u / u.sum() * R * R
    return f32(c), f32(k), float(R)


# ---------------------------------------------------------------------------
# the five benchmark configurations
# ---------------------------------------------------------------------------
def config1(seed=0):
    """64^3 closed box, tau 0.8, one 4-ball particle at (32, 32, 44), density 2.5,
    gravity 1e-5 lu/step^2 downward, 200 steps."""
    rng = np.random.default_rng(seed)
    c, k, r = blob_4(rng)
    p = ParticleSpec(c, k, 2.5, 1.0, f32([32.0, 32.0, 44.0]), random_unit_quaternion(rng), nominal_radius=r)
    return Scene("C1 64^3 one 4-ball particle", (64, 64, 64), 0.8, (0.0, 0.0, -1e-5), [p], 200, seed)


def config2(seed=0):
    """256x256x512 tank, three cobblestone-like particles (24-40 balls) at z = 400,
    spaced 80 lu apart in x, density 2.5, released from rest; 4000 steps."""
    rng = np.random.default_rng(seed)
    parts = []
    for j in range(3):
        c, k, r = cobble(rng)
        pos = f32([48.0 + 80.0 * j, 128.0 + (j - 1) * 20.0, 400.0])
        parts.append(ParticleSpec(c, k, 2.5, 1.0, pos, random_unit_quaternion(rng), nominal_radius=r))
    return Scene("C2 256x256x512 three cobbles", (256, 256, 512), 0.8, (0.0, 0.0, -1e-5), parts, 4000, seed)


def config3(seed=0):
    """192x192x768 channel: a 1-ball sphere (k = 100, r = 10) and a 32-ball prolate
    grain stacked on the axis 30 lu apart (leading one lower); density 2.87."""
    rng = np.random.default_rng(seed)
    sphere = ParticleSpec(f32(np.zeros((1, 3))), f32([100.0]), 2.87, 1.0, f32([96.0, 96.0, 650.0]),
                          f32([1.0, 0.0, 0.0, 0.0]), nominal_radius=10.0)
    c, k, r = grain_prolate(rng)
    grain = ParticleSpec(c, k, 2.87, 1.0, f32([96.0, 100.0, 680.0]), random_unit_quaternion(rng),
                         nominal_radius=r + 6.0)
    return Scene("C3 192x192x768 DKT pair", (192, 192, 768), 0.8, (0.0, 0.0, -1e-5), [sphere, grain], 20000, seed)


def _place_non_overlapping(rng, radii, box_lo, box_hi, margin, max_tries=200000):
    """Random sequential addition: each sphere (in the given order) at a uniform
    random position where it does not overlap any placed one (plus margin)."""
    pos = np.zeros((len(radii), 3))
    rad = np.asarray(radii, dtype=float)
    for n, r in enumerate(rad):
        for _ in range(max_tries // 64 + 1):
            cand = rng.uniform(box_lo + r, box_hi - r, (64, 3))
            if n == 0:
                pos[0] = cand[0]
                break
            d = np.sqrt(((cand[:, None, :] - pos[None, :n, :]) ** 2).sum(-1))
            ok = (d > rad[None, :n] + r + margin).all(1)
            if ok.any():
                pos[n] = cand[np.argmax(ok)]
                break
        else:
            raise RuntimeError("could not place particle")
    return [p for p in pos]


def config4(seed=0, shape=(512, 512, 512), n_particles=300):
    """512^3 tank, 300 particles of 8-64 balls, radius ~ U[8, 16], random
    orientation, non-overlapping random sequential placement."""
    rng = np.random.default_rng(seed)
    specs = []
    for _ in range(n_particles):
        n = int(rng.integers(8, 65))
        R = rng.uniform(8.0, 16.0)
        c, k, r = clustered(rng, n, R)
        specs.append((c, k, r))
    lo = np.array([4.0, 4.0, 4.0])
    hi = np.array(shape, dtype=float) - 4.0
    pos = _place_non_overlapping(rng, [1.3 * s[2] for s in specs], lo, hi, 2.0)
    parts = [ParticleSpec(c, k, 2.5, 1.0, f32(p), random_unit_quaternion(rng), nominal_radius=r)
             for (c, k, r), p in zip(specs, pos)]
    return Scene("C4 512^3 300 particles", shape, 0.8, (0.0, 0.0, -1e-5), parts, 2000, seed)


def config5(seed=0, shape=(384, 384, 768), n_particles=3000):
    """384x384x768 bed: 3000 particles of 4-128 balls (log-uniform), R ~ U[8, 16],
    packed into the lower 18 % of the box by random sequential addition of
    spheres of radius 0.5 R, so dense that neighbouring particles interpenetrate
    and the broad phase yields about 49k candidate pairs (the ~50k active pairs
    of the learned-proposal workload)."""
    rng = np.random.default_rng(seed)
    specs = []
    for _ in range(n_particles):
        n = int(np.round(np.exp(rng.uniform(np.log(4), np.log(128)))))
        R = rng.uniform(8.0, 16.0)
        c, k, r = clustered(rng, n, R)
        specs.append((c, k, r))
    lo = np.array([2.0, 2.0, 2.0])
    hi = np.array([shape[0] - 2.0, shape[1] - 2.0, shape[2] * 0.18])
    pos = _place_non_overlapping(rng, [0.5 * s[2] for s in specs], lo, hi, 0.0)
    parts = [ParticleSpec(c, k, 2.5, 1.0, f32(p), random_unit_quaternion(rng), nominal_radius=r)
             for (c, k, r), p in zip(specs, pos)]
    return Scene("C5 384x384x768 3000-particle bed", shape, 0.8, (0.0, 0.0, -1e-5), parts, 100, seed)


# ---------------------------------------------------------------------------
# Point hulls for the Gradient Search refinement (Sec. 2.2): the scanned hulls
# of the paper are not available; these stand in for them.
# ---------------------------------------------------------------------------
def ellipsoid_hull(rng, m, semi, bumps=0.0):
    """m points on the surface of an ellipsoid with semi-axes semi (a random
    direction each, radius scaled along it), optionally with a smooth radial
    modulation 1 + bumps * sin(3 theta) cos(2 phi); float32 values."""
    u = rng.normal(size=(m, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    theta = np.arccos(np.clip(u[:, 2], -1.0, 1.0))
    phi = np.arctan2(u[:, 1], u[:, 0])
    r = 1.0 + bumps * np.sin(3.0 * theta) * np.cos(2.0 * phi)
    return f32(u * r[:, None] * np.asarray(semi, dtype=np.float64)[None, :])


def hull_planes(H):
    """Facet planes (nx, ny, nz, d) of the convex hull of the points H:
    outward unit normals, n . x <= d inside; float32 values."""
    from scipy.spatial import ConvexHull
    eq = ConvexHull(np.asarray(H, dtype=np.float64)).equations  # n . x + off <= 0 inside
    return f32(np.concatenate([eq[:, :3], -eq[:, 3:4]], axis=1))


def gs_start_model(rng, n, semi):
    """A starting model for the refinement: n control points uniform inside
    the ellipsoid shrunk to half its size, with equal k that make a single
    coincident ball of the ellipsoid's volume; float32 values."""
    c = uniform_in_ball(rng, n, 1.0) * 0.5 * np.asarray(semi, dtype=np.float64)[None, :]
    r_eq = float(np.prod(semi)) ** (1.0 / 3.0)
    k = np.full(n, r_eq * r_eq / n)
    return f32(c), f32(k)
