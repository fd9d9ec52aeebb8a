"""Metaball field and solid flagging for the oracle (test infrastructure only),
float64.

Eq. 1 (Sec. 2.1): f(x) = sum_i k_i / |x - c_i|^2; the surface is f = 1, points
with f > 1 are inside, f ranges over (0, inf).  Readings:
  A1  a node exactly on a control point gives an infinite term: inside.
  A2  f >= 1 is solid (the surface itself counts as solid).
  A3  a particle's body frame has its origin at the particle position X and
      axes given by the unit quaternion q (w, x, y, z); a world point x maps
      to the body point x_b = R(q)^T (x - X).
  A4  a node inside several particles belongs to the lowest particle index
      (the paper does not treat overlapping solids).
  A5  node (i, j, k) sits at (i, j, k).
  A6  a particle's field is not wrapped across periodic faces.

Arithmetic order is spelled out (left to right, ball order) because the GPU
re-evaluates nodes within a guard band of f = 1 in FP64 in the same order.
"""
import numpy as np


def quat_to_matrix(q):
    """Rotation matrix (body -> world) of the quaternion q = (w, x, y, z),
    normalised first."""
    w, x, y, z = (float(v) for v in q)
    n = np.sqrt(((w * w + x * x) + y * y) + z * z)
    w, x, y, z = w / n, x / n, y / n, z / n
    return np.array([
        [1.0 - 2.0 * (y * y + z * z), 2.0 * (x * y - w * z), 2.0 * (x * z + w * y)],
        [2.0 * (x * y + w * z), 1.0 - 2.0 * (x * x + z * z), 2.0 * (y * z - w * x)],
        [2.0 * (x * z - w * y), 2.0 * (y * z + w * x), 1.0 - 2.0 * (x * x + y * y)],
    ])


def to_body(points, X, R):
    """x_b = R^T (x - X) for points of shape (..., 3)."""
    p = np.asarray(points, dtype=np.float64)
    d0 = p[..., 0] - X[0]
    d1 = p[..., 1] - X[1]
    d2 = p[..., 2] - X[2]
    b0 = (R[0, 0] * d0 + R[1, 0] * d1) + R[2, 0] * d2
    b1 = (R[0, 1] * d0 + R[1, 1] * d1) + R[2, 1] * d2
    b2 = (R[0, 2] * d0 + R[1, 2] * d1) + R[2, 2] * d2
    return np.stack([b0, b1, b2], axis=-1)


def field(xb, centers, k):
    """f(x_b) = sum_i k_i / |x_b - c_i|^2 (Eq. 1), summed in ball order."""
    xb = np.asarray(xb, dtype=np.float64)
    f = np.zeros(xb.shape[:-1])
    with np.errstate(divide="ignore"):
        for i in range(len(k)):
            d0 = xb[..., 0] - centers[i, 0]
            d1 = xb[..., 1] - centers[i, 1]
            d2 = xb[..., 2] - centers[i, 2]
            r2 = (d0 * d0 + d1 * d1) + d2 * d2
            f = f + k[i] / r2
    return f


def gradient(xb, centers, k):
    """grad f = sum_i -2 k_i (x - c_i) / |x - c_i|^4."""
    xb = np.asarray(xb, dtype=np.float64)
    g = np.zeros(xb.shape)
    for i in range(len(k)):
        d = xb - centers[i]
        r2 = (d * d).sum(-1)
        g = g + (-2.0 * k[i] / (r2 * r2))[..., None] * d
    return g


def hessian(xb, centers, k):
    """Hessian of f: sum_i k_i (8 d d^T / |d|^6 - 2 I / |d|^4), d = x - c_i."""
    xb = np.asarray(xb, dtype=np.float64)
    H = np.zeros(xb.shape[:-1] + (3, 3))
    eye = np.eye(3)
    for i in range(len(k)):
        d = xb - centers[i]
        r2 = (d * d).sum(-1)
        H = H + (8.0 * k[i] / r2 ** 3)[..., None, None] * (d[..., :, None] * d[..., None, :]) \
            - (2.0 * k[i] / (r2 * r2))[..., None, None] * eye
    return H


def bounding_radius(centers, k):
    """R_b = max_i |c_i| + sqrt(sum_i k_i).  Beyond it every term is below
    k_i / sum k, so f < 1: every solid node lies within R_b of the origin."""
    return float(np.sqrt((centers * centers).sum(1)).max() + np.sqrt(k.sum()))


def node_box(X, Rb, shape):
    """Integer node range [lo, hi) per axis covering |x - X| <= R_b, clipped."""
    lo = [max(0, int(np.floor(X[a] - Rb)) - 1) for a in range(3)]
    hi = [min(shape[a], int(np.ceil(X[a] + Rb)) + 2) for a in range(3)]
    return lo, hi


def flag_nodes(shape, particles):
    """Owner index per node (nz, ny, nx): the lowest particle index p with
    f_p(R_p^T (x - X_p)) >= 1, else -1 (fluid).

    particles: list of dicts with keys centers, k, pos, quat.
    shape: (nx, ny, nz).
    """
    nx, ny, nz = shape
    owner = np.full((nz, ny, nx), -1, dtype=np.int64)
    for p, P in enumerate(particles):
        X = np.asarray(P["pos"], dtype=np.float64)
        R = quat_to_matrix(P["quat"])
        Rb = bounding_radius(P["centers"], P["k"])
        lo, hi = node_box(X, Rb, shape)
        if any(hi[a] <= lo[a] for a in range(3)):
            continue
        zz, yy, xx = np.meshgrid(np.arange(lo[2], hi[2]), np.arange(lo[1], hi[1]), np.arange(lo[0], hi[0]),
                                 indexing="ij")
        pts = np.stack([xx, yy, zz], axis=-1).astype(np.float64)
        f = field(to_body(pts, X, R), P["centers"], P["k"])
        sub = owner[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]
        sub[(f >= 1.0) & (sub < 0)] = p
    return owner


def mass_properties(centers, k, density, h=0.25):
    """Volume, centroid, mass and inertia tensor (about the centroid, body
    axes) by midpoint quadrature of the indicator f >= 1 on a grid of spacing
    h over [-R_b, R_b]^3.  Reading A15: the paper defers these to its
    reference [zhang2021metaball]; grid quadrature is the plain definition of
    the integrals."""
    Rb = bounding_radius(centers, k)
    n = int(np.ceil(2 * Rb / h))
    ax = -Rb + (np.arange(n) + 0.5) * h
    V = 0.0
    S = np.zeros(3)
    SS = np.zeros((3, 3))
    for iz in range(n):  # slab by slab to bound memory
        zz, yy, xx = np.meshgrid(ax[iz:iz + 1], ax, ax, indexing="ij")
        pts = np.stack([xx, yy, zz], axis=-1).reshape(-1, 3)
        inside = field(pts, centers, k) >= 1.0
        q = pts[inside]
        V += inside.sum()
        S += q.sum(0)
        SS += q.T @ q
    dv = h ** 3
    vol = V * dv
    c = S * dv / vol
    second = SS * dv - vol * np.outer(c, c)  # about the centroid
    mass = density * vol
    I = density * (np.trace(second) * np.eye(3) - second)
    return {"volume": vol, "centroid": c, "mass": mass, "inertia": I}
