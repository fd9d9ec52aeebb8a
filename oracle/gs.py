"""Gradient Search refinement of a metaball model on a point hull (Sec. 2.2,
Algorithm 2, Eq. GSloss) for the oracle (test infrastructure only), float64.

A model M is n control points (c_j, k_j); its field at a hull point H_i is
f_i = sum_j k_j / |H_i - c_j|^2 (Eq. 1).  The refinement loss (Eq. GSloss) is
summed over the hull points, piecewise in f_i:
    (f - 1)^2                   for f in [2, inf)
    |f - 1|                     for f in [1, 2)
    (f - 1)^2 + 1/f - 1         for f in [0, 1)
and the search is full-batch gradient descent M <- M - eta grad L(M) for E
epochs, an anomaly detection, and E more epochs (Algorithm 2).

Readings (the paper leaves these open):
  G1  the branch intervals are taken as printed, with f = 2 in the first
      branch and f = 1 in the second (the pieces agree at both points).
  G2  dL/df = 2 (f - 1) on [2, inf), +1 on [1, 2) (the |f - 1| branch, f = 1
      included), 2 (f - 1) - 1/f^2 on [0, 1).
  G3  the parameters are every c_j and k_j; the gradient is the exact sum over
      all hull points (the paper computes the whole hull's gradient once per
      iteration); eta and E are inputs.
  G4  "cleared by assigning a zero weight": an anomalous control point gets
      k_j = 0 and takes no further part (it is not updated in the second
      descent).
  G5  a control point "outside the point hull" lies outside the convex hull of
      H: n . c > d for some facet plane (n, d) of it (outward unit normal n).
      The decision is an integer taken from floating point, so it is made in
      FP32 (single rounding of each product and sum, left to right), as the
      kernel makes it; the planes are inputs (the hull's facets).
  G6  a sign abnormality is k_j < 0.
"""
import numpy as np


def field(H, c, k):
    """f_i = sum_j k_j / |H_i - c_j|^2 for H (m, 3), c (n, 3), k (n,)."""
    d = np.asarray(H, dtype=np.float64)[:, None, :] - np.asarray(c, dtype=np.float64)[None, :, :]
    r2 = np.sum(d * d, axis=2)
    return np.sum(np.asarray(k, dtype=np.float64)[None, :] / r2, axis=1)


def loss_terms(f):
    """Per-point loss of Eq. GSloss (readings G1)."""
    f = np.asarray(f, dtype=np.float64)
    return np.where(f >= 2.0, (f - 1.0) ** 2,
                    np.where(f >= 1.0, np.abs(f - 1.0), (f - 1.0) ** 2 + 1.0 / f - 1.0))


def loss(H, c, k):
    return float(np.sum(loss_terms(field(H, c, k))))


def dloss_df(f):
    """dL/df per point (reading G2)."""
    f = np.asarray(f, dtype=np.float64)
    return np.where(f >= 2.0, 2.0 * (f - 1.0), np.where(f >= 1.0, 1.0, 2.0 * (f - 1.0) - 1.0 / (f * f)))


def gradient(H, c, k):
    """(dL/dc (n, 3), dL/dk (n,)) by the chain rule through f:
    df_i/dk_j = 1/r_ij^2, df_i/dc_j = 2 k_j (H_i - c_j) / r_ij^4."""
    H = np.asarray(H, dtype=np.float64)
    c = np.asarray(c, dtype=np.float64)
    k = np.asarray(k, dtype=np.float64)
    d = H[:, None, :] - c[None, :, :]           # (m, n, 3)
    r2 = np.sum(d * d, axis=2)                   # (m, n)
    f = np.sum(k[None, :] / r2, axis=1)
    w = dloss_df(f)                              # (m,)
    gk = np.sum(w[:, None] / r2, axis=0)
    gc = np.sum((w[:, None] * 2.0 * k[None, :] / (r2 * r2))[:, :, None] * d, axis=0)
    return gc, gk


def descend(H, c, k, epochs, lr, active=None):
    """E full-batch gradient-descent epochs; only active control points move."""
    c = np.array(c, dtype=np.float64)
    k = np.array(k, dtype=np.float64)
    act = np.ones(len(k), dtype=bool) if active is None else np.asarray(active, dtype=bool)
    for _ in range(epochs):
        gc, gk = gradient(H, c, k)
        c[act] -= lr * gc[act]
        k[act] -= lr * gk[act]
    return c, k


def outside_hull_f32(c, planes):
    """Reading G5: True where n . c > d for some plane (nx, ny, nz, d), the
    dot product and comparison in FP32, left to right (every product and sum
    an FP32 rounding of its own, as numpy float32 arrays compute them)."""
    c32 = np.asarray(c, dtype=np.float32).reshape(-1, 3)
    P = np.asarray(planes, dtype=np.float32)
    s = (P[None, :, 0] * c32[:, None, 0]) + (P[None, :, 1] * c32[:, None, 1])
    s = s + (P[None, :, 2] * c32[:, None, 2])
    return np.any(s > P[None, :, 3], axis=1)


def anomaly(c, k, planes):
    """Anomaly detection (readings G4-G6): the control points outside the
    hull or with k < 0 get k = 0 and become inactive."""
    k = np.array(k, dtype=np.float64)
    bad = outside_hull_f32(c, planes) | (k < 0.0)
    k[bad] = 0.0
    return k, ~bad


def gs_fit(H, c0, k0, epochs, lr, planes):
    """Algorithm 2: descent, anomaly detection, descent.  Returns the refined
    (c, k), the active mask, and the loss after each descent."""
    c, k = descend(H, c0, k0, epochs, lr)
    l1 = loss(H, c, k)
    k, active = anomaly(c, k, planes)
    c, k = descend(H, c, k, epochs, lr, active)
    return c, k, active, l1, loss(H, c, k)
