"""Shape descriptors of a metaball particle (Sec. 3, the sphericity, nominal
diameter, projected-area diameter and Corey shape factor of the DKT study)
for the oracle (test infrastructure only).

Definitions (the paper's):  Phi = S_sphere / S with S_sphere the surface of
the volume-equivalent sphere;  d_n = the diameter of the volume-equivalent
sphere;  d_s = sqrt(4 A_p / pi) with A_p the projected area;
CSF = d_s / sqrt(d_i d_l).

Readings (the paper leaves these open):
  D1  volume: midpoint quadrature of f >= 1 on a body-frame grid of spacing h
      over [-R_g, R_g]^3, R_g = max |c_j| + sqrt(sum k / (1 - eps)) (beyond
      it f < 1 - eps), cell centres at -R_g + (i + 1/2) h.
  D2  surface area: the coarea estimate S = (1 / 2 eps) sum over the cells
      with |f - 1| < eps of |grad f| h^3 (the band [1 - eps, 1 + eps] of the
      field holds 2 eps S to first order).
  D3  principal axes: the eigenvectors of the second moments of the solid
      cells about their centroid; the axis lengths d_l >= d_i >= d_sh are the
      extents of the solid along them, measured on a second grid of spacing h
      aligned with the axes (centred on the centroid, over R_g + 2 h): max -
      min of the solid cell centres' coordinates plus h.
  D4  A_p: the projection along the shortest axis (the largest projection of
      an ellipsoid-like body): h^2 times the number of columns of the second
      grid along that axis holding a solid cell.
  D5  the CSF's numerator is the shortest axis length d_sh (the Corey shape
      factor; the paper's symbol is also its projected-area diameter's).  For
      an ellipsoid these readings give d_n / d_s = CSF^(1/3) exactly, and the
      paper's table follows that relation within 0.9 % for all nine shapes.
The decision "f >= 1" and the band test are integers taken from FP32 values
the kernel computes, so they are taken here in FP32 with the same single
roundings (coordinates, differences, squares, sums, one IEEE division per
ball, ball order); the sums of the quadratures are FP64.
"""
import numpy as np



def _axis(n, lo, h):
    i = np.arange(n, dtype=np.float32)
    return np.float32(lo) + (i + np.float32(0.5)) * np.float32(h)


def field_f32(P, centers, k):
    """f at points P (..., 3) in FP32, ball order, single roundings."""
    P = np.asarray(P, dtype=np.float32)
    c = np.asarray(centers, dtype=np.float32)
    kk = np.asarray(k, dtype=np.float32)
    f = np.zeros(P.shape[:-1], dtype=np.float32)
    with np.errstate(divide="ignore"):
        for j in range(len(kk)):
            d0 = P[..., 0] - c[j, 0]
            d1 = P[..., 1] - c[j, 1]
            d2 = P[..., 2] - c[j, 2]
            r2 = (d0 * d0 + d1 * d1) + d2 * d2
            f = f + kk[j] / r2
    return f


def grad_norm(P, centers, k):
    """|grad f| at points P, FP64."""
    P = np.asarray(P, dtype=np.float64)
    g = np.zeros(P.shape)
    for j in range(len(k)):
        d = P - np.asarray(centers[j], dtype=np.float64)
        r2 = np.sum(d * d, axis=-1)
        g += (-2.0 * float(k[j]) / (r2 * r2))[..., None] * d
    return np.linalg.norm(g, axis=-1)


def grid_radius(centers, k, eps):
    """max |c_j| + sqrt(sum k / (1 - eps)): beyond it f < 1 - eps, so the
    grid holds the solid and the whole band (FP64, then FP32)."""
    c = np.asarray(centers, dtype=np.float64)
    kk = np.asarray(k, dtype=np.float64)
    return float(np.sqrt((c * c).sum(1)).max() + np.sqrt(kk.sum() / (1.0 - eps)))


def descriptors(centers, k, h, eps=0.1):
    """Volume, surface, principal axes, extents, projected area and the four
    descriptors of one metaball model (body frame)."""
    centers = np.asarray(centers, dtype=np.float32)
    k = np.asarray(k, dtype=np.float32)
    h = float(np.float32(h))  # the spacing is the FP32 value the coordinates use
    Rb = np.float32(grid_radius(centers, k, eps))
    n = int(np.ceil(2.0 * float(Rb) / h))
    ax = _axis(n, -Rb, h)
    vol_cells, s_band = 0, 0.0
    m1 = np.zeros(3)
    m2 = np.zeros((3, 3))
    for iz in range(n):
        zz, yy, xx = np.meshgrid(ax[iz:iz + 1], ax, ax, indexing="ij")
        P = np.stack([xx, yy, zz], axis=-1).reshape(-1, 3)
        f = field_f32(P, centers, k)
        inside = f >= np.float32(1.0)
        band = np.abs(f - np.float32(1.0)) < np.float32(eps)
        q = P[inside].astype(np.float64)
        vol_cells += int(inside.sum())
        m1 += q.sum(0)
        m2 += q.T @ q
        if band.any():
            s_band += float(grad_norm(P[band], centers, k).sum())
    dv = float(h) ** 3
    V = vol_cells * dv
    S = s_band * dv / (2.0 * eps)
    cen = m1 / vol_cells
    cov = m2 / vol_cells - np.outer(cen, cen)
    w, E = np.linalg.eigh(cov)          # ascending: shortest axis first
    E = E[:, ::-1]                      # longest, intermediate, shortest
    # second grid along the axes, centred on the centroid, two cells wider
    n2 = n + 4
    ax2 = _axis(n2, -(Rb + np.float32(2.0 * h)), h)
    ext_lo = np.full(3, np.inf)
    ext_hi = np.full(3, -np.inf)
    cols = set()
    A = E.astype(np.float32)
    c32 = cen.astype(np.float32)
    for iz in range(n2):
        u3, u2, u1 = np.meshgrid(ax2[iz:iz + 1], ax2, ax2, indexing="ij")
        U = np.stack([u1, u2, u3], axis=-1).reshape(-1, 3).astype(np.float32)
        B = c32[None, :] + U @ A.T
        inside = field_f32(B, centers, k) >= np.float32(1.0)
        if inside.any():
            Ui = U[inside].astype(np.float64)
            ext_lo = np.minimum(ext_lo, Ui.min(0))
            ext_hi = np.maximum(ext_hi, Ui.max(0))
            iu = np.nonzero(inside)[0]
            for a, b in zip(iu % n2, iu // n2):  # columns along the shortest axis (u3)
                cols.add((int(a), int(b)))
    L = ext_hi - ext_lo + h
    Ap = len(cols) * float(h) ** 2
    d_n = (6.0 * V / np.pi) ** (1.0 / 3.0)
    d_s = np.sqrt(4.0 * Ap / np.pi)
    return {"volume": V, "surface": S, "axes": E, "eigenvalues": w[::-1], "lengths": L, "projected_area": Ap,
            "sphericity": np.pi * d_n * d_n / S, "d_n": d_n, "d_s": d_s,
            "csf": L[2] / np.sqrt(L[1] * L[0]), "cells": vol_cells}
