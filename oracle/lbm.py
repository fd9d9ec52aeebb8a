"""Lattice Boltzmann part of the oracle (test infrastructure only), float64.

State convention (pull scheme): the stored array holds the POST-collision
populations f+(x, t), shape (19, nz, ny, nx), node (i, j, k) at position
(x=i, y=j, z=k) (reading A5).  One step is

    f_in(x, t+1)  = f+_i(x - e_i, t)          (streaming, pull form)
    f+(x, t+1)    = f_in - (f_in - f_eq)/tau   (BGK collision)

The paper introduces the distribution G_i, the weights omega_i and the lattice
speed C (Sec. 2.3.2); the lattice itself (D3Q19) and BGK collision are readings
A23.  Domain walls are halfway bounce-back at -1/2 and N-1/2 with an optional
wall velocity (moving-wall term 6 w_i rho0 e_i.u_wall / C^2, the same form the
paper uses for its particle walls in the bounce-back equation of Sec. 2.3.2).
Guo forcing (reading A27) is a test-only addition used by the Poiseuille pin.
"""
import functools

import numpy as np

from .d3q19 import E, W, OPP, Q

_EF = E.astype(np.float64)


def equilibrium(rho, u):
    """Second-order equilibrium f_i^eq = w_i rho (1 + 3 e.u + 9/2 (e.u)^2 - 3/2 u.u).

    rho: array of shape S; u: array of shape (3,) + S.  Returns (19,) + S.
    """
    rho = np.asarray(rho, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2]
    out = np.empty((Q,) + rho.shape, dtype=np.float64)
    for i in range(Q):
        eu = _EF[i, 0] * u[0] + _EF[i, 1] * u[1] + _EF[i, 2] * u[2]
        out[i] = W[i] * rho * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * usq)
    return out


def moments(f, force=None):
    """Density rho = sum_i f_i and velocity u = (sum_i e_i f_i + F/2) / rho.

    The F/2 shift is part of Guo forcing (reading A27); force=None means F = 0.
    """
    rho = f.sum(axis=0)
    mom = np.stack([(_EF[:, a].reshape((Q,) + (1,) * (f.ndim - 1)) * f).sum(axis=0)
                    for a in range(3)])
    if force is not None:
        mom = mom + 0.5 * np.asarray(force, dtype=np.float64).reshape((3,) + (1,) * (f.ndim - 1))
    return rho, mom / rho


def collide(f, tau, force=None):
    """BGK collision f+ = f - (f - f^eq(rho, u)) / tau, plus the Guo source term

        (1 - 1/(2 tau)) w_i [3 (e_i - u) + 9 (e_i.u) e_i] . F

    when a uniform body-force density F (3-vector) is given.
    """
    rho, u = moments(f, force)
    feq = equilibrium(rho, u)
    out = f - (f - feq) / tau
    if force is not None:
        F = np.asarray(force, dtype=np.float64)
        for i in range(Q):
            eu = _EF[i, 0] * u[0] + _EF[i, 1] * u[1] + _EF[i, 2] * u[2]
            s = 0.0
            for a in range(3):
                s = s + (3.0 * (_EF[i, a] - u[a]) + 9.0 * eu * _EF[i, a]) * F[a]
            out[i] = out[i] + (1.0 - 0.5 / tau) * W[i] * s
    return out


@functools.lru_cache(maxsize=256)
def _wall_face_cached(shape, e, periodic):
    face = wall_face_of_source(shape, e, periodic)
    face.setflags(write=False)
    return face


def wall_face_of_source(shape, e, periodic):
    """For destination nodes whose source x - e lies outside the domain along a
    non-periodic axis, return the index of the wall face crossed
    (0:x-, 1:x+, 2:y-, 3:y+, 4:z-, 5:z+), else -1.

    A corner crossing two faces is attributed to the first axis in the order
    x, y, z (the paper does not treat corners; only the face whose wall moves
    matters in the tests).
    """
    nz, ny, nx = shape
    Z, Y, X = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    face = np.full(shape, -1, dtype=np.int64)
    coords = (X, Y, Z)
    sizes = (nx, ny, nz)
    for a in (2, 1, 0):  # later assignment (lower axis) wins
        if periodic[a]:
            continue
        src = coords[a] - e[a]
        face[src < 0] = 2 * a
        face[src > sizes[a] - 1] = 2 * a + 1
    return face


def stream_pull(fpost, periodic=(False, False, False), wall_velocity=None, rho0=1.0):
    """Pull streaming f_in_i(x) = f+_i(x - e_i), with halfway bounce-back

        f_in_i(x) = f+_{opp i}(x) + 6 w_i rho0 (e_i . u_wall)

    where x - e_i is outside the domain along a non-periodic axis.
    wall_velocity: (6, 3) per face (0:x-, 1:x+, 2:y-, 3:y+, 4:z-, 5:z+).
    """
    wv = np.zeros((6, 3)) if wall_velocity is None else np.asarray(wall_velocity, dtype=np.float64)
    shape = fpost.shape[1:]
    fin = np.empty_like(fpost)
    for i in range(Q):
        ex, ey, ez = (int(v) for v in E[i])
        fin[i] = np.roll(fpost[i], shift=(ez, ey, ex), axis=(0, 1, 2))
        if i == 0:
            continue
        face = _wall_face_cached(tuple(shape), (ex, ey, ez), tuple(bool(p) for p in periodic))
        m = face >= 0
        if m.any():
            uw = wv[face[m]]
            eu = _EF[i, 0] * uw[:, 0] + _EF[i, 1] * uw[:, 1] + _EF[i, 2] * uw[:, 2]
            fin[i][m] = fpost[OPP[i]][m] + 6.0 * W[i] * rho0 * eu
    return fin


def step_bulk(fpost, tau, periodic=(False, False, False), wall_velocity=None, rho0=1.0, force=None):
    """One particle-free LBM step: stream (pull, walls) then BGK collide."""
    return collide(stream_pull(fpost, periodic, wall_velocity, rho0), tau, force)


def rest_state(shape, rho0=1.0):
    """f+ = f^eq(rho0, 0) = w_i rho0 at every node."""
    return np.broadcast_to((W * rho0).reshape((Q, 1, 1, 1)), (Q,) + tuple(shape)).copy()


def update_cells(fpost, cells, tau, periodic=(False, False, False), wall_velocity=None,
                 rho0=1.0, force=None):
    """The same stream + collide as `step_bulk`, evaluated only at the listed
    cells (array of (x, y, z) rows); returns f+(t+1) at those cells, shape
    (19, n).  Used to check sampled outputs of large lattices one by one.

    `fpost` may be any object indexable as fpost[i, z, y, x] with integer
    arrays (numpy array or a lazy gatherer).
    """
    wv = np.zeros((6, 3)) if wall_velocity is None else np.asarray(wall_velocity, dtype=np.float64)
    cells = np.asarray(cells, dtype=np.int64)
    nz, ny, nx = fpost.shape[1:]
    sizes = (nx, ny, nz)
    n = cells.shape[0]
    fin = np.empty((Q, n), dtype=np.float64)
    own = np.stack([np.asarray(fpost[j, cells[:, 2], cells[:, 1], cells[:, 0]], dtype=np.float64)
                    for j in range(Q)])
    for i in range(Q):
        src = cells - E[i][None, :]
        face = np.full(n, -1, dtype=np.int64)
        for a in (2, 1, 0):
            if periodic[a]:
                src[:, a] %= sizes[a]
                continue
            face[src[:, a] < 0] = 2 * a
            face[src[:, a] > sizes[a] - 1] = 2 * a + 1
        inside = face < 0
        vals = np.empty(n, dtype=np.float64)
        if inside.any():
            s = src[inside]
            vals[inside] = np.asarray(fpost[i, s[:, 2], s[:, 1], s[:, 0]], dtype=np.float64)
        if (~inside).any():
            uw = wv[face[~inside]]
            eu = _EF[i, 0] * uw[:, 0] + _EF[i, 1] * uw[:, 1] + _EF[i, 2] * uw[:, 2]
            vals[~inside] = own[OPP[i]][~inside] + 6.0 * W[i] * rho0 * eu
        fin[i] = vals
    return collide(fin, tau, force)
