"""Closed-form pin of the oracle's interpolated bounce-back population
(Sec. 2.3.2, Eqs. eqneq1, eqneq2, neqd; readings A8, A9) on single links cut
by a flat wall.

A linear velocity field u(x) = a (z - z_w) that vanishes on the plane
z = z_w, with a uniform first-order non-equilibrium part, is a flow that the
wall at rest does not disturb: extended into the solid, its populations are
what a link should pull back.  For a link (x_f, d) that crosses the plane at
x_w = x_f + q e_d, the returned population G_{opp d}(x_f, t+1) must equal
the extended field's f+_{opp d}(x_f + e_d).  The paper's scheme meets this
exactly (to rounding) for every q: u_d = u(x_f + (2q - 1) e_d) = a (1 - q)
mirrors the solid-side velocity u(x_f + e_d) = -a (1 - q), so the equilibria
differ only by the linear term that the moving-wall form of the rule restores,
and the non-equilibrium parts agree because the field's gradient is uniform
and even in e.  Halfway bounce-back (Ladd) meets it exactly at q = 1/2 only.
A wall moving along the plane keeps the identity to first order in u; the
quadratic remainder is bounded in closed form below.

A plausible slip in the oracle (u_f or u_ff in place of u_d, the
non-equilibrium part taken at u_ff, the neighbour x_f + e_d in place of
x_f - e_d, the sign of the moving-wall term) moves G by ~w_d |a| or more,
10^10 times the tolerance of the resting-wall case.  The choice between the
two branches of u* (q <= 1/2 or not) is not pinned here: both are exact for
any linear field.
"""
import numpy as np
import pytest

from oracle import coupling, lbm
from oracle.d3q19 import E, OPP, Q, W

EF = E.astype(np.float64)
SHAPE = (8, 8, 10)          # nx, ny, nz
Z_F = 4                     # row of fluid nodes next to the wall
A_SHEAR = np.array([2.0e-3, -1.5e-3, 4.0e-4])
TAU = 0.8
DOWN = [d for d in range(1, Q) if E[d][2] == -1]   # links from row Z_F into the solid below


def _neq(grad):
    """Uniform first-order non-equilibrium part of post-collision populations:
    -3 w_i (tau - 1) (e_i e_i - I/3) : grad u  (the Chapman-Enskog form; any
    constant multiple would do for the identity)."""
    out = np.empty(Q)
    for i in range(Q):
        Qi = np.outer(EF[i], EF[i]) - np.eye(3) / 3.0
        out[i] = -3.0 * W[i] * (TAU - 1.0) * np.sum(Qi * grad)
    return out


def _field(z_w, U, rho=1.0):
    """The extended field's post-collision populations on the whole lattice
    (solid nodes included) and a function giving them at any point."""
    grad = np.outer(np.array([0.0, 0.0, 1.0]), A_SHEAR)  # d u_b / d x_a: only d/dz
    neq = _neq(grad)

    def at(points):
        p = np.atleast_2d(points)
        u = U[None, :] + (p[:, 2] - z_w)[:, None] * A_SHEAR[None, :]
        feq = lbm.equilibrium(np.full(len(p), rho), u.T)
        return feq + neq[:, None]

    nx, ny, nz = SHAPE
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    pts = np.stack([xx.ravel(), yy.ravel(), zz.ravel()], 1).astype(np.float64)
    f = at(pts).reshape(Q, nz, ny, nx)
    return f, at


def _links(q):
    nx, ny, _ = SHAPE
    cells, dirs = [], []
    for y in range(ny):
        for x in range(nx):
            for d in DOWN:
                cells.append((x, y, Z_F))
                dirs.append(d)
    cell = np.array(cells, dtype=np.int64)
    d = np.array(dirs, dtype=np.int64)
    return cell, d, np.full(len(d), q)


def _solid():
    nx, ny, nz = SHAPE
    s = np.zeros((nz, ny, nx), dtype=bool)
    s[:Z_F] = True
    return s


def _returned_and_target(q, U, bb_mode):
    z_w = Z_F - q
    f, at = _field(z_w, U)
    cell, d, qv = _links(q)
    u_w = np.tile(U, (len(d), 1))   # the wall moves rigidly with U (rest: U = 0)
    G = coupling.bounce_back_populations(f, cell, d, qv, u_w, _solid(), (True, True, False), bb_mode)
    src = cell.astype(np.float64) + EF[d]             # x_f + e_d, inside the solid
    target = at(src)[OPP[d], np.arange(len(d))]       # f+_{opp d} of the extended field there
    return G, target, cell, d


@pytest.mark.parametrize("q", [0.05, 0.25, 0.4, 0.5, 0.6, 0.75, 0.95, 1.0])
def test_ibb_exact_for_linear_shear_past_resting_wall(q):
    G, target, _, d = _returned_and_target(q, np.zeros(3), "ibb")
    assert np.all(np.isin(d, [6, 12, 13, 16, 17]))
    err = np.abs(G - target).max()
    assert err <= 1e-15, err
    # the links carry the shear: a first-order slip would show
    assert np.abs(target - W[OPP[d]]).max() > 1e-5


def test_ladd_exact_only_at_half():
    G, target, _, _ = _returned_and_target(0.5, np.zeros(3), "ladd")
    assert np.abs(G - target).max() <= 1e-15
    G, target, _, d = _returned_and_target(0.2, np.zeros(3), "ladd")
    assert np.abs(G - target).max() > 1e-6      # halfway bounce-back is first order off elsewhere


@pytest.mark.parametrize("q", [0.1, 0.3, 0.7, 0.9])
def test_ibb_moving_wall_first_order(q):
    """Wall sliding at U = (0.004, -0.003, 0) along the plane: G equals the
    extended field's pulled population up to the quadratic terms of f^eq,
    w_d [4.5 |e.(u_d - u_s)| |e.(u_d + u_s)| + 1.5 |u_d - u_s| |u_d + u_s|],
    with u_d = u(x_f + (2q - 1) e_d), u_s = u(x_f + e_d)."""
    U = np.array([0.004, -0.003, 0.0])
    G, target, cell, d = _returned_and_target(q, U, "ibb")
    z_w = Z_F - q
    pd = cell + (2.0 * q - 1.0) * EF[d]
    ps = cell + EF[d]
    ud = U[None, :] + (pd[:, 2] - z_w)[:, None] * A_SHEAR
    us = U[None, :] + (ps[:, 2] - z_w)[:, None] * A_SHEAR
    e = EF[d]
    dm, sm = ud - us, ud + us
    bound = W[d] * (4.5 * np.abs((e * dm).sum(1)) * np.abs((e * sm).sum(1))
                    + 1.5 * np.linalg.norm(dm, axis=1) * np.linalg.norm(sm, axis=1))
    err = np.abs(G - target)
    assert np.all(err <= bound + 1e-15), (err / (bound + 1e-30)).max()
    # and the first-order term that u_d carries is far above that remainder
    first = 3.0 * W[d] * np.abs((e * (ud - (U + (cell[:, 2] - z_w)[:, None] * A_SHEAR))).sum(1))
    assert first.max() > 5.0 * bound.max()
