"""Fluid-particle coupling of the oracle (test infrastructure only), float64.

Sec. 2.3.2: nodes are fluid, solid, or boundary (fluid nodes next to a solid);
missing populations at boundary nodes come from the interpolated bounce-back
(IBB, Eqs. eqneq1, eqneq2, neqd); the hydrodynamic force is the Galilean-
invariant momentum exchange; nodes a particle uncovers are refilled by a local
bounce-back rule with an equilibrium fallback.

Readings (the paper leaves these open):
  A7   a link (x_f, d) joins a fluid node x_f to a solid neighbour x_f + e_d; q
       solves f_p(x_f + q e_d) = c0 with c0 = 1 (the fluid sees the same
       surface as the flagging), by 60 bisection steps on [0, 1].
  A8   IBB: G_{opp d}(x_f, t+1) = f^eq_d(rho_f, u_d) + [f+_d(x_f, t) -
       f^eq_d(rho_f, u_f)] + 6 w_d rho0 (e_{opp d} . u_w): the departure-point
       non-equilibrium part is taken at x_f; rho_f, u_f are the moments of the
       stored f+(x_f, t); u_ff those of x_ff = x_f - e_d when that node is fluid
       (else u_ff = u_f); u_w = v_p + omega_p x (x_w - X_p), x_w = x_f + q e_d.
  A9   the density in the moving-wall term is rho0.
  A10  momentum exchange per link: dP = (e_d - u_w) f+_d(x_f, t)
       - (e_{opp d} - u_w) G_{opp d}(x_f, t+1), summed per particle; torque
       arm x_w - X_p.
  A11  by default no momentum correction for covered/uncovered nodes.  As an
       option (cover_uncover), the correction of Lorenz et al. (2009), whom
       the paper cites for its momentum exchange: a node covered this step
       (fluid at the previous step, solid now) hands the momentum of its
       stored post-collision populations, J = sum_i e_i f+_i(x, t), to the
       particle that covers it (F += J, T += (x - X_p) x J); a node
       uncovered this step takes the momentum of its refilled populations,
       J' = sum_i e_i f+_i(x_new) after A12, from the particle that uncovered
       it (F -= J', T -= (x_new - X_p) x J').  With the plain exchange (u_w
       terms left out) fluid plus particles then conserve momentum exactly.
  A12  refill of a node x_new uncovered this step (fluid now, solid at the
       previous step), applied to its stored post-collision populations before
       streaming: f+_i(x_new) = f+_{opp i}(x_new + e_i) + 6 w_i rho0 (e_i .
       u_new) when x_new + e_i is a fluid node that was fluid at the previous
       step too (the population "exists": it streams into x_new), else
       f^eq_i(rho0, u_new); u_new is the velocity at x_new of the particle that
       covered it.
  A13  order within a step: flag at the current pose, links, refill, stream
       with bounce-back, collide, momentum exchange.
  MI_BB_LADD (alternative mode): G_{opp d} = f+_d(x_f, t) + 6 w_d rho0
       (e_{opp d} . u_w) with x_w = x_f + e_d / 2.
"""
import numpy as np

from . import lbm
from .d3q19 import E, OPP, Q, W
from .metaball import field, quat_to_matrix, to_body

_EF = E.astype(np.float64)


def _wrap(c, shape, periodic):
    """Wrap integer coordinates (..., 3) on periodic axes; return (coords,
    inside-domain mask)."""
    c = np.array(c, dtype=np.int64, copy=True)
    ok = np.ones(c.shape[:-1], dtype=bool)
    for a in range(3):
        if periodic[a]:
            c[..., a] %= shape[a]
        else:
            ok &= (c[..., a] >= 0) & (c[..., a] < shape[a])
    return c, ok


def classify(owner, owner_prev):
    """Boolean node classes from owner fields (-1 fluid): solid and new."""
    solid = owner >= 0
    new = (~solid) & (owner_prev >= 0)
    return solid, new


def find_links(owner, periodic=(False, False, False)):
    """Links (x_f, d, p): x_f fluid, x_f + e_d solid with owner p.
    Returns arrays cell (n, 3) as (x, y, z), dir (n,), particle (n,), sorted by
    (particle, linear cell index, dir)."""
    nz, ny, nx = owner.shape
    shape = (nx, ny, nz)
    fz, fy, fx = np.nonzero(owner < 0)
    fl = np.stack([fx, fy, fz], axis=1)
    cells, dirs, parts = [], [], []
    for d in range(1, Q):
        nb, ok = _wrap(fl + E[d], shape, periodic)
        o = np.full(len(fl), -1, dtype=np.int64)
        o[ok] = owner[nb[ok, 2], nb[ok, 1], nb[ok, 0]]
        m = o >= 0
        cells.append(fl[m])
        dirs.append(np.full(m.sum(), d, dtype=np.int64))
        parts.append(o[m])
    cell = np.concatenate(cells) if cells else np.zeros((0, 3), np.int64)
    dr = np.concatenate(dirs) if dirs else np.zeros(0, np.int64)
    pt = np.concatenate(parts) if parts else np.zeros(0, np.int64)
    lin = (cell[:, 2] * ny + cell[:, 1]) * nx + cell[:, 0]
    order = np.lexsort((dr, lin, pt))
    return cell[order], dr[order], pt[order]


def wall_fraction(cell, d, P, iters=60):
    """q in (0, 1] with f_p(x_f + q e_d) = 1, by bisection on [0, 1] (A7).
    f(x_f) < 1 (fluid) and f(x_f + e_d) >= 1 (solid) bracket the root."""
    X = np.asarray(P["pos"], dtype=np.float64)
    R = quat_to_matrix(P["quat"])
    x0 = np.asarray(cell, dtype=np.float64)
    e = _EF[np.asarray(d)]
    lo = np.zeros(len(x0))
    hi = np.ones(len(x0))
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        f = field(to_body(x0 + mid[:, None] * e, X, R), P["centers"], P["k"])
        inside = f >= 1.0
        hi = np.where(inside, mid, hi)
        lo = np.where(inside, lo, mid)
    return 0.5 * (lo + hi)


def rigid_velocity(P, x):
    """u = v + omega x (x - X) at world points x (..., 3)."""
    v = np.asarray(P["vel"], dtype=np.float64)
    w = np.asarray(P["omega"], dtype=np.float64)
    r = np.asarray(x, dtype=np.float64) - np.asarray(P["pos"], dtype=np.float64)
    return v + np.cross(w, r)


def departure_velocity(q, u_f, u_ff, u_w):
    """u_d = u*/3 + 2 u**/3 (Eq. neqd) with the paper's piecewise u* and u**."""
    q = np.asarray(q, dtype=np.float64)[..., None]
    u_star = np.where(q <= 0.5, 2.0 * q * u_f + (1.0 - 2.0 * q) * u_ff,
                      ((1.0 - q) / q) * u_f + ((2.0 * q - 1.0) / q) * u_w)
    u_2star = ((1.0 - q) / (1.0 + q)) * u_ff + (2.0 * q / (1.0 + q)) * u_w
    return u_star / 3.0 + 2.0 * u_2star / 3.0


def _node_moments(f, cells):
    vals = f[:, cells[:, 2], cells[:, 1], cells[:, 0]]
    rho = vals.sum(0)
    u = (_EF.T @ vals) / rho
    return rho, u.T


def refill(fpost, owner, owner_prev, particles, periodic=(False, False, False), rho0=1.0):
    """Refill of nodes uncovered this step (A12); returns a copy of fpost with
    the new nodes' post-collision populations replaced."""
    nz, ny, nx = owner.shape
    shape = (nx, ny, nz)
    solid, new = classify(owner, owner_prev)
    valid = (~solid) & (~new)
    out = fpost.copy()
    nzz, nyy, nxx = np.nonzero(new)
    for x, y, z in zip(nxx, nyy, nzz):
        P = particles[owner_prev[z, y, x]]
        u_new = rigid_velocity(P, np.array([x, y, z], dtype=np.float64))
        feq = lbm.equilibrium(np.array(rho0), u_new.reshape(3))
        for i in range(Q):
            nb, ok = _wrap(np.array([x, y, z]) + E[i], shape, periodic)
            if ok and valid[nb[2], nb[1], nb[0]]:
                out[i, z, y, x] = fpost[OPP[i], nb[2], nb[1], nb[0]] + 6.0 * W[i] * rho0 * (_EF[i] @ u_new)
            else:
                out[i, z, y, x] = feq[i]
    return out


def bounce_back_populations(fr, cell, d, q, u_w, solid, periodic=(False, False, False), bb_mode="ibb",
                            rho0=1.0):
    """The population G_{opp d}(x_f, t+1) that the wall returns on each link
    (x_f, d) (Sec. 2.3.2; readings A8, A9).

    fr: post-collision populations f+(t) after the refill, (19, nz, ny, nx);
    cell (n, 3) as (x, y, z), d (n,), q (n,): the links and their wall
    fractions; u_w (n, 3): the wall velocity at x_w; solid: node mask (nz, ny,
    nx) of the current flags.

    IBB (Eqs. eqneq1, eqneq2, neqd): G = f^eq_d(rho_f, u_d) + [f+_d(x_f) -
    f^eq_d(rho_f, u_f)] + 6 w_d rho0 (e_{opp d} . u_w), with rho_f, u_f the
    moments of f+(x_f), u_ff those of x_ff = x_f - e_d when it is a fluid node
    inside the domain (else u_f), and u_d from `departure_velocity`.
    Ladd: G = f+_d(x_f) + 6 w_d rho0 (e_{opp d} . u_w).
    """
    nz, ny, nx = solid.shape
    shape = (nx, ny, nz)
    j = OPP[d]
    e_j = _EF[j]
    wd = W[d]
    f_d = fr[d, cell[:, 2], cell[:, 1], cell[:, 0]]
    wall = 6.0 * wd * rho0 * (e_j * u_w).sum(1)
    if bb_mode == "ladd":
        return f_d + wall
    rho_f, u_f = _node_moments(fr, cell)
    ffc, ok = _wrap(cell - E[d], shape, periodic)
    okf = ok.copy()
    okf[ok] = ~solid[ffc[ok, 2], ffc[ok, 1], ffc[ok, 0]]
    u_ff = u_f.copy()
    if okf.any():
        _, u_ff[okf] = _node_moments(fr, ffc[okf])
    u_d = departure_velocity(q, u_f, u_ff, u_w)

    def feq_dir(rho, u, dd):
        eu = (_EF[dd] * u).sum(1)
        usq = (u * u).sum(1)
        return W[dd] * rho * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * usq)

    return feq_dir(rho_f, u_d, d) + (f_d - feq_dir(rho_f, u_f, d)) + wall


def coupled_lbm_step(fpost, owner, owner_prev, particles, tau, bb_mode="ibb",
                     periodic=(False, False, False), wall_velocity=None, rho0=1.0, force=None,
                     return_links=False, cover_uncover=False):
    """One LBM step with particles (A13): refill -> stream (domain walls,
    IBB/Ladd on particle links) -> collide -> momentum exchange.

    fpost: f+(t), (19, nz, ny, nx).  owner / owner_prev: node owners at the
    current and previous pose.  particles: list of dicts (centers, k, pos,
    quat, vel, omega).  Returns (f+(t+1) with NaN at solid nodes, F (np, 3),
    T (np, 3)) and, with return_links, a dict of per-link data.
    """
    nz, ny, nx = owner.shape
    shape = (nx, ny, nz)
    solid, new = classify(owner, owner_prev)
    fr = refill(fpost, owner, owner_prev, particles, periodic, rho0)
    fin = lbm.stream_pull(fr, periodic, wall_velocity, rho0)

    cell, d, p = find_links(owner, periodic)
    nl = len(d)
    q = np.empty(nl)
    for pi in np.unique(p):
        m = p == pi
        q[m] = wall_fraction(cell[m], d[m], particles[pi])
    if bb_mode == "ladd":
        q_w = np.full(nl, 0.5)
    else:
        q_w = q
    j = OPP[d]
    e_d = _EF[d]
    e_j = _EF[j]
    x_w = cell + q_w[:, None] * e_d
    u_w = np.zeros((nl, 3))
    X_p = np.zeros((nl, 3))
    for pi in np.unique(p):
        m = p == pi
        u_w[m] = rigid_velocity(particles[pi], x_w[m])
        X_p[m] = particles[pi]["pos"]
    f_d = fr[d, cell[:, 2], cell[:, 1], cell[:, 0]]
    G = bounce_back_populations(fr, cell, d, q, u_w, solid, periodic, bb_mode, rho0)
    # missing population j at x_f is replaced by G
    fin[j, cell[:, 2], cell[:, 1], cell[:, 0]] = G
    out = lbm.collide(fin, tau, force)
    out[:, solid] = np.nan

    dP = (e_d - u_w) * f_d[:, None] - (e_j - u_w) * G[:, None]
    dT = np.cross(x_w - X_p, dP)
    npart = len(particles)
    F = np.zeros((npart, 3))
    T = np.zeros((npart, 3))
    for pi in range(npart):
        m = p == pi
        F[pi] = dP[m].sum(0)
        T[pi] = dT[m].sum(0)
    if cover_uncover:
        # reading A11, optional: momentum of covered and uncovered nodes
        covered = (owner >= 0) & (owner_prev < 0)
        for sel, own, src, sign in ((covered, owner, fpost, 1.0), (new, owner_prev, fr, -1.0)):
            zz, yy, xx = np.nonzero(sel)
            if len(xx) == 0:
                continue
            J = (_EF.T @ src[:, zz, yy, xx]).T                      # (n, 3)
            pid = own[zz, yy, xx]
            xyz = np.stack([xx, yy, zz], axis=1).astype(np.float64)
            for pi in np.unique(pid):
                m = pid == pi
                arm = xyz[m] - np.asarray(particles[pi]["pos"], dtype=np.float64)
                F[pi] += sign * J[m].sum(0)
                T[pi] += sign * np.cross(arm, J[m]).sum(0)
    if return_links:
        links = {"cell": cell, "dir": d, "particle": p, "q": q, "G": G, "f_d": f_d, "u_w": u_w, "dP": dP}
        return out, F, T, links
    return out, F, T
