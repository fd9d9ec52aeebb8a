"""DEM contact between sphero-metaball particles for the oracle (test
infrastructure only), float64.

Sec. 2.3.1: each particle is taken as a shrunken ("zoomed") inner metaball
dilated by a sphere of radius R_s; the closest points follow from a stationary
point of f_0 + f_1 (Eq. CM_coreF; grad = 0, Eq. grad) found by Newton-Raphson,
a first-order Taylor step onto each core surface (Eq. cp), and the contact
point, normal and overlap of Eq. contactprop; walls use a Newton solve for the
core point whose gradient is along the wall normal (Eqs. metawallcp,
contactprop2); forces are linear spring-dashpot with a Coulomb-limited
tangential spring.

Readings:
  A16  the core is the iso-surface g = s f = 1 with s = ((r_e - R_s)/r_e)^2,
       r_e = sqrt(sum k): exact for coincident centres (core radius r_e - R_s),
       requires R_s < r_e.
  A17  Newton on grad(g_0 + g_1) = 0 (3x3 LU with partial pivoting, no line
       search; the stationary point of two spheres is a saddle).  Initial
       guess: for the pair of control points (a of particle 0, b of particle
       1) minimising |c_a - c_b| - sqrt(k_a) - sqrt(k_b) (world frame; ties to
       the lowest (a, b)), the midpoint of the two sphere surface points on
       the line c_a -> c_b.  Stop when |dx| <= 1e-10 R_b,max or after 50
       iterations.  Status: 0 ok, 1 not converged, 2 singular Hessian,
       3 inside a core (g_0 >= 1 or g_1 >= 1 at x_m), 4 out of range
       (g_0 or g_1 < c_tol = 1e-6).  |f_0| in the paper's constraint is read
       as f_0 (f > 0).
  A18  "Taylor" is first order: q_p = (1 - g_p(x_m)) / |grad g_p(x_m)|^2.
  A19  contact point x_cp = x_c0 - (R_s0 - delta/2) n with n = (x_c0 - x_c1)/|.|
       (pointing from particle 1 to particle 0): the paper's '+' sign would put
       x_cp outside the overlap with its own n.
  A20  forces: F_n = max(0, k_n delta + eta_n v_rel.n), v_rel = velocity of 1
       relative to 0 at x_cp; tangential spring xi += v_t dt (projected onto
       the current tangent plane), F_t = k_t xi + eta_t v_t on particle 0,
       Coulomb limit |F_t| <= mu_s F_n with xi reset to the limit; force on 0:
       F_n n + F_t, on 1 the opposite; torques (x_cp - X_p) x F_p.  The
       spring of a pair persists while the pair stays in contact.
  A21  walls: axis-aligned planes at -1/2 and N - 1/2 of every non-periodic
       axis, normal n_w pointing into the fluid; the core point x_cm solves
       grad g(x) = lam n_w, g(x) = 1 (4x4 Newton, guess: the control point
       minimising n_w.c_a - sqrt(s k_a), moved to its core sphere's extreme
       point); delta = R_s - n_w.(x_cm - p_w); n = n_w; x_cp = foot of x_cm
       on the plane + delta/2 n_w.
"""
import numpy as np

from .metaball import bounding_radius, quat_to_matrix, to_body

C_TOL = 1e-6
MAX_ITER = 50
OK, NOCONV, SINGULAR, INSIDE, OUT_OF_RANGE = 0, 1, 2, 3, 4


def core_scale(k, skin):
    re = np.sqrt(np.sum(k))
    return ((re - skin) / re) ** 2


def core_eval(P, x):
    """g = s f, grad g and Hessian of g at world point x (world frame)."""
    R = quat_to_matrix(P["quat"])
    s = core_scale(P["k"], P["skin"])
    xb = to_body(np.asarray(x, dtype=np.float64)[None], np.asarray(P["pos"], dtype=np.float64), R)[0]
    g = 0.0
    gb = np.zeros(3)
    Hb = np.zeros((3, 3))
    for c, k in zip(P["centers"], P["k"]):
        d = xb - c
        r2 = d @ d
        g += k / r2
        gb += -2.0 * k / (r2 * r2) * d
        Hb += 8.0 * k / r2 ** 3 * np.outer(d, d) - 2.0 * k / (r2 * r2) * np.eye(3)
    return s * g, s * (R @ gb), s * (R @ Hb @ R.T)


def world_centers(P):
    R = quat_to_matrix(P["quat"])
    return np.asarray(P["pos"], dtype=np.float64) + np.asarray(P["centers"]) @ R.T


def pair_guess(P0, P1):
    c0, c1 = world_centers(P0), world_centers(P1)
    r0, r1 = np.sqrt(P0["k"]), np.sqrt(P1["k"])
    best, arg = np.inf, (0, 0)
    for a in range(len(r0)):
        for b in range(len(r1)):
            gap = np.linalg.norm(c0[a] - c1[b]) - r0[a] - r1[b]
            if gap < best:
                best, arg = gap, (a, b)
    a, b = arg
    u = c1[b] - c0[a]
    D = np.linalg.norm(u)
    u = u / D if D > 0 else np.array([1.0, 0.0, 0.0])
    return 0.5 * ((c0[a] + r0[a] * u) + (c1[b] - r1[b] * u))


def lu_solve(A, b):
    """Gaussian elimination with partial pivoting; None if singular."""
    A = np.array(A, dtype=np.float64)
    b = np.array(b, dtype=np.float64)
    n = len(b)
    for i in range(n):
        p = i + int(np.argmax(np.abs(A[i:, i])))
        if A[p, i] == 0.0:
            return None
        if p != i:
            A[[i, p]] = A[[p, i]]
            b[[i, p]] = b[[p, i]]
        for r in range(i + 1, n):
            m = A[r, i] / A[i, i]
            A[r, i:] -= m * A[i, i:]
            b[r] -= m * b[i]
    x = np.zeros(n)
    for i in range(n - 1, -1, -1):
        x[i] = (b[i] - A[i, i + 1:] @ x[i + 1:]) / A[i, i]
    return x


def newton_pair(P0, P1, x0=None, tol_rel=1e-10, max_iter=MAX_ITER):
    """Closest points of two sphero-metaball particles (Eqs. CM_coreF, grad,
    cp, contactprop)."""
    Rb = max(bounding_radius(P0["centers"], P0["k"]), bounding_radius(P1["centers"], P1["k"]))
    x = pair_guess(P0, P1) if x0 is None else np.asarray(x0, dtype=np.float64)
    status, it = NOCONV, 0
    for it in range(1, max_iter + 1):
        _, g0, H0 = core_eval(P0, x)
        _, g1, H1 = core_eval(P1, x)
        dx = lu_solve(H0 + H1, g0 + g1)
        if dx is None or not np.all(np.isfinite(dx)):
            status = SINGULAR
            break
        x = x - dx
        if np.linalg.norm(dx) <= tol_rel * Rb:
            status = OK
            break
    G0, g0, _ = core_eval(P0, x)
    G1, g1, _ = core_eval(P1, x)
    if status == OK:
        if G0 >= 1.0 or G1 >= 1.0:
            status = INSIDE
        elif G0 < C_TOL or G1 < C_TOL:
            status = OUT_OF_RANGE
    xc0 = x + (1.0 - G0) / (g0 @ g0) * g0
    xc1 = x + (1.0 - G1) / (g1 @ g1) * g1
    d = xc0 - xc1
    dist = np.linalg.norm(d)
    n = d / dist if dist > 0 else np.zeros(3)
    delta = P0["skin"] + P1["skin"] - dist
    xcp = xc0 - (P0["skin"] - 0.5 * delta) * n
    return {"x_m": x, "iters": it, "status": status, "x_c0": xc0, "x_c1": xc1, "n": n, "delta": delta,
            "x_cp": xcp}


def wall_planes(shape, periodic):
    """(point on plane, inward normal, face index) of every wall face."""
    out = []
    for a in range(3):
        if periodic[a]:
            continue
        p = np.zeros(3)
        nrm = np.zeros(3)
        p[a], nrm[a] = -0.5, 1.0
        out.append((p.copy(), nrm.copy(), 2 * a))
        p[a], nrm[a] = shape[a] - 0.5, -1.0
        out.append((p.copy(), nrm.copy(), 2 * a + 1))
    return out


def newton_wall(P, p_w, n_w, tol_rel=1e-10, max_iter=MAX_ITER):
    """Core point of P extreme toward the wall and the contact geometry
    (Eqs. metawallcp, contactprop2)."""
    n_w = np.asarray(n_w, dtype=np.float64)
    s = core_scale(P["k"], P["skin"])
    cw = world_centers(P)
    rs = np.sqrt(s * P["k"])
    a = int(np.argmin(cw @ n_w - rs))
    x = cw[a] - rs[a] * n_w
    _, g, _ = core_eval(P, x)
    lam = np.linalg.norm(g)
    Rb = bounding_radius(P["centers"], P["k"])
    status, it = NOCONV, 0
    for it in range(1, max_iter + 1):
        G, g, H = core_eval(P, x)
        F = np.concatenate([g - lam * n_w, [G - 1.0]])
        J = np.zeros((4, 4))
        J[:3, :3] = H
        J[:3, 3] = -n_w
        J[3, :3] = g
        dz = lu_solve(J, F)
        if dz is None or not np.all(np.isfinite(dz)):
            status = SINGULAR
            break
        x = x - dz[:3]
        lam = lam - dz[3]
        if np.linalg.norm(dz[:3]) <= tol_rel * Rb:
            status = OK
            break
    dist = n_w @ (x - np.asarray(p_w, dtype=np.float64))
    delta = P["skin"] - dist
    foot = x - dist * n_w
    return {"x_cm": x, "iters": it, "status": status, "n": n_w.copy(), "delta": delta,
            "x_cp": foot + 0.5 * delta * n_w, "lam": lam}


def broad_phase(parts, margin=1.0):
    """Candidate pairs (i < j): |X_i - X_j| <= R_b,i + R_b,j + margin."""
    Rb = [bounding_radius(P["centers"], P["k"]) for P in parts]
    out = []
    for i in range(len(parts)):
        for j in range(i + 1, len(parts)):
            if np.linalg.norm(np.asarray(parts[i]["pos"]) - parts[j]["pos"]) <= Rb[i] + Rb[j] + margin:
                out.append((i, j))
    return out


def wall_candidates(parts, shape, periodic, margin=1.0):
    out = []
    for i, P in enumerate(parts):
        Rb = bounding_radius(P["centers"], P["k"])
        for p_w, n_w, face in wall_planes(shape, periodic):
            if n_w @ (np.asarray(P["pos"]) - p_w) <= Rb + margin:
                out.append((i, face))
    return out


def _point_velocity(P, x):
    return np.asarray(P["vel"], dtype=np.float64) + np.cross(P["omega"], np.asarray(x) - P["pos"])


def spring_dashpot(delta, n, x_cp, P0, P1, xi, params, dt):
    """Force on particle 0 (A20) and the updated tangential spring.  P1 may be
    None for a wall (at rest)."""
    kn, kt, eta_n, eta_t, mu = (params[k] for k in ("kn", "kt", "eta_n", "eta_t", "mu_s"))
    v0 = _point_velocity(P0, x_cp)
    v1 = np.zeros(3) if P1 is None else _point_velocity(P1, x_cp)
    vr = v1 - v0
    vn = vr @ n
    vt = vr - vn * n
    Fn = max(0.0, kn * delta + eta_n * vn)
    xi = np.asarray(xi, dtype=np.float64)
    xi = xi - (xi @ n) * n
    xi = xi + vt * dt
    Ft = kt * xi + eta_t * vt
    nt = np.linalg.norm(Ft)
    if nt > mu * Fn:
        if nt > 0:
            Ft = Ft * (mu * Fn / nt)
        xi = (Ft - eta_t * vt) / kt if kt > 0 else np.zeros(3)
    return Fn * n + Ft, xi


def contact_forces(parts, shape, periodic, params, history, dt, margin=1.0):
    """All contact forces of one DEM substep.

    history: dict keyed (i, j) (j = -1 - face for walls) -> xi of the previous
    substep (absent = new contact).  Returns F (np, 3), T (np, 3), the new
    history and the list of contacts (dicts)."""
    npart = len(parts)
    F = np.zeros((npart, 3))
    T = np.zeros((npart, 3))
    new_hist = {}
    contacts = []
    for i, j in broad_phase(parts, margin):
        c = newton_pair(parts[i], parts[j])
        c.update(i=i, j=j)
        contacts.append(c)
        if c["status"] != OK or c["delta"] <= 0:
            continue
        f, xi = spring_dashpot(c["delta"], c["n"], c["x_cp"], parts[i], parts[j],
                               history.get((i, j), np.zeros(3)), params, dt)
        new_hist[(i, j)] = xi
        F[i] += f
        F[j] -= f
        T[i] += np.cross(c["x_cp"] - parts[i]["pos"], f)
        T[j] -= np.cross(c["x_cp"] - parts[j]["pos"], f)
    planes = {face: (p, n) for p, n, face in wall_planes(shape, periodic)}
    for i, face in wall_candidates(parts, shape, periodic, margin):
        p_w, n_w = planes[face]
        c = newton_wall(parts[i], p_w, n_w)
        c.update(i=i, j=-1 - face)
        contacts.append(c)
        if c["status"] != OK or c["delta"] <= 0:
            continue
        f, xi = spring_dashpot(c["delta"], c["n"], c["x_cp"], parts[i], None,
                               history.get((i, -1 - face), np.zeros(3)), params, dt)
        new_hist[(i, -1 - face)] = xi
        F[i] += f
        T[i] += np.cross(c["x_cp"] - parts[i]["pos"], f)
    return F, T, new_hist, contacts
