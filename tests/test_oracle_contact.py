"""Pins of the oracle's contact model (no GPU): closed forms for two spheres
and a sphere at a wall, Newton's stationary point and closest points against
brute-force dense sampling on tiny metaball sets, and the spring-dashpot law
against the closed-form restitution and the Coulomb limit; the broad phase
at its threshold and against densely sampled solids."""
import numpy as np
import pytest

from oracle import contact, dem

RNG = np.random.default_rng(31)


def _sphere(c, k, skin, vel=(0, 0, 0), omega=(0, 0, 0), mass=10.0):
    return {"centers": np.zeros((1, 3)), "k": np.array([float(k)]), "pos": np.asarray(c, dtype=float),
            "quat": np.array([1.0, 0, 0, 0]), "skin": float(skin), "vel": np.asarray(vel, dtype=float),
            "omega": np.asarray(omega, dtype=float), "mass": mass, "volume": 0.0,
            "inertia": np.eye(3) * 0.4 * mass * k}


@pytest.mark.parametrize("k0,k1,R0,R1,D", [(9.0, 4.0, 0.5, 0.5, 5.3), (16.0, 9.0, 1.0, 0.4, 6.5),
                                          (4.0, 4.0, 0.3, 0.3, 3.5)])
def test_two_spheres_closed_form(k0, k1, R0, R1, D):
    u = RNG.normal(size=3)
    u /= np.linalg.norm(u)
    c0 = np.array([10.0, 11.0, 12.0])
    P0, P1 = _sphere(c0, k0, R0), _sphere(c0 + D * u, k1, R1)
    r = contact.newton_pair(P0, P1)
    a0 = contact.core_scale([k0], R0) * k0
    a1 = contact.core_scale([k1], R1) * k1
    r0 = D * a0 ** (1 / 3) / (a0 ** (1 / 3) + a1 ** (1 / 3))
    r1 = D - r0
    assert r["status"] == contact.OK
    assert np.allclose(r["x_m"], c0 + r0 * u, atol=1e-12 * D)
    # first-order projection onto each core sphere (the method's closed form)
    rho0 = r0 * (3 * a0 - r0 * r0) / (2 * a0)
    rho1 = r1 * (3 * a1 - r1 * r1) / (2 * a1)
    assert np.allclose(r["x_c0"], c0 + rho0 * u, atol=1e-12 * D)
    assert np.allclose(r["x_c1"], c0 + (D - rho1) * u, atol=1e-12 * D)
    gap = D - rho0 - rho1
    assert abs(r["delta"] - (R0 + R1 - abs(gap))) < 1e-12
    assert np.allclose(r["n"], -np.sign(gap) * u, atol=1e-12)
    # contact point in the middle of the skin overlap
    assert np.allclose(r["x_cp"], r["x_c0"] - (R0 - 0.5 * r["delta"]) * r["n"], atol=1e-13)


def test_single_ball_core_radius():
    # A16: the core of one ball is the sphere of radius sqrt(k) - R_s
    P = _sphere([0, 0, 0], 25.0, 1.5)
    g, _, _ = contact.core_eval(P, np.array([3.5, 0.0, 0.0]))
    assert abs(g - 1.0) < 1e-14


def test_equal_skins_contact_point_is_midpoint():
    P0, P1 = _sphere([0, 0, 0], 9.0, 0.6), _sphere([5.2, 0.3, -0.1], 16.0, 0.6)
    r = contact.newton_pair(P0, P1)
    assert np.allclose(r["x_cp"], 0.5 * (r["x_c0"] + r["x_c1"]), atol=1e-13)


def test_overlapping_cores_are_flagged():
    P0, P1 = _sphere([0, 0, 0], 9.0, 0.5), _sphere([2.0, 0, 0], 9.0, 0.5)
    r = contact.newton_pair(P0, P1)
    assert r["status"] in (contact.INSIDE, contact.SINGULAR, contact.NOCONV)


@pytest.mark.parametrize("axis,side", [(0, 0), (1, 1), (2, 0), (2, 1)])
def test_sphere_at_wall_closed_form(axis, side):
    shape = (40, 30, 50)
    planes = {face: (p, n) for p, n, face in contact.wall_planes(shape, (False, False, False))}
    p_w, n_w = planes[2 * axis + side]
    k, Rs = 16.0, 1.0
    c = np.array([20.0, 15.0, 25.0])
    c[axis] = p_w[axis] + n_w[axis] * 3.6  # core radius 3, skin 1: overlap 0.4
    r = contact.newton_wall(_sphere(c, k, Rs), p_w, n_w)
    assert r["status"] == contact.OK
    assert np.allclose(r["x_cm"], c - 3.0 * n_w, atol=1e-12)
    assert abs(r["delta"] - 0.4) < 1e-12
    foot = r["x_cm"] - 0.6 * n_w
    assert np.allclose(r["x_cp"], foot + 0.2 * n_w, atol=1e-12)


def _tiny(n, center, seed, spread=1.2):
    rng = np.random.default_rng(seed)
    c = rng.uniform(-spread, spread, (n, 3))
    c -= c.mean(0)
    k = rng.uniform(2.0, 4.0, n)
    q = rng.normal(size=4)
    return {"centers": c, "k": k, "pos": np.asarray(center, dtype=float), "quat": q / np.linalg.norm(q),
            "skin": 0.5, "vel": np.zeros(3), "omega": np.zeros(3)}


def _fib_dirs(m):
    i = np.arange(m) + 0.5
    phi = np.arccos(1 - 2 * i / m)
    th = np.pi * (1 + 5 ** 0.5) * i
    return np.stack([np.cos(th) * np.sin(phi), np.sin(th) * np.sin(phi), np.cos(phi)], 1)


def _core_surface(P, dirs):
    # radial bisection of g(X + r u) = 1 (tiny sets here are star-shaped about X)
    lo = np.zeros(len(dirs))
    hi = np.full(len(dirs), 12.0)
    for _ in range(50):
        mid = 0.5 * (lo + hi)
        g = np.array([contact.core_eval(P, P["pos"] + m * d)[0] for m, d in zip(mid, dirs)])
        inside = g >= 1.0
        lo = np.where(inside, mid, lo)
        hi = np.where(inside, hi, mid)
    return P["pos"] + (0.5 * (lo + hi))[:, None] * dirs


def test_newton_matches_dense_sampling_on_tiny_sets():
    P0 = _tiny(2, [10.0, 10.0, 10.0], 1)
    P1 = _tiny(3, [10.0, 10.0, 10.0], 2)
    # place P1 so that the cores are close: scan along x for a small gap
    for dxp in np.linspace(3.0, 9.0, 121):
        P1["pos"] = np.array([10.0 + dxp, 10.3, 9.8])
        r = contact.newton_pair(P0, P1)
        if r["status"] == contact.OK and 0.05 < np.linalg.norm(r["x_c1"] - r["x_c0"]) < 0.3:
            break
    assert r["status"] == contact.OK
    xm = r["x_m"]
    # (1) x_m is the zero of grad(g0 + g1): a dense grid around it has its
    # smallest |grad| at the centre cell
    h = 1e-3
    grid = np.stack(np.meshgrid(*[np.arange(-10, 11) * h] * 3, indexing="ij"), -1).reshape(-1, 3)
    gn = np.array([np.linalg.norm(contact.core_eval(P0, xm + d)[1] + contact.core_eval(P1, xm + d)[1])
                   for d in grid])
    assert np.linalg.norm(grid[np.argmin(gn)]) <= 1.5 * h
    # (2) the first-order closest points approach the true closest points of the
    # two core surfaces (dense sampling near x_m) within O(gap^2 / r)
    dirs = _fib_dirs(60000)
    u0 = (xm - P0["pos"]) / np.linalg.norm(xm - P0["pos"])
    u1 = (xm - P1["pos"]) / np.linalg.norm(xm - P1["pos"])
    S0 = _core_surface(P0, dirs[dirs @ u0 > 0.9])
    S1 = _core_surface(P1, dirs[dirs @ u1 > 0.9])
    d2 = ((S0[:, None, :] - S1[None, :, :]) ** 2).sum(-1)
    a, b = np.unravel_index(np.argmin(d2), d2.shape)
    gap = np.sqrt(d2[a, b])
    spacing = np.sqrt(4 * np.pi / 60000) * 4.0
    assert abs(np.linalg.norm(r["x_c1"] - r["x_c0"]) - gap) < 0.1 * gap + spacing
    assert np.linalg.norm(r["x_c0"] - S0[a]) < 0.5 * gap + 2 * spacing
    assert np.linalg.norm(r["x_c1"] - S1[b]) < 0.5 * gap + 2 * spacing


def test_wall_bounce_restitution_closed_form():
    # A sphere on a wall has an overlap exactly linear in its position (the wall
    # solve lands on the core's true extreme point), so the spring-dashpot law
    # must reproduce the clamped linear oscillator: the contact ends when
    # k delta + eta delta' = 0, at w_d t* = pi - atan(2 z sqrt(1-z^2)/(1-2z^2)),
    # with restitution e^(-z w t*) |cos(w_d t*) - (z w / w_d) sin(w_d t*)|.
    e = 0.8
    m = 10.0
    kn = 1.0
    ln = np.log(e)
    eta = -2.0 * ln * np.sqrt(m * kn) / np.sqrt(np.pi ** 2 + ln ** 2)
    params = {"kn": kn, "kt": 0.0, "eta_n": eta, "eta_t": 0.0, "mu_s": 0.4}
    v0 = 0.02
    # core radius 1.5, skin 0.5: touching when the centre is at z = -0.5 + 2.0
    P = _sphere([20.0, 20.0, 1.55], 4.0, 0.5, vel=(0, 0, -v0), mass=m)
    dt = 0.01
    hist = {}
    touched = False
    for _ in range(20000):
        F, T, hist, cs = contact.contact_forces([P], (40, 40, 40), (True, True, False), params, hist, dt)
        touched = touched or bool(hist)
        P = dem.integrate(P, F[0], T[0], (0, 0, 0), dt=dt)
        if touched and not hist:
            break
    z = -ln / np.sqrt(np.pi ** 2 + ln ** 2)
    w = np.sqrt(kn / m)
    wd = w * np.sqrt(1 - z * z)
    ts = (np.pi - np.arctan(2 * z * np.sqrt(1 - z * z) / (1 - 2 * z * z))) / wd
    e_clamped = np.exp(-z * w * ts) * abs(np.cos(wd * ts) - z * w / wd * np.sin(wd * ts))
    assert touched and P["vel"][2] > 0
    assert abs(P["vel"][2] / v0 - e_clamped) < 2e-3, (P["vel"][2] / v0, e_clamped)


def test_undamped_pair_collision_conserves_energy():
    params = {"kn": 1.0, "kt": 0.0, "eta_n": 0.0, "eta_t": 0.0, "mu_s": 0.4}
    v0 = 0.02
    P0 = _sphere([10.0, 10.0, 10.0], 4.0, 0.5, vel=(v0, 0, 0))
    P1 = _sphere([14.2, 10.0, 10.0], 4.0, 0.5, vel=(-v0, 0, 0))
    hist = {}
    touched = False
    for _ in range(20000):
        F, T, hist, cs = contact.contact_forces([P0, P1], (40, 40, 40), (True, True, True), params, hist, 0.01)
        touched = touched or bool(hist)
        P0 = dem.integrate(P0, F[0], T[0], (0, 0, 0), dt=0.01)
        P1 = dem.integrate(P1, F[1], T[1], (0, 0, 0), dt=0.01)
        if touched and not hist:
            break
    assert touched
    assert abs((P1["vel"][0] - P0["vel"][0]) / (2 * v0) - 1.0) < 2e-3
    assert abs(P0["vel"][0] + P1["vel"][0]) < 1e-15  # momentum


def test_coulomb_limit_sliding_on_a_wall():
    params = {"kn": 1.0, "kt": 0.5, "eta_n": 0.0, "eta_t": 0.0, "mu_s": 0.3}
    P = _sphere([20.0, 20.0, -0.5 + 3.0 + 0.8], 16.0, 1.0, vel=(0.05, 0, 0))  # overlap 0.2
    hist = {}
    for _ in range(50):
        F, T, hist, cs = contact.contact_forces([P], (40, 40, 40), (True, True, False), params, hist, 1.0)
    Fn = F[0][2]
    Ft = np.linalg.norm(F[0][:2])
    assert abs(Fn - 0.2) < 1e-12
    assert abs(Ft - 0.3 * Fn) < 1e-12
    assert F[0][0] < 0  # friction opposes the sliding of the particle


def test_broad_phase_threshold_and_completeness():
    """Candidates are the pairs with |X_i - X_j| <= R_b,i + R_b,j + margin
    (two single balls just inside and just outside the threshold), and no pair
    whose solids (f >= 1, sampled densely) come within the margin is missed."""
    from oracle import metaball
    a = _sphere([5.0, 5.0, 5.0], 4.0, 0.5)
    b = _sphere([5.0 + 6.0 - 1e-9, 5.0, 5.0], 9.0, 0.5)
    assert contact.broad_phase([a, b], margin=1.0) == [(0, 1)]
    b["pos"] = np.array([5.0 + 6.0 + 1e-9, 5.0, 5.0])
    assert contact.broad_phase([a, b], margin=1.0) == []

    rng = np.random.default_rng(5)
    parts = [_tiny(int(rng.integers(1, 4)), rng.uniform(4.0, 16.0, 3), 100 + s) for s in range(8)]
    cand = set(contact.broad_phase(parts, margin=1.0))
    solids = []
    for P in parts:
        Rb = metaball.bounding_radius(P["centers"], P["k"])
        ax = np.arange(-Rb, Rb + 1e-9, 0.2)
        g = np.stack(np.meshgrid(ax, ax, ax, indexing="ij"), -1).reshape(-1, 3) + P["pos"]
        R = metaball.quat_to_matrix(P["quat"])
        f = metaball.field(metaball.to_body(g, P["pos"], R), P["centers"], P["k"])
        solids.append(g[f >= 1.0])
    close = 0
    for i in range(len(parts)):
        for j in range(i + 1, len(parts)):
            d2 = ((solids[i][::7, None, :] - solids[j][None, ::7, :]) ** 2).sum(-1).min()
            if np.sqrt(d2) <= 1.0:
                close += 1
                assert (i, j) in cand, (i, j)
    assert close >= 1 and len(cand) > close   # the bounding spheres are conservative


def test_wall_candidates_threshold():
    """A particle is a wall candidate when its centre is within R_b + margin
    of the halfway wall plane (x = -0.5 or x = n - 0.5); periodic axes have
    no walls."""
    shape = (20, 20, 20)
    for x, expect in ((-0.5 + 4.0 - 1e-9, True), (-0.5 + 4.0 + 1e-9, False),
                      (19.5 - 4.0 + 1e-9, True), (19.5 - 4.0 - 1e-9, False)):
        P = _sphere([x, 10.0, 10.0], 9.0, 0.5)          # R_b = 3, margin 1
        faces = [f for _, f in contact.wall_candidates([P], shape, (False, True, True), margin=1.0)]
        assert (faces != []) == expect, (x, faces)
        if expect:
            assert faces == [0 if x < 10 else 1]
    P = _sphere([1.0, 1.0, 1.0], 9.0, 0.5)
    assert contact.wall_candidates([P], shape, (True, True, True), margin=1.0) == []
    assert sorted(f for _, f in contact.wall_candidates([P], shape, (False, False, False), margin=1.0)) == [0, 2, 4]
