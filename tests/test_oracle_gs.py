"""Pins of the Gradient Search oracle (Sec. 2.2, Algorithm 2, Eq. GSloss)
against what the definition and the mathematics fix: values and continuity
of the piecewise loss, the chain-rule gradient against finite differences of
the loss, symmetry and sign of the gradient for a single ball on a sphere,
descent lowering the loss towards a generator, and the anomaly detection."""
import numpy as np
import pytest

from oracle import gs
from paper_2209_10411_gb300 import scenes


def test_loss_pieces_values_and_continuity():
    # hand values: f = 0.5 -> 0.25 + 2 - 1; f = 1.5 -> 0.5; f = 3 -> 4; f = 1 -> 0
    assert gs.loss_terms(np.array([0.5]))[0] == pytest.approx(1.25, abs=1e-15)
    assert gs.loss_terms(np.array([1.5]))[0] == pytest.approx(0.5, abs=1e-15)
    assert gs.loss_terms(np.array([3.0]))[0] == pytest.approx(4.0, abs=1e-15)
    assert gs.loss_terms(np.array([1.0]))[0] == 0.0
    # the pieces meet at f = 1 and f = 2
    for f0 in (1.0, 2.0):
        lo, hi = gs.loss_terms(np.array([f0 - 1e-9, f0 + 1e-9]))
        assert abs(lo - hi) < 1e-8
    # the first branch owns f = 2 and the second f = 1 (reading G1)
    assert gs.dloss_df(np.array([2.0]))[0] == 2.0 and gs.dloss_df(np.array([1.0]))[0] == 1.0


@pytest.mark.parametrize("f", [0.3, 0.9, 1.2, 1.8, 2.5, 7.0])
def test_dloss_df_matches_finite_differences(f):
    h = 1e-6
    fd = (gs.loss_terms(np.array([f + h]))[0] - gs.loss_terms(np.array([f - h]))[0]) / (2 * h)
    assert gs.dloss_df(np.array([f]))[0] == pytest.approx(fd, rel=1e-6, abs=1e-8)


def _random_problem(seed, m=40, n=4):
    rng = np.random.default_rng(seed)
    H = scenes.ellipsoid_hull(rng, m, (6.0, 4.0, 3.0)).astype(np.float64)
    c, k = scenes.gs_start_model(rng, n, (6.0, 4.0, 3.0))
    return H, c.astype(np.float64), k.astype(np.float64) * rng.uniform(0.5, 2.0, n)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_gradient_matches_finite_differences(seed):
    H, c, k = _random_problem(seed)
    f = gs.field(H, c, k)
    # keep away from the kinks at f = 1 and f = 2, where finite differences do not apply
    keep = (np.abs(f - 1.0) > 0.05) & (np.abs(f - 2.0) > 0.05)
    H = H[keep]
    gc, gk = gs.gradient(H, c, k)
    h = 1e-6
    for j in range(len(k)):
        kp, km = k.copy(), k.copy()
        kp[j] += h
        km[j] -= h
        fd = (gs.loss(H, c, kp) - gs.loss(H, c, km)) / (2 * h)
        assert gk[j] == pytest.approx(fd, rel=1e-5, abs=1e-7)
        for a in range(3):
            cp, cm = c.copy(), c.copy()
            cp[j, a] += h
            cm[j, a] -= h
            fd = (gs.loss(H, cp, k) - gs.loss(H, cm, k)) / (2 * h)
            assert gc[j, a] == pytest.approx(fd, rel=1e-5, abs=1e-7)


def test_single_ball_on_a_sphere():
    """One ball at the centre of a symmetric point set on a sphere of radius
    R: f = k / R^2 everywhere, so the loss vanishes exactly at k = R^2, the
    centre gradient vanishes by symmetry for any k, and the k gradient pushes
    k towards R^2 from either side."""
    R = 3.0
    t = (1.0 + 5 ** 0.5) / 2.0
    ico = np.array([[0, 1, t], [0, -1, t], [0, 1, -t], [0, -1, -t], [1, t, 0], [-1, t, 0], [1, -t, 0], [-1, -t, 0],
                    [t, 0, 1], [-t, 0, 1], [t, 0, -1], [-t, 0, -1]], dtype=np.float64)
    H = R * ico / np.linalg.norm(ico, axis=1, keepdims=True)
    c = np.zeros((1, 3))
    assert gs.loss(H, c, np.array([R * R])) == pytest.approx(0.0, abs=1e-12)
    for k in (0.5 * R * R, 0.99 * R * R, 1.01 * R * R, 2.5 * R * R):
        gc, gk = gs.gradient(H, c, np.array([k]))
        assert np.abs(gc).max() < 1e-12
        assert np.sign(gk[0]) == np.sign(k - R * R)
        assert gs.loss(H, c, np.array([k])) > 0.0


def _generator_hull(rng, m):
    """Points of the f = 1 surface of a two-ball generator, by bisection along
    random rays from the origin (inside: f > 1 near the balls)."""
    c = np.array([[-1.5, 0.0, 0.0], [1.5, 0.3, 0.0]])
    k = np.array([6.0, 4.0])
    u = rng.normal(size=(m, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    pts = []
    for d in u:
        lo, hi = 0.0, 20.0
        for _ in range(80):
            mid = 0.5 * (lo + hi)
            if gs.field(mid * d[None, :], c, k)[0] >= 1.0:
                lo = mid
            else:
                hi = mid
        pts.append(lo * d)
    return np.array(pts), c, k


def test_descent_lowers_loss_towards_the_generator():
    rng = np.random.default_rng(7)
    H, cg, kg = _generator_hull(rng, 200)
    assert np.allclose(gs.field(H, cg, kg), 1.0, atol=1e-10)
    c0 = cg + rng.normal(scale=0.3, size=cg.shape)
    k0 = kg * 1.3
    l0 = gs.loss(H, c0, k0)
    c, k = gs.descend(H, c0, k0, 1000, 2e-4)
    # the generator is recovered: centres within 0.02 lu (from 0.5), k within 1 %
    assert gs.loss(H, c, k) < 0.01 * l0
    assert np.abs(c - cg).max() < 0.02
    assert np.abs(k / kg - 1.0).max() < 0.01


def test_anomaly_detection():
    rng = np.random.default_rng(3)
    H = scenes.ellipsoid_hull(rng, 300, (5.0, 4.0, 3.0))
    P = scenes.hull_planes(H)
    inside = np.array([[0.0, 0.0, 0.0], [1.0, -1.0, 0.5]])
    outside = np.array([[6.0, 0.0, 0.0], [0.0, 0.0, -3.5]])
    c = np.concatenate([inside, outside, [[0.5, 0.5, 0.5]]])
    k = np.array([1.0, 2.0, 1.0, 1.0, -0.5])
    k2, active = gs.anomaly(c, k, P)
    assert list(active) == [True, True, False, False, False]
    assert list(k2) == [1.0, 2.0, 0.0, 0.0, 0.0]
    # the centre of the hull is inside it
    assert not gs.outside_hull_f32(np.zeros((1, 3)), P)[0]


def test_gs_fit_keeps_cleared_points_out():
    rng = np.random.default_rng(5)
    H = scenes.ellipsoid_hull(rng, 120, (5.0, 4.0, 3.0)).astype(np.float64)
    P = scenes.hull_planes(H)
    c0, k0 = scenes.gs_start_model(rng, 6, (5.0, 4.0, 3.0))
    c0 = c0.astype(np.float64)
    c0[0] = (7.0, 0.0, 0.0)  # outside the hull from the start
    k0 = k0.astype(np.float64)
    c, k, active, l1, l2 = gs.gs_fit(H, c0, k0, 20, 1e-4, P)
    assert not active[0] and k[0] == 0.0
    assert np.array_equal(c[0], gs.descend(H, c0, k0, 20, 1e-4)[0][0])
    assert l2 <= l1 * 1.5
