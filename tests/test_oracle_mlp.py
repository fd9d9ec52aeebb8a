"""Pins of the oracle's learned-guess pieces (no GPU): backprop against central
finite differences, AdamW's first step against its closed form, training
reduces the loss, features are translation-invariant and match their
definitions on spheres, labels match the two-sphere closed form."""
import numpy as np

from oracle import contact, mlp


def _sphere(c, k, skin=0.5, quat=(1.0, 0.0, 0.0, 0.0)):
    return {"centers": np.zeros((1, 3)), "k": np.array([float(k)]), "pos": np.asarray(c, dtype=float),
            "quat": np.asarray(quat, dtype=float), "skin": skin, "vel": np.zeros(3), "omega": np.zeros(3)}


def _blob(seed, pos, n=4):
    rng = np.random.default_rng(seed)
    c = rng.uniform(-2, 2, (n, 3))
    q = rng.normal(size=4)
    return {"centers": c - c.mean(0), "k": rng.uniform(2, 5, n), "pos": np.asarray(pos, float),
            "quat": q / np.linalg.norm(q), "skin": 0.5, "vel": np.zeros(3), "omega": np.zeros(3)}


def test_backprop_matches_finite_differences():
    rng = np.random.default_rng(0)
    p = mlp.init_params(1)
    for k in p:
        if k.startswith("b"):
            p[k] = 0.1 * rng.normal(size=p[k].shape)
    X = rng.normal(size=(6, 64))
    T = rng.normal(size=(6, 4))
    Y, cache = mlp.forward(p, X)
    loss, dY = mlp.mse(Y, T)
    g = mlp.backward(p, cache, dY)
    h = 1e-6
    for key in ["W1", "b1", "W2", "b2", "W3", "b3"]:
        flat = p[key].reshape(-1)
        for idx in rng.choice(flat.size, min(12, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp, _ = mlp.mse(mlp.forward(p, X)[0], T)
            flat[idx] = old - h
            lm, _ = mlp.mse(mlp.forward(p, X)[0], T)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            an = g[key].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (key, idx, fd, an)


def test_adamw_first_step_closed_form():
    rng = np.random.default_rng(2)
    p = {"w": rng.normal(size=5)}
    g = {"w": rng.normal(size=5)}
    st = {}
    lr, eps, wd = 1e-2, 1e-8, 0.1
    q = mlp.adamw(p, g, st, lr=lr, eps=eps, wd=wd)
    # bias-corrected m = g, v = g^2 after one step
    expect = p["w"] - lr * (g["w"] / (np.abs(g["w"]) + eps) + wd * p["w"])
    assert np.allclose(q["w"], expect, rtol=0, atol=1e-14)
    assert st["t"] == 1


def test_training_reduces_loss_on_a_smooth_target():
    rng = np.random.default_rng(3)
    X = rng.normal(size=(256, 64))
    A = rng.normal(size=(64, 4)) / 8
    T = np.tanh(X @ A)
    p = mlp.init_params(4)
    st = {}
    l0 = mlp.mse(mlp.forward(p, X)[0], T)[0]
    for _ in range(60):
        Y, cache = mlp.forward(p, X)
        _, dY = mlp.mse(Y, T)
        p = mlp.adamw(p, mlp.backward(p, cache, dY), st, lr=3e-3)
    l1 = mlp.mse(mlp.forward(p, X)[0], T)[0]
    assert l1 < 0.2 * l0


def test_features_translation_invariant_and_defined():
    Pi, Pj = _blob(5, [10.0, 11.0, 12.0]), _blob(6, [14.5, 12.0, 11.0])
    f, xh = mlp.features(Pi, Pj)
    shift = np.array([3.25, -7.5, 100.0])
    g, xh2 = mlp.features(dict(Pi, pos=Pi["pos"] + shift), dict(Pj, pos=Pj["pos"] + shift))
    assert np.allclose(f, g, atol=1e-12) and np.allclose(xh2 - xh, shift)
    L = max(contact.bounding_radius(Pi["centers"], Pi["k"]), contact.bounding_radius(Pj["centers"], Pj["k"]))
    assert np.allclose(f[0:3], (Pj["pos"] - Pi["pos"]) / L)
    assert np.isclose(np.exp(f[14]), contact.core_eval(Pi, xh)[0])
    # nearest control points by brute force, in order
    cw = contact.world_centers(Pi)
    d = np.linalg.norm(cw - xh, axis=1)
    order = np.argsort(d, kind="stable")
    for r, b in enumerate(order[:4]):
        assert np.allclose(f[20 + 4 * r:23 + 4 * r], (cw[b] - xh) / L)
    assert np.all(f[20 + 16:20 + 20] == 0.0)  # only 4 balls: the fifth slot is empty


def test_two_sphere_guess_and_labels_closed_form():
    k0, k1, R = 9.0, 4.0, 0.5
    D = 5.2
    Pi, Pj = _sphere([0.0, 0.0, 0.0], k0, R), _sphere([D, 0.0, 0.0], k1, R)
    f, xh = mlp.features(Pi, Pj)
    # plain guess: midpoint of the two sphere surfaces on the centre line
    assert np.allclose(xh, [0.5 * (3.0 + D - 2.0), 0.0, 0.0])
    r = contact.newton_pair(Pi, Pj)
    lab = mlp.labels(Pi, Pj, r["x_m"], xh)
    L = 3.0  # bounding radius of the larger sphere: |c| + sqrt(k) = 3
    assert np.allclose(lab[:3], (r["x_m"] - xh) / L)
    a0, a1 = contact.core_scale([k0], R) * k0, contact.core_scale([k1], R) * k1
    r0 = np.linalg.norm(r["x_m"])
    r1 = D - r0
    w0, w1 = a0 / r0 ** 2, a1 / r1 ** 2
    near, far = (r0, r1) if r0 <= r1 else (r1, r0)
    wn = w0 if r0 <= r1 else w1
    expect = near if wn >= 0.99 * (w0 + w1) else far
    assert np.isclose(lab[3], np.log(expect / L))


def test_anchor_hand_computed():
    """Two unit balls at x = -1, +1 (body frame) and a ball of k = 4 six units
    away: the sphere of i reaching closest to X_j is the one facing it, the
    surface points are 2 and 4 along the axis, so x_a is 3 along it, whatever
    the rotation that brings the facing ball round."""
    bi = {"centers": np.array([[-1.0, 0, 0], [1.0, 0, 0]]), "k": np.array([1.0, 1.0]), "skin": 0.25,
          "vel": np.zeros(3), "omega": np.zeros(3), "pos": np.zeros(3)}
    s2 = np.sqrt(0.5)
    for quat, pj, expect in (((1.0, 0, 0, 0), (6.0, 0, 0), (3.0, 0, 0)),
                             ((0.0, 0, 0, 1.0), (6.0, 0, 0), (3.0, 0, 0)),      # 180 deg about z
                             ((s2, 0, 0, s2), (0, 6.0, 0), (0, 3.0, 0)),        # 90 deg about z
                             ((s2, 0, 0, -s2), (0, -6.0, 0), (0, -3.0, 0))):    # -90 deg about z
        Pi = dict(bi, quat=np.array(quat))
        Pj = _sphere(pj, 4.0)
        assert np.allclose(mlp.anchor(Pi, Pj), expect, atol=1e-12), (quat, pj)
        # for single-ball pairs the anchor is the plain guess
    Pa, Pb = _sphere([0.5, -1, 2], 3.0), _sphere([4, 1, 2.5], 5.0)
    assert np.allclose(mlp.anchor(Pa, Pb), contact.pair_guess(Pa, Pb), atol=1e-12)
