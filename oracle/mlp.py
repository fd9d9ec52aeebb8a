"""Learned Newton guess for contact detection: features, MLP, loss, AdamW
(oracle side, test infrastructure only; float64).

Not in the paper: the Newton-Raphson closest-point solve of Sec. 2.3.1 still
decides every point, and a small network proposes its starting point and the
set of control points that matter near the solution.

Features of a candidate pair (i, j), 64 numbers, lengths scaled by
L = max(R_b,i, R_b,j) and positions taken relative to O = (X_i + X_j)/2:
  0:3    (X_j - X_i) / L
  3:7    q_i, sign chosen so that w >= 0
  7:11   q_j, likewise
  11:14  (x_a - O) / L, x_a the anchor (below)
  14:16  log g_i(x_a), log g_j(x_a) (core fields)
  16:40  particle i: log(n)/5, log(sum k / L^2), R_b / L, R_s / L, then for
         the 5 control points nearest to x_a (by distance, ties to the lower
         index; zeros when fewer): (c - x_a)/L (world frame) and log(s k / L^2)
  40:64  particle j, likewise
Anchor x_a: the control-point sphere (radius sqrt k) of i that reaches
closest to the origin X_j of j, the one of j closest to X_i, and the midpoint
of their surface points on the line joining their centres.  It costs
O(n_i + n_j), against O(n_i n_j) for the plain guess of contact.py (the
closest pair of spheres); for single-ball particles the two coincide.
Outputs (4): (x_m - x_a)/L and log(r_act / L).  Labels: x_m the converged
plain Newton point; r_act the smallest radius around x_m whose control points
carry 99 % of g_i(x_m) + g_j(x_m).

Network: 64 -> 256 -> 256 -> 4, ReLU after the two hidden layers, weights
W1 (64x256), W2 (256x256), W3 (256x4) and biases; loss: mean over the batch
of the squared error summed over the 4 outputs.
"""
import numpy as np

from .contact import core_scale, world_centers
from .metaball import bounding_radius, field, quat_to_matrix, to_body

SIZES = (64, 256, 256, 4)
NEAREST = 5


def init_params(seed=0):
    """He-uniform weights, zero biases (a fixed, seeded initialisation)."""
    rng = np.random.default_rng(seed)
    p = {}
    for l, (a, b) in enumerate(zip(SIZES[:-1], SIZES[1:]), start=1):
        lim = np.sqrt(6.0 / a)
        p["W%d" % l] = rng.uniform(-lim, lim, (a, b))
        p["b%d" % l] = np.zeros(b)
    return p


def forward(p, X):
    """Y = relu(relu(X W1 + b1) W2 + b2) W3 + b3, with the cache for backprop."""
    Z1 = X @ p["W1"] + p["b1"]
    H1 = np.maximum(Z1, 0.0)
    Z2 = H1 @ p["W2"] + p["b2"]
    H2 = np.maximum(Z2, 0.0)
    Y = H2 @ p["W3"] + p["b3"]
    return Y, {"X": X, "Z1": Z1, "H1": H1, "Z2": Z2, "H2": H2}


def mse(Y, T):
    """Loss = mean over rows of sum over outputs of (Y - T)^2, and dLoss/dY."""
    n = Y.shape[0]
    d = Y - T
    return float((d * d).sum() / n), 2.0 * d / n


def backward(p, cache, dY):
    """Gradients of the loss with respect to every parameter (chain rule)."""
    g = {}
    g["W3"] = cache["H2"].T @ dY
    g["b3"] = dY.sum(0)
    dZ2 = (dY @ p["W3"].T) * (cache["Z2"] > 0)
    g["W2"] = cache["H1"].T @ dZ2
    g["b2"] = dZ2.sum(0)
    dZ1 = (dZ2 @ p["W2"].T) * (cache["Z1"] > 0)
    g["W1"] = cache["X"].T @ dZ1
    g["b1"] = dZ1.sum(0)
    return g


def adamw(p, g, state, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, wd=1e-4):
    """One AdamW step (decoupled weight decay, Loshchilov & Hutter): returns
    new parameters; `state` holds m, v and the step count t."""
    t = state.get("t", 0) + 1
    out = {}
    for k in p:
        m = beta1 * state.get("m" + k, 0.0) + (1 - beta1) * g[k]
        v = beta2 * state.get("v" + k, 0.0) + (1 - beta2) * g[k] * g[k]
        mh = m / (1 - beta1 ** t)
        vh = v / (1 - beta2 ** t)
        out[k] = p[k] - lr * (mh / (np.sqrt(vh) + eps) + wd * p[k])
        state["m" + k], state["v" + k] = m, v
    state["t"] = t
    return out


def _core_world(P, x):
    R = quat_to_matrix(P["quat"])
    xb = to_body(np.asarray(x, dtype=np.float64)[None], np.asarray(P["pos"], dtype=np.float64), R)[0]
    return core_scale(P["k"], P["skin"]) * field(xb[None], P["centers"], P["k"])[0]


def _reaching_ball(P, target):
    """Index of the sphere (centre c, radius sqrt k) of P whose surface comes
    closest to the point `target`: argmin |c - target| - sqrt k, ties to the
    lower index."""
    cw = world_centers(P)
    gap = np.sqrt(((cw - target) ** 2).sum(1)) - np.sqrt(np.asarray(P["k"], float))
    return int(np.argmin(gap)), cw


def anchor(Pi, Pj):
    """The anchor x_a of the pair (i, j) (module docstring)."""
    a, ci = _reaching_ball(Pi, np.asarray(Pj["pos"], float))
    b, cj = _reaching_ball(Pj, np.asarray(Pi["pos"], float))
    ra, rb = np.sqrt(float(Pi["k"][a])), np.sqrt(float(Pj["k"][b]))
    u = cj[b] - ci[a]
    D = np.linalg.norm(u)
    u = u / D if D > 0 else np.array([1.0, 0.0, 0.0])
    return 0.5 * ((ci[a] + ra * u) + (cj[b] - rb * u))


def features(Pi, Pj):
    """The 64 features of the pair (i, j) and the anchor x_a."""
    L = max(bounding_radius(Pi["centers"], Pi["k"]), bounding_radius(Pj["centers"], Pj["k"]))
    Xi, Xj = np.asarray(Pi["pos"], float), np.asarray(Pj["pos"], float)
    O = 0.5 * (Xi + Xj)
    xh = anchor(Pi, Pj)
    f = np.zeros(64)
    f[0:3] = (Xj - Xi) / L
    for off, P in ((3, Pi), (7, Pj)):
        q = np.asarray(P["quat"], float) / np.linalg.norm(P["quat"])
        f[off:off + 4] = q if q[0] >= 0 else -q
    f[11:14] = (xh - O) / L
    f[14] = np.log(_core_world(Pi, xh))
    f[15] = np.log(_core_world(Pj, xh))
    for off, P in ((16, Pi), (40, Pj)):
        k = np.asarray(P["k"], float)
        s = core_scale(k, P["skin"])
        f[off] = np.log(len(k)) / 5.0
        f[off + 1] = np.log(k.sum() / (L * L))
        f[off + 2] = bounding_radius(P["centers"], k) / L
        f[off + 3] = P["skin"] / L
        cw = world_centers(P)
        d = np.sqrt(((cw - xh) ** 2).sum(1))
        order = np.lexsort((np.arange(len(d)), d))[:NEAREST]
        for r, b in enumerate(order):
            f[off + 4 + 4 * r: off + 7 + 4 * r] = (cw[b] - xh) / L
            f[off + 7 + 4 * r] = np.log(s * k[b] / (L * L))
    return f, xh


def labels(Pi, Pj, xm, xh, frac=0.99):
    """Targets (x_m - x_a)/L and log(r_act/L) for a converged x_m (xh = x_a)."""
    L = max(bounding_radius(Pi["centers"], Pi["k"]), bounding_radius(Pj["centers"], Pj["k"]))
    d, w = [], []
    for P in (Pi, Pj):
        cw = world_centers(P)
        s = core_scale(P["k"], P["skin"])
        r = np.sqrt(((cw - xm) ** 2).sum(1))
        d.append(r)
        w.append(s * np.asarray(P["k"]) / (r * r))
    d, w = np.concatenate(d), np.concatenate(w)
    order = np.argsort(d, kind="stable")
    cum = np.cumsum(w[order])
    r_act = d[order][np.searchsorted(cum, frac * cum[-1])]
    return np.concatenate([(xm - xh) / L, [np.log(r_act / L)]])
