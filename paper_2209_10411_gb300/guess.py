"""Training driver of the learned Newton guess.

The closest-point solve between two metaball cores (Sec. 2.3.1) is
Newton-Raphson from a heuristic start.  This module makes training data from
that solve itself and fits the 64 -> 256 -> 256 -> 4 network on the GPU:

  * `pair_poses` draws pairs of particle shapes in random relative poses with
    the spacing of a dense bed (centre distance (R_i + R_j) times U[lo, hi],
    R the shapes' far-field radius, uniform random orientations);
  * `generate` runs them through `Simulation.pair_solve` with
    FEATURES | PLAIN | LABELS (features, plain Newton, targets from the
    converged point) and keeps the converged pairs;
  * `train` fits the network with the library's own forward, MSE, backward and
    AdamW kernels (mini-batches drawn by a seeded permutation).

The network's arithmetic (forward, loss, backward, AdamW) and the solves run
in the library's kernels; torch holds the device arrays, draws the
permutations and standardizes the features (folded into the first layer
after training).
"""
import numpy as np

from . import scenes
from ._binding import (PAIR_FEATURES, PAIR_LABELS, PAIR_LEARNED, PAIR_PLAIN, mlp_adamw, mlp_backward,
                       mlp_forward, mlp_infer, mlp_mse, mlp_pack, mlp_param_count, mlp_scale_columns)


def bed_shapes(seed, n_shapes, n_range=(4, 128), R_range=(8.0, 16.0), skin=1.0):
    """Shapes of the dense-bed workload: n log-uniform in n_range, far-field
    radius R ~ U[R_range], balls clustered within 0.5 R (scenes.clustered)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_shapes):
        n = int(np.round(np.exp(rng.uniform(np.log(n_range[0]), np.log(n_range[1])))))
        R = rng.uniform(*R_range)
        c, k, r = scenes.clustered(rng, n, R)
        out.append({"centers": c, "k": k, "R": r, "skin": skin})
    return out


def add_shapes(sim, shapes):
    """Add the shapes as particles of a handle used only for pair solves:
    parked at the origin (pair_solve takes its poses from its arguments) with
    placeholder mass properties (no dynamics runs on them)."""
    for s in shapes:
        sim.add_particle(s["centers"], s["k"], 2.5, s["skin"], (0.0, 0.0, 0.0), (1.0, 0.0, 0.0, 0.0),
                         mass_props={"mass": 1.0, "volume": 1.0, "inertia": np.eye(3)})


def pair_poses(seed, shapes, n, spacing=(0.9, 1.5)):
    """n random pairs: indices (n, 2) int32 and poses (n, 14) float64
    (pos_i, quat_i, pos_j, quat_j), rounded to float32 values."""
    rng = np.random.default_rng(seed)
    m = len(shapes)
    i = rng.integers(0, m, n)
    j = rng.integers(0, m - 1, n)
    j = j + (j >= i)  # distinct shapes
    R = np.array([s["R"] for s in shapes])
    u = rng.normal(size=(n, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    D = (R[i] + R[j]) * rng.uniform(spacing[0], spacing[1], n)
    base = rng.uniform(-50.0, 50.0, (n, 3))

    def quats():
        u1, u2, u3 = rng.random((3, n))
        q = np.stack([np.sqrt(u1) * np.cos(2 * np.pi * u3), np.sqrt(1 - u1) * np.sin(2 * np.pi * u2),
                      np.sqrt(1 - u1) * np.cos(2 * np.pi * u2), np.sqrt(u1) * np.sin(2 * np.pi * u3)], 1)
        return q

    poses = np.concatenate([base, quats(), base + D[:, None] * u, quats()], 1)
    ij = np.stack([i, j], 1).astype(np.int32)
    return ij, scenes.f32(poses)


def to_device(ij, poses, device="cuda"):
    import torch
    return (torch.as_tensor(ij, dtype=torch.int32, device=device),
            torch.as_tensor(poses, dtype=torch.float64, device=device))


def generate(sim, ij, poses, batch=1 << 18):
    """Features X and targets T (CUDA tensors) of the converged pairs, and
    the plain solves' statistics (iterations, ball evaluations, status)."""
    import torch
    Xs, Ts, its, evs, sts = [], [], [], [], []
    for a in range(0, ij.shape[0], batch):
        out = sim.pair_solve(ij[a:a + batch], poses[a:a + batch], PAIR_FEATURES | PAIR_PLAIN | PAIR_LABELS)
        ok = out["status"] == 0
        Xs.append(out["X"][ok])
        Ts.append(out["T"][ok])
        its.append(out["iters"])
        evs.append(out["evals"])
        sts.append(out["status"])
    return torch.cat(Xs), torch.cat(Ts), {"iters": torch.cat(its), "evals": torch.cat(evs),
                                          "status": torch.cat(sts)}


def init_params(seed=0, device="cuda"):
    """He-uniform weights, zero biases, in the library's parameter layout."""
    import torch
    rng = np.random.default_rng(seed)
    parts = []
    for a, b in ((64, 256), (256, 256), (256, 4)):
        lim = np.sqrt(6.0 / a)
        parts.append(rng.uniform(-lim, lim, (a, b)).ravel())
        parts.append(np.zeros(b))
    p = np.concatenate(parts).astype(np.float32)
    assert p.size == mlp_param_count()
    return torch.as_tensor(p, device=device)


def train(X, T, steps=3000, batch=4096, lr=1e-3, lr_final=5e-5, weight_decay=1e-4, seed=0, params=None,
          log_every=0, standardize=False, target_weights=None):
    """Fit the network to (X, T) with AdamW (cosine learning-rate decay from
    lr to lr_final); returns (params, list of (step, loss)).

    standardize: train on per-feature standardized inputs (X - mu) / sd;
    target_weights w: train on T * w (w = (10, 10, 10, 1) stresses the
    position outputs, which set the Newton start, over log r_act).  Both are
    folded back into the first and last layers afterwards (W1 <- W1 / sd by
    rows, b1 <- b1 - (mu / sd) W1; W3 <- W3 / w by columns, b3 <- b3 / w),
    so the returned parameters act on raw features and give raw targets.
    The statistics and the fold are FP64 host arithmetic; the device arrays
    are rescaled by the library's column kernel (mi_mlp_scale_columns)."""
    import torch
    dev = X.device
    mu = sd = None
    if standardize:
        Xh = X.cpu().numpy()
        mu = Xh.mean(0, dtype=np.float64)
        sd = np.maximum(Xh.std(0, dtype=np.float64), 1e-3)
        X = X.clone()
        mlp_scale_columns(X, torch.as_tensor(mu.astype(np.float32), device=dev),
                          torch.as_tensor((1.0 / sd).astype(np.float32), device=dev))
    wt = None
    if target_weights is not None:
        wt = np.asarray(target_weights, dtype=np.float64)
        T = T.clone()
        mlp_scale_columns(T, torch.zeros(T.shape[1], dtype=torch.float32, device=dev),
                          torch.as_tensor(wt.astype(np.float32), device=dev))
    p, history = _fit(X, T, steps, batch, lr, lr_final, weight_decay, seed, params, log_every)
    if mu is None and wt is None:
        return p, history
    o1 = 64 * 256
    o3 = o1 + 256 + 256 * 256 + 256
    ph = p.cpu().numpy().astype(np.float64)
    W1, b1 = ph[:o1].reshape(64, 256), ph[o1:o1 + 256]
    W3, b3 = ph[o3:o3 + 1024].reshape(256, 4), ph[o3 + 1024:o3 + 1028]
    if mu is not None:
        b1 -= (mu / sd) @ W1
        W1 /= sd[:, None]
    if wt is not None:
        W3 /= wt[None, :]
        b3 /= wt
    return torch.as_tensor(ph.astype(np.float32), device=dev), history


def _fit(X, T, steps, batch, lr, lr_final, weight_decay, seed, params, log_every):
    import torch
    dev = X.device
    p = init_params(seed, dev) if params is None else params.clone()
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    g = torch.Generator(device="cpu")
    g.manual_seed(seed)
    n = X.shape[0]
    perm = torch.randperm(n, generator=g).to(dev)
    pos = 0
    history = []
    for t in range(1, steps + 1):
        if pos + batch > n:
            perm = torch.randperm(n, generator=g).to(dev)
            pos = 0
        idx = perm[pos:pos + batch]
        pos += batch
        xb, tb = X[idx].contiguous(), T[idx].contiguous()
        Y, acts = mlp_forward(p, xb)
        loss, dY = mlp_mse(Y, tb)
        grads = mlp_backward(p, xb, acts, dY)
        rate = lr_final + 0.5 * (lr - lr_final) * (1 + np.cos(np.pi * (t - 1) / max(1, steps - 1)))
        mlp_adamw(p, grads, m, v, t, lr=rate, weight_decay=weight_decay)
        if log_every and (t % log_every == 0 or t == 1):
            history.append((t, float(loss.item())))
    return p, history


def predict(params, X):
    """Network outputs for X through the fused inference kernel."""
    return mlp_infer(mlp_pack(params), X.contiguous())


def compare(sim, params, ij, poses):
    """Plain and learned solves of the same pairs: per-pair iterations, ball
    evaluations, status and closest points of both (CUDA tensors)."""
    plain = sim.pair_solve(ij, poses, PAIR_FEATURES | PAIR_PLAIN)
    pred = predict(params, plain["X"])
    learned = sim.pair_solve(ij, poses, PAIR_LEARNED, pred=pred, X=plain["X"])
    return plain, learned
