"""GPU parity of the learned-guess network kernels (tensor-core BF16 GEMMs
with FP32 accumulation, MSE, AdamW) against the FP64 oracle, through the
C-ABI.

Two bars per quantity: against the FP64 oracle, relative Frobenius error
<= 1e-2 (BF16 operands carry 8 significant bits); for the gradients the
oracle's backprop takes its ReLU masks from the BF16 forward, since the
kernels decide them in that precision; and against the oracle fed with
BF16-rounded operands at every product (what the kernels multiply), relative
error <= 2e-4 forward, 2e-3 backward (FP32 accumulation order, and dY
inheriting the forward's difference).  The batch sizes span
several 64-row tiles and a ragged tail."""
import numpy as np
import pytest

from oracle import mlp
from tests.gpu_helpers import binding

pytestmark = pytest.mark.gpu

KEYS = ["W1", "b1", "W2", "b2", "W3", "b3"]


def _flat(p):
    return np.concatenate([p[k].ravel() for k in KEYS]).astype(np.float32)


def _unflat(v):
    out, o = {}, 0
    for k, shp in zip(KEYS, [(64, 256), (256,), (256, 256), (256,), (256, 4), (4,)]):
        n = int(np.prod(shp))
        out[k] = np.asarray(v[o:o + n], dtype=np.float64).reshape(shp)
        o += n
    return out


def bf16(a):
    """Round float64 values to the nearest BF16 (ties to even) via float32."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _oracle_bf16(p, X, T):
    """Forward, loss and gradients with every product's operands rounded to
    BF16; also the forward's cache (its ReLU decisions) for mlp.backward."""
    Z1 = bf16(X) @ bf16(p["W1"]) + p["b1"]
    H1 = np.maximum(Z1, 0)
    Z2 = bf16(H1) @ bf16(p["W2"]) + p["b2"]
    H2 = np.maximum(Z2, 0)
    Y = bf16(H2) @ bf16(p["W3"]) + p["b3"]
    cache = {"X": X, "Z1": Z1, "H1": H1, "Z2": Z2, "H2": H2}
    n = X.shape[0]
    dY = 2.0 * (Y - T) / n
    g = {"W3": bf16(H2).T @ bf16(dY), "b3": dY.sum(0)}
    dZ2 = (bf16(dY) @ bf16(p["W3"]).T) * (H2 > 0)
    g["W2"] = bf16(H1).T @ bf16(dZ2)
    g["b2"] = dZ2.sum(0)
    dZ1 = (bf16(dZ2) @ bf16(p["W2"]).T) * (H1 > 0)
    g["W1"] = bf16(X).T @ bf16(dZ1)
    g["b1"] = dZ1.sum(0)
    return Y, g, cache


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-30))


@pytest.fixture(scope="module")
def setup():
    B = binding()
    import torch
    rng = np.random.default_rng(11)
    p = mlp.init_params(3)
    for k in ("b1", "b2", "b3"):
        p[k] = 0.1 * rng.normal(size=p[k].shape)
    p = _unflat(_flat(p))  # the float32 values the GPU holds
    return B, torch, rng, p


@pytest.mark.parametrize("n", [1, 63, 200, 1000])
def test_forward_backward_against_oracle(setup, n):
    B, torch, rng, p = setup
    X = rng.normal(size=(n, 64)).astype(np.float32).astype(np.float64)
    T = rng.normal(size=(n, 4)).astype(np.float32).astype(np.float64)
    dp = torch.as_tensor(_flat(p), device="cuda")
    dX = torch.as_tensor(X, dtype=torch.float32, device="cuda")
    dT = torch.as_tensor(T, dtype=torch.float32, device="cuda")
    Y, acts = B.mlp_forward(dp, dX)
    loss, dY = B.mlp_mse(Y, dT)
    G = B.mlp_backward(dp, dX, acts, dY)
    torch.cuda.synchronize()
    Yg = Y.cpu().numpy().astype(np.float64)
    Gg = _unflat(G.cpu().numpy())

    Yo, _ = mlp.forward(p, X)
    lo, _ = mlp.mse(Yo, T)
    assert _rel(Yg, Yo) <= 1e-2
    assert abs(float(loss.item()) - lo) <= 2e-2 * lo

    # FP64 backprop taking the ReLU decisions where the kernels take them (a
    # unit whose pre-activation is within BF16 rounding of 0 may switch sides,
    # and one switched unit moves a whole row of a batch-1 gradient)
    Yb, Gb, cache_b = _oracle_bf16(p, X, T)
    _, dYb = mlp.mse(Yb, T)
    Go = mlp.backward(p, cache_b, dYb)
    for k in KEYS:
        assert _rel(Gg[k], Go[k]) <= 1e-2, (k, _rel(Gg[k], Go[k]))

    assert _rel(Yg, Yb) <= 2e-4, _rel(Yg, Yb)
    for k in KEYS:
        assert _rel(Gg[k], Gb[k]) <= 2e-3, (k, _rel(Gg[k], Gb[k]))


@pytest.mark.parametrize("n", [1, 63, 200, 20000])
def test_fused_inference_against_oracle(setup, n):
    """Both fused kernels (tcgen05 with 128-row tiles, and mma.sync with
    64-row tiles; output layer in the epilogue) against the BF16-operand
    oracle and against the GEMM path; 20000 rows exceed one tile per SM, so
    the persistent loops run."""
    B, torch, rng, p = setup
    X = rng.normal(size=(n, 64)).astype(np.float32).astype(np.float64)
    dp = torch.as_tensor(_flat(p), device="cuda")
    dX = torch.as_tensor(X, dtype=torch.float32, device="cuda")
    img = B.mlp_pack(dp)
    Yt = B.mlp_infer(img, dX)               # tcgen05 / TMEM
    Yf = B.mlp_infer(img, dX, engine="mma")  # mma.sync, network resident in shared memory
    Yg, _ = B.mlp_forward(dp, dX)
    torch.cuda.synchronize()
    Yt, Yf, Yg = (a.cpu().numpy().astype(np.float64) for a in (Yt, Yf, Yg))
    Yb, _, _ = _oracle_bf16(p, X, np.zeros((n, 4)))
    Yo, _ = mlp.forward(p, X)
    for Y in (Yt, Yf):
        assert np.isfinite(Y).all()
        assert _rel(Y, Yb) <= 2e-4, _rel(Y, Yb)
        assert _rel(Y, Yg) <= 2e-4, _rel(Y, Yg)
        assert _rel(Y, Yo) <= 1e-2


def test_empty_batch_forward(setup):
    B, torch, rng, p = setup
    dp = torch.as_tensor(_flat(p), device="cuda")
    Y, acts = B.mlp_forward(dp, torch.zeros((0, 64), device="cuda"))
    torch.cuda.synchronize()
    assert Y.shape == (0, 4)


def test_adamw_against_oracle(setup):
    B, torch, rng, p = setup
    q = _unflat(_flat(p))
    st = {}
    dp = torch.as_tensor(_flat(q), device="cuda")
    m = torch.zeros_like(dp)
    v = torch.zeros_like(dp)
    for t in range(1, 4):
        g = {k: rng.normal(size=q[k].shape) for k in KEYS}
        gf = _flat(g)
        B.mlp_adamw(dp, torch.as_tensor(gf, device="cuda"), m, v, t, lr=1e-2, weight_decay=0.1)
        q = mlp.adamw(q, _unflat(gf), st, lr=1e-2, wd=0.1)
    torch.cuda.synchronize()
    got = dp.cpu().numpy().astype(np.float64)
    want = _flat(q).astype(np.float64)
    assert np.max(np.abs(got - want)) <= 1e-5 * max(1.0, np.abs(want).max())


def test_gpu_training_reduces_loss(setup):
    """A smooth synthetic target: 300 GPU AdamW steps cut the loss fivefold
    (the same check the oracle's training passes)."""
    B, torch, rng, _ = setup
    from paper_2209_10411_gb300 import guess
    X = rng.normal(size=(4096, 64))
    A = rng.normal(size=(64, 4)) / 8
    T = np.tanh(X @ A)
    dX = torch.as_tensor(X, dtype=torch.float32, device="cuda")
    dT = torch.as_tensor(T, dtype=torch.float32, device="cuda")
    p0 = guess.init_params(4)
    Y, _ = B.mlp_forward(p0, dX)
    l0 = float(B.mlp_mse(Y, dT)[0].item())
    p, _ = guess.train(dX, dT, steps=300, batch=512, lr=3e-3, lr_final=3e-4, seed=1, params=p0)
    Y, _ = B.mlp_forward(p, dX)
    l1 = float(B.mlp_mse(Y, dT)[0].item())
    assert l1 < 0.2 * l0, (l0, l1)
