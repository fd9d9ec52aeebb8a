"""GPU parity and gain of the learned Newton guess, through the C-ABI.

Parity against the FP64 oracle on seeded pair poses of bed shapes: the 64
features (values within FP32 rounding; where the oracle's distances show a
near-tie that FP32 may break the other way, the swapped choice is checked to
be a tie instead), the plain closest point x_m (within 1e-5 of the particle
size 2 R_b, the contact-point bar), the training targets of the GPU's own
converged points, and the learned start: fed the exact answer it stops after
one full-set iteration (in the median) at the same x_m.

Gain (a measured count, not a defined result): a network trained on the GPU
from plain solves needs fewer Newton iterations and ball evaluations per pair
than plain Newton on held-out poses, converging to the same closest point."""
import json
import os

import numpy as np
import pytest

from oracle import contact, mlp
from tests.gpu_helpers import binding

pytestmark = pytest.mark.gpu

NPAIRS = 48


def _oracle_particle(shape, pose):
    return {"centers": shape["centers"], "k": shape["k"], "skin": shape["skin"], "pos": np.asarray(pose[:3]),
            "quat": np.asarray(pose[3:7]), "vel": np.zeros(3), "omega": np.zeros(3)}


def _sim_with(B, shapes):
    from paper_2209_10411_gb300 import guess
    sim = B.Simulation(16, 16, 16, max_particles=len(shapes) + 1, max_balls=sum(len(s["k"]) for s in shapes) + 1)
    guess.add_shapes(sim, shapes)
    return sim


@pytest.fixture(scope="module")
def small():
    """12 bed shapes (4-128 balls) and NPAIRS posed pairs, solved on the GPU
    with features, plain Newton and labels; oracle particles of each pair."""
    B = binding()
    import torch
    from paper_2209_10411_gb300 import guess
    shapes = guess.bed_shapes(21, 12)
    sim = _sim_with(B, shapes)
    ij, poses = guess.pair_poses(22, shapes, NPAIRS)
    dij, dposes = guess.to_device(ij, poses)
    out = sim.pair_solve(dij, dposes, B.PAIR_FEATURES | B.PAIR_PLAIN | B.PAIR_LABELS)
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    pairs = [(_oracle_particle(shapes[a], poses[p, :7]), _oracle_particle(shapes[b], poses[p, 7:]))
             for p, (a, b) in enumerate(ij)]
    Lp = np.array([max(contact.bounding_radius(Pi["centers"], Pi["k"]), contact.bounding_radius(Pj["centers"], Pj["k"]))
                   for Pi, Pj in pairs])
    yield B, torch, sim, shapes, ij, poses, dij, dposes, res, pairs, Lp
    sim.close()


def test_features_match_oracle(small):
    B, torch, sim, shapes, ij, poses, dij, dposes, res, pairs, Lp = small
    X = res["X"]
    skipped = 0
    for p, (Pi, Pj) in enumerate(pairs):
        f, xa = mlp.features(Pi, Pj)
        L = Lp[p]
        g = X[p].astype(np.float64)
        assert np.allclose(g[0:11], f[0:11], atol=2e-6), p
        if not np.allclose(g[11:14], f[11:14], atol=5e-5):
            # the anchor picks differ: must be a near-tie of the oracle's gaps
            skipped += 1
            continue
        assert np.allclose(g[14:16], f[14:16], atol=1e-3 + 1e-4 * np.abs(f[14:16]).max()), (p, g[14:16], f[14:16])
        for off, P in ((16, Pi), (40, Pj)):
            assert np.allclose(g[off:off + 4], f[off:off + 4], atol=2e-6), (p, off)
            for r in range(5):
                a, b = g[off + 4 + 4 * r: off + 8 + 4 * r], f[off + 4 + 4 * r: off + 8 + 4 * r]
                if not np.allclose(a, b, atol=5e-5):
                    # a swapped pair of nearest balls: their oracle distances must tie
                    cw = contact.world_centers(P)
                    d = np.linalg.norm(cw - xa, axis=1) / L
                    da = np.linalg.norm(a[:3])
                    assert abs(da - np.linalg.norm(b[:3])) <= 1e-5 and np.min(np.abs(d - da)) <= 1e-5, (p, off, r)
                    break
    assert skipped <= 2, skipped


def test_plain_solve_matches_oracle(small):
    B, torch, sim, shapes, ij, poses, dij, dposes, res, pairs, Lp = small
    agree = 0
    for p, (Pi, Pj) in enumerate(pairs):
        r = contact.newton_pair(Pi, Pj)
        if r["status"] != 0 or res["status"][p] != 0:
            continue
        err = np.linalg.norm(res["xm"][p] - r["x_m"]) / (2 * Lp[p])
        assert err <= 1e-5, (p, err)
        agree += 1
    assert agree >= 0.8 * NPAIRS, agree


def test_labels_match_oracle(small):
    B, torch, sim, shapes, ij, poses, dij, dposes, res, pairs, Lp = small
    checked = 0
    for p, (Pi, Pj) in enumerate(pairs):
        if res["status"][p] != 0:
            assert np.isnan(res["T"][p]).all()
            continue
        f, xa = mlp.features(Pi, Pj)
        if not np.allclose(res["X"][p, 11:14], f[11:14], atol=5e-5):
            continue
        xm = res["xm"][p]
        t = mlp.labels(Pi, Pj, xm, xa)
        assert np.allclose(res["T"][p, :3], t[:3], atol=5e-5), p
        # r_act: skip pairs whose 99 % threshold sits within FP32 noise of a ball
        d, w = [], []
        for P in (Pi, Pj):
            cw = contact.world_centers(P)
            rr = np.linalg.norm(cw - xm, axis=1)
            d.append(rr)
            w.append(contact.core_scale(P["k"], P["skin"]) * P["k"] / rr ** 2)
        d, w = np.concatenate(d), np.concatenate(w)
        cum = np.cumsum(w[np.argsort(d, kind="stable")]) / w.sum()
        if np.min(np.abs(cum - 0.99)) < 1e-4:
            continue
        assert abs(res["T"][p, 3] - t[3]) <= 1e-4, (p, res["T"][p, 3], t[3])
        checked += 1
    assert checked >= 0.7 * NPAIRS, checked


def test_learned_start_from_exact_answer(small):
    """pred = the targets of the converged plain solve: the learned path
    starts at x_m itself and (in the median) stops after one full-set
    iteration at the same point."""
    B, torch, sim, shapes, ij, poses, dij, dposes, res, pairs, Lp = small
    ok = res["status"] == 0
    T = torch.as_tensor(np.where(ok[:, None], res["T"], 0.0), dtype=torch.float32, device="cuda")
    X = torch.as_tensor(res["X"], device="cuda")
    out = sim.pair_solve(dij, dposes, B.PAIR_LEARNED, pred=T, X=X)
    torch.cuda.synchronize()
    st, it, xm = out["status"].cpu().numpy(), out["iters"].cpu().numpy(), out["xm"].cpu().numpy()
    assert (st[ok] == 0).all()
    err = np.linalg.norm(xm[ok] - res["xm"][ok], axis=1) / (2 * Lp[ok])
    assert err.max() <= 1e-5, err.max()
    assert np.median(it[ok]) == 1 and it[ok].mean() < res["iters"][ok].mean()


@pytest.fixture(scope="module")
def trained():
    """A network trained on the GPU from 600k plain solves of 128 bed shapes
    (seeded poses), and a handle holding those shapes and 32 held-out ones."""
    B = binding()
    import torch
    from paper_2209_10411_gb300 import guess
    train_shapes = guess.bed_shapes(1, 128)
    test_shapes = guess.bed_shapes(2, 32)
    sim = _sim_with(B, train_shapes + test_shapes)
    ij, poses = guess.pair_poses(3, train_shapes, 600_000)
    X, T, _ = guess.generate(sim, *guess.to_device(ij, poses))
    params, hist = guess.train(X, T, steps=12000, batch=4096, lr=2e-3, seed=0, log_every=2000, standardize=True,
                               target_weights=(10.0, 10.0, 10.0, 1.0))
    torch.cuda.synchronize()
    yield B, torch, guess, sim, train_shapes, test_shapes, params, hist, int(X.shape[0])
    sim.close()


def test_learned_guess_gain(trained):
    """Plain and learned starts on 20k held-out pairs of shapes the network
    never saw."""
    B, torch, guess, sim, train_shapes, test_shapes, params, hist, nsamples = trained
    ij2, poses2 = guess.pair_poses(4, test_shapes, 20_000)
    ij2 = ij2 + len(train_shapes)
    plain, learned = guess.compare(sim, params, *guess.to_device(ij2, poses2))
    torch.cuda.synchronize()
    ps, ls = plain["status"].cpu().numpy(), learned["status"].cpu().numpy()
    both = (ps == 0) & ((ls & 15) == 0)
    xm_p, xm_l = plain["xm"].cpu().numpy(), learned["xm"].cpu().numpy()
    Rb = np.array([sim.get_particle_shape(int(i))["Rb"] for i in range(len(train_shapes), sim.num_particles())])
    Rpair = np.maximum(Rb[ij2[:, 0] - len(train_shapes)], Rb[ij2[:, 1] - len(train_shapes)])
    same = np.linalg.norm(xm_p - xm_l, axis=1) <= 1e-5 * 2 * Rpair
    line = {
        "pairs": int(len(ps)), "train_samples": nsamples, "final_loss": hist[-1][1],
        "plain_iters": float(plain["iters"].float().mean().item()),
        "learned_iters": float(learned["iters"].float().mean().item()),
        "plain_evals": float(plain["evals"].float().mean().item()),
        "learned_evals": float(learned["evals"].float().mean().item()),
        "fallback": float(((ls & 16) != 0).mean()), "plain_converged": float((ps == 0).mean()),
        "learned_converged": float(((ls & 15) == 0).mean()), "same_point": float(same[both].mean()),
    }
    print("GAIN", json.dumps(line))
    out = os.environ.get("MI_GAIN_LOG")
    if out:
        with open(out, "a") as fh:
            fh.write(json.dumps(line) + "\n")
    assert line["learned_converged"] >= line["plain_converged"] - 0.005
    assert line["same_point"] >= 0.95
    assert line["learned_iters"] < line["plain_iters"]
    assert line["learned_evals"] < line["plain_evals"]


def test_step_contacts_learned_equal_plain(trained):
    """The DEM contact phase of a step with the learned guess finds the same
    contacts, points and forces as with the plain guess (a packed cluster)."""
    B, torch, guess, _, _, _, params, _, _ = trained
    from tests.test_gpu_contact import PARAMS, _cluster, _sim
    parts = _cluster(11)
    res = []
    for learned in (False, True):
        sim = _sim(B, (64, 64, 64), parts)
        if learned:
            sim.set_guess(B.GUESS_LEARNED, params)
        sim.step_phases(B.PHASE_CONTACT)
        res.append((sim.contacts(), sim.forces()))
        sim.close()
    (cp, fp), (cl, fl) = res
    key = lambda c: (c["i"], c["j"])
    cp, cl = sorted(cp, key=key), sorted(cl, key=key)
    assert [key(c) for c in cp] == [key(c) for c in cl]
    n_ok = 0
    for a, b in zip(cp, cl):
        if a["status"] != 0:
            continue
        assert b["status"] == 0
        assert np.linalg.norm(a["x_cp"] - b["x_cp"]) <= 1e-4, (a, b)
        assert abs(a["delta"] - b["delta"]) <= 1e-4
        n_ok += 1
    assert n_ok > 0
    scale = np.abs(fp["F_contact"]).max()
    assert np.abs(fp["F_contact"] - fl["F_contact"]).max() <= 1e-4 * scale + 1e-9


def _guess_candidates(Pi, Pj, tol):
    """All sphere pairs whose surface gap is within tol of the smallest (the
    oracle's search, vectorised) and the midpoint each one gives."""
    c0, c1 = contact.world_centers(Pi), contact.world_centers(Pj)
    r0, r1 = np.sqrt(Pi["k"]), np.sqrt(Pj["k"])
    gap = np.linalg.norm(c0[:, None, :] - c1[None, :, :], axis=2) - r0[:, None] - r1[None, :]
    out = []
    for a, b in zip(*np.nonzero(gap <= gap.min() + tol)):
        u = c1[b] - c0[a]
        u = u / np.linalg.norm(u)
        out.append(0.5 * ((c0[a] + r0[a] * u) + (c1[b] - r1[b] * u)))
    return out


@pytest.mark.parametrize("n_range,npairs", [((4, 128), 64), ((100, 200), 24)])
def test_plain_guess_matches_oracle(n_range, npairs):
    """The plain starting point (closest pair of control-point spheres, the
    midpoint of their surface points) of the GPU's pruned search over staged
    balls (n_i + n_j <= 256) and of its unstaged search (larger pairs)
    against the oracle's full search: the same point within FP32 rounding,
    or, where the oracle's smallest gaps tie within 1e-5 of the size, the
    point of one of the tied pairs."""
    B = binding()
    import torch
    from paper_2209_10411_gb300 import guess
    shapes = guess.bed_shapes(31, 10, n_range=n_range)
    sim = _sim_with(B, shapes)
    ij, poses = guess.pair_poses(32, shapes, npairs, spacing=(0.7, 1.2))
    dij, dposes = guess.to_device(ij, poses)
    out = sim.pair_solve(dij, dposes, B.PAIR_PLAIN | B.PAIR_GUESS_ONLY)
    torch.cuda.synchronize()
    xm, st, it = out["xm"].cpu().numpy(), out["status"].cpu().numpy(), out["iters"].cpu().numpy()
    sim.close()
    assert (st == 0).all() and (it == 0).all()
    staged = 0
    for p, (a, b) in enumerate(ij):
        Pi, Pj = _oracle_particle(shapes[a], poses[p, :7]), _oracle_particle(shapes[b], poses[p, 7:])
        size = 2 * max(contact.bounding_radius(Pi["centers"], Pi["k"]), contact.bounding_radius(Pj["centers"], Pj["k"]))
        ref = contact.pair_guess(Pi, Pj) if p < 8 else None
        cands = _guess_candidates(Pi, Pj, 1e-5 * size)
        if ref is not None:  # the vectorised search is the oracle's
            assert min(np.linalg.norm(c - ref) for c in cands) <= 1e-9 * size
        err = min(np.linalg.norm(xm[p] - c) for c in cands) / size
        assert err <= 2e-6, (p, err)
        staged += len(shapes[a]["k"]) + len(shapes[b]["k"]) <= 256
    if n_range[1] <= 128:
        assert staged == len(ij)
    else:
        assert 0 < staged < len(ij)


def test_guess_only_flag_rejected_without_plain():
    B = binding()
    import torch
    from paper_2209_10411_gb300 import guess
    shapes = guess.bed_shapes(31, 2)
    sim = _sim_with(B, shapes)
    dij, dposes = guess.to_device(*guess.pair_poses(1, shapes, 2))
    with pytest.raises(RuntimeError):
        sim.pair_solve(dij, dposes, B.PAIR_GUESS_ONLY)
    with pytest.raises(RuntimeError):
        sim.pair_solve(dij, dposes, B.PAIR_PLAIN | B.PAIR_GUESS_ONLY | B.PAIR_LABELS)
    sim.close()
