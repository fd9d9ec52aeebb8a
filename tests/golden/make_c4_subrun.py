"""Writes tests/golden/c4_subrun_fp64.npz: the FP64 oracle's reference for the
storage-precision test on a 128^3 sub-run of the 512^3 precision tank.

The sub-run: the 128^3 box of the precision tank (scenes.config4) at the
corner that holds the most whole particles (every particle whose bounding
sphere, plus 2 lu, lies inside; eight of them, 10-50 control points), fluid
at rest, each particle given a velocity of 0.015 lu/step in a seeded random
direction and a small spin, gravity 1e-5 lu/step^2, 30 coupled oracle steps
(flags, links, refill, IBB, momentum exchange, stream-collide, contacts,
rigid-body update).  Stored: the sub-run's definition, the velocity of the
fluid at 8192 sampled nodes that are fluid at the end (4096 uniform among
all fluid nodes, 4096 among fluid nodes within 3 lu of a solid node), and
each particle's hydrodynamic force and torque of the last step.

Only oracle/ and the seeded input generators are called.  Run:
    python tests/golden/make_c4_subrun.py      (about 10 minutes on one core)
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c4_subrun_fp64.npz")
SIDE = 128
STEPS = 30
SPEED = 0.015
SEED = 4


def subrun():
    """The sub-run's inputs: (shape, particle dicts, corner); the particle
    dicts hold control points about the oracle's quadrature centroid."""
    from oracle import metaball
    from paper_2209_10411_gb300 import scenes
    sc = scenes.config4()
    pos = np.array([p.pos for p in sc.particles])
    Rb = np.array([metaball.bounding_radius(p.centers, p.k) for p in sc.particles])
    best = None
    for cx in range(0, sc.shape[0] - SIDE + 1, 8):
        for cy in range(0, sc.shape[1] - SIDE + 1, 8):
            for cz in range(0, sc.shape[2] - SIDE + 1, 8):
                lo = np.array([cx, cy, cz])
                inside = ((pos - Rb[:, None] - 2 >= lo) & (pos + Rb[:, None] + 2 <= lo + SIDE - 1)).all(1)
                if best is None or inside.sum() > best[0]:
                    best = (int(inside.sum()), lo, np.nonzero(inside)[0])
    _, lo, idx = best
    rng = np.random.default_rng(SEED)
    parts = []
    for i in idx:
        s = sc.particles[i]
        mp = metaball.mass_properties(s.centers, s.k, s.density)
        c = s.centers - mp["centroid"]
        mp = metaball.mass_properties(c, s.k, s.density)
        v = rng.normal(size=3)
        v = scenes.f32(SPEED * v / np.linalg.norm(v))
        w = scenes.f32(rng.uniform(-1e-3, 1e-3, 3))
        # the control points about the quadrature centroid, the body origin at
        # the tank position (both sides get the same dict)
        X = s.pos - lo
        parts.append({"centers": c, "k": s.k.copy(), "pos": np.asarray(X, float), "quat": np.asarray(s.quat, float),
                      "vel": v, "omega": w, "density": s.density, "skin": s.skin, "mass": mp["mass"],
                      "volume": mp["volume"], "inertia": mp["inertia"]})
    return (SIDE, SIDE, SIDE), parts, lo, idx, tuple(float(g) for g in sc.gravity), sc.tau


def main():
    from oracle import lbm, metaball, step as ostep
    shape, parts, lo, idx, gravity, tau = subrun()
    S = ostep.OracleState(shape, lbm.rest_state(shape), parts, tau=tau, gravity=gravity)
    for n in range(STEPS):
        ostep.step(S)
        print("step", n + 1, flush=True)
    owner = metaball.flag_nodes(shape, S.particles)
    fluid = (owner < 0) & np.isfinite(S.f).all(0)
    solid = owner >= 0
    near = np.zeros_like(solid)
    zz, yy, xx = np.nonzero(solid)
    for dz in range(-3, 4):
        for dy in range(-3, 4):
            for dx in range(-3, 4):
                z, y, x = zz + dz, yy + dy, xx + dx
                ok = (z >= 0) & (z < shape[2]) & (y >= 0) & (y < shape[1]) & (x >= 0) & (x < shape[0])
                near[z[ok], y[ok], x[ok]] = True
    rng = np.random.default_rng(SEED + 1)
    all_f = np.stack(np.nonzero(fluid), 1)
    near_f = np.stack(np.nonzero(fluid & near), 1)
    pick = np.concatenate([all_f[rng.choice(len(all_f), 4096, replace=False)],
                           near_f[rng.choice(len(near_f), 4096, replace=False)]])   # (z, y, x)
    rho, u = lbm.moments(S.f[:, pick[:, 0], pick[:, 1], pick[:, 2]])
    np.savez_compressed(OUT, corner=np.asarray(lo), tank_indices=np.asarray(idx), steps=STEPS, speed=SPEED,
                        seed=SEED, nodes_zyx=pick.astype(np.int16), u=u.T, F_hydro=S.F_hydro, T_hydro=S.T_hydro,
                        pos=np.array([P["pos"] for P in S.particles]))
    print("wrote", OUT)


if __name__ == "__main__":
    main()
