"""GPU parity of one coupled LBM step at the benchmarks' particle sizes,
element by element against the FP64 oracle, through the C-ABI.

The particles are the settling tank's cobblestone-like particles (24-40
control points, semi-axes 12-20 lu, Sec. 2.1 Eq. 1 fields with R_b ~ 40 lu)
and the precision tank's / bed's many-ball particles (64-128 control points,
radius 16 lu), each on a cropped window around it, moving and rotating so
that the step covers and uncovers nodes.  Ball counts are chosen with
n % 4 != 0 so that the flagging kernel's four-wide ball loop and its tail both
run.  Every step of the particle phase is compared: owners and node classes
(Sec. 2.1 Eq. 1; node classes of Sec. 2.3.2) and the link set bit-exact, the
wall fractions q, the populations after refill, interpolated bounce-back and
collision (Sec. 2.3.2 Eqs. eqneq1, eqneq2, neqd, refill equation) and the
momentum-exchange force and torque, at the bars of tests/coupling_parity.py.
"""
import json
import os

import numpy as np
import pytest

from oracle import metaball
from paper_2209_10411_gb300 import scenes
from tests import coupling_parity as cp
from tests.gpu_helpers import binding

pytestmark = pytest.mark.gpu

OUT = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "gpurun_out")


def _record(name, res):
    """Append the measured errors to gpurun_out/parity_scale.jsonl (kept for
    the write-up; the assertions are in compare_step)."""
    os.makedirs(OUT, exist_ok=True)
    keep = {k: v for k, v in res.items() if k not in ("F", "T")}
    with open(os.path.join(OUT, "parity_scale.jsonl"), "a") as fh:
        fh.write(json.dumps(dict(keep, case=name)) + "\n")


def _moved(P, dX, dq):
    """The pose one step earlier: shifted by -dX, the quaternion perturbed by
    dq (then rounded to float32)."""
    return dict(P, pos=P["pos"] - np.asarray(dX, float), quat=scenes.f32(P["quat"] + np.asarray(dq, float)))


@pytest.mark.parametrize("index,mode", [(0, "ibb"), (2, "ibb"), (0, "ladd")])
def test_settling_cobble_window(index, mode):
    """One of the settling tank's cobbles (particle 0: 38 control points,
    particle 2: 31) on a 96^3 window: position with fractional parts, a step
    of (0.6, -0.4, 0.5) lu and a small rotation since the previous flags."""
    B = binding()
    spec = scenes.config2().particles[index]
    assert len(spec.k) % 4 != 0
    shape = (96, 96, 96)
    P = cp.prepared(spec, np.array([48.37, 47.61, 48.13]), spec.quat, (0.012, -0.008, 0.01), (0.002, -0.0015, 0.001))
    Pp = _moved(P, (0.6, -0.4, 0.5), (0.0, 0.02, -0.015, 0.01))
    f0 = cp.initial_flow(shape, seed=31 + index)
    sim = cp.run_one_step(B, shape, [Pp], [P], f0, mode)
    res = cp.compare_step(sim, shape, [Pp], [P], f0, mode)
    sim.close()
    assert res["links"] > 40000 and res["new_nodes"] > 100
    _record("cobble%d_%s" % (index, mode), res)


def test_two_cobbles_overlapping():
    """Two settling-tank cobbles (34 and 31 control points) whose boxes overlap
    and whose solids share 420 nodes (owner: the lower index, reading A4) on a
    128x96x96 window, both moving."""
    B = binding()
    specs = scenes.config2().particles
    shape = (128, 96, 96)
    A = cp.prepared(specs[1], np.array([37.3, 48.4, 47.7]), specs[1].quat, (0.01, 0.0, -0.006),
                    (0.001, 0.002, -0.001))
    C = cp.prepared(specs[2], np.array([87.3, 47.1, 48.6]), specs[2].quat, (-0.01, 0.004, 0.0),
                    (-0.002, 0.0, 0.0015))
    prev = [_moved(A, (0.5, 0.3, -0.4), (0.0, -0.01, 0.01, 0.0)), _moved(C, (-0.45, 0.2, 0.3), (0.0, 0.0, 0.01, -0.02))]
    both = ((metaball.flag_nodes(shape, [A]) >= 0) & (metaball.flag_nodes(shape, [C]) >= 0)).sum()
    assert both > 100   # the lowest-index owner rule decides these nodes
    f0 = cp.initial_flow(shape, seed=41)
    sim = cp.run_one_step(B, shape, prev, [A, C], f0, "ibb")
    res = cp.compare_step(sim, shape, prev, [A, C], f0, "ibb")
    sim.close()
    _record("two_cobbles_ibb", dict(res, shared_solid_nodes=int(both)))


@pytest.mark.parametrize("n_balls", [63, 101, 127])
def test_many_ball_particle(n_balls):
    """A precision-tank / bed particle of 63-127 control points (uniform in a
    ball of 8 lu, sum k = 16^2) on a 64^3 window."""
    B = binding()
    rng = np.random.default_rng(100 + n_balls)
    c, k, _ = scenes.clustered(rng, n_balls, 16.0)
    spec = scenes.ParticleSpec(c, k, 2.5, 1.0, None, None)
    shape = (64, 64, 64)
    P = cp.prepared(spec, np.array([32.21, 31.83, 32.47]), scenes.random_unit_quaternion(rng), (0.01, 0.01, -0.012),
                    (0.003, -0.002, 0.002))
    Pp = _moved(P, (0.55, 0.45, -0.6), (0.0, 0.015, 0.01, -0.02))
    f0 = cp.initial_flow(shape, seed=50 + n_balls)
    sim = cp.run_one_step(B, shape, [Pp], [P], f0, "ibb")
    res = cp.compare_step(sim, shape, [Pp], [P], f0, "ibb")
    sim.close()
    assert res["links"] > 10000 and res["new_nodes"] > 50
    _record("balls%d_ibb" % n_balls, res)
