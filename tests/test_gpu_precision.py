"""Error of the population storages against the FP64 oracle (a measured
number, not a defined result), in FP32, FP16-deviation and BF16-deviation
storage, on two workloads:

  * a particle moving at 0.02 lu/step through the 64^3 closed box of the
    oracle-size configuration, 40 coupled steps;
  * the 128^3 sub-run of the 512^3 precision tank: its eight whole particles
    (10-50 control points) moving at 0.015 lu/step, 30 coupled steps, against
    the FP64 reference stored by tests/golden/make_c4_subrun.py (velocities at
    8192 sampled fluid nodes, half of them within 3 lu of a particle, and each
    particle's hydrodynamic force).

Reported: the relative L2 error of the fluid velocity and the largest
relative error of a hydrodynamic force after the last step.  The asserted
bounds, about 2.5 times the measured errors, are the stated accuracy of each
storage."""
import json
import os

import numpy as np
import pytest

from oracle import lbm, metaball, step as ostep
from paper_2209_10411_gb300 import scenes
from tests.gpu_helpers import binding
from tests.coupling_parity import prepared as _prepared

pytestmark = pytest.mark.gpu

NSTEPS = 40
# (velocity, force) per storage, about 2.5 times the measured errors (FP32
# 1.1e-5 / 1.5e-6, FP16 2.7e-4 / 2.8e-4, BF16 1.2e-3 / 1.7e-3)
BOUNDS = {0: (3e-5, 4e-6), 1: (7e-4, 7e-4), 2: (3e-3, 4.5e-3)}


@pytest.fixture(scope="module")
def reference():
    sc = scenes.config1()
    spec = sc.particles[0]
    P = _prepared(spec, spec.pos, spec.quat, (0.0, 0.0, -0.02), (0.0, 0.0, 0.0))
    shape = sc.shape
    S = ostep.OracleState(shape, lbm.rest_state((shape[2], shape[1], shape[0])), [P], tau=sc.tau,
                          gravity=(0.0, 0.0, 0.0))
    for _ in range(NSTEPS):
        ostep.step(S)
    return sc, P, S


def _velocity(f, fluid):
    rho, u = lbm.moments(f)
    return u[:, fluid]


@pytest.mark.parametrize("storage", [0, 1, 2])
def test_storage_error_against_fp64(reference, storage):
    B = binding()
    sc, P, S = reference
    shape = sc.shape
    sim = B.Simulation(*shape, tau=sc.tau, storage=storage)
    sim.add_particle(P["centers"], P["k"], P["density"], P["skin"], P["pos"], P["quat"], P["vel"], P["omega"],
                     mass_props={"mass": P["mass"], "volume": P["volume"], "inertia": P["inertia"]})
    sim.step(NSTEPS)
    f = sim.get_populations().astype(np.float64)
    F = sim.forces()["F_hydro"][0]
    sim.close()
    fluid = (metaball.flag_nodes(shape, S.particles) < 0) & np.isfinite(S.f).all(0)
    u_ref = _velocity(S.f, fluid)
    u = _velocity(f, fluid)
    eu = np.linalg.norm(u - u_ref) / np.linalg.norm(u_ref)
    eF = np.linalg.norm(F - S.F_hydro[0]) / np.linalg.norm(S.F_hydro[0])
    line = {"storage": ["f32", "f16-dev", "bf16-dev"][storage], "steps": NSTEPS, "velocity_rel_l2": eu,
            "force_rel": eF, "u_max": float(np.abs(u_ref).max())}
    print("PRECISION", json.dumps(line))
    out = os.environ.get("MI_PRECISION_LOG")
    if out:
        with open(out, "a") as fh:
            fh.write(json.dumps(line) + "\n")
    bu, bf = BOUNDS[storage]
    assert eu < bu and eF < bf, line


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "c4_subrun_fp64.npz")
# (velocity rel. L2, force rel.) per storage on the 128^3 sub-run, about 2.5
# times the measured errors (FP32 1.4e-6 / 1.6e-6, FP16 1.3e-4 / 1.0e-4,
# BF16 1.1e-3 / 6.0e-4)
BOUNDS_C4 = {0: (3.5e-6, 4e-6), 1: (3.5e-4, 2.5e-4), 2: (2.7e-3, 1.5e-3)}


@pytest.mark.parametrize("storage", [0, 1, 2])
def test_storage_error_c4_subrun(storage):
    from tests.golden import make_c4_subrun as mk
    B = binding()
    ref = np.load(GOLDEN)
    shape, parts, lo, idx, gravity, tau = mk.subrun()
    assert np.array_equal(lo, ref["corner"]) and np.array_equal(idx, ref["tank_indices"])
    sim = B.Simulation(*shape, tau=tau, gravity=gravity, storage=storage, max_particles=len(parts))
    for P in parts:
        sim.add_particle(P["centers"], P["k"], P["density"], P["skin"], P["pos"], P["quat"], P["vel"], P["omega"],
                         mass_props={"mass": P["mass"], "volume": P["volume"], "inertia": P["inertia"]})
    sim.step(int(ref["steps"]))
    f = sim.get_populations().astype(np.float64)
    F = sim.forces()["F_hydro"]
    pos = np.array([sim.get_particle_state(i)["pos"] for i in range(len(parts))])
    sim.close()
    z, y, x = (ref["nodes_zyx"][:, a].astype(np.int64) for a in range(3))
    _, u = lbm.moments(f[:, z, y, x])
    u = u.T
    u_ref = ref["u"]
    eu = np.linalg.norm(u - u_ref) / np.linalg.norm(u_ref)
    eu_near = np.linalg.norm(u[4096:] - u_ref[4096:]) / np.linalg.norm(u_ref[4096:])
    F_ref = ref["F_hydro"]
    eF = float(max(np.linalg.norm(F[i] - F_ref[i]) / np.linalg.norm(F_ref[i]) for i in range(len(parts))))
    ep = float(np.abs(pos - ref["pos"]).max())
    line = {"workload": "128^3 sub-run of the 512^3 precision tank", "storage": ["f32", "f16-dev", "bf16-dev"][storage],
            "steps": int(ref["steps"]), "particles": len(parts), "velocity_rel_l2": eu,
            "velocity_rel_l2_near_particles": eu_near, "force_rel": eF, "position_abs": ep,
            "u_max": float(np.abs(u_ref).max())}
    print("PRECISION", json.dumps(line))
    out = os.environ.get("MI_PRECISION_LOG")
    if out:
        with open(out, "a") as fh:
            fh.write(json.dumps(line) + "\n")
    bu, bf = BOUNDS_C4[storage]
    assert eu < bu and eF < bf, line
