"""Error of the population storages against the FP64 oracle (a measured
number, not a defined result): a particle moving at 0.02 lu/step through the
64^3 closed box for 40 coupled steps, in FP32, FP16-deviation and
BF16-deviation storage.  Reported: the relative L2 error of the fluid
velocity field and the relative error of the hydrodynamic force after the
last step.  The asserted bounds are the stated accuracy of each storage."""
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
BOUNDS = {0: (1e-4, 1e-3), 1: (2e-2, 5e-2), 2: (1e-1, 2e-1)}  # (velocity, force) per storage


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
