"""Stokes drag of a periodic sphere array on the GPU path (the coupled step
of Sec. 2.3 on a resting particle, through the C-ABI), against the known
low-Reynolds limit and against the FP64 oracle run on the same inputs.

A sphere of radius 4.5 rests in a periodic 24^3 box and a uniform body force
drives the fluid; after 600 steps from a uniform stream, F / U (U the
superficial velocity) is within 6 % of Hasimoto's periodic-array drag
6 pi mu R K(c) and within 1e-3 of the oracle's F / U (FP32 populations
against FP64 over 600 steps); the fluid's momentum gains g N_fluid - F per
step up to the FP32 rounding of the populations."""
import numpy as np
import pytest

from oracle import coupling, lbm, metaball
from oracle.d3q19 import E
from tests.gpu_helpers import binding

pytestmark = pytest.mark.gpu

L, R, G, STEPS = 24, 4.5, 1e-5, 600
TAU = 0.5 + np.sqrt(3.0 / 16.0)
LBM_PHASES = 1 | 2 | 4 | 8 | 16 | 32   # flag, links, refill, bulk, boundary, swap: no rigid-body update


def _hasimoto_K(c):
    s = c ** (1.0 / 3.0)
    return 1.0 / (1.0 - 1.7601 * s + c - 1.5593 * c * c + 3.9799 * s ** 8 - 3.0734 * s ** 10)


def test_stokes_drag_gpu_matches_limit_and_oracle():
    B = binding()
    shape = (L, L, L)
    pos = np.array([12.3, 11.8, 12.1])
    quat = np.array([1.0, 0.0, 0.0, 0.0])
    P = {"centers": np.zeros((1, 3)), "k": np.array([R * R]), "pos": pos, "quat": quat,
         "vel": np.zeros(3), "omega": np.zeros(3)}
    owner = metaball.flag_nodes(shape, [P])
    fluid = owner < 0
    n_fl = int(fluid.sum())
    mu = (TAU - 0.5) / 3.0
    c = 4.0 / 3.0 * np.pi * R ** 3 / L ** 3
    stokes = 6.0 * np.pi * mu * R * _hasimoto_K(c)
    u0 = np.zeros((3, L, L, L))
    u0[0] = G * L ** 3 / stokes
    f0 = lbm.equilibrium(np.ones((L, L, L)), u0).astype(np.float32)
    ex = E[:, 0].astype(float)

    sim = B.Simulation(L, L, L, tau=TAU, periodic=(True, True, True), fluid_body_force=(G, 0.0, 0.0),
                       bb_mode=B.BB_IBB)
    sim.add_particle(P["centers"], P["k"], 2.5, 1.0, pos, quat)
    sim.step_phases(1)
    sim.set_populations(f0)
    mom_prev = np.einsum("i,in->", ex, f0[:, fluid].astype(np.float64))
    for s in range(STEPS):
        sim.step_phases(LBM_PHASES)
        if s < 3 or s == STEPS - 1:
            f = sim.get_populations().astype(np.float64)
            mom = np.einsum("i,in->", ex, f[:, fluid])
            F = sim.forces()["F_hydro"][0]
            if s < 3:
                # FP32 storage of ~2.5e5 populations near 0.05: ~1e-4 of the per-step gain
                assert abs((mom - mom_prev) - (G * n_fl - F[0])) < 1e-3 * G * n_fl
            mom_prev = mom
    _, own = sim.node_classes()
    own = own.astype(np.int64)
    own[own == 0xFFFFFFFF] = -1
    assert np.array_equal(own, owner)
    U = (mom - 0.5 * G * n_fl) / L ** 3
    ratio_gpu = F[0] / (U * stokes)
    assert abs(ratio_gpu - 1.0) < 0.06, ratio_gpu
    assert np.abs(F[1:]).max() < 2e-3 * F[0]

    fo = f0.astype(np.float64)
    fo[:, ~fluid] = np.nan
    for _ in range(STEPS):
        fo, Fo, _ = coupling.coupled_lbm_step(fo, owner, owner, [P], TAU, periodic=(True, True, True),
                                              force=(G, 0.0, 0.0))
    Uo = (np.einsum("i,in->", ex, fo[:, fluid]) - 0.5 * G * n_fl) / L ** 3
    ratio_oracle = Fo[0, 0] / (Uo * stokes)
    assert abs(ratio_gpu - ratio_oracle) < 1e-3, (ratio_gpu, ratio_oracle)
    assert F[0] == pytest.approx(Fo[0, 0], rel=2e-3)
