"""Pins of the oracle's whole coupled step (flag -> coupled LBM step -> DEM
substeps with the hydrodynamic force held): without particles it is the
bulk step; a particle at rest in fluid at rest feels no hydrodynamic force,
leaves the fluid unchanged, and its n substeps of the rigid-body update give
the closed form of n semi-implicit Euler steps under gravity and buoyancy."""
import numpy as np
import pytest

from oracle import lbm, metaball, step
from oracle.d3q19 import Q, W


@pytest.mark.parametrize("periodic", [(False, False, False), (True, False, True)])
def test_particle_free_step_is_the_bulk_step(periodic):
    shape = (12, 10, 9)
    rng = np.random.default_rng(3)
    f0 = W.reshape(Q, 1, 1, 1) * (1.0 + 0.05 * rng.standard_normal((Q, 9, 10, 12)))
    wv = np.zeros((6, 3))
    wv[3] = (0.02, 0.0, -0.01)
    S = step.OracleState(shape, f0, [], tau=0.7, periodic=periodic, wall_velocity=wv)
    step.step(S)
    ref = lbm.step_bulk(f0, 0.7, periodic=periodic, wall_velocity=wv)
    assert np.array_equal(S.f, ref)


@pytest.mark.parametrize("n_sub", [1, 4])
def test_resting_particle_substeps_closed_form(n_sub):
    shape = (20, 20, 20)
    c = np.array([[-0.8, 0.1, 0.0], [0.8, -0.1, 0.2]])
    k = np.array([4.0, 3.0])
    mp = metaball.mass_properties(c, k, 2.5, h=0.2)
    c = c - mp["centroid"]
    mp = metaball.mass_properties(c, k, 2.5, h=0.2)
    X = np.array([10.0, 9.7, 10.2])
    P = {"centers": c, "k": k, "pos": X, "quat": np.array([0.9, 0.1, -0.3, 0.2]) / np.linalg.norm([0.9, 0.1, -0.3, 0.2]),
         "vel": np.zeros(3), "omega": np.zeros(3), "skin": 0.5, "mass": mp["mass"], "volume": mp["volume"],
         "inertia": mp["inertia"]}
    g = np.array([0.0, 0.0, -1e-4])
    f0 = lbm.rest_state(shape)
    S = step.OracleState(shape, f0, [P], tau=0.8, gravity=g, dem_substeps=n_sub)
    step.step(S)
    owner = metaball.flag_nodes(shape, [P])
    fl = owner < 0
    assert np.abs(S.F_hydro).max() < 1e-13 and np.abs(S.T_hydro).max() < 1e-12
    assert np.abs(S.f[:, fl] - f0[:, fl]).max() < 1e-16
    assert len(S.contacts) == 0          # no wall within reach, no other particle
    a = (1.0 - P["volume"] / P["mass"]) * g
    Pn = S.particles[0]
    assert np.allclose(Pn["vel"], a, rtol=0, atol=1e-15)
    assert np.allclose(Pn["pos"], X + a * (n_sub + 1) / (2.0 * n_sub), rtol=0, atol=1e-14)
    assert np.allclose(Pn["quat"], P["quat"], rtol=0, atol=1e-15)
    assert np.abs(Pn["omega"]).max() < 1e-15


def test_cover_uncover_start_covers_nothing():
    """With the cover/uncover option the particles are not inserted into the
    fluid: the first step of a resting particle in moving fluid has the same
    hydrodynamic force as without the option."""
    shape = (16, 16, 16)
    P = {"centers": np.zeros((1, 3)), "k": np.array([6.0]), "pos": np.array([8.2, 7.9, 8.1]),
         "quat": np.array([1.0, 0.0, 0.0, 0.0]), "vel": np.zeros(3), "omega": np.zeros(3), "skin": 0.5,
         "mass": 100.0, "volume": 40.0, "inertia": np.eye(3) * 200.0}
    u = np.zeros((3, 16, 16, 16))
    u[0] = 0.02
    f0 = lbm.equilibrium(np.ones((16, 16, 16)), u)
    a = step.OracleState(shape, f0, [P], periodic=(True, True, True))
    b = step.OracleState(shape, f0, [P], periodic=(True, True, True), cover_uncover=True)
    step.step(a)
    step.step(b)
    assert np.abs(a.F_hydro).max() > 1e-3
    assert np.array_equal(a.F_hydro, b.F_hydro) and np.array_equal(a.T_hydro, b.T_hydro)
