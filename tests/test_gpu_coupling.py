"""GPU parity of the particle phases (flagging, links, refill, IBB, momentum
exchange, rigid-body update) against the FP64 oracle, through the C-ABI, on
small particles (1-4 control points); tests/test_gpu_parity_scale.py runs the
same comparison on the benchmarks' particle sizes.

Bars (tests/coupling_parity.py): node owners, node classes and the link set
bit-exact; wall fraction q within 1e-5 (FP32 root of an FP32 field whose
body-frame point carries ~1e-6 absolute rounding); populations at fluid nodes
within 1e-5 relative; hydrodynamic force and torque within
1e-4 * max(|F_ref|, 1e-3 * sum_links |dP|) per particle (the link-sum scale
guards the cancellation of O(0.1) link terms into a small net force).
"""
import numpy as np
import pytest

from oracle import coupling, dem, lbm, metaball
from oracle.d3q19 import E, W
from paper_2209_10411_gb300 import scenes
from tests import coupling_parity as cp
from tests.gpu_helpers import binding

pytestmark = pytest.mark.gpu

TAU = cp.TAU
_prepared = cp.prepared
_initial_flow = cp.initial_flow
_run_one_step = cp.run_one_step
_compare_step = cp.compare_step


@pytest.mark.parametrize("mode", ["ibb", "ladd"])
def test_one_step_moving_particle(mode):
    B = binding()
    shape = (40, 36, 44)
    rng = np.random.default_rng(7)
    c, k, _ = scenes.blob_4(rng)
    spec = scenes.ParticleSpec(c, k, 2.5, 1.0, None, None)
    q0 = scenes.random_unit_quaternion(rng)
    X = np.array([20.3, 17.6, 22.1])
    dX = np.array([0.7, 0.35, -0.2])
    P = _prepared(spec, X, q0, (0.02, -0.01, 0.015), (0.004, -0.003, 0.002))
    Pp = dict(P, pos=X - dX, quat=scenes.f32(q0 + np.array([0.0, 0.05, -0.03, 0.02])))
    f0 = _initial_flow(shape, seed=3)
    sim = _run_one_step(B, shape, [Pp], [P], f0, mode)
    owner_prev = metaball.flag_nodes(shape, [Pp])
    owner = metaball.flag_nodes(shape, [P])
    assert coupling.classify(owner, owner_prev)[1].sum() > 10  # uncovered nodes are exercised
    _compare_step(sim, shape, [Pp], [P], f0, mode)
    sim.close()


@pytest.mark.parametrize("mode", ["ibb", "ladd"])
def test_cover_uncover_rule(mode):
    """The optional cover/uncover momentum (Lorenz et al. 2009): one step of a
    particle that moves 0.8 lu; force and torque against the oracle's with
    the rule, at the same bar as the plain exchange, the rule's share of the
    force well above that bar, and the populations unchanged by it."""
    B = binding()
    shape = (40, 36, 44)
    rng = np.random.default_rng(7)
    c, k, _ = scenes.blob_4(rng)
    spec = scenes.ParticleSpec(c, k, 2.5, 1.0, None, None)
    q0 = scenes.random_unit_quaternion(rng)
    X = np.array([20.3, 17.6, 22.1])
    dX = np.array([0.7, 0.35, -0.2])
    P = _prepared(spec, X, q0, (0.02, -0.01, 0.015), (0.004, -0.003, 0.002))
    Pp = dict(P, pos=X - dX, quat=scenes.f32(q0 + np.array([0.0, 0.05, -0.03, 0.02])))
    f0 = _initial_flow(shape, seed=3)
    sim = _run_one_step(B, shape, [Pp], [P], f0, mode, cover_uncover=True)
    owner_prev = metaball.flag_nodes(shape, [Pp])
    owner = metaball.flag_nodes(shape, [P])
    assert ((owner >= 0) & (owner_prev < 0)).sum() > 10 and coupling.classify(owner, owner_prev)[1].sum() > 10
    ref, F, T, L = coupling.coupled_lbm_step(f0, owner, owner_prev, [P], TAU, bb_mode=mode, return_links=True,
                                             cover_uncover=True)
    _, F0, T0 = coupling.coupled_lbm_step(f0, owner, owner_prev, [P], TAU, bb_mode=mode)
    got = sim.get_populations().astype(np.float64)
    fl = owner < 0
    assert (np.abs(got[:, fl] - ref[:, fl]) / np.abs(ref[:, fl])).max() < 1e-5
    fr = sim.forces()
    qw = np.full(len(L["q"]), 0.5) if mode == "ladd" else L["q"]
    arm = L["cell"] + qw[:, None] * E[L["dir"]] - X
    scaleF = max(np.linalg.norm(F[0]), 1e-3 * np.abs(L["dP"]).sum())
    scaleT = max(np.linalg.norm(T[0]), 1e-3 * np.abs(np.cross(arm, L["dP"])).sum())
    assert np.linalg.norm(F[0] - F0[0]) > 10 * 1e-4 * scaleF        # the rule is exercised
    assert np.linalg.norm(fr["F_hydro"][0] - F[0]) <= 1e-4 * scaleF, (fr["F_hydro"][0], F[0])
    assert np.linalg.norm(fr["T_hydro"][0] - T[0]) <= 1e-4 * scaleT, (fr["T_hydro"][0], T[0])
    sim.close()


def test_one_step_two_particles_overlapping_boxes():
    B = binding()
    shape = (48, 40, 38)
    rng = np.random.default_rng(11)
    parts, prev = [], []
    for j, X in enumerate([np.array([17.2, 20.4, 19.1]), np.array([30.6, 19.3, 18.7])]):
        c, k, _ = scenes.blob_4(rng)
        spec = scenes.ParticleSpec(c, k, 2.5, 1.0, None, None)
        q = scenes.random_unit_quaternion(rng)
        v = rng.uniform(-0.02, 0.02, 3)
        w = rng.uniform(-0.005, 0.005, 3)
        P = _prepared(spec, X, q, v, w)
        parts.append(P)
        prev.append(dict(P, pos=X - np.array([0.4, -0.6, 0.5])))
    f0 = _initial_flow(shape, seed=4)
    sim = _run_one_step(B, shape, prev, parts, f0, "ibb")
    _compare_step(sim, shape, prev, parts, f0, "ibb")
    sim.close()


@pytest.mark.parametrize("mode", ["ibb", "ladd"])
def test_link_sums_without_block_partials(mode):
    """A handle sized for more than 1000 particles sums the links' momentum
    exchange with global 64-bit atomics instead of per-block shared-memory
    sums: the oracle's bars hold, and since the fixed-point sums do not depend
    on their order, forces, torques and populations equal the default path's
    bit for bit."""
    B = binding()
    shape = (48, 40, 38)
    rng = np.random.default_rng(12)
    parts, prev = [], []
    for X in (np.array([17.2, 20.4, 19.1]), np.array([30.6, 19.3, 18.7])):
        c, k, _ = scenes.blob_4(rng)
        spec = scenes.ParticleSpec(c, k, 2.5, 1.0, None, None)
        P = _prepared(spec, X, scenes.random_unit_quaternion(rng), rng.uniform(-0.02, 0.02, 3),
                      rng.uniform(-0.005, 0.005, 3))
        parts.append(P)
        prev.append(dict(P, pos=X - np.array([0.4, -0.6, 0.5])))
    f0 = _initial_flow(shape, seed=6)
    out = []
    for cap in (None, 1001):
        sim = _run_one_step(B, shape, prev, parts, f0, mode, max_particles=cap)
        if cap:
            _compare_step(sim, shape, prev, parts, f0, mode)
        out.append((sim.forces(), sim.get_populations()))
        sim.close()
    (fa, pa), (fb, pb) = out
    for key in ("F_hydro", "T_hydro"):
        assert np.array_equal(fa[key], fb[key]), key
    assert np.array_equal(pa, pb)


def test_rigid_body_update_after_step():
    B = binding()
    shape = (36, 34, 40)
    rng = np.random.default_rng(12)
    c, k, _ = scenes.blob_4(rng)
    spec = scenes.ParticleSpec(c, k, 2.5, 1.0, None, None)
    P = _prepared(spec, np.array([17.5, 16.2, 20.3]), scenes.random_unit_quaternion(rng),
                  (0.01, 0.0, -0.02), (0.002, 0.003, -0.001))
    f0 = _initial_flow(shape, seed=5)
    g = (0.0, 0.0, -1e-4)
    sim = B.Simulation(*shape, tau=TAU, gravity=g)
    sim.add_particle(P["centers"], P["k"], P["density"], P["skin"], P["pos"], P["quat"], P["vel"], P["omega"],
                     mass_props={"mass": P["mass"], "volume": P["volume"], "inertia": P["inertia"]})
    sim.set_populations(f0.astype(np.float32))
    sim.step(1)
    st = sim.get_particle_state(0)
    owner = metaball.flag_nodes(shape, [P])
    _, F, T = coupling.coupled_lbm_step(f0, owner, owner, [P], TAU)
    ref = dem.integrate(P, F[0], T[0], g)
    dv_ref = ref["vel"] - P["vel"]
    dv = st["vel"] - P["vel"]
    assert np.linalg.norm(dv - dv_ref) <= 1e-4 * np.linalg.norm(dv_ref) + 1e-12
    assert np.linalg.norm(st["pos"] - ref["pos"]) <= 1e-4 * np.linalg.norm(dv_ref) + 1e-12
    dw_ref = ref["omega"] - P["omega"]
    assert np.linalg.norm(st["omega"] - ref["omega"]) <= 1e-3 * np.linalg.norm(dw_ref) + 1e-10
    assert np.abs(np.abs(st["quat"] @ ref["quat"]) - 1.0) < 1e-12
    sim.close()


def test_short_trajectory_config1():
    """64^3 closed box, one 4-ball particle, density 2.5, gravity 1e-5 (the
    oracle-size settling case): 12 coupled steps, trajectory and forces vs the
    oracle."""
    B = binding()
    sc = scenes.config1()
    spec = sc.particles[0]
    P = _prepared(spec, spec.pos, spec.quat, (0, 0, 0), (0, 0, 0))
    shape = sc.shape
    nsteps = 12
    sim = B.Simulation(*shape, tau=sc.tau, gravity=sc.gravity)
    sim.add_particle(P["centers"], P["k"], P["density"], P["skin"], P["pos"], P["quat"], P["vel"], P["omega"],
                     mass_props={"mass": P["mass"], "volume": P["volume"], "inertia": P["inertia"]})
    f = lbm.rest_state((shape[2], shape[1], shape[0]))
    state = dict(P)
    owner_prev = metaball.flag_nodes(shape, [state])
    for n in range(nsteps):
        sim.step(1)
        fr = sim.forces()
        owner = metaball.flag_nodes(shape, [state])
        f, F, T = coupling.coupled_lbm_step(f, owner, owner_prev, [state], sc.tau)
        owner_prev = owner
        scale = max(np.linalg.norm(F[0]), 1e-9)
        assert np.linalg.norm(fr["F_hydro"][0] - F[0]) <= 1e-3 * scale + 1e-9, (n, fr["F_hydro"][0], F[0])
        state = dem.integrate(state, F[0], T[0], sc.gravity)
        st = sim.get_particle_state(0)
        assert np.linalg.norm(st["pos"] - state["pos"]) < 1e-7
        assert np.linalg.norm(st["vel"] - state["vel"]) < 1e-3 * np.linalg.norm(state["vel"]) + 1e-12
    got = sim.get_populations().astype(np.float64)
    fl = metaball.flag_nodes(shape, [state]) < 0
    fl = fl & np.isfinite(f).all(0)
    rel = np.abs(got[:, fl] - f[:, fl]) / np.abs(f[:, fl])
    assert rel.max() < 1e-4
    sim.close()


def test_mass_properties_quadrature_matches_oracle():
    B = binding()
    rng = np.random.default_rng(13)
    c, k, _ = scenes.blob_4(rng)
    X = np.array([20.0, 21.0, 22.0])
    q = scenes.random_unit_quaternion(rng)
    sim = B.Simulation(48, 48, 48, tau=TAU)
    sim.add_particle(c, k, 2.5, 1.0, X, q)
    sh = sim.get_particle_shape(0)
    st = sim.get_particle_state(0)
    mp = metaball.mass_properties(c, k, 2.5)
    assert abs(sh["volume"] - mp["volume"]) <= 1e-9 * mp["volume"]
    assert np.allclose(sh["inertia"], mp["inertia"], rtol=1e-8, atol=1e-8 * np.abs(mp["inertia"]).max())
    assert np.allclose(sh["centers"], c - mp["centroid"], atol=1e-9)
    R = metaball.quat_to_matrix(q)
    assert np.allclose(st["pos"], X + R @ mp["centroid"], atol=1e-9)
    sim.close()


@pytest.mark.parametrize("omega", [(0.01, -0.004, 0.002), (0.3, -0.2, 0.1), (0.0, 0.0, 0.0)])
def test_integrate_rotation_small_and_large_angles(omega):
    """The rigid-body update alone (no hydrodynamic or contact force): the
    half rotation angle |omega| dt / 2 below 1/64 takes the series branch,
    above it the library sin/cos; orientation, angular velocity and position
    against the oracle's update."""
    B = binding()
    rng = np.random.default_rng(21)
    c, k, _ = scenes.blob_4(rng)
    spec = scenes.ParticleSpec(c, k, 2.5, 1.0, None, None)
    P = _prepared(spec, np.array([16.0, 15.5, 17.25]), scenes.random_unit_quaternion(rng), (0.01, -0.02, 0.005),
                  omega)
    g = (0.0, 0.0, -1e-4)
    with B.Simulation(32, 32, 32, tau=TAU, gravity=g) as sim:
        sim.add_particle(P["centers"], P["k"], P["density"], P["skin"], P["pos"], P["quat"], P["vel"], P["omega"],
                         mass_props={"mass": P["mass"], "volume": P["volume"], "inertia": P["inertia"]})
        state = dict(P)
        for _ in range(3):
            sim.step_phases(B.PHASE_INTEGRATE)
            state = dem.integrate(state, np.zeros(3), np.zeros(3), g)
        st = sim.get_particle_state(0)
    assert np.abs(np.abs(st["quat"] @ state["quat"]) - 1.0) < 1e-14
    assert np.linalg.norm(st["quat"] - state["quat"]) < 1e-13
    assert np.linalg.norm(st["omega"] - state["omega"]) <= 1e-13 * max(np.linalg.norm(omega), 1.0)
    assert np.linalg.norm(st["pos"] - state["pos"]) < 1e-12
    assert np.linalg.norm(st["vel"] - state["vel"]) < 1e-15
