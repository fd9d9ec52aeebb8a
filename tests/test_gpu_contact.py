"""GPU parity of the DEM contact phase (broad phase, Newton closest points for
pairs and walls, spring-dashpot forces, DEM substeps) against the FP64
oracle, through the C-ABI.

Bars: candidate pair/wall lists bit-exact; contact point and overlap within
1e-5 of the particle size (the bounding diameter 2 R_b) -- the GPU solves in
FP32 in a frame centred between the particles and stops Newton at
|dx| <= 1e-5 R_b; normal within 1e-5; contact force and torque within 1e-4
relative (plus the same absolute slack propagated through k_n)."""
import numpy as np
import pytest

from oracle import contact, dem, metaball, step as ostep
from paper_2209_10411_gb300 import scenes
from tests.gpu_helpers import binding

pytestmark = pytest.mark.gpu

PARAMS = {"kn": 0.5, "kt": 0.15, "eta_n": 0.05, "eta_t": 0.02, "mu_s": 0.4}


def _particle(c, k, pos, quat, vel=(0, 0, 0), omega=(0, 0, 0), skin=0.6, density=2.5):
    c = np.asarray(c, dtype=float).reshape(-1, 3)
    k = np.asarray(k, dtype=float)
    mp = metaball.mass_properties(c, k, density)
    return {"centers": c - mp["centroid"], "k": k, "pos": np.asarray(pos, float), "quat": np.asarray(quat, float),
            "vel": np.asarray(vel, float), "omega": np.asarray(omega, float), "skin": skin, "density": density,
            "mass": mp["mass"], "volume": mp["volume"], "inertia": mp["inertia"]}


def _sim(B, shape, parts, periodic=(False, False, False), dem_substeps=1, **kw):
    sim = B.Simulation(*shape, tau=0.8, periodic=periodic, dem_substeps=dem_substeps, kn=PARAMS["kn"],
                       kt=PARAMS["kt"], eta_n=PARAMS["eta_n"], eta_t=PARAMS["eta_t"], mu_s=PARAMS["mu_s"],
                       max_particles=64, **kw)
    for P in parts:
        sim.add_particle(P["centers"], P["k"], P["density"], P["skin"], P["pos"], P["quat"], P["vel"], P["omega"],
                         mass_props={"mass": P["mass"], "volume": P["volume"], "inertia": P["inertia"]})
    return sim


def _compact(rng):
    """Three balls uniform in a 1.5-lu ball, k ~ U[3, 6]: a particle of radius ~3.5."""
    c = scenes.uniform_in_ball(rng, 3, 1.5)
    return scenes.f32(c), scenes.f32(rng.uniform(3.0, 6.0, 3))


def _cluster(seed, n=5, spacing=7.0):
    rng = np.random.default_rng(seed)
    parts = []
    base = np.array([20.0, 20.0, 3.6])
    offsets = [np.zeros(3), np.array([spacing, 0.3, 0.2]), np.array([0.2, spacing, -0.1]),
               np.array([spacing, spacing, 0.3]), np.array([0.5 * spacing, 0.5 * spacing, 5.5])][:n]
    for o in offsets:
        c, k = _compact(rng)
        parts.append(_particle(c, k, base + o, scenes.random_unit_quaternion(rng),
                               vel=rng.uniform(-0.01, 0.01, 3), omega=rng.uniform(-0.002, 0.002, 3)))
    return parts


def _key(c):
    return (c["i"], c["j"])


def _compare_contacts(gpu, ref, parts):
    g = {_key(c): c for c in gpu}
    r = {_key(c): c for c in ref}
    assert set(g) == set(r), (sorted(set(g) ^ set(r)))
    for key, rc in r.items():
        gc = g[key]
        i = key[0]
        size = 2 * max(metaball.bounding_radius(parts[i]["centers"], parts[i]["k"]),
                       metaball.bounding_radius(parts[key[1]]["centers"], parts[key[1]]["k"]) if key[1] >= 0 else 0)
        if rc["status"] != contact.OK:
            continue
        assert gc["status"] == contact.OK, key
        assert abs(gc["delta"] - rc["delta"]) <= 1e-5 * size, (key, gc["delta"], rc["delta"])
        assert np.linalg.norm(gc["x_cp"] - rc["x_cp"]) <= 1e-5 * size, (key, gc["x_cp"], rc["x_cp"])
        assert np.linalg.norm(gc["n"] - rc["n"]) <= 1e-5, key


def test_two_spheres_and_walls():
    B = binding()
    shape = (40, 40, 40)
    P0 = _particle([[0, 0, 0]], [16.0], [12.0, 20.0, 3.2], (1, 0, 0, 0), vel=(0.01, 0, -0.005), skin=0.7)
    P1 = _particle([[0, 0, 0]], [9.0], [18.3, 20.4, 4.3], (1, 0, 0, 0), vel=(-0.01, 0.002, 0), skin=0.5)
    parts = [P0, P1]
    sim = _sim(B, shape, parts)
    sim.step_phases(B.PHASE_CONTACT)
    gpu = sim.contacts()
    F, T, hist, ref = contact.contact_forces(parts, shape, (False, False, False), PARAMS, {}, 1.0)
    _compare_contacts(gpu, ref, parts)
    assert sum(1 for c in ref if c["status"] == contact.OK and c["delta"] > 0) >= 2
    fr = sim.forces()
    scale = np.abs(F).max()
    assert np.abs(fr["F_contact"] - F).max() <= 1e-4 * scale
    assert np.abs(fr["T_contact"] - T).max() <= 1e-4 * max(np.abs(T).max(), scale)
    sim.close()


def test_metaball_cluster_contacts():
    B = binding()
    shape = (48, 48, 40)
    for seed in (1, 2, 3):
        parts = _cluster(seed)
        sim = _sim(B, shape, parts)
        sim.step_phases(B.PHASE_CONTACT)
        gpu = sim.contacts()
        F, T, hist, ref = contact.contact_forces(parts, shape, (False, False, False), PARAMS, {}, 1.0)
        _compare_contacts(gpu, ref, parts)
        fr = sim.forces()
        scale = max(np.abs(F).max(), 1e-12)
        assert np.abs(fr["F_contact"] - F).max() <= 2e-4 * scale + 1e-12
        sim.close()


def test_dem_substeps_trajectory_without_fluid():
    """Contacts + rigid-body update only (no lattice phases), 4 substeps per
    step, 10 steps: springs carried over between substeps."""
    B = binding()
    shape = (48, 48, 40)
    parts = _cluster(4)
    parts[1]["vel"] = np.array([-0.05, 0.0, 0.0])
    nsub = 4
    sim = _sim(B, shape, parts, dem_substeps=nsub, gravity=(0, 0, -1e-4))
    hist = {}
    state = [dict(P) for P in parts]
    for n in range(10):
        sim.step_phases(B.PHASE_CONTACT | B.PHASE_INTEGRATE)
        for _ in range(nsub):
            F, T, hist, ref = contact.contact_forces(state, shape, (False,) * 3, PARAMS, hist, 1.0 / nsub)
            state = [dem.integrate(P, F[i], T[i], (0, 0, -1e-4), dt=1.0 / nsub) for i, P in enumerate(state)]
    for i, P in enumerate(state):
        st = sim.get_particle_state(i)
        assert np.linalg.norm(st["pos"] - P["pos"]) < 1e-5, (i, st["pos"], P["pos"])
        assert np.linalg.norm(st["vel"] - P["vel"]) < 1e-6, (i, st["vel"], P["vel"])
    sim.close()


def test_full_coupled_step_with_contacts():
    """Every phase of one step (flag, links, refill, LBM, boundary, contacts,
    rigid-body update) on a small tank with touching particles."""
    B = binding()
    shape = (48, 48, 40)
    parts = _cluster(5, n=4)
    sim = _sim(B, shape, parts, gravity=(0, 0, -1e-5))
    S = ostep.OracleState(shape, np.broadcast_to(np.array(
        [1 / 3] + [1 / 18] * 6 + [1 / 36] * 12).reshape(19, 1, 1, 1), (19, 40, 48, 48)).copy(), parts,
        gravity=(0, 0, -1e-5), contact_params=PARAMS)
    for n in range(3):
        sim.step(1)
        ostep.step(S)
        fr = sim.forces()
        for i in range(len(parts)):
            sF = max(np.linalg.norm(S.F_hydro[i]), 1e-7)
            assert np.linalg.norm(fr["F_hydro"][i] - S.F_hydro[i]) <= 1e-3 * sF + 1e-9
            sC = max(np.abs(S.F_contact).max(), 1e-12)
            assert np.linalg.norm(fr["F_contact"][i] - S.F_contact[i]) <= 2e-4 * sC + 1e-12
            st = sim.get_particle_state(i)
            assert np.linalg.norm(st["pos"] - S.particles[i]["pos"]) < 1e-6
    sim.close()


def test_add_particle_overlap_check():
    """With check_overlap, a particle whose core overlaps an existing one is
    rejected with MI_EOVERLAP (decided by the closest-point solve: the
    converged point lies inside a core) and nothing is added; a particle in
    skin contact only is accepted; without the check both are accepted."""
    B = binding()
    a = _particle([[-1, 0, 0], [1, 0, 0]], [3, 3], (13.0, 14.0, 14.0), (0.9, 0.1, 0.2, 0.1))
    overlapping = _particle([[0, 0, 0], [0.8, 0.3, 0]], [4, 2], (17.0, 14.3, 14.2), (0.8, 0.3, 0.1, 0.4))
    touching = _particle([[0, 0, 0], [0.8, 0.3, 0]], [4, 2], (17.8, 14.3, 14.2), (0.8, 0.3, 0.1, 0.4))
    assert contact.newton_pair(a, overlapping)["status"] == contact.INSIDE
    r = contact.newton_pair(a, touching)
    assert r["status"] == contact.OK and r["delta"] > 0

    def add(sim, P):
        sim.add_particle(P["centers"], P["k"], P["density"], P["skin"], P["pos"], P["quat"],
                         mass_props={"mass": P["mass"], "volume": P["volume"], "inertia": P["inertia"]})

    with B.Simulation(32, 28, 30, check_overlap=True, max_particles=8) as sim:
        add(sim, a)
        with pytest.raises(B.MiDelbmError) as ei:
            add(sim, overlapping)
        assert ei.value.status == B.MI_EOVERLAP
        assert sim.num_particles() == 1
        add(sim, touching)
        assert sim.num_particles() == 2
        sim.step(1)  # the rejected particle left nothing behind
        assert np.isfinite(sim.forces()["F_contact"]).all()
    with B.Simulation(32, 28, 30, max_particles=8) as sim:
        add(sim, a)
        add(sim, overlapping)
        assert sim.num_particles() == 2


def test_warm_guess_same_contacts_fewer_iterations():
    """MI_GUESS_WARM starts each pair's Newton solve at the pair's closest point
    of the previous DEM substep: over 8 substeps per step the cluster gets the
    same contacts, points and forces as with the plain guess (to the
    convergence tolerance) in fewer iterations."""
    B = binding()
    parts = _cluster(5)
    for P in parts:
        P["vel"] = P["vel"] * 10.0
    res = {}
    for mode in (B.GUESS_PLAIN, B.GUESS_WARM):
        sim = _sim(B, (48, 48, 40), parts, dem_substeps=8, guess_mode=mode)
        sim.step(2)
        recs = sorted(sim.contacts(), key=_key)
        res[mode] = (recs, sim.forces(), [sim.get_particle_state(i) for i in range(len(parts))])
        sim.close()
    (rp, fp, sp), (rw, fw, sw) = res[B.GUESS_PLAIN], res[B.GUESS_WARM]
    assert [_key(c) for c in rp] == [_key(c) for c in rw]
    pairs_p = [c for c in rp if c["j"] >= 0 and c["status"] == 0]
    pairs_w = [c for c in rw if c["j"] >= 0 and c["status"] == 0]
    assert len(pairs_p) == len(pairs_w) > 0
    for a, b in zip(pairs_p, pairs_w):
        assert np.linalg.norm(a["x_cp"] - b["x_cp"]) <= 1e-4, (a, b)
    scale = np.abs(fp["F_contact"]).max()
    assert np.abs(fp["F_contact"] - fw["F_contact"]).max() <= 1e-3 * scale + 1e-9
    it_p = np.mean([c["iters"] for c in pairs_p])
    it_w = np.mean([c["iters"] for c in pairs_w])
    assert it_w < it_p, (it_w, it_p)


def _dem_snapshot(sim, n):
    states = [sim.get_particle_state(i) for i in range(n)]
    key = lambda c: (c["i"], c["j"])
    recs = sorted(sim.contacts(), key=key)
    return states, recs, sim.forces()


def _assert_same_bits(a, b):
    (sa, ra, fa), (sb, rb, fb) = a, b
    for x, y in zip(sa, sb):
        for f in ("pos", "quat", "vel", "omega"):
            assert np.array_equal(x[f], y[f]), f
    assert [(c["i"], c["j"]) for c in ra] == [(c["i"], c["j"]) for c in rb]
    for x, y in zip(ra, rb):
        assert np.array_equal(x["x_cp"], y["x_cp"]) and np.array_equal(x["n"], y["n"])
        assert x["delta"] == y["delta"] and x["iters"] == y["iters"] and x["status"] == y["status"]
    for f in fa:
        assert np.array_equal(fa[f], fb[f]), f


@pytest.mark.parametrize("warm", [False, True])
def test_fused_dem_substeps_equal_per_substep_launches(warm):
    """The fused substep kernel (one CTA runs every substep of a step) against
    one launch sequence per substep: the same bits for the particle states,
    the contact records and the force sums after six steps of eight
    substeps, with the plain and with the warm start."""
    B = binding()
    shape = (48, 48, 40)
    parts = _cluster(5)
    parts[1]["vel"] = np.array([-0.05, 0.0, 0.0])
    parts[3]["vel"] = np.array([0.0, -0.04, 0.01])
    snaps = []
    for unfused in (False, True):
        sim = _sim(B, shape, parts, dem_substeps=8, gravity=(0, 0, -1e-4),
                   guess_mode=B.GUESS_WARM if warm else B.GUESS_PLAIN)
        sim.set_schedule(unfused_dem=unfused)
        for _ in range(6):
            sim.step_phases(B.PHASE_CONTACT | B.PHASE_INTEGRATE)
        snaps.append(_dem_snapshot(sim, len(parts)))
        sim.close()
    assert any(c["status"] == 0 and c["delta"] > 0 for c in snaps[0][1])
    _assert_same_bits(*snaps)


def test_fused_dem_substeps_in_coupled_steps():
    """Whole coupled steps (graph replay) of two particles in contact with
    five DEM substeps per step: fused and per-substep schedules give the same
    particle states, contacts, forces and populations."""
    B = binding()
    shape = (32, 28, 30)
    parts = [_particle([[-1, 0, 0], [1, 0, 0]], [3, 3], [13.0, 14.0, 14.0], (0.9, 0.1, 0.2, 0.1),
                       (0.004, 0.0, 0.001), (0.0, 0.002, 0.0)),
             _particle([[0, 0, 0], [0.8, 0.3, 0]], [4, 2], [17.8, 14.3, 14.2], (0.8, 0.3, 0.1, 0.4),
                       (-0.003, 0.001, 0.0), (0.001, 0.0, -0.002))]
    for P in parts:
        P["quat"] = P["quat"] / np.linalg.norm(P["quat"])
    snaps, pops = [], []
    for unfused in (False, True):
        sim = _sim(B, shape, parts, dem_substeps=5, gravity=(0.0, 0.0, -1e-4))
        sim.set_schedule(unfused_dem=unfused)
        sim.step(4)
        snaps.append(_dem_snapshot(sim, len(parts)))
        pops.append(sim.get_populations())
        sim.close()
    _assert_same_bits(*snaps)
    assert np.array_equal(pops[0], pops[1])
