"""Failure handling through the C-ABI, with every fault made on the host or
by a device wait on a flag that nothing sets (no fault, trap or hang of the
GPU):

  * lists forced too small: the step reports MI_ECAPACITY with the sizes it
    needed, the handle grows its lists and captures its graphs again, and the
    repeated step gives the bits of a handle that had room from the start;
  * the learned guess's tcgen05 kernel made to wait on an mbarrier nothing
    arrives at, with a short limit: MI_ETIMEOUT, the contacts of its rows
    fall back to plain Newton (the same contacts as the plain start), and
    the next phase with the wait restored is clean;
  * a NaN or an infinity planted in an uploaded population field: the state
    check reports it at its node (FP32 and FP16 storage), and ignores solid
    nodes;
  * bad particle parameters: MI_EINVAL, and the handle stays usable.
"""
import numpy as np
import pytest

from oracle import mlp
from paper_2209_10411_gb300 import scenes
from tests import coupling_parity as cp
from tests.gpu_helpers import binding

pytestmark = pytest.mark.gpu


def _one_particle(shape=(40, 36, 44)):
    rng = np.random.default_rng(7)
    c, k, _ = scenes.blob_4(rng)
    spec = scenes.ParticleSpec(c, k, 2.5, 1.0, None, None)
    P = cp.prepared(spec, np.array([20.3, 17.6, 22.1]), scenes.random_unit_quaternion(rng), (0.02, -0.01, 0.015),
                    (0.004, -0.003, 0.002))
    return P, cp.initial_flow(shape, seed=3)


def _sim(B, shape, P, f0, graphs=True):
    sim = B.Simulation(*shape, tau=cp.TAU, gravity=(0.0, 0.0, -1e-4))
    cp.add_particles(sim, [P])
    sim.set_graphs(graphs)
    sim.set_populations(f0.astype(np.float32))
    return sim


@pytest.mark.parametrize("graphs", [True, False])
def test_list_overflow_reports_then_grows(graphs):
    B = binding()
    shape = (40, 36, 44)
    P, f0 = _one_particle(shape)
    ref = _sim(B, shape, P, f0, graphs)
    ref.step(1)
    Fr = ref.forces()
    fr = ref.get_populations()
    st_ref = ref.get_particle_state(0)
    ref.close()

    sim = _sim(B, shape, P, f0, graphs)
    sim.reserve_lists(16, 32, 4)
    sim.step(1)
    with pytest.raises(B.MiDelbmError) as ei:
        sim.forces()
    assert ei.value.status == B.MI_ECAPACITY
    stats = sim.stats()   # the full counts of the step that overflowed
    # the boundary-node list overflowed (nodes beyond it append no links, so
    # whether the link list did too depends on the order of the appends)
    assert stats["boundary_nodes"] > 16 and stats["links"] > 32 and (stats["status"] & 1)
    assert "boundary nodes %d/16" % stats["boundary_nodes"] in str(ei.value)
    # repeat the step from the same state: the lists grow first
    sim.set_populations(f0.astype(np.float32))
    sim.set_particle_state(0, P["pos"], P["quat"], P["vel"], P["omega"])
    sim.step(1)
    F = sim.forces()
    assert sim.stats()["status"] == 0
    assert np.array_equal(F["F_hydro"], Fr["F_hydro"]) and np.array_equal(F["T_hydro"], Fr["T_hydro"])
    assert np.array_equal(sim.get_populations(), fr)
    st = sim.get_particle_state(0)
    assert np.array_equal(st["pos"], st_ref["pos"]) and np.array_equal(st["vel"], st_ref["vel"])
    sim.close()


def _params(seed):
    import torch
    p = mlp.init_params(seed)
    flat = np.concatenate([p[k].ravel() for k in ("W1", "b1", "W2", "b2", "W3", "b3")]).astype(np.float32)
    return torch.as_tensor(flat, device="cuda")


def _contact_pair_sim(B, mode, params=None):
    """Two small particles whose skins overlap (the smoke check's pair)."""
    parts = []
    for c, k, pos, q in (([[-1, 0, 0], [1, 0, 0]], [3, 3], [13.0, 14.0, 14.0], (0.9, 0.1, 0.2, 0.1)),
                         ([[0, 0, 0], [0.8, 0.3, 0]], [4, 2], [17.8, 14.3, 14.2], (0.8, 0.3, 0.1, 0.4))):
        c = np.asarray(c, float)
        k = np.asarray(k, float)
        spec = scenes.ParticleSpec(c, k, 2.5, 0.6, None, None)
        qq = np.asarray(q, float)
        parts.append(cp.prepared(spec, np.asarray(pos), qq / np.linalg.norm(qq), (0, 0, 0), (0, 0, 0)))
    sim = B.Simulation(32, 28, 30, tau=cp.TAU, max_particles=4)
    for P in parts:
        sim.add_particle(P["centers"], P["k"], P["density"], 0.6, P["pos"], P["quat"],
                         mass_props={"mass": P["mass"], "volume": P["volume"], "inertia": P["inertia"]})
    if mode == "learned":
        sim.set_guess(B.GUESS_LEARNED, params)
    return sim


def test_learned_guess_wait_runs_out():
    B = binding()
    params = _params(3)
    plain = _contact_pair_sim(B, "plain")
    plain.step_phases(B.PHASE_CONTACT)
    ref = plain.contacts()
    plain.close()
    assert any(c["status"] == 0 and c["delta"] > 0 for c in ref)

    sim = _contact_pair_sim(B, "learned", params)
    sim.set_guess_wait(4096, stall=True)       # a wait on a barrier nothing arrives at
    sim.step_phases(B.PHASE_CONTACT)
    with pytest.raises(B.MiDelbmError) as ei:
        sim.contacts()
    assert ei.value.status == B.MI_ETIMEOUT and "NaN" in str(ei.value)
    assert sim.stats()["status"] & 64          # the timeout bit (cleared by this read)
    sim.set_guess_wait(0, stall=False)
    sim.step_phases(B.PHASE_CONTACT)
    got = sim.contacts()                       # clean again (no MI_ETIMEOUT)
    assert sim.stats()["status"] == 0
    sim.close()
    assert sorted((c["i"], c["j"]) for c in got) == sorted((c["i"], c["j"]) for c in ref)


def test_timed_out_rows_fall_back_to_plain_newton():
    """While the wait runs out, every learned row is NaN, so each contact is
    solved from the plain guess: the same points as the plain start."""
    B = binding()
    params = _params(4)
    plain = _contact_pair_sim(B, "plain")
    plain.step_phases(B.PHASE_CONTACT)
    ref = plain.contacts()
    plain.close()
    sim = _contact_pair_sim(B, "learned", params)
    sim.set_guess_wait(2048, stall=True)
    sim.step_phases(B.PHASE_CONTACT)
    with pytest.raises(B.MiDelbmError):
        sim.contacts()
    sim.stats()                                # clears the timeout bit
    got = sim.contacts()
    sim.close()
    for a, b in zip(sorted(ref, key=lambda c: (c["i"], c["j"])), sorted(got, key=lambda c: (c["i"], c["j"]))):
        assert (a["i"], a["j"], a["status"], a["iters"]) == (b["i"], b["j"], b["status"], b["iters"])
        assert np.array_equal(a["x_cp"], b["x_cp"])


@pytest.mark.parametrize("storage", [0, 1])
def test_check_finds_planted_non_finite_population(storage):
    B = binding()
    shape = (24, 20, 22)
    rng = np.random.default_rng(3)
    c, k, _ = scenes.blob_4(rng)
    spec = scenes.ParticleSpec(c, k, 2.5, 1.0, None, None)
    P = cp.prepared(spec, np.array([11.2, 10.1, 10.9]), scenes.random_unit_quaternion(rng), (0, 0, 0), (0, 0, 0))
    f0 = cp.initial_flow(shape, seed=5).astype(np.float32)
    sim = B.Simulation(*shape, tau=cp.TAU, storage=storage)
    cp.add_particles(sim, [P])
    sim.step_phases(B.PHASE_FLAG)              # current flags
    sim.set_populations(f0)
    assert sim.check()["bad_populations"] == 0
    _, own = sim.node_classes()
    own = own.astype(np.int64)
    solid = np.argwhere(own != 0xFFFFFFFF)
    fluid_node = (3, 4, 5)                     # (z, y, x), far from the particle
    assert own[fluid_node] == 0xFFFFFFFF
    bad = f0.copy()
    bad[7][fluid_node] = np.nan
    bad[2][(5, 6, 7)] = np.inf
    bad[11][tuple(solid[0])] = np.nan          # ignored: values at solid nodes are unspecified
    sim.set_populations(bad)
    with pytest.raises(B.MiDelbmError) as ei:
        sim.check()
    assert ei.value.status == B.MI_ESTATE
    h = ei.value.health
    assert h["bad_populations"] == 2 and h["bad_particles"] == 0
    z, y, x = fluid_node
    assert h["first_bad_node"] == x + shape[0] * (y + shape[1] * z)
    sim.set_populations(f0)
    assert sim.check()["bad_populations"] == 0
    sim.close()


def test_add_particle_rejects_bad_parameters():
    B = binding()
    c = np.array([[0.0, 0.0, 0.0], [1.0, 0.5, 0.0]])
    k = np.array([4.0, 3.0])
    pos = np.array([16.0, 16.0, 16.0])
    quat = np.array([1.0, 0.0, 0.0, 0.0])
    bad = [
        dict(k=np.array([4.0, 0.0])),                      # k must be > 0
        dict(k=np.array([4.0, -1.0])),
        dict(centers=np.array([[0.0, np.nan, 0.0], [1.0, 0.5, 0.0]])),
        dict(skin=3.0),                                    # skin below sqrt(sum k) = 2.65
        dict(quat=np.zeros(4)),
        dict(density=0.0),
        dict(pos=np.array([16.0, np.inf, 16.0])),
        dict(vel=np.array([np.nan, 0.0, 0.0])),
    ]
    with B.Simulation(32, 32, 32, tau=cp.TAU) as sim:
        for b in bad:
            a = dict(centers=c, k=k, density=2.5, skin=0.5, pos=pos, quat=quat, vel=np.zeros(3))
            a.update(b)
            with pytest.raises(B.MiDelbmError) as ei:
                sim.add_particle(a["centers"], a["k"], a["density"], a["skin"], a["pos"], a["quat"], a["vel"])
            assert ei.value.status == B.MI_EINVAL, b
        assert sim.num_particles() == 0
        sim.add_particle(c, k, 2.5, 0.5, pos, quat)        # still usable
        sim.step(2)
        sim.synchronize()
        assert sim.num_particles() == 1 and sim.check()["bad_populations"] == 0
