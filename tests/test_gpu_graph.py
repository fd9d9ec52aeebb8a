"""A step replayed from a CUDA graph (with its concurrent wall-fraction and
contact branches) gives bit-identical results to the same step issued as
individual launches: every reduction on the path is an order-free
fixed-point sum, so neither the branch overlap nor the list order may change
a single bit."""
import numpy as np
import pytest

from oracle import lbm
from paper_2209_10411_gb300 import scenes
from tests.gpu_helpers import binding
from tests.test_gpu_contact import PARAMS, _cluster

pytestmark = pytest.mark.gpu


def _run(B, graphs, parts, shape, f0, nsteps, dem_substeps):
    sim = B.Simulation(*shape, tau=0.8, gravity=(0, 0, -1e-4), dem_substeps=dem_substeps, kn=PARAMS["kn"],
                       kt=PARAMS["kt"], eta_n=PARAMS["eta_n"], eta_t=PARAMS["eta_t"], mu_s=PARAMS["mu_s"],
                       max_particles=64)
    sim.set_graphs(graphs)
    for P in parts:
        sim.add_particle(P["centers"], P["k"], P["density"], P["skin"], P["pos"], P["quat"], P["vel"], P["omega"],
                         mass_props={"mass": P["mass"], "volume": P["volume"], "inertia": P["inertia"]})
    sim.set_populations(f0)
    out = []
    for _ in range(nsteps):
        sim.step(1)
        st = [sim.get_particle_state(i) for i in range(len(parts))]
        out.append((sim.forces(), st))
    pops = sim.get_raw_populations()
    cls, own = sim.node_classes()
    sim.close()
    return out, pops, cls, own


@pytest.mark.parametrize("dem_substeps", [1, 3])
def test_graph_replay_is_bitwise_identical(dem_substeps):
    B = binding()
    shape = (48, 48, 40)
    parts = _cluster(6)
    for P in parts:
        P["vel"] = P["vel"] * 20.0  # move enough to uncover nodes within a few steps
    nx, ny, nz = shape
    u = 0.02 * scenes.velocity_field_noise(shape, 9)
    f0 = lbm.equilibrium(np.ones((nz, ny, nx)), u).astype(np.float32)
    a = _run(B, True, parts, shape, f0, 6, dem_substeps)
    b = _run(B, False, parts, shape, f0, 6, dem_substeps)
    for (fa, sa), (fb, sb) in zip(a[0], b[0]):
        for key in fa:
            assert np.array_equal(fa[key], fb[key]), key
        for x, y in zip(sa, sb):
            for key in x:
                assert np.array_equal(x[key], y[key]), key
    assert np.array_equal(a[2], b[2]) and np.array_equal(a[3], b[3])
    fluid = a[3] == 0xFFFFFFFF  # values at solid nodes are unspecified
    assert np.array_equal(a[1][:, fluid].view(np.uint32), b[1][:, fluid].view(np.uint32))
    assert np.abs(a[0][-1][0]["F_contact"]).max() > 0  # contacts were exercised


def test_autotune_cache_and_bitwise_results(tmp_path):
    """The autotuner's launch shapes change no result bit (all sums are
    order-free), and a second handle reads the cached choice."""
    B = binding()
    shape = (48, 48, 40)
    parts = _cluster(7)
    nx, ny, nz = shape
    u = 0.02 * scenes.velocity_field_noise(shape, 3)
    f0 = lbm.equilibrium(np.ones((nz, ny, nx)), u).astype(np.float32)
    cache = str(tmp_path / "tune.json")

    def make():
        sim = B.Simulation(*shape, tau=0.8, kn=PARAMS["kn"], kt=PARAMS["kt"], eta_n=PARAMS["eta_n"],
                           eta_t=PARAMS["eta_t"], mu_s=PARAMS["mu_s"], max_particles=64)
        for P in parts:
            sim.add_particle(P["centers"], P["k"], P["density"], P["skin"], P["pos"], P["quat"], P["vel"],
                             P["omega"], mass_props={"mass": P["mass"], "volume": P["volume"],
                                                     "inertia": P["inertia"]})
        sim.set_populations(f0)
        return sim

    a, b = make(), make()
    a.step(1)
    b.step(1)
    t1 = a.autotune(cache)
    assert t1["bulk_block_x"] in (32, 64, 128, 256) and t1["list_blocks_per_sm"] in (2, 4, 8, 16, 32)
    lines = open(cache).read().strip().splitlines()
    assert len(lines) == 1 and '"bulk_block_x": %d' % t1["bulk_block_x"] in lines[0]
    t2 = b.autotune(cache)  # same key: read back, nothing appended
    assert t2 == t1 and len(open(cache).read().strip().splitlines()) == 1
    c = make()  # never tuned
    c.step(1)
    for sim in (a, b, c):
        sim.step(3)
    ra, rc = a.get_raw_populations(), c.get_raw_populations()
    _, own = a.node_classes()
    fluid = own == 0xFFFFFFFF
    assert np.array_equal(ra[:, fluid].view(np.uint32), rc[:, fluid].view(np.uint32))
    fa, fc = a.forces(), c.forces()
    for key in fa:
        assert np.array_equal(fa[key], fc[key]), key
    for sim in (a, b, c):
        sim.close()


@pytest.mark.parametrize("storage", [0, 1])
def test_overlapped_boundary_schedule_is_bitwise_identical(storage):
    """Computing the boundary nodes beside the bulk kernel into a side buffer
    and scattering them afterwards, or only the links' bounce-back beside it,
    changes no bit of the populations, the forces or the particle states
    (graph replay, moving particles, contacts)."""
    B = binding()
    shape = (48, 48, 40)
    parts = _cluster(8)
    for P in parts:
        P["vel"] = P["vel"] * 20.0
    nx, ny, nz = shape
    u = 0.02 * scenes.velocity_field_noise(shape, 5)
    f0 = lbm.equilibrium(np.ones((nz, ny, nx)), u).astype(np.float32)
    out = []
    for schedule in ({}, {"overlap_boundary": True}, {"links_beside": True}):
        sim = B.Simulation(*shape, tau=0.8, gravity=(0, 0, -1e-4), storage=storage, kn=PARAMS["kn"], kt=PARAMS["kt"],
                           eta_n=PARAMS["eta_n"], eta_t=PARAMS["eta_t"], mu_s=PARAMS["mu_s"], max_particles=64)
        sim.set_schedule(**schedule)
        for P in parts:
            sim.add_particle(P["centers"], P["k"], P["density"], P["skin"], P["pos"], P["quat"], P["vel"], P["omega"],
                             mass_props={"mass": P["mass"], "volume": P["volume"], "inertia": P["inertia"]})
        sim.set_populations(f0)
        sim.step(6)
        st = [sim.get_particle_state(i) for i in range(len(parts))]
        out.append((sim.get_raw_populations(), sim.forces(), st, sim.node_classes()))
        sim.close()
    pa, fa, sa, (ca, oa) = out[0]
    fluid = oa == 0xFFFFFFFF
    for pb, fb, sb, (cb, ob) in out[1:]:
        assert np.array_equal(ca, cb) and np.array_equal(oa, ob)
        assert np.ascontiguousarray(pa[:, fluid]).tobytes() == np.ascontiguousarray(pb[:, fluid]).tobytes()
        for key in fa:
            assert np.array_equal(fa[key], fb[key]), key
        for x, y in zip(sa, sb):
            for key in x:
                assert np.array_equal(x[key], y[key]), key


@pytest.mark.parametrize("nsteps,dem_substeps", [(7, 1), (8, 3)])
def test_device_loop_graph_is_bitwise_identical(nsteps, dem_substeps):
    """All steps of one call as one graph launch (a conditional while node
    over two-step bodies, the pair count on the device; an odd count adds a
    single-step graph) against one graph launch per step: the same bits, in
    two calls in a row (the second replays the instantiated loop)."""
    B = binding()
    shape = (48, 48, 40)
    parts = _cluster(6)
    for P in parts:
        P["vel"] = P["vel"] * 20.0
    nx, ny, nz = shape
    u = 0.02 * scenes.velocity_field_noise(shape, 11)
    f0 = lbm.equilibrium(np.ones((nz, ny, nx)), u).astype(np.float32)
    res = []
    for loop in (False, True):
        sim = B.Simulation(*shape, tau=0.8, gravity=(0, 0, -1e-4), dem_substeps=dem_substeps, kn=PARAMS["kn"],
                           kt=PARAMS["kt"], eta_n=PARAMS["eta_n"], eta_t=PARAMS["eta_t"], mu_s=PARAMS["mu_s"],
                           max_particles=64)
        sim.set_graphs(True, device_loop=loop)
        for P in parts:
            sim.add_particle(P["centers"], P["k"], P["density"], P["skin"], P["pos"], P["quat"], P["vel"],
                             P["omega"], mass_props={"mass": P["mass"], "volume": P["volume"],
                                                     "inertia": P["inertia"]})
        sim.set_populations(f0)
        l0 = sim.launch_count()
        sim.step(nsteps)
        sim.step(nsteps)
        launches = sim.launch_count() - l0
        st = [sim.get_particle_state(i) for i in range(len(parts))]
        res.append((sim.forces(), st, sim.get_raw_populations(), sim.node_classes(), launches))
        sim.close()
    (fa, sa, pa, (ca, oa), la), (fb, sb, pb, (cb, ob), lb) = res
    for key in fa:
        assert np.array_equal(fa[key], fb[key]), key
    for x, y in zip(sa, sb):
        for key in x:
            assert np.array_equal(x[key], y[key]), key
    assert np.array_equal(ca, cb) and np.array_equal(oa, ob)
    fluid = oa == 0xFFFFFFFF
    assert np.array_equal(pa[:, fluid].view(np.uint32), pb[:, fluid].view(np.uint32))
    # the same kernels, plus per call one counter kernel and one loop-tail kernel per step pair
    assert lb - la == 2 * (nsteps // 2 + 1)
