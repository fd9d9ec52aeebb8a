"""GPU parity of the bulk stream-collide (no particles) against the FP64
oracle, through the C-ABI.

Tolerances: FP32 storage, |f_gpu - f_ref| <= 1e-5 |f_ref| per population
(FP32 arithmetic of ~60 operations on O(1) values gives ~1e-7; the bound
leaves two orders of margin).  16-bit deviation storage: the stored value is
h = f - w_i with w_i the FP32 weight (|w32 - w| <= 1.5e-8); the GPU's stored
deviation may differ from the oracle's exact result by at most one unit in the
last place of the storage type (rounding of an FP32 value that is itself
within ~1e-7 of the oracle's), plus 1e-7 absolute.
"""
import numpy as np
import pytest

from oracle import lbm
from oracle.d3q19 import W
from paper_2209_10411_gb300 import scenes
from tests.gpu_helpers import DeviceGather, binding, decode, pop_tensor, ulp16

pytestmark = pytest.mark.gpu

TAU = 0.8


def _initial(shape, seed, amp=0.05):
    noise = scenes.lattice_noise(shape, seed).astype(np.float64)
    return (W.reshape(19, 1, 1, 1) * (1.0 + amp * noise)).astype(np.float32)


CASES = [
    # shape (nx, ny, nz), periodic, moving wall on face, body force
    ((37, 9, 11), (False, False, False), None, None),
    ((40, 12, 10), (True, False, True), (3, (0.03, 0.0, -0.02)), None),
    ((33, 7, 6), (True, True, True), None, (1e-5, -2e-5, 3e-5)),
    ((200, 5, 4), (False, True, False), (0, (0.0, 0.01, 0.02)), (0.0, 0.0, 1e-5)),
    ((1, 16, 1), (True, False, True), (3, (0.01, 0.0, 0.0)), None),
    ((130, 6, 5), (True, True, False), (5, (0.01, -0.02, 0.0)), (2e-5, 0.0, -1e-5)),
]


# launch variants of the bulk kernel: (threads per block, rows per thread, paired nodes)
VARIANTS = [(128, 1, 0), (32, 2, 0), (64, 1, 1), (32, 1, 1), (128, 1, 2), (32, 1, 3), (128, 1, 3)]


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("nsteps", [1, 3])
@pytest.mark.parametrize("variant", range(len(VARIANTS)))
def test_bulk_f32_matches_oracle(case, nsteps, variant):
    B = binding()
    shape, periodic, wall, force = CASES[case]
    wv = np.zeros((6, 3))
    if wall is not None:
        wv[wall[0]] = wall[1]
    f0 = _initial(shape, seed=case)
    bx, rows, pairs = VARIANTS[variant]
    with B.Simulation(*shape, tau=TAU, periodic=periodic, wall_velocity=wv,
                      fluid_body_force=force or (0, 0, 0)) as sim:
        sim.set_tuning(bx, rows, pairs, 8)
        sim.set_populations(f0)
        assert np.array_equal(sim.get_populations(), f0)
        sim.step(nsteps)
        got = sim.get_populations().astype(np.float64)
    ref = f0.astype(np.float64)
    for _ in range(nsteps):
        ref = lbm.step_bulk(ref, TAU, periodic=periodic, wall_velocity=wv, force=force)
    rel = np.abs(got - ref) / np.abs(ref)
    assert rel.max() < 1e-5, "max rel err %g" % rel.max()


@pytest.mark.parametrize("storage", [1, 2])
@pytest.mark.parametrize("shape,variant", [((45, 10, 9), 0), ((46, 10, 9), 2), ((70, 6, 5), 3), ((64, 7, 6), 1),
                                           ((262, 5, 4), 4), ((48, 10, 9), 5), ((264, 6, 5), 6), ((50, 8, 7), 5),
                                           ((12, 5, 4), 6)])
def test_bulk_16bit_deviation_storage(storage, shape, variant):
    B = binding()
    wv = np.zeros((6, 3))
    wv[5] = (0.02, -0.01, 0.0)
    f0 = _initial(shape, seed=21, amp=0.02)
    bx, rows, pairs = VARIANTS[variant]
    with B.Simulation(*shape, tau=TAU, wall_velocity=wv, storage=storage) as sim:
        sim.set_tuning(bx, rows, pairs, 8)
        sim.set_populations(f0)
        raw0 = sim.get_raw_populations()
        h0 = decode(raw0, storage)
        # stored value is f - w rounded to nearest even in the 16-bit type, with
        # w the FP32 weight (within 1.5e-8 of the exact one)
        exact = f0.astype(np.float64) - W.reshape(19, 1, 1, 1)
        assert np.all(np.abs(h0 - exact) <= 0.5 * ulp16(exact, storage) + 2e-8)
        sim.step(1)
        h1 = decode(sim.get_raw_populations(), storage)
    fin = h0 + W.reshape(19, 1, 1, 1)
    ref = lbm.step_bulk(fin, TAU, wall_velocity=wv) - W.reshape(19, 1, 1, 1)
    err = np.abs(h1 - ref)
    assert np.all(err <= ulp16(ref, storage) + 1e-7), "max err %g" % err.max()


@pytest.mark.parametrize("storage", [1, 2])
@pytest.mark.parametrize("shape,periodic,force", [((64, 6, 5), (True, True, False), (1e-5, -2e-5, 3e-5)),
                                                  ((40, 5, 7), (True, False, True), None),
                                                  ((48, 7, 4), (False, True, True), (0.0, 1e-5, 0.0)),
                                                  ((32, 4, 4), (True, True, True), None)])
@pytest.mark.parametrize("variant", [5, 6])
def test_bulk_16bit_periodic_and_forced(storage, shape, periodic, force, variant):
    """The four-node kernel with periodic x faces (the wrapped word), periodic
    or wall y / z faces, moving walls and Guo forcing, two steps against the
    oracle fed the decoded inputs of each step."""
    B = binding()
    wv = np.zeros((6, 3))
    wv[0] = (0.0, 0.01, -0.02)
    wv[5] = (0.02, -0.01, 0.0)
    f0 = _initial(shape, seed=33, amp=0.02)
    bx, rows, pairs = VARIANTS[variant]
    with B.Simulation(*shape, tau=TAU, periodic=periodic, wall_velocity=wv, storage=storage,
                      fluid_body_force=force or (0, 0, 0)) as sim:
        sim.set_tuning(bx, rows, pairs, 8)
        sim.set_populations(f0)
        for _ in range(2):
            h0 = decode(sim.get_raw_populations(), storage)
            sim.step(1)
            h1 = decode(sim.get_raw_populations(), storage)
            fin = h0 + W.reshape(19, 1, 1, 1)
            ref = lbm.step_bulk(fin, TAU, periodic=periodic, wall_velocity=wv, force=force) - W.reshape(19, 1, 1, 1)
            err = np.abs(h1 - ref)
            assert np.all(err <= ulp16(ref, storage) + 1e-7), "max err %g" % err.max()


def test_rest_state_and_mass_conservation():
    B = binding()
    shape = (64, 24, 20)
    with B.Simulation(*shape, tau=TAU) as sim:
        f = sim.get_populations()
        assert np.array_equal(f, np.broadcast_to(W.reshape(19, 1, 1, 1).astype(np.float32), f.shape))
        f0 = _initial(shape, seed=5)
        sim.set_populations(f0)
        m0 = f0.astype(np.float64).sum()
        sim.step(20)
        m1 = sim.get_populations().astype(np.float64).sum()
    assert abs(m1 - m0) / m0 < 1e-6


@pytest.mark.parametrize("variant", [0, 2])
def test_bulk_full_size_sampled(variant):
    """256x256x512 (the settling-tank lattice), one step in the benchmark's
    launch configurations (scalar and paired nodes), checked on 4096 random
    nodes plus every corner and edge-adjacent sample against the oracle
    evaluated node by node."""
    import torch
    B = binding()
    shape = (256, 256, 512)
    nx, ny, nz = shape
    bx, rows, pairs = VARIANTS[variant]
    with B.Simulation(*shape, tau=TAU) as sim:
        sim.set_tuning(bx, rows, pairs, 8)
        t = pop_tensor(sim)
        g = torch.Generator(device="cuda")
        g.manual_seed(1234)
        w = torch.tensor(W, dtype=torch.float32, device="cuda").reshape(19, 1)
        ncell = nx * ny * nz
        t[:, :ncell] = w * (1.0 + 0.05 * torch.randn((19, ncell), generator=g, device="cuda"))
        torch.cuda.synchronize()
        rng = np.random.default_rng(3)
        cells = np.stack([rng.integers(0, nx, 4096), rng.integers(0, ny, 4096), rng.integers(0, nz, 4096)], 1)
        corners = np.array([[x, y, z] for x in (0, nx - 1) for y in (0, ny - 1) for z in (0, nz - 1)])
        edges = np.array([[0, 5, 7], [nx - 1, 100, 200], [17, 0, 300], [18, ny - 1, 1], [200, 3, 0], [9, 9, nz - 1]])
        cells = np.concatenate([cells, corners, edges])
        before = DeviceGather(sim)
        ref = lbm.update_cells(before, cells, TAU)
        sim.step(1)
        after = DeviceGather(sim)
        got = np.stack([after[i, cells[:, 2], cells[:, 1], cells[:, 0]] for i in range(19)])
    rel = np.abs(got - ref) / np.abs(ref)
    assert rel.max() < 1e-5, "max rel err %g" % rel.max()


@pytest.mark.parametrize("storage", [1, 2])
def test_bulk_16bit_full_size_sampled(storage):
    """256x256x512 in 16-bit deviation storage, one step with the four-node
    kernel (the benchmark's 16-bit configuration), checked on 4096 random
    nodes plus corners and edges against the oracle fed the decoded inputs:
    within one unit in the last place of the stored type (plus 1e-7)."""
    import torch
    B = binding()
    shape = (256, 256, 512)
    nx, ny, nz = shape
    bx, rows, pairs = VARIANTS[6]
    with B.Simulation(*shape, tau=TAU, storage=storage) as sim:
        sim.set_tuning(bx, rows, pairs, 8)
        t = pop_tensor(sim)
        g = torch.Generator(device="cuda")
        g.manual_seed(4321)
        w = torch.tensor(W, dtype=torch.float32, device="cuda").reshape(19, 1)
        ncell = nx * ny * nz
        dev = w * 0.05 * torch.randn((19, ncell), generator=g, device="cuda")
        t[:, :ncell] = (dev.half() if storage == 1 else dev.bfloat16()).view(torch.int16)
        del dev
        torch.cuda.synchronize()
        rng = np.random.default_rng(4)
        cells = np.stack([rng.integers(0, nx, 4096), rng.integers(0, ny, 4096), rng.integers(0, nz, 4096)], 1)
        corners = np.array([[x, y, z] for x in (0, nx - 1) for y in (0, ny - 1) for z in (0, nz - 1)])
        edges = np.array([[0, 5, 7], [nx - 1, 100, 200], [3, 9, 9], [4, 9, 9], [nx - 5, 9, 9], [nx - 8, 9, 9],
                          [17, 0, 300], [18, ny - 1, 1], [200, 3, 0], [9, 9, nz - 1]])
        cells = np.concatenate([cells, corners, edges])
        before = DeviceGather(sim)
        ref = lbm.update_cells(before, cells, TAU)
        sim.step(1)
        after = DeviceGather(sim)
        got = np.stack([after[i, cells[:, 2], cells[:, 1], cells[:, 0]] for i in range(19)])
    Wc = W.reshape(19, 1)
    err = np.abs(got - ref)
    assert np.all(err <= ulp16(ref - Wc, storage) + 1e-7), "max err %g" % err.max()
