"""GPU parity of the Genetic Algorithm capture (Sec. 2.2, Algorithm 1;
mi_ga_run) against the oracle, through the C-ABI.

Bars: the initial population and the children of a generation are integer
decisions and FP32 values both sides take the same way (counter-based draws,
FP32 coordinates, the FP32 hull test, gene copies): bit-exact; fitness values
FP32 against FP64 within 1e-4 relative; the selection of the oracle fed the
GPU's own fitness values picks the same individuals in the same order (the
same bits); over a run the best fitness never rises and ends below the
initial best."""
import numpy as np
import pytest

from oracle import ga
from paper_2209_10411_gb300 import scenes
from tests.gpu_helpers import binding

pytestmark = pytest.mark.gpu

KR = (1.0, 6.0)


def _hull(seed=4, m=300, semi=(6.0, 4.0, 3.0)):
    rng = np.random.default_rng(seed)
    H = scenes.ellipsoid_hull(rng, m, semi, bumps=0.1)
    P = scenes.hull_planes(H)
    bbox = np.concatenate([H.min(0), H.max(0)]).astype(np.float32)
    return H, P, bbox


def test_initial_population_and_fitness():
    B = binding()
    H, P, bbox = _hull()
    pop, fit, _, _ = B.ga_run(H, P, bbox, KR, 64, 8, 0, 0.1, 0.5, 123)
    ref = ga.initial_population(123, 64, 8, bbox, KR, P)
    assert np.array_equal(pop, ref)
    fo = np.array([ga.fitness(H, ind) for ind in ref])
    assert np.allclose(fit, fo, rtol=1e-4)


@pytest.mark.parametrize("c_m,c_c", [(0.1, 0.5), (0.3, 0.25), (0.0, 0.75)])
def test_one_generation(c_m, c_c):
    B = binding()
    H, P, bbox = _hull()
    pop0, fit0, _, _ = B.ga_run(H, P, bbox, KR, 64, 8, 0, c_m, c_c, 77)
    pop1, fit1, off, fo = B.ga_run(H, P, bbox, KR, 64, 8, 1, c_m, c_c, 77, pop=pop0)
    ref_off = ga.offspring(pop0, 77, 0, c_m, c_c, bbox, KR, P)
    assert np.array_equal(off, ref_off)
    assert np.allclose(fo, [ga.fitness(H, ind) for ind in ref_off], rtol=1e-4)
    sel, sf, order = ga.select(pop0, fit0.astype(np.float64), off, fo.astype(np.float64))
    assert np.array_equal(pop1, sel)
    assert np.array_equal(fit1, sf.astype(np.float32))


def test_run_elitism_and_progress():
    B = binding()
    H, P, bbox = _hull(m=500)
    bests = []
    for g in (0, 5, 10, 20):
        pop, fit, _, _ = B.ga_run(H, P, bbox, KR, 200, 12, g, 0.05, 0.5, 5)
        assert np.all(np.diff(fit) >= 0) or g == 0
        bests.append(float(fit.min() if g == 0 else fit[0]))
    assert all(b2 <= b1 for b1, b2 in zip(bests, bests[1:]))
    assert bests[-1] < bests[0]
    assert abs(ga.fitness(H, pop[0]) - fit[0]) <= 1e-4 * fit[0]


def test_full_size_population():
    """1200 individuals of 32 genes on a 2048-point hull (the paper's
    population size), 10 generations: the best fitness falls, the population
    stays inside the hull."""
    B = binding()
    from oracle import gs
    H, P, bbox = _hull(seed=8, m=2048, semi=(12.0, 9.0, 7.0))
    pop0, fit0, _, _ = B.ga_run(H, P, bbox, (2.0, 12.0), 1200, 32, 0, 0.05, 0.5, 31)
    pop, fit, _, _ = B.ga_run(H, P, bbox, (2.0, 12.0), 1200, 32, 10, 0.05, 0.5, 31, pop=pop0)
    assert fit[0] < fit0.min()
    assert not gs.outside_hull_f32(pop.reshape(-1, 4)[:, :3], P).any()
