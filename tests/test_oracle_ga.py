"""Pins of the Genetic Algorithm oracle (Sec. 2.2, Algorithm 1): the
generator against SplitMix64's published first output, the fitness against
its closed form for one ball on a sphere, the genetic operators' special
cases (no mutation, crossover point at either end), initialisation inside
the hull, selection against a brute-force sort, and elitism."""
import numpy as np
import pytest

from oracle import ga, gs
from paper_2209_10411_gb300 import scenes


def test_splitmix64_published_first_output():
    # the first output of SplitMix64 from state 0
    assert ga.splitmix64(0) == 0xE220A8397B1DCDAF


def test_uniform_draws():
    u = np.array([ga.uniform(7, 3, i, i % 5, 1) for i in range(20000)], dtype=np.float64)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.01 and abs(u.var() - 1.0 / 12.0) < 0.003
    assert all(np.float32(x) == x for x in u[:100])


def _hull(seed=3, m=400, semi=(6.0, 4.0, 3.0)):
    rng = np.random.default_rng(seed)
    H = scenes.ellipsoid_hull(rng, m, semi)
    P = scenes.hull_planes(H)
    bbox = np.concatenate([H.min(0), H.max(0)]).astype(np.float32)
    return H, P, bbox


def test_fitness_closed_form_single_ball():
    R, k = 3.0, 5.0
    u = np.random.default_rng(1).normal(size=(50, 3))
    H = R * u / np.linalg.norm(u, axis=1, keepdims=True)
    F = ga.fitness(H, np.array([[0.0, 0.0, 0.0, k]]))
    assert F == pytest.approx(50 * (k / R ** 2 - 1.0) ** 2, rel=1e-12)
    assert ga.fitness(H, np.array([[0.0, 0.0, 0.0, R * R]])) == pytest.approx(0.0, abs=1e-20)


def test_initial_population_inside_hull():
    H, P, bbox = _hull()
    pop = ga.initial_population(11, 20, 6, bbox, (1.0, 4.0), P)
    g = pop.reshape(-1, 4)
    assert not gs.outside_hull_f32(g[:, :3], P).any()
    assert (g[:, 3] >= 1.0).all() and (g[:, 3] < 4.0).all()


def test_operators_special_cases():
    H, P, bbox = _hull()
    pop = ga.initial_population(5, 10, 6, bbox, (1.0, 4.0), P)
    # no mutation, crossover point 0: every pair swaps whole individuals
    off = ga.offspring(pop, 5, 0, 0.0, 0.0, bbox, (1.0, 4.0), P)
    assert sorted(map(bytes, off)) == sorted(map(bytes, pop))
    assert not np.array_equal(off, pop)
    # crossover point at the end: children are their parents
    assert np.array_equal(ga.offspring(pop, 5, 0, 0.0, 1.0, bbox, (1.0, 4.0), P), pop)
    # every gene mutated: all new genes inside the hull
    off = ga.offspring(pop, 5, 1, 1.0, 1.0, bbox, (1.0, 4.0), P)
    assert not gs.outside_hull_f32(off.reshape(-1, 4)[:, :3], P).any()
    assert np.mean(off != pop) > 0.9


def test_selection_is_the_sorted_best():
    rng = np.random.default_rng(2)
    pop = rng.normal(size=(8, 3, 4)).astype(np.float32)
    off = rng.normal(size=(8, 3, 4)).astype(np.float32)
    fp = rng.uniform(size=8)
    fo = rng.uniform(size=8)
    fo[3] = fp[5]  # a tie: the parent (lower index) comes first
    fo[6] = np.nan
    new, nf, order = ga.select(pop, fp, off, fo)
    allf = np.concatenate([fp, fo])
    brute = sorted(range(16), key=lambda c: (np.inf if np.isnan(allf[c]) else allf[c], c))[:8]
    assert list(order) == brute
    assert np.array_equal(new, np.concatenate([pop, off])[brute])


def test_elitism_and_progress():
    H, P, bbox = _hull(m=300)
    pop, fit, best = ga.run(H, P, bbox, (1.0, 6.0), 24, 4, 12, 0.1, 0.5, 9)
    assert all(b2 <= b1 for b1, b2 in zip(best, best[1:]))
    init = ga.initial_population(9, 24, 4, bbox, (1.0, 6.0), P)
    assert best[-1] < min(ga.fitness(H, ind) for ind in init)
    assert fit[0] == pytest.approx(ga.fitness(H, pop[0]))
