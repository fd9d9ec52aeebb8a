"""Genetic Algorithm capture of a principal outer contour (Sec. 2.2,
Algorithm 1) for the oracle (test infrastructure only).

A population of N_I individuals, each a metaball model of N_G genes (one
gene = one control point (x, y, z, k)), evolves for E generations: mutation,
crossover, evaluation of the fitness F(M) = sum_i (f_{H_i}(M) - 1)^2 over the
hull points (Eq. objF, f of Eq. 1), and selection of the fittest N_I.

Readings (the paper leaves these open):
  R1  a gene is one control point; crossover exchanges whole genes.
  R2  mutation: each gene of each individual mutates with probability C_m;
      a mutated gene is a new random control point inside the hull: x, y, z
      uniform in the hull's bounding box (accepted when inside the convex
      hull, up to 8 tries, else the gene is kept) and k uniform in
      [k_lo, k_hi].  Initialisation draws every gene the same way (64 tries,
      else the bounding-box centre).
  R3  crossover: the mutated individuals are paired at random (a shuffle of
      the population; pairs (perm[2q], perm[2q+1]), an odd last one stays
      single) and each pair swaps its genes from the crossover point
      p = floor(C_c N_G) on; the two children take their parents' places.
  R4  selection: parents and children together, the N_I smallest fitness
      values (ties to the lower index, parents before children) form the next
      population in that order; a NaN fitness ranks last.
  R5  random numbers: one counter-based generator, the SplitMix64 mixing
      function (Steele, Lea and Flood 2014) applied to a key chained from
      (seed, generation, individual, gene * 256 + slot); a uniform u in [0, 1)
      is the top 24 bits times 2^-24 (exact in FP32).  Coordinates are
      lo + u (hi - lo) with single FP32 roundings, and "inside the hull" is
      the FP32 facet-plane test of the Gradient Search (both are integers or
      values the kernel takes in FP32, so the oracle takes them in FP32).
  R6  the result is the fittest individual of the last population.
Fitness sums are FP64 here (FP32 on the GPU): selection parity is checked on
the GPU's own fitness values.
"""
import numpy as np

from .gs import outside_hull_f32

MASK = (1 << 64) - 1
INIT_GEN = 0xFFFFFFFF
SLOT_MUTATE, SLOT_K, SLOT_KEY = 0, 1, 2
TRIES_MUTATE, TRIES_INIT = 8, 64


def splitmix64(x):
    """SplitMix64 output for state x (the state advanced by the golden gamma,
    then the two xor-shift-multiply rounds and a final xor-shift)."""
    z = (x + 0x9E3779B97F4A7C15) & MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
    return z ^ (z >> 31)


def draw(seed, gen, ind, gene, slot):
    """64-bit random word for (seed, generation, individual, gene, slot)."""
    h = splitmix64(seed & MASK)
    h = splitmix64(h ^ (gen & MASK))
    h = splitmix64(h ^ (ind & MASK))
    return splitmix64(h ^ ((gene * 256 + slot) & MASK))


def uniform(seed, gen, ind, gene, slot):
    return np.float32((draw(seed, gen, ind, gene, slot) >> 40) * (2.0 ** -24))


def _lerp32(lo, hi, u):
    lo, hi = np.float32(lo), np.float32(hi)
    return np.float32(lo + np.float32(u * np.float32(hi - lo)))


def random_gene(seed, gen, ind, gene, bbox, krange, planes, tries):
    """(x, y, z, k) inside the hull, or None after `tries` rejected tries."""
    for t in range(tries):
        p = np.array([_lerp32(bbox[a], bbox[3 + a], uniform(seed, gen, ind, gene, 3 + 3 * t + a)) for a in range(3)],
                     dtype=np.float32)
        if not outside_hull_f32(p[None, :], planes)[0]:
            k = _lerp32(krange[0], krange[1], uniform(seed, gen, ind, gene, SLOT_K))
            return np.array([p[0], p[1], p[2], k], dtype=np.float32)
    return None


def initial_population(seed, n_ind, n_genes, bbox, krange, planes):
    pop = np.zeros((n_ind, n_genes, 4), dtype=np.float32)
    centre = [np.float32(np.float32(0.5) * np.float32(np.float32(bbox[a]) + np.float32(bbox[3 + a]))) for a in range(3)]
    for i in range(n_ind):
        for g in range(n_genes):
            v = random_gene(seed, INIT_GEN, i, g, bbox, krange, planes, TRIES_INIT)
            if v is None:
                v = np.array(centre + [_lerp32(krange[0], krange[1], uniform(seed, INIT_GEN, i, g, SLOT_K))],
                             dtype=np.float32)
            pop[i, g] = v
    return pop


def fitness(H, genes):
    """F(M) = sum_i (f_i - 1)^2 (Eq. objF), FP64."""
    H = np.asarray(H, dtype=np.float64)
    g = np.asarray(genes, dtype=np.float64)
    d = H[:, None, :] - g[None, :, :3]
    f = np.sum(g[None, :, 3] / np.sum(d * d, axis=2), axis=1)
    return float(np.sum((f - 1.0) ** 2))


def crossover_point(c_c, n_genes):
    """p = floor(C_c N_G), with C_c rounded to FP32 first (the kernel's
    argument type) and the product in FP64."""
    return int(np.floor(float(np.float32(c_c)) * n_genes))


def offspring(pop, seed, gen, c_m, c_c, bbox, krange, planes):
    """Mutation (R2) then crossover (R3) of one generation."""
    n_ind, n_genes, _ = pop.shape
    mut = pop.copy()
    for i in range(n_ind):
        for g in range(n_genes):
            if uniform(seed, gen, i, g, SLOT_MUTATE) < np.float32(c_m):
                v = random_gene(seed, gen, i, g, bbox, krange, planes, TRIES_MUTATE)
                if v is not None:
                    mut[i, g] = v
    keys = np.array([draw(seed, gen, i, 0, SLOT_KEY) for i in range(n_ind)], dtype=np.uint64)
    perm = np.argsort(keys, kind="stable")
    p = crossover_point(c_c, n_genes)
    out = mut.copy()
    for q in range(n_ind // 2):
        a, b = perm[2 * q], perm[2 * q + 1]
        out[a, :p], out[a, p:] = mut[a, :p], mut[b, p:]
        out[b, :p], out[b, p:] = mut[b, :p], mut[a, p:]
    return out


def select(pop, fit, off, fit_off):
    """R4: the N_I fittest of parents and children, ties to the lower index."""
    n_ind = len(pop)
    allf = np.concatenate([np.asarray(fit, dtype=np.float64), np.asarray(fit_off, dtype=np.float64)])
    allf = np.where(np.isnan(allf), np.inf, allf)
    order = np.lexsort((np.arange(2 * n_ind), allf))[:n_ind]
    cand = np.concatenate([pop, off])
    return cand[order], allf[order], order


def run(H, planes, bbox, krange, n_ind, n_genes, generations, c_m, c_c, seed, pop=None):
    """Algorithm 1; returns the final population (fittest first), its
    fitness values and the best fitness after every generation."""
    if pop is None:
        pop = initial_population(seed, n_ind, n_genes, bbox, krange, planes)
    fit = np.array([fitness(H, ind) for ind in pop])
    best = []
    for gen in range(generations):
        off = offspring(pop, seed, gen, c_m, c_c, bbox, krange, planes)
        fo = np.array([fitness(H, ind) for ind in off])
        pop, fit, _ = select(pop, fit, off, fo)
        best.append(float(fit[0]))
    return pop, fit, best
