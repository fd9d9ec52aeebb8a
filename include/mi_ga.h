/* Genetic Algorithm capture of the principal outer contour of a point hull
 * (Sec. 2.2, Algorithm 1): a population of metaball models evolves by
 * mutation, crossover, evaluation of the fitness
 *     F(M) = sum_i (f_{H_i}(M) - 1)^2,  f of Eq. 1 at the hull points,
 * and selection of the fittest.
 *
 *   gene        one control point (x, y, z, k); an individual has n_genes
 *   draws       SplitMix64 (Steele, Lea and Flood 2014) of a key chained from
 *               (seed, generation, individual, gene * 256 + slot); u in [0, 1)
 *               is the top 24 bits times 2^-24; the initialisation uses
 *               generation 0xFFFFFFFF
 *   new gene    x, y, z = lo + u (hi - lo) over the hull's bounding box (FP32,
 *               single roundings), tried until inside the convex hull (the
 *               facet-plane test of mi_gs.h) -- 64 tries at initialisation
 *               (else the box centre), 8 at mutation (else the gene is kept);
 *               k = k_lo + u (k_hi - k_lo) with the draw of slot 1; the tries
 *               use slots 3 + 3 t + axis
 *   mutation    each gene of each individual, when the draw of slot 0 is
 *               below c_m
 *   crossover   the individuals ordered by the 64-bit draw of (gene 0, slot 2)
 *               (ties to the lower index) are paired (perm[2q], perm[2q+1]);
 *               each pair swaps its genes from p = floor(c_c n_genes) on, and
 *               the children take their parents' places (an odd last
 *               individual is copied)
 *   selection   of parents (indices 0..n_ind-1) and children (n_ind..), the
 *               n_ind smallest fitness values, ties to the lower index, a NaN
 *               fitness last, in that order
 * The fitness is summed in FP32 (a fixed order per individual).
 */
#ifndef MI_GA_H
#define MI_GA_H

#include <stddef.h>

#include "mi_delbm.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Bytes of device scratch mi_ga_run needs for a population shape. */
size_t mi_ga_scratch_bytes(int n_ind, int n_genes);

/* Run `generations` generations asynchronously on `stream` (a cudaStream_t
 * or NULL) on the current device.  Device arrays (caller-owned): hull (m x 3
 * floats), planes (n_planes x 4 floats: nx, ny, nz, d with n . x <= d inside),
 * pop (n_ind x n_genes x 4 floats: the start population when init == 0,
 * ignored when init != 0; the final population, fittest first, on return),
 * fit (n_ind floats out: the final fitness values), offspring and
 * fit_offspring (optional, n_ind x n_genes x 4 and n_ind floats: the last
 * generation's children before selection and their fitness), scratch
 * (mi_ga_scratch_bytes).  Host arrays: bbox (lo x, y, z, hi x, y, z), krange
 * (k_lo, k_hi).  generations == 0 only initialises (init != 0) and evaluates.
 * Errors: MI_EINVAL (n_ind < 2, n_genes < 1, m < 1, n_planes < 1,
 * generations < 0, c_m or c_c outside [0, 1], a NULL required array),
 * MI_ECUDA (launch failure). */
mi_status mi_ga_run(int n_ind, int n_genes, const float *hull, int m, const float *planes, int n_planes,
                    const float *bbox, const float *krange, float c_m, float c_c, unsigned long long seed,
                    int generations, int init, float *pop, float *fit, float *offspring, float *fit_offspring,
                    void *scratch, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* MI_GA_H */
