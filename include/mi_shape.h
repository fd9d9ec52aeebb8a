/* Shape descriptors of metaball particles (Sec. 3: sphericity Phi, nominal
 * diameter d_n, projected-area diameter d_s, Corey shape factor CSF), by
 * quadrature on the GPU.
 *
 *   grid 1      body frame, cells of spacing h centred at -R_g + (i + 1/2) h,
 *               i < n, with R_g and n given per particle (R_g = max |c_j| +
 *               sqrt(sum k / (1 - eps)) holds the solid and the band below)
 *   field       f = sum_j k_j / |x - c_j|^2 in FP32 with single roundings:
 *               differences, squares, (d0^2 + d1^2) + d2^2, one IEEE
 *               division per ball, balls in order
 *   volume      V = h^3 #{cells with f >= 1}
 *   surface     S = h^3 / (2 eps) sum of |grad f| over the cells with
 *               |f - 1| < eps (coarea estimate)
 *   axes        eigenvectors of the solid cells' second moments about their
 *               centroid, longest first
 *   grid 2      n + 4 cells per axis along the axes, centred on the centroid,
 *               from -(R_g + 2 h): the extents L (max - min of the solid
 *               cells' coordinates, plus h) and the projection along the
 *               shortest axis, A_p = h^2 #{columns holding a solid cell}
 *   descriptors d_n = (6 V / pi)^(1/3), Phi = pi d_n^2 / S,
 *               d_s = sqrt(4 A_p / pi), CSF = L_short / sqrt(L_int L_long)
 */
#ifndef MI_SHAPE_H
#define MI_SHAPE_H

#include <stddef.h>

#include "mi_delbm.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Output row of one particle (doubles). */
enum {
  MI_SHAPE_VOLUME = 0, MI_SHAPE_SURFACE, MI_SHAPE_L_LONG, MI_SHAPE_L_INT, MI_SHAPE_L_SHORT,
  MI_SHAPE_PROJECTED_AREA, MI_SHAPE_SPHERICITY, MI_SHAPE_D_N, MI_SHAPE_D_S, MI_SHAPE_CSF,
  MI_SHAPE_CELLS, MI_SHAPE_FIELDS
};

/* Device scratch bytes for n_particles particles whose first grids have at
 * most max_n cells per axis. */
size_t mi_shape_scratch_bytes(int n_particles, int max_n);

/* Descriptors of n_particles metaball models, asynchronously on `stream` (a
 * cudaStream_t or NULL) on the current device.  Device arrays (caller-owned):
 * ball_off (n_particles + 1 ints), balls (4 floats x, y, z, k per ball, body
 * frame), grid_r (per particle R_g, float), grid_n (per particle n, int, at
 * most max_n), out (MI_SHAPE_FIELDS doubles per particle), axes (9 floats per
 * particle: the unit axes, longest first, as rows; may be NULL), scratch
 * (mi_shape_scratch_bytes).  h > 0 and 0 < eps < 1 are the spacing and the
 * band half-width.  A particle without a solid cell, or with more than 4096
 * balls, gets NaN descriptors.
 * Errors: MI_EINVAL (sizes, h, eps, NULL arrays), MI_ECUDA. */
mi_status mi_shape_descriptors(int n_particles, const int *ball_off, const float *balls, const float *grid_r,
                               const int *grid_n, int max_n, float h, float eps, double *out, float *axes,
                               void *scratch, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* MI_SHAPE_H */
