/* Gradient Search refinement of metaball models on point hulls (Sec. 2.2,
 * Algorithm 2 with the piecewise loss Eq. GSloss): full-batch gradient
 * descent on every control point (c_j, k_j) of a model, anomaly detection,
 * and a second descent.  Many independent fits run in one call, one CTA
 * each, in FP32.
 *
 *   field      f_i = sum_j k_j / |H_i - c_j|^2 at each hull point H_i (Eq. 1)
 *   loss       L = sum_i l(f_i), l = (f - 1)^2 on [2, inf), |f - 1| on [1, 2),
 *              (f - 1)^2 + 1/f - 1 on [0, 1)
 *   gradient   dl/df = 2 (f - 1), +1, 2 (f - 1) - 1/f^2 on those intervals;
 *              dL/dk_j = sum_i dl/df_i / r_ij^2,
 *              dL/dc_j = sum_i dl/df_i 2 k_j (H_i - c_j) / r_ij^4
 *   descent    every model value x <- x - lr dL/dx, `epochs` times
 *   anomalies  after the first descent, a control point with k_j < 0 or
 *              outside the convex hull of H (n . c_j > d for some facet
 *              plane, decided in FP32 with single roundings, left to right)
 *              gets k_j = 0 and is not updated by the second descent
 */
#ifndef MI_GS_H
#define MI_GS_H

#include "mi_delbm.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Largest hull and model one fit may have (shared-memory capacity). */
#define MI_GS_MAX_POINTS 10240
#define MI_GS_MAX_BALLS 256

/* Run n_fits refinements asynchronously on `stream` (a cudaStream_t, or
 * NULL for the default stream) on the current device.  All arrays are
 * device arrays owned by the caller:
 *   hull_off, ball_off, plane_off  n_fits + 1 ints each, prefix offsets of
 *                 fit f's rows in hull, balls and planes;
 *   hull          hull points, 3 floats (x, y, z) per row;
 *   balls         control points, 4 floats (x, y, z, k) per row: the start
 *                 model on entry, the refined model on return;
 *   planes        convex-hull facet planes of each fit, 4 floats
 *                 (nx, ny, nz, d) per row, outward unit normal, n . x <= d
 *                 inside;
 *   active        out, one int per ball row: 0 for the points the anomaly
 *                 detection cleared, else 1;
 *   loss          out, 2 floats per fit: L after the first descent and
 *                 after the second.
 * max_points and max_balls bound every fit's hull and model sizes (they size
 * the shared memory; at most MI_GS_MAX_POINTS and MI_GS_MAX_BALLS).  A fit
 * whose sizes exceed them, or that has no points or no balls, is left
 * unchanged with loss NaN.  Errors: MI_EINVAL (n_fits < 0, epochs < 0, lr
 * not finite, a bound out of range, a NULL array with n_fits > 0), MI_ECUDA
 * (launch failure).  Results are deterministic (fixed reduction orders).
 * The call takes n_fits + 1 ints of stream-ordered scratch (the fits'
 * largest-first order and a pick counter) from the device's default memory
 * pool on `stream` and frees them on the same stream. */
mi_status mi_gs_fit(int n_fits, const int *hull_off, const float *hull, const int *ball_off, float *balls,
                    const int *plane_off, const float *planes, int max_points, int max_balls, int epochs,
                    float lr, int *active, float *loss, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* MI_GS_H */
