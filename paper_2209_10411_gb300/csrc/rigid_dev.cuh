// Rigid-body update of one particle for one DEM substep (Sec. 2.3.1), shared
// by the per-substep kernel and the fused DEM substep loop.
#pragma once

#include "mi_internal.cuh"

namespace mi {

// FP64: semi-implicit Euler for the velocity, Euler's equations in the body
// frame, exponential map for the orientation; buoyancy-corrected gravity
// (m - rho0 V) g.  The few particles
// of a step share one warp, whose FP64 instructions issue at a small fraction
// of the FP32 rate on this part, so the chain is kept short: one reciprocal
// per normalisation, rotations from the unit quaternion without a second
// normalisation, and sin(a)/a, cos(a) of the half rotation angle a from their
// Taylor series when a <= 1/64 (terms to a^8: the first omitted term is below
// 2^-53 relative there), the library functions otherwise.
__device__ __forceinline__ void unit_quat_to_R(const double q[4], double R[9]) {
  const double w = q[0], x = q[1], y = q[2], z = q[3];
  R[0] = 1.0 - 2.0 * (y * y + z * z);
  R[1] = 2.0 * (x * y - w * z);
  R[2] = 2.0 * (x * z + w * y);
  R[3] = 2.0 * (x * y + w * z);
  R[4] = 1.0 - 2.0 * (x * x + z * z);
  R[5] = 2.0 * (y * z - w * x);
  R[6] = 2.0 * (x * z - w * y);
  R[7] = 2.0 * (y * z + w * x);
  R[8] = 1.0 - 2.0 * (x * x + y * y);
}

__device__ __forceinline__ void integrate_particle(const IntegrateLaunch& L, int p) {
  DevParticle& P = L.P[p];
  double F[3], T[3];
  for (int a = 0; a < 3; ++a) {
    // sums that other threads built with atomics: read past the L1
    F[a] = (double)__ldcg(L.facc + 6 * p + a) * FIX_INV;
    T[a] = (double)__ldcg(L.facc + 6 * p + 3 + a) * FIX_INV;
    if (L.fc) {
      F[a] += (double)__ldcg(L.fc + 6 * p + a) * FIX_INV;
      T[a] += (double)__ldcg(L.fc + 6 * p + 3 + a) * FIX_INV;
    }
  }
  const double m = P.mass, dt = L.dt;
  const double wg = m - L.rho0 * P.volume;
  const double dtm = dt / m;
  for (int a = 0; a < 3; ++a) P.vel[a] += dtm * (F[a] + wg * L.gravity[a]);
  // rotation at the current pose
  double q[4];
  const double iqn =
      1.0 / sqrt(P.quat[0] * P.quat[0] + P.quat[1] * P.quat[1] + P.quat[2] * P.quat[2] + P.quat[3] * P.quat[3]);
  for (int k = 0; k < 4; ++k) q[k] = P.quat[k] * iqn;
  double R[9];
  unit_quat_to_R(q, R);
  double wb[3], Tb[3];
  for (int a = 0; a < 3; ++a) {
    wb[a] = R[0 + a] * P.omega[0] + R[3 + a] * P.omega[1] + R[6 + a] * P.omega[2];
    Tb[a] = R[0 + a] * T[0] + R[3 + a] * T[1] + R[6 + a] * T[2];
  }
  const double* I = P.inertia;
  const double* Ii = P.inv_inertia;
  double Iw[3], rhs[3];
  for (int a = 0; a < 3; ++a) Iw[a] = I[3 * a] * wb[0] + I[3 * a + 1] * wb[1] + I[3 * a + 2] * wb[2];
  rhs[0] = Tb[0] - (wb[1] * Iw[2] - wb[2] * Iw[1]);
  rhs[1] = Tb[1] - (wb[2] * Iw[0] - wb[0] * Iw[2]);
  rhs[2] = Tb[2] - (wb[0] * Iw[1] - wb[1] * Iw[0]);
  for (int a = 0; a < 3; ++a) wb[a] += dt * (Ii[3 * a] * rhs[0] + Ii[3 * a + 1] * rhs[1] + Ii[3 * a + 2] * rhs[2]);
  // q <- normalize(q (x) exp(wb dt / 2)): dq = (cos a, (sin a / a) wb dt / 2), a = |wb| dt / 2
  const double th[3] = {wb[0] * dt, wb[1] * dt, wb[2] * dt};
  const double a2 = 0.25 * (th[0] * th[0] + th[1] * th[1] + th[2] * th[2]);
  double c, sa;  // cos a, sin(a) / a
  if (a2 <= 1.0 / 4096.0) {
    c = 1.0 + a2 * (-1.0 / 2 + a2 * (1.0 / 24 + a2 * (-1.0 / 720 + a2 * (1.0 / 40320))));
    sa = 1.0 + a2 * (-1.0 / 6 + a2 * (1.0 / 120 + a2 * (-1.0 / 5040 + a2 * (1.0 / 362880))));
  } else {
    const double an = sqrt(a2);
    c = cos(an);
    sa = sin(an) / an;
  }
  const double sn = 0.5 * sa;
  const double dq[4] = {c, sn * th[0], sn * th[1], sn * th[2]};
  double r[4];
  r[0] = q[0] * dq[0] - q[1] * dq[1] - q[2] * dq[2] - q[3] * dq[3];
  r[1] = q[0] * dq[1] + q[1] * dq[0] + q[2] * dq[3] - q[3] * dq[2];
  r[2] = q[0] * dq[2] - q[1] * dq[3] + q[2] * dq[0] + q[3] * dq[1];
  r[3] = q[0] * dq[3] + q[1] * dq[2] - q[2] * dq[1] + q[3] * dq[0];
  const double irn = 1.0 / sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2] + r[3] * r[3]);
  for (int k = 0; k < 4; ++k) {
    r[k] *= irn;
    P.quat[k] = r[k];
  }
  unit_quat_to_R(r, R);
  for (int a = 0; a < 3; ++a) P.omega[a] = R[3 * a] * wb[0] + R[3 * a + 1] * wb[1] + R[3 * a + 2] * wb[2];
  for (int a = 0; a < 3; ++a) P.pos[a] += dt * P.vel[a];
}

}  // namespace mi
