// Rigid-body update of one particle for one DEM substep (Sec. 2.3.1), shared
// by the per-substep kernel and the fused DEM substep loop.
#pragma once

#include "mi_internal.cuh"

namespace mi {

// FP64: semi-implicit Euler for the velocity, Euler's equations in the body
// frame, exponential map for the orientation; buoyancy-corrected gravity
// (m - rho0 V) g.  FP64 instructions issue at a small fraction of the FP32
// rate on this part and the update of one particle is one long dependent
// chain, so four lanes of a warp share it: lane a < 3 owns component a of
// every 3-vector (its column of R for R^T v, its row for R v), lane c < 4
// component c of the quaternion product, and the few values a lane needs
// from the others come by shuffles; scalars (norms, the half-angle series)
// are computed alike in the four lanes.  Rotations use
// R = (w^2 - v.v) I + 2 v v^T + 2 w [v]x of the unit quaternion (w, v);
// sin(a)/a and cos(a) of the half rotation angle a come from their Taylor
// series when a <= 1/64 (terms to a^8: the first omitted term is below 2^-53
// relative there), from the library functions otherwise.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double pick3(int a, double x, double y, double z) { return a == 0 ? x : (a == 1 ? y : z); }

// Lanes 0-3 of a warp update particle p (the other lanes return at once).
__device__ __forceinline__ void integrate_particle_lanes(const IntegrateLaunch& L, int p, int lane) {
  if (lane >= 4) return;
  constexpr unsigned M4 = 0xfu;
  DevParticle& P = L.P[p];
  const int a = lane < 3 ? lane : 2;  // lane 3 repeats component z and stores no 3-vector
  const int a1 = a == 2 ? 0 : a + 1, a2 = a == 0 ? 2 : a - 1;
  // force and torque: fixed-point sums that other threads built with atomics, read past the L1
  double F = (double)__ldcg(L.facc + 6 * p + a) * FIX_INV;
  double T = (double)__ldcg(L.facc + 6 * p + 3 + a) * FIX_INV;
  if (L.fc) {
    F += (double)__ldcg(L.fc + 6 * p + a) * FIX_INV;
    T += (double)__ldcg(L.fc + 6 * p + 3 + a) * FIX_INV;
  }
  const double m = P.mass, dt = L.dt;
  const double wg = m - L.rho0 * P.volume;
  const double vel = P.vel[a] + dt / m * (F + wg * L.gravity[a]);
  // unit quaternion of the current pose (w, v) and column a of its rotation
  const double q0 = P.quat[0], q1 = P.quat[1], q2 = P.quat[2], q3 = P.quat[3];
  const double iqn = 1.0 / sqrt(q0 * q0 + q1 * q1 + q2 * q2 + q3 * q3);
  const double w = q0 * iqn, vx = q1 * iqn, vy = q2 * iqn, vz = q3 * iqn;
  const double s = w * w - (vx * vx + vy * vy + vz * vz);
  const double va = pick3(a, vx, vy, vz), va1 = pick3(a1, vx, vy, vz), va2 = pick3(a2, vx, vy, vz);
  const double C_a = s + 2.0 * va * va;               // R[a][a]
  const double C_a1 = 2.0 * (va1 * va + w * va2);     // R[a1][a]
  const double C_a2 = 2.0 * (va2 * va - w * va1);     // R[a2][a]
  // body-frame angular velocity and torque: (R^T x)_a = R[a][a] x_a + R[a1][a] x_a1 + R[a2][a] x_a2
  const double om_a = P.omega[a], om_a1 = P.omega[a1], om_a2 = P.omega[a2];
  const double T_a1 = __shfl_sync(M4, T, a1), T_a2 = __shfl_sync(M4, T, a2);
  double wb = C_a * om_a + C_a1 * om_a1 + C_a2 * om_a2;
  const double Tb = C_a * T + C_a1 * T_a1 + C_a2 * T_a2;
  const double wb0 = __shfl_sync(M4, wb, 0), wb1 = __shfl_sync(M4, wb, 1), wb2 = __shfl_sync(M4, wb, 2);
  const double* I = P.inertia;
  const double* Ii = P.inv_inertia;
  const double Iw = I[3 * a] * wb0 + I[3 * a + 1] * wb1 + I[3 * a + 2] * wb2;
  const double Iw_a1 = __shfl_sync(M4, Iw, a1), Iw_a2 = __shfl_sync(M4, Iw, a2);
  const double wb_a1 = pick3(a1, wb0, wb1, wb2), wb_a2 = pick3(a2, wb0, wb1, wb2);
  const double rhs = Tb - (wb_a1 * Iw_a2 - wb_a2 * Iw_a1);
  const double r0 = __shfl_sync(M4, rhs, 0), r1 = __shfl_sync(M4, rhs, 1), r2 = __shfl_sync(M4, rhs, 2);
  wb += dt * (Ii[3 * a] * r0 + Ii[3 * a + 1] * r1 + Ii[3 * a + 2] * r2);
  // q <- normalize(q (x) exp(wb dt / 2)): dq = (cos h, (sin h / h) wb dt / 2), h = |wb| dt / 2
  const double th = wb * dt;
  const double t0 = __shfl_sync(M4, th, 0), t1 = __shfl_sync(M4, th, 1), t2 = __shfl_sync(M4, th, 2);
  const double h2 = 0.25 * (t0 * t0 + t1 * t1 + t2 * t2);
  double c, sa;  // cos h, sin(h) / h
  if (h2 <= 1.0 / 4096.0) {
    c = 1.0 + h2 * (-1.0 / 2 + h2 * (1.0 / 24 + h2 * (-1.0 / 720 + h2 * (1.0 / 40320))));
    sa = 1.0 + h2 * (-1.0 / 6 + h2 * (1.0 / 120 + h2 * (-1.0 / 5040 + h2 * (1.0 / 362880))));
  } else {
    const double hn = sqrt(h2);
    c = cos(hn);
    sa = sin(hn) / hn;
  }
  const double sn = 0.5 * sa;
  const double d0 = c, d1 = sn * t0, d2 = sn * t1, d3 = sn * t2;
  // component `lane` of q (x) dq: sum over k of sign * q_k * dq_perm(k)
  const int cq = lane;
  const double e0 = cq == 0 ? d0 : (cq == 1 ? d1 : (cq == 2 ? d2 : d3));   // with q0, sign +
  const double e1 = cq == 0 ? -d1 : (cq == 1 ? d0 : (cq == 2 ? -d3 : d2));  // with q1
  const double e2 = cq == 0 ? -d2 : (cq == 1 ? d3 : (cq == 2 ? d0 : -d1));  // with q2
  const double e3 = cq == 0 ? -d3 : (cq == 1 ? -d2 : (cq == 2 ? d1 : d0));  // with q3
  double r = w * e0 + vx * e1 + vy * e2 + vz * e3;
  const double n0 = __shfl_sync(M4, r, 0), n1 = __shfl_sync(M4, r, 1), n2 = __shfl_sync(M4, r, 2),
               n3 = __shfl_sync(M4, r, 3);
  const double irn = 1.0 / sqrt(n0 * n0 + n1 * n1 + n2 * n2 + n3 * n3);
  r *= irn;
  P.quat[cq] = r;
  // new angular velocity in the world frame: row a of the new rotation times wb
  const double W = n0 * irn, X = n1 * irn, Y = n2 * irn, Z = n3 * irn;
  const double s2 = W * W - (X * X + Y * Y + Z * Z);
  const double ua = pick3(a, X, Y, Z), ua1 = pick3(a1, X, Y, Z), ua2 = pick3(a2, X, Y, Z);
  const double wn0 = __shfl_sync(M4, wb, 0), wn1 = __shfl_sync(M4, wb, 1), wn2 = __shfl_sync(M4, wb, 2);
  const double wn_a = pick3(a, wn0, wn1, wn2), wn_a1 = pick3(a1, wn0, wn1, wn2), wn_a2 = pick3(a2, wn0, wn1, wn2);
  const double omega = (s2 + 2.0 * ua * ua) * wn_a + 2.0 * (ua * ua1 - W * ua2) * wn_a1 + 2.0 * (ua * ua2 + W * ua1) * wn_a2;
  if (lane < 3) {
    P.vel[a] = vel;
    P.omega[a] = omega;
    P.pos[a] += dt * vel;
  }
}

}  // namespace mi
