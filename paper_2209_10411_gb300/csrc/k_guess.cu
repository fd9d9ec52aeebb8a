// Learned Newton guess for the closest-point solve (the plain Newton-Raphson
// of Sec. 2.3.1 still decides every point): the feature kernel for the candidate pairs of
// a DEM substep, and the batch solver of explicitly posed pairs that makes the
// training data (features, plain solves, labels) and compares plain and
// learned starts on the same pairs.  One warp per pair, as in k_contacts.
#include "contact_dev.cuh"

namespace mi {
namespace {
using namespace cdev;

constexpr int WARPS = 4;

// Features of every particle-pair candidate of the substep (rows of wall
// candidates are left alone: walls always start from the plain guess).
__global__ void __launch_bounds__(WARPS * 32, 6) k_item_features(ContactLaunch L) {
  __shared__ float sh[WARPS][64];
  __shared__ float4 stage[WARPS][2][PG_CAP];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned n_items = min(L.ctr->n_pairs, L.cap_items);
  for (unsigned it = blockIdx.x * WARPS + w; it < n_items; it += gridDim.x * WARPS) {
    const int i = L.item_i[it], j = L.item_j[it];
    if (j < 0) continue;
    const DevParticle& Pi = L.P[i];
    const DevParticle& Pj = L.P[j];
    const float4 hi_i = L.pf[i], hi_j = L.pf[j], lo_i = L.plo[i], lo_j = L.plo[j];
    const float h[3] = {0.5f * ((hi_j.x - hi_i.x) + (lo_j.x - lo_i.x)), 0.5f * ((hi_j.y - hi_i.y) + (lo_j.y - lo_i.y)),
                        0.5f * ((hi_j.z - hi_i.z) + (lo_j.z - lo_i.z))};
    const float4 qi = L.qf[i], qj = L.qf[j];
    Frame F0, F1;
    pair_frames(Pi, Pj, qi, qj, h, F0, F1);
    float ya[3];
    pair_features_staged(Pi, Pj, h, qi, qj, F0, F1, L.balls, lane, sh[w], L.feat + (size_t)it * 64, ya, stage[w][0],
                         stage[w][1]);
  }
}

__global__ void __launch_bounds__(WARPS * 32) k_pair_solve(PairSolveLaunch S) {
  __shared__ float sh[WARPS][64];
  __shared__ unsigned short sub[WARPS][2][SUB_CAP];
  __shared__ float4 stage[WARPS][NT_CAP];
  __shared__ float rad[WARPS][NT_CAP];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int p = blockIdx.x * WARPS + w; p < S.n; p += gridDim.x * WARPS) {
    const int i = S.ij[2 * p], j = S.ij[2 * p + 1];
    if (i < 0 || j < 0 || i >= S.np || j >= S.np) {
      if (lane == 0) S.status[p] = 5;
      continue;
    }
    const DevParticle& Pi = S.P[i];
    const DevParticle& Pj = S.P[j];
    const double* pose = S.poses + (size_t)14 * p;
    const double *posi = pose, *qi = pose + 3, *posj = pose + 7, *qj = pose + 10;
    double O[3];
    float h[3];
    for (int a = 0; a < 3; ++a) {
      O[a] = 0.5 * (posi[a] + posj[a]);
      h[a] = (float)(0.5 * (posj[a] - posi[a]));
    }
    const float4 q0 = unit_quat_f32(qi), q1 = unit_quat_f32(qj);
    Frame F0, F1;
    pair_frames(Pi, Pj, q0, q1, h, F0, F1);
    const float Rb = fmaxf(Pi.Rb_f, Pj.Rb_f);
    float ya[3] = {0.f, 0.f, 0.f}, y[3];
    if (S.flags & MI_PAIR_FEATURES) {
      pair_features_staged(Pi, Pj, h, q0, q1, F0, F1, S.balls, lane, sh[w], S.X + (size_t)64 * p, ya, stage[w],
                           stage[w] + PG_CAP);
    } else if (S.flags & MI_PAIR_LEARNED) {
      for (int c = 0; c < 3; ++c) ya[c] = Rb * S.X[(size_t)64 * p + 11 + c];
    } else {
      anchor_guess(F0, F1, S.balls, lane, ya);
    }
    int status = -1;
    SolveCount sc = {0, 0, 0};
    if (!(S.flags & (MI_PAIR_LEARNED | MI_PAIR_PLAIN))) continue;  // features only
    __syncwarp();  // the features' use of the buffer is over
    const PairSolver PS(F0, F1, S.balls, stage[w], rad[w], &sub[w][0][0], lane);
    if (S.flags & MI_PAIR_LEARNED) {
      const float a[3] = {ya[0] / Rb, ya[1] / Rb, ya[2] / Rb};
      const float* pr = S.pred + (size_t)4 * p;
      const float d[4] = {pr[0], pr[1], pr[2], pr[3]};
      status = PS.learned(a, d, Rb, Rb, sub[w][0], sub[w][1], y, sc);
    } else if (S.flags & MI_PAIR_GUESS_ONLY) {
      PS.plain(y);
      if (lane == 0) {
        for (int c = 0; c < 3; ++c) S.xm[(size_t)3 * p + c] = O[c] + (double)y[c];
        S.iters[p] = 0;
        S.evals[p] = 0;
        S.status[p] = 0;
      }
      continue;
    } else {
      status = PS.plain_newton(y, NEWTON_TOL * Rb, sc.iters);
      sc.evals = sc.iters * (F0.n + F1.n);
    }
    GEval e0, e1;
    PS.final_eval(y, e0.g, e0.gr, e1.g, e1.gr);
    if (status == 0) {
      if (e0.g >= 1.f || e1.g >= 1.f) status = 3;
      else if (e0.g < C_TOL || e1.g < C_TOL) status = 4;
    }
    if ((S.flags & MI_PAIR_LABELS) && status == 0) pair_labels(F0, F1, S.balls, lane, y, ya, Rb, S.T + (size_t)4 * p);
    if (lane == 0) {
      for (int c = 0; c < 3; ++c) S.xm[(size_t)3 * p + c] = O[c] + (double)y[c];
      S.iters[p] = sc.iters;
      S.evals[p] = sc.evals;
      S.status[p] = status + (sc.fallback ? 16 : 0);
    }
  }
}

}  // namespace

cudaError_t launch_item_features(const ContactLaunch& L, cudaStream_t s) {
  k_item_features<<<L.grid, WARPS * 32, 0, s>>>(L);
  return cudaGetLastError();
}

cudaError_t launch_pair_solve(const PairSolveLaunch& S, cudaStream_t s) {
  if (S.n <= 0) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  long long blocks = ((long long)S.n + WARPS - 1) / WARPS;
  const long long cap = (long long)(sms > 0 ? sms : 1) * 16;
  if (blocks > cap) blocks = cap;
  k_pair_solve<<<(unsigned)blocks, WARPS * 32, 0, s>>>(S);
  return cudaGetLastError();
}

}  // namespace mi
