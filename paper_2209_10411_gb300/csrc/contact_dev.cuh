// Device-side pieces of the closest-point solve between sphero-metaball
// particles (Sec. 2.3.1), shared by the DEM contact kernel and the batch pair
// solver: the warp-cooperative core field with gradient and Hessian, the small
// dense solve, the starting guesses and the Newton iteration.  One warp works
// on one pair: the balls are spread over the lanes, the sums are
// shuffle-reduced and broadcast from lane 0, so every lane takes the same
// branches.  Geometry is FP32 in a local frame centred between the particles.
#pragma once

#include "mi_internal.cuh"

namespace mi {
namespace cdev {
constexpr unsigned FULL = 0xffffffffu;
constexpr int MAX_IT = 50;
constexpr float C_TOL = 1e-6f;
constexpr float NEWTON_TOL = 1e-5f;  // |dx| <= NEWTON_TOL * R_b,max

__device__ __forceinline__ float wsum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return __shfl_sync(FULL, v, 0);
}

// Order-preserving map of a float onto an unsigned key (-0 and +0 equal).
__device__ __forceinline__ unsigned fkey(float f) {
  const unsigned u = __float_as_uint(f + 0.0f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// Warp argmin: the smallest i among the lanes holding the smallest v (two
// integer warp reductions); the same in every lane.
__device__ __forceinline__ unsigned warp_argmin(float v, unsigned i) {
  const unsigned k = fkey(v);
  const unsigned m = __reduce_min_sync(FULL, k);
  return __reduce_min_sync(FULL, k == m ? i : 0xffffffffu);
}


// A particle seen from a local origin O: body point x_b = R^T y + o for local y.
struct Frame {
  float R[9];  // body -> world
  float o[3];  // R^T (O - X)
  float t[3];  // X - O (world offset of the particle origin)
  float s;     // core scale
  int off, n;
};

// Unit quaternion in FP32 (w, x, y, z) of an FP64 one.
__device__ __forceinline__ float4 unit_quat_f32(const double q[4]) {
  const float a = (float)q[0], b = (float)q[1], c = (float)q[2], d = (float)q[3];
  const float inv = 1.0f / sqrtf(a * a + b * b + c * c + d * d);
  return make_float4(a * inv, b * inv, c * inv, d * inv);
}

// The frame of particle P for a local origin O, given its unit quaternion q
// and the offset d = O - X, both FP32.  The geometry the frame serves is
// FP32; the callers take only the difference of two particle positions in
// FP64 before rounding, so that positions far from the origin keep their
// relative accuracy.  (FP64 runs at a small fraction of the FP32 rate on this
// part, and every candidate pair builds two frames.)
__device__ __forceinline__ Frame frame_f32(const DevParticle& P, const float4 q, const float d[3]) {
  Frame F;
  const float w = q.x, x = q.y, y = q.z, z = q.w;
  float* R = F.R;
  R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z);       R[2] = 2.f * (x * z + w * y);
  R[3] = 2.f * (x * y + w * z);       R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
  R[6] = 2.f * (x * z - w * y);       R[7] = 2.f * (y * z + w * x);       R[8] = 1.f - 2.f * (x * x + y * y);
  for (int a = 0; a < 3; ++a) {
    F.o[a] = R[a] * d[0] + R[3 + a] * d[1] + R[6 + a] * d[2];
    F.t[a] = -d[a];
  }
  F.s = P.core_s;
  F.off = P.ball_off;
  F.n = P.n_balls;
  return F;
}

// The two frames of a pair about O = (X_i + X_j) / 2 from h = (X_j - X_i) / 2
// (O - X_i = h, O - X_j = -h).
__device__ __forceinline__ void pair_frames(const DevParticle& Pi, const DevParticle& Pj, const float4 qi,
                                            const float4 qj, const float h[3], Frame& F0, Frame& F1) {
  const float mh[3] = {-h[0], -h[1], -h[2]};
  F0 = frame_f32(Pi, qi, h);
  F1 = frame_f32(Pj, qj, mh);
}

struct GEval {
  float g, gr[3], H[6];  // core value, world gradient, world Hessian (xx xy xz yy yz zz)
};

// Warp-cooperative g, grad g, Hessian of g at local point y (every lane passes
// the same y), over every ball of the particle or, with a list, over the m
// balls it names (an active subset).
__device__ __forceinline__ GEval eval(const Frame& F, const float4* __restrict__ balls, const float y[3], int lane,
                                      const unsigned short* list = nullptr, int m = 0) {
  float xb[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) xb[a] = F.R[a] * y[0] + F.R[3 + a] * y[1] + F.R[6 + a] * y[2] + F.o[a];
  float g = 0.f, gb0 = 0.f, gb1 = 0.f, gb2 = 0.f, h0 = 0.f, h1 = 0.f, h2 = 0.f, h3 = 0.f, h4 = 0.f, h5 = 0.f;
  const int cnt = list ? m : F.n;
  for (int u = lane; u < cnt; u += 32) {
    const int b = list ? (int)list[u] : u;
    const float4 c = __ldg(balls + F.off + b);
    const float d0 = xb[0] - c.x, d1 = xb[1] - c.y, d2 = xb[2] - c.z;
    const float ir2 = 1.0f / (d0 * d0 + d1 * d1 + d2 * d2);
    const float t = c.w * ir2;            // k / r^2
    const float t2 = -2.0f * t * ir2;     // -2 k / r^4
    const float t3 = 8.0f * t * ir2 * ir2;  // 8 k / r^6
    g += t;
    gb0 += t2 * d0;
    gb1 += t2 * d1;
    gb2 += t2 * d2;
    h0 += t3 * d0 * d0 + t2;
    h1 += t3 * d0 * d1;
    h2 += t3 * d0 * d2;
    h3 += t3 * d1 * d1 + t2;
    h4 += t3 * d1 * d2;
    h5 += t3 * d2 * d2 + t2;
  }
  g = wsum(g);
  gb0 = wsum(gb0); gb1 = wsum(gb1); gb2 = wsum(gb2);
  h0 = wsum(h0); h1 = wsum(h1); h2 = wsum(h2); h3 = wsum(h3); h4 = wsum(h4); h5 = wsum(h5);
  GEval e;
  const float s = F.s;
  e.g = s * g;
  const float* R = F.R;
  for (int a = 0; a < 3; ++a) e.gr[a] = s * (R[3 * a] * gb0 + R[3 * a + 1] * gb1 + R[3 * a + 2] * gb2);
  // H_w = R H_b R^T
  const float Hb[3][3] = {{h0, h1, h2}, {h1, h3, h4}, {h2, h4, h5}};
  float M[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) M[a][b] = R[3 * a] * Hb[0][b] + R[3 * a + 1] * Hb[1][b] + R[3 * a + 2] * Hb[2][b];
  float Hw[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) Hw[a][b] = s * (M[a][0] * R[3 * b] + M[a][1] * R[3 * b + 1] + M[a][2] * R[3 * b + 2]);
  e.H[0] = Hw[0][0]; e.H[1] = Hw[0][1]; e.H[2] = Hw[0][2];
  e.H[3] = Hw[1][1]; e.H[4] = Hw[1][2]; e.H[5] = Hw[2][2];
  return e;
}

// Gaussian elimination with partial pivoting (n <= 4); false if singular.
// The pivot search swaps row i with each later row whose entry in column i
// is larger in magnitude than the current pivot: the pivot chosen is the
// first largest, and every index is a compile-time constant, so the system
// stays in registers.  Each pivot is inverted once (correctly rounded) and
// its row's multipliers and unknown are products with that reciprocal.
template <int N>
__device__ __forceinline__ bool solve(float A[N][N], float b[N], float x[N]) {
  float ip[N];
#pragma unroll
  for (int i = 0; i < N; ++i) {
#pragma unroll
    for (int r = i + 1; r < N; ++r) {
      if (fabsf(A[r][i]) > fabsf(A[i][i])) {
#pragma unroll
        for (int c = i; c < N; ++c) { const float t = A[i][c]; A[i][c] = A[r][c]; A[r][c] = t; }
        const float t = b[i]; b[i] = b[r]; b[r] = t;
      }
    }
    if (!(fabsf(A[i][i]) > 0.f)) return false;
    ip[i] = __frcp_rn(A[i][i]);
#pragma unroll
    for (int r = i + 1; r < N; ++r) {
      const float m = A[r][i] * ip[i];
#pragma unroll
      for (int c = i; c < N; ++c) A[r][c] -= m * A[i][c];
      b[r] -= m * b[i];
    }
  }
#pragma unroll
  for (int i = N - 1; i >= 0; --i) {
    float acc = b[i];
#pragma unroll
    for (int c = i + 1; c < N; ++c) acc -= A[i][c] * x[c];
    x[i] = acc * ip[i];
  }
  return isfinite(x[0]) && isfinite(x[1]) && isfinite(x[2]) && (N < 4 || isfinite(x[N - 1]));
}

// Centre of ball c in the local frame.
__device__ __forceinline__ void ball_local(const Frame& F, const float4 c, float p[3]) {
#pragma unroll
  for (int k = 0; k < 3; ++k) p[k] = F.R[3 * k] * c.x + F.R[3 * k + 1] * c.y + F.R[3 * k + 2] * c.z + F.t[k];
}

// Midpoint of the surface points of ball a of F0 and ball b of F1 (spheres of
// radius sqrt k) on the line joining their centres.
__device__ __forceinline__ void sphere_midpoint(const Frame& F0, const Frame& F1, const float4* __restrict__ balls,
                                                int a, int b, float y[3]) {
  const float4 ca = __ldg(balls + F0.off + a), cb = __ldg(balls + F1.off + b);
  float pa[3], pb[3], u[3];
  ball_local(F0, ca, pa);
  ball_local(F1, cb, pb);
  for (int c = 0; c < 3; ++c) u[c] = pb[c] - pa[c];
  const float D = sqrtf(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  if (D > 0.f) for (int c = 0; c < 3; ++c) u[c] /= D;
  else { u[0] = 1.f; u[1] = u[2] = 0.f; }
  const float ra = sqrtf(ca.w), rb = sqrtf(cb.w);
  for (int c = 0; c < 3; ++c) y[c] = 0.5f * ((pa[c] + ra * u[c]) + (pb[c] - rb * u[c]));
}

constexpr int PG_CAP = 128;  // balls of particle 1 the plain guess stages in shared memory

// Plain starting guess: the closest pair of control-point spheres (smallest
// surface gap, ties to the lower (a, b)), O(n0 n1) per pair.  With a warp's
// shared buffer of PG_CAP float4 (and n1 <= PG_CAP), particle 1's spheres
// (local centre, radius) are formed once and read back by broadcast instead
// of being transformed again for every ball of particle 0; the arithmetic
// and the order are the same either way.
static __device__ __noinline__ void plain_guess(const Frame& F0, const Frame& F1, const float4* __restrict__ balls,
                                            int lane, float y[3], float4* stage = nullptr) {
  float best = 3.4e38f;
  int ba = 0, bb = 0;
  if (stage && F1.n <= PG_CAP) {
    for (int b = lane; b < F1.n; b += 32) {
      const float4 cb = __ldg(balls + F1.off + b);
      float pb[3];
      ball_local(F1, cb, pb);
      stage[b] = make_float4(pb[0], pb[1], pb[2], sqrtf(cb.w));
    }
    __syncwarp();
    for (int a = lane; a < F0.n; a += 32) {
      const float4 ca = __ldg(balls + F0.off + a);
      float pa[3];
      ball_local(F0, ca, pa);
      const float ra = sqrtf(ca.w);
      for (int b = 0; b < F1.n; ++b) {
        const float4 q = stage[b];
        const float gap = sqrtf((pa[0] - q.x) * (pa[0] - q.x) + (pa[1] - q.y) * (pa[1] - q.y) +
                                (pa[2] - q.z) * (pa[2] - q.z)) - ra - q.w;
        if (gap < best) { best = gap; ba = a; bb = b; }
      }
    }
    __syncwarp();  // the buffer is free again
  } else {
    for (int a = lane; a < F0.n; a += 32) {
      const float4 ca = __ldg(balls + F0.off + a);
      float pa[3];
      ball_local(F0, ca, pa);
      const float ra = sqrtf(ca.w);
      for (int b = 0; b < F1.n; ++b) {
        const float4 cb = __ldg(balls + F1.off + b);
        float pb[3];
        ball_local(F1, cb, pb);
        const float gap = sqrtf((pa[0] - pb[0]) * (pa[0] - pb[0]) + (pa[1] - pb[1]) * (pa[1] - pb[1]) +
                                (pa[2] - pb[2]) * (pa[2] - pb[2])) - ra - sqrtf(cb.w);
        if (gap < best) { best = gap; ba = a; bb = b; }
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const float g2 = __shfl_xor_sync(FULL, best, o);
    const int a2 = __shfl_xor_sync(FULL, ba, o), b2 = __shfl_xor_sync(FULL, bb, o);
    if (g2 < best || (g2 == best && (a2 < ba || (a2 == ba && b2 < bb)))) { best = g2; ba = a2; bb = b2; }
  }
  ba = __shfl_sync(FULL, ba, 0);
  bb = __shfl_sync(FULL, bb, 0);
  sphere_midpoint(F0, F1, balls, ba, bb, y);
}

// The ball of F whose sphere surface comes closest to the local point tgt:
// argmin |c - tgt| - sqrt k, ties to the lower index (warp-uniform result).
__device__ __forceinline__ int reaching_ball(const Frame& F, const float4* __restrict__ balls, const float tgt[3],
                                             int lane) {
  float best = 3.4e38f;
  int bi = 0x7fffffff;
  for (int b = lane; b < F.n; b += 32) {
    const float4 c = __ldg(balls + F.off + b);
    float p[3];
    ball_local(F, c, p);
    const float gap = sqrtf((p[0] - tgt[0]) * (p[0] - tgt[0]) + (p[1] - tgt[1]) * (p[1] - tgt[1]) +
                            (p[2] - tgt[2]) * (p[2] - tgt[2])) - sqrtf(c.w);
    if (gap < best) { best = gap; bi = b; }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const float g2 = __shfl_xor_sync(FULL, best, o);
    const int b2 = __shfl_xor_sync(FULL, bi, o);
    if (g2 < best || (g2 == best && b2 < bi)) { best = g2; bi = b2; }
  }
  return __shfl_sync(FULL, bi, 0);
}

// Anchor of the learned guess, O(n0 + n1): the ball of particle 0 reaching
// closest to the origin of particle 1 and vice versa, and the midpoint of
// their surface points (the particle origins are F.t in the local frame).
__device__ __forceinline__ void anchor_guess(const Frame& F0, const Frame& F1, const float4* __restrict__ balls,
                                             int lane, float y[3]) {
  const int a = reaching_ball(F0, balls, F1.t, lane);
  const int b = reaching_ball(F1, balls, F0.t, lane);
  sphere_midpoint(F0, F1, balls, a, b, y);
}

// Newton-Raphson on grad(g0 + g1) = 0 (the closest-point condition of the two
// cores) from y, over all balls or over the listed subsets.  Stops when
// |dx| <= tol; returns 0 converged, 1 not converged in max_it, 2 singular;
// iters counts the iterations taken (a failed solve included).
static __device__ __noinline__ int newton_pair(const Frame& F0, const Frame& F1, const float4* __restrict__ balls,
                                           int lane, float y[3], float tol, int max_it, int& iters,
                                           const unsigned short* l0 = nullptr, int m0 = 0,
                                           const unsigned short* l1 = nullptr, int m1 = 0) {
  int status = 1;
  for (iters = 1; iters <= max_it; ++iters) {
    const GEval e0 = eval(F0, balls, y, lane, l0, m0), e1 = eval(F1, balls, y, lane, l1, m1);
    float A[3][3] = {{e0.H[0] + e1.H[0], e0.H[1] + e1.H[1], e0.H[2] + e1.H[2]},
                     {e0.H[1] + e1.H[1], e0.H[3] + e1.H[3], e0.H[4] + e1.H[4]},
                     {e0.H[2] + e1.H[2], e0.H[4] + e1.H[4], e0.H[5] + e1.H[5]}};
    float b[3] = {e0.gr[0] + e1.gr[0], e0.gr[1] + e1.gr[1], e0.gr[2] + e1.gr[2]};
    float dx[3];
    if (!solve<3>(A, b, dx)) { status = 2; break; }
    for (int c = 0; c < 3; ++c) y[c] -= dx[c];
    if (sqrtf(dx[0] * dx[0] + dx[1] * dx[1] + dx[2] * dx[2]) <= tol) { status = 0; break; }
  }
  if (iters > max_it) iters = max_it;
  return status;
}

constexpr int SUB_CAP = 128;   // largest active subset per particle kept in shared memory
constexpr int SUB_IT = 3;      // subset Newton iterations at most
constexpr float SUB_TOL = 1e-3f;  // subset stop: |dx| <= SUB_TOL * R_b,max (a coarse pre-solve)

// Indices of the balls of F whose centre lies within r of y, compacted into
// list (warp ballot); returns their count (which may exceed SUB_CAP: then the
// list holds only the first SUB_CAP).
__device__ __forceinline__ int active_subset(const Frame& F, const float4* __restrict__ balls, const float y[3],
                                             float r, int lane, unsigned short* list) {
  int cnt = 0;
  const float r2 = r * r;
  for (int base = 0; base < F.n; base += 32) {
    const int b = base + lane;
    bool in = false;
    if (b < F.n) {
      float p[3];
      ball_local(F, __ldg(balls + F.off + b), p);
      const float d2 = (p[0] - y[0]) * (p[0] - y[0]) + (p[1] - y[1]) * (p[1] - y[1]) + (p[2] - y[2]) * (p[2] - y[2]);
      in = d2 <= r2;
    }
    const unsigned m = __ballot_sync(FULL, in);
    const int pos = cnt + __popc(m & ((1u << lane) - 1u));
    if (in && pos < SUB_CAP) list[pos] = (unsigned short)b;
    cnt += __popc(m);
  }
  __syncwarp();
  return cnt;
}

struct SolveCount {
  int iters;       // Newton iterations: subset + full set (+ plain fallback)
  int evals;       // ball evaluations of those iterations (one per ball per iteration)
  int fallback;    // 1 when the learned start failed and plain Newton took over
};

// Learned start: y0 = L (a + d), with a the anchor / L and d the predicted
// offset; active subset = balls within r_act = L exp(log_r) of y0.  Newton
// runs on the subsets first when that at least halves the work of an
// iteration (both non-empty, within SUB_CAP, together at most half the
// balls), for at most SUB_IT iterations to the coarse SUB_TOL, and its point
// is kept only if it converged; then on the full set to the plain tolerance.
// If the full-set solve fails, plain Newton from the plain guess decides.
static __device__ __noinline__ int learned_newton(const Frame& F0, const Frame& F1, const float4* __restrict__ balls,
                                              int lane, const float a[3], const float d[4], float L, float Rb,
                                              unsigned short* l0, unsigned short* l1, float y[3], SolveCount& sc,
                                              float4* stage = nullptr) {
  sc.iters = sc.evals = sc.fallback = 0;
  for (int c = 0; c < 3; ++c) y[c] = L * (a[c] + d[c]);
  bool ok = isfinite(y[0]) && isfinite(y[1]) && isfinite(y[2]);
  if (ok) {
    const float r_act = L * expf(fminf(fmaxf(d[3], -8.f), 2.f));
    const int m0 = active_subset(F0, balls, y, r_act, lane, l0);
    const int m1 = active_subset(F1, balls, y, r_act, lane, l1);
    if (m0 > 0 && m1 > 0 && m0 <= SUB_CAP && m1 <= SUB_CAP && 2 * (m0 + m1) <= F0.n + F1.n) {
      float ys[3] = {y[0], y[1], y[2]};
      int it = 0;
      const int st = newton_pair(F0, F1, balls, lane, ys, SUB_TOL * Rb, SUB_IT, it, l0, m0, l1, m1);
      sc.iters += it;
      sc.evals += it * (m0 + m1);
      if (st == 0)
        for (int c = 0; c < 3; ++c) y[c] = ys[c];
    }
    int it = 0;
    const int st = newton_pair(F0, F1, balls, lane, y, NEWTON_TOL * Rb, MAX_IT, it);
    sc.iters += it;
    sc.evals += it * (F0.n + F1.n);
    ok = st == 0;
  }
  if (ok) return 0;
  sc.fallback = 1;
  plain_guess(F0, F1, balls, lane, y, stage);
  int it = 0;
  const int st = newton_pair(F0, F1, balls, lane, y, NEWTON_TOL * Rb, MAX_IT, it);
  sc.iters += it;
  sc.evals += it * (F0.n + F1.n);
  return st;
}

constexpr int NEAREST = 5;     // nearest balls per particle in the features
constexpr float ACT_FRAC = 0.99f;  // share of g0 + g1 the active radius label must carry

// One pass over the balls of F around the local point y: the core field
// g(y) = s sum k / |c - y|^2 (warp sum, broadcast) and the NEAREST balls
// closest to y, ties to the lower index, written by lane 0 into row[4 r ..]
// as (c - y) / L and log(s k / L^2), zeros when F has fewer balls.  Each lane
// keeps a sorted list of its own nearest balls in registers; NEAREST rounds
// of a warp argmin over the lanes' list heads then merge them.
__device__ __forceinline__ float field_and_nearest(const Frame& F, const float4* __restrict__ balls, const float y[3],
                                                   float iL, int lane, float* row) {
  float kd[NEAREST];
  int kb[NEAREST];
#pragma unroll
  for (int r = 0; r < NEAREST; ++r) { kd[r] = 3.4e38f; kb[r] = 0x7fffffff; }
  float g = 0.f;
  for (int b = lane; b < F.n; b += 32) {
    const float4 c = __ldg(balls + F.off + b);
    float p[3];
    ball_local(F, c, p);
    const float d2 = (p[0] - y[0]) * (p[0] - y[0]) + (p[1] - y[1]) * (p[1] - y[1]) + (p[2] - y[2]) * (p[2] - y[2]);
    g += c.w / d2;
    float cd = sqrtf(d2);
    int cb = b;
#pragma unroll
    for (int r = 0; r < NEAREST; ++r)  // this lane's balls arrive in index order: strict < keeps ties in order
      if (cd < kd[r]) {
        const float td = kd[r]; kd[r] = cd; cd = td;
        const int tb = kb[r]; kb[r] = cb; cb = tb;
      }
  }
  g = F.s * wsum(g);
  for (int r = 0; r < NEAREST; ++r) {
    float best = kd[0];
    int bi = kb[0];
    for (int o = 16; o > 0; o >>= 1) {
      const float d2 = __shfl_xor_sync(FULL, best, o);
      const int b2 = __shfl_xor_sync(FULL, bi, o);
      if (d2 < best || (d2 == best && b2 < bi)) { best = d2; bi = b2; }
    }
    bi = __shfl_sync(FULL, bi, 0);
    if (kb[0] == bi && bi != 0x7fffffff) {  // the owning lane pops its head
#pragma unroll
      for (int q = 0; q < NEAREST - 1; ++q) { kd[q] = kd[q + 1]; kb[q] = kb[q + 1]; }
      kd[NEAREST - 1] = 3.4e38f;
      kb[NEAREST - 1] = 0x7fffffff;
    }
    if (lane == 0) {
      float* out = row + 4 * r;
      if (bi < F.n) {
        const float4 c = __ldg(balls + F.off + bi);
        float p[3];
        ball_local(F, c, p);
        for (int k = 0; k < 3; ++k) out[k] = (p[k] - y[k]) * iL;
        out[3] = logf(F.s * c.w * iL * iL);
      } else {
        out[0] = out[1] = out[2] = out[3] = 0.f;
      }
    }
  }
  return g;
}

// The 64 features of a candidate pair (lengths / L, L = max R_b, positions
// relative to the pair centre O; the layout of the learned-guess oracle):
// 0:3 (X_j - X_i)/L, 3:11 unit quaternions with w >= 0, 11:14 anchor, 14:16
// log g at the anchor, then per particle (16:40, 40:64) log(n)/5,
// log(sum k / L^2), R_b/L, R_s/L and the 5 balls nearest the anchor (ties to
// the lower index; zeros when fewer) as (c - x_a)/L and log(s k / L^2).
// Lane 0 fills the warp's shared row sh, the warp stores it to out; ya
// returns the anchor in the local frame; h = (X_j - X_i) / 2 and the unit
// quaternions are FP32 (the features are FP32 network inputs).
__device__ __forceinline__ void pair_features(const DevParticle& Pi, const DevParticle& Pj, const float h[3],
                                              const float4 qi, const float4 qj, const Frame& F0, const Frame& F1,
                                              const float4* __restrict__ balls, int lane, float* sh, float* out,
                                              float ya[3]) {
  const float L = fmaxf(Pi.Rb_f, Pj.Rb_f);
  const float iL = 1.0f / L;
  anchor_guess(F0, F1, balls, lane, ya);
  const float g0 = field_and_nearest(F0, balls, ya, iL, lane, sh + 20);
  const float g1 = field_and_nearest(F1, balls, ya, iL, lane, sh + 44);
  if (lane == 0) {
    for (int c = 0; c < 3; ++c) sh[c] = 2.0f * h[c] * iL;
    for (int side = 0; side < 2; ++side) {
      const float4 q = side ? qj : qi;
      const float sg = q.x >= 0.f ? 1.f : -1.f;
      sh[3 + 4 * side] = sg * q.x;
      sh[4 + 4 * side] = sg * q.y;
      sh[5 + 4 * side] = sg * q.z;
      sh[6 + 4 * side] = sg * q.w;
    }
    for (int c = 0; c < 3; ++c) sh[11 + c] = ya[c] * iL;
    sh[14] = logf(g0);
    sh[15] = logf(g1);
    for (int side = 0; side < 2; ++side) {
      const Frame& F = side ? F1 : F0;
      const DevParticle& P = side ? Pj : Pi;
      const int off = side ? 40 : 16;
      sh[off] = logf((float)F.n) / 5.0f;
      sh[off + 1] = 2.0f * logf(P.re_f * iL);
      sh[off + 2] = P.Rb_f * iL;
      sh[off + 3] = P.skin_f * iL;
    }
  }
  __syncwarp();
  out[lane] = sh[lane];
  out[lane + 32] = sh[lane + 32];
  __syncwarp();
}

// Distance from y and core weight s k / d^2 of ball t of the pair (balls of
// particle 0 first, then those of particle 1).
__device__ __forceinline__ void ball_weight(const Frame& F0, const Frame& F1, const float4* __restrict__ balls, int t,
                                            const float y[3], float& d, float& w) {
  const Frame& F = t < F0.n ? F0 : F1;
  const int b = t < F0.n ? t : t - F0.n;
  const float4 c = __ldg(balls + F.off + b);
  float p[3];
  ball_local(F, c, p);
  const float d2 = (p[0] - y[0]) * (p[0] - y[0]) + (p[1] - y[1]) * (p[1] - y[1]) + (p[2] - y[2]) * (p[2] - y[2]);
  d = sqrtf(d2);
  w = F.s * c.w / d2;
}

// Training targets of a converged pair: (x_m - x_a)/L and log(r_act/L), with
// r_act the smallest distance from x_m such that the balls no farther away
// (ties by index) carry ACT_FRAC of g0(x_m) + g1(x_m).  O((n0 + n1)^2 / 32)
// per lane: it runs only when training data is generated.
__device__ __forceinline__ void pair_labels(const Frame& F0, const Frame& F1, const float4* __restrict__ balls,
                                            int lane, const float ym[3], const float ya[3], float L, float* out) {
  const int N = F0.n + F1.n;
  float W = 0.f;
  for (int t = lane; t < N; t += 32) {
    float d, w;
    ball_weight(F0, F1, balls, t, ym, d, w);
    W += w;
  }
  W = wsum(W);
  float best = 3.4e38f;
  for (int t = lane; t < N; t += 32) {
    float dt, wt;
    ball_weight(F0, F1, balls, t, ym, dt, wt);
    float cum = 0.f;
    for (int u = 0; u < N; ++u) {
      float du, wu;
      ball_weight(F0, F1, balls, u, ym, du, wu);
      if (du < dt || (du == dt && u <= t)) cum += wu;
    }
    if (cum >= ACT_FRAC * W && dt < best) best = dt;
  }
  for (int o = 16; o > 0; o >>= 1) best = fminf(best, __shfl_xor_sync(FULL, best, o));
  if (lane == 0) {
    for (int c = 0; c < 3; ++c) out[c] = (ym[c] - ya[c]) / L;
    out[3] = logf(best / L);
  }
}

}  // namespace cdev
}  // namespace mi

namespace mi {
namespace cdev {

__device__ __forceinline__ void reaching_staged2(const float4* s0, int n0, const float t0[3], const float4* s1, int n1,
                                                 const float t1[3], int lane, int& a, int& b);
__device__ __forceinline__ void field_nearest_staged2(const float4* s0, int n0, float sc0, const float4* s1, int n1,
                                                      float sc1, const float y[3], float iL, int lane, float* row0,
                                                      float* row1, float& g0, float& g1);

// Staged form of the feature computation: the local centres and k of both
// particles' balls (at most PG_CAP each) are formed once into the warp's
// shared buffers s0, s1 and every scan reads them back; the five nearest-ball
// rows of a particle are written by lanes 0..4 at once.  The values are those
// of pair_features (same operations on the same operands).
// pair_features with both particles staged in s0, s1 (PG_CAP float4 each);
// falls back to pair_features when a particle has more balls.
__device__ __forceinline__ void pair_features_staged(const DevParticle& Pi, const DevParticle& Pj, const float h[3],
                                                     const float4 qi, const float4 qj, const Frame& F0,
                                                     const Frame& F1, const float4* __restrict__ balls, int lane,
                                                     float* sh, float* out, float ya[3], float4* s0, float4* s1) {
  if (F0.n > PG_CAP || F1.n > PG_CAP) {
    pair_features(Pi, Pj, h, qi, qj, F0, F1, balls, lane, sh, out, ya);
    return;
  }
  for (int b = lane; b < F0.n; b += 32) {
    const float4 c = __ldg(balls + F0.off + b);
    float p[3];
    ball_local(F0, c, p);
    s0[b] = make_float4(p[0], p[1], p[2], c.w);
  }
  for (int b = lane; b < F1.n; b += 32) {
    const float4 c = __ldg(balls + F1.off + b);
    float p[3];
    ball_local(F1, c, p);
    s1[b] = make_float4(p[0], p[1], p[2], c.w);
  }
  __syncwarp();
  const float L = fmaxf(Pi.Rb_f, Pj.Rb_f);
  const float iL = 1.0f / L;
  {
    // anchor: the sphere of each particle reaching closest to the other's origin
    int a, b;
    reaching_staged2(s0, F0.n, F1.t, s1, F1.n, F0.t, lane, a, b);
    const float4 pa = s0[a], pb = s1[b];
    float u[3] = {pb.x - pa.x, pb.y - pa.y, pb.z - pa.z};
    const float D = sqrtf(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    if (D > 0.f) for (int c = 0; c < 3; ++c) u[c] /= D;
    else { u[0] = 1.f; u[1] = u[2] = 0.f; }
    const float ra = sqrtf(pa.w), rb = sqrtf(pb.w);
    ya[0] = 0.5f * ((pa.x + ra * u[0]) + (pb.x - rb * u[0]));
    ya[1] = 0.5f * ((pa.y + ra * u[1]) + (pb.y - rb * u[1]));
    ya[2] = 0.5f * ((pa.z + ra * u[2]) + (pb.z - rb * u[2]));
  }
  float g0, g1;
  field_nearest_staged2(s0, F0.n, F0.s, s1, F1.n, F1.s, ya, iL, lane, sh + 20, sh + 44, g0, g1);
  // the six logarithms, one per lane 0-5, written by their lanes
  {
    float arg = 1.f, scale = 1.f;
    int slot = 0;
    if (lane == 0) { arg = g0; slot = 14; }
    else if (lane == 1) { arg = g1; slot = 15; }
    else if (lane == 2) { arg = (float)F0.n; slot = 16; scale = 0.2f; }
    else if (lane == 3) { arg = (float)F1.n; slot = 40; scale = 0.2f; }
    else if (lane == 4) { arg = Pi.re_f * iL; slot = 17; scale = 2.0f; }
    else if (lane == 5) { arg = Pj.re_f * iL; slot = 41; scale = 2.0f; }
    const float lg = logf(arg);
    if (lane < 6) sh[slot] = lane >= 2 && lane < 4 ? lg / 5.0f : scale * lg;
  }
  if (lane == 0) {
    for (int c = 0; c < 3; ++c) sh[c] = 2.0f * h[c] * iL;
    for (int side = 0; side < 2; ++side) {
      const float4 q = side ? qj : qi;
      const float sg = q.x >= 0.f ? 1.f : -1.f;
      sh[3 + 4 * side] = sg * q.x;
      sh[4 + 4 * side] = sg * q.y;
      sh[5 + 4 * side] = sg * q.z;
      sh[6 + 4 * side] = sg * q.w;
    }
    for (int c = 0; c < 3; ++c) sh[11 + c] = ya[c] * iL;
    sh[18] = Pi.Rb_f * iL;
    sh[19] = Pi.skin_f * iL;
    sh[42] = Pj.Rb_f * iL;
    sh[43] = Pj.skin_f * iL;
  }
  __syncwarp();
  out[lane] = sh[lane];
  out[lane + 32] = sh[lane + 32];
  __syncwarp();
}

}  // namespace cdev
}  // namespace mi

namespace mi {
namespace cdev {

// Both particles at once (the same values as two reaching_staged /
// field_nearest_staged calls): the two independent reductions of every step
// are interleaved, which halves the dependent shuffle latency per pair.
__device__ __forceinline__ void argmin2(float& b0, int& i0, float& b1, int& i1) {
  i0 = (int)warp_argmin(b0, (unsigned)i0);
  i1 = (int)warp_argmin(b1, (unsigned)i1);
}

__device__ __forceinline__ void reaching_staged2(const float4* s0, int n0, const float t0[3], const float4* s1, int n1,
                                                 const float t1[3], int lane, int& a, int& b) {
  float b0 = 3.4e38f, b1 = 3.4e38f;
  int i0 = 0x7fffffff, i1 = 0x7fffffff;
  const int n = max(n0, n1);
  for (int k = lane; k < n; k += 32) {
    if (k < n0) {
      const float4 q = s0[k];
      const float gap = sqrtf((q.x - t0[0]) * (q.x - t0[0]) + (q.y - t0[1]) * (q.y - t0[1]) +
                              (q.z - t0[2]) * (q.z - t0[2])) - sqrtf(q.w);
      if (gap < b0) { b0 = gap; i0 = k; }
    }
    if (k < n1) {
      const float4 q = s1[k];
      const float gap = sqrtf((q.x - t1[0]) * (q.x - t1[0]) + (q.y - t1[1]) * (q.y - t1[1]) +
                              (q.z - t1[2]) * (q.z - t1[2])) - sqrtf(q.w);
      if (gap < b1) { b1 = gap; i1 = k; }
    }
  }
  argmin2(b0, i0, b1, i1);
  a = i0;
  b = i1;
}

__device__ __forceinline__ void topk_insert(float (&kd)[NEAREST], int (&kb)[NEAREST], float cd, int cb) {
#pragma unroll
  for (int r = 0; r < NEAREST; ++r)  // a lane's balls arrive in index order: strict < keeps ties in order
    if (cd < kd[r]) {
      const float td = kd[r]; kd[r] = cd; cd = td;
      const int tb = kb[r]; kb[r] = cb; cb = tb;
    }
}

__device__ __forceinline__ void topk_pop(float (&kd)[NEAREST], int (&kb)[NEAREST], int bi) {
  if (kb[0] == bi && bi != 0x7fffffff) {
#pragma unroll
    for (int q = 0; q < NEAREST - 1; ++q) { kd[q] = kd[q + 1]; kb[q] = kb[q + 1]; }
    kd[NEAREST - 1] = 3.4e38f;
    kb[NEAREST - 1] = 0x7fffffff;
  }
}

__device__ __forceinline__ void nearest_row(const float4* st, int n, float s, const float y[3], float iL, int mine,
                                            float* out) {
  if (mine < n) {
    const float4 q = st[mine];
    out[0] = (q.x - y[0]) * iL;
    out[1] = (q.y - y[1]) * iL;
    out[2] = (q.z - y[2]) * iL;
    out[3] = logf(s * q.w * iL * iL);
  } else {
    out[0] = out[1] = out[2] = out[3] = 0.f;
  }
}

__device__ __forceinline__ void field_nearest_staged2(const float4* s0, int n0, float sc0, const float4* s1, int n1,
                                                      float sc1, const float y[3], float iL, int lane, float* row0,
                                                      float* row1, float& g0, float& g1) {
  float kd0[NEAREST], kd1[NEAREST];
  int kb0[NEAREST], kb1[NEAREST];
#pragma unroll
  for (int r = 0; r < NEAREST; ++r) {
    kd0[r] = kd1[r] = 3.4e38f;
    kb0[r] = kb1[r] = 0x7fffffff;
  }
  float a0 = 0.f, a1 = 0.f;
  const int n = max(n0, n1);
  for (int k = lane; k < n; k += 32) {
    if (k < n0) {
      const float4 q = s0[k];
      const float d2 = (q.x - y[0]) * (q.x - y[0]) + (q.y - y[1]) * (q.y - y[1]) + (q.z - y[2]) * (q.z - y[2]);
      a0 += q.w / d2;
      topk_insert(kd0, kb0, d2, k);  // squared distances order the same
    }
    if (k < n1) {
      const float4 q = s1[k];
      const float d2 = (q.x - y[0]) * (q.x - y[0]) + (q.y - y[1]) * (q.y - y[1]) + (q.z - y[2]) * (q.z - y[2]);
      a1 += q.w / d2;
      topk_insert(kd1, kb1, d2, k);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a0 += __shfl_xor_sync(FULL, a0, o);
    a1 += __shfl_xor_sync(FULL, a1, o);
  }
  g0 = sc0 * __shfl_sync(FULL, a0, 0);
  g1 = sc1 * __shfl_sync(FULL, a1, 0);
  int mine0 = 0x7fffffff, mine1 = 0x7fffffff;
  for (int r = 0; r < NEAREST; ++r) {
    float b0 = kd0[0], b1 = kd1[0];
    int i0 = kb0[0], i1 = kb1[0];
    argmin2(b0, i0, b1, i1);
    topk_pop(kd0, kb0, i0);
    topk_pop(kd1, kb1, i1);
    if (lane == r) { mine0 = i0; mine1 = i1; }
  }
  if (lane < NEAREST) {
    nearest_row(s0, n0, sc0, y, iL, mine0, row0 + 4 * lane);
    nearest_row(s1, n1, sc1, y, iL, mine1, row1 + 4 * lane);
  }
}

}  // namespace cdev
}  // namespace mi


namespace mi {
namespace cdev {

// ---------------------------------------------------------------------------
// Staged pair solve.  When both particles together have at most NT_CAP balls,
// their centres in the pair's local frame are formed once per pair into a
// warp's shared buffer: st[k] = (p_k, s k_k) and rad[k] = sqrt k_k, particle 0
// first (k < n0).  The core field of the pair at a local point y is then
// sum_k w_k / |y - p_k|^2 with its gradient and Hessian in the local frame
// directly, so a Newton iteration accumulates both particles' terms in the
// same lanes and reduces nine sums once, with no rotation per evaluation.
// The guesses read the same staged centres; their arithmetic is that of the
// unstaged versions (ball_local of the same frame), term for term.
// ---------------------------------------------------------------------------
constexpr int NT_CAP = 2 * PG_CAP;

__device__ __forceinline__ bool stage_pair(const Frame& F0, const Frame& F1, const float4* __restrict__ balls, int lane,
                                           float4* st, float* rad) {
  if (F0.n + F1.n > NT_CAP) return false;
  for (int b = lane; b < F0.n; b += 32) {
    const float4 c = __ldg(balls + F0.off + b);
    float p[3];
    ball_local(F0, c, p);
    st[b] = make_float4(p[0], p[1], p[2], F0.s * c.w);
    rad[b] = sqrtf(c.w);
  }
  for (int b = lane; b < F1.n; b += 32) {
    const float4 c = __ldg(balls + F1.off + b);
    float p[3];
    ball_local(F1, c, p);
    st[F0.n + b] = make_float4(p[0], p[1], p[2], F1.s * c.w);
    rad[F0.n + b] = sqrtf(c.w);
  }
  __syncwarp();
  return true;
}

// Warp sum of eight values per lane, each total broadcast to every lane:
// three halving exchanges leave lane l with the partial sum of value
// 4 b4 + 2 b3 + b2 (b = bits of l) over the eight lanes that share l's low
// two bits; two butterflies finish it and the totals are read from lanes
// 0, 4, ..., 28.  Seventeen shuffles instead of forty-eight.
__device__ __forceinline__ void wsum8(float v[8], int lane) {
  const bool u4 = lane & 16, u3 = lane & 8, u2 = lane & 4;
  float w[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float keep = u4 ? v[j + 4] : v[j], send = u4 ? v[j] : v[j + 4];
    w[j] = keep + __shfl_xor_sync(FULL, send, 16);
  }
  float x[2];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const float keep = u3 ? w[j + 2] : w[j], send = u3 ? w[j] : w[j + 2];
    x[j] = keep + __shfl_xor_sync(FULL, send, 8);
  }
  float z;
  {
    const float keep = u2 ? x[1] : x[0], send = u2 ? x[0] : x[1];
    z = keep + __shfl_xor_sync(FULL, send, 4);
  }
  z += __shfl_xor_sync(FULL, z, 2);
  z += __shfl_xor_sync(FULL, z, 1);
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = __shfl_sync(FULL, z, 4 * j);
}

// Newton-Raphson on grad(g0 + g1) = 0 from the staged balls, over all n of
// them or over the listed subsets (l0: indices of particle 0's balls, l1 of
// particle 1's, offset by n0 in st).  Step, stopping rule, status and
// iteration count as in newton_pair.
__device__ __forceinline__ int newton_staged(const float4* st, int n, int lane, float y[3], float tol, int max_it,
                                             int& iters, const unsigned short* l0 = nullptr, int m0 = 0,
                                             const unsigned short* l1 = nullptr, int m1 = 0, int n0 = 0) {
  int status = 1;
  const int cnt = l0 ? m0 + m1 : n;
  for (iters = 1; iters <= max_it; ++iters) {
    float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // grad (3), Hessian xx xy xz yy yz
    float h5 = 0.f;                                          // Hessian zz
    for (int u = lane; u < cnt; u += 32) {
      const int k = l0 ? (u < m0 ? (int)l0[u] : n0 + (int)l1[u - m0]) : u;
      const float4 q = st[k];
      const float d0 = y[0] - q.x, d1 = y[1] - q.y, d2 = y[2] - q.z;
      const float ir2 = 1.0f / (d0 * d0 + d1 * d1 + d2 * d2);
      const float t = q.w * ir2;              // w / r^2
      const float t2 = -2.0f * t * ir2;       // -2 w / r^4
      const float t3 = 8.0f * t * ir2 * ir2;  // 8 w / r^6
      v[0] += t2 * d0;
      v[1] += t2 * d1;
      v[2] += t2 * d2;
      v[3] += t3 * d0 * d0 + t2;
      v[4] += t3 * d0 * d1;
      v[5] += t3 * d0 * d2;
      v[6] += t3 * d1 * d1 + t2;
      v[7] += t3 * d1 * d2;
      h5 += t3 * d2 * d2 + t2;
    }
    wsum8(v, lane);
    h5 = wsum(h5);
    float A[3][3] = {{v[3], v[4], v[5]}, {v[4], v[6], v[7]}, {v[5], v[7], h5}};
    float b[3] = {v[0], v[1], v[2]};
    float dx[3];
    if (!solve<3>(A, b, dx)) { status = 2; break; }
    for (int c = 0; c < 3; ++c) y[c] -= dx[c];
    if (sqrtf(dx[0] * dx[0] + dx[1] * dx[1] + dx[2] * dx[2]) <= tol) { status = 0; break; }
  }
  if (iters > max_it) iters = max_it;
  return status;
}

// Core values and gradients of each particle at y from the staged balls (the
// final evaluation of a pair solve: status, projections, normal).
__device__ __forceinline__ void final_staged(const float4* st, int n0, int n, int lane, const float y[3], float& g0,
                                             float gr0[3], float& g1, float gr1[3]) {
  float a[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (int k = lane; k < n; k += 32) {
    const float4 q = st[k];
    const float d0 = y[0] - q.x, d1 = y[1] - q.y, d2 = y[2] - q.z;
    const float ir2 = 1.0f / (d0 * d0 + d1 * d1 + d2 * d2);
    const float t = q.w * ir2, t2 = -2.0f * t * ir2;
    if (k < n0) {
      a[0] += t; a[1] += t2 * d0; a[2] += t2 * d1; a[3] += t2 * d2;
    } else {
      a[4] += t; a[5] += t2 * d0; a[6] += t2 * d1; a[7] += t2 * d2;
    }
  }
  wsum8(a, lane);
  g0 = a[0];
  g1 = a[4];
  for (int c = 0; c < 3; ++c) {
    gr0[c] = a[1 + c];
    gr1[c] = a[5 + c];
  }
}

// sphere_midpoint of staged balls a (particle 0) and b (particle 1).
__device__ __forceinline__ void sphere_midpoint_staged(const float4* st, const float* rad, int n0, int a, int b,
                                                       float y[3]) {
  const float4 qa = st[a], qb = st[n0 + b];
  const float pa[3] = {qa.x, qa.y, qa.z}, pb[3] = {qb.x, qb.y, qb.z};
  float u[3];
  for (int c = 0; c < 3; ++c) u[c] = pb[c] - pa[c];
  const float D = sqrtf(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  if (D > 0.f) for (int c = 0; c < 3; ++c) u[c] /= D;
  else { u[0] = 1.f; u[1] = u[2] = 0.f; }
  const float ra = rad[a], rb = rad[n0 + b];
  for (int c = 0; c < 3; ++c) y[c] = 0.5f * ((pa[c] + ra * u[c]) + (pb[c] - rb * u[c]));
}

// plain_guess from the staged balls, with the search pruned so that its
// result is unchanged.  With c0, c1 the particle origins and R0, R1 the radii
// about them that hold every sphere of the particle, the triangle inequality
// bounds the gap of any pair from below by |p_a - c1| - R1 - r_a (and by
// |p_b - c0| - R0 - r_b).  The gap of the pair formed by each particle's
// sphere reaching closest to the other's origin is an upper bound ub on the
// smallest gap; balls whose bound exceeds ub (plus a margin far above FP32
// rounding of these sums) cannot take part in a pair that reaches the minimum
// or ties with it, so the O(n0 n1) search runs over the surviving balls only,
// in the same ascending order (cand: NT_CAP indices of scratch).
__device__ __forceinline__ void plain_staged(const float4* st, const float* rad, int n0, int n1, int lane,
                                             const float c0[3], const float c1[3], unsigned short* cand, float y[3]) {
  // radii about the origins, and each particle's sphere reaching closest to the other's origin
  float R0 = 0.f, R1 = 0.f, ra_best = 3.4e38f, rb_best = 3.4e38f;
  int sa = 0x7fffffff, sb = 0x7fffffff;
  for (int a = lane; a < n0; a += 32) {
    const float4 p = st[a];
    const float r = rad[a];
    R0 = fmaxf(R0, sqrtf((p.x - c0[0]) * (p.x - c0[0]) + (p.y - c0[1]) * (p.y - c0[1]) + (p.z - c0[2]) * (p.z - c0[2])) + r);
    const float g = sqrtf((p.x - c1[0]) * (p.x - c1[0]) + (p.y - c1[1]) * (p.y - c1[1]) + (p.z - c1[2]) * (p.z - c1[2])) - r;
    if (g < ra_best) { ra_best = g; sa = a; }
  }
  for (int b = lane; b < n1; b += 32) {
    const float4 p = st[n0 + b];
    const float r = rad[n0 + b];
    R1 = fmaxf(R1, sqrtf((p.x - c1[0]) * (p.x - c1[0]) + (p.y - c1[1]) * (p.y - c1[1]) + (p.z - c1[2]) * (p.z - c1[2])) + r);
    const float g = sqrtf((p.x - c0[0]) * (p.x - c0[0]) + (p.y - c0[1]) * (p.y - c0[1]) + (p.z - c0[2]) * (p.z - c0[2])) - r;
    if (g < rb_best) { rb_best = g; sb = b; }
  }
  // non-negative floats order as their bit patterns
  R0 = __uint_as_float(__reduce_max_sync(FULL, __float_as_uint(R0)));
  R1 = __uint_as_float(__reduce_max_sync(FULL, __float_as_uint(R1)));
  sa = (int)warp_argmin(ra_best, (unsigned)sa);
  sb = (int)warp_argmin(rb_best, (unsigned)sb);
  float ub = 3.4e38f;
  if (sa < n0 && sb < n1) {
    const float4 pa = st[sa], q = st[n0 + sb];
    ub = sqrtf((pa.x - q.x) * (pa.x - q.x) + (pa.y - q.y) * (pa.y - q.y) + (pa.z - q.z) * (pa.z - q.z)) - rad[sa] -
         rad[n0 + sb];
  }
  const float dc = sqrtf((c0[0] - c1[0]) * (c0[0] - c1[0]) + (c0[1] - c1[1]) * (c0[1] - c1[1]) +
                         (c0[2] - c1[2]) * (c0[2] - c1[2]));
  const float lim = ub + 1e-5f * (R0 + R1 + dc);
  // survivors, ascending: particle 0's in cand[0, ma), particle 1's in cand[ma, ma + mb)
  int ma = 0, mb = 0;
  for (int base = 0; base < n0; base += 32) {
    const int a = base + lane;
    bool in = false;
    if (a < n0) {
      const float4 p = st[a];
      in = sqrtf((p.x - c1[0]) * (p.x - c1[0]) + (p.y - c1[1]) * (p.y - c1[1]) + (p.z - c1[2]) * (p.z - c1[2])) - R1 -
               rad[a] <= lim;
    }
    const unsigned m = __ballot_sync(FULL, in);
    if (in) cand[ma + __popc(m & ((1u << lane) - 1u))] = (unsigned short)a;
    ma += __popc(m);
  }
  for (int base = 0; base < n1; base += 32) {
    const int b = base + lane;
    bool in = false;
    if (b < n1) {
      const float4 p = st[n0 + b];
      in = sqrtf((p.x - c0[0]) * (p.x - c0[0]) + (p.y - c0[1]) * (p.y - c0[1]) + (p.z - c0[2]) * (p.z - c0[2])) - R0 -
               rad[n0 + b] <= lim;
    }
    const unsigned m = __ballot_sync(FULL, in);
    if (in) cand[ma + mb + __popc(m & ((1u << lane) - 1u))] = (unsigned short)b;
    mb += __popc(m);
  }
  __syncwarp();
  float best = 3.4e38f;
  int ba = 0, bb = 0;
  if (ma > 0 && mb > 0) {
    // the ma x mb surviving pairs over the lanes, 32 at a time: lane l takes
    // pairs l, l + 32, ... of the row-major (survivor a, survivor b) order,
    // its indices advanced by 32 without a division per step
    const int q32 = 32 / mb, r32 = 32 - q32 * mb;
    int ia = lane / mb, ib = lane - (lane / mb) * mb;
    for (int u = lane; u < ma * mb; u += 32) {
      const int a = cand[ia], b = cand[ma + ib];
      const float4 pa = st[a], q = st[n0 + b];
      const float gap = sqrtf((pa.x - q.x) * (pa.x - q.x) + (pa.y - q.y) * (pa.y - q.y) + (pa.z - q.z) * (pa.z - q.z)) -
                        rad[a] - rad[n0 + b];
      if (gap < best || (gap == best && (((unsigned)a << 16) | (unsigned)b) < (((unsigned)ba << 16) | (unsigned)bb))) {
        best = gap;
        ba = a;
        bb = b;
      }
      ia += q32;
      ib += r32;
      if (ib >= mb) {
        ib -= mb;
        ++ia;
      }
    }
  }
  // smallest gap, ties to the lower (a, b): a, b < 256 here
  const unsigned ab = warp_argmin(best, ((unsigned)ba << 16) | (unsigned)bb);
  sphere_midpoint_staged(st, rad, n0, (int)(ab >> 16), (int)(ab & 0xffffu), y);
}

// active_subset over the staged balls st[base, base + n).
__device__ __forceinline__ int active_staged(const float4* st, int base, int n, const float y[3], float r, int lane,
                                             unsigned short* list) {
  int cnt = 0;
  const float r2 = r * r;
  for (int b0 = 0; b0 < n; b0 += 32) {
    const int b = b0 + lane;
    bool in = false;
    if (b < n) {
      const float4 p = st[base + b];
      const float d2 = (p.x - y[0]) * (p.x - y[0]) + (p.y - y[1]) * (p.y - y[1]) + (p.z - y[2]) * (p.z - y[2]);
      in = d2 <= r2;
    }
    const unsigned m = __ballot_sync(FULL, in);
    const int pos = cnt + __popc(m & ((1u << lane) - 1u));
    if (in && pos < SUB_CAP) list[pos] = (unsigned short)b;
    cnt += __popc(m);
  }
  __syncwarp();
  return cnt;
}

// Core values and gradients of both particles at y from the ball table (the
// final evaluation of a pair too large to stage).  Out of line: the staged
// path is the common one, and the kernel's hot code stays small.
static __device__ __noinline__ void final_unstaged(const Frame& F0, const Frame& F1, const float4* __restrict__ balls,
                                            int lane, const float y[3], float& g0, float gr0[3], float& g1,
                                            float gr1[3]) {
  const GEval e0 = eval(F0, balls, y, lane), e1 = eval(F1, balls, y, lane);
  g0 = e0.g;
  g1 = e1.g;
  for (int c = 0; c < 3; ++c) {
    gr0[c] = e0.gr[c];
    gr1[c] = e1.gr[c];
  }
}

// A pair's solver state: the frames, and (when the pair fits) its staged
// balls; every piece of the solve goes through the staged path when it can
// and through the unstaged warp evaluation otherwise.
struct PairSolver {
  const Frame& F0;
  const Frame& F1;
  const float4* __restrict__ balls;
  float4* st;
  float* rad;
  unsigned short* cand;  // NT_CAP indices of scratch (the plain guess's survivors)
  int lane;
  bool staged;

  __device__ __forceinline__ PairSolver(const Frame& f0, const Frame& f1, const float4* __restrict__ b, float4* s,
                                        float* r, unsigned short* cd, int ln)
      : F0(f0), F1(f1), balls(b), st(s), rad(r), cand(cd), lane(ln) {
    staged = stage_pair(F0, F1, balls, lane, st, rad);
  }
  __device__ __forceinline__ int nballs() const { return F0.n + F1.n; }
  __device__ __forceinline__ void plain(float y[3]) const {
    if (staged) plain_staged(st, rad, F0.n, F1.n, lane, F0.t, F1.t, cand, y);
    else plain_guess(F0, F1, balls, lane, y, st);
  }
  __device__ __forceinline__ int newton(float y[3], float tol, int max_it, int& iters) const {
    return staged ? newton_staged(st, F0.n + F1.n, lane, y, tol, max_it, iters)
                  : newton_pair(F0, F1, balls, lane, y, tol, max_it, iters);
  }
  // plain start, then Newton to the contact tolerance
  __device__ __forceinline__ int plain_newton(float y[3], float tol, int& iters) const {
    plain(y);
    return newton(y, tol, MAX_IT, iters);
  }
  __device__ __forceinline__ void final_eval(const float y[3], float& g0, float gr0[3], float& g1, float gr1[3]) const {
    if (staged) final_staged(st, F0.n, F0.n + F1.n, lane, y, g0, gr0, g1, gr1);
    else final_unstaged(F0, F1, balls, lane, y, g0, gr0, g1, gr1);
  }
  // learned_newton through the staged path (same stages, gates and fallback)
  __device__ __forceinline__ int learned(const float a[3], const float d[4], float L, float Rb, unsigned short* l0,
                                         unsigned short* l1, float y[3], SolveCount& sc) const {
    if (!staged) return learned_newton(F0, F1, balls, lane, a, d, L, Rb, l0, l1, y, sc, st);
    const int n0 = F0.n, n1 = F1.n;
    sc.iters = sc.evals = sc.fallback = 0;
    for (int c = 0; c < 3; ++c) y[c] = L * (a[c] + d[c]);
    bool ok = isfinite(y[0]) && isfinite(y[1]) && isfinite(y[2]);
    if (ok) {
      const float r_act = L * expf(fminf(fmaxf(d[3], -8.f), 2.f));
      const int m0 = active_staged(st, 0, n0, y, r_act, lane, l0);
      const int m1 = active_staged(st, n0, n1, y, r_act, lane, l1);
      if (m0 > 0 && m1 > 0 && m0 <= SUB_CAP && m1 <= SUB_CAP && 2 * (m0 + m1) <= n0 + n1) {
        float ys[3] = {y[0], y[1], y[2]};
        int it = 0;
        const int s = newton_staged(st, n0 + n1, lane, ys, SUB_TOL * Rb, SUB_IT, it, l0, m0, l1, m1, n0);
        sc.iters += it;
        sc.evals += it * (m0 + m1);
        if (s == 0)
          for (int c = 0; c < 3; ++c) y[c] = ys[c];
      }
      int it = 0;
      const int s = newton_staged(st, n0 + n1, lane, y, NEWTON_TOL * Rb, MAX_IT, it);
      sc.iters += it;
      sc.evals += it * (n0 + n1);
      ok = s == 0;
    }
    if (ok) return 0;
    sc.fallback = 1;
    __syncwarp();  // the subset lists share cand's memory
    plain_staged(st, rad, n0, n1, lane, F0.t, F1.t, cand, y);
    int it = 0;
    const int s = newton_staged(st, n0 + n1, lane, y, NEWTON_TOL * Rb, MAX_IT, it);
    sc.iters += it;
    sc.evals += it * (n0 + n1);
    return s;
  }
};

}  // namespace cdev
}  // namespace mi
