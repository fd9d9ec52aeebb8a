// Particle-side kernels: per-step prologue, solid flagging from the metaball
// field (Eq. 1), node classification with boundary/uncovered lists, the wall
// fraction q of every boundary link, the rigid-body update (Newton-Euler,
// Sec. 2.3.1) and mass-property quadrature.
//
// Flagging decides f >= 1 exactly as an FP64 evaluation would: an FP32 pass
// with the body-frame point formed in FP64 decides every node whose FP32 value
// is farther than GUARD from 1 (its error is below 3e-5 for control points at
// least 0.3 lu from the node), and the rare nodes inside the guard band are
// re-evaluated in FP64 with unfused operations in the order: x - X, R^T,
// ball by ball k / |x_b - c|^2 accumulated left to right.
#include <cfloat>
#include <climits>

#include <cooperative_groups.h>
#include <cooperative_groups/scan.h>

#include "mi_internal.cuh"
#include "rigid_dev.cuh"

namespace cg = cooperative_groups;

namespace mi {

namespace {
constexpr float GUARD = FIELD_GUARD;

__device__ __forceinline__ void quat_to_R_exact(const double q[4], double R[9]) {
  // body -> world rotation of the normalised quaternion, unfused FP64
  double n = __dsqrt_rn(__dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(q[0], q[0]), __dmul_rn(q[1], q[1])),
                                            __dmul_rn(q[2], q[2])),
                                  __dmul_rn(q[3], q[3])));
  const double w = __ddiv_rn(q[0], n), x = __ddiv_rn(q[1], n), y = __ddiv_rn(q[2], n), z = __ddiv_rn(q[3], n);
  R[0] = __dsub_rn(1.0, __dmul_rn(2.0, __dadd_rn(__dmul_rn(y, y), __dmul_rn(z, z))));
  R[1] = __dmul_rn(2.0, __dsub_rn(__dmul_rn(x, y), __dmul_rn(w, z)));
  R[2] = __dmul_rn(2.0, __dadd_rn(__dmul_rn(x, z), __dmul_rn(w, y)));
  R[3] = __dmul_rn(2.0, __dadd_rn(__dmul_rn(x, y), __dmul_rn(w, z)));
  R[4] = __dsub_rn(1.0, __dmul_rn(2.0, __dadd_rn(__dmul_rn(x, x), __dmul_rn(z, z))));
  R[5] = __dmul_rn(2.0, __dsub_rn(__dmul_rn(y, z), __dmul_rn(w, x)));
  R[6] = __dmul_rn(2.0, __dsub_rn(__dmul_rn(x, z), __dmul_rn(w, y)));
  R[7] = __dmul_rn(2.0, __dadd_rn(__dmul_rn(y, z), __dmul_rn(w, x)));
  R[8] = __dsub_rn(1.0, __dmul_rn(2.0, __dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y))));
}

// f(x) >= 1 in FP64, unfused, same operation order as the definition above,
// for the node (x, y, z) that every lane of the warp passes: the lanes form
// the terms of 32 balls at a time and the sum is taken in ball order, so the
// value is that of one thread summing ball after ball.
__device__ __noinline__ bool inside_exact_warp(const DevParticle& P, const double* balls_d, int x, int y, int z,
                                               unsigned lane) {
  const double d0 = __dsub_rn((double)x, P.pos[0]), d1 = __dsub_rn((double)y, P.pos[1]),
               d2 = __dsub_rn((double)z, P.pos[2]);
  const double* R = P.R;
  const double b0 = __dadd_rn(__dadd_rn(__dmul_rn(R[0], d0), __dmul_rn(R[3], d1)), __dmul_rn(R[6], d2));
  const double b1 = __dadd_rn(__dadd_rn(__dmul_rn(R[1], d0), __dmul_rn(R[4], d1)), __dmul_rn(R[7], d2));
  const double b2 = __dadd_rn(__dadd_rn(__dmul_rn(R[2], d0), __dmul_rn(R[5], d1)), __dmul_rn(R[8], d2));
  const int nb = P.n_balls;
  double f = 0.0;
  for (int base = 0; base < nb; base += 32) {
    double t = 0.0;
    const int i = base + (int)lane;
    if (i < nb) {
      const double* c = balls_d + 4 * (size_t)(P.ball_off + i);
      const double e0 = __dsub_rn(b0, c[0]), e1 = __dsub_rn(b1, c[1]), e2 = __dsub_rn(b2, c[2]);
      const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(e0, e0), __dmul_rn(e1, e1)), __dmul_rn(e2, e2));
      t = __ddiv_rn(c[3], r2);
    }
    const int m = nb - base < 32 ? nb - base : 32;
    for (int j = 0; j < m; ++j) f = __dadd_rn(f, __shfl_sync(0xffffffffu, t, j));
  }
  return f >= 1.0;
}

// Region of a box kernel: box [lo, lo + ext) widened by `pad`, clipped.
struct Region {
  int lo[3], n[3];
  unsigned total;
};
__device__ __forceinline__ Region clip_region(const int lo[3], const int ext[3], int pad, const LatticeGeom& g) {
  Region r;
  const int sz[3] = {g.nx, g.ny, g.nz};
  r.total = 1u;
  for (int a = 0; a < 3; ++a) {
    int l = lo[a] - pad, h = lo[a] + ext[a] + pad;
    l = l < 0 ? 0 : l;
    h = h > sz[a] ? sz[a] : h;
    r.lo[a] = l;
    r.n[a] = h > l ? h - l : 0;
    r.total *= (unsigned)r.n[a];
  }
  return r;
}

__device__ __forceinline__ long long lin(int x, int y, int z, const LatticeGeom& g) {
  return x + (long long)g.nx * (y + (long long)g.ny * z);
}

// Neighbour along direction d with periodic wrap; false if outside the domain.
__device__ __forceinline__ bool neighbour(int x, int y, int z, int dx, int dy, int dz, const LatticeGeom& g,
                                          long long& out) {
  // |dx|, |dy|, |dz| <= 1: one wrap at most
  int a = x + dx, b = y + dy, c = z + dz;
  if (a < 0 || a >= g.nx) {
    if (!g.periodic[0]) return false;
    a += a < 0 ? g.nx : -g.nx;
  }
  if (b < 0 || b >= g.ny) {
    if (!g.periodic[1]) return false;
    b += b < 0 ? g.ny : -g.ny;
  }
  if (c < 0 || c >= g.nz) {
    if (!g.periodic[2]) return false;
    c += c < 0 ? g.nz : -g.nz;
  }
  out = lin(a, b, c, g);
  return true;
}
}  // namespace

// ---------------------------------------------------------------------------
// Prologue: bump the flag generation, zero counters and hydrodynamic force
// sums, rotation matrices and node boxes at the current pose.
// ---------------------------------------------------------------------------
__global__ void k_prologue(ParticleLaunch L) {
  // one warp per particle: every lane forms the rotation (the same FP64
  // operations, so the same bits), then the lanes share out the float pairs
  // of its entries and of the directions
  const int p = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (p == 0 && lane == 0) {
    L.ctr->gen += 1u;
    L.ctr->n_bc = 0;
    L.ctr->n_links = 0;
    L.ctr->n_new = 0;
    L.ctr->n_cov = 0;
  }
  if (p >= L.np) return;
  DevParticle& P = L.P[p];
  double R[9];
  quat_to_R_exact(P.quat, R);
  if (lane < 9) {
    double r = R[0];
#pragma unroll
    for (int k = 1; k < 9; ++k) r = lane == k ? R[k] : r;
    const float rf = (float)r;
    P.R[lane] = r;
    P.Rf[lane] = rf;
    P.Rs[0][lane] = rf;
    P.Rs[1][lane] = (float)(r - (double)rf);
  } else if (lane < 12) {
    // R^T (X - floor X), entry k
    const int k = lane - 9;
    double fr[3], c[3];
    for (int a = 0; a < 3; ++a) fr[a] = P.pos[a] - floor(P.pos[a]);
#pragma unroll
    for (int a = 0; a < 3; ++a) c[a] = k == 0 ? R[3 * a] : (k == 1 ? R[3 * a + 1] : R[3 * a + 2]);
    const double t = c[0] * fr[0] + c[1] * fr[1] + c[2] * fr[2];
    P.Ts[0][k] = (float)t;
    P.Ts[1][k] = (float)(t - (double)P.Ts[0][k]);
  }
  if (lane < 19) {
    // R^T e_d for direction d = lane
    const int d = lane;
    const double ex = lex(d), ey = ley(d), ez = lez(d);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const double e = R[k] * ex + R[3 + k] * ey + R[6 + k] * ez;
      P.Es[d][k] = (float)e;
      P.Es[d][3 + k] = (float)(e - (double)P.Es[d][k]);
    }
  }
  if (lane == 0) {
    for (int a = 0; a < 3; ++a) {
      P.lo[a] = (int)floor(P.pos[a] - P.Rt) - 1;
      P.posf[a] = (float)P.pos[a];
      const double fl = floor(P.pos[a]);
      P.pos_i[a] = (int)fl;
      P.pos_fr[a] = (float)(P.pos[a] - fl);
      P.velf[a] = (float)P.vel[a];
      P.omegaf[a] = (float)P.omega[a];
      const int prev = P.lo_hist[L.prev_buf][a];
      if (prev != BOX_NONE && abs(P.lo[a] - prev) > 2) atomicOr(&L.ctr->status, STATUS_MOVED_TOO_FAR);
    }
    P.srad2[L.cur_buf] = -1;  // the solid radius of this step, grown by k_flag
    for (int a = 0; a < 3; ++a) P.sctr[L.cur_buf][a] = (float)P.pos[a];
  }
  if (lane < 6) L.facc[6 * p + lane] = 0;
}

cudaError_t launch_prologue(const ParticleLaunch& L, cudaStream_t s) {
  const int blocks = L.np > 0 ? (L.np + 3) / 4 : 1;  // four warps per block, a warp per particle
  k_prologue<<<blocks, 128, 0, s>>>(L);
  return cudaGetLastError();
}

// The particle owning block b of a box kernel's 1D grid (off[p] <= b <
// off[p + 1], off[0] = 0) by binary search, its first block and block count.
struct BoxBlock {
  int p, b, nb;
};
__device__ __forceinline__ BoxBlock box_block(const int* __restrict__ off, int np, int b) {
  int lo = 0, hi = np;  // off[lo] <= b < off[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= b) lo = mid;
    else hi = mid;
  }
  const int o = off[lo];
  return {lo, b - o, off[lo + 1] - o};
}

// ---------------------------------------------------------------------------
// Clear the owner buffer about to be rewritten, over the boxes it was last
// written with.
// ---------------------------------------------------------------------------
__global__ void k_clear(ParticleLaunch L) {
  const BoxBlock bb = box_block(L.flag_off, L.np, blockIdx.x);
  const DevParticle& P = L.P[bb.p];
  const int* lo = P.lo_hist[L.cur_buf];
  if (lo[0] == BOX_NONE) return;
  const Region r = clip_region(lo, P.ext, 0, L.g);
  const unsigned n0 = (unsigned)r.n[0], n01 = n0 * (unsigned)r.n[1];
  for (unsigned i = bb.b * blockDim.x + threadIdx.x; i < r.total; i += bb.nb * blockDim.x) {
    const unsigned zi = i / n01, rem = i - zi * n01, yi = rem / n0;
    const int x = r.lo[0] + (int)(rem - yi * n0);
    const int y = r.lo[1] + (int)yi;
    const int z = r.lo[2] + (int)zi;
    L.owner_cur[lin(x, y, z, L.g)] = OWNER_NONE;
  }
}

cudaError_t launch_clear(const ParticleLaunch& L, cudaStream_t s) {
  if (L.np == 0) return cudaSuccess;
  k_clear<<<L.flag_blocks, 256, 0, s>>>(L);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Solid flagging: node x of particle p's box is solid for p when
// f_p(R_p^T (x - X_p)) >= 1; the owner is the lowest such p (atomicMin).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256, 3) k_flag(ParticleLaunch L) {
  extern __shared__ float4 sb[];
  const BoxBlock bb = box_block(L.flag_off, L.np, blockIdx.x);
  const int p = bb.p;
  const DevParticle& P = L.P[p];
  const int nb = P.n_balls;
  const bool staged = nb <= L.max_balls_per_particle;
  __shared__ int rr_s;  // the block's largest squared solid distance (float bits)
  volatile int* rr = &rr_s;
  if (threadIdx.x == 0) rr_s = -1;
  if (staged)
    for (int i = threadIdx.x; i < nb; i += blockDim.x) sb[i] = L.balls[P.ball_off + i];
  __syncthreads();
  const float4* bl = staged ? sb : L.balls + P.ball_off;
  if (bb.b == 0 && threadIdx.x == 0)
    for (int a = 0; a < 3; ++a) L.P[p].lo_hist[L.cur_buf][a] = P.lo[a];
  const Region r = clip_region(P.lo, P.ext, 0, L.g);
  // x - X = (x - Xi) - Xf with Xi = floor(X): the integer part is exact in
  // FP32, the fraction carries one FP32 rounding (both set once per particle
  // by the prologue, with R in FP32: FP64 set-up in every thread would cost
  // more than the field evaluations on this part)
  const int xi0 = P.pos_i[0], xi1 = P.pos_i[1], xi2 = P.pos_i[2];
  const float xf0 = P.pos_fr[0], xf1 = P.pos_fr[1], xf2 = P.pos_fr[2];
  float Rf[9];
  for (int k = 0; k < 9; ++k) Rf[k] = P.Rf[k];
  const float rt = (float)P.Rt * (1.0f + 1e-6f) + 1e-4f, rt2 = rt * rt;
  const unsigned n0 = (unsigned)r.n[0], n01 = n0 * (unsigned)r.n[1];
  // whole warps step together (the guard band's FP64 field is a warp collective)
  const unsigned lane = threadIdx.x & 31u;
  for (unsigned base = bb.b * blockDim.x + (threadIdx.x & ~31u); base < r.total; base += bb.nb * blockDim.x) {
    const unsigned i = base + lane;
    int x = 0, y = 0, z = 0;
    bool inside = false, band = false;
    if (i < r.total) {
      const unsigned zi = i / n01, rem = i - zi * n01, yi = rem / n0;
      x = r.lo[0] + (int)(rem - yi * n0);
      y = r.lo[1] + (int)yi;
      z = r.lo[2] + (int)zi;
      const float d0 = (float)(x - xi0) - xf0, d1 = (float)(y - xi1) - xf1, d2 = (float)(z - xi2) - xf2;
      // beyond the tight radius: fluid
      if (d0 * d0 + d1 * d1 + d2 * d2 <= rt2) {
        const float b0 = Rf[0] * d0 + Rf[3] * d1 + Rf[6] * d2;
        const float b1 = Rf[1] * d0 + Rf[4] * d1 + Rf[7] * d2;
        const float b2 = Rf[2] * d0 + Rf[5] * d1 + Rf[8] * d2;
        // four independent partial sums (the terms are positive, so any partial
        // sum above 1 + GUARD decides "inside"; FP32 reordering moves the sum by
        // far less than GUARD, and sums within GUARD of 1 are redone in FP64)
        float f0 = 0.f, f1 = 0.f, f2 = 0.f, f3 = 0.f;
        bool decided = false;
        int b = 0;
        for (; b + 4 <= nb; b += 4) {
          const float4 c0 = bl[b], c1 = bl[b + 1], c2 = bl[b + 2], c3 = bl[b + 3];
          f0 += __fdividef(c0.w, (b0 - c0.x) * (b0 - c0.x) + (b1 - c0.y) * (b1 - c0.y) + (b2 - c0.z) * (b2 - c0.z));
          f1 += __fdividef(c1.w, (b0 - c1.x) * (b0 - c1.x) + (b1 - c1.y) * (b1 - c1.y) + (b2 - c1.z) * (b2 - c1.z));
          f2 += __fdividef(c2.w, (b0 - c2.x) * (b0 - c2.x) + (b1 - c2.y) * (b1 - c2.y) + (b2 - c2.z) * (b2 - c2.z));
          f3 += __fdividef(c3.w, (b0 - c3.x) * (b0 - c3.x) + (b1 - c3.y) * (b1 - c3.y) + (b2 - c3.z) * (b2 - c3.z));
          if ((f0 + f1) + (f2 + f3) > 1.0f + GUARD) {  // partial sums only grow: inside for sure
            inside = decided = true;
            break;
          }
        }
        if (!decided) {
          for (; b < nb; ++b) {
            const float4 c = bl[b];
            const float e0 = b0 - c.x, e1 = b1 - c.y, e2 = b2 - c.z;
            f0 += __fdividef(c.w, e0 * e0 + e1 * e1 + e2 * e2);
          }
          const float f = (f0 + f1) + (f2 + f3);
          if (f > 1.0f + GUARD) inside = true;
          else if (f < 1.0f - GUARD) inside = false;
          else band = true;  // within GUARD of 1 (or not a number): decided in FP64 below
        }
      }
    }
    // the nodes in the guard band, one at a time by the whole warp
    for (unsigned m = __ballot_sync(0xffffffffu, band); m; m &= m - 1u) {
      const int src = __ffs(m) - 1;
      const bool in = inside_exact_warp(P, L.balls_d, __shfl_sync(0xffffffffu, x, src),
                                        __shfl_sync(0xffffffffu, y, src), __shfl_sync(0xffffffffu, z, src), lane);
      if ((int)lane == src) inside = in;
    }
    if (inside) {
      atomicMin(L.owner_cur + lin(x, y, z, L.g), (uint32_t)p);
      // the block's solid radius in shared memory (non-negative floats
      // order as their bits): an atomic only where it grows; the distance is
      // formed again here rather than kept live through the ball loop
      const float e0 = (float)(x - xi0) - xf0, e1 = (float)(y - xi1) - xf1, e2 = (float)(z - xi2) - xf2;
      const int dd = __float_as_int(e0 * e0 + e1 * e1 + e2 * e2);
      if (dd > *rr) atomicMax((int*)rr, dd);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && *rr >= 0) atomicMax(&L.P[p].srad2[L.cur_buf], *rr);
}

cudaError_t launch_flag(const ParticleLaunch& L, cudaStream_t s) {
  if (L.np == 0) return cudaSuccess;
  const size_t smem = sizeof(float4) * (size_t)L.max_balls_per_particle;
  k_flag<<<L.flag_blocks, 256, smem, s>>>(L);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Classification over each particle's old and new boxes widened by 2: solid,
// boundary (fluid with a solid neighbour; 18-bit link mask), uncovered (fluid
// now, solid at the previous step), and with the cover/uncover rule covered
// (solid now, fluid at the previous step).  Boxes may overlap: every block
// writes the same class for a node, and a per-node generation stamp lets
// exactly one block append it to the boundary / uncovered / covered lists.
// ---------------------------------------------------------------------------
template <bool COV>
__global__ void __launch_bounds__(256) k_classify(ParticleLaunch L) {
  const BoxBlock bb = box_block(L.cls_off, L.np, blockIdx.x);
  const DevParticle& P = L.P[bb.p];
  int lo[3], ext[3];
  const int* lp = P.lo_hist[L.prev_buf];
  const bool had = lp[0] != BOX_NONE;
  for (int a = 0; a < 3; ++a) {
    if (!had) {
      lo[a] = P.lo[a];
      ext[a] = P.ext[a];
    } else {
      lo[a] = min(P.lo[a], lp[a]);
      ext[a] = max(P.lo[a], lp[a]) + P.ext[a] - lo[a];
    }
  }
  // nodes whose class can change: the solid nodes of this step and of the
  // previous one (within their solid radii of the positions they were
  // flagged at), the fluid nodes next to them (a link is at most sqrt 2
  // long), and the nodes uncovered at the previous step (solid two steps ago:
  // within a move of the previous solid, and a particle moves at most two
  // nodes per step): both spheres widened by 3
  const int sc = P.srad2[L.cur_buf], sp = had ? P.srad2[L.prev_buf] : -1;
  if (sc < 0 && sp < 0) return;
  const float rc = sc >= 0 ? sqrtf(__int_as_float(sc)) + 3.0f : -1.0f;
  const float rp = sp >= 0 ? sqrtf(__int_as_float(sp)) + 3.0f : -1.0f;
  const float rc2 = rc * rc, rp2 = rp * rp;
  const float cc0 = P.sctr[L.cur_buf][0], cc1 = P.sctr[L.cur_buf][1], cc2 = P.sctr[L.cur_buf][2];
  const float cp0 = P.sctr[L.prev_buf][0], cp1 = P.sctr[L.prev_buf][1], cp2 = P.sctr[L.prev_buf][2];
  const Region r = clip_region(lo, ext, 2, L.g);
  const unsigned gen = L.ctr->gen;
  // one warp per (y, z) row of the region: the row's x-interval inside
  // either sphere, computed once per row (rows that miss both are skipped by
  // the whole warp), its nodes taken 32 at a time
  const int lane = threadIdx.x & 31;
  const unsigned rows = (unsigned)r.n[1] * (unsigned)r.n[2];
  const unsigned wid = (bb.b * blockDim.x + threadIdx.x) >> 5, nw = (bb.nb * blockDim.x) >> 5;
  for (unsigned row = wid; row < rows; row += nw) {
    const unsigned zi = row / (unsigned)r.n[1];
    const int y = r.lo[1] + (int)(row - zi * (unsigned)r.n[1]);
    const int z = r.lo[2] + (int)zi;
    int xa = INT_MAX, xb = INT_MIN;
    {
      const float hc = rc2 - ((y - cc1) * (y - cc1) + (z - cc2) * (z - cc2));
      if (rc >= 0.f && hc >= 0.f) {
        const float w = sqrtf(hc);
        xa = (int)ceilf(cc0 - w);
        xb = (int)floorf(cc0 + w);
      }
      const float hp = rp2 - ((y - cp1) * (y - cp1) + (z - cp2) * (z - cp2));
      if (rp >= 0.f && hp >= 0.f) {
        const float w = sqrtf(hp);
        xa = min(xa, (int)ceilf(cp0 - w));
        xb = max(xb, (int)floorf(cp0 + w));
      }
      xa = max(xa, r.lo[0]);
      xb = min(xb, r.lo[0] + r.n[0] - 1);
    }
    // a row outside both spheres (xa > xb) is skipped before any index is
    // formed: xa = INT_MAX + lane would overflow
    if (xa > xb) continue;
    for (int x = xa + lane; x <= xb; x += 32) {
    const long long c = lin(x, y, z, L.g);
    const bool solid = L.owner_cur[c] != OWNER_NONE;
    const bool was = L.owner_prev[c] != OWNER_NONE;
    uint32_t mask = 0;
    if (!solid) {
      const bool interior = (x > 0) & (x < L.g.nx - 1) & (y > 0) & (y < L.g.ny - 1) & (z > 0) & (z < L.g.nz - 1);
      if (interior) {
        const long long sy = L.g.nx, sz = (long long)L.g.nx * L.g.ny;
#pragma unroll
        for (int d = 1; d < 19; ++d)
          if (__ldg(L.owner_cur + c + cx(d) + sy * cy(d) + sz * cz(d)) != OWNER_NONE) mask |= 1u << d;
      } else {
#pragma unroll 1
        for (int d = 1; d < 19; ++d) {
          long long nbr;
          if (neighbour(x, y, z, cx(d), cy(d), cz(d), L.g, nbr) && L.owner_cur[nbr] != OWNER_NONE) mask |= 1u << d;
        }
      }
    }
    const bool isnew = !solid && was;
    // covered: listed for the cover/uncover rule only, and not in the step
    // that first flags the covering particle (it was not there before)
    const bool iscov = COV && solid && !was && L.P[L.owner_cur[c]].lo_hist[L.prev_buf][0] != BOX_NONE;
    L.cls[c] = (uint8_t)((solid ? CLS_SOLID : 0) | (mask ? CLS_BOUNDARY : 0) | (isnew ? CLS_NEW : 0));
    if (!(mask || isnew || iscov)) continue;
    if (atomicExch(L.stamp + c, gen) == gen) continue;  // another block listed it
    // list appends aggregated over the lanes that got here: one atomic per
    // counter and warp (all boundary nodes share the counters, and
    // same-address atomics serialise in L2), offsets by ballot ranks and a scan
    const cg::coalesced_group grp = cg::coalesced_threads();
    const unsigned below = (1u << grp.thread_rank()) - 1u;
    const unsigned newm = grp.ballot(isnew), bcm = grp.ballot(mask != 0);
    const unsigned m = __popc(mask);
    const unsigned m_excl = cg::exclusive_scan(grp, m);
    unsigned base_new = 0, base_bc = 0, base_l = 0;
    if (grp.thread_rank() == 0) {
      if (newm) base_new = atomicAdd(&L.ctr->n_new, (unsigned)__popc(newm));
      if (bcm) base_bc = atomicAdd(&L.ctr->n_bc, (unsigned)__popc(bcm));
    }
    if (grp.thread_rank() == grp.size() - 1) {
      const unsigned total = m_excl + m;
      if (total) base_l = atomicAdd(&L.ctr->n_links, total);
    }
    base_new = grp.shfl(base_new, 0);
    base_bc = grp.shfl(base_bc, 0);
    base_l = grp.shfl(base_l, grp.size() - 1);
    if (isnew) {
      const unsigned k = base_new + __popc(newm & below);
      if (k < L.cap_new) L.new_cell[k] = (uint32_t)c;
      else atomicOr(&L.ctr->status, STATUS_NEW_OVERFLOW);
    }
    if constexpr (COV) {
      const unsigned covm = grp.ballot(iscov);
      unsigned base_cov = 0;
      if (grp.thread_rank() == 0 && covm) base_cov = atomicAdd(&L.ctr->n_cov, (unsigned)__popc(covm));
      base_cov = grp.shfl(base_cov, 0);
      if (iscov) {
        const unsigned k = base_cov + __popc(covm & below);
        if (k < L.cap_new) L.cov_cell[k] = (uint32_t)c;
        else atomicOr(&L.ctr->status, STATUS_NEW_OVERFLOW);
      }
    }
    if (mask) {
      const unsigned bi = base_bc + __popc(bcm & below);
      const unsigned lo_l = base_l + m_excl;
      if (bi >= L.cap_bc) {
        atomicOr(&L.ctr->status, STATUS_BC_OVERFLOW);
        continue;
      }
      L.bc_cell[bi] = (uint32_t)c;
      L.bc_mask[bi] = mask;
      L.bc_loff[bi] = lo_l;
      if (lo_l + m > L.cap_links) {
        atomicOr(&L.ctr->status, STATUS_LINK_OVERFLOW);
        continue;
      }
      unsigned k = 0;
      for (int d = 1; d < 19; ++d) {
        if (!((mask >> d) & 1u)) continue;
        long long nbr;
        neighbour(x, y, z, cx(d), cy(d), cz(d), L.g, nbr);
        L.link_bc[lo_l + k] = bi;
        L.link_dir[lo_l + k] = (uint8_t)d;
        L.link_p[lo_l + k] = L.owner_cur[nbr];
        ++k;
      }
    }
  }
  }
}

cudaError_t launch_classify(const ParticleLaunch& L, cudaStream_t s) {
  if (L.np == 0) return cudaSuccess;
  // a warp per (y, z) row, about 64 rows per warp
  if (L.cover_uncover) k_classify<true><<<L.classify_blocks, 256, 0, s>>>(L);
  else k_classify<false><<<L.classify_blocks, 256, 0, s>>>(L);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Wall fraction of each link: root q in (0, 1] of g(q) = f_p(x_f + q e_d) - 1
// (Sec. 2.3.2; reading A7: along the link that points into the solid, c0 = 1).
//
// Inputs: the body-frame link origin p and direction e as float pairs hi + lo
// (the prologue forms the particle's frame in FP64 once per step; each link
// combines it in float-float arithmetic, without FP64, which runs at a small
// fraction of the FP32 rate on this part), and the ball table's split copy; origins
// and centres are split on the grid of 2^-12 when the particle's bounding
// radius is below 1000, so that p_hi - c_hi is exact in FP32 (otherwise the
// difference goes through TwoSum).
//
// Stage 1, FP32: Newton steps on h(q) = f^(-1/2) - 1, which has the same root
// and is close to linear along a link for fields of the form k / r^2 (the
// distance to a lone ball over its radius), kept inside a shrinking bracket
// [lo, hi] (bisection when a step leaves it), the field summed as two
// independent partial sums from the hi parts of the centres, until a step is
// below 1e-3.  With the exact
// differences the body-frame point carries ~1e-7 of rounding, but the FP32
// field's noise, divided by g'(q) = e . grad f (small on large smooth
// particles and on links that meet the surface at a grazing angle), still
// leaves errors up to ~1e-4.
// Stage 2, double-float: Newton steps whose residual g(q) is evaluated in
// float-float arithmetic (an unevaluated sum hi + lo of two floats, ~44
// significant bits; Knuth's TwoSum and the fused-multiply-add form of
// Dekker's product are exact), the derivative in FP32, inside a bracket that
// starts at [0, 1] (the exact flags guarantee g(0) < 0 <= g(1)) and moves with
// the accurate signs.  A step ends it when it is below 2e-5 or when the error
// Newton's quadratic convergence leaves behind, |g''/2g'| step^2 with g'' in
// FP32 from the same sums, is below 1e-7 (usually the first step); at most
// four steps.
// ---------------------------------------------------------------------------
namespace {
struct F2 {
  float hi, lo;
};
__device__ __forceinline__ F2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bv = __fsub_rn(s, a);
  const float av = __fsub_rn(s, bv);
  return {s, __fadd_rn(__fsub_rn(a, av), __fsub_rn(b, bv))};
}
__device__ __forceinline__ F2 two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ F2 df_add(F2 a, F2 b) {
  const F2 s = two_sum(a.hi, b.hi);
  return two_sum(s.hi, s.lo + (a.lo + b.lo));
}
// a float pair re-split with hi on the grid of 2^-12 (|hi| < 2^11: exact)
__device__ __forceinline__ F2 to_grid(F2 v) {
  const float h = rintf(v.hi * 4096.0f) * (1.0f / 4096.0f);
  return {h, (v.hi - h) + v.lo};
}
// p_hi - c_hi as hi + lo (exact on the grid)
__device__ __forceinline__ F2 diff_hi(float p, float c, bool grid) {
  return grid ? F2{__fsub_rn(p, c), 0.f} : two_sum(p, -c);
}

// g(q) = f(p + q e) - 1 in float-float; g'(q) and g''(q) in FP32 (ee = e . e).
template <bool GRID>
__device__ __forceinline__ float residual_ff(const float4* __restrict__ bs, int nb, const F2 p[3], const F2 e[3],
                                             float q, float ee, float& gp, float& gpp) {
  float gh = 0.f, gl = 0.f, d1 = 0.f, d2 = 0.f;
  for (int b = 0; b < nb; ++b) {
    const float4 ch = __ldg(bs + 2 * b), cl = __ldg(bs + 2 * b + 1);
    const float c_hi[3] = {ch.x, ch.y, ch.z}, c_lo[3] = {cl.x, cl.y, cl.z};
    float r2h = 0.f, r2l = 0.f, ae = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      // a = (p - c) + q e as ah + al
      const F2 d = diff_hi(p[k].hi, c_hi[k], GRID);
      const float dl = GRID ? p[k].lo - c_lo[k] : d.lo + (p[k].lo - c_lo[k]);
      const F2 m = two_prod(q, e[k].hi);
      const float ml = __fmaf_rn(q, e[k].lo, m.lo);
      const F2 a = two_sum(d.hi, m.hi);
      const float al = a.lo + dl + ml;
      // a^2 = ah^2 + 2 ah al (al^2 is below the working precision)
      const F2 sq = two_prod(a.hi, a.hi);
      const float sql = __fmaf_rn(2.0f * a.hi, al, sq.lo);
      if (k == 0) {
        r2h = sq.hi;
        r2l = sql;
      } else {
        const F2 t = two_sum(r2h, sq.hi);
        r2h = t.hi;
        r2l += t.lo + sql;
      }
      ae = __fmaf_rn(a.hi, e[k].hi, ae);
    }
    const F2 r2 = two_sum(r2h, r2l);
    // k / r^2: a quotient of the hi parts (within 2 ulps), corrected by its
    // residual (formed by FMA, rounded at ~2^-46 of k)
    const float th = __fdividef(ch.w, r2.hi);
    float res = __fmaf_rn(-th, r2.hi, ch.w);
    res = __fmaf_rn(-th, r2.lo, res + cl.w);
    const float tl = __fdividef(res, r2.hi);
    const F2 s = two_sum(gh, th);
    gh = s.hi;
    gl += s.lo + tl;
    // k / r^2 along the link: r^2' = 2 a.e, r^2'' = 2 e.e, so
    // g' = -2 t (a.e) / r^2 and g'' = t / r^2 (8 (a.e)^2 / r^2 - 2 e.e), t = k / r^2
    const float ir2 = __fdividef(1.0f, r2.hi), u = ae * ir2;
    d1 = __fmaf_rn(-2.0f * th, u, d1);
    d2 = __fmaf_rn(th * ir2, __fmaf_rn(8.0f * ae, u, -2.0f * ee), d2);
  }
  gp = d1;
  gpp = d2;
  const F2 g = two_sum(gh, -1.0f);
  return g.hi + (g.lo + gl);
}
}  // namespace

// The root q of one link from its body-frame origin ps and direction es
// (float pairs) over the particle's nb split balls bs; GRID: ps and the
// centres share the 2^-12 grid (hi parts subtract exactly).
template <bool GRID>
__device__ __forceinline__ float link_root(const float4* __restrict__ bs, int nb, const F2 ps[3], const F2 es[3]) {
  // stage 1: FP32 Newton on h = f^(-1/2) - 1
  float lo = 0.f, hi = 1.f, q = 0.5f;
  for (int it = 0; it < 24; ++it) {
    float f0 = 0.f, f1 = 0.f, s0 = 0.f, s1 = 0.f;
    // p_lo + q e, then + (p_hi - c_hi) per ball: the centres' lo parts (2^-24
    // of a centre) are left to the accurate stage
    float a[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) a[k] = __fmaf_rn(q, es[k].hi, ps[k].lo);
    int b = 0;
    for (; b + 2 <= nb; b += 2) {
      const float4 ha = __ldg(bs + 2 * b), hb = __ldg(bs + 2 * b + 2);
      const float u0 = diff_hi(ps[0].hi, ha.x, GRID).hi + a[0];
      const float u1 = diff_hi(ps[1].hi, ha.y, GRID).hi + a[1];
      const float u2 = diff_hi(ps[2].hi, ha.z, GRID).hi + a[2];
      const float v0 = diff_hi(ps[0].hi, hb.x, GRID).hi + a[0];
      const float v1 = diff_hi(ps[1].hi, hb.y, GRID).hi + a[1];
      const float v2 = diff_hi(ps[2].hi, hb.z, GRID).hi + a[2];
      const float iu = __fdividef(1.f, u0 * u0 + u1 * u1 + u2 * u2), iv = __fdividef(1.f, v0 * v0 + v1 * v1 + v2 * v2);
      const float tu = ha.w * iu, tv = hb.w * iv;
      f0 += tu;
      f1 += tv;
      // f' = -2 sum k (a . e) / r^4: the factor -2 is applied to the sums
      s0 = __fmaf_rn(tu * iu, u0 * es[0].hi + u1 * es[1].hi + u2 * es[2].hi, s0);
      s1 = __fmaf_rn(tv * iv, v0 * es[0].hi + v1 * es[1].hi + v2 * es[2].hi, s1);
    }
    if (b < nb) {
      const float4 ha = __ldg(bs + 2 * b);
      const float u0 = diff_hi(ps[0].hi, ha.x, GRID).hi + a[0];
      const float u1 = diff_hi(ps[1].hi, ha.y, GRID).hi + a[1];
      const float u2 = diff_hi(ps[2].hi, ha.z, GRID).hi + a[2];
      const float iu = __fdividef(1.f, u0 * u0 + u1 * u1 + u2 * u2);
      const float tu = ha.w * iu;
      f0 += tu;
      s0 = __fmaf_rn(tu * iu, u0 * es[0].hi + u1 * es[1].hi + u2 * es[2].hi, s0);
    }
    const float f = f0 + f1, fp = -2.f * (s0 + s1);
    if (f >= 1.f) hi = q;
    else lo = q;
    // Newton on h: q + 2 f (1 - sqrt f) / f'
    const float step = 2.f * f * (1.f - f * rsqrtf(f)) / fp;
    float qn = q + step;
    // a step below 1e-3 ends the stage (taken, clamped to the bracket): h is
    // close to linear, so the step leaves far less than the FP32 field's
    // noise behind, which the accurate stage removes
    if (fabsf(step) < 1e-3f) {
      q = fminf(fmaxf(qn, lo), hi);
      break;
    }
    if (!(qn > lo && qn < hi)) qn = 0.5f * (lo + hi);
    q = qn;
    if (hi - lo < 1e-6f) break;
  }
  // stage 2: double-float Newton
  lo = 0.f;
  hi = 1.f;
  const float ee = es[0].hi * es[0].hi + es[1].hi * es[1].hi + es[2].hi * es[2].hi;
  for (int it = 0; it < 4; ++it) {
    float gp, gpp;
    const float g = residual_ff<GRID>(bs, nb, ps, es, q, ee, gp, gpp);
    if (g >= 0.f) hi = q;
    else lo = q;
    const float step = g / gp;
    float qn = q - step;
    // the step ends the stage when it is below 2e-5, or when Newton's error
    // after it, |g'' / 2 g'| step^2, is below 1e-7 (and it stays in the bracket)
    if (fabsf(step) < 2e-5f || (qn >= lo && qn <= hi && fabsf(gpp) * step * step <= 2e-7f * fabsf(gp))) {
      q = fminf(fmaxf(qn, lo), hi);
      break;
    }
    if (!(qn > lo && qn < hi)) qn = 0.5f * (lo + hi);
    q = qn;
  }
  return q;
}

__global__ void __launch_bounds__(256) k_links_q(ParticleLaunch L) {
  const unsigned nl = min(L.ctr->n_links, L.cap_links);
  const unsigned nbc = min(L.ctr->n_bc, L.cap_bc);
  for (unsigned l = blockIdx.x * blockDim.x + threadIdx.x; l < nl; l += gridDim.x * blockDim.x) {
    const unsigned bi = L.link_bc[l];
    if (bi >= nbc) continue;
    // an entry of this step: inside the range of the node it names, whose
    // links all fitted (entries of a node that overflowed were not written)
    const unsigned loff = L.bc_loff[bi], m = __popc(L.bc_mask[bi]);
    if (l < loff || l - loff >= m || (unsigned long long)loff + m > (unsigned long long)L.cap_links) continue;
    const long long c = L.bc_cell[bi];
    const int d = L.link_dir[l];
    const DevParticle& P = L.P[L.link_p[l]];
    // node indices of particle lists fit in 32 bits (the lists store them as uint32)
    const unsigned cu = (unsigned)c, row = cu / (unsigned)L.g.nx;
    const int x = (int)(cu - row * (unsigned)L.g.nx), z = (int)(row / (unsigned)L.g.ny), y = (int)(row - (unsigned)z * L.g.ny);
    // body-frame link origin p = R^T (x - X) = R^T n - R^T (X - floor X), n = x - floor X
    // an exact small integer vector, in float-float arithmetic from the
    // prologue's float pairs (TwoProduct of R_hi n exact, R_lo n below it)
    const float n[3] = {(float)(x - P.pos_i[0]), (float)(y - P.pos_i[1]), (float)(z - P.pos_i[2])};
    F2 ps[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      F2 acc = {-P.Ts[0][k], -P.Ts[1][k]};
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        F2 t = two_prod(P.Rs[0][3 * a + k], n[a]);
        t.lo = __fmaf_rn(P.Rs[1][3 * a + k], n[a], t.lo);
        acc = df_add(acc, t);
      }
      ps[k] = acc;
    }
    // on the 2^-12 grid (|p|, |c| < 1024, split the same way by the host) the
    // hi parts subtract exactly; larger particles take TwoSum
    const bool grid = P.Rb_f < 1000.f;
    if (grid)
      for (int k = 0; k < 3; ++k) ps[k] = to_grid(ps[k]);
    const F2 es[3] = {{P.Es[d][0], P.Es[d][3]}, {P.Es[d][1], P.Es[d][4]}, {P.Es[d][2], P.Es[d][5]}};
    const float4* bs = L.balls_s + 2 * (size_t)P.ball_off;
    const int nb = P.n_balls;
    const float q = grid ? link_root<true>(bs, nb, ps, es) : link_root<false>(bs, nb, ps, es);
    L.link_q[l] = fminf(fmaxf(q, 1e-6f), 1.0f);
  }
}

cudaError_t launch_links_q(const ParticleLaunch& L, int grid, cudaStream_t s) {
  if (L.np == 0) return cudaSuccess;
  // no more blocks than the link list's capacity can use
  const unsigned long long need = ((unsigned long long)L.cap_links + 255ull) / 256ull;
  if (need < (unsigned long long)grid) grid = need < 1 ? 1 : (int)need;
  k_links_q<<<grid, 256, 0, s>>>(L);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Rigid-body update, four lanes of a warp per particle (rigid_dev.cuh).
// ---------------------------------------------------------------------------
__global__ void k_integrate(IntegrateLaunch L) {
  const int p = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (p < L.np) integrate_particle_lanes(L, p, threadIdx.x & 31);
}

cudaError_t launch_integrate(const IntegrateLaunch& L, cudaStream_t s) {
  if (L.np == 0) return cudaSuccess;
  k_integrate<<<(L.np + 3) / 4, 128, 0, s>>>(L);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Mass properties: midpoint quadrature of the indicator f >= 1 (FP32 with the
// FP64 guard band), FP64 moment sums per block.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_mass(const float4* balls, const double* balls_d, int nb, double Rb,
                                              double h, int n, double* partials) {
  __shared__ double red[10][256];
  double acc[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  const long long total = (long long)n * n * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int ix = (int)(i % n), iy = (int)((i / n) % n), iz = (int)(i / ((long long)n * n));
    const double X = __dadd_rn(-Rb, __dmul_rn(ix + 0.5, h));
    const double Y = __dadd_rn(-Rb, __dmul_rn(iy + 0.5, h));
    const double Z = __dadd_rn(-Rb, __dmul_rn(iz + 0.5, h));
    if (mass_sample_inside(balls, balls_d, nb, X, Y, Z)) mass_sample_accumulate(acc, X, Y, Z);
  }
  for (int k = 0; k < 10; ++k) red[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st)
      for (int k = 0; k < 10; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int k = 0; k < 10; ++k) partials[10 * blockIdx.x + k] = red[k][0];
}

cudaError_t launch_mass_quadrature(const float4* balls, const double* balls_d, int n_balls, double Rb, double h,
                                   int n_side, double* partials, int blocks, cudaStream_t s) {
  k_mass<<<blocks, 256, 0, s>>>(balls, balls_d, n_balls, Rb, h, n_side, partials);
  return cudaGetLastError();
}

}  // namespace mi
