// DEM contact kernels (Sec. 2.3.1): broad phase, Newton-Raphson closest points
// between sphero-metaball particles (Eqs. CM_coreF, grad, cp, contactprop) and
// between a particle and an axis-aligned wall (Eqs. metawallcp, contactprop2),
// linear spring-dashpot forces with a Coulomb-limited tangential spring.
//
// The core of a particle is the iso-surface g = s f = 1, s = ((r_e - R_s)/r_e)^2,
// r_e = sqrt(sum k).  One warp solves one candidate: the balls of each particle
// are spread over the lanes, the 10 sums of g, grad g and the Hessian are
// shuffle-reduced (and broadcast from lane 0, so every lane takes identical
// branches), and the 3x3 (4x4 for walls) Newton system is solved redundantly
// in every lane.  Work is taken from an atomic counter (no inter-block waits);
// a warp leaves when the queue is empty.  Geometry is FP32 in a local frame
// centred between the particles; the spring-dashpot forces are FP32 from
// velocities staged per substep, summed per particle in 2^-40 fixed point
// (order-free); the tangential spring is stored in FP64.
#include "contact_dev.cuh"
#include "rigid_dev.cuh"

namespace mi {

namespace {
using namespace cdev;

__device__ __forceinline__ void add_fixed6(long long* acc, int p, const float v[6]) {
  for (int k = 0; k < 6; ++k)
    atomicAdd(reinterpret_cast<unsigned long long*>(acc + 6 * p + k),
              (unsigned long long)__float2ll_rn(v[k] * (float)FIX_SCALE));
}

// Velocity of the material point at offset r from the origin of a particle
// whose staged (v, omega) are vw[0], vw[1]: v + omega x r.
__device__ __forceinline__ void point_velocity(const float4* vw, const float r[3], float v[3]) {
  const float4 a = vw[0], w = vw[1];
  v[0] = a.x + w.y * r[2] - w.z * r[1];
  v[1] = a.y + w.z * r[0] - w.x * r[2];
  v[2] = a.z + w.x * r[1] - w.y * r[0];
}

// Spring-dashpot force on particle i at the contact point x_c = X_i + ri
// (the partner j at x_c = X_j + rj, or a wall at rest when vwj == nullptr):
// normal n (from i towards j), overlap delta.  FP32; the tangential spring
// of the history entry is FP64 in memory.
__device__ void spring_dashpot(const DashF& c, const float4* vwi, const float4* vwj, const float ri[3],
                               const float rj[3], const float n[3], float delta, HistEntry* h, long long substep,
                               float f[3]) {
  float v0[3], v1[3] = {0.f, 0.f, 0.f};
  point_velocity(vwi, ri, v0);
  if (vwj) point_velocity(vwj, rj, v1);
  float vr[3], vt[3];
  for (int a = 0; a < 3; ++a) vr[a] = v1[a] - v0[a];
  const float vn = vr[0] * n[0] + vr[1] * n[1] + vr[2] * n[2];
  for (int a = 0; a < 3; ++a) vt[a] = vr[a] - vn * n[a];
  const float Fn = fmaxf(0.f, c.kn * delta + c.eta_n * vn);
  float xi[3] = {0.f, 0.f, 0.f};
  if (h->stamp == substep - 1)
    for (int a = 0; a < 3; ++a) xi[a] = (float)h->xi[a];
  const float xn = xi[0] * n[0] + xi[1] * n[1] + xi[2] * n[2];
  for (int a = 0; a < 3; ++a) xi[a] = xi[a] - xn * n[a] + vt[a] * c.dt;
  float Ft[3];
  for (int a = 0; a < 3; ++a) Ft[a] = c.kt * xi[a] + c.eta_t * vt[a];
  const float nt = sqrtf(Ft[0] * Ft[0] + Ft[1] * Ft[1] + Ft[2] * Ft[2]);
  if (nt > c.mu_s * Fn) {
    if (nt > 0.f)
      for (int a = 0; a < 3; ++a) Ft[a] *= c.mu_s * Fn / nt;
    for (int a = 0; a < 3; ++a) xi[a] = c.kt > 0.f ? (Ft[a] - c.eta_t * vt[a]) / c.kt : 0.f;
  }
  for (int a = 0; a < 3; ++a) {
    f[a] = Fn * n[a] + Ft[a];
    h->xi[a] = (double)xi[a];
  }
  h->stamp = substep;
}
}  // namespace

// Per-substep FP32 staging of particle k: position split as hi + lo (hi = the
// position rounded to FP32, lo = the remainder rounded), radius, unit
// quaternion, velocity and angular velocity.
__device__ __forceinline__ void stage_particle(const ContactLaunch& L, int k) {
  const DevParticle& P = L.P[k];
  const float hx = (float)P.pos[0], hy = (float)P.pos[1], hz = (float)P.pos[2];
  L.pf[k] = make_float4(hx, hy, hz, P.Rb_f);
  L.plo[k] = make_float4((float)(P.pos[0] - hx), (float)(P.pos[1] - hy), (float)(P.pos[2] - hz), 0.f);
  L.qf[k] = unit_quat_f32(P.quat);
  L.vw[2 * k] = make_float4((float)P.vel[0], (float)P.vel[1], (float)P.vel[2], 0.f);
  L.vw[2 * k + 1] = make_float4((float)P.omega[0], (float)P.omega[1], (float)P.omega[2], 0.f);
}

// ---------------------------------------------------------------------------
__global__ void k_dem_prologue(ContactLaunch L) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    *L.substep += 1;
    L.ctr->n_pairs = 0;
    L.ctr->n_contacts = 0;
    *L.work = 0;
  }
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < 6 * L.np; k += gridDim.x * blockDim.x) L.fcacc[k] = 0;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < L.np; k += gridDim.x * blockDim.x) stage_particle(L, k);
}

cudaError_t launch_dem_prologue(const ContactLaunch& L, cudaStream_t s) {
  k_dem_prologue<<<(L.np + 255) / 256 + 1, 256, 0, s>>>(L);
  return cudaGetLastError();
}

__device__ __forceinline__ void append_item(const ContactLaunch& L, int i, int j) {
  const unsigned k = atomicAdd(&L.ctr->n_pairs, 1u);
  if (k < L.cap_items) {
    L.item_i[k] = i;
    L.item_j[k] = j;
  } else {
    atomicOr(&L.ctr->status, STATUS_PAIR_OVERFLOW);
  }
}

constexpr int BP_TILE = 64;

// Pair (i, j) with staged (FP32 position, R_b) pa, pb: FP32 filter with an
// error band, FP64 decision inside it (the decision is the FP64 one).
__device__ __forceinline__ bool pair_candidate(const ContactLaunch& L, int i, int j, const float4 pa, const float4 pb) {
  const float dx = pa.x - pb.x, dy = pa.y - pb.y, dz = pa.z - pb.z;
  const float dd = sqrtf(dx * dx + dy * dy + dz * dz);
  const float thr = pa.w + pb.w + (float)L.cp.margin;
  const float band = 2.4e-7f * (fabsf(pa.x) + fabsf(pa.y) + fabsf(pa.z) + fabsf(pb.x) + fabsf(pb.y) + fabsf(pb.z)) +
                     1e-5f * thr + 1e-6f;
  if (dd > thr + band) return false;
  if (dd >= thr - band) {
    const DevParticle& P = L.P[i];
    const DevParticle& Q = L.P[j];
    const double d0 = P.pos[0] - Q.pos[0], d1 = P.pos[1] - Q.pos[1], d2 = P.pos[2] - Q.pos[2];
    if (!(sqrt(d0 * d0 + d1 * d1 + d2 * d2) <= P.Rb + Q.Rb + L.cp.margin)) return false;
  }
  return true;
}

// Particle j against the domain wall on face (0..5), FP64.
__device__ __forceinline__ bool wall_candidate(const ContactLaunch& L, int j, int face) {
  const int axis = face / 2;
  if (L.cp.periodic[axis]) return false;
  const double pw = (face & 1) ? L.cp.n[axis] - 0.5 : -0.5;
  const double nw = (face & 1) ? -1.0 : 1.0;
  return nw * (L.P[j].pos[axis] - pw) <= L.P[j].Rb + L.cp.margin;
}

// Candidates: pairs i < j with |X_i - X_j| <= R_b,i + R_b,j + margin, and
// particle-wall items with n_w.(X_i - p_w) <= R_b,i + margin, both decided in
// FP64.  The pairs come in 64 x 64 tiles of the upper triangle, one block per
// tile, with both particle ranges staged in shared memory; the blocks after
// the tiles take the particle-wall items.  An FP32 filter settles every pair
// whose FP32 distance lies farther from the threshold than a bound on its
// error (each coordinate carries at most 2^-24 of its magnitude from rounding,
// taken four times over; 1e-5 of the threshold covers the radii and the FP32
// arithmetic); the rest take the FP64 test, so the list is the FP64 one.
__global__ void __launch_bounds__(128) k_broad_phase(ContactLaunch L, int n_tiles) {
  __shared__ float4 A[BP_TILE], Bt[BP_TILE];
  const int np = L.np;
  const int b = blockIdx.x;
  if (b < n_tiles) {
    // tile (ti, tj), ti <= tj, enumerated as b = tj (tj + 1) / 2 + ti
    int tj = (int)((sqrtf(8.0f * (float)b + 1.0f) - 1.0f) * 0.5f);
    while (tj * (tj + 1) / 2 > b) --tj;
    while ((tj + 1) * (tj + 2) / 2 <= b) ++tj;
    const int ti = b - tj * (tj + 1) / 2;
    const int i0 = ti * BP_TILE, j0 = tj * BP_TILE;
    if (threadIdx.x < BP_TILE) {
      const int k = i0 + threadIdx.x;
      A[threadIdx.x] = k < np ? L.pf[k] : make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
      const int k = j0 + threadIdx.x - BP_TILE;
      Bt[threadIdx.x - BP_TILE] = k < np ? L.pf[k] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < BP_TILE * BP_TILE; e += 128) {
      const int a = e / BP_TILE, c = e % BP_TILE;
      const int i = i0 + a, j = j0 + c;
      if (i >= j || j >= np) continue;
      if (pair_candidate(L, i, j, A[a], Bt[c])) append_item(L, i, j);
    }
  } else {
    const int t = (b - n_tiles) * 128 + threadIdx.x;
    if (t >= 6 * np) return;
    if (wall_candidate(L, t / 6, t % 6)) append_item(L, t / 6, -1 - t % 6);
  }
}

cudaError_t launch_broad_phase(const ContactLaunch& L, cudaStream_t s) {
  if (L.np <= 0) return cudaSuccess;
  const int nt = (L.np + BP_TILE - 1) / BP_TILE;
  const int n_tiles = nt * (nt + 1) / 2;
  const int wall_blocks = (6 * L.np + 127) / 128;
  k_broad_phase<<<n_tiles + wall_blocks, 128, 0, s>>>(L, n_tiles);
  return cudaGetLastError();
}

// One candidate item (a particle pair or a particle-wall pair) by one warp:
// Newton closest point, contact geometry, spring-dashpot force into the
// fixed-point sums, and the item's record.  sub, stage and rad are the warp's
// shared scratch (2 x SUB_CAP indices, NT_CAP balls).  WARM and LEARNED are
// the handle's warm-start and learned-start switches, fixed per kernel
// variant so that each variant holds only the code of its starts.
template <bool WARM, bool LEARNED>
__device__ __forceinline__ void contact_item(const ContactLaunch& L, unsigned it, long long substep, int lane,
                                             unsigned short (*sub)[SUB_CAP], float4* stage, float* rad) {
  const float4* balls = L.balls;
  {
    const int i = L.item_i[it], j = L.item_j[it];
    const DevParticle& Pi = L.P[i];
    int status = 1, iters = 0;
    float rel[3], nf[3], dl;  // contact point - X_i, normal, overlap (FP32)
    if (j >= 0) {
      // ---------------- particle pair ----------------
      const DevParticle& Pj = L.P[j];
      // h = (X_j - X_i) / 2 from the hi/lo split: the hi parts of nearby
      // particles subtract exactly, so h carries FP32 accuracy relative to
      // the pair's own size, not to the distance from the origin
      const float4 hi_i = L.pf[i], hi_j = L.pf[j], lo_i = L.plo[i], lo_j = L.plo[j];
      const float h[3] = {0.5f * ((hi_j.x - hi_i.x) + (lo_j.x - lo_i.x)), 0.5f * ((hi_j.y - hi_i.y) + (lo_j.y - lo_i.y)),
                          0.5f * ((hi_j.z - hi_i.z) + (lo_j.z - lo_i.z))};
      Frame F0, F1;
      pair_frames(Pi, Pj, L.qf[i], L.qf[j], h, F0, F1);
      const float Rb = fmaxf(Pi.Rb_f, Pj.Rb_f);
      const PairSolver S(F0, F1, balls, stage, rad, &sub[0][0], lane);
      float y[3];
      const int lo = min(i, j), hi = max(i, j);
      HistEntry* hp = L.hist_pair + ((long long)lo * L.ncap - (long long)lo * (lo + 1) / 2 + (hi - lo - 1));
      // substeps count from 1 and the history starts zeroed: a stamp is valid from 1 on
      const bool have_warm = WARM && substep >= 2 && hp->xm_stamp == substep - 1;
      if (have_warm) {
        // warm start: the pair's closest point of the previous substep (x - O = (x - X_i) - h)
        for (int c = 0; c < 3; ++c) y[c] = hp->xm_rel[c] - h[c];
        status = S.newton(y, NEWTON_TOL * Rb, MAX_IT, iters);
        if (status != 0) {  // the plain start decides
          int more = 0;
          status = S.plain_newton(y, NEWTON_TOL * Rb, more);
          iters += more;
        }
      } else if (LEARNED) {
        // learned start: anchor and prediction of this item (features and MLP ran before)
        const float* x = L.feat + (size_t)it * 64;
        const float* pr = L.pred + (size_t)it * 4;
        const float a[3] = {x[11], x[12], x[13]}, d[4] = {pr[0], pr[1], pr[2], pr[3]};
        SolveCount sc;
        status = S.learned(a, d, Rb, Rb, sub[0], sub[1], y, sc);
        iters = sc.iters;
      } else {
        // plain start: closest pair of control-point spheres, midpoint of their surface points
        status = S.plain_newton(y, NEWTON_TOL * Rb, iters);
      }
      GEval e0, e1;
      S.final_eval(y, e0.g, e0.gr, e1.g, e1.gr);
      if (status == 0) {
        if (e0.g >= 1.f || e1.g >= 1.f) status = 3;
        else if (e0.g < C_TOL || e1.g < C_TOL) status = 4;
      }
      // first-order projections onto the two cores, the normal between them,
      // the overlap of the skins and the contact point (Eqs. cp, contactprop)
      const float q0 = (1.f - e0.g) / (e0.gr[0] * e0.gr[0] + e0.gr[1] * e0.gr[1] + e0.gr[2] * e0.gr[2]);
      const float q1 = (1.f - e1.g) / (e1.gr[0] * e1.gr[0] + e1.gr[1] * e1.gr[1] + e1.gr[2] * e1.gr[2]);
      float xc0[3], xc1[3], d[3];
      for (int c = 0; c < 3; ++c) {
        xc0[c] = y[c] + q0 * e0.gr[c];
        xc1[c] = y[c] + q1 * e1.gr[c];
        d[c] = xc0[c] - xc1[c];
      }
      const float dist = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      dl = Pi.skin_f + Pj.skin_f - dist;
      for (int c = 0; c < 3; ++c) {
        nf[c] = dist > 0.f ? d[c] / dist : 0.f;
        rel[c] = h[c] + xc0[c] - (Pi.skin_f - 0.5f * dl) * nf[c];
      }
      if (lane == 0 && WARM && status == 0) {
        for (int c = 0; c < 3; ++c) hp->xm_rel[c] = y[c] + h[c];
        hp->xm_stamp = substep;
      }
      if (lane == 0 && status == 0 && dl > 0.f) {
        // x_c - X_j = (x_c - X_i) - (X_j - X_i) = rel - 2 h
        const float rj[3] = {rel[0] - 2.f * h[0], rel[1] - 2.f * h[1], rel[2] - 2.f * h[2]};
        float f[3];
        spring_dashpot(L.cf, L.vw + 2 * i, L.vw + 2 * j, rel, rj, nf, dl, hp, substep, f);
        const float vi[6] = {f[0], f[1], f[2], rel[1] * f[2] - rel[2] * f[1], rel[2] * f[0] - rel[0] * f[2],
                             rel[0] * f[1] - rel[1] * f[0]};
        const float vj[6] = {-f[0], -f[1], -f[2], -(rj[1] * f[2] - rj[2] * f[1]), -(rj[2] * f[0] - rj[0] * f[2]),
                             -(rj[0] * f[1] - rj[1] * f[0])};
        add_fixed6(L.fcacc, i, vi);
        add_fixed6(L.fcacc, j, vj);
        atomicAdd(&L.ctr->n_contacts, 1u);
      }
    } else {
      // ---------------- particle - wall ----------------
      const int face = -1 - j, axis = face / 2;
      const float zero[3] = {0.f, 0.f, 0.f};
      const Frame F0 = frame_f32(Pi, L.qf[i], zero);  // local origin X_i
      float nw[3] = {0.f, 0.f, 0.f};
      nw[axis] = (face & 1) ? -1.f : 1.f;
      const double pw = (face & 1) ? L.cp.n[axis] - 0.5 : -0.5;
      const float distO = (float)((double)nw[axis] * (Pi.pos[axis] - pw));
      const float Rb = Pi.Rb_f;
      // guess: the core sphere reaching deepest towards the wall
      float best = 3.4e38f;
      int ba = 0;
      for (int a = lane; a < F0.n; a += 32) {
        const float4 ca = __ldg(balls + F0.off + a);
        const float pn = (F0.R[3 * axis] * ca.x + F0.R[3 * axis + 1] * ca.y + F0.R[3 * axis + 2] * ca.z + F0.t[axis]) * nw[axis];
        const float v = pn - sqrtf(F0.s * ca.w);
        if (v < best) { best = v; ba = a; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const float g2 = __shfl_xor_sync(FULL, best, o);
        const int a2 = __shfl_xor_sync(FULL, ba, o);
        if (g2 < best || (g2 == best && a2 < ba)) { best = g2; ba = a2; }
      }
      ba = __shfl_sync(FULL, ba, 0);
      float y[3];
      {
        const float4 ca = __ldg(balls + F0.off + ba);
        const float rs = sqrtf(F0.s * ca.w);
        for (int c = 0; c < 3; ++c)
          y[c] = F0.R[3 * c] * ca.x + F0.R[3 * c + 1] * ca.y + F0.R[3 * c + 2] * ca.z + F0.t[c] - rs * nw[c];
      }
      GEval e = eval(F0, balls, y, lane);
      float lam = sqrtf(e.gr[0] * e.gr[0] + e.gr[1] * e.gr[1] + e.gr[2] * e.gr[2]);
      for (iters = 1; iters <= MAX_IT; ++iters) {
        e = eval(F0, balls, y, lane);
        float A[4][4] = {{e.H[0], e.H[1], e.H[2], -nw[0]},
                         {e.H[1], e.H[3], e.H[4], -nw[1]},
                         {e.H[2], e.H[4], e.H[5], -nw[2]},
                         {e.gr[0], e.gr[1], e.gr[2], 0.f}};
        float b[4] = {e.gr[0] - lam * nw[0], e.gr[1] - lam * nw[1], e.gr[2] - lam * nw[2], e.g - 1.f};
        float dz[4];
        if (!solve<4>(A, b, dz)) { status = 2; break; }
        for (int c = 0; c < 3; ++c) y[c] -= dz[c];
        lam -= dz[3];
        if (sqrtf(dz[0] * dz[0] + dz[1] * dz[1] + dz[2] * dz[2]) <= NEWTON_TOL * Rb) { status = 0; break; }
      }
      if (iters > MAX_IT) iters = MAX_IT;
      const float dist = nw[0] * y[0] + nw[1] * y[1] + nw[2] * y[2] + distO;
      dl = Pi.skin_f - dist;
      for (int c = 0; c < 3; ++c) {
        nf[c] = nw[c];
        rel[c] = (y[c] - dist * nw[c]) + 0.5f * dl * nw[c];
      }
      if (lane == 0 && status == 0 && dl > 0.f) {
        HistEntry* hp = L.hist_wall + ((long long)i * 6 + face);
        float f[3];
        spring_dashpot(L.cf, L.vw + 2 * i, nullptr, rel, nullptr, nw, dl, hp, substep, f);
        const float vi[6] = {f[0], f[1], f[2], rel[1] * f[2] - rel[2] * f[1], rel[2] * f[0] - rel[0] * f[2],
                             rel[0] * f[1] - rel[1] * f[0]};
        add_fixed6(L.fcacc, i, vi);
        atomicAdd(&L.ctr->n_contacts, 1u);
      }
    }
    if (lane == 0) {
      ContactRec& r = L.recs[it];
      r.i = i;
      r.j = j;
      for (int c = 0; c < 3; ++c) {
        r.X[c] = Pi.pos[c];
        r.r[c] = rel[c];
        r.n[c] = nf[c];
      }
      r.delta = dl;
      r.iters = iters;
      r.status = status;
    }
  }
}

// Persistent warp-per-candidate Newton solver and forces.
template <bool WARM, bool LEARNED>
__global__ void __launch_bounds__(128, 6) k_contacts(ContactLaunch L) {
  __shared__ unsigned short sub[4][2][SUB_CAP];  // active subsets of the learned start, per warp
  __shared__ float4 stage[4][NT_CAP];              // the pair's staged balls, per warp
  __shared__ float rad[4][NT_CAP];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned n_items = min(L.ctr->n_pairs, L.cap_items);
  const long long substep = *L.substep;
  for (;;) {
    unsigned it = 0;
    if (lane == 0) it = atomicAdd(L.work, 1u);
    it = __shfl_sync(FULL, it, 0);
    if (it >= n_items) break;
    contact_item<WARM, LEARNED>(L, it, substep, lane, sub[w], stage[w], rad[w]);
  }
}

cudaError_t launch_contacts(const ContactLaunch& L, cudaStream_t s) {
  // the starts are exclusive (the handle's guess mode)
  if (L.learned) k_contacts<false, true><<<L.grid, 128, 0, s>>>(L);
  else if (L.warm) k_contacts<true, false><<<L.grid, 128, 0, s>>>(L);
  else k_contacts<false, false><<<L.grid, 128, 0, s>>>(L);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// The DEM substeps of one LBM step for a handful of particles in one CTA:
// the first substep's rigid-body update (its contacts ran beside the bulk
// kernel), then for every further substep the prologue, every pair and wall
// candidate test, the warp-per-item solves and the rigid-body update, with
// block barriers between them instead of launches.  The work per item is the
// per-kernel path's (same device functions), so the results are the same
// bits.  Counters and force sums that other threads updated with atomics are
// read past the L1 (__ldcg); everything else is written and read by this
// block only.
// ---------------------------------------------------------------------------
template <bool WARM>
__global__ void __launch_bounds__(128) k_dem_substeps(ContactLaunch L, IntegrateLaunch I, int n_sub) {
  __shared__ unsigned short sub[4][2][SUB_CAP];
  __shared__ float4 stage[4][NT_CAP];
  __shared__ float rad[4][NT_CAP];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int np = L.np;
  for (int p = w; p < np; p += 4) integrate_particle_lanes(I, p, lane);
  __syncthreads();
  const int npairs = np * (np - 1) / 2;
  for (int k = 1; k < n_sub; ++k) {
    if (t == 0) {
      *L.substep += 1;
      L.ctr->n_pairs = 0;
      L.ctr->n_contacts = 0;
    }
    for (int q = t; q < 6 * np; q += blockDim.x) L.fcacc[q] = 0;
    for (int q = t; q < np; q += blockDim.x) stage_particle(L, q);
    __syncthreads();
    for (int e = t; e < npairs + 6 * np; e += blockDim.x) {
      if (e < npairs) {
        // e = j (j - 1) / 2 + i, 0 <= i < j
        int j = (int)((1.0f + sqrtf(1.0f + 8.0f * (float)e)) * 0.5f);
        while (j * (j - 1) / 2 > e) --j;
        while ((j + 1) * j / 2 <= e) ++j;
        const int i = e - j * (j - 1) / 2;
        if (pair_candidate(L, i, j, L.pf[i], L.pf[j])) append_item(L, i, j);
      } else {
        const int u = e - npairs;
        if (wall_candidate(L, u / 6, u % 6)) append_item(L, u / 6, -1 - u % 6);
      }
    }
    __syncthreads();
    const unsigned n_items = min(__ldcg(&L.ctr->n_pairs), L.cap_items);
    const long long substep = *L.substep;
    for (unsigned it = w; it < n_items; it += 4) contact_item<WARM, false>(L, it, substep, lane, sub[w], stage[w], rad[w]);
    __syncthreads();
    for (int p = w; p < np; p += 4) integrate_particle_lanes(I, p, lane);
    __syncthreads();
  }
}

cudaError_t launch_dem_substeps(const ContactLaunch& L, const IntegrateLaunch& I, int n_sub, cudaStream_t s) {
  if (L.np <= 0 || n_sub <= 0) return cudaSuccess;
  if (L.warm) k_dem_substeps<true><<<1, 128, 0, s>>>(L, I, n_sub);
  else k_dem_substeps<false><<<1, 128, 0, s>>>(L, I, n_sub);
  return cudaGetLastError();
}

}  // namespace mi
