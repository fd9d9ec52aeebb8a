// Internal declarations shared by the CUDA translation units of libmi_delbm.
// Nothing here is part of the C-ABI (include/mi_delbm.h is).
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "mi_delbm.h"

namespace mi {

// ---------------------------------------------------------------------------
// D3Q19 lattice (C = 1, c_s^2 = 1/3).  Order: rest, +x,-x,+y,-y,+z,-z, then
// the twelve edge diagonals each followed by its opposite.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int cx(int i) {
  constexpr int t[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
  return t[i];
}
__host__ __device__ constexpr int cy(int i) {
  constexpr int t[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
  return t[i];
}
__host__ __device__ constexpr int cz(int i) {
  constexpr int t[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
  return t[i];
}
__host__ __device__ constexpr float wq(int i) {
  return i == 0 ? (1.0f / 3.0f) : (i <= 6 ? (1.0f / 18.0f) : (1.0f / 36.0f));
}
__host__ __device__ constexpr double wq_d(int i) {
  return i == 0 ? (1.0 / 3.0) : (i <= 6 ? (1.0 / 18.0) : (1.0 / 36.0));
}
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }

// Direction components as 2-bit fields (value + 1), so that a thread can look
// up a direction given at run time without local or constant memory.
__host__ __device__ constexpr unsigned long long dir_pack(int axis) {
  unsigned long long v = 0;
  for (int i = 0; i < 19; ++i)
    v |= (unsigned long long)((axis == 0 ? cx(i) : (axis == 1 ? cy(i) : cz(i))) + 1) << (2 * i);
  return v;
}
constexpr unsigned long long EXB = dir_pack(0), EYB = dir_pack(1), EZB = dir_pack(2);
__device__ __forceinline__ int lex(int j) { return (int)((EXB >> (2 * j)) & 3ull) - 1; }
__device__ __forceinline__ int ley(int j) { return (int)((EYB >> (2 * j)) & 3ull) - 1; }
__device__ __forceinline__ int lez(int j) { return (int)((EZB >> (2 * j)) & 3ull) - 1; }

constexpr uint32_t OWNER_NONE = 0xFFFFFFFFu;

// node class bits
constexpr uint8_t CLS_SOLID = 1u;
constexpr uint8_t CLS_BOUNDARY = 2u;
constexpr uint8_t CLS_NEW = 4u;

// ---------------------------------------------------------------------------
// Population storage.  Every storage hands the kernels the deviation
// h_i = f_i - w_i as float; F32 stores f_i itself (f - w is exact in FP32 for
// f within a factor two of w), the 16-bit storages store h_i rounded to
// nearest even.
// ---------------------------------------------------------------------------
template <int ST> struct Store;
template <> struct Store<MI_STORE_F32> {
  using T = float;
  static __device__ __forceinline__ float dev(const float* p, int i) { return __ldg(p) - wq(i); }
  static __device__ __forceinline__ void put(float* p, int i, float h) { __stcs(p, h + wq(i)); }
};
template <> struct Store<MI_STORE_F16_DEV> {
  using T = __half;
  static __device__ __forceinline__ float dev(const __half* p, int) {
    return __half2float(__ushort_as_half(__ldg(reinterpret_cast<const unsigned short*>(p))));
  }
  static __device__ __forceinline__ void put(__half* p, int, float h) {
    __stcs(reinterpret_cast<unsigned short*>(p), __half_as_ushort(__float2half_rn(h)));
  }
};
template <> struct Store<MI_STORE_BF16_DEV> {
  using T = __nv_bfloat16;
  static __device__ __forceinline__ float dev(const __nv_bfloat16* p, int) {
    return __bfloat162float(__ushort_as_bfloat16(__ldg(reinterpret_cast<const unsigned short*>(p))));
  }
  static __device__ __forceinline__ void put(__nv_bfloat16* p, int, float h) {
    __stcs(reinterpret_cast<unsigned short*>(p), __bfloat16_as_ushort(__float2bfloat16_rn(h)));
  }
};

inline size_t store_bytes(int st) { return st == MI_STORE_F32 ? 4 : 2; }

// Two x-adjacent stored elements read or written as one aligned access
// (the first element at an even index).  P is the register type of a pair.
template <int ST> struct Pair;
template <> struct Pair<MI_STORE_F32> {
  using P = float2;
  static __device__ __forceinline__ P load(const float* p) { return __ldg(reinterpret_cast<const float2*>(p)); }
  static __device__ __forceinline__ float lo(P v, int i) { return v.x - wq(i); }
  static __device__ __forceinline__ float hi(P v, int i) { return v.y - wq(i); }
  static __device__ __forceinline__ void put(float* p, int i, float a, float b) {
    __stcs(reinterpret_cast<float2*>(p), make_float2(a + wq(i), b + wq(i)));
  }
  static __device__ __forceinline__ P shfl_up(P v) {
    return make_float2(__shfl_up_sync(0xffffffffu, v.x, 1), __shfl_up_sync(0xffffffffu, v.y, 1));
  }
  static __device__ __forceinline__ P shfl_down(P v) {
    return make_float2(__shfl_down_sync(0xffffffffu, v.x, 1), __shfl_down_sync(0xffffffffu, v.y, 1));
  }
};
template <> struct Pair<MI_STORE_F16_DEV> {
  using P = unsigned int;
  static __device__ __forceinline__ P load(const __half* p) { return __ldg(reinterpret_cast<const unsigned int*>(p)); }
  static __device__ __forceinline__ float lo(P v, int) { return __half2float(__ushort_as_half((unsigned short)(v & 0xFFFFu))); }
  static __device__ __forceinline__ float hi(P v, int) { return __half2float(__ushort_as_half((unsigned short)(v >> 16))); }
  static __device__ __forceinline__ void put(__half* p, int, float a, float b) {
    const unsigned int v = (unsigned int)__half_as_ushort(__float2half_rn(a)) |
                           ((unsigned int)__half_as_ushort(__float2half_rn(b)) << 16);
    __stcs(reinterpret_cast<unsigned int*>(p), v);
  }
  static __device__ __forceinline__ P shfl_up(P v) { return __shfl_up_sync(0xffffffffu, v, 1); }
  static __device__ __forceinline__ P shfl_down(P v) { return __shfl_down_sync(0xffffffffu, v, 1); }
};
// 16-bit storage element <-> FP32 deviation
template <int ST> __device__ __forceinline__ float dev16(unsigned short u);
template <> __device__ __forceinline__ float dev16<MI_STORE_F16_DEV>(unsigned short u) {
  return __half2float(__ushort_as_half(u));
}
template <> __device__ __forceinline__ float dev16<MI_STORE_BF16_DEV>(unsigned short u) {
  return __uint_as_float((unsigned)u << 16);
}
template <int ST> __device__ __forceinline__ unsigned short pack16(float h);
template <> __device__ __forceinline__ unsigned short pack16<MI_STORE_F16_DEV>(float h) {
  return __half_as_ushort(__float2half_rn(h));
}
template <> __device__ __forceinline__ unsigned short pack16<MI_STORE_BF16_DEV>(float h) {
  return __bfloat16_as_ushort(__float2bfloat16_rn(h));
}

template <> struct Pair<MI_STORE_BF16_DEV> {
  using P = unsigned int;
  static __device__ __forceinline__ P load(const __nv_bfloat16* p) { return __ldg(reinterpret_cast<const unsigned int*>(p)); }
  static __device__ __forceinline__ float lo(P v, int) { return __uint_as_float(v << 16); }
  static __device__ __forceinline__ float hi(P v, int) { return __uint_as_float(v & 0xFFFF0000u); }
  static __device__ __forceinline__ void put(__nv_bfloat16* p, int, float a, float b) {
    const unsigned int v = (unsigned int)__bfloat16_as_ushort(__float2bfloat16_rn(a)) |
                           ((unsigned int)__bfloat16_as_ushort(__float2bfloat16_rn(b)) << 16);
    __stcs(reinterpret_cast<unsigned int*>(p), v);
  }
  static __device__ __forceinline__ P shfl_up(P v) { return __shfl_up_sync(0xffffffffu, v, 1); }
  static __device__ __forceinline__ P shfl_down(P v) { return __shfl_down_sync(0xffffffffu, v, 1); }
};

// ---------------------------------------------------------------------------
// Launch parameters of the lattice kernels.
// ---------------------------------------------------------------------------
struct LatticeGeom {
  int nx, ny, nz;
  int periodic[3];
  long long plane;   // elements between q planes
};

struct CollideParams {
  float omega;          // 1 / tau
  float force[3];       // Guo body force density (zero unless set)
  float bb_wall[6][19]; // 6 w_i rho0 (e_i . u_wall[face]) per face and direction
  float rho0;
};

// Bulk stream-collide launch (kernels in k_lbm.cu).
struct BulkLaunch {
  const void* A;       // f+(t)
  void* B;             // f+(t+1)
  LatticeGeom g;
  CollideParams p;
  int storage;
  bool forcing;
  int block_x;         // threads per block along x
  int rows = 1;        // consecutive rows (y) per thread: 1 or 2
  bool pairs = false;  // two x-adjacent nodes per thread with paired accesses (nx even)
  int pair_mode = 1;   // 16-bit paired kernel occupancy: 1 = up to 64 registers, 2 = up to 80
};
cudaError_t launch_bulk(const BulkLaunch& L, cudaStream_t s);

// Fill every node with the rest state f_i = w_i rho0.
cudaError_t launch_fill_rest(void* pop, const LatticeGeom& g, int storage, float rho0, cudaStream_t s);
// mi_delbm_check: out[0] = non-finite stored populations at non-solid nodes, out[1] = the first such node
cudaError_t launch_check(const void* pop, const LatticeGeom& g, int storage, const uint32_t* owner, long long* out,
                         int sm_count, cudaStream_t s);
// Convert float populations [19][ncell] (dense) to/from the storage layout.
cudaError_t launch_pack(const float* src, void* pop, const LatticeGeom& g, int storage, cudaStream_t s);
cudaError_t launch_unpack(const void* pop, float* dst, const LatticeGeom& g, int storage, cudaStream_t s);

// ---------------------------------------------------------------------------
// Particles
// ---------------------------------------------------------------------------
constexpr int BOX_NONE = -(1 << 30);  // "no box written" marker in box histories
constexpr double FIX_SCALE = 1099511627776.0;  // 2^40: fixed-point scale of force sums
constexpr double FIX_INV = 1.0 / 1099511627776.0;

// FP64 state of one particle (device table, one entry per particle).
struct DevParticle {
  double pos[3], quat[4], vel[3], omega[3];  // world frame; quat = (w, x, y, z)
  double mass, volume, density, skin, Rb, re;
  double Rt;                                 // tight radius: f < 1 beyond it (root of sum k/(r-|c|)^2 = 1)
  double inertia[9], inv_inertia[9];         // body frame, about the centroid
  double R[9];                               // body -> world rotation at the current pose
  float posf[3], velf[3], omegaf[3];         // FP32 copies for the lattice kernels
  int pos_i[3];                              // floor(pos), and pos - floor(pos) in FP32: node offsets
  float pos_fr[3];                           //   x - X = (x - pos_i) - pos_fr without FP64 arithmetic
  float Rf[9];                               // R rounded to FP32 (set with pos_i, pos_fr each step)
  // float pairs (hi, lo) of the body frame at the current pose, for the wall
  // fraction's float-float arithmetic (set by the prologue each step):
  float Rs[2][9];                            //   R
  float Ts[2][3];                            //   R^T (X - floor X)
  float Es[19][6];                           //   R^T e_d: hi xyz, lo xyz per direction d
  float core_s;                              // core scale s = ((r_e - R_s) / r_e)^2 (constant)
  float Rb_f, re_f, skin_f;                  // FP32 copies of R_b, r_e, R_s (constant)
  int ball_off, n_balls;
  int ext[3];                                // node box extent per axis (constant)
  int lo[3];                                 // node box origin at the current pose
  int lo_hist[2][3];                         // box origin last flagged into owner buffer b
  int srad2[2];                              // largest squared distance from the position of that step of a
                                             //   solid node flagged into owner buffer b, as float bits (-1: none)
  float sctr[2][3];                          // the position (FP32) the solid nodes of buffer b were flagged at
};

// Per-step device counters and status (one instance per handle).
struct DevCounters {
  unsigned int gen;      // flag generation stamp (bumped once per flag phase)
  unsigned int n_bc;     // boundary nodes
  unsigned int n_links;  // boundary links
  unsigned int n_new;    // uncovered nodes
  unsigned int status;   // STATUS_* bits, sticky until read
  unsigned int n_contacts;
  unsigned int n_pairs;
  unsigned int n_cov;    // covered nodes (cover/uncover rule)
};
constexpr unsigned STATUS_BC_OVERFLOW = 1u, STATUS_LINK_OVERFLOW = 2u, STATUS_NEW_OVERFLOW = 4u,
                   STATUS_PAIR_OVERFLOW = 8u, STATUS_CONTACT_OVERFLOW = 16u, STATUS_MOVED_TOO_FAR = 32u,
                   STATUS_GUESS_TIMEOUT = 64u;  // a bounded wait of the tcgen05 MLP kernel gave up

struct ParticleLaunch {
  DevParticle* P;
  int np;
  const float4* balls;        // (c_x, c_y, c_z, k) FP32
  const double* balls_d;      // (c_x, c_y, c_z, k) FP64, 4 per ball
  const float4* balls_s;      // per ball two float4: FP32 (c, k) and the FP32 remainders of the FP64 values
  int max_balls_per_particle;
  uint32_t* owner_cur;        // buffer being written this step
  const uint32_t* owner_prev; // flags of the previous step
  int cur_buf, prev_buf;      // their indices (for the box histories)
  uint8_t* cls;
  uint32_t* stamp;
  DevCounters* ctr;
  long long* facc;            // np x 6 fixed-point (F_h, T_h)
  // lists
  uint32_t *bc_cell, *bc_mask, *bc_loff;
  uint32_t *link_bc, *link_p;
  uint8_t* link_dir;
  float* link_q;
  float* link_g;               // interpolated bounce-back population of each link (k_links_ibb)
  uint32_t* new_cell;
  uint32_t* cov_cell;         // covered nodes, listed only when cover_uncover (capacity cap_new)
  unsigned cap_bc, cap_links, cap_new;
  int cover_uncover;
  // box kernels: particle p owns blocks [off[p], off[p + 1]) of a 1D grid,
  // flag_off for the flag and clear kernels (flag_blocks in all), cls_off for
  // the row-per-warp classification (classify_blocks in all)
  const int* flag_off;
  const int* cls_off;
  int flag_blocks, classify_blocks;
  LatticeGeom g;
};
cudaError_t launch_prologue(const ParticleLaunch& L, cudaStream_t s);
cudaError_t launch_clear(const ParticleLaunch& L, cudaStream_t s);
cudaError_t launch_flag(const ParticleLaunch& L, cudaStream_t s);
cudaError_t launch_classify(const ParticleLaunch& L, cudaStream_t s);
cudaError_t launch_links_q(const ParticleLaunch& L, int grid, cudaStream_t s);

struct BoundaryLaunch {
  ParticleLaunch pl;
  void* A;  // f+(t); the refill writes into it at uncovered nodes
  void* B;  // f+(t+1)
  CollideParams p;
  int storage;
  bool forcing;
  int bb_mode;
  int grid;
  void* tmp;  // when set, k_boundary writes node k's 19 values to tmp[19 k ..] instead of B
  // per-block momentum-exchange sums of k_links_ibb (part_blocks x 6 np
  // int64), or null: the link kernel then adds into pl.facc directly
  long long* part;
  int part_blocks;
};
// Up to this many particles the link kernel sums the momentum exchange per
// block in shared memory and the boundary-node kernel adds the blocks' sums,
// so that warps do not contend for the same global addresses (thousands of
// 64-bit atomics on the same few addresses serialise).
constexpr int IBB_SHARED_PARTICLES = 1000;
constexpr int IBB_BLOCKS_PER_SM = 4;
cudaError_t launch_refill(const BoundaryLaunch& L, cudaStream_t s);
// Every link's bounce-back population into L.pl.link_g and its momentum exchange
// into the fixed-point sums (reads A only).
cudaError_t launch_links_ibb(const BoundaryLaunch& L, cudaStream_t s);
cudaError_t launch_boundary(const BoundaryLaunch& L, cudaStream_t s);
cudaError_t launch_near(const BoundaryLaunch& L, cudaStream_t s);
// Copy the boundary nodes' values from L.tmp into B (stored format, no arithmetic).
cudaError_t launch_scatter_boundary(const BoundaryLaunch& L, cudaStream_t s);

// ---------------------------------------------------------------------------
// DEM contacts (k_contact.cu)
// ---------------------------------------------------------------------------
struct ContactRec {       // one candidate (pair or particle-wall) of the last substep
  int i, j;               // j >= 0 particle, j = -1 - face for a wall
  double X[3];            // origin of particle i at the substep (copied, for the world contact point)
  float r[3];             // contact point - X_i
  float n[3];             // unit normal (towards particle i for pairs, into the domain for walls)
  float delta;            // overlap of the skins
  int iters, status;      // status: 0 ok, 1 not converged, 2 singular, 3 inside a core, 4 out of range
};
struct HistEntry {        // tangential spring of a pair / particle-wall contact
  double xi[3];
  long long stamp;        // DEM substep index of the last update (valid if previous substep)
  float xm_rel[3];        // last converged closest point of the pair, relative to particle i (warm start)
  int pad;
  long long xm_stamp;     // DEM substep of xm_rel
};
struct ContactParams {
  double kn, kt, eta_n, eta_t, mu_s, dt, margin;
  int periodic[3];
  int n[3];               // lattice sizes (walls at -1/2 and n - 1/2)
};
struct DashF {            // FP32 copy of the spring-dashpot parameters of ContactParams
  float kn, kt, eta_n, eta_t, mu_s, dt;
};
struct ContactLaunch {
  DevParticle* P;
  int np, ncap;           // particles, capacity used to index the pair-history triangle
  const float4* balls;
  DevCounters* ctr;
  unsigned* work;         // persistent-kernel work counter
  int* item_i;
  int* item_j;
  unsigned cap_items;
  ContactRec* recs;
  HistEntry* hist_pair;   // ncap (ncap - 1) / 2
  HistEntry* hist_wall;   // ncap x 6
  long long* fcacc;       // np x 6 fixed point (contact F, T)
  long long* substep;     // device substep counter
  ContactParams cp;
  int grid;
  float4* pf;             // np FP32 (position rounded to FP32, R_b) of the substep
  float4* plo;            // np FP32 remainders (position - pf.xyz) of the substep
  float4* qf;             // np FP32 unit quaternions (w, x, y, z) of the substep
  float4* vw;             // 2 np FP32 (velocity, 0), (angular velocity, 0) of the substep
  DashF cf;               // FP32 spring-dashpot parameters
  int learned;            // 1: pair items start from the learned guess (feat, pred), else the plain guess
  int warm;               // 1: pair items start from the previous substep's closest point when it exists
  float* feat;            // cap_items x 64 features of the pair items (learned)
  const float* pred;      // cap_items x 4 MLP outputs (learned)
};
cudaError_t launch_dem_prologue(const ContactLaunch& L, cudaStream_t s);
cudaError_t launch_broad_phase(const ContactLaunch& L, cudaStream_t s);
cudaError_t launch_contacts(const ContactLaunch& L, cudaStream_t s);
cudaError_t launch_item_features(const ContactLaunch& L, cudaStream_t s);

// Batch closest-point solve of explicitly posed particle pairs (shapes of the
// handle's particles, poses given per pair).
struct PairSolveLaunch {
  const DevParticle* P;
  int np;
  const float4* balls;
  int n;                  // pairs
  const int* ij;          // n x 2 particle indices (shapes)
  const double* poses;    // n x 14: pos_i, quat_i, pos_j, quat_j
  int flags;              // MI_PAIR_* bits
  const float* pred;      // n x 4 (learned start)
  float* X;               // n x 64 features (in: learned start without FEATURES; out: FEATURES)
  float* T;               // n x 4 labels (LABELS)
  double* xm;             // n x 3 closest point (world)
  int* iters;             // n Newton iterations
  int* evals;             // n ball evaluations
  int* status;            // n status (+ 16 when the learned start fell back to plain Newton)
};
cudaError_t launch_pair_solve(const PairSolveLaunch& S, cudaStream_t s);

// Fused MLP inference of the learned guess from a packed BF16 image
// (mlp_pack): Y (M x 4) for X (M x 64, 16-byte aligned), the row count read
// on the device from *Mdev when given (capped at M), as a step needs: its
// number of candidates is known only on the device.  mlp_infer_prepare sets
// the kernel's shared-memory limit; call it outside any stream capture.
size_t mlp_image_bytes();
cudaError_t mlp_pack(const float* params, void* image, cudaStream_t s);
cudaError_t mlp_infer_prepare();
cudaError_t mlp_infer(const void* image, const float* X, int M, const unsigned* Mdev, float* Y, cudaStream_t s);
// The same network on tcgen05/TMEM from its own packed image (mlp_tc_pack);
// on a wait timeout the kernel ORs err_bit into *err and writes NaN rows.
size_t mlp_tc_image_bytes();
size_t mlp_image_total();  // both images back to back (the C-ABI's packed image)
cudaError_t mlp_tc_pack(const float* params, void* image, cudaStream_t s);
cudaError_t mlp_tc_prepare();
cudaError_t mlp_tc_infer(const void* image, const float* X, int M, const unsigned* Mdev, float* Y, unsigned* err,
                         unsigned err_bit, cudaStream_t s, unsigned wait_limit = 0, int stall = 0);

struct IntegrateLaunch {
  DevParticle* P;
  int np;
  const long long* facc;   // hydrodynamic F, T (fixed point)
  const long long* fc;     // contact F, T (np x 6, fixed point) or nullptr
  double gravity[3];
  double rho0;
  double dt;
};
cudaError_t launch_integrate(const IntegrateLaunch& L, cudaStream_t s);
// Fused DEM loop of one LBM step for at most FUSED_DEM_MAX_PARTICLES particles
// (one CTA): the first substep's rigid-body update, then n_sub - 1 substeps of
// prologue, candidates, solves and update.  The plain or warm start only.
constexpr int FUSED_DEM_MAX_PARTICLES = 64;
cudaError_t launch_dem_substeps(const ContactLaunch& L, const IntegrateLaunch& I, int n_sub, cudaStream_t s);

// Half-width of the band around f = 1 inside which an FP32 field value does
// not decide solid or fluid and the node or sample is re-evaluated in FP64.
constexpr float FIELD_GUARD = 1e-4f;

// One sample (X, Y, Z) of the midpoint quadrature of the indicator f >= 1
// (Sec. 2.1 Eq. 1; reading A15), in the body frame: the FP32 field summed ball
// by ball with an early exit once it passes 1 + FIELD_GUARD (the terms are
// positive), and inside the band an unfused FP64 re-evaluation in ball order,
// so that the decision is the FP64 one.  balls: FP32 (c, k); balls_d: the
// same table as 4 doubles per ball.
__device__ __forceinline__ bool mass_sample_inside(const float4* balls, const double* balls_d, int nb, double X,
                                                   double Y, double Z) {
  const float xf = (float)X, yf = (float)Y, zf = (float)Z;
  float f = 0.f;
  for (int b = 0; b < nb; ++b) {
    const float4 c = balls[b];
    const float e0 = xf - c.x, e1 = yf - c.y, e2 = zf - c.z;
    f += __fdividef(c.w, e0 * e0 + e1 * e1 + e2 * e2);
    if (f > 1.0f + FIELD_GUARD) return true;
  }
  if (f < 1.0f - FIELD_GUARD) return false;
  double fd = 0.0;
  for (int b = 0; b < nb; ++b) {
    const double* c = balls_d + 4 * b;
    const double e0 = __dsub_rn(X, c[0]), e1 = __dsub_rn(Y, c[1]), e2 = __dsub_rn(Z, c[2]);
    const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(e0, e0), __dmul_rn(e1, e1)), __dmul_rn(e2, e2));
    fd = __dadd_rn(fd, __ddiv_rn(c[3], r2));
  }
  return fd >= 1.0;
}

// Moment sums of an inside sample: [count, x, y, z, xx, xy, xz, yy, yz, zz].
__device__ __forceinline__ void mass_sample_accumulate(double acc[10], double X, double Y, double Z) {
  acc[0] += 1.0;
  acc[1] += X;
  acc[2] += Y;
  acc[3] += Z;
  acc[4] += X * X;
  acc[5] += X * Y;
  acc[6] += X * Z;
  acc[7] += Y * Y;
  acc[8] += Y * Z;
  acc[9] += Z * Z;
}

// Mass properties by midpoint quadrature of f >= 1 on a grid of spacing h over
// [-Rb, Rb]^3 (body frame); out: [count, sx, sy, sz, sxx, sxy, sxz, syy, syz, szz]
// per block, summed on the host in block order.
cudaError_t launch_mass_quadrature(const float4* balls, const double* balls_d, int n_balls, double Rb,
                                   double h, int n_side, double* partials, int blocks, cudaStream_t s);


// D3Q19 direction of the integer offset, or -1.
__host__ __device__ inline int dir_of(int x, int y, int z) {
  for (int i = 0; i < 19; ++i)
    if (cx(i) == x && cy(i) == y && cz(i) == z) return i;
  return -1;
}

}  // namespace mi
