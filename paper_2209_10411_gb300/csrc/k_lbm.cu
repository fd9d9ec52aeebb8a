// Lattice kernels: bulk pull stream-collide (D3Q19 BGK) and population
// packing.  The stream-collide follows the LBM basis of the paper's
// Sec. 2.3.2 (distributions G_i, weights omega_i, C = 1) with the D3Q19 BGK
// lattice; domain walls are halfway bounce-back with the moving-wall term
// 6 w_i rho0 (e_i . u_wall), the same form the paper gives for moving
// particle walls.
//
// Memory: populations are SoA, one plane of ncell elements per direction,
// x fastest.  One thread updates one node: 19 pulled loads (neighbour x - e_i,
// misaligned by one element for the 10 directions with e_x != 0; the L1/L2
// absorb the sector overlap so DRAM sees each element once), FP32 collision,
// 19 streaming stores.  Algorithmic traffic: 19 * 2 * sizeof(storage) bytes
// per node update (+1 byte of node class when particles are present).
#include <climits>
#include "mi_internal.cuh"

namespace mi {

// BGK collision on deviations h_i = f_i - w_i and store of the result.
//   rho = 1 + sum h_i, j = sum e_i h_i (sum w_i = 1, sum w_i e_i = 0)
//   f_eq,i - w_i = w_i (rho - 1) + w_i rho (3 e.u + 4.5 (e.u)^2 - 1.5 u.u)
//   h+_i = h_i + omega (f_eq,i - w_i - h_i)   [+ Guo source]
template <bool FORCE>
__device__ __forceinline__ void collide_inplace(float (&h)[19], const CollideParams& P) {
  float drho = 0.f;
#pragma unroll
  for (int i = 0; i < 19; ++i) drho += h[i];
  const float jx = (h[1] - h[2]) + (h[7] - h[8]) + (h[9] - h[10]) + (h[11] - h[12]) + (h[13] - h[14]);
  const float jy = (h[3] - h[4]) + (h[7] - h[8]) + (h[10] - h[9]) + (h[15] - h[16]) + (h[17] - h[18]);
  const float jz = (h[5] - h[6]) + (h[11] - h[12]) + (h[14] - h[13]) + (h[15] - h[16]) + (h[18] - h[17]);
  const float rho = 1.0f + drho;
  const float irho = 1.0f / rho;
  float ux, uy, uz;
  if (FORCE) {
    ux = (jx + 0.5f * P.force[0]) * irho;
    uy = (jy + 0.5f * P.force[1]) * irho;
    uz = (jz + 0.5f * P.force[2]) * irho;
  } else {
    ux = jx * irho;
    uy = jy * irho;
    uz = jz * irho;
  }
  const float usq15 = 1.5f * (ux * ux + uy * uy + uz * uz);
  const float om = P.omega;
#pragma unroll
  for (int i = 0; i < 19; ++i) {
    const float eu = cx(i) * ux + cy(i) * uy + cz(i) * uz;
    const float feq_dev = wq(i) * (drho + rho * (3.0f * eu + 4.5f * eu * eu - usq15));
    float hp = h[i] + om * (feq_dev - h[i]);
    if (FORCE) {
      const float eF = cx(i) * P.force[0] + cy(i) * P.force[1] + cz(i) * P.force[2];
      const float uF = ux * P.force[0] + uy * P.force[1] + uz * P.force[2];
      hp += (1.0f - 0.5f * om) * wq(i) * (3.0f * (eF - uF) + 9.0f * eu * eF);
    }
    h[i] = hp;
  }
}

template <int ST, bool FORCE>
__device__ __forceinline__ void collide_store(float (&h)[19], typename Store<ST>::T* __restrict__ B,
                                              long long plane, long long c, const CollideParams& P) {
  collide_inplace<FORCE>(h, P);
#pragma unroll
  for (int i = 0; i < 19; ++i) Store<ST>::put(B + i * plane + c, i, h[i]);
}

// Pull streaming (with halfway bounce-back at domain walls) of node (x, y, z),
// c its linear index: the 19 incoming deviations h_i = f_i - w_i.
template <int ST>
__device__ __forceinline__ void pull_node(const typename Store<ST>::T* __restrict__ A, const LatticeGeom& g,
                                          const CollideParams& P, int x, int y, int z, long long c, float (&h)[19]) {
  const long long nxy = (long long)g.nx * g.ny;
  const bool interior = (x > 0) & (x < g.nx - 1) & (y > 0) & (y < g.ny - 1) & (z > 0) & (z < g.nz - 1);
  if (interior) {
#pragma unroll
    for (int i = 0; i < 19; ++i) {
      const long long off = cx(i) + (long long)g.nx * cy(i) + nxy * cz(i);
      h[i] = Store<ST>::dev(A + i * g.plane + (c - off), i);
    }
  } else {
#pragma unroll
    for (int i = 0; i < 19; ++i) {
      int sx = x - cx(i), sy = y - cy(i), sz = z - cz(i);
      int face = -1;  // a corner crossing is attributed to x, then y, then z
      if (sz < 0) { if (g.periodic[2]) sz += g.nz; else face = 4; }
      else if (sz >= g.nz) { if (g.periodic[2]) sz -= g.nz; else face = 5; }
      if (sy < 0) { if (g.periodic[1]) sy += g.ny; else face = 2; }
      else if (sy >= g.ny) { if (g.periodic[1]) sy -= g.ny; else face = 3; }
      if (sx < 0) { if (g.periodic[0]) sx += g.nx; else face = 0; }
      else if (sx >= g.nx) { if (g.periodic[0]) sx -= g.nx; else face = 1; }
      if (face < 0) {
        h[i] = Store<ST>::dev(A + i * g.plane + (sx + (long long)g.nx * sy + nxy * sz), i);
      } else {
        // halfway bounce-back: f_in,i(x) = f+_opp(i)(x) + 6 w_i rho0 e_i.u_wall (w_opp = w_i)
        h[i] = Store<ST>::dev(A + opp(i) * g.plane + c, opp(i)) + P.bb_wall[face][i];
      }
    }
  }
}

// Pull and collide one node.
template <int ST, bool FORCE>
__device__ __forceinline__ void update_node(const typename Store<ST>::T* __restrict__ A,
                                            typename Store<ST>::T* __restrict__ B, const LatticeGeom& g,
                                            const CollideParams& P, int x, int y, int z, long long c) {
  float h[19];
  pull_node<ST>(A, g, P, x, y, z, c, h);
  collide_store<ST, FORCE>(h, B, g.plane, c, P);
}

// Every node of the lattice, ROWS consecutive rows (y) per thread: all pulls
// of a thread are issued before its collisions, so that 16-bit storages keep
// as many bytes in flight as FP32.  With particles this runs concurrently with
// the particle phases: boundary nodes are rewritten afterwards by k_boundary,
// solid nodes hold unspecified values, and the nodes next to a node uncovered
// this step (whose refilled populations this kernel may not have seen) are
// recomputed by k_near.  Nodes anywhere else have no solid or uncovered
// neighbour, so their update here is final.
template <int ST, bool FORCE, int ROWS>
__global__ void __launch_bounds__(256) k_bulk(const typename Store<ST>::T* __restrict__ A,
                                              typename Store<ST>::T* __restrict__ B, LatticeGeom g,
                                              CollideParams P) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y0 = blockIdx.y * ROWS, z = blockIdx.z;
  if (x >= g.nx) return;
  float h[ROWS][19];
#pragma unroll
  for (int r = 0; r < ROWS; ++r)
    if (y0 + r < g.ny) pull_node<ST>(A, g, P, x, y0 + r, z, x + (long long)g.nx * (y0 + r + (long long)g.ny * z), h[r]);
#pragma unroll
  for (int r = 0; r < ROWS; ++r)
    if (y0 + r < g.ny) collide_store<ST, FORCE>(h[r], B, g.plane, x + (long long)g.nx * (y0 + r + (long long)g.ny * z), P);
}

template <int ST, bool FORCE, int ROWS>
static cudaError_t launch_bulk_t(const BulkLaunch& L, cudaStream_t s) {
  using T = typename Store<ST>::T;
  const int bx = L.block_x;
  dim3 grid((L.g.nx + bx - 1) / bx, (L.g.ny + ROWS - 1) / ROWS, L.g.nz);
  k_bulk<ST, FORCE, ROWS><<<grid, bx, 0, s>>>(static_cast<const T*>(L.A), static_cast<T*>(L.B), L.g, L.p);
  return cudaGetLastError();
}

// Every node, two x-adjacent nodes (x0, x0 + 1), x0 even, per thread: the
// pulls of the 9 directions with e_x = 0 are one paired load each; for
// e_x = +1 (-1) the pair is completed by the high (low) element of the
// previous (next) lane's paired load, fetched by a shuffle (a scalar load at
// the warp's edge).  Both collisions store paired.  Nodes on the lattice's
// boundary rows and edge columns are pulled again by the general path.  The
// same concurrency contract as k_bulk.  Requires nx even.
template <int ST, bool FORCE>
__global__ void __launch_bounds__(128) k_bulk_pairs(const typename Store<ST>::T* __restrict__ A,
                                                    typename Store<ST>::T* __restrict__ B, LatticeGeom g,
                                                    CollideParams P) {
  using T = typename Store<ST>::T;
  using PR = Pair<ST>;
  const int lane = threadIdx.x & 31;
  const int x0 = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
  const int y = blockIdx.y, z = blockIdx.z;
  const bool active = x0 < g.nx;
  const int xc = active ? x0 : g.nx - 2;  // idle lanes still take part in the shuffles
  float h0[19], h1[19];
#pragma unroll
  for (int i = 0; i < 19; ++i) {
    const int ys = min(max(y - cy(i), 0), g.ny - 1), zs = min(max(z - cz(i), 0), g.nz - 1);
    const T* row = A + i * g.plane + ((long long)zs * g.ny + ys) * g.nx;
    const typename PR::P v = PR::load(row + xc);
    if (cx(i) == 0) {
      h0[i] = PR::lo(v, i);
      h1[i] = PR::hi(v, i);
    } else if (cx(i) == 1) {  // node x0 pulls from x0 - 1
      const typename PR::P u = PR::shfl_up(v);
      float prev = PR::hi(u, i);
      if (lane == 0) prev = xc > 0 ? Store<ST>::dev(row + xc - 1, i) : 0.f;
      h0[i] = prev;
      h1[i] = PR::lo(v, i);
    } else {  // node x0 + 1 pulls from x0 + 2
      const typename PR::P u = PR::shfl_down(v);
      float next = PR::lo(u, i);
      if (lane == 31) next = xc + 2 < g.nx ? Store<ST>::dev(row + xc + 2, i) : 0.f;
      h0[i] = PR::hi(v, i);
      h1[i] = next;
    }
  }
  if (!active) return;
  const long long c0 = x0 + (long long)g.nx * (y + (long long)g.ny * z);
  const bool rows_interior = (y > 0) & (y < g.ny - 1) & (z > 0) & (z < g.nz - 1);
  if (!rows_interior || x0 == 0) pull_node<ST>(A, g, P, x0, y, z, c0, h0);
  if (!rows_interior || x0 + 1 == g.nx - 1) pull_node<ST>(A, g, P, x0 + 1, y, z, c0 + 1, h1);
  collide_inplace<FORCE>(h0, P);
  collide_inplace<FORCE>(h1, P);
#pragma unroll
  for (int i = 0; i < 19; ++i) PR::put(B + i * g.plane + c0, i, h0[i], h1[i]);
}

// 16-bit storages: the same paired scheme with both nodes' incoming and
// outgoing values kept packed, one 32-bit register per direction for the two
// nodes, so that a thread needs about as many registers as the scalar kernel
// and a warp keeps twice the bytes in flight.
template <int ST, bool FORCE, int MINB>
__global__ void __launch_bounds__(128, MINB) k_bulk_pairs16(const typename Store<ST>::T* __restrict__ A,
                                                         typename Store<ST>::T* __restrict__ B, LatticeGeom g,
                                                         CollideParams P) {
  using T = typename Store<ST>::T;
  const int lane = threadIdx.x & 31;
  const int x0 = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
  const int y = blockIdx.y, z = blockIdx.z;
  const bool active = x0 < g.nx;
  const int xc = active ? x0 : g.nx - 2;
  unsigned in[19];  // low half: node x0, high half: node x0 + 1
#pragma unroll
  for (int i = 0; i < 19; ++i) {
    const int ys = min(max(y - cy(i), 0), g.ny - 1), zs = min(max(z - cz(i), 0), g.nz - 1);
    const unsigned short* row =
        reinterpret_cast<const unsigned short*>(A + i * g.plane + ((long long)zs * g.ny + ys) * g.nx);
    const unsigned v = __ldg(reinterpret_cast<const unsigned*>(row + xc));
    if (cx(i) == 0) {
      in[i] = v;
    } else if (cx(i) == 1) {
      const unsigned u = __shfl_up_sync(0xffffffffu, v, 1);
      unsigned prev = u >> 16;
      if (lane == 0) prev = xc > 0 ? (unsigned)__ldg(row + xc - 1) : 0u;
      in[i] = prev | (v << 16);
    } else {
      const unsigned u = __shfl_down_sync(0xffffffffu, v, 1);
      unsigned next = u & 0xFFFFu;
      if (lane == 31) next = xc + 2 < g.nx ? (unsigned)__ldg(row + xc + 2) : 0u;
      in[i] = (v >> 16) | (next << 16);
    }
  }
  if (!active) return;
  const long long c0 = x0 + (long long)g.nx * (y + (long long)g.ny * z);
  const bool rows_interior = (y > 0) & (y < g.ny - 1) & (z > 0) & (z < g.nz - 1);
  unsigned out[19];
  {
    float h[19];
    if (!rows_interior || x0 == 0) {
      pull_node<ST>(A, g, P, x0, y, z, c0, h);
    } else {
#pragma unroll
      for (int i = 0; i < 19; ++i) h[i] = dev16<ST>((unsigned short)(in[i] & 0xFFFFu));
    }
    collide_inplace<FORCE>(h, P);
#pragma unroll
    for (int i = 0; i < 19; ++i) out[i] = pack16<ST>(h[i]);
  }
  {
    float h[19];
    if (!rows_interior || x0 + 1 == g.nx - 1) {
      pull_node<ST>(A, g, P, x0 + 1, y, z, c0 + 1, h);
    } else {
#pragma unroll
      for (int i = 0; i < 19; ++i) h[i] = dev16<ST>((unsigned short)(in[i] >> 16));
    }
    collide_inplace<FORCE>(h, P);
#pragma unroll
    for (int i = 0; i < 19; ++i) out[i] |= (unsigned)pack16<ST>(h[i]) << 16;
  }
#pragma unroll
  for (int i = 0; i < 19; ++i) __stcs(reinterpret_cast<unsigned*>(B + i * g.plane + c0), out[i]);
}

// 16-bit storages: four x-adjacent nodes (x0 .. x0 + 3, x0 a multiple of 4)
// per thread.  Each pull is one aligned 64-bit load per direction when e_x = 0;
// for e_x = +1 (-1) the four shifted elements x0 - 1 .. x0 + 2 (x0 + 1 ..
// x0 + 4) are the quad's own aligned 64-bit word plus the aligned 32-bit
// word beside it, joined by two byte permutes.  The 16-bit values stay packed
// in registers until each node's collision, and every direction is stored as
// one 64-bit streaming store: a 16-bit storage moves half the bytes of FP32
// per instruction, and the wider accesses keep the instruction count per
// byte near that of the FP32 kernel.  The quads at the x faces stay on this
// path (no warp mixes paths): the word beside them comes from the other end
// of the row when x is periodic, else the face node's pulled value is
// replaced after unpacking by its halfway bounce-back.  Rows on the y and z
// faces (whole warps) take the general per-node path.  The same concurrency
// contract as k_bulk.  Requires nx % 4 == 0.
template <int ST> __device__ __forceinline__ float2 unpack2(unsigned w);
template <> __device__ __forceinline__ float2 unpack2<MI_STORE_F16_DEV>(unsigned w) {
  return __half22float2(*reinterpret_cast<const __half2*>(&w));
}
template <> __device__ __forceinline__ float2 unpack2<MI_STORE_BF16_DEV>(unsigned w) {
  return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xFFFF0000u));
}
template <int ST> __device__ __forceinline__ unsigned pack2(float a, float b);
template <> __device__ __forceinline__ unsigned pack2<MI_STORE_F16_DEV>(float a, float b) {
  const __half2 v = __floats2half2_rn(a, b);
  return *reinterpret_cast<const unsigned*>(&v);
}
template <> __device__ __forceinline__ unsigned pack2<MI_STORE_BF16_DEV>(float a, float b) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const unsigned*>(&v);
}

template <int ST, bool FORCE>
__global__ void __launch_bounds__(128, FORCE ? 3 : 5) k_bulk_quad16(const typename Store<ST>::T* __restrict__ A,
                                                     typename Store<ST>::T* __restrict__ B, LatticeGeom g,
                                                     CollideParams P) {
  const int x0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
  const int y = blockIdx.y, z = blockIdx.z;
  if (x0 >= g.nx) return;
  const long long c0 = x0 + (long long)g.nx * (y + (long long)g.ny * z);
  if (!((y > 0) & (y < g.ny - 1) & (z > 0) & (z < g.nz - 1))) {
#pragma unroll 1
    for (int k = 0; k < 4; ++k) update_node<ST, FORCE>(A, B, g, P, x0 + k, y, z, c0 + k);
    return;
  }
  const bool lo_edge = x0 == 0, hi_edge = x0 == g.nx - 4, xper = g.periodic[0] != 0;
  const unsigned short* Au = reinterpret_cast<const unsigned short*>(A);
  const long long nxy = (long long)g.nx * g.ny;
  uint2 in[19];
#pragma unroll
  for (int i = 0; i < 19; ++i) {
    // aligned position of node x0 in the source row of direction i
    const unsigned short* row = Au + i * g.plane + (c0 - ((long long)g.nx * cy(i) + nxy * cz(i)));
    const uint2 w = __ldg(reinterpret_cast<const uint2*>(row));
    if (cx(i) == 0) {
      in[i] = w;
    } else if (cx(i) == 1) {  // elements x0 - 1 .. x0 + 2
      unsigned before;        // its high half: element x0 - 1
      if (!lo_edge) before = __ldg(reinterpret_cast<const unsigned*>(row - 2));
      else before = xper ? (unsigned)__ldg(row + g.nx - 1) << 16 : 0u;  // wall: replaced below
      in[i] = make_uint2(__byte_perm(before, w.x, 0x5432), __byte_perm(w.x, w.y, 0x5432));
    } else {                  // elements x0 + 1 .. x0 + 4
      unsigned after;         // its low half: element x0 + 4
      if (!hi_edge) after = __ldg(reinterpret_cast<const unsigned*>(row + 4));
      else after = xper ? (unsigned)__ldg(row - x0) : 0u;  // wall: replaced below
      in[i] = make_uint2(__byte_perm(w.x, w.y, 0x5432), __byte_perm(w.y, after, 0x5432));
    }
  }
  uint2 out[19];
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    float h0[19], h1[19];
#pragma unroll
    for (int i = 0; i < 19; ++i) {
      const float2 v = unpack2<ST>(half ? in[i].y : in[i].x);
      h0[i] = v.x;
      h1[i] = v.y;
    }
    if (!xper) {
      // halfway bounce-back at the x faces: f_in,i(x) = f+_opp(i)(x) + 6 w_i rho0 e_i.u_wall
      if (half == 0 && lo_edge) {
#pragma unroll
        for (int i = 0; i < 19; ++i)
          if (cx(i) == 1) h0[i] = dev16<ST>(__ldg(Au + opp(i) * g.plane + c0)) + P.bb_wall[0][i];
      }
      if (half == 1 && hi_edge) {
#pragma unroll
        for (int i = 0; i < 19; ++i)
          if (cx(i) == -1) h1[i] = dev16<ST>(__ldg(Au + opp(i) * g.plane + c0 + 3)) + P.bb_wall[1][i];
      }
    }
    collide_inplace<FORCE>(h0, P);
    collide_inplace<FORCE>(h1, P);
#pragma unroll
    for (int i = 0; i < 19; ++i) {
      const unsigned wv = pack2<ST>(h0[i], h1[i]);
      if (half) out[i].y = wv; else out[i].x = wv;
    }
  }
  unsigned short* Bu = reinterpret_cast<unsigned short*>(B);
#pragma unroll
  for (int i = 0; i < 19; ++i) __stcs(reinterpret_cast<uint2*>(Bu + i * g.plane + c0), out[i]);
}

template <int ST, bool FORCE>
static cudaError_t launch_bulk_pairs_t(const BulkLaunch& L, cudaStream_t s) {
  using T = typename Store<ST>::T;
  const int bx = L.block_x;
  const int npair = L.g.nx / 2;
  dim3 grid((npair + bx - 1) / bx, L.g.ny, L.g.nz);
  if (ST == MI_STORE_F32)
    k_bulk_pairs<ST, FORCE><<<grid, bx, 0, s>>>(static_cast<const T*>(L.A), static_cast<T*>(L.B), L.g, L.p);
  else {
    constexpr int S16 = ST == MI_STORE_F32 ? MI_STORE_F16_DEV : ST;
    using T16 = typename Store<S16>::T;
    if (L.pair_mode == 2)
      k_bulk_pairs16<S16, FORCE, 6><<<grid, bx, 0, s>>>(reinterpret_cast<const T16*>(L.A), reinterpret_cast<T16*>(L.B),
                                                        L.g, L.p);
    else
      k_bulk_pairs16<S16, FORCE, 8><<<grid, bx, 0, s>>>(reinterpret_cast<const T16*>(L.A), reinterpret_cast<T16*>(L.B),
                                                        L.g, L.p);
  }
  return cudaGetLastError();
}

template <int ST, bool FORCE>
static cudaError_t launch_bulk_quad_t(const BulkLaunch& L, cudaStream_t s) {
  constexpr int S16 = ST == MI_STORE_F32 ? MI_STORE_F16_DEV : ST;
  using T16 = typename Store<S16>::T;
  const int bx = L.block_x;
  const int nq = L.g.nx / 4;
  dim3 grid((nq + bx - 1) / bx, L.g.ny, L.g.nz);
  k_bulk_quad16<S16, FORCE><<<grid, bx, 0, s>>>(reinterpret_cast<const T16*>(L.A), reinterpret_cast<T16*>(L.B), L.g,
                                                L.p);
  return cudaGetLastError();
}

template <int ST>
static cudaError_t launch_bulk_st(const BulkLaunch& L, cudaStream_t s) {
  if (ST != MI_STORE_F32 && L.pair_mode == 3 && L.g.nx % 4 == 0 && L.g.nx >= 4)
    return L.forcing ? launch_bulk_quad_t<ST, true>(L, s) : launch_bulk_quad_t<ST, false>(L, s);
  if (L.pairs && L.pair_mode != 3 && L.g.nx % 2 == 0 && L.g.nx >= 2)
    return L.forcing ? launch_bulk_pairs_t<ST, true>(L, s) : launch_bulk_pairs_t<ST, false>(L, s);
  if (L.rows == 2) return L.forcing ? launch_bulk_t<ST, true, 2>(L, s) : launch_bulk_t<ST, false, 2>(L, s);
  return L.forcing ? launch_bulk_t<ST, true, 1>(L, s) : launch_bulk_t<ST, false, 1>(L, s);
}

cudaError_t launch_bulk(const BulkLaunch& L, cudaStream_t s) {
  if (L.block_x <= 0 || L.block_x > 256 || (L.block_x % 32) != 0) return cudaErrorInvalidValue;
  if (L.pairs && L.block_x > 128) return cudaErrorInvalidValue;
  switch (L.storage) {
    case MI_STORE_F32: return launch_bulk_st<MI_STORE_F32>(L, s);
    case MI_STORE_F16_DEV: return launch_bulk_st<MI_STORE_F16_DEV>(L, s);
    case MI_STORE_BF16_DEV: return launch_bulk_st<MI_STORE_BF16_DEV>(L, s);
  }
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// Refill of uncovered nodes (the paper's local bounce-back refill, Sec. 2.3.2),
// applied to the stored post-collision populations f+(t) before streaming:
//   f+_i(x_new) = f+_opp(i)(x_new + e_i) + 6 w_i rho0 (e_i . u_new)
// when x_new + e_i is a fluid node that was also fluid at the previous step,
// else f_eq,i(rho0, u_new); u_new is the rigid velocity at x_new of the
// particle that covered it.  One thread per uncovered node.  With the
// cover/uncover rule the same launch also moves node momenta: an uncovered
// node's refilled momentum is taken from its particle, a covered node's
// post-collision momentum is given to the particle that covers it.
// ---------------------------------------------------------------------------
namespace {
__device__ __forceinline__ bool nbr_wrap(int x, int y, int z, int dx, int dy, int dz, const LatticeGeom& g,
                                         long long& out) {
  int a = x + dx, b = y + dy, c = z + dz;
  if (a < 0 || a >= g.nx) {
    if (!g.periodic[0]) return false;
    a = (a + g.nx) % g.nx;
  }
  if (b < 0 || b >= g.ny) {
    if (!g.periodic[1]) return false;
    b = (b + g.ny) % g.ny;
  }
  if (c < 0 || c >= g.nz) {
    if (!g.periodic[2]) return false;
    c = (c + g.nz) % g.nz;
  }
  out = a + (long long)g.nx * (b + (long long)g.ny * c);
  return true;
}

__device__ __forceinline__ void rigid_u(const DevParticle& P, double px, double py, double pz, float u[3]) {
  const float r0 = (float)(px - P.pos[0]), r1 = (float)(py - P.pos[1]), r2 = (float)(pz - P.pos[2]);
  u[0] = P.velf[0] + (P.omegaf[1] * r2 - P.omegaf[2] * r1);
  u[1] = P.velf[1] + (P.omegaf[2] * r0 - P.omegaf[0] * r2);
  u[2] = P.velf[2] + (P.omegaf[0] * r1 - P.omegaf[1] * r0);
}

// Node coordinates of a list entry (particle lists store node indices as
// uint32, so 32-bit divisions suffice).
__device__ __forceinline__ void coords(long long c, const LatticeGeom& g, int& x, int& y, int& z) {
  const unsigned cu = (unsigned)c, row = cu / (unsigned)g.nx;
  x = (int)(cu - row * (unsigned)g.nx);
  z = (int)(row / (unsigned)g.ny);
  y = (int)(row - (unsigned)z * (unsigned)g.ny);
}

template <int ST>
__device__ __forceinline__ void moments_at(const typename Store<ST>::T* __restrict__ A, long long plane,
                                           long long c, float& rho, float u[3]) {
  float h[19];
#pragma unroll
  for (int i = 0; i < 19; ++i) h[i] = Store<ST>::dev(A + i * plane + c, i);
  float dr = 0.f;
#pragma unroll
  for (int i = 0; i < 19; ++i) dr += h[i];
  rho = 1.0f + dr;
  const float jx = (h[1] - h[2]) + (h[7] - h[8]) + (h[9] - h[10]) + (h[11] - h[12]) + (h[13] - h[14]);
  const float jy = (h[3] - h[4]) + (h[7] - h[8]) + (h[10] - h[9]) + (h[15] - h[16]) + (h[17] - h[18]);
  const float jz = (h[5] - h[6]) + (h[11] - h[12]) + (h[14] - h[13]) + (h[15] - h[16]) + (h[18] - h[17]);
  u[0] = jx / rho;
  u[1] = jy / rho;
  u[2] = jz / rho;
}
}  // namespace

namespace {
// Cover/uncover rule: a node's population momentum J (FP32) and its torque
// about the particle's position, sign * (J, (x - X_p) x J), added to the
// particle's fixed-point hydrodynamic sums.
__device__ __forceinline__ void add_node_momentum(long long* facc, const DevParticle* Ps, uint32_t p, int x, int y,
                                                  int z, const float J[3], float sign) {
  const DevParticle& P = Ps[p];
  const float r0 = (float)(x - P.pos[0]), r1 = (float)(y - P.pos[1]), r2 = (float)(z - P.pos[2]);
  const float v[6] = {J[0], J[1], J[2], r1 * J[2] - r2 * J[1], r2 * J[0] - r0 * J[2], r0 * J[1] - r1 * J[0]};
  for (int k = 0; k < 6; ++k) {
    const long long iv = __float2ll_rn(sign * v[k] * 1099511627776.0f);
    atomicAdd(reinterpret_cast<unsigned long long*>(facc + 6 * (size_t)p + k), (unsigned long long)iv);
  }
}
}  // namespace

template <int ST>
__global__ void __launch_bounds__(128) k_refill(BoundaryLaunch L) {
  using T = typename Store<ST>::T;
  T* A = static_cast<T*>(L.A);
  const LatticeGeom& g = L.pl.g;
  const unsigned nn = min(L.pl.ctr->n_new, L.pl.cap_new);
  const float rho0 = L.p.rho0;
  for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < nn; k += gridDim.x * blockDim.x) {
    const long long c = L.pl.new_cell[k];
    int x, y, z;
    coords(c, g, x, y, z);
    const uint32_t pid = L.pl.owner_prev[c];
    const DevParticle& P = L.pl.P[pid];
    float u[3];
    rigid_u(P, x, y, z, u);
    const float usq15 = 1.5f * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    float J[3] = {0.f, 0.f, 0.f};  // momentum of the refilled populations (sum e_i (f_i - w_i))
#pragma unroll
    for (int i = 0; i < 19; ++i) {
      const float eu = cx(i) * u[0] + cy(i) * u[1] + cz(i) * u[2];
      long long nb;
      float h;
      if (i != 0 && nbr_wrap(x, y, z, cx(i), cy(i), cz(i), g, nb) && L.pl.owner_cur[nb] == OWNER_NONE &&
          L.pl.owner_prev[nb] == OWNER_NONE) {
        h = Store<ST>::dev(A + opp(i) * g.plane + nb, opp(i)) + 6.0f * wq(i) * rho0 * eu;
      } else {
        h = wq(i) * (rho0 - 1.0f) + wq(i) * rho0 * (3.0f * eu + 4.5f * eu * eu - usq15);
      }
      Store<ST>::put(A + i * g.plane + c, i, h);
      J[0] += cx(i) * h;
      J[1] += cy(i) * h;
      J[2] += cz(i) * h;
    }
    // cover/uncover rule: the particle that uncovered the node gives up this momentum
    if (L.pl.cover_uncover) add_node_momentum(L.pl.facc, L.pl.P, pid, x, y, z, J, -1.0f);
  }
  if (!L.pl.cover_uncover) return;
  // covered nodes: the momentum of their post-collision populations f+(t)
  // (still in A: they were fluid) goes to the particle that covered them
  const unsigned nc = min(L.pl.ctr->n_cov, L.pl.cap_new);
  for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < nc; k += gridDim.x * blockDim.x) {
    const long long c = L.pl.cov_cell[k];
    int x, y, z;
    coords(c, g, x, y, z);
    float J[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 1; i < 19; ++i) {
      const float h = Store<ST>::dev(A + i * g.plane + c, i);
      J[0] += cx(i) * h;
      J[1] += cy(i) * h;
      J[2] += cz(i) * h;
    }
    add_node_momentum(L.pl.facc, L.pl.P, L.pl.owner_cur[c], x, y, z, J, 1.0f);
  }
}

// ---------------------------------------------------------------------------
// Nodes next to an uncovered node: recomputed after the refill (the bulk
// kernel may have read their neighbour's populations before it was refilled).
// One thread per (uncovered node, direction); a node reached twice is written
// twice with the same values.
// ---------------------------------------------------------------------------
template <int ST, bool FORCE>
__global__ void __launch_bounds__(128) k_near(BoundaryLaunch L) {
  using T = typename Store<ST>::T;
  const T* __restrict__ A = static_cast<const T*>(L.A);
  T* __restrict__ B = static_cast<T*>(L.B);
  const LatticeGeom& g = L.pl.g;
  const unsigned nn = min(L.pl.ctr->n_new, L.pl.cap_new);
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < nn * 18u; t += gridDim.x * blockDim.x) {
    const unsigned k = t / 18u;
    const int d = 1 + (int)(t - 18u * k);
    int x, y, z;
    coords(L.pl.new_cell[k], g, x, y, z);
    long long nb;
    if (!nbr_wrap(x, y, z, cx(d), cy(d), cz(d), g, nb)) continue;
    if (L.pl.owner_cur[nb] != OWNER_NONE || (L.pl.cls[nb] & CLS_BOUNDARY)) continue;
    int a, b, c;
    coords(nb, g, a, b, c);
    update_node<ST, FORCE>(A, B, g, L.p, a, b, c, nb);
  }
}

// ---------------------------------------------------------------------------
// Boundary nodes (Sec. 2.3.2) in two kernels.
//
// k_links_ibb, one thread per link (x_f, d): x_f a fluid boundary node,
// x_f + e_d a solid node of particle p at wall fraction q.  The population
// that would have streamed from the solid neighbour into x_f along
// j = opp(d) is the paper's interpolated bounce-back (Eqs. eqneq1, eqneq2,
// neqd):
//   G_j = f_eq,d(rho_f, u_d) + [f+_d(x_f) - f_eq,d(rho_f, u_f)] + 6 w_d rho0 (e_j . u_w)
//   u_d = u*/3 + 2 u**/3 (piecewise in q), u_w = v_p + omega_p x (x_w - X_p)
// (or the halfway rule f+_d + 6 w_d rho0 e_j.u_w in Ladd mode), kept per
// link.  The Galilean-invariant momentum exchange of the link,
//   dP = (e_d - u_w) f+_d - (e_j - u_w) G_j = e_d (2 w_d + h_d + h_G) - u_w (h_d - h_G),
// and its torque about X_p are rounded to 2^-40 fixed point per link and
// summed in integers (over the warp, then per block, then over the blocks):
// the sums do not depend on the order in which links are visited.  It reads
// f+(t) only (A, after the refill), so it may run beside the bulk kernel
// (a schedule option); by default it runs after it.
//
// k_boundary, one thread per boundary node, for each direction j: pull
// streaming where the source is fluid, halfway bounce-back where it is
// outside the domain, the link's G_j where it is solid; then BGK collision,
// written into f+(t+1).  Up to IBB_SHARED_PARTICLES particles the link kernel
// leaves its momentum exchange as per-block sums, which this kernel adds into
// the particles' sums first (no launch of its own).
//
// A link is used only when every link of its node fitted into the link list
// (an overflow, reported by the classification, leaves the node on halfway
// bounce-back without momentum exchange until the lists grow).
// ---------------------------------------------------------------------------
namespace {
constexpr unsigned FULLW = 0xffffffffu;
// weight and opposite of a direction given at run time (lex, ley, lez: the
// shared header's packed direction tables)
__device__ __forceinline__ float lw(int j) { return j == 0 ? (1.0f / 3.0f) : (j <= 6 ? (1.0f / 18.0f) : (1.0f / 36.0f)); }
__device__ __forceinline__ int lopp(int j) { return j == 0 ? 0 : ((j & 1) ? j + 1 : j - 1); }

// Exact warp sum of 64-bit fixed-point values (|v| < 2^62): three 22-bit
// pieces, each summed by one integer warp reduction (at most 32 x 2^22 < 2^27,
// no overflow), recombined; the result is in every lane.
__device__ __forceinline__ long long warp_sum_fixed(long long v) {
  const unsigned c0 = (unsigned)(v & 0x3FFFFFLL);
  const unsigned c1 = (unsigned)((v >> 22) & 0x3FFFFFLL);
  const int c2 = (int)(v >> 44);
  const unsigned s0 = __reduce_add_sync(FULLW, c0);
  const unsigned s1 = __reduce_add_sync(FULLW, c1);
  const int s2 = __reduce_add_sync(FULLW, c2);
  return (long long)s0 + ((long long)s1 << 22) + ((long long)s2 << 44);
}

// v * 2^40 rounded to the nearest integer, ties to even: the same value as
// __float2ll_rn(v * 2^40) without a 64-bit conversion.  f = v 2^40 is exact;
// f = h 2^20 + r with h = rint(f 2^-20) (an integer-valued float) and the
// remainder r, |r| <= 2^19, exact in FP32; h 2^20 is an even integer, so the
// nearest-even integer to f is h 2^20 plus the nearest-even integer to r,
// which adding and removing 1.5 2^23 gives (|r| < 2^22).  |v| < 2^10.
__device__ __forceinline__ long long fixed_2m40(float v) {
  const float f = v * 1099511627776.0f;
  const float h = rintf(f * (1.0f / 1048576.0f));
  const float r = f - h * 1048576.0f;
  const int ir = __float_as_int(r + 12582912.0f) - 0x4B400000;
  return ((long long)__float2int_rn(h) << 20) + (long long)ir;
}

}  // namespace

// The link entries of node bi fit into the list (its links were written by
// the classification of this step).
__device__ __forceinline__ bool links_fit(uint32_t loff, uint32_t mask, unsigned cap_links) {
  return (unsigned long long)loff + (unsigned)__popc(mask) <= (unsigned long long)cap_links;
}

template <int ST, bool LADD, bool SHARED>
__global__ void __launch_bounds__(256) k_links_ibb(BoundaryLaunch L) {
  // the block's sums per particle (SHARED) as 64-bit integers in two 32-bit
  // words (native 32-bit shared atomics, the carry of the low word added to
  // the high word), else the global sums directly
  __shared__ unsigned s_lo[SHARED ? 6 * IBB_SHARED_PARTICLES : 1], s_hi[SHARED ? 6 * IBB_SHARED_PARTICLES : 1];
  using T = typename Store<ST>::T;
  const T* __restrict__ A = static_cast<const T*>(L.A);
  const ParticleLaunch& pl = L.pl;
  const LatticeGeom& g = pl.g;
  const unsigned nl = min(pl.ctr->n_links, pl.cap_links);
  const unsigned nbc = min(pl.ctr->n_bc, pl.cap_bc);
  const float rho0 = L.p.rho0;
  const unsigned lane = threadIdx.x & 31u;
  const unsigned stride = gridDim.x * blockDim.x;
  const int n6 = 6 * pl.np;
  if constexpr (SHARED) {
    for (int k = threadIdx.x; k < n6; k += blockDim.x) s_lo[k] = s_hi[k] = 0u;
    __syncthreads();
  }
  const auto flush = [&](int q, const long long* w) {
    for (int k = 0; k < 6; ++k) {
      if constexpr (SHARED) {
        // (hi, lo) += w modulo 2^64: every wrap of the low word is seen by
        // exactly the addition that made it, which carries it into the high word
        const unsigned long long u = (unsigned long long)w[k];
        const unsigned lo = (unsigned)u, old = atomicAdd(&s_lo[6 * q + k], lo);
        const unsigned hi = (unsigned)(u >> 32) + (old + lo < old ? 1u : 0u);
        if (hi) atomicAdd(&s_hi[6 * q + k], hi);
      } else {
        atomicAdd(reinterpret_cast<unsigned long long*>(pl.facc + 6 * q + k), (unsigned long long)w[k]);
      }
    }
  };
  int pacc = -1;  // lane 0: particle of the running fixed-point sums
  long long iacc[6] = {0, 0, 0, 0, 0, 0};
  // whole warps step together (the sums below are warp collectives)
  for (unsigned base = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < nl; base += stride) {
    const unsigned l = base + lane;
    int p = -1;
    float v[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    const unsigned bi = l < nl ? pl.link_bc[l] : 0xffffffffu;
    uint32_t loff = 0, mask = 0;
    if (bi < nbc) {
      loff = pl.bc_loff[bi];
      mask = pl.bc_mask[bi];
    }
    // an entry of this step: inside the range of the node it names, which fitted
    if (bi < nbc && l >= loff && l - loff < (unsigned)__popc(mask) && links_fit(loff, mask, pl.cap_links)) {
      const long long c = pl.bc_cell[bi];
      int x, y, z;
      coords(c, g, x, y, z);
      const int d = pl.link_dir[l];
      const int j = lopp(d);
      const int ed[3] = {lex(d), ley(d), lez(d)};
      const bool inside = (g.periodic[0] || (unsigned)(x + ed[0]) < (unsigned)g.nx) &&
                          (g.periodic[1] || (unsigned)(y + ed[1]) < (unsigned)g.ny) &&
                          (g.periodic[2] || (unsigned)(z + ed[2]) < (unsigned)g.nz);
      if (inside) {
        // own post-collision populations and moments (rho_f, u_f)
        float h[19];
#pragma unroll
        for (int i = 0; i < 19; ++i) h[i] = Store<ST>::dev(A + i * g.plane + c, i);
        float dr = 0.f, j0 = 0.f, j1 = 0.f, j2 = 0.f;
#pragma unroll
        for (int i = 0; i < 19; ++i) {
          dr += h[i];
          j0 += cx(i) * h[i];
          j1 += cy(i) * h[i];
          j2 += cz(i) * h[i];
        }
        float hopp = h[0];  // f+_d(x_f) - w_d
#pragma unroll
        for (int i = 1; i < 19; ++i) hopp = i == d ? h[i] : hopp;
        const float rho_f = 1.0f + dr;
        const float irho_f = 1.0f / rho_f;
        const float uf[3] = {j0 * irho_f, j1 * irho_f, j2 * irho_f};
        p = (int)pl.link_p[l];
        const DevParticle& P = pl.P[p];
        const float q = LADD ? 0.5f : pl.link_q[l];
        const float wj = lw(j);
        // wall point relative to the particle position: x - X = (x - floor X) - frac X,
        // the integer part exact and the fraction rounded once to FP32
        const float r0 = ((float)(x - P.pos_i[0]) - P.pos_fr[0]) + q * ed[0];
        const float r1 = ((float)(y - P.pos_i[1]) - P.pos_fr[1]) + q * ed[1];
        const float r2 = ((float)(z - P.pos_i[2]) - P.pos_fr[2]) + q * ed[2];
        float uw[3];
        uw[0] = P.velf[0] + (P.omegaf[1] * r2 - P.omegaf[2] * r1);
        uw[1] = P.velf[1] + (P.omegaf[2] * r0 - P.omegaf[0] * r2);
        uw[2] = P.velf[2] + (P.omegaf[0] * r1 - P.omegaf[1] * r0);
        const float wall = 6.0f * wj * rho0 * (-ed[0] * uw[0] - ed[1] * uw[1] - ed[2] * uw[2]);
        float G;
        if (LADD) {
          G = hopp + wall;
        } else {
          // u at the second fluid node x_f - e_d when it is fluid, else u_f
          float uff[3] = {uf[0], uf[1], uf[2]};
          long long ff;
          if (nbr_wrap(x, y, z, -ed[0], -ed[1], -ed[2], g, ff) && pl.owner_cur[ff] == OWNER_NONE) {
            float rr;
            moments_at<ST>(A, g.plane, ff, rr, uff);
          }
          float ud[3];
          const float i1q = 1.0f / (1.0f + q), iq = 1.0f / q;
          const float a1 = (1.0f - q) * i1q, a2 = 2.0f * q * i1q;
          const float b1 = (1.0f - q) * iq, b2 = (2.0f * q - 1.0f) * iq;
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            const float us = q <= 0.5f ? 2.0f * q * uf[a] + (1.0f - 2.0f * q) * uff[a] : b1 * uf[a] + b2 * uw[a];
            ud[a] = us / 3.0f + 2.0f * (a1 * uff[a] + a2 * uw[a]) / 3.0f;
          }
          const float eud = ed[0] * ud[0] + ed[1] * ud[1] + ed[2] * ud[2];
          const float euf = ed[0] * uf[0] + ed[1] * uf[1] + ed[2] * uf[2];
          const float ud2 = ud[0] * ud[0] + ud[1] * ud[1] + ud[2] * ud[2];
          const float uf2 = uf[0] * uf[0] + uf[1] * uf[1] + uf[2] * uf[2];
          G = hopp + wj * rho_f * (3.0f * (eud - euf) + 4.5f * (eud * eud - euf * euf) - 1.5f * (ud2 - uf2)) + wall;
        }
        pl.link_g[l] = G;
        const float s2 = 2.0f * wj + hopp + G, dl = hopp - G;
        v[0] = ed[0] * s2 - uw[0] * dl;
        v[1] = ed[1] * s2 - uw[1] * dl;
        v[2] = ed[2] * s2 - uw[2] * dl;
        v[3] = r1 * v[2] - r2 * v[1];
        v[4] = r2 * v[0] - r0 * v[2];
        v[5] = r0 * v[1] - r1 * v[0];
      }
    }
    // momentum exchange: each link's contribution rounded to 2^-40 fixed point
    // in its own lane (v * 2^40 is exact in FP32 and the rounding is to nearest
    // even: odd-symmetric, so opposite links of a closed body cancel exactly),
    // summed over the warp in integers and kept by lane 0 while the particle
    // does not change
    if (__any_sync(FULLW, p >= 0)) {
      const int pmin = __reduce_min_sync(FULLW, p >= 0 ? p : 0x7fffffff);
      const bool single = __all_sync(FULLW, p < 0 || p == pmin);
      long long iv[6];
#pragma unroll
      for (int k = 0; k < 6; ++k) iv[k] = p >= 0 ? fixed_2m40(v[k]) : 0LL;
      if (single) {
#pragma unroll
        for (int k = 0; k < 6; ++k) iv[k] = warp_sum_fixed(iv[k]);
        if (lane == 0) {
          if (pacc != pmin) {
            if (pacc >= 0) flush(pacc, iacc);
            pacc = pmin;
            for (int k = 0; k < 6; ++k) iacc[k] = 0;
          }
          for (int k = 0; k < 6; ++k) iacc[k] += iv[k];
        }
      } else if (p >= 0) {  // links to several particles: per-link atomics
        flush(p, iv);
      }
    }
  }
  if (lane == 0 && pacc >= 0) flush(pacc, iacc);
  if constexpr (SHARED) {
    __syncthreads();
    long long* out = L.part + (size_t)blockIdx.x * n6;
    for (int k = threadIdx.x; k < n6; k += blockDim.x)
      out[k] = (long long)(((unsigned long long)s_hi[k] << 32) | (unsigned long long)s_lo[k]);
  }
}

template <int ST, bool FORCE>
__global__ void __launch_bounds__(256) k_boundary(BoundaryLaunch L) {
  using T = typename Store<ST>::T;
  const T* __restrict__ A = static_cast<const T*>(L.A);
  T* __restrict__ B = static_cast<T*>(L.B);
  const LatticeGeom& g = L.pl.g;
  const ParticleLaunch& pl = L.pl;
  const unsigned nbc = min(pl.ctr->n_bc, pl.cap_bc);
  const float om = L.p.omega;
  if (L.part && pl.np <= IBB_SHARED_PARTICLES) {
    // the link kernel's per-block momentum-exchange sums into the particles'
    // fixed-point sums (it ran before this kernel), a warp per component
    const int n6 = 6 * pl.np;
    const unsigned lane = threadIdx.x & 31u;
    for (unsigned k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < (unsigned)n6;
         k += (gridDim.x * blockDim.x) >> 5) {
      long long v = 0;
      for (int b = (int)lane; b < L.part_blocks; b += 32) v += L.part[(size_t)b * n6 + k];
      v = warp_sum_fixed(v);
      if (lane == 0 && v) atomicAdd(reinterpret_cast<unsigned long long*>(pl.facc + k), (unsigned long long)v);
    }
  }
  for (unsigned bi = blockIdx.x * blockDim.x + threadIdx.x; bi < nbc; bi += gridDim.x * blockDim.x) {
    const long long c = pl.bc_cell[bi];
    const uint32_t mask = pl.bc_mask[bi];
    const uint32_t loff = pl.bc_loff[bi];
    const bool fit = links_fit(loff, mask, pl.cap_links);
    int x, y, z;
    coords(c, g, x, y, z);
    float h[19];
#pragma unroll
    for (int j = 0; j < 19; ++j) {
      const int d = opp(j);  // link direction of j (towards the source node)
      int sx = x - cx(j), sy = y - cy(j), sz = z - cz(j);
      int face = -1;  // a corner crossing is attributed to x, then y, then z
      if (sz < 0) { if (g.periodic[2]) sz += g.nz; else face = 4; }
      else if (sz >= g.nz) { if (g.periodic[2]) sz -= g.nz; else face = 5; }
      if (sy < 0) { if (g.periodic[1]) sy += g.ny; else face = 2; }
      else if (sy >= g.ny) { if (g.periodic[1]) sy -= g.ny; else face = 3; }
      if (sx < 0) { if (g.periodic[0]) sx += g.nx; else face = 0; }
      else if (sx >= g.nx) { if (g.periodic[0]) sx -= g.nx; else face = 1; }
      if (face >= 0) {
        h[j] = Store<ST>::dev(A + d * g.plane + c, d) + L.p.bb_wall[face][j];
      } else if (j == 0 || !((mask >> d) & 1u)) {
        h[j] = Store<ST>::dev(A + j * g.plane + (sx + (long long)g.nx * (sy + (long long)g.ny * sz)), j);
      } else if (fit) {
        h[j] = pl.link_g[loff + __popc(mask & ((1u << d) - 1u))];
      } else {
        h[j] = Store<ST>::dev(A + d * g.plane + c, d);
      }
    }
    // BGK collision of the node
    float drho = 0.f, j0 = 0.f, j1 = 0.f, j2 = 0.f;
#pragma unroll
    for (int i = 0; i < 19; ++i) {
      drho += h[i];
      j0 += cx(i) * h[i];
      j1 += cy(i) * h[i];
      j2 += cz(i) * h[i];
    }
    const float rho = 1.0f + drho;
    const float irho = 1.0f / rho;
    float u0, u1, u2;
    if (FORCE) {
      u0 = (j0 + 0.5f * L.p.force[0]) * irho;
      u1 = (j1 + 0.5f * L.p.force[1]) * irho;
      u2 = (j2 + 0.5f * L.p.force[2]) * irho;
    } else {
      u0 = j0 * irho;
      u1 = j1 * irho;
      u2 = j2 * irho;
    }
    const float usq15 = 1.5f * (u0 * u0 + u1 * u1 + u2 * u2);
#pragma unroll
    for (int j = 0; j < 19; ++j) {
      const float eu = cx(j) * u0 + cy(j) * u1 + cz(j) * u2;
      const float feq_dev = wq(j) * (drho + rho * (3.0f * eu + 4.5f * eu * eu - usq15));
      float hp = h[j] + om * (feq_dev - h[j]);
      if (FORCE) {
        const float eF = cx(j) * L.p.force[0] + cy(j) * L.p.force[1] + cz(j) * L.p.force[2];
        const float uF = u0 * L.p.force[0] + u1 * L.p.force[1] + u2 * L.p.force[2];
        hp += (1.0f - 0.5f * om) * wq(j) * (3.0f * (eF - uF) + 9.0f * eu * eF);
      }
      if (L.tmp) Store<ST>::put(static_cast<T*>(L.tmp) + 19 * (size_t)bi + j, j, hp);
      else Store<ST>::put(B + j * g.plane + c, j, hp);
    }
  }
}

// A list kernel's grid: the tuned block count, but no more blocks than the
// list's capacity (`items` work units at `threads` per block) can use, so
// that small lists do not dispatch thousands of empty blocks.
static inline int list_grid(int tuned, unsigned long long items, int threads) {
  const unsigned long long need = (items + (unsigned long long)threads - 1) / (unsigned long long)threads;
  return (int)(need < 1 ? 1 : (need < (unsigned long long)tuned ? need : (unsigned long long)tuned));
}

template <int ST>
static cudaError_t launch_refill_st(const BoundaryLaunch& L, cudaStream_t s) {
  k_refill<ST><<<list_grid(L.grid, L.pl.cap_new, 128), 128, 0, s>>>(L);
  return cudaGetLastError();
}

cudaError_t launch_refill(const BoundaryLaunch& L, cudaStream_t s) {
  if (L.pl.np == 0) return cudaSuccess;
  switch (L.storage) {
    case MI_STORE_F32: return launch_refill_st<MI_STORE_F32>(L, s);
    case MI_STORE_F16_DEV: return launch_refill_st<MI_STORE_F16_DEV>(L, s);
    case MI_STORE_BF16_DEV: return launch_refill_st<MI_STORE_BF16_DEV>(L, s);
  }
  return cudaErrorInvalidValue;
}

template <int ST>
static cudaError_t launch_links_ibb_st(const BoundaryLaunch& L, cudaStream_t s) {
  const bool ladd = L.bb_mode == MI_BB_LADD;
  if (L.part && L.pl.np <= IBB_SHARED_PARTICLES) {
    if (ladd) k_links_ibb<ST, true, true><<<L.part_blocks, 256, 0, s>>>(L);
    else k_links_ibb<ST, false, true><<<L.part_blocks, 256, 0, s>>>(L);
  } else {
    const int grid = list_grid(L.grid, L.pl.cap_links, 256);
    if (ladd) k_links_ibb<ST, true, false><<<grid, 256, 0, s>>>(L);
    else k_links_ibb<ST, false, false><<<grid, 256, 0, s>>>(L);
  }
  return cudaGetLastError();
}

cudaError_t launch_links_ibb(const BoundaryLaunch& L, cudaStream_t s) {
  if (L.pl.np == 0) return cudaSuccess;
  switch (L.storage) {
    case MI_STORE_F32: return launch_links_ibb_st<MI_STORE_F32>(L, s);
    case MI_STORE_F16_DEV: return launch_links_ibb_st<MI_STORE_F16_DEV>(L, s);
    case MI_STORE_BF16_DEV: return launch_links_ibb_st<MI_STORE_BF16_DEV>(L, s);
  }
  return cudaErrorInvalidValue;
}

template <int ST>
static cudaError_t launch_near_st(const BoundaryLaunch& L, cudaStream_t s) {
  const int grid = list_grid(L.grid, 18ull * L.pl.cap_new, 128);
  if (L.forcing) k_near<ST, true><<<grid, 128, 0, s>>>(L);
  else k_near<ST, false><<<grid, 128, 0, s>>>(L);
  return cudaGetLastError();
}

cudaError_t launch_near(const BoundaryLaunch& L, cudaStream_t s) {
  if (L.pl.np == 0) return cudaSuccess;
  switch (L.storage) {
    case MI_STORE_F32: return launch_near_st<MI_STORE_F32>(L, s);
    case MI_STORE_F16_DEV: return launch_near_st<MI_STORE_F16_DEV>(L, s);
    case MI_STORE_BF16_DEV: return launch_near_st<MI_STORE_BF16_DEV>(L, s);
  }
  return cudaErrorInvalidValue;
}

template <int ST>
static cudaError_t launch_boundary_st(const BoundaryLaunch& L, cudaStream_t s) {
  const int grid = list_grid(L.grid, L.pl.cap_bc, 256);
  if (L.forcing) k_boundary<ST, true><<<grid, 256, 0, s>>>(L);
  else k_boundary<ST, false><<<grid, 256, 0, s>>>(L);
  return cudaGetLastError();
}

template <typename T>
__global__ void __launch_bounds__(256) k_scatter_boundary(BoundaryLaunch L) {
  const unsigned nbc = min(L.pl.ctr->n_bc, L.pl.cap_bc);
  const T* __restrict__ tmp = static_cast<const T*>(L.tmp);
  T* __restrict__ B = static_cast<T*>(L.B);
  for (unsigned e = blockIdx.x * blockDim.x + threadIdx.x; e < 19u * nbc; e += gridDim.x * blockDim.x) {
    const unsigned k = e / 19u, j = e - 19u * k;
    B[j * L.pl.g.plane + L.pl.bc_cell[k]] = tmp[e];
  }
}

cudaError_t launch_scatter_boundary(const BoundaryLaunch& L, cudaStream_t s) {
  if (L.pl.np == 0 || !L.tmp) return cudaSuccess;
  const int grid = list_grid(L.grid, 19ull * L.pl.cap_bc, 256);
  if (L.storage == MI_STORE_F32) k_scatter_boundary<float><<<grid, 256, 0, s>>>(L);
  else k_scatter_boundary<unsigned short><<<grid, 256, 0, s>>>(L);
  return cudaGetLastError();
}

cudaError_t launch_boundary(const BoundaryLaunch& L, cudaStream_t s) {
  if (L.pl.np == 0) return cudaSuccess;
  switch (L.storage) {
    case MI_STORE_F32: return launch_boundary_st<MI_STORE_F32>(L, s);
    case MI_STORE_F16_DEV: return launch_boundary_st<MI_STORE_F16_DEV>(L, s);
    case MI_STORE_BF16_DEV: return launch_boundary_st<MI_STORE_BF16_DEV>(L, s);
  }
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// Fill / pack / unpack (set-up and inspection, not on the step path).
// ---------------------------------------------------------------------------
template <int ST>
__global__ void k_fill_rest(typename Store<ST>::T* pop, long long ncell, long long plane, float rho0) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= ncell) return;
#pragma unroll
  for (int i = 0; i < 19; ++i) Store<ST>::put(pop + i * plane + n, i, wq(i) * (rho0 - 1.0f));
}

template <int ST>
__global__ void k_pack(const float* __restrict__ src, typename Store<ST>::T* pop, long long ncell, long long plane) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= ncell) return;
#pragma unroll
  for (int i = 0; i < 19; ++i) Store<ST>::put(pop + i * plane + n, i, src[i * ncell + n] - wq(i));
}

// F32 storage keeps f itself: copy the bits so that a set/get round trip is exact.
__global__ void k_pack_f32(const float* __restrict__ src, float* pop, long long ncell, long long plane) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= ncell) return;
#pragma unroll
  for (int i = 0; i < 19; ++i) pop[i * plane + n] = src[i * ncell + n];
}
__global__ void k_unpack_f32(const float* pop, float* __restrict__ dst, long long ncell, long long plane) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= ncell) return;
#pragma unroll
  for (int i = 0; i < 19; ++i) dst[i * ncell + n] = pop[i * plane + n];
}

template <int ST>
__global__ void k_unpack(const typename Store<ST>::T* pop, float* __restrict__ dst, long long ncell, long long plane) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= ncell) return;
#pragma unroll
  for (int i = 0; i < 19; ++i) dst[i * ncell + n] = Store<ST>::dev(pop + i * plane + n, i) + wq(i);
}

static inline long long ncell_of(const LatticeGeom& g) { return (long long)g.nx * g.ny * g.nz; }

// Non-finite stored populations (NaN or infinite) at nodes that are not solid
// (owner NULL: every node): out[0] += their count, out[1] = the smallest
// such node index.  For 16-bit storages the test is on the bits (an all-ones
// exponent).
__device__ __forceinline__ bool bad_value(float v) { return !isfinite(v); }
__device__ __forceinline__ bool bad_value(__half v) { return (__half_as_ushort(v) & 0x7C00u) == 0x7C00u; }
__device__ __forceinline__ bool bad_value(__nv_bfloat16 v) { return (__bfloat16_as_ushort(v) & 0x7F80u) == 0x7F80u; }

template <int ST>
__global__ void __launch_bounds__(256) k_check(const typename Store<ST>::T* __restrict__ pop, long long ncell,
                                               long long plane, const uint32_t* __restrict__ owner,
                                               long long* __restrict__ out) {
  long long nbad = 0, first = LLONG_MAX;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell; c += (long long)gridDim.x * blockDim.x) {
    if (owner && owner[c] != OWNER_NONE) continue;
    int k = 0;
#pragma unroll
    for (int i = 0; i < 19; ++i) k += bad_value(pop[i * plane + c]) ? 1 : 0;
    if (k) {
      nbad += k;
      first = c < first ? c : first;
    }
  }
  if (nbad) {
    atomicAdd(reinterpret_cast<unsigned long long*>(out), (unsigned long long)nbad);
    atomicMin(out + 1, first);
  }
}

cudaError_t launch_check(const void* pop, const LatticeGeom& g, int storage, const uint32_t* owner, long long* out,
                         int sm_count, cudaStream_t s) {
  const long long init[2] = {0, LLONG_MAX};
  cudaError_t e = cudaMemcpyAsync(out, init, sizeof(init), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  const long long ncell = (long long)g.nx * g.ny * g.nz;
  const int grid = sm_count * 8;
  if (storage == MI_STORE_F16_DEV)
    k_check<MI_STORE_F16_DEV><<<grid, 256, 0, s>>>(static_cast<const __half*>(pop), ncell, g.plane, owner, out);
  else if (storage == MI_STORE_BF16_DEV)
    k_check<MI_STORE_BF16_DEV><<<grid, 256, 0, s>>>(static_cast<const __nv_bfloat16*>(pop), ncell, g.plane, owner, out);
  else
    k_check<MI_STORE_F32><<<grid, 256, 0, s>>>(static_cast<const float*>(pop), ncell, g.plane, owner, out);
  return cudaGetLastError();
}

cudaError_t launch_fill_rest(void* pop, const LatticeGeom& g, int storage, float rho0, cudaStream_t s) {
  const long long n = ncell_of(g);
  const unsigned blocks = (unsigned)((n + 255) / 256);
  switch (storage) {
    case MI_STORE_F32: k_fill_rest<MI_STORE_F32><<<blocks, 256, 0, s>>>((float*)pop, n, g.plane, rho0); break;
    case MI_STORE_F16_DEV: k_fill_rest<MI_STORE_F16_DEV><<<blocks, 256, 0, s>>>((__half*)pop, n, g.plane, rho0); break;
    case MI_STORE_BF16_DEV: k_fill_rest<MI_STORE_BF16_DEV><<<blocks, 256, 0, s>>>((__nv_bfloat16*)pop, n, g.plane, rho0); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_pack(const float* src, void* pop, const LatticeGeom& g, int storage, cudaStream_t s) {
  const long long n = ncell_of(g);
  const unsigned blocks = (unsigned)((n + 255) / 256);
  switch (storage) {
    case MI_STORE_F32: k_pack_f32<<<blocks, 256, 0, s>>>(src, (float*)pop, n, g.plane); break;
    case MI_STORE_F16_DEV: k_pack<MI_STORE_F16_DEV><<<blocks, 256, 0, s>>>(src, (__half*)pop, n, g.plane); break;
    case MI_STORE_BF16_DEV: k_pack<MI_STORE_BF16_DEV><<<blocks, 256, 0, s>>>(src, (__nv_bfloat16*)pop, n, g.plane); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_unpack(const void* pop, float* dst, const LatticeGeom& g, int storage, cudaStream_t s) {
  const long long n = ncell_of(g);
  const unsigned blocks = (unsigned)((n + 255) / 256);
  switch (storage) {
    case MI_STORE_F32: k_unpack_f32<<<blocks, 256, 0, s>>>((const float*)pop, dst, n, g.plane); break;
    case MI_STORE_F16_DEV: k_unpack<MI_STORE_F16_DEV><<<blocks, 256, 0, s>>>((const __half*)pop, dst, n, g.plane); break;
    case MI_STORE_BF16_DEV: k_unpack<MI_STORE_BF16_DEV><<<blocks, 256, 0, s>>>((const __nv_bfloat16*)pop, dst, n, g.plane); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace mi
