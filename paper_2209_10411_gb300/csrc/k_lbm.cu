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
#include "mi_internal.cuh"

namespace mi {

// BGK collision on deviations h_i = f_i - w_i and store of the result.
//   rho = 1 + sum h_i, j = sum e_i h_i (sum w_i = 1, sum w_i e_i = 0)
//   f_eq,i - w_i = w_i (rho - 1) + w_i rho (3 e.u + 4.5 (e.u)^2 - 1.5 u.u)
//   h+_i = h_i + omega (f_eq,i - w_i - h_i)   [+ Guo source]
template <int ST, bool FORCE>
__device__ __forceinline__ void collide_store(const float (&h)[19], typename Store<ST>::T* __restrict__ B,
                                              long long plane, long long c, const CollideParams& P) {
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
    Store<ST>::put(B + i * plane + c, i, hp);
  }
}

template <int ST, bool FORCE, bool HAS_CLS>
__global__ void __launch_bounds__(256) k_bulk(const typename Store<ST>::T* __restrict__ A,
                                              typename Store<ST>::T* __restrict__ B,
                                              const uint8_t* __restrict__ cls, LatticeGeom g,
                                              CollideParams P) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y, z = blockIdx.z;
  if (x >= g.nx) return;
  const long long nxy = (long long)g.nx * g.ny;
  const long long c = x + (long long)g.nx * y + nxy * z;
  if (HAS_CLS) {
    if (__ldg(cls + c) != 0) return;  // solid, boundary and new nodes go elsewhere
  }
  float h[19];
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
  collide_store<ST, FORCE>(h, B, g.plane, c, P);
}

template <int ST, bool FORCE, bool HAS_CLS>
static cudaError_t launch_bulk_t(const BulkLaunch& L, cudaStream_t s) {
  using T = typename Store<ST>::T;
  const int bx = L.block_x;
  dim3 grid((L.g.nx + bx - 1) / bx, L.g.ny, L.g.nz);
  k_bulk<ST, FORCE, HAS_CLS><<<grid, bx, 0, s>>>(static_cast<const T*>(L.A), static_cast<T*>(L.B), L.cls, L.g, L.p);
  return cudaGetLastError();
}

template <int ST>
static cudaError_t launch_bulk_st(const BulkLaunch& L, cudaStream_t s) {
  if (L.forcing) return L.cls ? launch_bulk_t<ST, true, true>(L, s) : launch_bulk_t<ST, true, false>(L, s);
  return L.cls ? launch_bulk_t<ST, false, true>(L, s) : launch_bulk_t<ST, false, false>(L, s);
}

cudaError_t launch_bulk(const BulkLaunch& L, cudaStream_t s) {
  if (L.block_x <= 0 || L.block_x > 256 || (L.block_x % 32) != 0) return cudaErrorInvalidValue;
  switch (L.storage) {
    case MI_STORE_F32: return launch_bulk_st<MI_STORE_F32>(L, s);
    case MI_STORE_F16_DEV: return launch_bulk_st<MI_STORE_F16_DEV>(L, s);
    case MI_STORE_BF16_DEV: return launch_bulk_st<MI_STORE_BF16_DEV>(L, s);
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
