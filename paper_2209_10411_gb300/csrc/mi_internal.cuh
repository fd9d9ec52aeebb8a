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
  const uint8_t* cls;  // node classes, or nullptr when no node is solid/boundary
  LatticeGeom g;
  CollideParams p;
  int storage;
  bool forcing;
  int block_x;         // threads per block along x
};
cudaError_t launch_bulk(const BulkLaunch& L, cudaStream_t s);

// Fill every node with the rest state f_i = w_i rho0.
cudaError_t launch_fill_rest(void* pop, const LatticeGeom& g, int storage, float rho0, cudaStream_t s);
// Convert float populations [19][ncell] (dense) to/from the storage layout.
cudaError_t launch_pack(const float* src, void* pop, const LatticeGeom& g, int storage, cudaStream_t s);
cudaError_t launch_unpack(const void* pop, float* dst, const LatticeGeom& g, int storage, cudaStream_t s);

}  // namespace mi
