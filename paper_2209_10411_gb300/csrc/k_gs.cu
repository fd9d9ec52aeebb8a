// Gradient Search refinement of metaball models on point hulls (Sec. 2.2,
// Algorithm 2, Eq. GSloss), one fit at a time per CTA, the fits taken
// largest first by persistent CTAs.  The fit's hull points, model
// and gradients stay in shared memory for all epochs; an epoch is two passes:
// threads over hull points evaluate the field and dl/df (kept beside each
// point; two points per thread at a time for two independent sums), then the
// (control point, chunk of GS_CHUNKS points) units are spread over the warps,
// each summing its four gradient components with a fixed lane order and
// butterfly, and one thread per control point adds its chunks in order.
// Everything is FP32; the reductions have a fixed order, so a fit's result
// does not depend on the other fits of the call.
#include <cmath>

#include "mi_gs.h"
#include "mi_internal.cuh"

namespace mi {
namespace {

constexpr int GS_THREADS = 1024;
constexpr int GS_CHUNKS = 8;  // hull-point chunks per control point in the gradient pass
constexpr unsigned GS_FULL = 0xffffffffu;

// dl/df of Eq. GSloss: 2 (f - 1) on [2, inf), +1 on [1, 2), 2 (f - 1) - 1/f^2 below
__device__ __forceinline__ float gs_dl(float f) {
  return f >= 2.0f ? 2.0f * (f - 1.0f) : (f >= 1.0f ? 1.0f : 2.0f * (f - 1.0f) - 1.0f / (f * f));
}

// l(f) of Eq. GSloss
__device__ __forceinline__ float gs_l(float f) {
  return f >= 2.0f ? (f - 1.0f) * (f - 1.0f) : (f >= 1.0f ? f - 1.0f : (f - 1.0f) * (f - 1.0f) + 1.0f / f - 1.0f);
}

// f at (x, y, z): sum over the model's balls in order
__device__ __forceinline__ float gs_field(const float4* M, int n, float x, float y, float z) {
  float f = 0.f;
  for (int j = 0; j < n; ++j) {
    const float4 b = M[j];
    const float dx = x - b.x, dy = y - b.y, dz = z - b.z;
    f += b.w * __fdividef(1.0f, dx * dx + dy * dy + dz * dz);
  }
  return f;
}

// Sum of one value per thread in a fixed tree order; the result in every thread.
__device__ __forceinline__ float gs_block_sum(float v, float* red) {
  const int t = threadIdx.x;
  red[t] = v;
  __syncthreads();
  for (int s = GS_THREADS / 2; s > 0; s >>= 1) {
    if (t < s) red[t] += red[t + s];
    __syncthreads();
  }
  const float r = red[0];
  __syncthreads();
  return r;
}

struct GsLaunch {
  const int* hull_off;
  const float* hull;
  const int* ball_off;
  float* balls;
  const int* plane_off;
  const float* planes;
  int max_points, max_balls, epochs;
  float lr;
  int* active;
  float* loss;
};

// One fit by the whole CTA (every thread calls it with the same fit).
__device__ __forceinline__ void gs_fit_one(const GsLaunch& G, int fit, float4* gsm, float* red) {
  float4* Hs = gsm;                      // hull points (x, y, z, dl/df of the last pass)
  float4* Ms = Hs + G.max_points;        // model (x, y, z, k)
  float4* Ps = Ms + G.max_balls;         // gradient partial sums per (control point, chunk)
  int* act = reinterpret_cast<int*>(Ps + (size_t)G.max_balls * GS_CHUNKS);
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int h0 = G.hull_off[fit], m = G.hull_off[fit + 1] - h0;
  const int b0 = G.ball_off[fit], n = G.ball_off[fit + 1] - b0;
  const int p0 = G.plane_off[fit], np_ = G.plane_off[fit + 1] - p0;
  if (m <= 0 || n <= 0 || m > G.max_points || n > G.max_balls) {
    if (t == 0) G.loss[2 * fit] = G.loss[2 * fit + 1] = __int_as_float(0x7fc00000);
    return;
  }
  for (int i = t; i < m; i += GS_THREADS)
    Hs[i] = make_float4(G.hull[3 * (h0 + i)], G.hull[3 * (h0 + i) + 1], G.hull[3 * (h0 + i) + 2], 0.f);
  for (int j = t; j < n; j += GS_THREADS) {
    const float* b = G.balls + 4 * (b0 + j);
    Ms[j] = make_float4(b[0], b[1], b[2], b[3]);
    act[j] = 1;
  }
  __syncthreads();
  float loss1 = 0.f;
  for (int round = 0; round < 2; ++round) {
    for (int e = 0; e < G.epochs; ++e) {
      // dl/df at every hull point, two points per thread at a time
      for (int i = t; i < m; i += 2 * GS_THREADS) {
        const int i2 = i + GS_THREADS;
        const float4 ha = Hs[i], hb = Hs[i2 < m ? i2 : i];
        float fa = 0.f, fb = 0.f;
        for (int j = 0; j < n; ++j) {
          const float4 b = Ms[j];
          const float ax = ha.x - b.x, ay = ha.y - b.y, az = ha.z - b.z;
          const float bx = hb.x - b.x, by = hb.y - b.y, bz = hb.z - b.z;
          fa += b.w * __fdividef(1.0f, ax * ax + ay * ay + az * az);
          fb += b.w * __fdividef(1.0f, bx * bx + by * by + bz * bz);
        }
        Hs[i].w = gs_dl(fa);
        if (i2 < m) Hs[i2].w = gs_dl(fb);
      }
      __syncthreads();
      // gradient of every control point: dL/dk = sum w / r^2, dL/dc = sum w 2 k (H - c) / r^4,
      // as GS_CHUNKS partial sums over contiguous chunks of the points
      const int csz = (m + GS_CHUNKS - 1) / GS_CHUNKS;
      for (int u = w; u < n * GS_CHUNKS; u += GS_THREADS / 32) {
        const int j = u / GS_CHUNKS, ch = u - j * GS_CHUNKS;
        const int i0 = ch * csz, i1 = min(m, i0 + csz);
        const float4 b = Ms[j];
        float gx = 0.f, gy = 0.f, gz = 0.f, gk = 0.f;
        for (int i = i0 + lane; i < i1; i += 32) {
          const float4 h = Hs[i];
          const float dx = h.x - b.x, dy = h.y - b.y, dz = h.z - b.z;
          const float inv = __fdividef(1.0f, dx * dx + dy * dy + dz * dz);
          gk += h.w * inv;
          const float s = h.w * 2.0f * b.w * inv * inv;
          gx += s * dx;
          gy += s * dy;
          gz += s * dz;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          gx += __shfl_xor_sync(GS_FULL, gx, o);
          gy += __shfl_xor_sync(GS_FULL, gy, o);
          gz += __shfl_xor_sync(GS_FULL, gz, o);
          gk += __shfl_xor_sync(GS_FULL, gk, o);
        }
        if (lane == 0) Ps[u] = make_float4(gx, gy, gz, gk);
      }
      __syncthreads();
      for (int j = t; j < n; j += GS_THREADS)
        if (act[j]) {
          float4 g = Ps[j * GS_CHUNKS];
          for (int ch = 1; ch < GS_CHUNKS; ++ch) {
            const float4 q = Ps[j * GS_CHUNKS + ch];
            g.x += q.x;
            g.y += q.y;
            g.z += q.z;
            g.w += q.w;
          }
          float4 b = Ms[j];
          b.x -= G.lr * g.x;
          b.y -= G.lr * g.y;
          b.z -= G.lr * g.z;
          b.w -= G.lr * g.w;
          Ms[j] = b;
        }
      __syncthreads();
    }
    // the loss of the model after this descent
    float part = 0.f;
    for (int i = t; i < m; i += GS_THREADS) {
      const float4 h = Hs[i];
      part += gs_l(gs_field(Ms, n, h.x, h.y, h.z));
    }
    const float L = gs_block_sum(part, red);
    if (round == 0) {
      loss1 = L;
      // anomalies: k < 0, or outside a facet plane (FP32, single roundings, left to right)
      for (int j = t; j < n; j += GS_THREADS) {
        const float4 b = Ms[j];
        bool bad = b.w < 0.f;
        for (int p = 0; p < np_ && !bad; ++p) {
          const float* P = G.planes + 4 * (p0 + p);
          const float s = __fadd_rn(__fadd_rn(__fmul_rn(P[0], b.x), __fmul_rn(P[1], b.y)), __fmul_rn(P[2], b.z));
          bad = s > P[3];
        }
        if (bad) {
          Ms[j].w = 0.f;
          act[j] = 0;
        }
      }
      __syncthreads();
    } else if (t == 0) {
      G.loss[2 * fit] = loss1;
      G.loss[2 * fit + 1] = L;
    }
  }
  for (int j = t; j < n; j += GS_THREADS) {
    float* b = G.balls + 4 * (b0 + j);
    const float4 v = Ms[j];
    b[0] = v.x;
    b[1] = v.y;
    b[2] = v.z;
    b[3] = v.w;
    G.active[b0 + j] = act[j];
  }
  __syncthreads();  // the shared buffers are free for the next fit
}

// Fits in decreasing order of work (hull points x control points, ties to the
// lower index): order[r] is the fit of rank r.
__global__ void k_gs_order(GsLaunch G, int n_fits, int* order) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n_fits) return;
  auto work = [&](int f) {
    return (long long)(G.hull_off[f + 1] - G.hull_off[f]) * (long long)(G.ball_off[f + 1] - G.ball_off[f]);
  };
  const long long wj = work(j);
  int r = 0;
  for (int i = 0; i < n_fits; ++i) {
    const long long wi = work(i);
    r += (wi > wj) || (wi == wj && i < j);
  }
  order[r] = j;
}

// Persistent CTAs take the fits largest first from a counter, so that the
// SMs' loads even out (longest-processing-time-first scheduling).
__global__ void __launch_bounds__(GS_THREADS) k_gs_fit(GsLaunch G, int n_fits, const int* order, int* next) {
  extern __shared__ __align__(16) float4 gsm[];
  __shared__ float red[GS_THREADS];
  __shared__ int pick;
  for (;;) {
    if (threadIdx.x == 0) pick = atomicAdd(next, 1);
    __syncthreads();
    const int q = pick;
    __syncthreads();
    if (q >= n_fits) break;
    gs_fit_one(G, order[q], gsm, red);
  }
}

}  // namespace
}  // namespace mi

extern "C" mi_status mi_gs_fit(int n_fits, const int* hull_off, const float* hull, const int* ball_off, float* balls,
                               const int* plane_off, const float* planes, int max_points, int max_balls, int epochs,
                               float lr, int* active, float* loss, void* stream) {
  using namespace mi;
  if (n_fits < 0 || epochs < 0 || !std::isfinite(lr) || max_points < 1 || max_points > MI_GS_MAX_POINTS ||
      max_balls < 1 || max_balls > MI_GS_MAX_BALLS)
    return MI_EINVAL;
  if (n_fits == 0) return MI_OK;
  if (!hull_off || !hull || !ball_off || !balls || !plane_off || !planes || !active || !loss) return MI_EINVAL;
  GsLaunch G;
  G.hull_off = hull_off;
  G.hull = hull;
  G.ball_off = ball_off;
  G.balls = balls;
  G.plane_off = plane_off;
  G.planes = planes;
  G.max_points = max_points;
  G.max_balls = max_balls;
  G.epochs = epochs;
  G.lr = lr;
  G.active = active;
  G.loss = loss;
  const size_t smem =
      sizeof(float4) * ((size_t)max_points + (size_t)(1 + GS_CHUNKS) * max_balls) + sizeof(int) * max_balls;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaFuncSetAttribute(k_gs_fit, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return MI_ECUDA;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gs_fit, GS_THREADS, smem) != cudaSuccess)
    return MI_ECUDA;
  // the fit order and the pick counter, stream-ordered scratch
  int* tmp = nullptr;
  if (cudaMallocAsync(reinterpret_cast<void**>(&tmp), sizeof(int) * ((size_t)n_fits + 1), s) != cudaSuccess)
    return MI_ECUDA;
  int* order = tmp + 1;
  e = cudaMemsetAsync(tmp, 0, sizeof(int), s);
  if (e == cudaSuccess) {
    k_gs_order<<<(n_fits + 255) / 256, 256, 0, s>>>(G, n_fits, order);
    long long grid = (long long)(sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
    if (grid > n_fits) grid = n_fits;
    k_gs_fit<<<(unsigned)grid, GS_THREADS, smem, s>>>(G, n_fits, order, tmp);
    e = cudaGetLastError();
  }
  const cudaError_t ef = cudaFreeAsync(tmp, s);
  return e == cudaSuccess && ef == cudaSuccess ? MI_OK : MI_ECUDA;
}
