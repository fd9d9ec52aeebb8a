// Shape descriptors of metaball particles (Sec. 3: sphericity, nominal
// diameter, projected-area diameter, Corey shape factor) by quadrature.  A
// thread walks one column of a particle's grid (a fixed (x, y), all z), so
// the field of a column's cells and the per-column results (any solid cell,
// its extent along the column) stay in registers; a block sums its threads'
// moments with shuffles and adds them to the particle's FP64 accumulators.
// The principal axes come from a cyclic Jacobi diagonalisation of the 3x3
// second moments, one thread per particle.
#include <cmath>

#include "mi_internal.cuh"
#include "mi_shape.h"

namespace mi {
namespace {

constexpr int SH_THREADS = 256;
constexpr int SH_MAX_BALLS = 4096;  // balls of one particle staged in shared memory (64 KB)
constexpr unsigned SH_FULL = 0xffffffffu;

struct ShapeLaunch {
  int np;
  const int* ball_off;
  const float* balls;
  const float* grid_r;
  const int* grid_n;
  float h, eps;
  int words;                 // bitmap words per particle
  unsigned long long* cnt;   // solid cells per particle
  double* acc;               // per particle: band sum, m1 (3), m2 (xx xy xz yy yz zz)
  int* ext;                  // per particle: ordered-int min u (3), max u (3)
  float* frame;              // per particle: centroid (3), axes rows (9)
  unsigned* bits;            // per particle: column bitmap of grid 2
  double* out;
  float* axes;
};

// cell centre -lo + (i + 1/2) h with single FP32 roundings
__device__ __forceinline__ float sh_coord(float lo, int i, float h) {
  return __fadd_rn(lo, __fmul_rn(__fadd_rn((float)i, 0.5f), h));
}

// f at (x, y, z): differences, squares, (d0^2 + d1^2) + d2^2 and one IEEE
// division per ball, each a single FP32 rounding, balls in order
__device__ __forceinline__ float sh_field(const float4* B, int nb, float x, float y, float z) {
  float f = 0.f;
  for (int j = 0; j < nb; ++j) {
    const float4 b = B[j];
    const float d0 = __fsub_rn(x, b.x), d1 = __fsub_rn(y, b.y), d2 = __fsub_rn(z, b.z);
    const float r2 = __fadd_rn(__fadd_rn(__fmul_rn(d0, d0), __fmul_rn(d1, d1)), __fmul_rn(d2, d2));
    f = __fadd_rn(f, __fdiv_rn(b.w, r2));
  }
  return f;
}

__device__ __forceinline__ float sh_gradnorm(const float4* B, int nb, float x, float y, float z) {
  float gx = 0.f, gy = 0.f, gz = 0.f;
  for (int j = 0; j < nb; ++j) {
    const float4 b = B[j];
    const float d0 = x - b.x, d1 = y - b.y, d2 = z - b.z;
    const float r2 = d0 * d0 + d1 * d1 + d2 * d2;
    const float s = -2.0f * b.w / (r2 * r2);
    gx += s * d0;
    gy += s * d1;
    gz += s * d2;
  }
  return sqrtf(gx * gx + gy * gy + gz * gz);
}

__device__ __forceinline__ int sh_key(float v) {
  const int i = __float_as_int(v);
  return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float sh_unkey(int k) { return __int_as_float(k >= 0 ? k : k ^ 0x7fffffff); }

__global__ void k_shape_clear(ShapeLaunch S) {
  const int p = blockIdx.y;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < S.words; i += gridDim.x * blockDim.x)
    S.bits[(size_t)p * S.words + i] = 0u;
  if (blockIdx.x == 0 && threadIdx.x < 10) S.acc[10 * p + threadIdx.x] = 0.0;
  if (blockIdx.x == 0 && threadIdx.x == 10) S.cnt[p] = 0ull;
  if (blockIdx.x == 0 && threadIdx.x >= 16 && threadIdx.x < 22) {
    const int a = threadIdx.x - 16;
    S.ext[6 * p + a] = a < 3 ? sh_key(INFINITY) : sh_key(-INFINITY);
  }
}

// block sum of v added to *dst (FP64)
__device__ __forceinline__ void sh_add(float v, double* dst, float* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(SH_FULL, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.f;
    for (int i = 0; i < SH_THREADS / 32; ++i) s += red[i];
    atomicAdd(dst, (double)s);
  }
}

// grid 1: solid cells, their first and second moments, the surface band
__global__ void __launch_bounds__(SH_THREADS) k_shape_pass1(ShapeLaunch S) {
  extern __shared__ float4 sb[];
  __shared__ float red[SH_THREADS / 32];
  const int p = blockIdx.y;
  const int b0 = S.ball_off[p], nb = S.ball_off[p + 1] - b0;
  if (nb < 1 || nb > SH_MAX_BALLS) return;  // no solid cell counted: NaN descriptors
  for (int j = threadIdx.x; j < nb; j += SH_THREADS)
    sb[j] = make_float4(S.balls[4 * (b0 + j)], S.balls[4 * (b0 + j) + 1], S.balls[4 * (b0 + j) + 2],
                        S.balls[4 * (b0 + j) + 3]);
  __syncthreads();
  const int n = S.grid_n[p];
  const float lo = -S.grid_r[p], h = S.h;
  unsigned cnt = 0;
  float m[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, band = 0.f;
  for (long long col = (long long)blockIdx.x * SH_THREADS + threadIdx.x; col < (long long)n * n;
       col += (long long)gridDim.x * SH_THREADS) {
    const int ix = (int)(col % n), iy = (int)(col / n);
    const float x = sh_coord(lo, ix, h), y = sh_coord(lo, iy, h);
    for (int iz = 0; iz < n; ++iz) {
      const float z = sh_coord(lo, iz, h);
      const float f = sh_field(sb, nb, x, y, z);
      if (f >= 1.0f) {
        ++cnt;
        m[0] += x;
        m[1] += y;
        m[2] += z;
        m[3] += x * x;
        m[4] += x * y;
        m[5] += x * z;
        m[6] += y * y;
        m[7] += y * z;
        m[8] += z * z;
      }
      if (fabsf(__fsub_rn(f, 1.0f)) < S.eps) band += sh_gradnorm(sb, nb, x, y, z);
    }
  }
  unsigned c = cnt;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(SH_FULL, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(S.cnt + p, (unsigned long long)c);
  sh_add(band, S.acc + 10 * p, red);
  for (int a = 0; a < 9; ++a) sh_add(m[a], S.acc + 10 * p + 1 + a, red);
}

// principal axes by cyclic Jacobi rotations of the centred second moments
__global__ void k_shape_axes(ShapeLaunch S) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= S.np) return;
  const double N = (double)S.cnt[p];
  const double* A = S.acc + 10 * p;
  float* fr = S.frame + 12 * p;
  if (N <= 0.0) {
    for (int i = 0; i < 12; ++i) fr[i] = 0.f;
    return;
  }
  const double c[3] = {A[1] / N, A[2] / N, A[3] / N};
  double M[3][3] = {{A[4] / N - c[0] * c[0], A[5] / N - c[0] * c[1], A[6] / N - c[0] * c[2]},
                    {0.0, A[7] / N - c[1] * c[1], A[8] / N - c[1] * c[2]},
                    {0.0, 0.0, A[9] / N - c[2] * c[2]}};
  M[1][0] = M[0][1];
  M[2][0] = M[0][2];
  M[2][1] = M[1][2];
  double V[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  for (int sweep = 0; sweep < 50; ++sweep) {
    const double off = M[0][1] * M[0][1] + M[0][2] * M[0][2] + M[1][2] * M[1][2];
    if (off <= 1e-30 * (M[0][0] * M[0][0] + M[1][1] * M[1][1] + M[2][2] * M[2][2])) break;
    for (int pq = 0; pq < 3; ++pq) {
      const int a = pq == 2 ? 1 : 0, b = pq == 0 ? 1 : 2;
      if (M[a][b] == 0.0) continue;
      const double th = (M[b][b] - M[a][a]) / (2.0 * M[a][b]);
      const double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
      const double cs = 1.0 / sqrt(t * t + 1.0), sn = t * cs;
      for (int k = 0; k < 3; ++k) {  // M <- J^T M J, V <- V J
        const double mka = M[k][a], mkb = M[k][b];
        M[k][a] = cs * mka - sn * mkb;
        M[k][b] = sn * mka + cs * mkb;
      }
      for (int k = 0; k < 3; ++k) {
        const double mak = M[a][k], mbk = M[b][k];
        M[a][k] = cs * mak - sn * mbk;
        M[b][k] = sn * mak + cs * mbk;
      }
      for (int k = 0; k < 3; ++k) {
        const double vka = V[k][a], vkb = V[k][b];
        V[k][a] = cs * vka - sn * vkb;
        V[k][b] = sn * vka + cs * vkb;
      }
    }
  }
  // eigenvalues descending: longest axis first
  int ord[3] = {0, 1, 2};
  for (int i = 0; i < 3; ++i)
    for (int j = i + 1; j < 3; ++j)
      if (M[ord[j]][ord[j]] > M[ord[i]][ord[i]]) {
        const int t = ord[i];
        ord[i] = ord[j];
        ord[j] = t;
      }
  for (int a = 0; a < 3; ++a) fr[a] = (float)c[a];
  for (int r = 0; r < 3; ++r)
    for (int k = 0; k < 3; ++k) fr[3 + 3 * r + k] = (float)V[k][ord[r]];  // row r = axis r
}

// grid 2 along the axes: extents and the columns along the shortest axis
__global__ void __launch_bounds__(SH_THREADS) k_shape_pass2(ShapeLaunch S) {
  extern __shared__ float4 sb[];
  const int p = blockIdx.y;
  const int b0 = S.ball_off[p], nb = S.ball_off[p + 1] - b0;
  if (S.cnt[p] == 0 || nb > SH_MAX_BALLS) return;
  for (int j = threadIdx.x; j < nb; j += SH_THREADS)
    sb[j] = make_float4(S.balls[4 * (b0 + j)], S.balls[4 * (b0 + j) + 1], S.balls[4 * (b0 + j) + 2],
                        S.balls[4 * (b0 + j) + 3]);
  __syncthreads();
  const float* fr = S.frame + 12 * p;
  const float cx = fr[0], cy = fr[1], cz = fr[2];
  const float* E = fr + 3;  // rows: long, intermediate, short axes
  const int n2 = S.grid_n[p] + 4;
  const float h = S.h, lo = -(S.grid_r[p] + 2.0f * h);
  float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (long long col = (long long)blockIdx.x * SH_THREADS + threadIdx.x; col < (long long)n2 * n2;
       col += (long long)gridDim.x * SH_THREADS) {
    const int i1 = (int)(col % n2), i2 = (int)(col / n2);
    const float u1 = sh_coord(lo, i1, h), u2 = sh_coord(lo, i2, h);
    const float px = cx + u1 * E[0] + u2 * E[3], py = cy + u1 * E[1] + u2 * E[4], pz = cz + u1 * E[2] + u2 * E[5];
    bool any = false;
    for (int i3 = 0; i3 < n2; ++i3) {
      const float u3 = sh_coord(lo, i3, h);
      if (sh_field(sb, nb, px + u3 * E[6], py + u3 * E[7], pz + u3 * E[8]) >= 1.0f) {
        any = true;
        mn[2] = fminf(mn[2], u3);
        mx[2] = fmaxf(mx[2], u3);
      }
    }
    if (any) {
      mn[0] = fminf(mn[0], u1);
      mx[0] = fmaxf(mx[0], u1);
      mn[1] = fminf(mn[1], u2);
      mx[1] = fmaxf(mx[1], u2);
      const long long bit = col;
      atomicOr(S.bits + (size_t)p * S.words + (bit >> 5), 1u << (bit & 31));
    }
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      mn[a] = fminf(mn[a], __shfl_xor_sync(SH_FULL, mn[a], o));
      mx[a] = fmaxf(mx[a], __shfl_xor_sync(SH_FULL, mx[a], o));
    }
  }
  if ((threadIdx.x & 31) == 0) {
    for (int a = 0; a < 3; ++a) {
      if (mn[a] <= mx[a]) {
        atomicMin(S.ext + 6 * p + a, sh_key(mn[a]));
        atomicMax(S.ext + 6 * p + 3 + a, sh_key(mx[a]));
      }
    }
  }
}

__global__ void k_shape_final(ShapeLaunch S) {
  __shared__ unsigned red[SH_THREADS];
  const int p = blockIdx.x;
  unsigned c = 0;
  for (int i = threadIdx.x; i < S.words; i += SH_THREADS) c += __popc(S.bits[(size_t)p * S.words + i]);
  red[threadIdx.x] = c;
  __syncthreads();
  for (int s = SH_THREADS / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  double* o = S.out + (size_t)MI_SHAPE_FIELDS * p;
  const double h = S.h, dv = h * h * h;
  const unsigned long long N = S.cnt[p];
  if (N == 0) {
    for (int i = 0; i < MI_SHAPE_FIELDS; ++i) o[i] = NAN;
    o[MI_SHAPE_CELLS] = 0.0;
    return;
  }
  const double V = (double)N * dv;
  const double Sa = S.acc[10 * p] * dv / (2.0 * (double)S.eps);
  double L[3];
  for (int a = 0; a < 3; ++a)
    L[a] = (double)sh_unkey(S.ext[6 * p + 3 + a]) - (double)sh_unkey(S.ext[6 * p + a]) + h;
  const double Ap = (double)red[0] * h * h;
  const double dn = cbrt(6.0 * V / 3.14159265358979323846);
  o[MI_SHAPE_VOLUME] = V;
  o[MI_SHAPE_SURFACE] = Sa;
  o[MI_SHAPE_L_LONG] = L[0];
  o[MI_SHAPE_L_INT] = L[1];
  o[MI_SHAPE_L_SHORT] = L[2];
  o[MI_SHAPE_PROJECTED_AREA] = Ap;
  o[MI_SHAPE_SPHERICITY] = 3.14159265358979323846 * dn * dn / Sa;
  o[MI_SHAPE_D_N] = dn;
  o[MI_SHAPE_D_S] = sqrt(4.0 * Ap / 3.14159265358979323846);
  o[MI_SHAPE_CSF] = L[2] / sqrt(L[1] * L[0]);
  o[MI_SHAPE_CELLS] = (double)N;
  if (S.axes)
    for (int i = 0; i < 9; ++i) S.axes[9 * p + i] = S.frame[12 * p + 3 + i];
}

inline size_t sh_align(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace
}  // namespace mi

extern "C" size_t mi_shape_scratch_bytes(int n_particles, int max_n) {
  using namespace mi;
  if (n_particles < 1 || max_n < 1) return 0;
  const size_t n2 = (size_t)max_n + 4, words = (n2 * n2 + 31) / 32;
  return sh_align(sizeof(unsigned long long) * n_particles) + sh_align(sizeof(double) * 10 * n_particles) +
         sh_align(sizeof(int) * 6 * n_particles) + sh_align(sizeof(float) * 12 * n_particles) +
         sh_align(sizeof(unsigned) * words * n_particles);
}

extern "C" mi_status mi_shape_descriptors(int n_particles, const int* ball_off, const float* balls,
                                          const float* grid_r, const int* grid_n, int max_n, float h, float eps,
                                          double* out, float* axes, void* scratch, void* stream) {
  using namespace mi;
  if (n_particles < 0 || max_n < 1 || !(h > 0.f) || !(eps > 0.f && eps < 1.f)) return MI_EINVAL;
  if (n_particles == 0) return MI_OK;
  if (!ball_off || !balls || !grid_r || !grid_n || !out || !scratch) return MI_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t n2 = (size_t)max_n + 4, words = (n2 * n2 + 31) / 32;
  unsigned char* sp = static_cast<unsigned char*>(scratch);
  ShapeLaunch S;
  S.np = n_particles;
  S.ball_off = ball_off;
  S.balls = balls;
  S.grid_r = grid_r;
  S.grid_n = grid_n;
  S.h = h;
  S.eps = eps;
  S.words = (int)words;
  S.cnt = reinterpret_cast<unsigned long long*>(sp);
  sp += sh_align(sizeof(unsigned long long) * n_particles);
  S.acc = reinterpret_cast<double*>(sp);
  sp += sh_align(sizeof(double) * 10 * n_particles);
  S.ext = reinterpret_cast<int*>(sp);
  sp += sh_align(sizeof(int) * 6 * n_particles);
  S.frame = reinterpret_cast<float*>(sp);
  sp += sh_align(sizeof(float) * 12 * n_particles);
  S.bits = reinterpret_cast<unsigned*>(sp);
  S.out = out;
  S.axes = axes;
  const size_t smem = sizeof(float4) * (size_t)SH_MAX_BALLS;
  if (cudaFuncSetAttribute(k_shape_pass1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      cudaFuncSetAttribute(k_shape_pass2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return MI_ECUDA;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return MI_ECUDA;
  const long long cols1 = (long long)max_n * max_n, cols2 = (long long)n2 * n2;
  long long bx1 = (cols1 + SH_THREADS - 1) / SH_THREADS, bx2 = (cols2 + SH_THREADS - 1) / SH_THREADS;
  const long long cap = (long long)sms * 4;
  if (bx1 > cap) bx1 = cap;
  if (bx2 > cap) bx2 = cap;
  k_shape_clear<<<dim3((unsigned)((words + 255) / 256 + 1), n_particles), 256, 0, s>>>(S);
  k_shape_pass1<<<dim3((unsigned)bx1, n_particles), SH_THREADS, smem, s>>>(S);
  k_shape_axes<<<(n_particles + 127) / 128, 128, 0, s>>>(S);
  k_shape_pass2<<<dim3((unsigned)bx2, n_particles), SH_THREADS, smem, s>>>(S);
  k_shape_final<<<n_particles, SH_THREADS, 0, s>>>(S);
  return cudaGetLastError() == cudaSuccess ? MI_OK : MI_ECUDA;
}
