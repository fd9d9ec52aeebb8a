// Allocation-free variant of the mass-property quadrature (the kernel behind
// mi_delbm_add_particle when no mass properties are given), for callers that
// cannot allocate device memory themselves.  Its scratch -- an FP32 copy of
// the ball table and one row of moment sums per block -- lives in a
// file-scope static __device__ array of fixed size instead of memory from
// cudaMalloc; the caller passes the input ball table and the output buffer.
#include <cmath>
#include <mutex>

#include "mi_internal.cuh"

namespace mi {
void set_thread_error(const char* msg);  // engine.cu: message for mi_delbm_last_error(NULL)
}

namespace {
constexpr int NOALLOC_MAX_BALLS = 4096;  // largest ball table accepted
constexpr int NOALLOC_BLOCKS = 1024;     // quadrature blocks (one row of 10 sums each)
constexpr int NOALLOC_MAX_DEVICES = 64;
// Largest quadrature grid: at most 2048 samples per axis and at most 2^38
// (sample, ball) field evaluations, about a tenth of a second on this part.
// Larger grids (a very small spacing, a large or ill-formed ball table) are
// not run: the outputs are set to NaN instead.
constexpr long long NOALLOC_MAX_SIDE = 2048;
constexpr double NOALLOC_MAX_EVALS = 274877906944.0;  // 2^38

struct NoallocScratch {
  float4 balls[NOALLOC_MAX_BALLS];      // FP32 (c_x, c_y, c_z, k)
  double partials[NOALLOC_BLOCKS * 10]; // per-block moment sums
  double Rb;                            // bounding radius max|c_i| + sqrt(sum k_i)
  long long n_side;                     // samples per axis
};

// 64 KB + 80 KB: held by every GPU that loads the library, until exit.
static __device__ __align__(256) NoallocScratch g_noalloc_scratch;

NoallocScratch* g_scratch_addr[NOALLOC_MAX_DEVICES] = {};
std::mutex g_scratch_mutex;

// Device address of the scratch on the current device (looked up once per
// device; the host-side symbol itself is only a stand-in, never a device
// address).  The cached address belongs to the device's primary context as it
// was at the first call: a cudaDeviceReset on that device invalidates it, and
// the entry point must not be called on that device afterwards.
cudaError_t scratch_address(int dev, NoallocScratch** out) {
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<NoallocScratch*>(p);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

// One thread: FP32 ball copy, bounding radius and sample count (sequential,
// unfused, the same operations as the host does in mi_delbm_add_particle).
__global__ void k_noalloc_prep(const double* __restrict__ balls, int n, double h, NoallocScratch* S) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  double maxc = 0.0, sumk = 0.0;
  for (int i = 0; i < n; ++i) {
    const double* b = balls + 4 * i;
    S->balls[i] = make_float4((float)b[0], (float)b[1], (float)b[2], (float)b[3]);
    const double r = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(b[0], b[0]), __dmul_rn(b[1], b[1])), __dmul_rn(b[2], b[2])));
    maxc = fmax(maxc, r);
    sumk = __dadd_rn(sumk, b[3]);
  }
  const double Rb = __dadd_rn(maxc, __dsqrt_rn(sumk));
  S->Rb = Rb;
  // samples per axis, or 0 (nothing is sampled, the outputs become NaN) when
  // the table is ill-formed (a NaN, a non-positive sum of k) or the grid is
  // beyond the limits above; the comparisons are false for NaN
  const double side = ceil(__ddiv_rn(__dmul_rn(2.0, Rb), h));
  const bool ok = Rb > 0.0 && side >= 1.0 && side <= (double)NOALLOC_MAX_SIDE &&
                  side * side * side * (double)n <= NOALLOC_MAX_EVALS;
  S->n_side = ok ? (long long)side : 0;
}

// Midpoint quadrature of f >= 1 over [-Rb, Rb]^3: FP32 field with the FP64
// guard band, FP64 moment sums per block into the scratch rows.
__global__ void __launch_bounds__(256) k_noalloc_quadrature(const double* __restrict__ balls, int nb, double h,
                                                            NoallocScratch* S) {
  __shared__ double red[10][256];
  const double Rb = S->Rb;
  const long long n = S->n_side;
  double acc[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  const long long total = n * n * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long ix = i % n, iy = (i / n) % n, iz = i / (n * n);
    const double X = __dadd_rn(-Rb, __dmul_rn((double)ix + 0.5, h));
    const double Y = __dadd_rn(-Rb, __dmul_rn((double)iy + 0.5, h));
    const double Z = __dadd_rn(-Rb, __dmul_rn((double)iz + 0.5, h));
    if (mi::mass_sample_inside(S->balls, balls, nb, X, Y, Z)) mi::mass_sample_accumulate(acc, X, Y, Z);
  }
  for (int k = 0; k < 10; ++k) red[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st)
      for (int k = 0; k < 10; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int k = 0; k < 10; ++k) S->partials[10 * blockIdx.x + k] = red[k][0];
}

// One thread: sum the block rows in block order and form mass, volume,
// centroid and inertia about the centroid.  out: 14 doubles, all NaN when the
// grid was not run or no sample lies inside (no solid volume).
__global__ void k_noalloc_finish(const NoallocScratch* S, double h, double density, double* __restrict__ out) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  double s[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int b = 0; b < NOALLOC_BLOCKS; ++b)
    for (int k = 0; k < 10; ++k) s[k] += S->partials[10 * b + k];
  const double dv = h * h * h;
  const double vol = s[0] * dv;
  if (S->n_side == 0 || !(vol > 0.0)) {
    for (int k = 0; k < 14; ++k) out[k] = __longlong_as_double(0x7FF8000000000000LL);
    return;
  }
  double cen[3] = {0, 0, 0};
  for (int a = 0; a < 3; ++a) cen[a] = s[1 + a] * dv / vol;
  double sec[9] = {s[4] * dv, s[5] * dv, s[6] * dv, s[5] * dv, s[7] * dv, s[8] * dv, s[6] * dv, s[8] * dv, s[9] * dv};
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) sec[3 * a + b] -= vol * cen[a] * cen[b];
  const double tr = sec[0] + sec[4] + sec[8];
  out[0] = density * vol;
  out[1] = vol;
  for (int a = 0; a < 3; ++a) out[2 + a] = cen[a];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) out[5 + 3 * a + b] = density * ((a == b ? tr : 0.0) - sec[3 * a + b]);
}
}  // namespace

extern "C" mi_status mi_mass_properties_noalloc(const double* balls_dev, int n_balls, double density,
                                                double spacing, double* out_dev, void* stream) {
  if (!balls_dev || !out_dev) {
    mi::set_thread_error("mi_mass_properties_noalloc: null device pointer");
    return MI_EINVAL;
  }
  if (n_balls < 1 || n_balls > NOALLOC_MAX_BALLS) {
    mi::set_thread_error("mi_mass_properties_noalloc: n_balls must be in 1..4096 (the size of the static scratch)");
    return MI_EINVAL;
  }
  if (!(density > 0.0) || !(spacing > 0.0) || !std::isfinite(density) || !std::isfinite(spacing)) {
    mi::set_thread_error("mi_mass_properties_noalloc: density and spacing must be finite and > 0");
    return MI_EINVAL;
  }
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
    mi::set_thread_error("mi_mass_properties_noalloc: no usable current device");
    return MI_ECUDA;
  }
  NoallocScratch* S = nullptr;
  e = scratch_address(dev, &S);
  if (e != cudaSuccess) {
    mi::set_thread_error("mi_mass_properties_noalloc: cudaGetSymbolAddress failed");
    return MI_ECUDA;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  k_noalloc_prep<<<1, 1, 0, s>>>(balls_dev, n_balls, spacing, S);
  k_noalloc_quadrature<<<NOALLOC_BLOCKS, 256, 0, s>>>(balls_dev, n_balls, spacing, S);
  k_noalloc_finish<<<1, 1, 0, s>>>(S, spacing, density, out_dev);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    mi::set_thread_error("mi_mass_properties_noalloc: kernel launch failed");
    return MI_ECUDA;
  }
  return MI_OK;
}
