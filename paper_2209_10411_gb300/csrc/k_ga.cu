// Genetic Algorithm capture of the principal outer contour (Sec. 2.2,
// Algorithm 1).  One generation: the pairing keys and their ranks (the random
// pairing); the mutation draws (a thread per gene, the mutating genes
// appended to a list) and the new genes (a warp per listed gene: the convex-
// hull test of a candidate point spreads the facet planes over the lanes);
// the crossover (a thread per gene pair); the children's fitness (a CTA per
// individual, threads over hull points, fixed-order block sum); and the
// selection (a warp per candidate, its rank by counting over parents and
// children).  Random numbers come from a counter-based SplitMix64, so every
// draw is a function of (seed, generation, individual, gene, slot) and the
// run does not depend on the launch shapes.
#include <cmath>

#include "mi_ga.h"
#include "mi_internal.cuh"

namespace mi {
namespace {

constexpr unsigned GA_INIT_GEN = 0xFFFFFFFFu;
constexpr int GA_SLOT_MUTATE = 0, GA_SLOT_K = 1, GA_SLOT_KEY = 2;
constexpr int GA_TRIES_MUTATE = 8, GA_TRIES_INIT = 64;
constexpr int GA_FIT_THREADS = 256;

// SplitMix64 output for state x: the golden-gamma step, two xor-shift-multiply
// rounds and a final xor-shift (constants of the published generator).
__host__ __device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
  unsigned long long z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ unsigned long long ga_draw(unsigned long long seed, unsigned long long gen,
                                                      unsigned long long ind, int gene, int slot) {
  unsigned long long h = splitmix64(seed);
  h = splitmix64(h ^ gen);
  h = splitmix64(h ^ ind);
  return splitmix64(h ^ ((unsigned long long)gene * 256ull + (unsigned long long)slot));
}

// top 24 bits times 2^-24: exact in FP32
__device__ __forceinline__ float ga_uniform(unsigned long long seed, unsigned long long gen, unsigned long long ind,
                                            int gene, int slot) {
  return (float)(unsigned)(ga_draw(seed, gen, ind, gene, slot) >> 40) * 5.9604644775390625e-8f;
}

// lo + u (hi - lo), single FP32 roundings
__device__ __forceinline__ float ga_lerp(float lo, float hi, float u) {
  return __fadd_rn(lo, __fmul_rn(u, __fsub_rn(hi, lo)));
}

struct GaLaunch {
  int n_ind, n_genes, m, n_planes;
  const float* hull;
  const float* planes;
  float lo[3], hi[3], klo, khi;
  float c_m;
  int p;  // crossover point
  unsigned long long seed;
};

// outside the convex hull: n . p > d for some facet plane (FP32, single
// roundings, left to right), the planes spread over the lanes of a warp
// (every lane passes the same point)
__device__ __forceinline__ bool ga_outside_warp(const float* planes, int n_planes, float x, float y, float z,
                                                int lane) {
  bool out = false;
  for (int p = lane; p < n_planes && !out; p += 32) {
    const float* P = planes + 4 * p;
    const float s = __fadd_rn(__fadd_rn(__fmul_rn(P[0], x), __fmul_rn(P[1], y)), __fmul_rn(P[2], z));
    out = s > P[3];
  }
  return __any_sync(0xffffffffu, out);
}

// a new gene inside the hull for (gen, ind, gene) by one warp; false after
// `tries` rejections
__device__ __forceinline__ bool ga_new_gene(const GaLaunch& G, unsigned long long gen, int ind, int gene, int tries,
                                            int lane, float4& out) {
  for (int t = 0; t < tries; ++t) {
    const float x = ga_lerp(G.lo[0], G.hi[0], ga_uniform(G.seed, gen, ind, gene, 3 + 3 * t));
    const float y = ga_lerp(G.lo[1], G.hi[1], ga_uniform(G.seed, gen, ind, gene, 3 + 3 * t + 1));
    const float z = ga_lerp(G.lo[2], G.hi[2], ga_uniform(G.seed, gen, ind, gene, 3 + 3 * t + 2));
    if (!ga_outside_warp(G.planes, G.n_planes, x, y, z, lane)) {
      out = make_float4(x, y, z, ga_lerp(G.klo, G.khi, ga_uniform(G.seed, gen, ind, gene, GA_SLOT_K)));
      return true;
    }
  }
  return false;
}

// one warp per gene of the initial population
__global__ void k_ga_init(GaLaunch G, float4* pop) {
  const long long e = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (e >= (long long)G.n_ind * G.n_genes) return;
  const int ind = (int)(e / G.n_genes), gene = (int)(e - (long long)ind * G.n_genes);
  float4 v;
  if (!ga_new_gene(G, GA_INIT_GEN, ind, gene, GA_TRIES_INIT, lane, v)) {
    v = make_float4(__fmul_rn(0.5f, __fadd_rn(G.lo[0], G.hi[0])), __fmul_rn(0.5f, __fadd_rn(G.lo[1], G.hi[1])),
                    __fmul_rn(0.5f, __fadd_rn(G.lo[2], G.hi[2])),
                    ga_lerp(G.klo, G.khi, ga_uniform(G.seed, GA_INIT_GEN, ind, gene, GA_SLOT_K)));
  }
  if (lane == 0) pop[e] = v;
}

// F = sum_i (f_i - 1)^2 of one individual per CTA (fixed-order block sum)
__global__ void __launch_bounds__(GA_FIT_THREADS) k_ga_fitness(GaLaunch G, const float4* pop, float* fit) {
  extern __shared__ float4 genes[];
  __shared__ float red[GA_FIT_THREADS];
  const int ind = blockIdx.x, t = threadIdx.x;
  for (int g = t; g < G.n_genes; g += GA_FIT_THREADS) genes[g] = pop[(long long)ind * G.n_genes + g];
  __syncthreads();
  float part = 0.f;
  for (int i = t; i < G.m; i += GA_FIT_THREADS) {
    const float x = G.hull[3 * i], y = G.hull[3 * i + 1], z = G.hull[3 * i + 2];
    float f = 0.f;
    for (int g = 0; g < G.n_genes; ++g) {
      const float4 b = genes[g];
      const float dx = x - b.x, dy = y - b.y, dz = z - b.z;
      f += b.w * __fdividef(1.0f, dx * dx + dy * dy + dz * dz);
    }
    part += (f - 1.0f) * (f - 1.0f);
  }
  red[t] = part;
  __syncthreads();
  for (int s = GA_FIT_THREADS / 2; s > 0; s >>= 1) {
    if (t < s) red[t] += red[t + s];
    __syncthreads();
  }
  if (t == 0) fit[ind] = red[0];
}

__global__ void k_ga_keys(GaLaunch G, unsigned gen, unsigned long long* keys) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < G.n_ind) keys[i] = ga_draw(G.seed, gen, (unsigned long long)i, 0, GA_SLOT_KEY);
}

// perm[rank of key i] = i, ranks ascending with ties to the lower index; a
// warp per key, its lanes counting over strided keys
__global__ void k_ga_perm(GaLaunch G, const unsigned long long* keys, int* perm) {
  const int i = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (i >= G.n_ind) return;
  const unsigned long long ki = keys[i];
  int r = 0;
  for (int j = lane; j < G.n_ind; j += 32) {
    const unsigned long long kj = keys[j];
    r += (kj < ki) || (kj == ki && j < i);
  }
  r = __reduce_add_sync(0xffffffffu, r);
  if (lane == 0) perm[r] = i;
}

// the genes whose mutation draw falls below c_m, appended to a list
__global__ void k_ga_mutflags(GaLaunch G, unsigned gen, int* list, int* count) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)G.n_ind * G.n_genes) return;
  const int ind = (int)(e / G.n_genes), gene = (int)(e - (long long)ind * G.n_genes);
  if (ga_uniform(G.seed, gen, ind, gene, GA_SLOT_MUTATE) < G.c_m) list[atomicAdd(count, 1)] = (int)e;
}

// a new gene for every listed gene, one warp each (the list order does not
// matter: every gene's draws are its own)
__global__ void k_ga_mutate(GaLaunch G, unsigned gen, const int* list, const int* count, float4* mut) {
  const int lane = threadIdx.x & 31;
  const int n = *count;
  for (long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < n;
       w += ((long long)gridDim.x * blockDim.x) >> 5) {
    const int e = list[w];
    const int ind = e / G.n_genes, gene = e - ind * G.n_genes;
    float4 v;
    if (ga_new_gene(G, gen, ind, gene, GA_TRIES_MUTATE, lane, v) && lane == 0) mut[e] = v;
  }
}

// children of the pairs (perm[2q], perm[2q+1]) of the mutated individuals, one
// thread per (pair, gene)
__global__ void k_ga_crossover(GaLaunch G, const float4* mut, const int* perm, float4* off) {
  const int npair = (G.n_ind + 1) / 2;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)npair * G.n_genes) return;
  const int q = (int)(e / G.n_genes), g = (int)(e - (long long)q * G.n_genes);
  const int a = perm[2 * q];
  const float4 ma = mut[(long long)a * G.n_genes + g];
  if (2 * q + 1 >= G.n_ind) {  // odd last individual: copied
    off[(long long)a * G.n_genes + g] = ma;
    return;
  }
  const int b = perm[2 * q + 1];
  const float4 mb = mut[(long long)b * G.n_genes + g];
  off[(long long)a * G.n_genes + g] = g < G.p ? ma : mb;
  off[(long long)b * G.n_genes + g] = g < G.p ? mb : ma;
}

// the n_ind fittest of parents (0..n_ind-1) and children (n_ind..), by
// counting: a warp per candidate, its lanes over strided candidates
__global__ void k_ga_select(GaLaunch G, const float4* pop, const float* fit, const float4* off, const float* fit_off,
                            float4* npop, float* nfit) {
  const int n2 = 2 * G.n_ind;
  const int c = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (c >= n2) return;
  auto val = [&](int d) {
    const float v = d < G.n_ind ? fit[d] : fit_off[d - G.n_ind];
    return isnan(v) ? INFINITY : v;
  };
  const float fc = val(c);
  int r = 0;
  for (int d = lane; d < n2; d += 32) {
    const float fd = val(d);
    r += (fd < fc) || (fd == fc && d < c);
  }
  r = __reduce_add_sync(0xffffffffu, r);
  if (r >= G.n_ind) return;
  const float4* src = c < G.n_ind ? pop + (long long)c * G.n_genes : off + (long long)(c - G.n_ind) * G.n_genes;
  for (int g = lane; g < G.n_genes; g += 32) npop[(long long)r * G.n_genes + g] = src[g];
  if (lane == 0) nfit[r] = fc;
}

inline size_t align256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace
}  // namespace mi

extern "C" size_t mi_ga_scratch_bytes(int n_ind, int n_genes) {
  using namespace mi;
  if (n_ind < 1 || n_genes < 1) return 0;
  const size_t popb = align256(sizeof(float4) * (size_t)n_ind * n_genes);
  return 3 * popb + 3 * align256(sizeof(float) * n_ind) + align256(sizeof(unsigned long long) * n_ind) +
         align256(sizeof(int) * n_ind) + align256(sizeof(int) * (size_t)n_ind * n_genes) + 256;
}

extern "C" mi_status mi_ga_run(int n_ind, int n_genes, const float* hull, int m, const float* planes, int n_planes,
                               const float* bbox, const float* krange, float c_m, float c_c, unsigned long long seed,
                               int generations, int init, float* pop, float* fit, float* offspring,
                               float* fit_offspring, void* scratch, void* stream) {
  using namespace mi;
  if (n_ind < 2 || n_genes < 1 || m < 1 || n_planes < 1 || generations < 0 || !(c_m >= 0.f && c_m <= 1.f) ||
      !(c_c >= 0.f && c_c <= 1.f) || !hull || !planes || !bbox || !krange || !pop || !fit || !scratch)
    return MI_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  GaLaunch G;
  G.n_ind = n_ind;
  G.n_genes = n_genes;
  G.m = m;
  G.n_planes = n_planes;
  G.hull = hull;
  G.planes = planes;
  for (int a = 0; a < 3; ++a) {
    G.lo[a] = bbox[a];
    G.hi[a] = bbox[3 + a];
  }
  G.klo = krange[0];
  G.khi = krange[1];
  G.c_m = c_m;
  G.p = (int)std::floor((double)c_c * n_genes);
  G.seed = seed;
  // scratch: a second population, the children, three fitness arrays, keys, ranks
  unsigned char* sp = static_cast<unsigned char*>(scratch);
  const size_t popb = align256(sizeof(float4) * (size_t)n_ind * n_genes);
  float4* popB = reinterpret_cast<float4*>(sp);
  float4* off = reinterpret_cast<float4*>(sp + popb);
  float* fitB = reinterpret_cast<float*>(sp + 2 * popb);
  float* fitO = reinterpret_cast<float*>(sp + 2 * popb + align256(sizeof(float) * n_ind));
  unsigned long long* keys =
      reinterpret_cast<unsigned long long*>(sp + 2 * popb + 3 * align256(sizeof(float) * n_ind));
  int* perm = reinterpret_cast<int*>(sp + 2 * popb + 3 * align256(sizeof(float) * n_ind) +
                                     align256(sizeof(unsigned long long) * n_ind));
  unsigned char* sp2 = reinterpret_cast<unsigned char*>(perm) + align256(sizeof(int) * n_ind);
  float4* mut = reinterpret_cast<float4*>(sp2);
  int* mlist = reinterpret_cast<int*>(sp2 + popb);
  int* mcount = reinterpret_cast<int*>(sp2 + popb + align256(sizeof(int) * (size_t)n_ind * n_genes));
  float4* cur = reinterpret_cast<float4*>(pop);
  float4* nxt = popB;
  float* fcur = fit;
  float* fnxt = fitB;
  const long long ng = (long long)n_ind * n_genes;
  const size_t gsm = sizeof(float4) * (size_t)n_genes;
  if (gsm > 48 * 1024 &&
      cudaFuncSetAttribute(k_ga_fitness, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsm) != cudaSuccess)
    return MI_ECUDA;
  if (init) k_ga_init<<<(unsigned)((ng * 32 + 255) / 256), 256, 0, s>>>(G, cur);
  k_ga_fitness<<<n_ind, GA_FIT_THREADS, gsm, s>>>(G, cur, fcur);
  const long long npair_genes = (long long)((n_ind + 1) / 2) * n_genes;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return MI_ECUDA;
  const unsigned mut_blocks = (unsigned)(sms > 0 ? 8 * sms : 1024);  // 8 warps per block, grid-strided over the list
  for (int gen = 0; gen < generations; ++gen) {
    k_ga_keys<<<(n_ind + 255) / 256, 256, 0, s>>>(G, (unsigned)gen, keys);
    k_ga_perm<<<(unsigned)(((long long)n_ind * 32 + 255) / 256), 256, 0, s>>>(G, keys, perm);
    if (cudaMemcpyAsync(mut, cur, sizeof(float4) * ng, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(mcount, 0, sizeof(int), s) != cudaSuccess)
      return MI_ECUDA;
    k_ga_mutflags<<<(unsigned)((ng + 255) / 256), 256, 0, s>>>(G, (unsigned)gen, mlist, mcount);
    k_ga_mutate<<<mut_blocks, 256, 0, s>>>(G, (unsigned)gen, mlist, mcount, mut);
    k_ga_crossover<<<(unsigned)((npair_genes + 255) / 256), 256, 0, s>>>(G, mut, perm, off);
    k_ga_fitness<<<n_ind, GA_FIT_THREADS, gsm, s>>>(G, off, fitO);
    if (gen == generations - 1 && offspring) {
      if (cudaMemcpyAsync(offspring, off, sizeof(float4) * ng, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return MI_ECUDA;
      if (fit_offspring &&
          cudaMemcpyAsync(fit_offspring, fitO, sizeof(float) * n_ind, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return MI_ECUDA;
    }
    k_ga_select<<<(unsigned)(((long long)2 * n_ind * 32 + 255) / 256), 256, 0, s>>>(G, cur, fcur, off, fitO, nxt, fnxt);
    float4* t4 = cur;
    cur = nxt;
    nxt = t4;
    float* tf = fcur;
    fcur = fnxt;
    fnxt = tf;
  }
  if (cur != reinterpret_cast<float4*>(pop)) {
    if (cudaMemcpyAsync(pop, cur, sizeof(float4) * ng, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(fit, fcur, sizeof(float) * n_ind, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return MI_ECUDA;
  }
  return cudaGetLastError() == cudaSuccess ? MI_OK : MI_ECUDA;
}
