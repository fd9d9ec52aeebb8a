// MLP of the learned Newton guess (64 -> 256 -> 256 -> 4, ReLU): forward,
// backward, MSE loss and AdamW on the GPU.  Every matrix product runs on the
// tensor cores as BF16 x BF16 -> FP32 (mma.sync m16n8k16); parameters,
// activations and gradients live in FP32 and are rounded to BF16 when a tile
// is staged in shared memory, so the network computes with BF16 weights and
// FP32 accumulation while the optimizer keeps FP32 master weights.
#include <cstring>
#include <string>

#include "mi_internal.cuh"

namespace mi {
void set_thread_error(const char* msg);  // engine.cu: message for mi_delbm_last_error(NULL)

namespace {

constexpr int BM = 64, BN = 64, BK = 32, PAD = 8;

struct GemmArgs {
  int M, N, K;
  const unsigned* Mdev;  // when set, the row count is min(M, *Mdev), read on the device
  const float* A;
  int lda, transA;   // op(A) is M x K; A is M x K row-major, or K x M when transA
  const float* B;
  int ldb, transB;   // op(B) is K x N; B is K x N row-major, or N x K when transB
  const float* bias; // N, or nullptr
  const float* mask; // M x N (ldmask): the result is zeroed where mask <= 0, or nullptr
  int ldmask;
  int relu;
  float* C;
  int ldc;
};

// Two consecutive BF16 of a shared-memory row (even column: 4-byte aligned,
// the lower column in the lower half, as the mma fragments want them).
__device__ __forceinline__ unsigned ld32(const __nv_bfloat16* p) { return *reinterpret_cast<const unsigned*>(p); }

__device__ __forceinline__ void mma_bf16(float (&d)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                         unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// C = op(A) op(B) (+ bias) (ReLU) (masked).  Block tile 64 x 64, K step 32,
// 4 warps in 2 x 2, each warp 32 x 32 = 2 x 4 mma tiles of 16 x 8.
__global__ void __launch_bounds__(128) k_gemm(GemmArgs g) {
  __shared__ __nv_bfloat16 As[BM][BK + PAD];  // (m, k)
  __shared__ __nv_bfloat16 Bs[BN][BK + PAD];  // (n, k)
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int gid = lane >> 2, tig = lane & 3;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  if (g.Mdev) {
    const int Md = (int)min((unsigned)g.M, *g.Mdev);
    g.M = Md;
    if (m0 >= Md) return;  // uniform over the block
  }
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  float acc[2][4][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;

  for (int k0 = 0; k0 < g.K; k0 += BK) {
    // stage op(A)[m0:m0+64, k0:k0+32] and op(B)[k0:k0+32, n0:n0+64] as BF16
    for (int e = tid; e < BM * BK; e += 128) {
      int m, k;
      if (g.transA) { m = e % BM; k = e / BM; } else { k = e % BK; m = e / BK; }
      const int gm = m0 + m, gk = k0 + k;
      float v = 0.f;
      if (gm < g.M && gk < g.K) v = g.transA ? g.A[(long long)gk * g.lda + gm] : g.A[(long long)gm * g.lda + gk];
      As[m][k] = __float2bfloat16_rn(v);
    }
    for (int e = tid; e < BN * BK; e += 128) {
      int n, k;
      if (g.transB) { k = e % BK; n = e / BK; } else { n = e % BN; k = e / BN; }
      const int gn = n0 + n, gk = k0 + k;
      float v = 0.f;
      if (gn < g.N && gk < g.K) v = g.transB ? g.B[(long long)gn * g.ldb + gk] : g.B[(long long)gk * g.ldb + gn];
      Bs[n][k] = __float2bfloat16_rn(v);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; kk += 16) {
      unsigned a[2][4], b[4][2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int r = wm + 16 * i + gid;
        a[i][0] = ld32(&As[r][kk + 2 * tig]);
        a[i][1] = ld32(&As[r + 8][kk + 2 * tig]);
        a[i][2] = ld32(&As[r][kk + 2 * tig + 8]);
        a[i][3] = ld32(&As[r + 8][kk + 2 * tig + 8]);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = wn + 8 * j + gid;
        b[j][0] = ld32(&Bs[c][kk + 2 * tig]);
        b[j][1] = ld32(&Bs[c][kk + 2 * tig + 8]);
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], a[i][0], a[i][1], a[i][2], a[i][3], b[j][0], b[j][1]);
    }
    __syncthreads();
  }
  // epilogue
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int row = m0 + wm + 16 * i + gid + (c >= 2 ? 8 : 0);
        const int col = n0 + wn + 8 * j + 2 * tig + (c & 1);
        if (row >= g.M || col >= g.N) continue;
        float v = acc[i][j][c];
        if (g.bias) v += g.bias[col];
        if (g.relu) v = fmaxf(v, 0.f);
        if (g.mask && !(g.mask[(long long)row * g.ldmask + col] > 0.f)) v = 0.f;
        g.C[(long long)row * g.ldc + col] = v;
      }
}

cudaError_t gemm(const GemmArgs& a, cudaStream_t s) {
  dim3 grid((a.N + BN - 1) / BN, (a.M + BM - 1) / BM);
  if (grid.x == 0 || grid.y == 0) return cudaSuccess;
  k_gemm<<<grid, 128, 0, s>>>(a);
  return cudaGetLastError();
}

GemmArgs gemm_args(int M, int N, int K, const float* A, int lda, int tA, const float* B, int ldb, int tB,
                   const float* bias, int relu, const float* mask, int ldm, float* C, int ldc) {
  GemmArgs g;
  g.M = M; g.N = N; g.K = K;
  g.Mdev = nullptr;
  g.A = A; g.lda = lda; g.transA = tA;
  g.B = B; g.ldb = ldb; g.transB = tB;
  g.bias = bias; g.relu = relu; g.mask = mask; g.ldmask = ldm;
  g.C = C; g.ldc = ldc;
  return g;
}

// dY = 2 (Y - T) / n and per-block partial sums of (Y - T)^2 (summed in block order).
__global__ void k_mse(const float* __restrict__ Y, const float* __restrict__ T, int count, float inv_n,
                      float* __restrict__ dY, double* __restrict__ partial) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    const float d = Y[i] - T[i];
    dY[i] = 2.0f * d * inv_n;
    acc += (double)d * d;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void k_loss_finish(const double* partial, int nb, double inv_n, float* loss) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += partial[b];
  *loss = (float)(s * inv_n);
}

// Column sums of an M x N matrix (bias gradients): block (32, 8) covers 32
// columns, the 8 row phases are added in a fixed order (deterministic).
__global__ void k_colsum(const float* __restrict__ D, int M, int N, float* __restrict__ out) {
  __shared__ float red[8][33];
  const int c = blockIdx.x * 32 + threadIdx.x;
  float s = 0.f;
  if (c < N)
    for (int r = threadIdx.y; r < M; r += 8) s += D[(long long)r * N + c];
  red[threadIdx.y][threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.y == 0 && c < N) {
    float t = red[0][threadIdx.x];
    for (int y = 1; y < 8; ++y) t += red[y][threadIdx.x];
    out[c] = t;
  }
}

cudaError_t colsum(const float* D, int M, int N, float* out, cudaStream_t s) {
  k_colsum<<<(N + 31) / 32, dim3(32, 8), 0, s>>>(D, M, N, out);
  return cudaGetLastError();
}

// AdamW (decoupled weight decay) on FP32 master parameters.
__global__ void k_adamw(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                        float* __restrict__ v, int n, float lr, float b1, float b2, float eps, float wd, float c1,
                        float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float mi = b1 * m[i] + (1.f - b1) * g[i];
  const float vi = b2 * v[i] + (1.f - b2) * g[i] * g[i];
  m[i] = mi;
  v[i] = vi;
  const float mh = mi / c1, vh = vi / c2;
  p[i] = p[i] - lr * (mh / (sqrtf(vh) + eps) + wd * p[i]);
}

}  // namespace


}  // namespace mi

using namespace mi;

namespace mi {
// X[r][c] = (X[r][c] - shift[c]) * scale[c]: the training driver's feature
// standardisation and target weighting
__global__ void k_scale_columns(float* __restrict__ X, long long n, int cols, const float* __restrict__ shift,
                                const float* __restrict__ scale) {
  const long long total = n * cols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(e % cols);
    X[e] = (X[e] - shift[c]) * scale[c];
  }
}
}  // namespace mi

extern "C" {

// Parameter block layout (floats): W1 64x256, b1 256, W2 256x256, b2 256, W3 256x4, b3 4.
size_t mi_mlp_param_count(void) { return 64 * 256 + 256 + 256 * 256 + 256 + 256 * 4 + 4; }

static void split(const float* base, const float* P[6]) {
  P[0] = base;
  P[1] = P[0] + 64 * 256;
  P[2] = P[1] + 256;
  P[3] = P[2] + 256 * 256;
  P[4] = P[3] + 256;
  P[5] = P[4] + 256 * 4;
}

mi_status mi_mlp_forward(const float* params, const float* X, int n, float* Y, float* acts, void* stream) {
  if (n < 0 || (n > 0 && (!params || !X || !Y || !acts))) {
    set_thread_error("mi_mlp_forward: null pointer or negative batch");
    return MI_EINVAL;
  }
  if (n == 0) return MI_OK;
  const float* P[6];
  split(params, P);
  cudaStream_t s = (cudaStream_t)stream;
  float* H1 = acts;                    // n x 256, relu(X W1 + b1)
  float* H2 = acts + (size_t)n * 256;  // n x 256, relu(H1 W2 + b2)
  cudaError_t e = gemm(gemm_args(n, 256, 64, X, 64, 0, P[0], 256, 0, P[1], 1, nullptr, 0, H1, 256), s);
  if (e == cudaSuccess) e = gemm(gemm_args(n, 256, 256, H1, 256, 0, P[2], 256, 0, P[3], 1, nullptr, 0, H2, 256), s);
  if (e == cudaSuccess) e = gemm(gemm_args(n, 4, 256, H2, 256, 0, P[4], 4, 0, P[5], 0, nullptr, 0, Y, 4), s);
  if (e != cudaSuccess) {
    set_thread_error("mi_mlp_forward: launch failed");
    return MI_ECUDA;
  }
  return MI_OK;
}

mi_status mi_mlp_mse(const float* Y, const float* T, int n, float* dY, float* loss, double* scratch, void* stream) {
  if (!Y || !T || !dY || !loss || !scratch || n <= 0) {
    set_thread_error("mi_mlp_mse: null pointer or empty batch");
    return MI_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int blocks = 64;
  k_mse<<<blocks, 256, 0, s>>>(Y, T, 4 * n, 1.0f / n, dY, scratch);
  k_loss_finish<<<1, 32, 0, s>>>(scratch, blocks, 1.0 / n, loss);
  if (cudaGetLastError() != cudaSuccess) {
    set_thread_error("mi_mlp_mse: launch failed");
    return MI_ECUDA;
  }
  return MI_OK;
}

mi_status mi_mlp_backward(const float* params, const float* X, const float* acts, const float* dY, int n,
                          float* grads, float* scratch, void* stream) {
  if (!params || !X || !acts || !dY || !grads || !scratch || n <= 0) {
    set_thread_error("mi_mlp_backward: null pointer or empty batch");
    return MI_EINVAL;
  }
  const float* P[6];
  split(params, P);
  float* G[6];
  {
    const float* Gc[6];
    split(grads, Gc);
    for (int i = 0; i < 6; ++i) G[i] = const_cast<float*>(Gc[i]);
  }
  // relu(z) > 0 exactly where z > 0, so the saved activations give the masks.
  const float* H1 = acts;
  const float* H2 = acts + (size_t)n * 256;
  float* dZ2 = scratch;                    // n x 256
  float* dZ1 = scratch + (size_t)n * 256;  // n x 256
  cudaStream_t s = (cudaStream_t)stream;
  // layer 3: dW3 = H2^T dY, db3 = colsum dY
  cudaError_t e = gemm(gemm_args(256, 4, n, H2, 256, 1, dY, 4, 0, nullptr, 0, nullptr, 0, G[4], 4), s);
  if (e == cudaSuccess) e = colsum(dY, n, 4, G[5], s);
  // dZ2 = (dY W3^T) masked by H2 > 0
  if (e == cudaSuccess) e = gemm(gemm_args(n, 256, 4, dY, 4, 0, P[4], 4, 1, nullptr, 0, H2, 256, dZ2, 256), s);
  // layer 2: dW2 = H1^T dZ2, db2 = colsum dZ2
  if (e == cudaSuccess) e = gemm(gemm_args(256, 256, n, H1, 256, 1, dZ2, 256, 0, nullptr, 0, nullptr, 0, G[2], 256), s);
  if (e == cudaSuccess) e = colsum(dZ2, n, 256, G[3], s);
  // dZ1 = (dZ2 W2^T) masked by H1 > 0
  if (e == cudaSuccess) e = gemm(gemm_args(n, 256, 256, dZ2, 256, 0, P[2], 256, 1, nullptr, 0, H1, 256, dZ1, 256), s);
  // layer 1: dW1 = X^T dZ1, db1 = colsum dZ1
  if (e == cudaSuccess) e = gemm(gemm_args(64, 256, n, X, 64, 1, dZ1, 256, 0, nullptr, 0, nullptr, 0, G[0], 256), s);
  if (e == cudaSuccess) e = colsum(dZ1, n, 256, G[1], s);
  if (e != cudaSuccess) {
    set_thread_error("mi_mlp_backward: launch failed");
    return MI_ECUDA;
  }
  return MI_OK;
}

mi_status mi_mlp_adamw(float* params, const float* grads, float* m, float* v, int step, float lr, float beta1,
                       float beta2, float eps, float weight_decay, void* stream) {
  if (!params || !grads || !m || !v || step < 1) {
    set_thread_error("mi_mlp_adamw: null pointer or step < 1");
    return MI_EINVAL;
  }
  const int n = (int)mi_mlp_param_count();
  const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
  k_adamw<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(params, grads, m, v, n, lr, beta1, beta2, eps,
                                                             weight_decay, c1, c2);
  if (cudaGetLastError() != cudaSuccess) {
    set_thread_error("mi_mlp_adamw: launch failed");
    return MI_ECUDA;
  }
  return MI_OK;
}

mi_status mi_mlp_scale_columns(float* X, long long n, int cols, const float* shift, const float* scale, void* stream) {
  if (n < 0 || cols < 1 || (n > 0 && (!X || !shift || !scale))) {
    set_thread_error("mi_mlp_scale_columns: null pointer, n < 0 or cols < 1");
    return MI_EINVAL;
  }
  if (n == 0) return MI_OK;
  mi::k_scale_columns<<<2048, 256, 0, (cudaStream_t)stream>>>(X, n, cols, shift, scale);
  if (cudaGetLastError() != cudaSuccess) {
    set_thread_error("mi_mlp_scale_columns: launch failed");
    return MI_ECUDA;
  }
  return MI_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Fused inference: the whole network for a 64-row tile in one CTA.  The
// parameters are packed once into a BF16 image laid out as the CTA's shared
// memory wants it (weights transposed to (n, k) with padded rows, so that
// every fragment load is one conflict-free 32-bit word); each CTA copies the
// image with 16-byte loads and then loops over row tiles (persistent).
// Layers 1 and 2 run on the tensor cores; the 256 -> 4 output layer is done
// in the epilogue of layer 2 with the same BF16 operands (their products are
// exact in FP32) and FP32 sums, so H2 never leaves registers.
// ---------------------------------------------------------------------------
namespace mi {
namespace {

constexpr int FT_ROWS = 64;                       // rows per tile
constexpr int FW1_LD = 72, FW2_LD = 264;          // padded row lengths (bf16) of W1^T, W2^T
constexpr int FX_LD = 72, FH_LD = 264;            // padded row lengths of the X and H1 tiles
constexpr size_t IMG_W1 = 0;
constexpr size_t IMG_W2 = IMG_W1 + 256 * FW1_LD * 2;       // 36864
constexpr size_t IMG_W3 = IMG_W2 + 256 * FW2_LD * 2;       // 172032: W3^T (4 x 256) as BF16-valued floats
constexpr size_t IMG_B1 = IMG_W3 + 4 * 256 * 4;
constexpr size_t IMG_B2 = IMG_B1 + 256 * 4;
constexpr size_t IMG_B3 = IMG_B2 + 256 * 4;
constexpr size_t IMG_BYTES = IMG_B3 + 16;                  // 178192 (a multiple of 16)
constexpr size_t SM_X = IMG_BYTES;
constexpr size_t SM_H1 = SM_X + FT_ROWS * FX_LD * 2;
constexpr size_t SM_Y = SM_H1 + FT_ROWS * FH_LD * 2;
constexpr size_t SM_BYTES = SM_Y + 8 * FT_ROWS * 4 * 4;    // 229392
static_assert(IMG_BYTES % 16 == 0 && SM_BYTES <= 232448, "fused MLP shared memory layout");

__global__ void k_mlp_pack(const float* __restrict__ p, unsigned char* __restrict__ img) {
  const float* W1 = p;
  const float* b1 = W1 + 64 * 256;
  const float* W2 = b1 + 256;
  const float* b2 = W2 + 256 * 256;
  const float* W3 = b2 + 256;
  const float* b3 = W3 + 256 * 4;
  __nv_bfloat16* w1t = reinterpret_cast<__nv_bfloat16*>(img + IMG_W1);
  __nv_bfloat16* w2t = reinterpret_cast<__nv_bfloat16*>(img + IMG_W2);
  float* w3t = reinterpret_cast<float*>(img + IMG_W3);
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
  for (int e = tid; e < 256 * FW1_LD; e += nt) {
    const int n = e / FW1_LD, k = e % FW1_LD;
    w1t[e] = __float2bfloat16_rn(k < 64 ? W1[k * 256 + n] : 0.f);
  }
  for (int e = tid; e < 256 * FW2_LD; e += nt) {
    const int n = e / FW2_LD, k = e % FW2_LD;
    w2t[e] = __float2bfloat16_rn(k < 256 ? W2[k * 256 + n] : 0.f);
  }
  for (int e = tid; e < 4 * 256; e += nt) {
    const int o = e / 256, c = e % 256;
    w3t[e] = __bfloat162float(__float2bfloat16_rn(W3[c * 4 + o]));
  }
  for (int e = tid; e < 256; e += nt) {
    reinterpret_cast<float*>(img + IMG_B1)[e] = b1[e];
    reinterpret_cast<float*>(img + IMG_B2)[e] = b2[e];
  }
  if (tid < 4) reinterpret_cast<float*>(img + IMG_B3)[tid] = b3[tid];
}

__global__ void __launch_bounds__(256, 1) k_mlp_fused(const uint4* __restrict__ img, const float* __restrict__ X,
                                                      int M, const unsigned* __restrict__ Mdev,
                                                      float* __restrict__ Y) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, gid = lane >> 2, tig = lane & 3;
  if (Mdev) M = min(M, (int)*Mdev);
  const int tiles = (M + FT_ROWS - 1) / FT_ROWS;
  if ((int)blockIdx.x >= tiles) return;
  for (int e = tid; e < (int)(IMG_BYTES / 16); e += 256) reinterpret_cast<uint4*>(sm)[e] = img[e];
  const __nv_bfloat16(*W1t)[FW1_LD] = reinterpret_cast<const __nv_bfloat16(*)[FW1_LD]>(sm + IMG_W1);
  const __nv_bfloat16(*W2t)[FW2_LD] = reinterpret_cast<const __nv_bfloat16(*)[FW2_LD]>(sm + IMG_W2);
  const float* W3t = reinterpret_cast<const float*>(sm + IMG_W3);
  const float* b1 = reinterpret_cast<const float*>(sm + IMG_B1);
  const float* b2 = reinterpret_cast<const float*>(sm + IMG_B2);
  const float* b3 = reinterpret_cast<const float*>(sm + IMG_B3);
  __nv_bfloat16(*Xs)[FX_LD] = reinterpret_cast<__nv_bfloat16(*)[FX_LD]>(sm + SM_X);
  __nv_bfloat16(*H1)[FH_LD] = reinterpret_cast<__nv_bfloat16(*)[FH_LD]>(sm + SM_H1);
  float(*Yp)[FT_ROWS][4] = reinterpret_cast<float(*)[FT_ROWS][4]>(sm + SM_Y);
  const int wn = warp * 32;  // this warp's 32 output columns of layers 1 and 2

  for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
    const int r0 = t * FT_ROWS;
    __syncthreads();  // previous tile's readers of Xs, H1 and Yp are done (and the image is in place)
    for (int e = tid; e < FT_ROWS * 16; e += 256) {
      const int r = e >> 4, c4 = (e & 15) * 4;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (r0 + r < M) v = *reinterpret_cast<const float4*>(X + (size_t)(r0 + r) * 64 + c4);
      Xs[r][c4] = __float2bfloat16_rn(v.x);
      Xs[r][c4 + 1] = __float2bfloat16_rn(v.y);
      Xs[r][c4 + 2] = __float2bfloat16_rn(v.z);
      Xs[r][c4 + 3] = __float2bfloat16_rn(v.w);
    }
    __syncthreads();
    float acc[4][4][4];
    // ---- layer 1: H1 = relu(X W1 + b1), rows 0..63 x columns wn..wn+31 ----
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[i][j][c] = 0.f;
#pragma unroll
    for (int kk = 0; kk < 64; kk += 16) {
      unsigned a[4][4], b[4][2];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int r = 16 * i + gid;
        a[i][0] = ld32(&Xs[r][kk + 2 * tig]);
        a[i][1] = ld32(&Xs[r + 8][kk + 2 * tig]);
        a[i][2] = ld32(&Xs[r][kk + 2 * tig + 8]);
        a[i][3] = ld32(&Xs[r + 8][kk + 2 * tig + 8]);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int n = wn + 8 * j + gid;
        b[j][0] = ld32(&W1t[n][kk + 2 * tig]);
        b[j][1] = ld32(&W1t[n][kk + 2 * tig + 8]);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], a[i][0], a[i][1], a[i][2], a[i][3], b[j][0], b[j][1]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int row = 16 * i + gid + 8 * h, col = wn + 8 * j + 2 * tig;
          const float v0 = fmaxf(acc[i][j][2 * h] + b1[col], 0.f);
          const float v1 = fmaxf(acc[i][j][2 * h + 1] + b1[col + 1], 0.f);
          __nv_bfloat162 pr;
          pr.x = __float2bfloat16_rn(v0);
          pr.y = __float2bfloat16_rn(v1);
          *reinterpret_cast<__nv_bfloat162*>(&H1[row][col]) = pr;
        }
    __syncthreads();
    // ---- layer 2: H2 = relu(H1 W2 + b2), same warp tiling, K = 256 ----
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[i][j][c] = 0.f;
#pragma unroll 4
    for (int kk = 0; kk < 256; kk += 16) {
      unsigned a[4][4], b[4][2];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int r = 16 * i + gid;
        a[i][0] = ld32(&H1[r][kk + 2 * tig]);
        a[i][1] = ld32(&H1[r + 8][kk + 2 * tig]);
        a[i][2] = ld32(&H1[r][kk + 2 * tig + 8]);
        a[i][3] = ld32(&H1[r + 8][kk + 2 * tig + 8]);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int n = wn + 8 * j + gid;
        b[j][0] = ld32(&W2t[n][kk + 2 * tig]);
        b[j][1] = ld32(&W2t[n][kk + 2 * tig + 8]);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], a[i][0], a[i][1], a[i][2], a[i][3], b[j][0], b[j][1]);
    }
    // ---- layer 3 in the epilogue: partial Y over this warp's 32 columns ----
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float y[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const int col = wn + 8 * j + 2 * tig + e;
            const float hv = __bfloat162float(__float2bfloat16_rn(fmaxf(acc[i][j][2 * h + e] + b2[col], 0.f)));
#pragma unroll
            for (int o = 0; o < 4; ++o) y[o] += hv * W3t[o * 256 + col];
          }
#pragma unroll
        for (int o = 0; o < 4; ++o) {
          y[o] += __shfl_xor_sync(0xffffffffu, y[o], 1);
          y[o] += __shfl_xor_sync(0xffffffffu, y[o], 2);
        }
        if (tig == 0) {
          const int row = 16 * i + gid + 8 * h;
#pragma unroll
          for (int o = 0; o < 4; ++o) Yp[warp][row][o] = y[o];
        }
      }
    __syncthreads();
    {
      const int row = tid >> 2, o = tid & 3;
      float v = b3[o];
#pragma unroll
      for (int w = 0; w < 8; ++w) v += Yp[w][row][o];
      if (r0 + row < M) Y[(size_t)(r0 + row) * 4 + o] = v;
    }
  }
}

}  // namespace

size_t mlp_image_bytes() { return IMG_BYTES; }

cudaError_t mlp_pack(const float* params, void* image, cudaStream_t s) {
  k_mlp_pack<<<64, 256, 0, s>>>(params, reinterpret_cast<unsigned char*>(image));
  return cudaGetLastError();
}

cudaError_t mlp_infer_prepare() {
  return cudaFuncSetAttribute(k_mlp_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM_BYTES);
}

cudaError_t mlp_infer(const void* image, const float* X, int M, const unsigned* Mdev, float* Y, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const int tiles = (M + FT_ROWS - 1) / FT_ROWS;
  if (tiles <= 0) return cudaSuccess;
  const int grid = tiles < sms ? tiles : sms;
  k_mlp_fused<<<grid, 256, SM_BYTES, s>>>(reinterpret_cast<const uint4*>(image), X, M, Mdev, Y);
  return cudaGetLastError();
}

}  // namespace mi



// ---------------------------------------------------------------------------
// Fused inference on the 5th-generation tensor cores (tcgen05, TMEM).
//
// One CTA of 256 threads per 128-row tile, persistent over tiles.  Operands are BF16 in shared memory in the no-swizzle K-major
// "core matrix" layout (8 rows x 16 bytes contiguous; adjacent core
// matrices 128 bytes apart along K, a whole K extent apart along M/N).  The
// weights are packed once into five 32 KB chunks of (N = 256) x (K = 64):
// W1^T, then W2^T in four K ranges; a single thread streams them through a
// two-slot shared-memory ring with cp.async.bulk (completion on an
// mbarrier) and issues the MMAs (M = 128, N = 256, K = 16 each) into one
// FP32 accumulator of 256 TMEM columns; tcgen05.commit arrives on an
// mbarrier when they complete (which also frees the ring slot).  Two
// threads own each row of the tile (warp w reads TMEM lanes 32 (w % 4) ..,
// column half w / 4): they read their half of the accumulator row back with
// tcgen05.ld for the bias + ReLU epilogue of layer 1 (written back as BF16
// for layer 2's A operand) and for layer 2's epilogue, which also applies
// the 256 -> 4 output layer with the same BF16-rounded operands as the
// other paths (the two half-row partial sums meet in shared memory).  Every wait is bounded: on a timeout the kernel raises its
// error flag, stops issuing work, waits (bounded) for what it issued and
// frees its TMEM.
// ---------------------------------------------------------------------------
namespace mi {
namespace {

constexpr int TC_M = 128;
constexpr unsigned TC_CHUNK = 256 * 64 * 2;                 // one (N=256) x (K=64) BF16 chunk: 32 KB
constexpr size_t TCI_W = 0;                                  // 5 chunks
constexpr size_t TCI_W3 = TCI_W + 5 * (size_t)TC_CHUNK;      // W3^T as BF16-valued floats, [4][256]
constexpr size_t TCI_B1 = TCI_W3 + 4 * 256 * 4;
constexpr size_t TCI_B2 = TCI_B1 + 256 * 4;
constexpr size_t TCI_B3 = TCI_B2 + 256 * 4;
constexpr size_t TC_IMG_BYTES = TCI_B3 + 16;                 // 170000
// shared memory of the tcgen05 kernel
constexpr unsigned TS_X = 0;                                 // 128 x 64 BF16 core matrices: 16 KB
constexpr unsigned TS_H = TS_X + TC_M * 64 * 2;              // 128 x 256 BF16: 64 KB
constexpr unsigned TS_W = TS_H + TC_M * 256 * 2;             // ring: 2 x 32 KB
constexpr unsigned TS_P = TS_W + 2 * TC_CHUNK;               // W3^T, b1, b2, b3: 6160 B
constexpr unsigned TS_YP = TS_P + 4 * 256 * 4 + 2 * 256 * 4 + 16;  // output-layer partials [2][128][4]
constexpr unsigned TS_BAR = TS_YP + 2 * TC_M * 4 * 4;               // mbarriers (8 B each)
constexpr unsigned TS_BYTES = TS_BAR + 64;
constexpr int TC_THREADS = 256;  // two threads per tile row: one per half of the 256 columns
static_assert(TC_IMG_BYTES % 16 == 0 && TS_BYTES <= 232448 && TS_BAR % 8 == 0, "tcgen05 MLP layout");

// byte offset of element (row r, k) in a core-matrix K-major tile with K extent kext
__host__ __device__ __forceinline__ unsigned cm_off(unsigned r, unsigned k, unsigned kext) {
  return ((r >> 3) * (kext >> 3) + (k >> 3)) * 128u + (r & 7u) * 16u + (k & 7u) * 2u;
}

__global__ void k_mlp_pack_tc(const float* __restrict__ p, unsigned char* __restrict__ img) {
  const float* W1 = p;
  const float* b1 = W1 + 64 * 256;
  const float* W2 = b1 + 256;
  const float* b2 = W2 + 256 * 256;
  const float* W3 = b2 + 256;
  const float* b3 = W3 + 256 * 4;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
  // chunk c, element (n, k): B operand row n (output column), K index k within the chunk
  for (int e = tid; e < 5 * 256 * 64; e += nt) {
    const int c = e / (256 * 64), r = e % (256 * 64), n = r / 64, k = r % 64;
    const float v = c == 0 ? W1[k * 256 + n] : W2[((c - 1) * 64 + k) * 256 + n];
    *reinterpret_cast<__nv_bfloat16*>(img + TCI_W + (size_t)c * TC_CHUNK + cm_off(n, k, 64)) = __float2bfloat16_rn(v);
  }
  for (int e = tid; e < 4 * 256; e += nt) {
    const int o = e / 256, c = e % 256;
    reinterpret_cast<float*>(img + TCI_W3)[e] = __bfloat162float(__float2bfloat16_rn(W3[c * 4 + o]));
  }
  for (int e = tid; e < 256; e += nt) {
    reinterpret_cast<float*>(img + TCI_B1)[e] = b1[e];
    reinterpret_cast<float*>(img + TCI_B2)[e] = b2[e];
  }
  if (tid < 4) reinterpret_cast<float*>(img + TCI_B3)[tid] = b3[tid];
}

}  // namespace
}  // namespace mi

namespace mi {
namespace {

constexpr unsigned TC_WAIT_LIMIT = 1u << 24;  // default: try_wait rounds before a wait gives up

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned a, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned a, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
// Bounded wait for the completion of the phase with the given parity; false
// after `limit` try_wait rounds.
__device__ __forceinline__ bool mbar_wait(unsigned a, unsigned parity, unsigned limit = TC_WAIT_LIMIT) {
  for (unsigned it = 0; it < limit; ++it) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}
__device__ __forceinline__ void bulk_g2s(unsigned dst, const void* src, unsigned bytes, unsigned mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(mbar)
               : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: no swizzle, K-major core matrices; lbo =
// byte step between core matrices along K, sbo = along M/N.
__device__ __forceinline__ unsigned long long smem_desc(unsigned saddr, unsigned lbo, unsigned sbo) {
  unsigned long long d = (unsigned long long)((saddr >> 4) & 0x3FFFu);
  d |= (unsigned long long)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (unsigned long long)((sbo >> 4) & 0x3FFFu) << 32;
  d |= 1ull << 46;  // descriptor version of tcgen05
  return d;         // base offset 0, layout type 0 (no swizzle)
}
// Instruction descriptor of kind::f16: D FP32, A and B BF16, both K-major, M = 128, N = 256.
constexpr unsigned TC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((256u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void tc_mma(unsigned d_tmem, unsigned long long a, unsigned long long b, unsigned acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          d_tmem),
      "l"(a), "l"(b), "r"(TC_IDESC), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void tc_commit(unsigned mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}
// 32 consecutive FP32 columns of this warp's 32 TMEM lanes (one row per thread).
__device__ __forceinline__ void tc_ld32(unsigned taddr, float (&v)[32]) {
  unsigned r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
      "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ unsigned pack_bf2(float a, float b) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const unsigned*>(&v);
}

}  // namespace
}  // namespace mi

namespace mi {
namespace {

// wait_limit: try_wait rounds of every wait on the work's progress (0: the
// default).  stall != 0 (fault-injection tests only): before any work is
// issued, thread 0 waits, with that limit, on an mbarrier that nothing
// arrives at, so that the wait runs out and the abort path runs with no copy
// or MMA in flight.
__global__ void __launch_bounds__(TC_THREADS, 1) k_mlp_tc(const unsigned char* __restrict__ img, const float* __restrict__ X,
                                                   int M, const unsigned* __restrict__ Mdev, float* __restrict__ Y,
                                                   unsigned* __restrict__ err, unsigned err_bit, unsigned wait_limit,
                                                   int stall) {
  const unsigned wl = wait_limit ? wait_limit : TC_WAIT_LIMIT;
  extern __shared__ __align__(16) unsigned char sm[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // warp w reads TMEM lanes 32 (w % 4) ..: this thread's tile row, and column half w / 4
  const int row_t = 32 * (warp & 3) + lane, half = warp >> 2;
  if (Mdev) M = min(M, (int)*Mdev);
  const int tiles = (M + TC_M - 1) / TC_M;
  if ((int)blockIdx.x >= tiles) return;  // uniform over the block

  const unsigned sbase = smem_u32(sm);
  const unsigned full0 = sbase + TS_BAR, empty0 = sbase + TS_BAR + 16, done = sbase + TS_BAR + 32;
  const unsigned never = sbase + TS_BAR + 48;  // the stall test's barrier: nothing arrives at it
  unsigned* tmem_slot = reinterpret_cast<unsigned*>(sm + TS_BAR + 40);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + TS_BAR + 44);
  float* W3t = reinterpret_cast<float*>(sm + TS_P);
  float* b1 = W3t + 4 * 256;
  float* b2 = b1 + 256;
  float* b3 = b2 + 256;

  if (tid == 0) {
    for (int s = 0; s < 2; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(done, 1);
    mbar_init(never, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(256u)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  {
    const float* src = reinterpret_cast<const float*>(img + TCI_W3);
    for (int e = tid; e < 4 * 256 + 2 * 256 + 4; e += TC_THREADS) W3t[e] = src[e];
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned tmem = *reinterpret_cast<volatile unsigned*>(tmem_slot);
  const unsigned lane_base = (unsigned)(32 * (warp & 3)) << 16;  // this warp's TMEM lanes
  float(*Yp)[TC_M][4] = reinterpret_cast<float(*)[TC_M][4]>(sm + TS_YP);

  // producer / MMA issuer state (thread 0)
  unsigned g_issued = 0, g_used = 0;   // chunks copied, chunks consumed
  unsigned n_done = 0;                 // done-barrier completions waited for (every thread)
  bool ok = true;

  auto issue = [&](int c) {  // thread 0: copy weight chunk c into the next ring slot
    const unsigned s = g_issued & 1u, use = g_issued >> 1;
    if (use > 0 && !mbar_wait(empty0 + 8 * s, (use - 1) & 1u, wl)) { ok = false; return; }
    mbar_expect_tx(full0 + 8 * s, TC_CHUNK);
    bulk_g2s(sbase + TS_W + s * TC_CHUNK, img + TCI_W + (size_t)c * TC_CHUNK, TC_CHUNK, full0 + 8 * s);
    ++g_issued;
  };
  // thread 0: MMAs of the next copied chunk: A (K extent a_kext, starting K a_k0), accumulate into D
  auto consume = [&](unsigned a_base, unsigned a_kext, unsigned a_k0, bool first) {
    const unsigned s = g_used & 1u, use = g_used >> 1;
    if (!mbar_wait(full0 + 8 * s, use & 1u, wl)) { ok = false; return; }
    tc_fence_after();
    const unsigned b_base = sbase + TS_W + s * TC_CHUNK;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const unsigned long long a = smem_desc(a_base + cm_off(0, a_k0 + 16 * k, a_kext), 128, (a_kext / 8) * 128);
      const unsigned long long b = smem_desc(b_base + cm_off(0, 16 * k, 64), 128, (64 / 8) * 128);
      tc_mma(tmem, a, b, (first && k == 0) ? 0u : 1u);
    }
    tc_commit(empty0 + 8 * s);  // the slot is free once these MMAs have read it
    ++g_used;
  };

  if (stall) {
    if (tid == 0 && !mbar_wait(never, 0u, wl)) *abort_flag = 1;
    __syncthreads();
  }
  int t = blockIdx.x;
  for (; t < tiles && !*abort_flag; t += gridDim.x) {
    const int r0 = t * TC_M;
    // X tile: this thread's half of its row, BF16, core-matrix layout (K extent 64)
    {
      const int row = r0 + row_t;
#pragma unroll
      for (int q = 4 * half; q < 4 * half + 4; ++q) {
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
        if (row < M) {
          a = *reinterpret_cast<const float4*>(X + (size_t)row * 64 + 8 * q);
          b = *reinterpret_cast<const float4*>(X + (size_t)row * 64 + 8 * q + 4);
        }
        *reinterpret_cast<uint4*>(sm + TS_X + cm_off(row_t, 8 * q, 64)) =
            make_uint4(pack_bf2(a.x, a.y), pack_bf2(a.z, a.w), pack_bf2(b.x, b.y), pack_bf2(b.z, b.w));
      }
    }
    fence_proxy_async();  // generic-proxy smem writes -> visible to the tensor core
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0 && ok) {
      issue(0);
      if (ok) issue(1);
      if (ok) consume(sbase + TS_X, 64, 0, true);  // layer 1: D = X W1
      if (ok) tc_commit(done);
      if (!ok) *abort_flag = 1;
    }
    __syncthreads();
    if (*abort_flag) break;
    // ---- layer-1 epilogue: H1 = relu(D + b1) as BF16 (A operand of layer 2) ----
    if (!mbar_wait(done, n_done & 1u, wl)) *abort_flag = 1;
    ++n_done;
    tc_fence_after();
    __syncthreads();
    if (*abort_flag) break;
#pragma unroll 1
    for (int cb = 4 * half; cb < 4 * half + 4; ++cb) {
      float v[32];
      tc_ld32(tmem + lane_base + 32 * cb, v);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int c = 32 * cb + 8 * q;
        uint4 w;
        w.x = pack_bf2(fmaxf(v[8 * q] + b1[c], 0.f), fmaxf(v[8 * q + 1] + b1[c + 1], 0.f));
        w.y = pack_bf2(fmaxf(v[8 * q + 2] + b1[c + 2], 0.f), fmaxf(v[8 * q + 3] + b1[c + 3], 0.f));
        w.z = pack_bf2(fmaxf(v[8 * q + 4] + b1[c + 4], 0.f), fmaxf(v[8 * q + 5] + b1[c + 5], 0.f));
        w.w = pack_bf2(fmaxf(v[8 * q + 6] + b1[c + 6], 0.f), fmaxf(v[8 * q + 7] + b1[c + 7], 0.f));
        *reinterpret_cast<uint4*>(sm + TS_H + cm_off(row_t, c, 256)) = w;
      }
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0 && ok) {
      for (int c = 1; c <= 4 && ok; ++c) {
        if (c + 1 <= 4) issue(c + 1);
        if (ok) consume(sbase + TS_H, 256, 64 * (c - 1), c == 1);  // layer 2: D = H1 W2
      }
      if (ok) tc_commit(done);
      if (!ok) *abort_flag = 1;
    }
    __syncthreads();
    if (*abort_flag) break;
    // ---- layer-2 epilogue and the output layer ----
    if (!mbar_wait(done, n_done & 1u, wl)) *abort_flag = 1;
    ++n_done;
    tc_fence_after();
    __syncthreads();
    if (*abort_flag) break;
    float y[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 1
    for (int cb = 4 * half; cb < 4 * half + 4; ++cb) {
      float v[32];
      tc_ld32(tmem + lane_base + 32 * cb, v);
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int c = 32 * cb + j;
        const float h = __bfloat162float(__float2bfloat16_rn(fmaxf(v[j] + b2[c], 0.f)));
#pragma unroll
        for (int o = 0; o < 4; ++o) y[o] += h * W3t[o * 256 + c];
      }
    }
#pragma unroll
    for (int o = 0; o < 4; ++o) Yp[half][row_t][o] = y[o];
    __syncthreads();
    if (half == 0 && r0 + row_t < M) {
      float r[4];
#pragma unroll
      for (int o = 0; o < 4; ++o) r[o] = b3[o] + (Yp[0][row_t][o] + Yp[1][row_t][o]);
      *reinterpret_cast<float4*>(Y + (size_t)(r0 + row_t) * 4) = make_float4(r[0], r[1], r[2], r[3]);
    }
    tc_fence_before();
    __syncthreads();  // TMEM, X and H1 are reused by the next tile
    tc_fence_after();
  }
  // teardown: after an abort, wait (bounded) for what was issued, then free the TMEM
  if (*abort_flag) {
    // rows this block did not finish are marked NaN
    for (int tt = t; tt < tiles; tt += gridDim.x)
      if (half == 0 && tt * TC_M + row_t < M)
        *reinterpret_cast<float4*>(Y + (size_t)(tt * TC_M + row_t) * 4) = make_float4(NAN, NAN, NAN, NAN);
    if (tid == 0) {
      atomicOr(err, err_bit);
      for (unsigned s = 0; s < 2; ++s) {
        const unsigned uses = (g_issued + (s == 0 ? 1u : 0u)) >> 1;  // copies into slot s
        const unsigned consumed = (g_used + (s == 0 ? 1u : 0u)) >> 1;
        if (uses > consumed) mbar_wait(full0 + 8 * s, consumed & 1u);
        if (consumed > 0) mbar_wait(empty0 + 8 * s, (consumed - 1) & 1u);
      }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
  }
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256u) : "memory");
}

}  // namespace

size_t mlp_tc_image_bytes() { return TC_IMG_BYTES; }

cudaError_t mlp_tc_pack(const float* params, void* image, cudaStream_t s) {
  k_mlp_pack_tc<<<64, 256, 0, s>>>(params, reinterpret_cast<unsigned char*>(image));
  return cudaGetLastError();
}

cudaError_t mlp_tc_prepare() {
  return cudaFuncSetAttribute(k_mlp_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TS_BYTES);
}

cudaError_t mlp_tc_infer(const void* image, const float* X, int M, const unsigned* Mdev, float* Y, unsigned* err,
                         unsigned err_bit, cudaStream_t s, unsigned wait_limit, int stall) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const int tiles = (M + TC_M - 1) / TC_M;
  if (tiles <= 0) return cudaSuccess;
  const int grid = tiles < sms ? tiles : sms;
  k_mlp_tc<<<grid, TC_THREADS, TS_BYTES, s>>>(reinterpret_cast<const unsigned char*>(image), X, M, Mdev, Y, err, err_bit,
                                              wait_limit, stall);
  return cudaGetLastError();
}

}  // namespace mi

namespace mi {
// Device word the standalone inference reports a tcgen05 wait timeout in.
__device__ unsigned g_mlp_tc_error;

size_t mlp_image_total() { return IMG_BYTES + TC_IMG_BYTES; }
}  // namespace mi

extern "C" {

// The packed image holds both layouts: the mma.sync kernel's (first
// IMG_BYTES bytes) and the tcgen05 kernel's (the rest).
size_t mi_mlp_image_bytes(void) { return mi::mlp_image_total(); }

mi_status mi_mlp_pack(const float* params, void* image, void* stream) {
  if (!params || !image || (reinterpret_cast<uintptr_t>(image) & 15)) {
    mi::set_thread_error("mi_mlp_pack: null pointer or image not 16-byte aligned");
    return MI_EINVAL;
  }
  cudaError_t e = mi::mlp_pack(params, image, (cudaStream_t)stream);
  if (e == cudaSuccess) e = mi::mlp_tc_pack(params, static_cast<unsigned char*>(image) + mi::IMG_BYTES, (cudaStream_t)stream);
  if (e != cudaSuccess) {
    mi::set_thread_error("mi_mlp_pack: launch failed");
    return MI_ECUDA;
  }
  return MI_OK;
}

static mi_status infer_args(const void* image, const float* X, int n, float* Y, const char* who) {
  if (n < 0 || (n > 0 && (!image || !X || !Y)) || (reinterpret_cast<uintptr_t>(image) & 15) ||
      (reinterpret_cast<uintptr_t>(X) & 15) || (reinterpret_cast<uintptr_t>(Y) & 15)) {
    mi::set_thread_error((std::string(who) + ": null pointer, negative batch, or image/X/Y not 16-byte aligned").c_str());
    return MI_EINVAL;
  }
  return MI_OK;
}

mi_status mi_mlp_infer(const void* image, const float* X, int n, float* Y, void* stream) {
  mi_status st = infer_args(image, X, n, Y, "mi_mlp_infer");
  if (st != MI_OK || n == 0) return st;
  unsigned* err = nullptr;
  if (cudaGetSymbolAddress(reinterpret_cast<void**>(&err), mi::g_mlp_tc_error) != cudaSuccess ||
      mi::mlp_tc_prepare() != cudaSuccess ||
      mi::mlp_tc_infer(static_cast<const unsigned char*>(image) + mi::IMG_BYTES, X, n, nullptr, Y, err, 1u,
                       (cudaStream_t)stream) != cudaSuccess) {
    mi::set_thread_error("mi_mlp_infer: launch failed");
    return MI_ECUDA;
  }
  return MI_OK;
}

mi_status mi_mlp_infer_mma(const void* image, const float* X, int n, float* Y, void* stream) {
  mi_status st = infer_args(image, X, n, Y, "mi_mlp_infer_mma");
  if (st != MI_OK || n == 0) return st;
  if (mi::mlp_infer_prepare() != cudaSuccess || mi::mlp_infer(image, X, n, nullptr, Y, (cudaStream_t)stream) != cudaSuccess) {
    mi::set_thread_error("mi_mlp_infer_mma: launch failed");
    return MI_ECUDA;
  }
  return MI_OK;
}

}  // extern "C"
