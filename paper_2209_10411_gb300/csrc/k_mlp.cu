// MLP of the learned Newton guess (64 -> 256 -> 256 -> 4, ReLU): forward,
// backward, MSE loss and AdamW on the GPU.  Every matrix product runs on the
// tensor cores as BF16 x BF16 -> FP32 (mma.sync m16n8k16); parameters,
// activations and gradients live in FP32 and are rounded to BF16 when a tile
// is staged in shared memory, so the network computes with BF16 weights and
// FP32 accumulation while the optimizer keeps FP32 master weights.
#include <cstring>

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

extern "C" {

size_t mi_mlp_image_bytes(void) { return mi::IMG_BYTES; }

mi_status mi_mlp_pack(const float* params, void* image, void* stream) {
  if (!params || !image || (reinterpret_cast<uintptr_t>(image) & 15)) {
    mi::set_thread_error("mi_mlp_pack: null pointer or image not 16-byte aligned");
    return MI_EINVAL;
  }
  if (mi::mlp_pack(params, image, (cudaStream_t)stream) != cudaSuccess) {
    mi::set_thread_error("mi_mlp_pack: launch failed");
    return MI_ECUDA;
  }
  return MI_OK;
}

mi_status mi_mlp_infer(const void* image, const float* X, int n, float* Y, void* stream) {
  if (n < 0 || (n > 0 && (!image || !X || !Y)) || (reinterpret_cast<uintptr_t>(image) & 15) ||
      (reinterpret_cast<uintptr_t>(X) & 15)) {
    mi::set_thread_error("mi_mlp_infer: null pointer, negative batch, or image/X not 16-byte aligned");
    return MI_EINVAL;
  }
  if (n == 0) return MI_OK;
  if (mi::mlp_infer_prepare() != cudaSuccess || mi::mlp_infer(image, X, n, nullptr, Y, (cudaStream_t)stream) != cudaSuccess) {
    mi::set_thread_error("mi_mlp_infer: launch failed");
    return MI_ECUDA;
  }
  return MI_OK;
}

}  // extern "C"
