// Learned warm start: per-contact MLP 32 -> 128 -> 128 -> 128 -> 3 with GELU
// (exact erf form), BF16 weights and activations, FP32 accumulation, on the
// tensor cores (mma.sync m16n8k16 BF16).
//
// Inference (k_mlp_fwd): one warp per 16 contact rows; the block stages every
// weight once in shared memory (rows padded by 8 BF16 so the 8 row-groups of a
// fragment load hit distinct banks); each layer's FP32 accumulators become the
// next layer's A fragments in registers (the C fragment of n-tiles 2kk, 2kk+1
// is exactly the A fragment of k-tile kk), so activations never leave the SM.
// Training: the same forward kernel stores Z (pre-activation, FP32) and H (BF16)
// per layer; the backward pass is a tiled BF16 GEMM (k_gemm) plus elementwise
// kernels (MSE gradient, GELU', bias sums) and Adam on FP32 master weights.
//
// Parameter layout (FP32, shared with the CPU reference): W1[128][32] b1[128]
// W2[128][128] b2[128] W3[128][128] b3[128] W4[3][128] b4[3].
#include <cuda_bf16.h>

#include <string>
#include <vector>

#include "../../include/sim.h"
#include "sim_internal.cuh"

namespace gb {

constexpr int HID = 128, NIN = 32, NOUT = 3;
constexpr int MLP_NPARAM = HID * NIN + HID + HID * HID + HID + HID * HID + HID + NOUT * HID + NOUT;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + HID * NIN, OFF_W2 = OFF_B1 + HID, OFF_B2 = OFF_W2 + HID * HID,
              OFF_W3 = OFF_B2 + HID, OFF_B3 = OFF_W3 + HID * HID, OFF_W4 = OFF_B3 + HID, OFF_B4 = OFF_W4 + NOUT * HID;
constexpr int LD1 = NIN + 8;   // padded row length (BF16) of W1
constexpr int LDH = HID + 8;   // padded row length of W2, W3, W4

// device weights: BF16 padded, biases FP32 (b4 padded to 8), input normalisation
struct MlpDev {
  __nv_bfloat16 *W1, *W2, *W3, *W4;  // [128][40], [128][136], [128][136], [8][136]
  float *b1, *b2, *b3, *b4;          // [128] x3, [8]
  float *mean, *invstd;              // [32]
};

constexpr size_t SMEM_W1 = (size_t)HID * LD1 * 2, SMEM_W23 = (size_t)HID * LDH * 2, SMEM_W4 = (size_t)8 * LDH * 2;
constexpr size_t SMEM_MLP = SMEM_W1 + 2 * SMEM_W23 + SMEM_W4 + (3 * HID + 8 + 2 * NIN) * 4;

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}
__device__ __forceinline__ void mma16816(float* c, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x) {
  return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * expf(-0.5f * x * x) * 0.39894228040143267794f;
}

struct FwdOut {       // training-mode outputs (nullptr in inference)
  float *Z1, *Z2, *Z3;  // [n][128]
  __nv_bfloat16 *X, *H1, *H2, *H3;  // [n][32], [n][128] x3
  float* Y;           // [n][3]
};

// Rows: inference reads feature row `slot` of environment `env` (rows 0..n_contacts-1
// of each environment, 16 per warp pass); training reads rows 0..n-1 of X.
template <bool TRAIN>
__global__ void __launch_bounds__(128) k_mlp_fwd(MlpDev w, const float* feat, const int* n_contacts, int E, int C,
                                                 float4* pred, int n_rows, FwdOut out) {
  extern __shared__ __align__(16) unsigned char smm[];
  __nv_bfloat16* sW1 = reinterpret_cast<__nv_bfloat16*>(smm);
  __nv_bfloat16* sW2 = reinterpret_cast<__nv_bfloat16*>(smm + SMEM_W1);
  __nv_bfloat16* sW3 = reinterpret_cast<__nv_bfloat16*>(smm + SMEM_W1 + SMEM_W23);
  __nv_bfloat16* sW4 = reinterpret_cast<__nv_bfloat16*>(smm + SMEM_W1 + 2 * SMEM_W23);
  float* sb = reinterpret_cast<float*>(smm + SMEM_W1 + 2 * SMEM_W23 + SMEM_W4);  // b1 b2 b3 b4(8) mean invstd
  // stage weights (16-byte copies)
  {
    const int4* src;
    int4* dst;
    src = reinterpret_cast<const int4*>(w.W1); dst = reinterpret_cast<int4*>(sW1);
    for (int i = threadIdx.x; i < (int)(SMEM_W1 / 16); i += blockDim.x) dst[i] = src[i];
    src = reinterpret_cast<const int4*>(w.W2); dst = reinterpret_cast<int4*>(sW2);
    for (int i = threadIdx.x; i < (int)(SMEM_W23 / 16); i += blockDim.x) dst[i] = src[i];
    src = reinterpret_cast<const int4*>(w.W3); dst = reinterpret_cast<int4*>(sW3);
    for (int i = threadIdx.x; i < (int)(SMEM_W23 / 16); i += blockDim.x) dst[i] = src[i];
    src = reinterpret_cast<const int4*>(w.W4); dst = reinterpret_cast<int4*>(sW4);
    for (int i = threadIdx.x; i < (int)(SMEM_W4 / 16); i += blockDim.x) dst[i] = src[i];
    for (int i = threadIdx.x; i < HID; i += blockDim.x) {
      sb[i] = w.b1[i]; sb[HID + i] = w.b2[i]; sb[2 * HID + i] = w.b3[i];
    }
    for (int i = threadIdx.x; i < 8; i += blockDim.x) sb[3 * HID + i] = w.b4[i];
    for (int i = threadIdx.x; i < NIN; i += blockDim.x) {
      sb[3 * HID + 8 + i] = w.mean[i];
      sb[3 * HID + 8 + NIN + i] = w.invstd[i];
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const float* smean = sb + 3 * HID + 8;
  const float* sinv = smean + NIN;

  // work list, walked by the warps of the grid: inference = (environment, 16-row tile)
  // items over each environment's contacts; training = 16-row tiles of X
  const int gwarp = blockIdx.x * 4 + warp, nwarps = gridDim.x * 4;
  for (int item = gwarp;; item += nwarps) {
    int row0, nvalid, e_item = 0;
    if (TRAIN) {
      row0 = item * 16;
      if (row0 >= n_rows) break;
      nvalid = min(16, n_rows - row0);
    } else {
      if (item >= E * ((C + 15) / 16)) break;
      e_item = item / ((C + 15) / 16);
      int tile = item % ((C + 15) / 16);
      int nc = n_contacts[e_item];
      row0 = tile * 16;
      if (row0 >= nc) continue;
      nvalid = min(16, nc - row0);
    }
    const int r0 = g, r1 = g + 8;
    const bool v0 = r0 < nvalid, v1 = r1 < nvalid;
    const float* x0 = TRAIN ? feat + (size_t)(row0 + r0) * NIN : feat + ((size_t)e_item * C + row0 + r0) * NIN;
    const float* x1 = TRAIN ? feat + (size_t)(row0 + r1) * NIN : feat + ((size_t)e_item * C + row0 + r1) * NIN;
    // ---- layer 1 A fragments from the (normalised) features
    uint32_t a[8][4];
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
      int c0 = 16 * kk + 2 * t, c1 = c0 + 8;
      float f00 = v0 ? (x0[c0] - smean[c0]) * sinv[c0] : 0.f, f01 = v0 ? (x0[c0 + 1] - smean[c0 + 1]) * sinv[c0 + 1] : 0.f;
      float f10 = v1 ? (x1[c0] - smean[c0]) * sinv[c0] : 0.f, f11 = v1 ? (x1[c0 + 1] - smean[c0 + 1]) * sinv[c0 + 1] : 0.f;
      float f02 = v0 ? (x0[c1] - smean[c1]) * sinv[c1] : 0.f, f03 = v0 ? (x0[c1 + 1] - smean[c1 + 1]) * sinv[c1 + 1] : 0.f;
      float f12 = v1 ? (x1[c1] - smean[c1]) * sinv[c1] : 0.f, f13 = v1 ? (x1[c1 + 1] - smean[c1 + 1]) * sinv[c1 + 1] : 0.f;
      a[kk][0] = pack2(f00, f01);
      a[kk][1] = pack2(f10, f11);
      a[kk][2] = pack2(f02, f03);
      a[kk][3] = pack2(f12, f13);
      if (TRAIN) {
        if (v0) {
          *reinterpret_cast<uint32_t*>(out.X + (size_t)(row0 + r0) * NIN + c0) = a[kk][0];
          *reinterpret_cast<uint32_t*>(out.X + (size_t)(row0 + r0) * NIN + c1) = a[kk][2];
        }
        if (v1) {
          *reinterpret_cast<uint32_t*>(out.X + (size_t)(row0 + r1) * NIN + c0) = a[kk][1];
          *reinterpret_cast<uint32_t*>(out.X + (size_t)(row0 + r1) * NIN + c1) = a[kk][3];
        }
      }
    }
    // ---- layers 1..3: 16 n-tiles of 8 outputs
    float acc[16][4];
#pragma unroll
    for (int layer = 0; layer < 3; ++layer) {
      const __nv_bfloat16* sW = layer == 0 ? sW1 : (layer == 1 ? sW2 : sW3);
      const int ld = layer == 0 ? LD1 : LDH;
      const int nk = layer == 0 ? 2 : 8;
      const float* bias = sb + layer * HID;
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
        const __nv_bfloat16* wrow = sW + (size_t)(8 * j + g) * ld + 2 * t;
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
          if (kk < nk) {
            uint32_t b0 = *reinterpret_cast<const uint32_t*>(wrow + 16 * kk);
            uint32_t b1 = *reinterpret_cast<const uint32_t*>(wrow + 16 * kk + 8);
            mma16816(acc[j], a[kk], b0, b1);
          }
        }
      }
      // bias + GELU, stored for training, packed into the next layer's A fragments
      float* Zo = layer == 0 ? out.Z1 : (layer == 1 ? out.Z2 : out.Z3);
      __nv_bfloat16* Ho = layer == 0 ? out.H1 : (layer == 1 ? out.H2 : out.H3);
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        int col = 8 * j + 2 * t;
        float z0 = acc[j][0] + bias[col], z1 = acc[j][1] + bias[col + 1];
        float z2 = acc[j][2] + bias[col], z3 = acc[j][3] + bias[col + 1];
        uint32_t p01 = pack2(gelu(z0), gelu(z1)), p23 = pack2(gelu(z2), gelu(z3));
        if (TRAIN) {
          if (v0) {
            *reinterpret_cast<float2*>(Zo + (size_t)(row0 + r0) * HID + col) = make_float2(z0, z1);
            *reinterpret_cast<uint32_t*>(Ho + (size_t)(row0 + r0) * HID + col) = p01;
          }
          if (v1) {
            *reinterpret_cast<float2*>(Zo + (size_t)(row0 + r1) * HID + col) = make_float2(z2, z3);
            *reinterpret_cast<uint32_t*>(Ho + (size_t)(row0 + r1) * HID + col) = p23;
          }
        }
        if ((j & 1) == 0) { a[j >> 1][0] = p01; a[j >> 1][1] = p23; }
        else { a[j >> 1][2] = p01; a[j >> 1][3] = p23; }
      }
    }
    // ---- layer 4: one n-tile (3 outputs padded to 8)
    float y[4] = {0.f, 0.f, 0.f, 0.f};
    const __nv_bfloat16* w4row = sW4 + (size_t)g * LDH + 2 * t;
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
      uint32_t b0 = *reinterpret_cast<const uint32_t*>(w4row + 16 * kk);
      uint32_t b1 = *reinterpret_cast<const uint32_t*>(w4row + 16 * kk + 8);
      mma16816(y, a[kk], b0, b1);
    }
    // lane (g, t) holds cols 2t, 2t+1 of rows g (y0, y1) and g+8 (y2, y3); outputs are cols 0..2
    const float* b4 = sb + 3 * HID;
    float c2_r0 = __shfl_down_sync(0xffffffffu, y[0], 1);  // col 2 of row g, from lane t = 1
    float c2_r1 = __shfl_down_sync(0xffffffffu, y[2], 1);
    if (t == 0) {
      float o0[3] = {y[0] + b4[0], y[1] + b4[1], c2_r0 + b4[2]};
      float o1[3] = {y[2] + b4[0], y[3] + b4[1], c2_r1 + b4[2]};
      if (TRAIN) {
        if (v0) for (int k = 0; k < 3; ++k) out.Y[(size_t)(row0 + r0) * 3 + k] = o0[k];
        if (v1) for (int k = 0; k < 3; ++k) out.Y[(size_t)(row0 + r1) * 3 + k] = o1[k];
      } else {
        if (v0) pred[(size_t)e_item * C + row0 + r0] = make_float4(o0[0], o0[1], o0[2], 0.f);
        if (v1) pred[(size_t)e_item * C + row0 + r1] = make_float4(o1[0], o1[1], o1[2], 0.f);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// C[M x N] (FP32, row-major, ldc) = op(A)[M x K] * op(B)[K x N], BF16 operands:
// A(m, k) = A[a_t ? k * lda + m : m * lda + k], B(k, n) = B[b_t ? n * ldb + k : k * ldb + n].
// Block tile 64 x 64, K step 32, 4 warps of 32 x 32 (2 x 4 mma tiles).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_gemm(int M, int N, int K, const __nv_bfloat16* A, int lda, int a_t,
                                              const __nv_bfloat16* B, int ldb, int b_t, float* C, int ldc) {
  __shared__ __align__(16) __nv_bfloat16 sA[64][40];  // [m][k]
  __shared__ __align__(16) __nv_bfloat16 sB[64][40];  // [n][k]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  float acc[2][4][4];
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 4; ++j)
      for (int k = 0; k < 4; ++k) acc[i][j][k] = 0.f;
  const __nv_bfloat16 zero = __float2bfloat16_rn(0.f);
  for (int k0 = 0; k0 < K; k0 += 32) {
    for (int i = threadIdx.x; i < 64 * 32; i += 128) {
      int r = i / 32, k = i % 32;
      int m = m0 + r, kk = k0 + k;
      sA[r][k] = (m < M && kk < K) ? A[a_t ? (size_t)kk * lda + m : (size_t)m * lda + kk] : zero;
      int n = n0 + r;
      sB[r][k] = (n < N && kk < K) ? B[b_t ? (size_t)n * ldb + kk : (size_t)kk * ldb + n] : zero;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
      uint32_t af[2][4];
      for (int i = 0; i < 2; ++i) {
        int r = wm + 16 * i + g, c = 16 * kk + 2 * t;
        af[i][0] = *reinterpret_cast<const uint32_t*>(&sA[r][c]);
        af[i][1] = *reinterpret_cast<const uint32_t*>(&sA[r + 8][c]);
        af[i][2] = *reinterpret_cast<const uint32_t*>(&sA[r][c + 8]);
        af[i][3] = *reinterpret_cast<const uint32_t*>(&sA[r + 8][c + 8]);
      }
      for (int j = 0; j < 4; ++j) {
        int n = wn + 8 * j + g, c = 16 * kk + 2 * t;
        uint32_t b0 = *reinterpret_cast<const uint32_t*>(&sB[n][c]);
        uint32_t b1 = *reinterpret_cast<const uint32_t*>(&sB[n][c + 8]);
        for (int i = 0; i < 2; ++i) mma16816(acc[i][j], af[i], b0, b1);
      }
    }
    __syncthreads();
  }
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 4; ++j) {
      int r = m0 + wm + 16 * i + g, c = n0 + wn + 8 * j + 2 * t;
      if (r < M && c < N) C[(size_t)r * ldc + c] = acc[i][j][0];
      if (r < M && c + 1 < N) C[(size_t)r * ldc + c + 1] = acc[i][j][1];
      if (r + 8 < M && c < N) C[(size_t)(r + 8) * ldc + c] = acc[i][j][2];
      if (r + 8 < M && c + 1 < N) C[(size_t)(r + 8) * ldc + c + 1] = acc[i][j][3];
    }
}

// dY = 2 (Y - T) / (3 n) as BF16 [n][8] (columns 3..7 zero); loss partial sums per block
__global__ void k_mse_grad(const float* Y, const float* T, int n, __nv_bfloat16* dY, float* loss_acc) {
  __shared__ float red[256];
  float s = 0.f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n * 8; i += gridDim.x * blockDim.x) {
    int r = i / 8, k = i % 8;
    float gval = 0.f;
    if (k < 3) {
      float d = Y[(size_t)r * 3 + k] - T[(size_t)r * 3 + k];
      s += d * d;
      gval = 2.f * d / (3.f * n);
    }
    dY[i] = __float2bfloat16_rn(gval);
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(loss_acc, red[0]);
}

// dZ = dH (FP32 [n][128]) * GELU'(Z) -> BF16
__global__ void k_gelu_back(const float* dH, const float* Z, int n, __nv_bfloat16* dZ) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= (size_t)n * HID) return;
  dZ[i] = __float2bfloat16_rn(dH[i] * gelu_grad(Z[i]));
}

// column sums of a BF16 [n][ld] matrix (first `cols` columns) -> out[cols] (FP32)
__global__ void k_colsum(const __nv_bfloat16* X, int n, int ld, int cols, float* out) {
  int c = blockIdx.x;
  if (c >= cols) return;
  __shared__ float red[256];
  float s = 0.f;
  for (int r = threadIdx.x; r < n; r += blockDim.x) s += __bfloat162float(X[(size_t)r * ld + c]);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[c] = red[0];
}

// Adam (Kingma & Ba 2015) on FP32 master parameters
__global__ void k_adam(float* p, const float* gr, float* m, float* v, int n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float gi = gr[i];
  float mi = b1 * m[i] + (1.f - b1) * gi;
  float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// FP32 flat parameters -> padded BF16 weights and FP32 biases
__global__ void k_pack_params(const float* P, MlpDev w) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < HID * LD1) {
    int r = i / LD1, c = i % LD1;
    w.W1[i] = __float2bfloat16_rn(c < NIN ? P[OFF_W1 + r * NIN + c] : 0.f);
  }
  if (i < HID * LDH) {
    int r = i / LDH, c = i % LDH;
    w.W2[i] = __float2bfloat16_rn(c < HID ? P[OFF_W2 + r * HID + c] : 0.f);
    w.W3[i] = __float2bfloat16_rn(c < HID ? P[OFF_W3 + r * HID + c] : 0.f);
  }
  if (i < 8 * LDH) {
    int r = i / LDH, c = i % LDH;
    w.W4[i] = __float2bfloat16_rn(r < NOUT && c < HID ? P[OFF_W4 + r * HID + c] : 0.f);
  }
  if (i < HID) {
    w.b1[i] = P[OFF_B1 + i];
    w.b2[i] = P[OFF_B2 + i];
    w.b3[i] = P[OFF_B3 + i];
  }
  if (i < 8) w.b4[i] = i < NOUT ? P[OFF_B4 + i] : 0.f;
}

__global__ void k_fill(float* p, int n, float v) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct Mlp {
  MlpDev w;
  float* params;  // FP32 flat master copy
  std::vector<void*> allocs;
};

template <typename T>
static bool dmalloc(Mlp* m, T** p, size_t n) {
  if (cudaMalloc((void**)p, sizeof(T) * (n ? n : 1)) != cudaSuccess) return false;
  m->allocs.push_back(*p);
  return true;
}

static bool mlp_alloc(Mlp* m) {
  return dmalloc(m, &m->w.W1, (size_t)HID * LD1) && dmalloc(m, &m->w.W2, (size_t)HID * LDH) &&
         dmalloc(m, &m->w.W3, (size_t)HID * LDH) && dmalloc(m, &m->w.W4, (size_t)8 * LDH) &&
         dmalloc(m, &m->w.b1, HID) && dmalloc(m, &m->w.b2, HID) && dmalloc(m, &m->w.b3, HID) &&
         dmalloc(m, &m->w.b4, 8) && dmalloc(m, &m->w.mean, NIN) && dmalloc(m, &m->w.invstd, NIN) &&
         dmalloc(m, &m->params, MLP_NPARAM);
}

static void mlp_free(Mlp* m) {
  for (void* p : m->allocs) cudaFree(p);
  delete m;
}

static void mlp_repack(Mlp* m, cudaStream_t s) {
  k_pack_params<<<(HID * LDH + 255) / 256, 256, 0, s>>>(m->params, m->w);
}

void* mlp_create(const float* params, int on_device, cudaStream_t s, std::string& err) {
  Mlp* m = new Mlp();
  if (!mlp_alloc(m)) {
    err = "allocation failed";
    mlp_free(m);
    return nullptr;
  }
  cudaMemcpyAsync(m->params, params, sizeof(float) * MLP_NPARAM,
                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s);
  k_fill<<<1, NIN, 0, s>>>(m->w.mean, NIN, 0.f);
  k_fill<<<1, NIN, 0, s>>>(m->w.invstd, NIN, 1.f);
  mlp_repack(m, s);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    err = cudaGetErrorString(e);
    mlp_free(m);
    return nullptr;
  }
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_mlp_fwd<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_MLP);
    cudaFuncSetAttribute(k_mlp_fwd<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_MLP);
    attr = true;
  }
  return m;
}

void mlp_destroy(void* p) {
  if (p) mlp_free((Mlp*)p);
}

void launch_mlp_infer(const Dev& d, const void* mlp, cudaStream_t s) {
  const Mlp* m = (const Mlp*)mlp;
  if (d.E == 0) return;
  int tiles = d.E * ((d.C + 15) / 16);
  int blocks = min((tiles + 3) / 4, 152 * 2 * 8);
  FwdOut none = {};
  k_mlp_fwd<false><<<blocks, 128, SMEM_MLP, s>>>(m->w, d.feat, d.n_contacts, d.E, d.C, d.pred, 0, none);
}

}  // namespace gb

// ---------------------------------------------------------------------------
// C ABI: trainer (see include/sim.h)
// ---------------------------------------------------------------------------
struct MlpTrainer {
  gb::Mlp* m;
  cudaStream_t stream;
  int batch;
  float *grad, *am, *av, *Z, *dH, *loss;
  __nv_bfloat16 *X, *H, *dY, *dZ;
  float* Y;
  long long t;
  std::string err;
};

namespace gb {
int report_error(int code, const std::string& msg);
}

static int tr_fail(int code, const std::string& msg) { return gb::report_error(code, msg); }

extern "C" {

int mlp_train_create(const float* init_params, int on_device, int batch, const float* feat_mean,
                     const float* feat_std, void* cuda_stream, MlpTrainer** out) {
  using namespace gb;
  if (!out || !init_params || batch < 1 || batch > (1 << 20)) return tr_fail(SIM_ERR_INVALID_ARG, "mlp_train_create: bad argument");
  *out = nullptr;
  MlpTrainer* T = new MlpTrainer();
  T->stream = (cudaStream_t)cuda_stream;
  T->batch = batch;
  T->t = 0;
  std::string err;
  T->m = (Mlp*)mlp_create(init_params, on_device, T->stream, err);
  if (!T->m) { delete T; return tr_fail(SIM_ERR_CUDA, "mlp_train_create: " + err); }
  Mlp* m = T->m;
  size_t B = batch;
  bool ok = dmalloc(m, &T->grad, MLP_NPARAM) && dmalloc(m, &T->am, MLP_NPARAM) && dmalloc(m, &T->av, MLP_NPARAM) &&
            dmalloc(m, &T->Z, 3 * B * HID) && dmalloc(m, &T->dH, B * HID) && dmalloc(m, &T->loss, 1) &&
            dmalloc(m, &T->X, B * NIN) && dmalloc(m, &T->H, 3 * B * HID) && dmalloc(m, &T->dY, B * 8) &&
            dmalloc(m, &T->dZ, B * HID) && dmalloc(m, &T->Y, B * 3);
  if (!ok) { mlp_free(m); delete T; return tr_fail(SIM_ERR_OOM, "mlp_train_create: allocation failed"); }
  cudaMemsetAsync(T->am, 0, sizeof(float) * MLP_NPARAM, T->stream);
  cudaMemsetAsync(T->av, 0, sizeof(float) * MLP_NPARAM, T->stream);
  std::vector<float> mean(NIN, 0.f), inv(NIN, 1.f);
  for (int i = 0; i < NIN; ++i) {
    if (feat_mean) mean[i] = feat_mean[i];
    if (feat_std) inv[i] = feat_std[i] > 0.f ? 1.f / feat_std[i] : 1.f;
  }
  cudaMemcpyAsync(m->w.mean, mean.data(), sizeof(float) * NIN, cudaMemcpyHostToDevice, T->stream);
  cudaMemcpyAsync(m->w.invstd, inv.data(), sizeof(float) * NIN, cudaMemcpyHostToDevice, T->stream);
  cudaError_t e = cudaStreamSynchronize(T->stream);
  if (e != cudaSuccess) { mlp_free(m); delete T; return tr_fail(SIM_ERR_CUDA, cudaGetErrorString(e)); }
  *out = T;
  return SIM_OK;
}

void mlp_train_destroy(MlpTrainer* T) {
  if (!T) return;
  cudaStreamSynchronize(T->stream);
  gb::mlp_free(T->m);
  delete T;
}

// Forward + backward on n <= batch rows (device X [n][32] raw features, T [n][3]);
// gradient into the trainer's buffer; loss (mean squared error) to *loss_out if not NULL.
static int train_fwd_bwd(MlpTrainer* T, const float* X, const float* Tg, int n, float* loss_out) {
  using namespace gb;
  if (!T || !X || !Tg || n < 1 || n > T->batch) return tr_fail(SIM_ERR_INVALID_ARG, "mlp: bad batch");
  Mlp* m = T->m;
  cudaStream_t s = T->stream;
  size_t B = T->batch;
  float *Z1 = T->Z, *Z2 = T->Z + B * HID, *Z3 = T->Z + 2 * B * HID;
  __nv_bfloat16 *H1 = T->H, *H2 = T->H + B * HID, *H3 = T->H + 2 * B * HID;
  FwdOut fo = {Z1, Z2, Z3, T->X, H1, H2, H3, T->Y};
  int blocks = min((n + 63) / 64, 152 * 2 * 8);
  k_mlp_fwd<true><<<blocks, 128, SMEM_MLP, s>>>(m->w, X, nullptr, 0, 0, nullptr, n, fo);
  cudaMemsetAsync(T->loss, 0, sizeof(float), s);
  k_mse_grad<<<min((n * 8 + 255) / 256, 1024), 256, 0, s>>>(T->Y, Tg, n, T->dY, T->loss);
  float* G = T->grad;
  auto gemm = [&](int M, int N, int K, const __nv_bfloat16* A, int lda, int at, const __nv_bfloat16* Bm, int ldb,
                  int bt, float* Cm, int ldc) {
    dim3 grid((N + 63) / 64, (M + 63) / 64);
    k_gemm<<<grid, 128, 0, s>>>(M, N, K, A, lda, at, Bm, ldb, bt, Cm, ldc);
  };
  // layer 4: dW4 = dY^T H3, db4 = sum dY, dH3 = dY W4
  gemm(NOUT, HID, n, T->dY, 8, 1, H3, HID, 0, G + OFF_W4, HID);
  k_colsum<<<NOUT, 256, 0, s>>>(T->dY, n, 8, NOUT, G + OFF_B4);
  gemm(n, HID, 8, T->dY, 8, 0, m->w.W4, LDH, 0, T->dH, HID);
  const int offW[3] = {OFF_W1, OFF_W2, OFF_W3}, offB[3] = {OFF_B1, OFF_B2, OFF_B3};
  __nv_bfloat16* Ws[3] = {m->w.W1, m->w.W2, m->w.W3};
  float* Zs[3] = {Z1, Z2, Z3};
  __nv_bfloat16* Hin[3] = {T->X, H1, H2};
  for (int l = 2; l >= 0; --l) {
    unsigned nb = (unsigned)(((size_t)n * HID + 255) / 256);
    k_gelu_back<<<nb, 256, 0, s>>>(T->dH, Zs[l], n, T->dZ);
    int nin = l == 0 ? NIN : HID;
    gemm(HID, nin, n, T->dZ, HID, 1, Hin[l], nin, 0, G + offW[l], nin);
    k_colsum<<<HID, 256, 0, s>>>(T->dZ, n, HID, HID, G + offB[l]);
    if (l > 0) gemm(n, HID, HID, T->dZ, HID, 0, Ws[l], LDH, 0, T->dH, HID);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return tr_fail(SIM_ERR_CUDA, std::string("mlp train: ") + cudaGetErrorString(e));
  if (loss_out) {
    float l = 0.f;
    e = cudaMemcpyAsync(&l, T->loss, sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return tr_fail(SIM_ERR_CUDA, cudaGetErrorString(e));
    *loss_out = l / (3.f * n);
  }
  return SIM_OK;
}

int mlp_loss_grad(MlpTrainer* T, const float* X, const float* Tg, int n, float* grad_out, float* loss_out) {
  int r = train_fwd_bwd(T, X, Tg, n, loss_out);
  if (r) return r;
  if (grad_out) {
    cudaError_t e = cudaMemcpyAsync(grad_out, T->grad, sizeof(float) * gb::MLP_NPARAM, cudaMemcpyDeviceToDevice, T->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(T->stream);
    if (e != cudaSuccess) return tr_fail(SIM_ERR_CUDA, cudaGetErrorString(e));
  }
  return SIM_OK;
}

int mlp_train_step(MlpTrainer* T, const float* X, const float* Tg, int n, float lr, float* loss_out) {
  using namespace gb;
  int r = train_fwd_bwd(T, X, Tg, n, loss_out);
  if (r) return r;
  T->t += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  float c1 = 1.f - powf(b1, (float)T->t), c2 = 1.f - powf(b2, (float)T->t);
  k_adam<<<(MLP_NPARAM + 255) / 256, 256, 0, T->stream>>>(T->m->params, T->grad, T->am, T->av, MLP_NPARAM, lr, b1, b2,
                                                         1e-8f, c1, c2);
  mlp_repack(T->m, T->stream);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return tr_fail(SIM_ERR_CUDA, cudaGetErrorString(e));
  return SIM_OK;
}

// Forward only (inference kernel in training layout) on n rows: Y[n][3] (device).
int mlp_forward(MlpTrainer* T, const float* X, int n, float* Y) {
  using namespace gb;
  if (!T || !X || !Y || n < 1 || n > T->batch) return tr_fail(SIM_ERR_INVALID_ARG, "mlp_forward: bad argument");
  size_t B = T->batch;
  FwdOut fo = {T->Z, T->Z + B * HID, T->Z + 2 * B * HID, T->X, T->H, T->H + B * HID, T->H + 2 * B * HID, Y};
  int blocks = min((n + 63) / 64, 152 * 2 * 8);
  k_mlp_fwd<true><<<blocks, 128, SMEM_MLP, T->stream>>>(T->m->w, X, nullptr, 0, 0, nullptr, n, fo);
  cudaError_t e = cudaStreamSynchronize(T->stream);
  if (e != cudaSuccess) return tr_fail(SIM_ERR_CUDA, cudaGetErrorString(e));
  return SIM_OK;
}

// Parameters for raw (unnormalised) features: W1 / std per input column and
// b1 - W1 (mean / std) folded in, FP32 flat layout, into params_out (host or device).
int mlp_get_params(MlpTrainer* T, float* params_out, int to_device) {
  using namespace gb;
  if (!T || !params_out) return tr_fail(SIM_ERR_INVALID_ARG, "mlp_get_params: NULL argument");
  std::vector<float> P(MLP_NPARAM), mean(NIN), inv(NIN);
  cudaError_t e = cudaMemcpyAsync(P.data(), T->m->params, sizeof(float) * MLP_NPARAM, cudaMemcpyDeviceToHost, T->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(mean.data(), T->m->w.mean, sizeof(float) * NIN, cudaMemcpyDeviceToHost, T->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(inv.data(), T->m->w.invstd, sizeof(float) * NIN, cudaMemcpyDeviceToHost, T->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(T->stream);
  if (e != cudaSuccess) return tr_fail(SIM_ERR_CUDA, cudaGetErrorString(e));
  for (int o = 0; o < HID; ++o) {
    double shift = 0.0;
    for (int i = 0; i < NIN; ++i) {
      float w = P[OFF_W1 + o * NIN + i] * inv[i];
      P[OFF_W1 + o * NIN + i] = w;
      shift += (double)w * mean[i];
    }
    P[OFF_B1 + o] = (float)(P[OFF_B1 + o] - shift);
  }
  e = cudaMemcpy(params_out, P.data(), sizeof(float) * MLP_NPARAM, to_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost);
  if (e != cudaSuccess) return tr_fail(SIM_ERR_CUDA, cudaGetErrorString(e));
  return SIM_OK;
}

}  // extern "C"
