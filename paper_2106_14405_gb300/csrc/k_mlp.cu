// Learned warm start: per-contact MLP 32 -> 128 -> 128 -> 128 -> 3 with GELU
// (exact erf form), BF16 weights and activations, FP32 accumulation.
//
// Forward (inference and training, k_mlp_tc): layers 1-3 on the 5th-generation
// tensor cores -- tcgen05.mma (kind::f16, M = N = 128) from shared-memory
// operands into a TMEM accumulator, read back with tcgen05.ld -- one 128-row tile
// per block; inference runs over the contacts the row kernel lists (those without a
// prior-frame match and the fast matched ones, the only ones whose warm start uses the
// network).  Training: the forward stores Z (pre-activation, FP32)
// and H (BF16) per layer; the backward pass is a BF16 GEMM on the same tensor
// cores (k_gemm, 128 x 128 tiles) plus elementwise kernels (MSE gradient, GELU',
// bias sums) and Adam on FP32 master weights.
//
// Parameter layout (FP32, shared with the CPU reference): W1[128][32] b1[128]
// W2[128][128] b2[128] W3[128][128] b3[128] W4[3][128] b4[3].
#include <cuda_bf16.h>

#include <algorithm>
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
// In-step inference limits each finite output to the range of the training targets
// (+-10 units of learn_scale); beyond it the network extrapolates, and an
// extrapolated correction on a contact with a large effective mass is an impulse
// that a fixed number of sweeps cannot undo.  Non-finite outputs pass through, so
// that the solver falls back to the prior-frame impulse.
constexpr float PRED_LIMIT = 10.f;
constexpr int LDH = HID + 8;   // padded row length of W2, W3, W4
constexpr int GEMM_SPLITS = 32;  // most K splits of a training GEMM

// device weights: BF16 padded, biases FP32 (b4 padded to 8), input normalisation
struct MlpDev {
  __nv_bfloat16 *W1, *W2, *W3, *W4;  // [128][40], [128][136], [128][136], [8][136]
  float *b1, *b2, *b3, *b4;          // [128] x3, [8]
  float *mean, *invstd;              // [32]
};


__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}
__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
// In-step inference: GELU by its tanh form, 0.5 x (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3)))
// (Hendrycks & Gimpel 2016), with the hardware tanh approximation: the tanh form
// departs from the erf form by at most 4.7e-4 (at x = 2.7), the approximation adds a
// few 1e-4 of x, both below the BF16 rounding (2^-8 relative) of the activations it
// feeds; training and the FP64 reference keep the erf form.
__device__ __forceinline__ float gelu_infer(float x) {
  const float u = 0.7978845608028654f * fmaf(0.044715f * x, x * x, x);
  float th;
  asm("tanh.approx.f32 %0, %1;" : "=f"(th) : "f"(u));
  return 0.5f * x * (1.f + th);
}
__device__ __forceinline__ float gelu_grad(float x) {
  return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * expf(-0.5f * x * x) * 0.39894228040143267794f;
}

struct FwdOut {       // training-mode outputs (nullptr in inference)
  float *Z1, *Z2, *Z3;  // [n][128]
  __nv_bfloat16 *X, *H1, *H2, *H3;  // [n][32], [n][128] x3
  float* Y;           // [n][3]
};

// ---------------------------------------------------------------------------
// Forward on the 5th-generation tensor cores (tcgen05): one 512-thread block per
// 128-row tile at a time; threads m, m + 128, m + 256 and m + 384 share row m = TMEM
// lane m (warps w, w + 4, w + 8 and w + 12 read the same TMEM lane quarter) and take
// a quarter of the columns each, so every epilogue (bias, GELU, BF16 packing) is
// spread over four threads per row.  Layers 1-3 are D = A W^T with
// M = N = 128 (K = 32, 128): A (activations) and W (weights) in shared memory in
// the no-swizzle K-major core-matrix layout (8 rows x 16 bytes per core matrix;
// element (r, k) of a K-column matrix at (r/8)*16K + (k/8)*128 + (r%8)*16 +
// (k%8)*2 bytes), the FP32 accumulator in 128 TMEM columns; one thread issues the
// K/16 MMAs and commits them to an mbarrier; every thread then reads its row
// from TMEM (tcgen05.ld, 32 columns at a time), adds the bias, applies GELU and
// writes the BF16 activations back into the A buffer for the next layer (the
// MMAs that read it have completed).  Layer 4 (3 outputs) is a dot product per
// row on the CUDA cores from the BF16 activations, each thread's quarter summed
// into the first quarter's through shared memory (the A buffer beyond the 8 KB
// that the next tile's layer-1 input occupies: free from the last layer's
// completion until the next tile's first epilogue).  Every wait is bounded: on a
// timeout the block flags it (environment status bit / trainer flag), skips the
// rest and frees its TMEM.
// ---------------------------------------------------------------------------
constexpr int TC_ROWS = 128, TC_PARTS = 4, TC_THREADS = TC_ROWS * TC_PARTS;
constexpr int TC_COLS = HID / TC_PARTS;  // epilogue columns per thread: one 32-column TMEM load
constexpr size_t TC_W1 = 0, TC_W2 = TC_W1 + 128 * 32 * 2, TC_W3 = TC_W2 + 128 * 128 * 2,
                 TC_A = TC_W3 + 128 * 128 * 2, TC_W4 = TC_A + 128 * 128 * 2, TC_B = TC_W4 + 3 * HID * 4,
                 TC_BAR = TC_B + (3 * HID + 8 + 2 * NIN) * 4, SMEM_TC = TC_BAR + 16;
// layer-4 partial sums of quarters 1..3 ([3][128][4] floats) inside the A buffer,
// after the K = 32 layer-1 input (128 x 32 BF16)
constexpr size_t TC_Y_IN_A = 128 * 32 * 2;
static_assert(TC_COLS == 32 && NIN / 8 == TC_PARTS, "one TMEM load and one input chunk per thread");
static_assert(TC_Y_IN_A + (TC_PARTS - 1) * TC_ROWS * 4 * 4 <= 128 * 128 * 2, "partial sums fit in the A buffer");
constexpr uint32_t TC_TMEM_COLS = 128;
constexpr unsigned long long TC_WAIT_NS = 500000000ull;  // a completion wait gives up after 0.5 s
constexpr unsigned long long TC_WAIT_POLLS = 1ull << 26; // and after this many polls in any case

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: no swizzle, K-major; start, leading (K) and
// stride (row-group) byte offsets; descriptor version 1
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both K-major, N = M = 128
constexpr uint32_t TC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((128u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(TC_IDESC), "r"(acc));
}
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool tc_wait(uint32_t bar, uint32_t parity) {
  const unsigned long long t0 = globaltimer_ns();
  for (unsigned long long it = 0; it < TC_WAIT_POLLS; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (globaltimer_ns() - t0 > TC_WAIT_NS) return false;
  }
  return false;
}
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16-byte chunk j (columns 8j..8j+7) of row r of a K-column core-matrix-layout matrix
__device__ __forceinline__ uint4* tc_chunk(unsigned char* base, int r, int j, int K) {
  return reinterpret_cast<uint4*>(base + (size_t)(r >> 3) * (16 * K) + j * 128 + (r & 7) * 16);
}

template <bool TRAIN>
__global__ void __launch_bounds__(TC_THREADS, 2) k_mlp_tc(MlpDev w, const float* feat, int C, float4* pred,
                                                       const int* rows, const int* n_list, int* env_status, int n_rows,
                                                       FwdOut out, int* err, int hold) {
  extern __shared__ __align__(1024) unsigned char smt[];
  const int t = threadIdx.x, warp = t >> 5;
  const int m = t & (TC_ROWS - 1), part = t >> 7;  // row (TMEM lane) and column quarter
  const int nrows = TRAIN ? n_rows : *n_list;
  const int ntiles = (nrows + TC_ROWS - 1) / TC_ROWS;
  if ((int)blockIdx.x >= ntiles) return;  // no tile for this block: skip the weight staging
  unsigned char* sW1 = smt + TC_W1;
  unsigned char* sW2 = smt + TC_W2;
  unsigned char* sW3 = smt + TC_W3;
  unsigned char* sA = smt + TC_A;
  float* sW4 = reinterpret_cast<float*>(smt + TC_W4);
  float* sb = reinterpret_cast<float*>(smt + TC_B);  // b1 b2 b3 b4(8) mean invstd
  float* sy = reinterpret_cast<float*>(sA + TC_Y_IN_A);  // [3][128][4]: quarters 1-3's layer-4 partial sums
  uint64_t* bar = reinterpret_cast<uint64_t*>(smt + TC_BAR);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smt + TC_BAR + 8);
  // ---- weights into the core-matrix layout (16-byte chunks), biases, normalisation
  for (int i = t; i < 128 * 4; i += TC_THREADS) {
    const int n = i >> 2, j = i & 3;
    *tc_chunk(sW1, n, j, 32) = *reinterpret_cast<const uint4*>(w.W1 + (size_t)n * LD1 + 8 * j);
  }
  for (int i = t; i < 128 * 16; i += TC_THREADS) {
    const int n = i >> 4, j = i & 15;
    *tc_chunk(sW2, n, j, 128) = *reinterpret_cast<const uint4*>(w.W2 + (size_t)n * LDH + 8 * j);
    *tc_chunk(sW3, n, j, 128) = *reinterpret_cast<const uint4*>(w.W3 + (size_t)n * LDH + 8 * j);
  }
  for (int i = t; i < 3 * HID; i += TC_THREADS) sW4[i] = __bfloat162float(w.W4[(size_t)(i / HID) * LDH + i % HID]);
  for (int i = t; i < HID; i += TC_THREADS) {
    sb[i] = w.b1[i]; sb[HID + i] = w.b2[i]; sb[2 * HID + i] = w.b3[i];
  }
  if (t < 8) sb[3 * HID + t] = w.b4[t];
  if (t < NIN) { sb[3 * HID + 8 + t] = w.mean[t]; sb[3 * HID + 8 + NIN + t] = w.invstd[t]; }
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(TC_TMEM_COLS) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t tl = tmem + ((uint32_t)((warp & 3) * 32) << 16);  // this warp's 32 lanes
  const uint32_t ubar = smem_u32(bar), uA = smem_u32(sA), uW1 = smem_u32(sW1), uW2 = smem_u32(sW2), uW3 = smem_u32(sW3);
  const float* smean = sb + 3 * HID + 8;
  const float* sinv = smean + NIN;
  uint32_t phase = 0;
  bool ok = true;
  int fail_tile = 0;
  for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
    fail_tile = tile;
    // ---- this thread's row: a training row, or entry tile * 128 + m of the list of
    //      contact rows (e * C + slot) the network runs on
    int row = -1;
    if (tile * TC_ROWS + m < nrows) row = TRAIN ? tile * TC_ROWS + m : rows[tile * TC_ROWS + m];
    // ---- layer 1 input: normalised features, BF16, K = 32 (each quarter one of the
    //      four 16-byte chunks of its row: two 16-byte loads of its eight features)
    {
      const int j = part;
      float4 xa = make_float4(0.f, 0.f, 0.f, 0.f), xb = xa;
      if (row >= 0) {
        const float4* x4 = reinterpret_cast<const float4*>(feat + (size_t)row * NIN + 8 * j);
        xa = x4[0];
        xb = x4[1];
      }
      const float4 ma = *reinterpret_cast<const float4*>(smean + 8 * j), mb = *reinterpret_cast<const float4*>(smean + 8 * j + 4);
      const float4 ia = *reinterpret_cast<const float4*>(sinv + 8 * j), ib = *reinterpret_cast<const float4*>(sinv + 8 * j + 4);
      const float xs[8] = {xa.x, xa.y, xa.z, xa.w, xb.x, xb.y, xb.z, xb.w};
      const float ms[8] = {ma.x, ma.y, ma.z, ma.w, mb.x, mb.y, mb.z, mb.w};
      const float is[8] = {ia.x, ia.y, ia.z, ia.w, ib.x, ib.y, ib.z, ib.w};
      float f[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) f[q] = row >= 0 ? (xs[q] - ms[q]) * is[q] : 0.f;
      uint4 v = make_uint4(pack2(f[0], f[1]), pack2(f[2], f[3]), pack2(f[4], f[5]), pack2(f[6], f[7]));
      *tc_chunk(sA, m, j, 32) = v;
      if (TRAIN && row >= 0) *reinterpret_cast<uint4*>(out.X + (size_t)row * NIN + 8 * j) = v;
    }
    float y[3] = {0.f, 0.f, 0.f};
#pragma unroll 1
    for (int layer = 0; layer < 3; ++layer) {
      const int K = layer == 0 ? 32 : 128;
      fence_async_smem();
      tc_fence_before();
      __syncthreads();
      if (t == 0) {
        tc_fence_after();
        const uint32_t uW = layer == 0 ? uW1 : (layer == 1 ? uW2 : uW3);
        for (int s = 0; s < K / 16; ++s)
          tc_mma(tmem, tc_desc(uA + 256 * s, 128, 16 * K), tc_desc(uW + 256 * s, 128, 16 * K), s > 0);
        if (!hold) tc_commit(ubar);  // hold: testing the bounded wait
      }
      if (!__syncthreads_and(tc_wait(ubar, phase))) { ok = false; break; }  // one decision for the block
      phase ^= 1u;
      tc_fence_after();
      // epilogue: bias + GELU, BF16 into the A buffer (K = 128 layout) or, after
      // layer 3, the output dot products
      const float* bias = sb + layer * HID;
      float* Zo = layer == 0 ? out.Z1 : (layer == 1 ? out.Z2 : out.Z3);
      __nv_bfloat16* Ho = layer == 0 ? out.H1 : (layer == 1 ? out.H2 : out.H3);
      {
        const int cb = part;  // this quarter's 32 columns
        float v[32];
        tc_ld32(tl + 32 * cb, v);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float4 ba = *reinterpret_cast<const float4*>(bias + 32 * cb + 8 * j);
          const float4 bb = *reinterpret_cast<const float4*>(bias + 32 * cb + 8 * j + 4);
          const float bs[8] = {ba.x, ba.y, ba.z, ba.w, bb.x, bb.y, bb.z, bb.w};
          float h[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int c = 32 * cb + 8 * j + q;
            const float z = v[8 * j + q] + bs[q];
            if (TRAIN && row >= 0) Zo[(size_t)row * HID + c] = z;
            h[q] = TRAIN ? gelu(z) : gelu_infer(z);
          }
          const uint4 hv = make_uint4(pack2(h[0], h[1]), pack2(h[2], h[3]), pack2(h[4], h[5]), pack2(h[6], h[7]));
          if (TRAIN && row >= 0) *reinterpret_cast<uint4*>(Ho + (size_t)row * HID + 32 * cb + 8 * j) = hv;
          if (layer < 2) {
            *tc_chunk(sA, m, 4 * cb + j, 128) = hv;
          } else {
            const __nv_bfloat16* hb = reinterpret_cast<const __nv_bfloat16*>(&hv);
            float hq[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) hq[q] = __bfloat162float(hb[q]);
#pragma unroll
            for (int o = 0; o < 3; ++o) {  // each output's sum in column order
              const float4 wa = *reinterpret_cast<const float4*>(sW4 + o * HID + 32 * cb + 8 * j);
              const float4 wb = *reinterpret_cast<const float4*>(sW4 + o * HID + 32 * cb + 8 * j + 4);
              const float w8[8] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
#pragma unroll
              for (int q = 0; q < 8; ++q) y[o] += hq[q] * w8[q];
            }
          }
        }
      }
    }
    if (!ok) break;
    // layer 4: quarters 1-3's partial sums to shared memory, added to the first's
    if (part) {
      float* q = sy + (size_t)(part - 1) * TC_ROWS * 4 + 4 * m;
      q[0] = y[0]; q[1] = y[1]; q[2] = y[2];
    }
    __syncthreads();
    if (!part && row >= 0) {
      const float* b4 = sb + 3 * HID;
      const float* q1 = sy + 4 * m;
      const float* q2 = q1 + TC_ROWS * 4;
      const float* q3 = q2 + TC_ROWS * 4;
      const float o0 = ((y[0] + q1[0]) + (q2[0] + q3[0])) + b4[0], o1 = ((y[1] + q1[1]) + (q2[1] + q3[1])) + b4[1],
                  o2 = ((y[2] + q1[2]) + (q2[2] + q3[2])) + b4[2];
      if (TRAIN) {
        out.Y[(size_t)row * 3 + 0] = o0; out.Y[(size_t)row * 3 + 1] = o1; out.Y[(size_t)row * 3 + 2] = o2;
      } else {
        auto lim = [](float o) { return isfinite(o) ? fminf(PRED_LIMIT, fmaxf(-PRED_LIMIT, o)) : o; };
        pred[row] = make_float4(lim(o0), lim(o1), lim(o2), 0.f);
      }
    }
    // (the next tile's layer-1 input stays below sy; its first barrier orders these
    //  reads before the first epilogue overwrites the A buffer)
  }
  if (!ok) {
    // a wait gave up: wait once more (bounded) for the MMAs in flight, then flag the
    // environments of this block's unfinished tiles (or the trainer's flag)
    tc_wait(ubar, phase);
    if (TRAIN) {
      if (t == 0) atomicOr(err, 1);
    } else {
      for (int t2 = fail_tile; t2 < ntiles && !part; t2 += gridDim.x)
        if (t2 * TC_ROWS + m < nrows) atomicOr(&env_status[rows[t2 * TC_ROWS + m] / C], ST_DEVICE_WAIT);
    }
  }
  // ---- free the TMEM (after every thread's reads and the last MMA)
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS) : "memory");
  }
}


// ---------------------------------------------------------------------------
// C[M x N] (FP32, row-major, ldc) = op(A)[M x K] * op(B)[K x N], BF16 operands:
// A(m, k) = A[a_t ? k * lda + m : m * lda + k], B(k, n) = B[b_t ? n * ldb + k : k * ldb + n].
// tcgen05: one 128 x 128 output tile per block, K steps of 64 (four kind::f16
// MMAs, FP32 accumulator in TMEM).  Both operands are staged into the K-major
// core-matrix layout through registers (the operand of B is its N x K
// transpose): a row with contiguous K by 16-byte loads, a transposed one read
// coalesced along M (N) by the threads and written element by element; rows,
// columns and K beyond the matrix are zero.  Bounded waits as in k_mlp_tc.
// ---------------------------------------------------------------------------
constexpr size_t GT_A = 0, GT_B = 128 * 64 * 2, GT_BAR = GT_B + 128 * 64 * 2, SMEM_GT = GT_BAR + 16;

// rows r0..r0+127 x k0..k0+63 of an operand X(r, k) = X[t ? k * ld + r : r * ld + k] (R rows, K columns)
__device__ __forceinline__ void gt_stage(unsigned char* dst, const __nv_bfloat16* X, int ld, int t, int R, int K,
                                         int r0, int k0) {
  const int i = threadIdx.x;
  if (!t) {
    const int r = r0 + i;
#pragma unroll 1
    for (int j = 0; j < 8; ++j) {
      const int k = k0 + 8 * j;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (r < R) {
        if (k + 8 <= K && ((((size_t)r * ld + k) & 7) == 0) && ((reinterpret_cast<uintptr_t>(X) & 15) == 0)) {
          v = *reinterpret_cast<const uint4*>(X + (size_t)r * ld + k);
        } else {
          __nv_bfloat16 e[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) e[q] = k + q < K ? X[(size_t)r * ld + k + q] : __float2bfloat16_rn(0.f);
          v = *reinterpret_cast<const uint4*>(e);
        }
      }
      *tc_chunk(dst, i, j, 64) = v;
    }
  } else {
    // thread i: rows 8 (i % 16) .. +7 of the tile at columns kk = 8 it + i / 16 -- one
    // 16-byte load of 8 consecutive rows (contiguous in X) per column, 8 columns per
    // thread, scattered into the layout
    const int rg = i & 15, kq = i >> 4;
    const int r = r0 + 8 * rg;
    __nv_bfloat16* d = reinterpret_cast<__nv_bfloat16*>(dst);
    const bool vec = r + 8 <= R && ((ld & 7) == 0) && ((reinterpret_cast<uintptr_t>(X) & 15) == 0);
#pragma unroll 2
    for (int it = 0; it < 8; ++it) {
      const int kk = 8 * it + kq, k = k0 + kk;
      __nv_bfloat16 e[8];
      if (k < K && vec) {
        *reinterpret_cast<uint4*>(e) = *reinterpret_cast<const uint4*>(X + (size_t)k * ld + r);
      } else {
#pragma unroll
        for (int q = 0; q < 8; ++q) e[q] = (k < K && r + q < R) ? X[(size_t)k * ld + r + q] : __float2bfloat16_rn(0.f);
      }
#pragma unroll
      for (int q = 0; q < 8; ++q)  // tile row 8 rg + q: row group rg, row q within it
        d[((size_t)rg * (16 * 64) + (kk >> 3) * 128 + q * 16 + (kk & 7) * 2) / 2] = e[q];
    }
  }
}

// Split K: block z sums K range [z kchunk, (z + 1) kchunk) into its own partial output
// C + z M ldc (gridDim.z = 1: the whole K into C); k_sum_splits then adds the partials.
__global__ void __launch_bounds__(128) k_gemm(int M, int N, int K, int kchunk, const __nv_bfloat16* A, int lda,
                                              int a_t, const __nv_bfloat16* B, int ldb, int b_t, float* C, int ldc,
                                              int* err) {
  extern __shared__ __align__(1024) unsigned char smg[];
  unsigned char* sA = smg + GT_A;
  unsigned char* sB = smg + GT_B;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smg + GT_BAR);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smg + GT_BAR + 8);
  const int m = threadIdx.x, warp = m >> 5;
  const int m0 = blockIdx.y * 128, n0 = blockIdx.x * 128;
  if (m == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(TC_TMEM_COLS) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t ubar = smem_u32(bar), uA = smem_u32(sA), uB = smem_u32(sB);
  const int kbeg = blockIdx.z * kchunk, kend = min(K, kbeg + kchunk);
  C += (size_t)blockIdx.z * M * ldc;
  uint32_t phase = 0;
  bool ok = true;
  for (int k0 = kbeg; k0 < kend; k0 += 64) {
    gt_stage(sA, A, lda, a_t, M, kend, m0, k0);
    gt_stage(sB, B, ldb, !b_t, N, kend, n0, k0);  // B's operand row n, column k: B(k, n)
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (m == 0) {
      tc_fence_after();
      for (int s = 0; s < 4; ++s)
        tc_mma(tmem, tc_desc(uA + 256 * s, 128, 16 * 64), tc_desc(uB + 256 * s, 128, 16 * 64), (k0 > kbeg || s > 0));
      tc_commit(ubar);
    }
    if (!__syncthreads_and(tc_wait(ubar, phase))) { ok = false; break; }
    phase ^= 1u;
    tc_fence_after();
  }
  if (ok && kend <= kbeg) {  // an empty split: its partial is zero
    const int row = m0 + m;
    if (row < M)
      for (int n = n0; n < min(N, n0 + 128); ++n) C[(size_t)row * ldc + n] = 0.f;
  } else if (ok) {
    const int row = m0 + m;
    const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
    for (int cb = 0; cb < 4; ++cb) {
      float v[32];
      tc_ld32(tl + 32 * cb, v);
      if (row < M)
#pragma unroll
        for (int c = 0; c < 32; ++c) {
          const int n = n0 + 32 * cb + c;
          if (n < N) C[(size_t)row * ldc + n] = v[c];
        }
    }
  } else if (!ok) {
    tc_wait(ubar, phase);  // the MMAs in flight, bounded
    if (m == 0) atomicOr(err, 1);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS) : "memory");
  }
}

// C[m][n] = sum over z = 0 .. Z-1, in order, of the split partials P[z][m][n] (ld N)
__global__ void k_sum_splits(const float* P, int Z, int M, int N, float* C, int ldc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M * N) return;
  const int r = i / N, c = i % N;
  float acc = 0.f;
  for (int z = 0; z < Z; ++z) acc += P[(size_t)z * M * N + i];
  C[(size_t)r * ldc + c] = acc;
}

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
  int* err;       // set by a tensor-core forward whose bounded wait gave up (training)
  int grid = 0;   // persistent grid of the tensor-core forward
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
         dmalloc(m, &m->params, MLP_NPARAM) && dmalloc(m, &m->err, 1);
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
  cudaMemsetAsync(m->err, 0, sizeof(int), s);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_mlp_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_TC);
    cudaFuncSetAttribute(k_mlp_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_TC);
    cudaFuncSetAttribute(k_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_GT);
    // all of the unified L1 as shared memory: two 107 KB forward blocks per SM
    cudaFuncSetAttribute(k_mlp_tc<false>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    cudaFuncSetAttribute(k_mlp_tc<true>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    attr = true;
  }
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // resident blocks per SM: the occupancy calculator, or the shared-memory arithmetic
  // (the SM's shared memory over a block's, with the per-block reservation), at most two
  // (2 x 128 TMEM columns of the SM's 512 for the two forward blocks and headroom)
  int smem_sm = 0, reserved = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mlp_tc<false>, TC_THREADS, SMEM_TC);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  const int fit = smem_sm / (int)(SMEM_TC + (size_t)reserved);
  m->grid = std::max(1, sms * std::max(1, std::min(std::max(per_sm, fit), 2)));
  return m;
}

void mlp_destroy(void* p) {
  if (p) mlp_free((Mlp*)p);
}

// the tensor-core forward over the rows the row kernel listed (see LEARN_GATE)
void launch_mlp_infer(const Dev& d, const void* mlp, cudaStream_t s) {
  const Mlp* m = (const Mlp*)mlp;
  if (d.E == 0) return;
  FwdOut none = {};
  k_mlp_tc<false><<<m->grid, TC_THREADS, SMEM_TC, s>>>(m->w, d.feat, d.C, d.pred, d.mlp_rows, d.mlp_count, d.status, 0,
                                                none, m->err, d.hold_async);
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
  float* part;  // split-K partials of the weight-gradient GEMMs: [GEMM_SPLITS][128][128]
  __nv_bfloat16 *X, *H, *dY, *dZ;
  float* Y;
  long long t;
  std::string err;
};

namespace gb {
int report_error(int code, const std::string& msg);
}

static int tr_fail(int code, const std::string& msg) { return gb::report_error(code, msg); }

// after a stream synchronisation: a tensor-core forward whose bounded wait gave up
static int check_err(MlpTrainer* T) {
  int f = 0;
  cudaError_t e = cudaMemcpy(&f, T->m->err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return tr_fail(SIM_ERR_CUDA, cudaGetErrorString(e));
  if (f) {
    cudaMemset(T->m->err, 0, sizeof(int));
    return tr_fail(SIM_ERR_CUDA, "mlp: a tensor-core completion wait timed out");
  }
  return SIM_OK;
}

// ---------------------------------------------------------------------------
// Training-set preparation (the learned warm start's recipe, on the device)
// ---------------------------------------------------------------------------
namespace {
constexpr int SEL_ROWS = 256;  // rows per block of the selection

__device__ __forceinline__ bool row_selected(const float* X, const float* T, size_t i, int only_used, float gate) {
  const float* t = T + 3 * i;
  if (!(isfinite(t[0]) && isfinite(t[1]) && isfinite(t[2]))) return false;
  if (!only_used) return true;
  const float* f = X + i * gb::NIN;
  return f[26] == 0.f || sqrtf(f[9] * f[9] + f[10] * f[10] + f[11] * f[11]) > gate;
}

// WRITE = false: rows kept per block into cnt[block]; WRITE = true: the kept rows, in
// order, from row cnt[block] (exclusive prefix) on, targets clipped to [-clip, clip].
template <bool WRITE>
__global__ void __launch_bounds__(SEL_ROWS) k_select_rows(const float* X, const float* T, int n, int only_used,
                                                          float gate, float clip, int* cnt, float* Xo, float* To) {
  __shared__ int warp_tot[SEL_ROWS / 32];
  const size_t i = (size_t)blockIdx.x * SEL_ROWS + threadIdx.x;
  const bool keep = i < (size_t)n && row_selected(X, T, i, only_used, gate);
  const unsigned bal = __ballot_sync(0xffffffffu, keep);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) warp_tot[w] = __popc(bal);
  __syncthreads();
  int before = 0, total = 0;
  for (int k = 0; k < SEL_ROWS / 32; ++k) {
    before += k < w ? warp_tot[k] : 0;
    total += warp_tot[k];
  }
  if (!WRITE) {
    if (threadIdx.x == 0) cnt[blockIdx.x] = total;
    return;
  }
  if (!keep) return;
  const size_t o = (size_t)cnt[blockIdx.x] + before + __popc(bal & ((1u << lane) - 1u));
  for (int k = 0; k < gb::NIN; ++k) Xo[o * gb::NIN + k] = X[i * gb::NIN + k];
  for (int r = 0; r < 3; ++r) To[3 * o + r] = fmaxf(-clip, fminf(clip, T[3 * i + r]));
}

// Per-feature sums and sums of squares (FP64) of a fixed set of row strides: block b
// covers rows b*8 + j, stepping gridDim.x*8 (8 row lanes x 32 features per block);
// part[b][0..31] sums, part[b][32..63] sums of squares.
__global__ void __launch_bounds__(256) k_feature_partials(const float* X, int n, double* part) {
  __shared__ double sh[2][8][32];
  const int f = threadIdx.x & 31, j = threadIdx.x >> 5;
  double s = 0.0, q = 0.0;
  for (size_t r = (size_t)blockIdx.x * 8 + j; r < (size_t)n; r += (size_t)gridDim.x * 8) {
    const double x = X[r * gb::NIN + f];
    s += x;
    q += x * x;
  }
  sh[0][j][f] = s;
  sh[1][j][f] = q;
  __syncthreads();
  if (j == 0) {
    double ss = 0.0, qq = 0.0;
    for (int k = 0; k < 8; ++k) {
      ss += sh[0][k][f];
      qq += sh[1][k][f];
    }
    part[(size_t)blockIdx.x * 64 + f] = ss;
    part[(size_t)blockIdx.x * 64 + 32 + f] = qq;
  }
}
// One thread per feature: the partials in block order (deterministic) -> mean and
// population standard deviation (below 1e-6 reported as 1: a constant feature).
__global__ void k_feature_finish(const double* part, int blocks, int n, float* mean, float* sd) {
  const int f = threadIdx.x;
  if (f >= gb::NIN) return;
  double s = 0.0, q = 0.0;
  for (int b = 0; b < blocks; ++b) {
    s += part[(size_t)b * 64 + f];
    q += part[(size_t)b * 64 + 32 + f];
  }
  const double m = s / n;
  const double v = fmax(0.0, q / n - m * m);
  const double d = sqrt(v);
  mean[f] = (float)m;
  sd[f] = d < 1e-6 ? 1.f : (float)d;
}
constexpr int STAT_BLOCKS = 256;
}  // namespace

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
            dmalloc(m, &T->dZ, B * HID) && dmalloc(m, &T->Y, B * 3) &&
            dmalloc(m, &T->part, (size_t)GEMM_SPLITS * HID * HID);
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
  if (reinterpret_cast<uintptr_t>(X) & 15u) return tr_fail(SIM_ERR_INVALID_ARG, "mlp: X not 16-byte aligned");
  Mlp* m = T->m;
  cudaStream_t s = T->stream;
  size_t B = T->batch;
  float *Z1 = T->Z, *Z2 = T->Z + B * HID, *Z3 = T->Z + 2 * B * HID;
  __nv_bfloat16 *H1 = T->H, *H2 = T->H + B * HID, *H3 = T->H + 2 * B * HID;
  FwdOut fo = {Z1, Z2, Z3, T->X, H1, H2, H3, T->Y};
  k_mlp_tc<true><<<std::min((n + TC_ROWS - 1) / TC_ROWS, m->grid), TC_THREADS, SMEM_TC, s>>>(
      m->w, X, 0, nullptr, nullptr, nullptr, nullptr, n, fo, m->err, 0);
  cudaMemsetAsync(T->loss, 0, sizeof(float), s);
  k_mse_grad<<<min((n * 8 + 255) / 256, 1024), 256, 0, s>>>(T->Y, Tg, n, T->dY, T->loss);
  float* G = T->grad;
  // a single-tile output over a long K (the weight gradients, K = batch rows) is split
  // along K over up to GEMM_SPLITS blocks, its partials summed in order afterwards
  auto gemm = [&](int M, int N, int K, const __nv_bfloat16* A, int lda, int at, const __nv_bfloat16* Bm, int ldb,
                  int bt, float* Cm, int ldc) {
    int Z = (M <= 128 && N <= 128 && K > 512) ? std::min(GEMM_SPLITS, (K + 255) / 256) : 1;
    const int kchunk = Z > 1 ? ((K + Z - 1) / Z + 63) / 64 * 64 : K;
    if (Z > 1) Z = (K + kchunk - 1) / kchunk;
    dim3 grid((N + 127) / 128, (M + 127) / 128, Z);
    if (Z == 1) {
      k_gemm<<<grid, 128, SMEM_GT, s>>>(M, N, K, K, A, lda, at, Bm, ldb, bt, Cm, ldc, m->err);
    } else {
      k_gemm<<<grid, 128, SMEM_GT, s>>>(M, N, K, kchunk, A, lda, at, Bm, ldb, bt, T->part, N, m->err);
      k_sum_splits<<<(M * N + 255) / 256, 256, 0, s>>>(T->part, Z, M, N, Cm, ldc);
    }
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
    if (int r = check_err(T)) return r;
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
  if (reinterpret_cast<uintptr_t>(X) & 15u) return tr_fail(SIM_ERR_INVALID_ARG, "mlp_forward: X not 16-byte aligned");
  size_t B = T->batch;
  FwdOut fo = {T->Z, T->Z + B * HID, T->Z + 2 * B * HID, T->X, T->H, T->H + B * HID, T->H + 2 * B * HID, Y};
  k_mlp_tc<true><<<std::min((n + TC_ROWS - 1) / TC_ROWS, T->m->grid), TC_THREADS, SMEM_TC, T->stream>>>(
      T->m->w, X, 0, nullptr, nullptr, nullptr, nullptr, n, fo, T->m->err, 0);
  cudaError_t e = cudaStreamSynchronize(T->stream);
  if (e != cudaSuccess) return tr_fail(SIM_ERR_CUDA, cudaGetErrorString(e));
  return check_err(T);
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



int mlp_select_rows(const float* X, const float* T, int n, int only_used, float gate_speed, float clip, float* X_out,
                    float* T_out, int* n_out, void* cuda_stream) {
  if (!X || !T || !X_out || !T_out || !n_out || n < 0 || !(clip > 0.f) || !(gate_speed >= 0.f))
    return tr_fail(SIM_ERR_INVALID_ARG, "mlp_select_rows: bad argument");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const int blocks = (n + SEL_ROWS - 1) / SEL_ROWS;
  int* cnt = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&cnt, sizeof(int) * ((size_t)blocks + 1), s);
  if (e != cudaSuccess) return tr_fail(SIM_ERR_OOM, "mlp_select_rows: scratch");
  if (blocks) k_select_rows<false><<<blocks, SEL_ROWS, 0, s>>>(X, T, n, only_used, gate_speed, clip, cnt, nullptr, nullptr);
  gb::k_exclusive_scan<<<1, 1024, 0, s>>>(cnt, blocks);
  if (blocks) k_select_rows<true><<<blocks, SEL_ROWS, 0, s>>>(X, T, n, only_used, gate_speed, clip, cnt, X_out, T_out);
  e = cudaGetLastError();
  int kept = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&kept, cnt + blocks, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(cnt, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return tr_fail(SIM_ERR_CUDA, std::string("mlp_select_rows: ") + cudaGetErrorString(e));
  *n_out = kept;
  return SIM_OK;
}

int mlp_feature_stats(const float* X, int n, float* mean, float* std_out, int to_device, void* cuda_stream) {
  if (!X || !mean || !std_out || n < 1) return tr_fail(SIM_ERR_INVALID_ARG, "mlp_feature_stats: bad argument");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  double* part = nullptr;
  float* out = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&part, sizeof(double) * STAT_BLOCKS * 64, s);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&out, sizeof(float) * 2 * gb::NIN, s);
  if (e != cudaSuccess) {
    if (part) cudaFreeAsync(part, s);
    return tr_fail(SIM_ERR_OOM, "mlp_feature_stats: scratch");
  }
  k_feature_partials<<<STAT_BLOCKS, 256, 0, s>>>(X, n, part);
  k_feature_finish<<<1, 32, 0, s>>>(part, STAT_BLOCKS, n, out, out + gb::NIN);
  e = cudaGetLastError();
  const cudaMemcpyKind kind = to_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (e == cudaSuccess) e = cudaMemcpyAsync(mean, out, sizeof(float) * gb::NIN, kind, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(std_out, out + gb::NIN, sizeof(float) * gb::NIN, kind, s);
  cudaFreeAsync(part, s);
  cudaFreeAsync(out, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return tr_fail(SIM_ERR_CUDA, std::string("mlp_feature_stats: ") + cudaGetErrorString(e));
  return SIM_OK;
}

}  // extern "C"
