// Learned warm start: per-contact MLP 32 -> 128 -> 128 -> 128 -> 3 (GELU),
// BF16 weights and activations, FP32 accumulation.
//
// Parameters arrive in FP32 (W1[128][32] b1 W2[128][128] b2 W3[128][128] b3
// W4[3][128] b4); weights are stored on the device in BF16, biases in FP32.
#include <cuda_bf16.h>

#include <string>

#include "sim_internal.cuh"

namespace gb {

constexpr int MLP_NPARAM = 128 * 32 + 128 + 128 * 128 + 128 + 128 * 128 + 128 + 3 * 128 + 3;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + 128 * 32, OFF_W2 = OFF_B1 + 128, OFF_B2 = OFF_W2 + 128 * 128,
              OFF_W3 = OFF_B2 + 128, OFF_B3 = OFF_W3 + 128 * 128, OFF_W4 = OFF_B3 + 128, OFF_B4 = OFF_W4 + 3 * 128;

struct Mlp {
  __nv_bfloat16* w;  // all parameters in BF16 (biases unused in this copy)
  float* p;          // all parameters in FP32 (biases read from here)
};

__global__ void k_to_bf16(const float* src, __nv_bfloat16* dst, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = __float2bfloat16_rn(src[i]);
}

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float bfr(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// One thread per contact; activations rounded to BF16 between layers.
__global__ void k_mlp_simple(Dev d, const __nv_bfloat16* W, const float* P) {
  long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
  long total = (long)d.E * d.C;
  if (idx >= total) return;
  int e = (int)(idx / d.C), i = (int)(idx % d.C);
  if (i >= d.n_contacts[e]) return;
  float x[128], h[128];
  const float* f = d.feat + idx * NFEAT;
  for (int k = 0; k < 32; ++k) x[k] = bfr(f[k]);
  const int offs[3][2] = {{OFF_W1, OFF_B1}, {OFF_W2, OFF_B2}, {OFF_W3, OFF_B3}};
  int nin = 32;
  for (int l = 0; l < 3; ++l) {
    for (int o = 0; o < 128; ++o) {
      float s = 0.f;
      for (int k = 0; k < nin; ++k) s += __bfloat162float(W[offs[l][0] + o * nin + k]) * x[k];
      h[o] = bfr(gelu(s + P[offs[l][1] + o]));
    }
    for (int o = 0; o < 128; ++o) x[o] = h[o];
    nin = 128;
  }
  float y[3];
  for (int o = 0; o < 3; ++o) {
    float s = 0.f;
    for (int k = 0; k < 128; ++k) s += __bfloat162float(W[OFF_W4 + o * 128 + k]) * x[k];
    y[o] = s + P[OFF_B4 + o];
  }
  d.pred[idx] = make_float4(y[0], y[1], y[2], 0.f);
}

void* mlp_create(const float* params, int on_device, cudaStream_t s, std::string& err) {
  Mlp* m = new Mlp();
  if (cudaMalloc((void**)&m->p, sizeof(float) * MLP_NPARAM) != cudaSuccess ||
      cudaMalloc((void**)&m->w, sizeof(__nv_bfloat16) * MLP_NPARAM) != cudaSuccess) {
    err = "allocation failed";
    delete m;
    return nullptr;
  }
  cudaMemcpyAsync(m->p, params, sizeof(float) * MLP_NPARAM, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s);
  k_to_bf16<<<(MLP_NPARAM + 255) / 256, 256, 0, s>>>(m->p, m->w, MLP_NPARAM);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    err = cudaGetErrorString(e);
    return nullptr;
  }
  return m;
}

void mlp_destroy(void* p) {
  Mlp* m = (Mlp*)p;
  if (!m) return;
  cudaFree(m->p);
  cudaFree(m->w);
  delete m;
}

void launch_mlp_infer(const Dev& d, const void* mlp, cudaStream_t s) {
  const Mlp* m = (const Mlp*)mlp;
  long total = (long)d.E * d.C;
  if (total == 0) return;
  k_mlp_simple<<<(unsigned)((total + 127) / 128), 128, 0, s>>>(d, m->w, m->p);
}

}  // namespace gb
