// Articulated-body kernels: one warp per multi-joint articulation (aba_multi),
// one thread per single-joint articulation (aba_single), and the forward
// kinematics the collision kernel reads (fk_multi, fk_single); the device code is
// in aba.cuh.
#include "aba.cuh"

namespace gb {

template <int G>
__global__ void __launch_bounds__(128, 7) k_aba(Dev d) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int lane = threadIdx.x & 31;
  const int gl = lane & (G - 1), g0 = lane & ~(G - 1);
  const unsigned gm = G == 32 ? 0xffffffffu : (((1u << (G & 31)) - 1u) << g0);
  const int grp = threadIdx.x / G;
  const int slot = blockIdx.x * (blockDim.x / G) + grp;
  if (slot >= d.n_art_multi) return;
  aba_multi<G>(d, d.art_multi[slot], gl, gm, reinterpret_cast<AbaSh*>(sm_raw)[grp]);
}

__global__ void __launch_bounds__(256) k_aba1(Dev d) {
  int slot = blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= d.n_art_single) return;
  aba_single(d, d.art_single[slot]);
}

// forward kinematics: blocks 0 .. nb_multi-1 take the multi-joint articulations (a
// 16-lane group each, 8 per block), the rest the single-joint ones (a thread each)
__global__ void __launch_bounds__(128) k_fk(Dev d, int nb_multi) {
  __shared__ FkSh sh[8];
  if ((int)blockIdx.x < nb_multi) {
    const int lane = threadIdx.x & 31;
    const int gl = lane & 15, g0 = lane & ~15;
    const unsigned gm = 0xffffu << g0;
    const int slot = blockIdx.x * 8 + threadIdx.x / 16;
    if (slot < d.n_art_multi) fk_multi<16>(d, d.art_multi[slot], gl, gm, sh[threadIdx.x / 16]);
  } else {
    const int slot = (blockIdx.x - nb_multi) * 128 + threadIdx.x;
    if (slot < d.n_art_single) fk_single(d, d.art_single[slot]);
  }
}

void launch_fk(const Dev& d, cudaStream_t st) {
  const int nb_multi = (d.n_art_multi + 7) / 8, nb_single = (d.n_art_single + 127) / 128;
  if (nb_multi + nb_single > 0) k_fk<<<nb_multi + nb_single, 128, 0, st>>>(d, nb_multi);
}

void configure_aba() {
  cudaFuncSetAttribute(k_aba<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(sizeof(AbaSh) * 4));
  cudaFuncSetAttribute(k_aba<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(sizeof(AbaSh) * 8));
}

// lanes: 32 (one articulation per warp) or 16 (two per warp); 4 warps per block
void launch_aba(const Dev& d, cudaStream_t st, int lanes) {
  if (d.n_art_multi > 0) {
    const int per_block = lanes == 16 ? 8 : 4;
    const int blocks = (d.n_art_multi + per_block - 1) / per_block;
    if (lanes == 16) k_aba<16><<<blocks, 128, sizeof(AbaSh) * per_block, st>>>(d);
    else k_aba<32><<<blocks, 128, sizeof(AbaSh) * per_block, st>>>(d);
  }
  if (d.n_art_single > 0) k_aba1<<<(d.n_art_single + 255) / 256, 256, 0, st>>>(d);
}

}  // namespace gb
