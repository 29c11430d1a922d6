// The whole step as one persistent launch (SimLaunchShape.fused): each warp takes an
// environment from a work queue and carries it through every stage of all n physics
// steps of a sim_step call -- link poses and forward dynamics of its articulations,
// collision, rows, projected Gauss-Seidel with integration and sleeping -- with no
// synchronisation between environments, which never interact, so no stage waits for
// the slowest environment of the batch and the n steps are one launch.  Every stage
// runs the same device code as the stage kernels.  Shared memory per warp holds the
// largest stage's working set and the stages use it in turn; the PGS layout's
// mbarrier (the row pool's bulk copy) is placed above every other stage's use of it.
// One register build (up to 128 registers, four resident 128-thread blocks per SM),
// whose results are those of the stage kernels bit for bit.  The learned warm start
// (its inference is one tensor-core tile over many environments' contacts) and kernel
// timing keep the stage kernels.
#include "aba.cuh"
#include "collide.cuh"
#include "solve.cuh"

namespace gb {

constexpr int FUSED_WARPS = 4;

__global__ void __launch_bounds__(32 * FUSED_WARPS, 4)
    k_step_fused(Dev d, int nsub, int NC, PgsLayout L, int warp_bytes, WorkQueue q) {
  extern __shared__ __align__(16) unsigned char smf[];
  const int lane = threadIdx.x & 31;
  unsigned char* base = smf + (size_t)(threadIdx.x >> 5) * warp_bytes;
  if (lane == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"((uint32_t)__cvta_generic_to_shared(base + L.off_bar()))
                 : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  uint32_t bar_phase = 0;
  int pending = -1;
  for (int s = wq_first(q, lane); s < d.E; s = wq_next(q, lane)) {
    const int e = wq_env(q, s);
    const int a0 = d.art_off[e], a1 = d.art_off[e + 1];
    for (int sub = 0; sub < nsub; ++sub) {
      // link poses, then forward dynamics: multi-joint articulations on the warp, the
      // others (one joint) a lane each
      for (int a = a0; a < a1; ++a)
        if (d.joint_off[a + 1] - d.joint_off[a] > 1) {
          fk_multi<32>(d, a, lane, 0xffffffffu, *reinterpret_cast<FkSh*>(base));
          __syncwarp();
          aba_multi<32>(d, a, lane, 0xffffffffu, *reinterpret_cast<AbaSh*>(base));
          __syncwarp();
        }
      for (int a = a0 + lane; a < a1; a += 32)
        if (d.joint_off[a + 1] - d.joint_off[a] <= 1) {
          fk_single(d, a);
          aba_single(d, a);
        }
      __syncwarp();
      collide_env(d, NC, reinterpret_cast<float*>(base), e, lane);
      __syncwarp();
      rows_env(d, e, lane);
      // the row pool just written is read next by a bulk copy (the async proxy)
      asm volatile("fence.proxy.async;" ::: "memory");
      __syncwarp();
      pgs_env<32>(d, L, base, e, lane, 0xffffffffu, 0, bar_phase, pending);
      __syncwarp();
      // a pool copy given up on may still land: wait for it (bounded) before the next
      // stage writes this warp's shared memory
      if (pending >= 0) {
        if (lane == 0) mbar_wait_bounded((uint32_t)__cvta_generic_to_shared(base + L.off_bar()), (uint32_t)pending);
        pending = -1;
        __syncwarp();
      }
    }
  }
  wq_done(q, lane);
}

// The PGS layout of the fused step: the shape's staging, with the mbarrier raised
// above the collision, forward-kinematics and ABA working sets, which share the
// warp's shared memory.
static PgsLayout fused_layout(const Dev& d, int max_coll, int max_obj, int max_arts, int stage_contacts,
                              int stage_pool) {
  PgsLayout L = pgs_layout(d, max_obj, max_arts, stage_contacts, stage_pool);
  const size_t coll = sizeof(float) * CollLayout{(max_coll + 3) & ~3}.floats();
  L.bar_floor = (int)std::max(std::max(coll, sizeof(AbaSh)), sizeof(FkSh));
  return L;
}

static int max_optin_smem() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return v;
}

int fused_warp_bytes(const Dev& d, int max_coll, int max_obj, int max_arts, int stage_contacts, int stage_pool) {
  const size_t w = fused_layout(d, max_coll, max_obj, max_arts, stage_contacts, stage_pool).bytes();
  return w * FUSED_WARPS > (size_t)max_optin_smem() ? 0 : (int)w;
}

void configure_fused() {
  cudaFuncSetAttribute(k_step_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, max_optin_smem());
}

void launch_fused(const Dev& d, cudaStream_t st, int n, int max_coll, int max_obj, int max_arts, int stage_contacts,
                  int stage_pool, int sms, const int* perm) {
  if (d.E == 0 || n <= 0) return;
  const PgsLayout L = fused_layout(d, max_coll, max_obj, max_arts, stage_contacts, stage_pool);
  const int warp_bytes = fused_warp_bytes(d, max_coll, max_obj, max_arts, stage_contacts, stage_pool);
  if (warp_bytes == 0) return;  // the launch shape is validated against this
  const size_t smem = (size_t)warp_bytes * FUSED_WARPS;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step_fused, 32 * FUSED_WARPS, smem) != cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  const int blocks = std::min((d.E + FUSED_WARPS - 1) / FUSED_WARPS, per_sm * sms);
  // the collision kernel's queue counters: that kernel does not run in a fused step
  WorkQueue q{d.wq + 0, perm, 1};
  k_step_fused<<<blocks, 32 * FUSED_WARPS, smem, st>>>(d, n, (max_coll + 3) & ~3, L, warp_bytes, q);
}

}  // namespace gb
