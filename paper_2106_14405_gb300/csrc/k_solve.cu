// Row-build, PGS, ordering and integration kernels (device code in solve.cuh).
#include "solve.cuh"

namespace gb {

__global__ void __launch_bounds__(256, 3) k_rows(Dev d, WorkQueue q) {
  const int lane = threadIdx.x & 31;
  for (int s = wq_first(q, lane); s < d.E; s = wq_next(q, lane)) {
    rows_env(d, wq_env(q, s), lane);
    __syncwarp();
  }
  wq_done(q, lane);
}

// MINB: resident 256-thread blocks per SM the register allocation is built for
// (1: up to 255 registers per thread; 2: up to 128; 3: up to 85, the rest spilled to local memory)
template <int G, int MINB>
__global__ void __launch_bounds__(256, MINB) k_pgs(Dev d, PgsLayout L, WorkQueue q, int heavy_sms, int heavy_base) {
  extern __shared__ __align__(16) unsigned char smp[];
  __shared__ int s_role;
  const int lane = threadIdx.x & 31;
  const int gl = lane & (G - 1), g0 = lane & ~(G - 1);
  const unsigned gm = G == 32 ? 0xffffffffu : (((1u << (G & 31)) - 1u) << g0);
  unsigned char* base = smp + (size_t)(threadIdx.x / G) * L.bytes();
  const int groups_per_block = blockDim.x / G;
  PgsSched S;
  S.ctr = q.ctr;
  S.sm_rank = d.sm_rank;
  S.heavy_sms = q.persistent ? heavy_sms : 0;
  S.persistent = q.persistent;
  S.pass = 0;
  S.E = d.E;
  S.first = blockIdx.x * groups_per_block + threadIdx.x / G;
  S.H = min(d.E, S.heavy_sms * groups_per_block);
  S.role = 0;
  if (S.heavy_sms > 0) {
    if (threadIdx.x == 0) {
      unsigned smid;
      asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
      const int r = (int)smid - heavy_base;  // this launch's heavy SMs: heavy_base .. heavy_base + heavy_sms - 1
      s_role = (r >= 0 && r < S.heavy_sms) ? (atomicAdd(S.sm_rank + r, 1) == 0 ? 1 : 2) : 0;
    }
    __syncthreads();
    S.role = s_role;
    if (S.role == 2) S.pass = 2;
  }
  // the group's mbarrier for the bulk copy of each environment's row pool
  if (gl == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"((uint32_t)__cvta_generic_to_shared(base + L.off_bar()))
                 : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp(gm);
  uint32_t bar_phase = 0;
  int pending = -1;  // parity of a pool copy whose bounded wait ran out, while it may still land
  for (int s = S.next<G>(gl, gm, g0); s >= 0; s = S.next<G>(gl, gm, g0)) {
    pgs_env<G>(d, L, base, wq_env(q, s), gl, gm, g0, bar_phase, pending);
    __syncwarp(gm);
  }
  // a copy given up on may still be in flight: wait for it once more (bounded) before
  // the block's shared memory is released
  if (pending >= 0 && gl == 0)
    mbar_wait_bounded((uint32_t)__cvta_generic_to_shared(base + L.off_bar()), (uint32_t)pending);
  if (q.persistent && gl == 0) {  // the last group to finish resets the counters for the next launch
    const int total = (int)gridDim.x * groups_per_block;
    if (atomicAdd(q.ctr + 1, 1) == total - 1) {
      atomicExch(q.ctr, 0);
      atomicExch(q.ctr + 1, 0);
      atomicExch(q.ctr + 2, 0);
      for (int i = 0; i < S.heavy_sms; ++i) atomicExch(S.sm_rank + i, 0);
    }
  }
}

// ---------------------------------------------------------------------------
static int max_optin_smem() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return v;
}

int occupancy_rows(int warps) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_rows, 32 * warps, 0) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

void launch_rows(const Dev& d, cudaStream_t st, KShape k) {
  if (d.E == 0) return;
  int blocks = (d.E + k.warps - 1) / k.warps;
  if (k.persistent) blocks = min(blocks, k.grid_cap);
  WorkQueue q{d.wq + 2, nullptr, k.persistent};
  k_rows<<<blocks, 32 * k.warps, 0, st>>>(d, q);
}

static PgsLayout make_layout(const Dev& d, int max_obj, int max_arts, int S, int AS) {
  PgsLayout L;
  L.C = d.C;
  L.nobj = max(max_obj, 1);
  L.narts = max(max_arts, 1);
  L.S = S;
  L.LS = 16;
  L.AS = AS;
  L.bar_floor = 0;
  return L;
}

// Default staging: contacts 4 per object + 8 (32 .. max_contacts); articulation row
// endpoints 32, halved (down to 8) while an environment needs more than 19 KB, about
// the share of an SM's shared memory that keeps 12 environments resident.
void pgs_stage_defaults(const Dev& d, int max_obj, int max_arts, int* stage_contacts, int* stage_pool) {
  const int S = min(d.C, max(32, 4 * max_obj + 8));
  int AS = 32;
  while (AS > 8 && make_layout(d, max_obj, max_arts, S, AS).bytes() > 19 * 1024) AS >>= 1;
  *stage_contacts = S;
  *stage_pool = AS;
}

PgsLayout pgs_layout(const Dev& d, int max_obj, int max_arts, int stage_contacts, int stage_pool) {
  int S0, AS0;
  pgs_stage_defaults(d, max_obj, max_arts, &S0, &AS0);
  return make_layout(d, max_obj, max_arts, stage_contacts > 0 ? min(d.C, stage_contacts) : S0,
                     stage_pool > 0 ? min(APOOL, stage_pool) : AS0);
}

using PgsKernel = void (*)(Dev, PgsLayout, WorkQueue, int, int);

static PgsKernel pgs_kernel(int lanes, int min_blocks) {
  if (min_blocks == 2) {
    if (lanes == 32) return k_pgs<32, 2>;
    if (lanes == 16) return k_pgs<16, 2>;
    if (lanes == 8) return k_pgs<8, 2>;
  }
  if (min_blocks == 3 && lanes == 32) return k_pgs<32, 3>;
  if (min_blocks == 1 && lanes == 32) return k_pgs<32, 1>;
  return nullptr;
}

// every PGS build may take the whole opt-in shared memory of a block (less its static part)
void configure_pgs(const Dev& d, int max_obj, int max_arts) {
  (void)d; (void)max_obj; (void)max_arts;
  for (int lanes = 8; lanes <= 32; lanes *= 2)
    for (int mb = 1; mb <= 3; ++mb) {
      PgsKernel k = pgs_kernel(lanes, mb);
      if (k) cudaFuncSetAttribute((const void*)k, cudaFuncAttributeMaxDynamicSharedMemorySize, max_optin_smem() - 64);
    }
}

int occupancy_pgs(const Dev& d, int max_obj, int max_arts, int warps, int lanes, int min_blocks, int stage_contacts,
                  int stage_pool) {
  PgsKernel k = pgs_kernel(lanes, min_blocks);
  if (!k || warps < 1 || warps * 32 < lanes) return 0;
  const size_t smem =
      pgs_layout(d, max_obj, max_arts, stage_contacts, stage_pool).bytes() * (size_t)(warps * 32 / lanes);
  if (smem + 64 > (size_t)max_optin_smem()) return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, 32 * warps, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

void launch_pgs(const Dev& d, cudaStream_t st, int max_obj, int max_arts, KShape k, int lpt, int heavy_base) {
  if (d.E == 0) return;
  PgsLayout L = pgs_layout(d, max_obj, max_arts, k.stage_contacts, k.stage_pool);
  const int envs = k.warps * 32 / k.lanes;  // environments per block
  int blocks = (d.E + envs - 1) / envs;
  if (k.persistent) blocks = min(blocks, k.grid_cap);
  WorkQueue q{d.wq + 4, lpt ? d.perm : nullptr, k.persistent};
  pgs_kernel(k.lanes, k.min_blocks)<<<blocks, 32 * k.warps, L.bytes() * envs, st>>>(d, L, q, k.heavy_sms,
                                                                                     heavy_base);
}

// Longest-processing-time-first schedule for k_pgs: environments sorted by the
// length of their Gauss-Seidel chain, descending, so the longest chains start
// first and overlap the short ones.  An environment's chain is its colour count
// times the sweeps; the key is the colour count of its previous step (the
// contact set changes slowly), then its row count.  One block; the order within
// a bucket may vary between runs, which changes only which warp runs an
// environment, never its result.
__device__ __forceinline__ int lpt_key(const int* n_rows, const int* n_colours, int e) {
  return 1023 - (16 * min(n_colours[e], 63) + min(n_rows[e] >> 4, 15));
}

// counting sort on the 1024 keys: histogram, block-wide exclusive scan (one key
// per thread: warp scans, then a scan of the 32 warp totals), scatter.  Each
// thread takes four consecutive environments per pass, their counts loaded
// together (one round trip per pass instead of one per environment).  The order
// within a key depends on atomics; it only changes which warp takes which slot.
__global__ void __launch_bounds__(1024) k_lpt_order(const int* n_rows, const int* n_colours, int E, int* perm) {
  __shared__ int h[1024];
  __shared__ int wsum[32];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  h[t] = 0;
  __syncthreads();
  for (int e0 = 4 * t; e0 < E; e0 += 4096) {
    int key[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) key[i] = e0 + i < E ? lpt_key(n_rows, n_colours, e0 + i) : -1;
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (key[i] >= 0) atomicAdd(&h[key[i]], 1);
  }
  __syncthreads();
  const int c = h[t];
  int incl = c;
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) wsum[w] = incl;
  __syncthreads();
  if (w == 0) {
    int x = wsum[lane];
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += v;
    }
    wsum[lane] = x;  // inclusive over warps
  }
  __syncthreads();
  h[t] = (w > 0 ? wsum[w - 1] : 0) + incl - c;
  __syncthreads();
  for (int e0 = 4 * t; e0 < E; e0 += 4096) {
    int key[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) key[i] = e0 + i < E ? lpt_key(n_rows, n_colours, e0 + i) : -1;
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (key[i] >= 0) perm[atomicAdd(&h[key[i]], 1)] = e0 + i;
  }
}

void launch_lpt_order(const Dev& d, cudaStream_t st) {
  if (d.E == 0 || !d.perm) return;
  k_lpt_order<<<1, 1024, 0, st>>>(d.n_rows, d.n_colours, d.E, d.perm);
}

}  // namespace gb
