// Internal device layout and helpers of the batched physics step (CUDA, sm_103a).
//
// Layout in HBM: structure of arrays, one array per field, each field a float4
// (or int) per item so that a warp reading the consecutive items of one
// environment issues 16-byte coalesced loads.  Items of one environment are
// contiguous (CSR offsets per environment), so every per-environment kernel
// reads one contiguous range per field.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gb {

constexpr int MAX_DOF = 9;
constexpr int MAX_OBJ = 64;
constexpr int MAX_COLL = 128;
constexpr int MAX_ARTS = 8;
constexpr int MAX_CONTACTS = 256;
constexpr int PAIR_CAP = 1024;    // candidate pairs per env
constexpr int APOOL = 64;         // articulation row endpoints per env
constexpr int APS = 72;           // floats per endpoint: J rows at 0, 12, 24, M^-1 J^T rows at 36, 48, 60 (9 of 12 used)
constexpr int LCAP = 32;          // joint-limit rows per env
constexpr int NFEAT = 32;

enum { SHAPE_SPHERE = 0, SHAPE_BOX = 1, SHAPE_PLANE = 2 };
enum { CK_OBJ = 0, CK_LINK = 1, CK_BASE = 2, CK_STATIC = 3, CK_PLANE = 4 };
enum { ST_OVERFLOW = 1, ST_NUMERIC = 2, ST_ITER_CAP = 4, ST_FORCE = 8, ST_DEVICE_WAIT = 16 };

// Row endpoint codes: -1 static, 0..63 object (local index), or
// ART_TAG | art_local << 8 | pool slot.
constexpr int ART_TAG = 0x10000;

struct Dev {
  int E, NO, NS, NA, NJ, C;
  // first environment of this view: a partition of the batch (see partition_view) sees
  // environments env0 .. env0 + E - 1 as 0 .. E - 1 through offset per-environment
  // arrays; objects, joints and articulations keep their batch-wide indices
  int env0;
  // parameters
  float dt, gx, gy, gz;
  int pgs_iters; float pgs_tol; int pgs_max_iters;
  float baumgarte, slop, margin, rest_thresh;
  float sleep_lin, sleep_ang; int sleep_steps, sleep_enabled, warm_mode;
  float plane_mu, lambda_floor, match_dist, fp64_cond;
  float force_limit;  // N; accumulated robot contact force that flags an env (<= 0: off)
  int hold_async;     // testing: withhold async completions so that the bounded device waits run out
  int motor_mode;     // 1: joints of kinematic-base articulations driven by motor rows instead of the implicit PD
  float motor_kp, motor_max_impulse;
  int log_features;  // K_rows writes per-contact features
  // per env
  const int *obj_off, *stat_off, *art_off, *env_plane, *base_off, *base_art;
  int *status, *iters, *n_contacts, *n_rows, *n_limit, *n_colours, *fp64_used, *pair_count, *pairs;
  float *robot_force, *robot_force_acc;  // [E] contact force on the robot: this step, accumulated (N)
  float* resid;
  // objects
  float4 *obj_pos, *obj_comp, *obj_quat, *obj_vel, *obj_omega;
  float4 *obj_vstar, *obj_wstar;  // velocities after gravity (zero while asleep), before the solve
  const int *obj_env, *j_env;     // owning environment of each object / joint
  const float4 *obj_half;   // half extents (sphere: radius in x), w = shape
  const float4 *obj_inv;    // inv mass, inverse principal inertia
  const float2 *obj_mat;    // mu, restitution
  int *obj_awake, *obj_ctr;
  // statics
  const float4 *stat_pos;   // w = mu
  const float4 *stat_quat, *stat_half;
  // articulations
  const int *joint_off, *art_has_bc, *art_kin, *j_art;
  float4 *art_base_pos, *art_base_quat;
  const float4 *art_bc_off, *art_bc_half;
  // articulations by size: multi-joint ones (warp kernel), single-joint ones (thread kernel)
  const int *art_multi, *art_single;
  int n_art_multi, n_art_single;
  // joints (constants)
  const int *j_parent, *j_type;
  const unsigned* j_anc;    // joints on the path from the articulation's root to this joint (bit per local joint)
  const float4 *j_axis, *j_opos, *j_oquat;
  const float4 *j_com;      // w = mass
  const float4 *j_half;     // w = mu
  const float4 *j_lim;      // lo, hi, has_limit
  const float2 *j_gain;     // kp, kd
  // joints (state)
  float *j_q, *j_qcomp, *j_qd, *j_target, *j_lim_lambda, *j_motor_lambda;
  int* j_lim_side;
  // ABA outputs (at q_t)
  float4 *l_com, *l_r0, *l_r1, *l_r2, *l_ja, *l_jo;  // link COM, rotation rows, joint axis, joint origin
  float *j_qdd, *j_qdstar;
  float* a_minv;  // [NA][81]
  // contacts [E*C]
  int4* c_key;    // a, b, feature
  float4 *c_p;    // point, separation
  float4 *c_n;    // normal B->A
  float4 *c_lam;  // final impulses
  // prior-frame cache [E*C]
  int* cache_count;
  int4* cache_key;
  float4 *cache_p, *cache_lam;  // lam: normal, friction world vector
  // rows [E*C]
  float4 *r_t1;    // t1, mu
  float4 *r_meff;  // m_eff n, t1, t2, target
  float4 *r_lam;   // warm start, then current
  float4 *r_ra, *r_rb;  // contact point minus COM for object endpoints
  int2* r_ends;    // endpoint codes A, B
  float* ap;            // [E*APOOL][APS]: the PGS kernel's shared-memory layout, staged by a plain copy
  int* ap_count;
  // limit rows [E*LCAP]
  int4* lr_info;   // art local, joint local, sign (+1/-1), global joint
  float4* lr_data; // m_eff, target, lambda, 0
  float* lr_w;     // [E*LCAP][MAX_DOF]
  // longest-processing-time-first order of the solver's environments (heaviest first)
  int* perm;       // [E]; NULL = identity
  // work queues of the persistent launches: {next slot, warps finished} for collide and rows
  int* wq;         // [8], zero between launches (PGS: {light next, finished, heavy next})
  int* sm_rank;    // [MAX_HEAVY_SMS] blocks started per heavy SM in the PGS launch, zero between launches
  // learned warm start
  float* feat;     // [E*C][32]
  float4* pred;    // [E*C] network output (normalised impulses)
  int* mlp_rows;   // [E*C] contact rows (e*C + slot) the network runs on this step (see LEARN_GATE)
  int* mlp_count;  // their number (zeroed before the row kernel)
};

// ---------------------------------------------------------------------------
// small vector helpers
// ---------------------------------------------------------------------------
struct V3 { float x, y, z; };
__device__ __forceinline__ V3 v3(float x, float y, float z) { return V3{x, y, z}; }
__device__ __forceinline__ V3 v3(float4 a) { return V3{a.x, a.y, a.z}; }
__device__ __forceinline__ V3 operator+(V3 a, V3 b) { return V3{a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ V3 operator-(V3 a, V3 b) { return V3{a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ V3 operator-(V3 a) { return V3{-a.x, -a.y, -a.z}; }
__device__ __forceinline__ V3 operator*(V3 a, float s) { return V3{a.x * s, a.y * s, a.z * s}; }
__device__ __forceinline__ V3 operator*(float s, V3 a) { return V3{a.x * s, a.y * s, a.z * s}; }
__device__ __forceinline__ float dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ V3 cross(V3 a, V3 b) {
  return V3{a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ float norm(V3 a) { return sqrtf(dot(a, a)); }
__device__ __forceinline__ float comp(V3 a, int i) { return i == 0 ? a.x : (i == 1 ? a.y : a.z); }
__device__ __forceinline__ float4 f4(V3 a, float w) { return make_float4(a.x, a.y, a.z, w); }

// Learned warm start (warm_mode 2).  Unit of its impulses for one contact: the normal
// effective mass times the velocity change the step can ask of the contact -- the
// free-fall increment |g| dt plus the size of its relative velocity before the solve
// (features 9-11): about one |g| dt for a resting contact, about the approach speed for
// an impact.  `f` is the contact's 32 features, gdt = |g| dt.
__device__ __forceinline__ float learn_scale(float meff_n, const float* f, float gdt) {
  return meff_n * (gdt + sqrtf(f[9] * f[9] + f[10] * f[10] + f[11] * f[11]));
}
// The network starts the contacts without a prior-frame match and the matched ones whose
// relative velocity exceeds LEARN_GATE |g| dt; persistent resting contacts keep their
// prior-frame impulse.
constexpr float LEARN_GATE = 4.f;

// In place: v[0..n) counts -> exclusive prefix sums, v[n] = their total.  One block
// of 1024 threads, each scanning a contiguous chunk (stable compaction of rows).
static __global__ void __launch_bounds__(1024) k_exclusive_scan(int* v, int n) {
  __shared__ int part[1024];
  const int t = threadIdx.x;
  const int chunk = (n + 1023) / 1024;
  const int b = min(n, t * chunk), e2 = min(n, b + chunk);
  int sum = 0;
  for (int i = b; i < e2; ++i) sum += v[i];
  part[t] = sum;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {  // inclusive scan of the chunk sums
    const int x = t >= o ? part[t - o] : 0;
    __syncthreads();
    part[t] += x;
    __syncthreads();
  }
  int acc = part[t] - sum;
  for (int i = b; i < e2; ++i) {
    const int c = v[i];
    v[i] = acc;
    acc += c;
  }
  if (t == 1023) v[n] = part[1023];
}

struct M3 { V3 r0, r1, r2; };  // rows
__device__ __forceinline__ V3 mv(const M3& m, V3 v) { return V3{dot(m.r0, v), dot(m.r1, v), dot(m.r2, v)}; }
__device__ __forceinline__ V3 mtv(const M3& m, V3 v) { return m.r0 * v.x + m.r1 * v.y + m.r2 * v.z; }
__device__ __forceinline__ V3 mcol(const M3& m, int j) {
  return j == 0 ? V3{m.r0.x, m.r1.x, m.r2.x} : (j == 1 ? V3{m.r0.y, m.r1.y, m.r2.y} : V3{m.r0.z, m.r1.z, m.r2.z});
}
__device__ __forceinline__ M3 quat_mat(float4 q) {  // (w, x, y, z)
  float w = q.x, x = q.y, y = q.z, z = q.w;
  M3 r;
  r.r0 = V3{1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z), 2.f * (x * z + w * y)};
  r.r1 = V3{2.f * (x * y + w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x)};
  r.r2 = V3{2.f * (x * z - w * y), 2.f * (y * z + w * x), 1.f - 2.f * (x * x + y * y)};
  return r;
}

__device__ __forceinline__ float warp_sum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
// sum over the G lanes of a group (mask gm)
template <int G>
__device__ __forceinline__ float group_sum(float v, unsigned gm) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(gm, v, o);
  return v;
}

// ---------------------------------------------------------------------------
// Environment scheduling of the warp-per-environment kernels.  In a plain grid
// warp w of block b runs environment slot b * warps + w.  In a persistent grid
// (as many blocks as stay resident) each warp takes the next slot from a device
// counter until the slots run out, so a warp that finishes a light environment
// starts the next one at once instead of waiting for its block; the last warp
// to finish zeroes the counters for the next launch.  A slot maps to an
// environment through perm when given.  Either way every environment runs the
// same code on one warp, so the results do not depend on the schedule.
// ---------------------------------------------------------------------------
struct WorkQueue {
  int* ctr;         // {next slot, warps finished}
  const int* perm;  // slot -> environment, or NULL for the identity
  int persistent;
};

// G = lanes per environment (32: one warp; 16 or 8: several environments per
// warp); gm = the lane mask of this lane's group, g0 = the group's first lane.
template <int G = 32>
__device__ __forceinline__ int wq_first(const WorkQueue& q, int gl, unsigned gm = 0xffffffffu, int g0 = 0) {
  if (!q.persistent) return blockIdx.x * (blockDim.x / G) + threadIdx.x / G;
  int s = 0;
  if (gl == 0) s = atomicAdd(q.ctr, 1);
  return __shfl_sync(gm, s, g0);
}
template <int G = 32>
__device__ __forceinline__ int wq_next(const WorkQueue& q, int gl, unsigned gm = 0xffffffffu, int g0 = 0) {
  if (!q.persistent) return 0x7fffffff;
  int s = 0;
  if (gl == 0) s = atomicAdd(q.ctr, 1);
  return __shfl_sync(gm, s, g0);
}
// every group of a persistent grid calls this once, after its last (failed) take
template <int G = 32>
__device__ __forceinline__ void wq_done(const WorkQueue& q, int gl) {
  if (!q.persistent || gl != 0) return;
  const int total = (int)(gridDim.x * (blockDim.x / G));
  if (atomicAdd(q.ctr + 1, 1) == total - 1) {
    atomicExch(q.ctr, 0);
    atomicExch(q.ctr + 1, 0);
  }
}
__device__ __forceinline__ int wq_env(const WorkQueue& q, int slot) { return q.perm ? q.perm[slot] : slot; }

// launch shape of one warp-per-environment kernel
struct KShape {
  int warps;       // warps per block
  int persistent;  // 1: grid of grid_cap blocks pulling from the work queue
  int grid_cap;    // blocks resident on the device at this shape
  int lanes;       // lanes per environment (32, or 16 / 8 for the PGS kernel)
  int min_blocks;  // PGS register build: 2 or 3 resident 256-thread blocks per SM
  int heavy_sms;   // PGS: SMs given to the heaviest environments (persistent grid with LPT order only)
  int stage_contacts, stage_pool;  // PGS: contacts / articulation row endpoints staged in shared memory (0: default)
};
static const int MAX_WARPS_PER_CTA = 8;
static const int MAX_HEAVY_SMS = 256;

// ---------------------------------------------------------------------------
// kernel launchers (defined in the kernel translation units)
// ---------------------------------------------------------------------------
void launch_aba(const Dev& d, cudaStream_t s, int lanes);
void launch_collide(const Dev& d, cudaStream_t s, int max_coll, KShape k);
void launch_rows(const Dev& d, cudaStream_t s, KShape k);
void launch_pgs(const Dev& d, cudaStream_t s, int max_obj, int max_arts, KShape k, int lpt, int heavy_base);
// resident blocks per SM of each kernel at `warps` warps per block (0: does not fit)
int occupancy_collide(int max_coll, int warps);
int occupancy_rows(int warps);
int occupancy_pgs(const Dev& d, int max_obj, int max_arts, int warps, int lanes, int min_blocks, int stage_contacts,
                  int stage_pool);
void pgs_stage_defaults(const Dev& d, int max_obj, int max_arts, int* stage_contacts, int* stage_pool);
void launch_lpt_order(const Dev& d, cudaStream_t s);
// the whole step in one persistent launch (k_fused.cu): shared memory per warp (0 if four
// warps' do not fit a block), and the launch of n physics steps (perm: slot order or NULL)
int fused_warp_bytes(const Dev& d, int max_coll, int max_obj, int max_arts, int stage_contacts, int stage_pool);
void launch_fused(const Dev& d, cudaStream_t s, int n, int max_coll, int max_obj, int max_arts, int stage_contacts,
                  int stage_pool, int sms, const int* perm);
void configure_fused();
void launch_fk(const Dev& d, cudaStream_t s);  // link poses of the view's articulations
// set dynamic shared-memory limits once, outside any stream capture
void configure_aba();
void configure_collide(int max_coll);
void configure_pgs(const Dev& d, int max_obj, int max_arts);

}  // namespace gb
