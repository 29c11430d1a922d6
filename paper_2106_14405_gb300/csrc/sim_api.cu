// C ABI of the batched physics step: handle creation (validation, SoA upload),
// step scheduling (optionally replayed from a captured CUDA graph), state and
// diagnostics transfer.  See include/sim.h for the contract of every call.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/sim.h"
#include "sim_internal.cuh"

using gb::Dev;

static thread_local std::string g_err;
static thread_local unsigned long long g_err_count = 0;  // errors recorded on this thread

static int fail(int code, const std::string& msg) {
  g_err = msg;
  ++g_err_count;
  return code;
}

// Selects the handle's device for the duration of a call and restores the caller's
// current device afterwards (no device change, and no runtime call beyond the query,
// when they are the same).
// It also copies an error recorded during the call into the handle (sim_last_error(h)).
struct DevGuard {
  int prev = -1, want = -1;
  bool ok = true;
  std::string* err = nullptr;
  unsigned long long count0 = 0;
  DevGuard(int dev, std::string* handle_err) : want(dev), err(handle_err), count0(g_err_count) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != want) ok = cudaSetDevice(want) == cudaSuccess;
  }
  ~DevGuard() {
    if (prev >= 0 && prev != want) cudaSetDevice(prev);
    if (err && g_err_count != count0) *err = g_err;
  }
};
#define ON_DEVICE(h)                                                          \
  DevGuard dev_guard_((h)->device, &(h)->last_err);                           \
  if (!dev_guard_.ok) return fail(SIM_ERR_CUDA, "cannot select the handle's device")

#define CK(call)                                                                                     \
  do {                                                                                               \
    cudaError_t e_ = (call);                                                                         \
    if (e_ != cudaSuccess) return fail(SIM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

struct SimHandle {
  int device;               // CUDA device the handle was created on; every call selects it
  std::string last_err;     // the last error of a call on this handle (sim_last_error(h))
  Dev d;
  SimParams p;
  cudaStream_t stream;      // the caller's stream: every launch and graph replay goes here
  cudaStream_t cap_stream;  // private non-blocking stream the step graph is captured on
  int max_coll, max_obj, max_arts;  // per-env maxima of the batch (launch shapes)
  std::vector<void*> allocs;
  float* stage;  // device staging buffer for packed transfers
  size_t stage_floats;
  cudaGraphExec_t graph;
  int graph_n;
  long long graph_kernels;  // kernels in one replay of the captured graph
  int* art_env;  // env of each articulation (device)
  int mlp_ready;
  void* mlp;     // learned warm-start weights (see k_mlp.cu)
  // kernel timing: events[substep][stage boundary]
  int profiling;
  std::vector<cudaEvent_t> events;
  int prof_n;                // substeps of the last profiled sim_step
  int stage_launches[SIM_N_STAGES];  // kernels per stage in the last enqueued sim_step call
  long long launches;        // kernels enqueued since creation
  int kernels_per_step;
  // launch shapes of the warp-per-environment kernels
  SimLaunchShape shape;
  int sm_count;
  // reset template (sim_reset_envs): the per-environment state that a reset restores
  struct {
    float4 *obj_pos, *obj_comp, *obj_quat, *obj_vel, *obj_omega, *base_pos, *base_quat;
    int *obj_awake, *obj_ctr, *j_lim_side;
    float *j_q, *j_qcomp, *j_qd, *j_target, *j_lim_lambda, *j_motor_lambda;
  } tmpl;
  int occ[2][4];  // resident blocks per SM: [collide, rows][1, 2, 4, 8 warps per block]
  int pgs_occ;    // resident PGS blocks per SM at the current shape
  // environment partitions (SimLaunchShape.partitions): each partition's kernels run on
  // a stream of their own, forked from and joined to the handle's stream (or the capture)
  cudaStream_t pstream[SIM_MAX_PARTITIONS];
  cudaEvent_t fork_ev, join_ev[SIM_MAX_PARTITIONS];
  std::vector<int> art_off_h, multi_h, single_h;  // host copies: articulation ranges of partitions
  int last_parts;  // partitions of the last enqueued steps (each lists its own network rows)
  // the ABA kernels beside forward kinematics and collision (SimLaunchShape.aba_overlap):
  // per partition a side stream, forked from the partition's stream and joined before
  // the row kernel
  cudaStream_t astream[SIM_MAX_PARTITIONS];
  cudaEvent_t afork_ev[SIM_MAX_PARTITIONS], ajoin_ev[SIM_MAX_PARTITIONS];
};

namespace gb {
// defined in sim_noalloc.cu: looks up the fixed scratch's address on the current device
int noalloc_scratch_refresh();
// defined in k_mlp.cu
void launch_mlp_infer(const Dev& d, const void* mlp, cudaStream_t s);
void* mlp_create(const float* params, int on_device, cudaStream_t s, std::string& err);
void mlp_destroy(void* mlp);
}  // namespace gb

// ---------------------------------------------------------------------------
// small kernels: body constants, base pose, pack / unpack
// ---------------------------------------------------------------------------
__global__ void k_init_bodies(int NO, const float4* half, const float* mass, float4* inv) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NO) return;
  float4 h = half[i];
  float m = mass[i];
  float im = 1.f / m;
  if (h.w == 0.f) {  // solid sphere
    float I = 0.4f * m * h.x * h.x;
    inv[i] = make_float4(im, 1.f / I, 1.f / I, 1.f / I);
  } else {  // solid box
    float Ix = m * (h.y * h.y + h.z * h.z) / 3.f, Iy = m * (h.x * h.x + h.z * h.z) / 3.f,
          Iz = m * (h.x * h.x + h.y * h.y) / 3.f;
    inv[i] = make_float4(im, 1.f / Ix, 1.f / Iy, 1.f / Iz);
  }
}

__global__ void k_set_base(int NA, const int* art_env, const int* kin, const float* xy_yaw, float4* pos, float4* quat) {
  int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= NA || !kin[a]) return;
  int e = art_env[a];
  float x = xy_yaw[3 * e], y = xy_yaw[3 * e + 1], yaw = xy_yaw[3 * e + 2];
  float4 p = pos[a];
  pos[a] = make_float4(x, y, p.z, 0.f);
  quat[a] = make_float4(cosf(0.5f * yaw), 0.f, 0.f, sinf(0.5f * yaw));
}

// float4 array -> packed [n][w] floats (w <= 4)
__global__ void k_pack(const float4* src, float* dst, long n, int w) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  float4 v = src[i];
  float c[4] = {v.x, v.y, v.z, v.w};
  for (int k = 0; k < w; ++k) dst[i * w + k] = c[k];
}
__global__ void k_unpack(const float* src, float4* dst, long n, int w) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  float c[4] = {0.f, 0.f, 0.f, 0.f};
  float4 o = dst[i];
  c[3] = o.w;  // keep the unused lane (e.g. a constant packed there)
  for (int k = 0; k < w; ++k) c[k] = src[i * w + k];
  dst[i] = make_float4(c[0], c[1], c[2], c[3]);
}
__global__ void k_pack_i4(const int4* src, int* dst, long n) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int4 v = src[i];
  dst[3 * i] = v.x; dst[3 * i + 1] = v.y; dst[3 * i + 2] = v.z;
}
__global__ void k_unpack_i4(const int* src, int4* dst, long n) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  dst[i] = make_int4(src[3 * i], src[3 * i + 1], src[3 * i + 2], 0);
}
__global__ void k_pack_rot(const float4* r0, const float4* r1, const float4* r2, float* dst, long n) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  float4 a = r0[i], b = r1[i], c = r2[i];
  float* o = dst + 9 * i;
  o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = b.x; o[4] = b.y; o[5] = b.z; o[6] = c.x; o[7] = c.y; o[8] = c.z;
}
__global__ void k_pack_w(const float4* src, float* dst, long n) {  // the .w lane
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  dst[i] = src[i].w;
}
__global__ void k_pairs_out(const int* pairs, int cap, int* dst, int E) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= (long)E * cap) return;
  long e = i / cap, k = i % cap;
  dst[i] = pairs[e * gb::PAIR_CAP + k];
}
// Contact-impulse log for training the learned warm start.  A contact is logged when
// its environment's solve met the residual target in the last step (a fixed sweep count
// always does: only converged impulses are training targets) and its target,
// (final - prior-frame impulses) / learn_scale, is finite (a degenerate row, m_eff,n = 0,
// or a contact with no velocity change to ask for has no scale).  One warp per
// environment.  MODE 0: the env's logged contacts into count[e].  MODE 1: their
// features and targets, in contact order, from row prefix[e] on; MODE 2: the learned
// warm start's network outputs of the same rows into feats[row * 3 + k] (rows >= cap
// are dropped).
template <int MODE>
__global__ void k_log_rows(Dev d, const int* prefix, int* count, float* feats, float* lams, int cap) {
  constexpr bool WRITE = MODE != 0;
  const int lane = threadIdx.x & 31;
  const int e = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (e >= d.E) return;
  const bool conv = d.pgs_tol <= 0.f || d.resid[e] <= d.pgs_tol;
  const int n = conv ? d.n_contacts[e] : 0;
  const float gdt = sqrtf(d.gx * d.gx + d.gy * d.gy + d.gz * d.gz) * d.dt;
  const int base = WRITE ? prefix[e] : 0;
  int cnt = 0;
  for (int i0 = 0; i0 < n; i0 += 32) {
    const int i = i0 + lane;
    const size_t g = (size_t)e * d.C + i;
    bool ok = false;
    float t[3] = {0.f, 0.f, 0.f};
    if (i < n) {
      const float* f = d.feat + g * gb::NFEAT;
      const float sc = gb::learn_scale(d.r_meff[g].x, f, gdt);
      const float4 l = d.c_lam[g];
      t[0] = (l.x - f[23]) / sc;  // prior-frame impulses are features 23..25
      t[1] = (l.y - f[24]) / sc;
      t[2] = (l.z - f[25]) / sc;
      ok = sc > 0.f && isfinite(t[0]) && isfinite(t[1]) && isfinite(t[2]);
    }
    const unsigned bal = __ballot_sync(0xffffffffu, ok);
    if (MODE == 2 && ok) {
      const int o = base + cnt + __popc(bal & ((1u << lane) - 1u));
      if (o < cap) {
        const float4 y = d.pred[g];
        feats[3 * (size_t)o] = y.x;
        feats[3 * (size_t)o + 1] = y.y;
        feats[3 * (size_t)o + 2] = y.z;
      }
    } else if (MODE == 1 && ok) {
      const int o = base + cnt + __popc(bal & ((1u << lane) - 1u));
      if (o < cap) {
        const float4* src = reinterpret_cast<const float4*>(d.feat + g * gb::NFEAT);
        for (int k = 0; k < gb::NFEAT / 4; ++k) {
          const float4 v = src[k];
          float* dst = feats + (size_t)o * gb::NFEAT + 4 * k;
          dst[0] = v.x; dst[1] = v.y; dst[2] = v.z; dst[3] = v.w;
        }
        for (int r = 0; r < 3; ++r) lams[3 * (size_t)o + r] = t[r];
      }
    }
    cnt += __popc(bal);
  }
  if (!WRITE && lane == 0) count[e] = cnt;
}

static inline unsigned nblk(long n, int t) { return (unsigned)((n + t - 1) / t); }

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
template <typename T>
static int dalloc(SimHandle* h, T** p, size_t n) {
  if (n == 0) n = 1;
  cudaError_t e = cudaMalloc((void**)p, n * sizeof(T));
  if (e != cudaSuccess) return fail(SIM_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  h->allocs.push_back(*p);
  e = cudaMemsetAsync(*p, 0, n * sizeof(T), h->stream);
  if (e != cudaSuccess) return fail(SIM_ERR_CUDA, cudaGetErrorString(e));
  return SIM_OK;
}
template <typename T>
static int upload(SimHandle* h, T** p, const std::vector<T>& v) {
  int r = dalloc(h, p, v.size());
  if (r) return r;
  if (!v.empty()) CK(cudaMemcpyAsync(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, h->stream));
  return SIM_OK;
}

static void apply_params(SimHandle* h, const SimParams* p) {
  Dev& d = h->d;
  h->p = *p;
  d.dt = (float)p->dt;
  d.gx = (float)p->gravity[0]; d.gy = (float)p->gravity[1]; d.gz = (float)p->gravity[2];
  d.pgs_iters = p->pgs_iters; d.pgs_tol = (float)p->pgs_tol; d.pgs_max_iters = p->pgs_max_iters;
  d.baumgarte = (float)p->baumgarte; d.slop = (float)p->slop; d.margin = (float)p->margin;
  d.rest_thresh = (float)p->rest_thresh; d.sleep_lin = (float)p->sleep_lin; d.sleep_ang = (float)p->sleep_ang;
  d.sleep_steps = p->sleep_steps; d.sleep_enabled = p->sleep_enabled; d.warm_mode = p->warm_mode;
  d.plane_mu = (float)p->plane_mu; d.lambda_floor = (float)p->lambda_floor; d.match_dist = (float)p->match_dist;
  d.fp64_cond = (float)p->fp64_cond; d.log_features = p->log_features;
  d.force_limit = (float)p->force_limit;
  d.motor_mode = p->motor_mode;
  d.motor_kp = (float)p->motor_kp;
  d.motor_max_impulse = (float)p->motor_max_impulse;
}

static int check_params(const SimParams* p, int C_alloc) {
  if (!p) return fail(SIM_ERR_INVALID_ARG, "params is NULL");
  if (!(p->dt > 0) || !std::isfinite(p->dt)) return fail(SIM_ERR_INVALID_ARG, "dt must be positive");
  if (p->pgs_iters < 0 || p->pgs_max_iters < 0 || p->pgs_tol < 0) return fail(SIM_ERR_INVALID_ARG, "bad PGS settings");
  if (p->max_contacts < 1 || p->max_contacts > SIM_MAX_CONTACTS)
    return fail(SIM_ERR_INVALID_ARG, "max_contacts out of [1, SIM_MAX_CONTACTS]");
  if (C_alloc > 0 && p->max_contacts != C_alloc) return fail(SIM_ERR_INVALID_ARG, "max_contacts cannot change");
  if (p->warm_mode < 0 || p->warm_mode > 2) return fail(SIM_ERR_INVALID_ARG, "warm_mode must be 0, 1 or 2");
  if (p->sleep_steps < 1) return fail(SIM_ERR_INVALID_ARG, "sleep_steps must be >= 1");
  if (!(p->margin >= 0)) return fail(SIM_ERR_INVALID_ARG, "margin must be >= 0");
  if (!std::isfinite(p->force_limit)) return fail(SIM_ERR_INVALID_ARG, "force_limit must be finite");
  if (p->motor_mode != 0 && p->motor_mode != 1) return fail(SIM_ERR_INVALID_ARG, "motor_mode must be 0 or 1");
  if (p->motor_mode && !(p->motor_kp >= 0 && p->motor_max_impulse >= 0 && std::isfinite(p->motor_kp) &&
                         std::isfinite(p->motor_max_impulse)))
    return fail(SIM_ERR_INVALID_ARG, "motor_kp and motor_max_impulse must be finite and >= 0");
  return SIM_OK;
}

static void reset_graph(SimHandle* h) {
  if (h->graph) cudaGraphExecDestroy(h->graph);
  h->graph = nullptr;
  h->graph_n = 0;
}

static int ensure_stage(SimHandle* h, size_t floats) {
  if (floats <= h->stage_floats) return SIM_OK;
  if (h->stage) { cudaStreamSynchronize(h->stream); cudaFree(h->stage); }
  h->stage = nullptr;
  cudaError_t e = cudaMalloc((void**)&h->stage, floats * sizeof(float));
  if (e != cudaSuccess) { h->stage_floats = 0; return fail(SIM_ERR_OOM, "staging buffer"); }
  h->stage_floats = floats;
  return SIM_OK;
}

namespace gb {
// internal access for entry points defined in other translation units
int handle_internals(SimHandle* h, const Dev** d, cudaStream_t* s, int* device) {
  if (!h) return fail(SIM_ERR_INVALID_ARG, "handle is NULL");
  *d = &h->d;
  *s = h->stream;
  *device = h->device;
  return SIM_OK;
}
int report_error(int code, const std::string& msg) { return fail(code, msg); }
// the thread's last error becomes the handle's (calls defined in other translation units)
void note_handle_error(SimHandle* h) {
  if (h) h->last_err = g_err;
}

// The contact-impulse log of the last step (sim_log_contacts and its allocation-free
// variant): per-environment counts of logged contacts into prefix[0..E), their
// exclusive prefix sums and total into prefix[0..E] (E + 1 device ints owned by the
// caller), then the rows, enqueued on s.  With preds the network outputs of the same
// rows go to feats (3 per row) instead of features and targets (sim_log_predictions).
int enqueue_contact_log(const Dev& d, cudaStream_t s, int* prefix, float* feats, float* lams, int cap,
                        bool preds) {
  constexpr int WPB = 4;  // environments (warps) per block
  const unsigned blocks = (unsigned)((d.E + WPB - 1) / WPB);
  if (d.E) k_log_rows<0><<<blocks, 32 * WPB, 0, s>>>(d, nullptr, prefix, nullptr, nullptr, 0);
  gb::k_exclusive_scan<<<1, 1024, 0, s>>>(prefix, d.E);
  if (cap > 0 && d.E) {
    if (preds) k_log_rows<2><<<blocks, 32 * WPB, 0, s>>>(d, prefix, nullptr, feats, nullptr, cap);
    else k_log_rows<1><<<blocks, 32 * WPB, 0, s>>>(d, prefix, nullptr, feats, lams, cap);
  }
  CK(cudaGetLastError());
  return SIM_OK;
}
}  // namespace gb

extern "C" {

const char* sim_last_error(const SimHandle* h) { return h ? h->last_err.c_str() : g_err.c_str(); }

static SimLaunchShape default_shape() {
  SimLaunchShape k;
  k.collide_warps = 4; k.collide_persistent = 0;
  k.rows_warps = 4; k.rows_persistent = 0;
  k.pgs_warps = 4; k.pgs_persistent = 0; k.pgs_lpt = 1; k.pgs_lanes = 32; k.pgs_min_blocks = 2;
  k.pgs_heavy_sms = 0; k.pgs_stage_contacts = 0; k.pgs_stage_pool = 0;
  k.aba_lanes = 32;
  k.partitions = 1;
  k.aba_overlap = 1;
  k.fused = 0;
  return k;
}

static int warps_index(int w) { return w == 1 ? 0 : w == 2 ? 1 : w == 4 ? 2 : w == 8 ? 3 : -1; }

// collision (0) and row-build (1) kernels: resident blocks per SM at `warps` warps per block
static int occupancy(const SimHandle* h, int kernel, int warps) {
  int i = warps_index(warps);
  return i < 0 ? 0 : h->occ[kernel][i];
}

static gb::KShape kshape(const SimHandle* h, int kernel, int warps, int persistent) {
  gb::KShape k{};
  k.warps = warps;
  k.persistent = persistent;
  k.grid_cap = occupancy(h, kernel, warps) * h->sm_count;
  k.lanes = 32;
  k.min_blocks = 2;
  return k;
}

static bool shape_ok(const SimHandle* h, int kernel, int warps, int persistent) {
  return (persistent == 0 || persistent == 1) && occupancy(h, kernel, warps) > 0;
}

// PGS: resident blocks per SM of shape k (0: invalid or does not fit)
static int pgs_occupancy(const SimHandle* h, const SimLaunchShape& k) {
  const bool ok = warps_index(k.pgs_warps) >= 0 && (k.pgs_lanes == 32 || k.pgs_lanes == 16 || k.pgs_lanes == 8) &&
                  (k.pgs_persistent == 0 || k.pgs_persistent == 1) && (k.pgs_lpt == 0 || k.pgs_lpt == 1) &&
                  (k.pgs_min_blocks == 2 || ((k.pgs_min_blocks == 1 || k.pgs_min_blocks == 3) && k.pgs_lanes == 32)) &&
                  k.pgs_stage_contacts >= 0 && k.pgs_stage_pool >= 0 &&
                  (k.pgs_heavy_sms == 0 || (k.pgs_heavy_sms > 0 && k.pgs_heavy_sms <= std::min(h->sm_count, gb::MAX_HEAVY_SMS) &&
                                            k.pgs_persistent == 1 && k.pgs_lpt == 1));
  if (!ok) return 0;
  return gb::occupancy_pgs(h->d, h->max_obj, h->max_arts, k.pgs_warps, k.pgs_lanes, k.pgs_min_blocks,
                           k.pgs_stage_contacts, k.pgs_stage_pool);
}

static gb::KShape pgs_kshape(const SimHandle* h, const SimLaunchShape& s) {
  gb::KShape k{};
  k.warps = s.pgs_warps;
  k.persistent = s.pgs_persistent;
  k.grid_cap = h->pgs_occ * h->sm_count;
  k.lanes = s.pgs_lanes;
  k.min_blocks = s.pgs_min_blocks;
  k.heavy_sms = s.pgs_heavy_sms;
  k.stage_contacts = s.pgs_stage_contacts;
  k.stage_pool = s.pgs_stage_pool;
  return k;
}

// applies a validated shape
static void apply_shape(SimHandle* h, const SimLaunchShape& k) {
  h->shape = k;
  h->pgs_occ = pgs_occupancy(h, k);
}

// Copy the live per-environment state into the reset template (to_template) or back.
static int copy_template(SimHandle* h, bool to_template) {
  const Dev& d = h->d;
  auto& t = h->tmpl;
  auto cp = [&](void* live, void* tm, size_t bytes) -> cudaError_t {
    if (bytes == 0) return cudaSuccess;
    return to_template ? cudaMemcpyAsync(tm, live, bytes, cudaMemcpyDeviceToDevice, h->stream)
                       : cudaMemcpyAsync(live, tm, bytes, cudaMemcpyDeviceToDevice, h->stream);
  };
  const size_t f4o = sizeof(float4) * d.NO, f4a = sizeof(float4) * d.NA, fj = sizeof(float) * d.NJ;
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cp(d.obj_pos, t.obj_pos, f4o);
  if (e == cudaSuccess) e = cp(d.obj_comp, t.obj_comp, f4o);
  if (e == cudaSuccess) e = cp(d.obj_quat, t.obj_quat, f4o);
  if (e == cudaSuccess) e = cp(d.obj_vel, t.obj_vel, f4o);
  if (e == cudaSuccess) e = cp(d.obj_omega, t.obj_omega, f4o);
  if (e == cudaSuccess) e = cp(d.obj_awake, t.obj_awake, sizeof(int) * d.NO);
  if (e == cudaSuccess) e = cp(d.obj_ctr, t.obj_ctr, sizeof(int) * d.NO);
  if (e == cudaSuccess) e = cp(d.j_q, t.j_q, fj);
  if (e == cudaSuccess) e = cp(d.j_qcomp, t.j_qcomp, fj);
  if (e == cudaSuccess) e = cp(d.j_qd, t.j_qd, fj);
  if (e == cudaSuccess) e = cp(d.j_target, t.j_target, fj);
  if (e == cudaSuccess) e = cp(d.j_lim_lambda, t.j_lim_lambda, fj);
  if (e == cudaSuccess) e = cp(d.j_motor_lambda, t.j_motor_lambda, fj);
  if (e == cudaSuccess) e = cp(d.j_lim_side, t.j_lim_side, sizeof(int) * d.NJ);
  if (e == cudaSuccess) e = cp(d.art_base_pos, t.base_pos, f4a);
  if (e == cudaSuccess) e = cp(d.art_base_quat, t.base_quat, f4a);
  if (e != cudaSuccess) return fail(SIM_ERR_CUDA, std::string("reset template: ") + cudaGetErrorString(e));
  return SIM_OK;
}

int sim_create(const SimBatchDesc* desc, const SimParams* params, void* cuda_stream, SimHandle** out) {
  if (!out) return fail(SIM_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!desc) return fail(SIM_ERR_INVALID_ARG, "desc is NULL");
  int r = check_params(params, 0);
  if (r) return r;
  const SimBatchDesc& D = *desc;
  const int E = D.n_envs;
  if (E < 0) return fail(SIM_ERR_INVALID_ARG, "n_envs < 0");
  if (!D.obj_off || !D.stat_off || !D.art_off || !D.joint_off || !D.env_plane)
    return fail(SIM_ERR_INVALID_ARG, "missing offset arrays");
  const int NO = D.obj_off[E], NS = D.stat_off[E], NA = D.art_off[E];
  if (D.obj_off[0] != 0 || D.stat_off[0] != 0 || D.art_off[0] != 0) return fail(SIM_ERR_INVALID_ARG, "offsets must start at 0");
  for (int e = 0; e < E; ++e)
    if (D.obj_off[e + 1] < D.obj_off[e] || D.stat_off[e + 1] < D.stat_off[e] || D.art_off[e + 1] < D.art_off[e])
      return fail(SIM_ERR_INVALID_ARG, "offsets must be non-decreasing");
  if (D.joint_off[0] != 0) return fail(SIM_ERR_INVALID_ARG, "joint_off must start at 0");
  for (int a = 0; a < NA; ++a) {
    int n = D.joint_off[a + 1] - D.joint_off[a];
    if (n < 1 || n > SIM_MAX_DOF) return fail(SIM_ERR_INVALID_ARG, "articulation joint count out of [1, 9]");
  }
  const int NJ = D.joint_off[NA];
  auto need = [&](const void* p, const char* name) { return p ? 0 : fail(SIM_ERR_INVALID_ARG, std::string(name) + " is NULL"); };
  if (NO && (need(D.obj_shape, "obj_shape") || need(D.obj_half, "obj_half") || need(D.obj_mass, "obj_mass") ||
             need(D.obj_mu, "obj_mu") || need(D.obj_rest, "obj_rest") || need(D.obj_pos, "obj_pos") ||
             need(D.obj_quat, "obj_quat") || need(D.obj_vel, "obj_vel") || need(D.obj_omega, "obj_omega")))
    return SIM_ERR_INVALID_ARG;
  if (NS && (need(D.stat_pos, "stat_pos") || need(D.stat_quat, "stat_quat") || need(D.stat_half, "stat_half") ||
             need(D.stat_mu, "stat_mu")))
    return SIM_ERR_INVALID_ARG;
  if (NA && (need(D.art_base_pos, "art_base_pos") || need(D.art_base_quat, "art_base_quat") ||
             need(D.art_has_base_coll, "art_has_base_coll") || need(D.art_base_coll_off, "art_base_coll_off") ||
             need(D.art_base_coll_half, "art_base_coll_half") || need(D.art_kinematic, "art_kinematic") ||
             need(D.joint_parent, "joint_parent") || need(D.joint_type, "joint_type") || need(D.joint_axis, "joint_axis") ||
             need(D.joint_origin_pos, "joint_origin_pos") || need(D.joint_origin_quat, "joint_origin_quat") ||
             need(D.joint_com, "joint_com") || need(D.joint_half, "joint_half") || need(D.joint_mass, "joint_mass") ||
             need(D.joint_lo, "joint_lo") || need(D.joint_hi, "joint_hi") || need(D.joint_has_limit, "joint_has_limit") ||
             need(D.joint_kp, "joint_kp") || need(D.joint_kd, "joint_kd") || need(D.joint_mu, "joint_mu") ||
             need(D.joint_q0, "joint_q0") || need(D.joint_qd0, "joint_qd0") || need(D.joint_target, "joint_target")))
    return SIM_ERR_INVALID_ARG;
  for (int i = 0; i < NO; ++i) {
    if (D.obj_shape[i] != 0 && D.obj_shape[i] != 1) return fail(SIM_ERR_INVALID_ARG, "obj_shape must be 0 or 1");
    if (!(D.obj_mass[i] > 0)) return fail(SIM_ERR_INVALID_ARG, "obj_mass must be positive");
    for (int k = 0; k < 3; ++k)
      if (!(D.obj_half[3 * i + k] > 0) && (D.obj_shape[i] == 1 || k == 0))
        return fail(SIM_ERR_INVALID_ARG, "object sizes must be positive");
  }
  for (int j = 0; j < NJ; ++j) {
    if (!(D.joint_mass[j] > 0)) return fail(SIM_ERR_INVALID_ARG, "joint_mass must be positive");
    if (D.joint_type[j] != 0 && D.joint_type[j] != 1) return fail(SIM_ERR_INVALID_ARG, "joint_type must be 0 or 1");
  }
  // derived per-env tables
  std::vector<int> base_off(E + 1, 0), base_art, obj_env(NO), j_env(NJ), j_art(NJ), art_env(NA);
  int max_coll = 1, max_obj = 0, max_arts = 0;
  for (int e = 0; e < E; ++e) {
    int nobj = D.obj_off[e + 1] - D.obj_off[e];
    int narts = D.art_off[e + 1] - D.art_off[e];
    if (nobj > max_obj) max_obj = nobj;
    if (narts > max_arts) max_arts = narts;
    if (nobj > SIM_MAX_OBJECTS) return fail(SIM_ERR_INVALID_ARG, "more than SIM_MAX_OBJECTS objects in an env");
    if (narts > SIM_MAX_ARTS) return fail(SIM_ERR_INVALID_ARG, "more than SIM_MAX_ARTS articulations in an env");
    for (int i = D.obj_off[e]; i < D.obj_off[e + 1]; ++i) obj_env[i] = e;
    int nlinks = 0;
    for (int a = D.art_off[e]; a < D.art_off[e + 1]; ++a) {
      art_env[a] = e;
      if (D.art_has_base_coll[a]) base_art.push_back(a);
      for (int j = D.joint_off[a]; j < D.joint_off[a + 1]; ++j) {
        int jl = j - D.joint_off[a];
        if (D.joint_parent[j] < -1 || D.joint_parent[j] >= jl)
          return fail(SIM_ERR_INVALID_ARG, "joint_parent must be -1 or a smaller joint index");
        j_env[j] = e;
        j_art[j] = a;
        ++nlinks;
      }
    }
    base_off[e + 1] = (int)base_art.size();
    int nc = nobj + nlinks + (base_off[e + 1] - base_off[e]) + (D.stat_off[e + 1] - D.stat_off[e]) + (D.env_plane[e] ? 1 : 0);
    if (nc > SIM_MAX_COLLIDERS) return fail(SIM_ERR_INVALID_ARG, "more than SIM_MAX_COLLIDERS colliders in an env");
    if (nc > max_coll) max_coll = nc;
  }

  SimHandle* h = new SimHandle();
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    delete h;
    return fail(SIM_ERR_CUDA, "cudaGetDevice failed");
  }
  h->stream = (cudaStream_t)cuda_stream;
  h->cap_stream = nullptr;
  if (cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    delete h;
    return fail(SIM_ERR_CUDA, "cudaStreamCreateWithFlags failed");
  }
  for (int p = 0; p < SIM_MAX_PARTITIONS; ++p) { h->pstream[p] = nullptr; h->join_ev[p] = nullptr; }
  h->fork_ev = nullptr;
  {
    bool ok = cudaEventCreateWithFlags(&h->fork_ev, cudaEventDisableTiming) == cudaSuccess;
    for (int p = 0; p < SIM_MAX_PARTITIONS && ok; ++p)
      ok = cudaStreamCreateWithFlags(&h->pstream[p], cudaStreamNonBlocking) == cudaSuccess &&
           cudaEventCreateWithFlags(&h->join_ev[p], cudaEventDisableTiming) == cudaSuccess &&
           cudaStreamCreateWithFlags(&h->astream[p], cudaStreamNonBlocking) == cudaSuccess &&
           cudaEventCreateWithFlags(&h->afork_ev[p], cudaEventDisableTiming) == cudaSuccess &&
           cudaEventCreateWithFlags(&h->ajoin_ev[p], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
      sim_destroy(h);
      return fail(SIM_ERR_CUDA, "partition streams / events");
    }
  }
  h->graph = nullptr;
  h->graph_n = 0;
  h->stage = nullptr;
  h->stage_floats = 0;
  h->mlp_ready = 0;
  h->mlp = nullptr;
  h->max_coll = max_coll;
  h->max_obj = max_obj;
  h->max_arts = max_arts;
  h->profiling = 0;
  h->prof_n = 0;
  h->launches = 0;
  h->kernels_per_step = 0;
  for (int k = 0; k < SIM_N_STAGES; ++k) h->stage_launches[k] = 0;
  h->graph_kernels = 0;
  Dev& d = h->d;
  std::memset(&d, 0, sizeof(d));
  d.E = E; d.NO = NO; d.NS = NS; d.NA = NA; d.NJ = NJ; d.C = params->max_contacts;
  apply_params(h, params);
  const int C = d.C;
  auto F4 = [](const double* p, int w, int n, float fill = 0.f) {
    std::vector<float4> v(n);
    for (int i = 0; i < n; ++i) {
      float c[4] = {fill, fill, fill, fill};
      for (int k = 0; k < w; ++k) c[k] = (float)p[(size_t)w * i + k];
      v[i] = make_float4(c[0], c[1], c[2], c[3]);
    }
    return v;
  };
  auto I1 = [](const int* p, int n) { return std::vector<int>(p, p + n); };
  auto Fv = [](const double* p, int n) {
    std::vector<float> v(n);
    for (int i = 0; i < n; ++i) v[i] = (float)p[i];
    return v;
  };
  int rc = 0;
#define UP(field, vec) do { rc = upload(h, &field, vec); if (rc != 0) { sim_destroy(h); return rc; } } while (0)
#define AL(field, n) do { rc = dalloc(h, &field, (size_t)(n)); if (rc != 0) { sim_destroy(h); return rc; } } while (0)
  {
    const int* tmp;
    int* p;
    UP(p, I1(D.obj_off, E + 1)); d.obj_off = p;
    UP(p, I1(D.stat_off, E + 1)); d.stat_off = p;
    UP(p, I1(D.art_off, E + 1)); d.art_off = p;
    UP(p, I1(D.env_plane, E)); d.env_plane = p;
    UP(p, base_off); d.base_off = p;
    UP(p, base_art); d.base_art = p;
    UP(p, obj_env); d.obj_env = p;
    UP(p, j_env); d.j_env = p;
    UP(p, j_art); d.j_art = p;
    UP(p, art_env); h->art_env = p;
    UP(p, I1(D.joint_off, NA + 1)); d.joint_off = p;
    std::vector<int> multi, single;
    for (int a = 0; a < NA; ++a) (D.joint_off[a + 1] - D.joint_off[a] > 1 ? multi : single).push_back(a);
    UP(p, multi); d.art_multi = p; d.n_art_multi = (int)multi.size();
    UP(p, single); d.art_single = p; d.n_art_single = (int)single.size();
    h->art_off_h.assign(D.art_off, D.art_off + E + 1);
    h->multi_h = multi;
    h->single_h = single;
    (void)tmp;
  }
  AL(d.status, E); AL(d.iters, E); AL(d.n_contacts, E); AL(d.n_rows, E); AL(d.n_limit, E); AL(d.n_colours, E);
  AL(d.robot_force, E); AL(d.robot_force_acc, E);
  AL(d.fp64_used, E); AL(d.pair_count, E); AL(d.pairs, (size_t)E * gb::PAIR_CAP); AL(d.resid, E);
  // objects
  {
    std::vector<float4> pos = F4(D.obj_pos, 3, NO), quat = F4(D.obj_quat, 4, NO), vel = F4(D.obj_vel, 3, NO),
                        om = F4(D.obj_omega, 3, NO), half = F4(D.obj_half, 3, NO);
    for (int i = 0; i < NO; ++i) {
      half[i].w = (float)D.obj_shape[i];
      if (D.obj_shape[i] == 0) half[i].y = half[i].z = half[i].x;
    }
    std::vector<float2> mat(NO);
    for (int i = 0; i < NO; ++i) mat[i] = make_float2((float)D.obj_mu[i], (float)D.obj_rest[i]);
    std::vector<int> awake(NO, 1);
    float4* f;
    UP(d.obj_pos, pos); AL(d.obj_comp, NO); UP(d.obj_quat, quat); UP(d.obj_vel, vel); UP(d.obj_omega, om);
    AL(d.obj_vstar, NO); AL(d.obj_wstar, NO);
    UP(f, half); d.obj_half = f;
    float* mass;
    UP(mass, Fv(D.obj_mass, NO));
    float4* inv;
    AL(inv, NO); d.obj_inv = inv;
    float2* m2;
    UP(m2, mat); d.obj_mat = m2;
    UP(d.obj_awake, awake); AL(d.obj_ctr, NO);
    if (NO) k_init_bodies<<<nblk(NO, 256), 256, 0, h->stream>>>(NO, d.obj_half, mass, inv);
  }
  // statics
  {
    std::vector<float4> sp = F4(D.stat_pos, 3, NS);
    for (int i = 0; i < NS; ++i) sp[i].w = (float)D.stat_mu[i];
    float4* f;
    UP(f, sp); d.stat_pos = f;
    UP(f, F4(D.stat_quat, 4, NS)); d.stat_quat = f;
    UP(f, F4(D.stat_half, 3, NS)); d.stat_half = f;
  }
  // articulations and joints
  {
    float4* f;
    int* p;
    UP(d.art_base_pos, F4(D.art_base_pos, 3, NA)); UP(d.art_base_quat, F4(D.art_base_quat, 4, NA));
    UP(p, I1(D.art_has_base_coll, NA)); d.art_has_bc = p;
    UP(p, I1(D.art_kinematic, NA)); d.art_kin = p;
    UP(f, F4(D.art_base_coll_off, 3, NA)); d.art_bc_off = f;
    UP(f, F4(D.art_base_coll_half, 3, NA)); d.art_bc_half = f;
    UP(p, I1(D.joint_parent, NJ)); d.j_parent = p;
    {
      std::vector<unsigned> anc(NJ);
      for (int a = 0; a < NA; ++a)
        for (int j = D.joint_off[a]; j < D.joint_off[a + 1]; ++j) {
          unsigned m = 0;
          for (int k = j - D.joint_off[a]; k >= 0; k = D.joint_parent[D.joint_off[a] + k]) m |= 1u << k;
          anc[j] = m;
        }
      unsigned* pa;
      UP(pa, anc); d.j_anc = pa;
    }
    UP(p, I1(D.joint_type, NJ)); d.j_type = p;
    UP(f, F4(D.joint_axis, 3, NJ)); d.j_axis = f;
    UP(f, F4(D.joint_origin_pos, 3, NJ)); d.j_opos = f;
    UP(f, F4(D.joint_origin_quat, 4, NJ)); d.j_oquat = f;
    std::vector<float4> com = F4(D.joint_com, 3, NJ), half = F4(D.joint_half, 3, NJ), lim(NJ);
    std::vector<float2> gain(NJ);
    for (int j = 0; j < NJ; ++j) {
      com[j].w = (float)D.joint_mass[j];
      half[j].w = (float)D.joint_mu[j];
      lim[j] = make_float4((float)D.joint_lo[j], (float)D.joint_hi[j], (float)D.joint_has_limit[j], 0.f);
      gain[j] = make_float2((float)D.joint_kp[j], (float)D.joint_kd[j]);
    }
    UP(f, com); d.j_com = f;
    UP(f, half); d.j_half = f;
    UP(f, lim); d.j_lim = f;
    float2* g2;
    UP(g2, gain); d.j_gain = g2;
    UP(d.j_q, Fv(D.joint_q0, NJ)); AL(d.j_qcomp, NJ); UP(d.j_qd, Fv(D.joint_qd0, NJ));
    UP(d.j_target, Fv(D.joint_target, NJ)); AL(d.j_lim_lambda, NJ); AL(d.j_lim_side, NJ);
    AL(d.j_motor_lambda, NJ);
    AL(d.l_com, NJ); AL(d.l_r0, NJ); AL(d.l_r1, NJ); AL(d.l_r2, NJ); AL(d.l_ja, NJ); AL(d.l_jo, NJ);
    AL(d.j_qdd, NJ); AL(d.j_qdstar, NJ); AL(d.a_minv, (size_t)NA * 81);
  }
  // contacts, cache, rows
  {
    size_t EC = (size_t)E * C;
    AL(d.c_key, EC); AL(d.c_p, EC); AL(d.c_n, EC); AL(d.c_lam, EC);
    AL(d.cache_count, E); AL(d.cache_key, EC); AL(d.cache_p, EC); AL(d.cache_lam, EC);
    AL(d.r_t1, EC); AL(d.r_meff, EC); AL(d.r_lam, EC); AL(d.r_ra, EC); AL(d.r_rb, EC); AL(d.r_ends, EC);
    AL(d.ap, (size_t)E * gb::APOOL * gb::APS);
    AL(d.ap_count, E);
    AL(d.perm, E);
    AL(d.wq, 8 * SIM_MAX_PARTITIONS);  // 8 counters per partition
    AL(d.sm_rank, (size_t)gb::MAX_HEAVY_SMS * SIM_MAX_PARTITIONS);
    AL(d.lr_info, (size_t)E * gb::LCAP); AL(d.lr_data, (size_t)E * gb::LCAP); AL(d.lr_w, (size_t)E * gb::LCAP * gb::MAX_DOF);
    if (params->log_features || params->warm_mode == 2) {
      AL(d.feat, EC * gb::NFEAT); AL(d.pred, EC); AL(d.mlp_rows, EC); AL(d.mlp_count, SIM_MAX_PARTITIONS);
    }
  }
  // the reset template starts as the batch's initial state
  {
    auto& t = h->tmpl;
    AL(t.obj_pos, NO); AL(t.obj_comp, NO); AL(t.obj_quat, NO); AL(t.obj_vel, NO); AL(t.obj_omega, NO);
    AL(t.obj_awake, NO); AL(t.obj_ctr, NO);
    AL(t.j_q, NJ); AL(t.j_qcomp, NJ); AL(t.j_qd, NJ); AL(t.j_target, NJ); AL(t.j_lim_lambda, NJ);
    AL(t.j_motor_lambda, NJ);
    AL(t.j_lim_side, NJ); AL(t.base_pos, NA); AL(t.base_quat, NA);
    if ((rc = copy_template(h, true))) { sim_destroy(h); return rc; }
  }
#undef UP
#undef AL
  gb::configure_aba();
  gb::configure_collide(max_coll);
  gb::configure_pgs(d, max_obj, max_arts);
  gb::configure_fused();
  {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, dev);
    for (int i = 0; i < 4; ++i) {
      h->occ[0][i] = gb::occupancy_collide(max_coll, 1 << i);
      h->occ[1][i] = gb::occupancy_rows(1 << i);
    }
    SimLaunchShape k = default_shape();
    // fewer warps per block where four environments' shared memory does not fit one block
    while (k.collide_warps > 1 && !shape_ok(h, 0, k.collide_warps, 0)) k.collide_warps >>= 1;
    while (k.pgs_warps > 1 && pgs_occupancy(h, k) == 0) k.pgs_warps >>= 1;
    apply_shape(h, k);
  }
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    sim_destroy(h);
    return fail(SIM_ERR_CUDA, std::string("sim_create: ") + cudaGetErrorString(e));
  }
  // (re)read the device address of sim_log_contacts_noalloc's fixed scratch on this
  // device: creation is never inside a stream capture (it allocates), and a handle
  // created after a device reset must not see an address cached before it
  if ((r = gb::noalloc_scratch_refresh())) {
    sim_destroy(h);
    return r;
  }
  *out = h;
  return SIM_OK;
}

void sim_destroy(SimHandle* h) {
  if (!h) return;
  DevGuard dev_guard_(h->device, nullptr);
  cudaStreamSynchronize(h->stream);
  reset_graph(h);
  for (void* p : h->allocs) cudaFree(p);
  if (h->stage) cudaFree(h->stage);
  if (h->mlp) gb::mlp_destroy(h->mlp);
  for (cudaEvent_t ev : h->events) cudaEventDestroy(ev);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  for (int p = 0; p < SIM_MAX_PARTITIONS; ++p) {
    if (h->pstream[p]) cudaStreamDestroy(h->pstream[p]);
    if (h->join_ev[p]) cudaEventDestroy(h->join_ev[p]);
    if (h->astream[p]) cudaStreamDestroy(h->astream[p]);
    if (h->afork_ev[p]) cudaEventDestroy(h->afork_ev[p]);
    if (h->ajoin_ev[p]) cudaEventDestroy(h->ajoin_ev[p]);
  }
  if (h->fork_ev) cudaEventDestroy(h->fork_ev);
  delete h;
}

int sim_set_params(SimHandle* h, const SimParams* params) {
  if (!h) return fail(SIM_ERR_INVALID_ARG, "handle is NULL");
  ON_DEVICE(h);
  int r = check_params(params, h->d.C);
  if (r) return r;
  if ((params->log_features || params->warm_mode == 2) && !h->d.feat) {
    size_t EC = (size_t)h->d.E * h->d.C;
    if ((r = dalloc(h, &h->d.feat, EC * gb::NFEAT))) return r;
    if ((r = dalloc(h, &h->d.pred, EC))) return r;
    if ((r = dalloc(h, &h->d.mlp_rows, EC))) return r;
    if ((r = dalloc(h, &h->d.mlp_count, SIM_MAX_PARTITIONS))) return r;
  }
  apply_params(h, params);
  reset_graph(h);
  return SIM_OK;
}

int sim_set_joint_targets(SimHandle* h, const float* targets, int on_device) {
  if (!h || !targets) return fail(SIM_ERR_INVALID_ARG, "NULL argument");
  ON_DEVICE(h);
  if (h->d.NJ == 0) return SIM_OK;
  CK(cudaMemcpyAsync(h->d.j_target, targets, sizeof(float) * h->d.NJ,
                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
  if (!on_device) CK(cudaStreamSynchronize(h->stream));  // the caller may reuse its host buffer
  return SIM_OK;
}

int sim_set_base_pose(SimHandle* h, const float* xy_yaw, int on_device) {
  if (!h || !xy_yaw) return fail(SIM_ERR_INVALID_ARG, "NULL argument");
  ON_DEVICE(h);
  if (h->d.E == 0 || h->d.NA == 0) return SIM_OK;
  const float* src = xy_yaw;
  if (!on_device) {
    int r = ensure_stage(h, (size_t)h->d.E * 3);
    if (r) return r;
    CK(cudaMemcpyAsync(h->stage, xy_yaw, sizeof(float) * 3 * h->d.E, cudaMemcpyHostToDevice, h->stream));
    src = h->stage;
  }
  k_set_base<<<nblk(h->d.NA, 256), 256, 0, h->stream>>>(h->d.NA, h->art_env, h->d.art_kin, src, h->d.art_base_pos,
                                                          h->d.art_base_quat);
  CK(cudaGetLastError());
  if (!on_device) CK(cudaStreamSynchronize(h->stream));
  return SIM_OK;
}

static int ensure_events(SimHandle* h, int n) {
  size_t need = (size_t)n * (SIM_N_STAGES + 1);
  while (h->events.size() < need) {
    cudaEvent_t ev;
    CK(cudaEventCreate(&ev));
    h->events.push_back(ev);
  }
  return SIM_OK;
}

// Enqueue one physics step; with profiling, events bracket every stage.
// During stream capture an event record must be an external node to be timed at replay.
static inline void record(cudaEvent_t ev, cudaStream_t st, bool capturing) {
  if (capturing) cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal);
  else cudaEventRecord(ev, st);
}

// The batch's environments [e0, e1) of partition p of P (equal shares in environment
// order): per-environment arrays offset by e0, work-queue counters, heavy-SM ranks and
// the network's row count of its own, the articulation lists restricted to its
// articulations.  Objects, joints and articulations keep their batch-wide indices (the
// CSR offsets hold them), so every kernel runs unchanged on a view.
static Dev partition_view(const SimHandle* h, int p, int P) {
  const Dev& d = h->d;
  if (P <= 1) return d;
  const int e0 = (int)((long long)d.E * p / P), e1 = (int)((long long)d.E * (p + 1) / P);
  const size_t C = d.C, e0c = (size_t)e0 * C;
  Dev v = d;
  v.E = e1 - e0;
  v.env0 = e0;
  v.obj_off += e0; v.stat_off += e0; v.art_off += e0; v.env_plane += e0; v.base_off += e0;
  v.status += e0; v.iters += e0; v.n_contacts += e0; v.n_rows += e0; v.n_limit += e0; v.n_colours += e0;
  v.fp64_used += e0; v.pair_count += e0; v.pairs += (size_t)e0 * gb::PAIR_CAP;
  v.robot_force += e0; v.robot_force_acc += e0; v.resid += e0;
  v.c_key += e0c; v.c_p += e0c; v.c_n += e0c; v.c_lam += e0c;
  v.cache_count += e0; v.cache_key += e0c; v.cache_p += e0c; v.cache_lam += e0c;
  v.r_t1 += e0c; v.r_meff += e0c; v.r_lam += e0c; v.r_ra += e0c; v.r_rb += e0c; v.r_ends += e0c;
  v.ap += (size_t)e0 * gb::APOOL * gb::APS; v.ap_count += e0;
  v.lr_info += (size_t)e0 * gb::LCAP; v.lr_data += (size_t)e0 * gb::LCAP;
  v.lr_w += (size_t)e0 * gb::LCAP * gb::MAX_DOF;
  v.perm += e0;
  v.wq += 8 * p;
  v.sm_rank += (size_t)gb::MAX_HEAVY_SMS * p;
  if (d.feat) {
    v.feat += e0c * gb::NFEAT; v.pred += e0c; v.mlp_rows += e0c; v.mlp_count += p;
  }
  const int a0 = h->art_off_h[e0], a1 = h->art_off_h[e1];
  auto range = [&](const std::vector<int>& l, const int* dev, const int** out, int* n) {
    const int i0 = (int)(std::lower_bound(l.begin(), l.end(), a0) - l.begin());
    const int i1 = (int)(std::lower_bound(l.begin(), l.end(), a1) - l.begin());
    *out = dev + i0;
    *n = i1 - i0;
  };
  range(h->multi_h, d.art_multi, &v.art_multi, &v.n_art_multi);
  range(h->single_h, d.art_single, &v.art_single, &v.n_art_single);
  return v;
}

// One physics step of the environments of view d on stream st (heavy SMs of the PGS
// launch: heavy_base .. heavy_base + heavy - 1); returns the kernels enqueued.
static int enqueue_step(SimHandle* h, const Dev& d, int sub, cudaStream_t st, bool capturing, int heavy,
                        int heavy_base, int part) {
  cudaEvent_t* ev = h->profiling == 1 ? &h->events[(size_t)sub * (SIM_N_STAGES + 1)] : nullptr;
  // mode 2: events around the PGS kernel only (each event node in a graph costs a few us)
  cudaEvent_t* evp = h->profiling == 2 ? &h->events[(size_t)sub * (SIM_N_STAGES + 1)] : nullptr;
  // the LPT order only schedules PGS work (any order gives the same results): it is
  // recomputed on the first physics step of each sim_step call
  const bool lpt = h->shape.pgs_lpt != 0 && sub == 0;
  // ABA on the side stream beside forward kinematics and collision, which need only the
  // link poses; in sequence while kernel timing is on (each kernel timed alone)
  const bool side = h->shape.aba_overlap != 0 && !h->profiling && d.n_art_multi + d.n_art_single > 0;
  const bool arts = d.n_art_multi > 0 || d.n_art_single > 0;
  int nk[SIM_N_STAGES] = {(d.n_art_multi > 0) + (d.n_art_single > 0) + arts, d.E > 0, d.E > 0,
                          d.warm_mode == 2 && h->mlp_ready && d.E > 0, d.E > 0 && lpt, d.E > 0,
                          0};  // integration runs in the PGS kernel's write-back
  if (ev) record(ev[0], st, capturing);
  if (side) {
    cudaEventRecord(h->afork_ev[part], st);
    cudaStreamWaitEvent(h->astream[part], h->afork_ev[part], 0);
    gb::launch_aba(d, h->astream[part], h->shape.aba_lanes);
    cudaEventRecord(h->ajoin_ev[part], h->astream[part]);
    gb::launch_fk(d, st);
  } else {
    gb::launch_fk(d, st);
    gb::launch_aba(d, st, h->shape.aba_lanes);
  }
  if (ev) record(ev[1], st, capturing);
  const SimLaunchShape& k = h->shape;
  gb::launch_collide(d, st, h->max_coll, kshape(h, 0, k.collide_warps, k.collide_persistent));
  if (side) cudaStreamWaitEvent(st, h->ajoin_ev[part], 0);  // the rows read M^-1 and q̇*
  if (ev) record(ev[2], st, capturing);
  if (nk[3]) cudaMemsetAsync(d.mlp_count, 0, sizeof(int), st);  // the row kernel lists the network's rows
  gb::launch_rows(d, st, kshape(h, 1, k.rows_warps, k.rows_persistent));
  if (ev) record(ev[3], st, capturing);
  if (nk[3]) gb::launch_mlp_infer(d, h->mlp, st);
  if (ev) record(ev[4], st, capturing);
  if (lpt) gb::launch_lpt_order(d, st);
  if (ev) record(ev[5], st, capturing);
  if (evp) record(evp[5], st, capturing);
  gb::KShape ks = pgs_kshape(h, k);
  ks.heavy_sms = heavy;
  gb::launch_pgs(d, st, h->max_obj, h->max_arts, ks, k.pgs_lpt, heavy_base);
  if (ev) record(ev[6], st, capturing);
  if (evp) record(evp[6], st, capturing);
  if (ev) record(ev[7], st, capturing);
  int tot = 0;
  for (int k = 0; k < SIM_N_STAGES; ++k) { h->stage_launches[k] += nk[k]; tot += nk[k]; }
  return tot;
}

// The fused step kernel runs for shape.fused except while kernel timing is on (stage
// events time each stage kernel) and in warm mode 2 (the network's inference is one
// tensor-core launch over every environment's contacts between rows and PGS).
static bool fused_active(const SimHandle* h) {
  return h->shape.fused != 0 && !h->profiling && h->d.warm_mode != 2 && h->d.E > 0;
}

// Partitions in use: the shape's, or one while profiling (stage events time each
// kernel alone, and concurrent partitions would overlap them).
static int active_partitions(const SimHandle* h) {
  return h->profiling ? 1 : std::max(1, std::min(h->shape.partitions, std::max(1, h->d.E)));
}

// Enqueue n physics steps on st; returns the number of kernels enqueued.  With P
// partitions every partition's n steps go to a stream of its own, forked from st and
// joined back to it (inside a capture, parallel branches of the graph), so one
// partition's kernels fill the SMs that another's leave idle at the end of its kernels.
// The heavy SMs of the PGS launches are split between the partitions.
static long long enqueue_steps(SimHandle* h, int n, cudaStream_t st, bool capturing) {
  for (int k = 0; k < SIM_N_STAGES; ++k) h->stage_launches[k] = 0;
  long long tot = 0;
  if (fused_active(h)) {
    // the LPT order from the last step's colour and row counts, then all n steps in one
    // launch (counted with the PGS stage)
    const SimLaunchShape& k = h->shape;
    if (k.pgs_lpt) gb::launch_lpt_order(h->d, st);
    gb::launch_fused(h->d, st, n, h->max_coll, h->max_obj, h->max_arts, k.pgs_stage_contacts, k.pgs_stage_pool,
                     h->sm_count, k.pgs_lpt ? h->d.perm : nullptr);
    h->stage_launches[4] = k.pgs_lpt ? 1 : 0;
    h->stage_launches[5] = 1;
    tot = h->stage_launches[4] + 1;
    h->kernels_per_step = n > 0 ? (int)((tot + n - 1) / n) : 0;
    return tot;
  }
  const int P = active_partitions(h);
  h->last_parts = P;
  if (P == 1) {
    for (int i = 0; i < n; ++i) tot += enqueue_step(h, h->d, i, st, capturing, h->shape.pgs_heavy_sms, 0, 0);
    h->kernels_per_step = n > 0 ? (int)(tot / n) : 0;
    return tot;
  }
  const int heavy = h->shape.pgs_heavy_sms / P;
  cudaEventRecord(h->fork_ev, st);
  for (int p = 0; p < P; ++p) {
    cudaStreamWaitEvent(h->pstream[p], h->fork_ev, 0);
    const Dev v = partition_view(h, p, P);
    for (int i = 0; i < n; ++i) tot += enqueue_step(h, v, i, h->pstream[p], capturing, heavy, heavy * p, p);
    cudaEventRecord(h->join_ev[p], h->pstream[p]);
    cudaStreamWaitEvent(st, h->join_ev[p], 0);
  }
  h->kernels_per_step = n > 0 ? (int)(tot / n) : 0;
  return tot;
}

int sim_step(SimHandle* h, int n) {
  if (!h) return fail(SIM_ERR_INVALID_ARG, "handle is NULL");
  ON_DEVICE(h);
  if (n < 0) return fail(SIM_ERR_INVALID_ARG, "n < 0");
  if (n == 0) return SIM_OK;
  if (h->d.warm_mode == 2 && !h->mlp_ready) return fail(SIM_ERR_STATE, "warm_mode 2 needs sim_set_mlp first");
  if (h->profiling) {
    int r = ensure_events(h, n);
    if (r) return r;
    h->prof_n = n;
  }
  if (!h->p.use_graph) {
    long long nk = enqueue_steps(h, n, h->stream, false);
    CK(cudaGetLastError());
    h->launches += nk;
    return SIM_OK;
  }
  if (!h->graph || h->graph_n != n) {
    reset_graph(h);
    cudaGraph_t g;
    // captured on the private stream (the legacy default stream cannot be captured),
    // replayed on the caller's stream
    CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    h->graph_kernels = enqueue_steps(h, n, h->cap_stream, true);
    cudaError_t le = cudaGetLastError();
    cudaError_t ce = cudaStreamEndCapture(h->cap_stream, &g);
    if (le != cudaSuccess) return fail(SIM_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(le));
    if (ce != cudaSuccess) return fail(SIM_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(ce));
    cudaError_t ie = cudaGraphInstantiate(&h->graph, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) { h->graph = nullptr; return fail(SIM_ERR_CUDA, std::string("instantiate: ") + cudaGetErrorString(ie)); }
    h->graph_n = n;
  }
  CK(cudaGraphLaunch(h->graph, h->stream));
  h->launches += h->graph_kernels;
  return SIM_OK;
}

int sim_set_profiling(SimHandle* h, int enable) {
  if (!h) return fail(SIM_ERR_INVALID_ARG, "handle is NULL");
  ON_DEVICE(h);
  if (enable < 0 || enable > 2) return fail(SIM_ERR_INVALID_ARG, "profiling mode must be 0, 1 or 2");
  if (h->profiling != enable) reset_graph(h);
  h->profiling = enable;
  h->prof_n = 0;
  return SIM_OK;
}

int sim_kernel_times(SimHandle* h, float* ms, int* launches) {
  if (!h) return fail(SIM_ERR_INVALID_ARG, "handle is NULL");
  ON_DEVICE(h);
  if (!h->profiling || h->prof_n == 0) return fail(SIM_ERR_STATE, "no profiled sim_step");
  CK(cudaStreamSynchronize(h->stream));
  for (int k = 0; k < SIM_N_STAGES; ++k) {
    float acc = 0.f;
    const bool timed = h->profiling == 1 || k == 5;  // mode 2 times the PGS stage only
    for (int i = 0; timed && i < h->prof_n; ++i) {
      float t = 0.f;
      const size_t b = (size_t)i * (SIM_N_STAGES + 1) + k;
      CK(cudaEventElapsedTime(&t, h->events[b], h->events[b + 1]));
      acc += t;
    }
    if (ms) ms[k] = acc;
    if (launches) launches[k] = h->stage_launches[k];
  }
  return SIM_OK;
}

int sim_get_launch_shape(SimHandle* h, SimLaunchShape* out) {
  if (!h || !out) return fail(SIM_ERR_INVALID_ARG, "NULL argument");
  ON_DEVICE(h);
  *out = h->shape;
  return SIM_OK;
}

int sim_set_launch_shape(SimHandle* h, const SimLaunchShape* in) {
  if (!h || !in) return fail(SIM_ERR_INVALID_ARG, "NULL argument");
  ON_DEVICE(h);
  if (!shape_ok(h, 0, in->collide_warps, in->collide_persistent))
    return fail(SIM_ERR_INVALID_ARG, "collide_warps must be 1, 2, 4 or 8 with its shared memory within a block, "
                                     "collide_persistent 0 or 1");
  if (!shape_ok(h, 1, in->rows_warps, in->rows_persistent))
    return fail(SIM_ERR_INVALID_ARG, "rows_warps must be 1, 2, 4 or 8, rows_persistent 0 or 1");
  if (in->aba_lanes != 32 && in->aba_lanes != 16)
    return fail(SIM_ERR_INVALID_ARG, "aba_lanes must be 32 or 16");
  if (in->partitions < 1 || in->partitions > SIM_MAX_PARTITIONS || (h->d.E > 0 && in->partitions > h->d.E))
    return fail(SIM_ERR_INVALID_ARG, "partitions must be 1 .. SIM_MAX_PARTITIONS and at most the environments");
  if (in->aba_overlap != 0 && in->aba_overlap != 1) return fail(SIM_ERR_INVALID_ARG, "aba_overlap must be 0 or 1");
  if (in->fused != 0 && (in->fused != 1 || in->partitions != 1 ||
                         gb::fused_warp_bytes(h->d, h->max_coll, h->max_obj, h->max_arts, in->pgs_stage_contacts,
                                              in->pgs_stage_pool) == 0))
    return fail(SIM_ERR_INVALID_ARG, "fused must be 0 or 1, with partitions 1 and four warps' shared memory "
                                     "(stage working sets and the PGS layout) within a block");
  if (pgs_occupancy(h, *in) == 0)
    return fail(SIM_ERR_INVALID_ARG, "PGS shape: pgs_warps must be 1, 2, 4 or 8, pgs_lanes 32, 16 or 8, "
                                     "pgs_min_blocks 2 (or 1 or 3 with 32 lanes), pgs_persistent and pgs_lpt 0 or 1, "
                                     "pgs_stage_contacts and pgs_stage_pool >= 0, pgs_heavy_sms 0 or at most the SM "
                                     "count (and 256) with pgs_persistent = pgs_lpt = 1, and the block's shared "
                                     "memory must fit the device");
  apply_shape(h, *in);
  reset_graph(h);
  return SIM_OK;
}

static float median_of(std::vector<float> v) {
  if (v.empty()) return 0.f;
  std::sort(v.begin(), v.end());
  size_t n = v.size();
  return n % 2 ? v[n / 2] : 0.5f * (v[n / 2 - 1] + v[n / 2]);
}

// Runs `trials` round-robin (round 0 untimed) and returns, per trial, the median
// device ms per physics step of the collision, row-build and PGS stages and of
// the whole step (med[4 t + 0..3]).
// The state a physics step reads and writes -- the reset template's fields, the
// warm-start cache, the robot's contact forces and the status flags -- as (address,
// bytes) pairs: the autotuner saves it at the start of each round and restores it
// before every trial of the round, so that all trials of a round time the same steps.
static std::vector<std::pair<void*, size_t>> step_state(const SimHandle* h) {
  const Dev& d = h->d;
  const size_t f4o = sizeof(float4) * d.NO, f4a = sizeof(float4) * d.NA, fj = sizeof(float) * d.NJ;
  const size_t EC = (size_t)d.E * d.C;
  return {{d.obj_pos, f4o}, {d.obj_comp, f4o}, {d.obj_quat, f4o}, {d.obj_vel, f4o}, {d.obj_omega, f4o},
          {d.obj_awake, sizeof(int) * d.NO}, {d.obj_ctr, sizeof(int) * d.NO}, {d.j_q, fj}, {d.j_qcomp, fj},
          {d.j_qd, fj}, {d.j_target, fj}, {d.j_lim_lambda, fj}, {d.j_motor_lambda, fj},
          {d.j_lim_side, sizeof(int) * d.NJ}, {d.art_base_pos, f4a}, {d.art_base_quat, f4a},
          {d.cache_count, sizeof(int) * d.E}, {d.cache_key, sizeof(int4) * EC}, {d.cache_p, sizeof(float4) * EC},
          {d.cache_lam, sizeof(float4) * EC}, {d.robot_force, sizeof(float) * d.E},
          {d.robot_force_acc, sizeof(float) * d.E}, {d.status, sizeof(int) * d.E}};
}
// save (to the snapshot) or restore (from it) the step state on the handle's stream
static cudaError_t state_snapshot(const SimHandle* h, unsigned char* snap, bool save) {
  size_t off = 0;
  for (const auto& f : step_state(h)) {
    if (f.second == 0) continue;
    cudaError_t e = save ? cudaMemcpyAsync(snap + off, f.first, f.second, cudaMemcpyDeviceToDevice, h->stream)
                         : cudaMemcpyAsync(f.first, snap + off, f.second, cudaMemcpyDeviceToDevice, h->stream);
    if (e != cudaSuccess) return e;
    off += (f.second + 255) & ~(size_t)255;
  }
  return cudaSuccess;
}
static size_t state_snapshot_bytes(const SimHandle* h) {
  size_t b = 0;
  for (const auto& f : step_state(h)) b += (f.second + 255) & ~(size_t)255;
  return b;
}

// Every round: the state saved, then each trial from it (restored before all but the
// first), so the batch advances by steps_per_trial per round -- the last trial's steps.
static int time_trials(SimHandle* h, const std::vector<SimLaunchShape>& trials, int steps_per_trial, int rounds,
                       int& steps, std::vector<float>& med, unsigned char* snap, bool graph = false) {
  const int n = (int)trials.size();
  std::vector<std::vector<float>> ms(n * 5);
  for (int round = 0; round <= rounds; ++round) {
    cudaError_t se = state_snapshot(h, snap, true);
    if (se != cudaSuccess) return fail(SIM_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(se));
    for (int i = 0; i < n; ++i) {
      // forward on even rounds, backward on odd ones (the order only matters for the
      // caches each trial finds warm)
      const int t = round % 2 ? n - 1 - i : i;
      if (i > 0 && (se = state_snapshot(h, snap, false)) != cudaSuccess)
        return fail(SIM_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(se));
      apply_shape(h, trials[t]);
      if (graph) {  // captured for this shape and replayed, as sim_step runs it
        reset_graph(h);
        int r = sim_step(h, steps_per_trial);
        if (r) return r;
      } else {
        h->prof_n = steps_per_trial;
        h->launches += enqueue_steps(h, steps_per_trial, h->stream, false);
      }
      cudaError_t e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
      if (e != cudaSuccess) return fail(SIM_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(e));
      if (round == 0) continue;
      float st[SIM_N_STAGES];
      int r = sim_kernel_times(h, st, nullptr);
      if (r) return r;
      float tot = 0.f;
      for (int k = 0; k < SIM_N_STAGES; ++k) tot += st[k];
      ms[5 * t + 0].push_back(st[1] / steps_per_trial);
      ms[5 * t + 1].push_back(st[2] / steps_per_trial);
      ms[5 * t + 2].push_back((st[4] + st[5]) / steps_per_trial);  // PGS with its LPT ordering
      ms[5 * t + 3].push_back(tot / steps_per_trial);
      ms[5 * t + 4].push_back(st[0] / steps_per_trial);
    }
  }
  steps += (rounds + 1) * steps_per_trial;
  med.assign(n * 5, 0.f);
  for (int i = 0; i < n * 5; ++i) med[i] = median_of(ms[i]);
  return SIM_OK;
}

// Three phases on the live batch.  Phase 1 times every admissible launch option
// of each kernel (trial t runs option t mod #options of every kernel, so the
// kernels are tuned side by side) and keeps for each kernel the option with the
// lowest mean of its trials' median stage time.  Phase 2 times the PGS staging
// capacities (contacts and articulation row endpoints held in shared memory),
// with the 128- and (for 32 lanes) the 255-register build, under the phase-1
// shape.  Phase 3 re-times the best PGS grid options under that staging from
// CUDA graphs.  Each round's trials run from the same saved state (the scene's cost
// changes from step to step, most of all while objects fall and settle), forward
// and backward on alternate rounds.
int sim_autotune(SimHandle* h, int steps_per_trial, int rounds, SimLaunchShape* chosen, SimTuneReport* report) {
  if (!h) return fail(SIM_ERR_INVALID_ARG, "handle is NULL");
  ON_DEVICE(h);
  if (steps_per_trial < 1 || rounds < 1) return fail(SIM_ERR_INVALID_ARG, "steps_per_trial and rounds must be >= 1");
  if (h->d.warm_mode == 2 && !h->mlp_ready) return fail(SIM_ERR_STATE, "warm_mode 2 needs sim_set_mlp first");
  // phase-1 options.  PGS: 32 or 16 lanes per environment with the 128-register build
  // (the 8-lane and 85-register builds stay settable but are not searched); heavy SMs
  // with 32 lanes, persistent grids and LPT order.
  std::vector<SimLaunchShape> opt[4];  // collide, rows, pgs, aba
  const SimLaunchShape base = default_shape();
  for (int g = 32; g >= 16; g >>= 1) {
    SimLaunchShape k = base;
    k.aba_lanes = g;
    opt[3].push_back(k);
  }
  for (int w = 1; w <= gb::MAX_WARPS_PER_CTA; w <<= 1)
    for (int p = 0; p <= 1; ++p) {
      SimLaunchShape k = base;
      k.collide_warps = w; k.collide_persistent = p;
      if (shape_ok(h, 0, w, p)) opt[0].push_back(k);
      k = base;
      k.rows_warps = w; k.rows_persistent = p;
      if (shape_ok(h, 1, w, p)) opt[1].push_back(k);
      for (int g = 32; g >= 16; g >>= 1)
        for (int lpt = 0; lpt <= 1; ++lpt) {
          k = base;
          k.pgs_warps = w; k.pgs_persistent = p; k.pgs_lanes = g; k.pgs_lpt = lpt;
          if (pgs_occupancy(h, k) > 0) opt[2].push_back(k);
          if (g == 32 && p == 1 && lpt == 1)
            for (int div = 16; div >= 4; div >>= 1) {
              k.pgs_heavy_sms = h->sm_count / div;
              if (k.pgs_heavy_sms > 0 && pgs_occupancy(h, k) > 0) opt[2].push_back(k);
            }
        }
    }
  for (int k = 0; k < 4; ++k)
    if (opt[k].empty()) return fail(SIM_ERR_STATE, "no launch shape fits the device");
  const int n1 = (int)std::max(std::max(opt[0].size(), opt[1].size()), std::max(opt[2].size(), opt[3].size()));
  auto merge = [&](const SimLaunchShape& c, const SimLaunchShape& r, const SimLaunchShape& p,
                   const SimLaunchShape& ab) {
    SimLaunchShape k = p;
    k.collide_warps = c.collide_warps; k.collide_persistent = c.collide_persistent;
    k.rows_warps = r.rows_warps; k.rows_persistent = r.rows_persistent;
    k.aba_lanes = ab.aba_lanes;
    return k;
  };
  std::vector<SimLaunchShape> trials;
  for (int t = 0; t < n1; ++t)
    trials.push_back(merge(opt[0][t % opt[0].size()], opt[1][t % opt[1].size()], opt[2][t % opt[2].size()],
                           opt[3][t % opt[3].size()]));

  const SimLaunchShape old_shape = h->shape;
  const int old_prof = h->profiling, old_graph = h->p.use_graph;
  auto restore = [&](const SimLaunchShape& k) {
    apply_shape(h, k);
    h->profiling = old_prof;
    h->prof_n = 0;
    h->p.use_graph = old_graph;
    reset_graph(h);
  };
  reset_graph(h);
  h->profiling = 1;
  h->p.use_graph = 0;
  int r = ensure_events(h, steps_per_trial);
  if (r) { restore(old_shape); return r; }
  // the device copy of the step state each round's trials start from, freed on return
  struct SnapBuf {
    unsigned char* p = nullptr;
    ~SnapBuf() { if (p) cudaFree(p); }
  } snap;
  if (cudaMalloc(&snap.p, std::max<size_t>(state_snapshot_bytes(h), 256)) != cudaSuccess) {
    cudaGetLastError();
    restore(old_shape);
    return fail(SIM_ERR_CUDA, "autotune: state snapshot allocation");
  }
  int steps = 0;
  std::vector<float> med1, med2;
  if ((r = time_trials(h, trials, steps_per_trial, rounds, steps, med1, snap.p))) { restore(old_shape); return r; }
  int best[4];
  float best_ms[4];
  const int med_index[4] = {0, 1, 2, 4};  // per-trial medians: collide, rows, pgs, step, aba
  std::vector<float> pgs_score(opt[2].size());
  for (int k = 0; k < 4; ++k) {
    const int no = (int)opt[k].size();
    best[k] = 0;
    best_ms[k] = 3.4e38f;
    for (int o = 0; o < no; ++o) {
      float acc = 0.f;
      int cnt = 0;
      for (int t = o; t < n1; t += no) { acc += med1[5 * t + med_index[k]]; ++cnt; }
      float m = acc / (float)cnt;
      if (k == 2) pgs_score[o] = m;
      if (m < best_ms[k]) { best_ms[k] = m; best[k] = o; }
    }
  }
  SimLaunchShape b = merge(opt[0][best[0]], opt[1][best[1]], opt[2][best[2]], opt[3][best[3]]);

  // phase 2: PGS staging capacities under the phase-1 shape
  // (the phase-1 shape itself is a candidate: the scene moves on between the phases)
  int S0 = 0, AS0 = 0;
  gb::pgs_stage_defaults(h->d, h->max_obj, h->max_arts, &S0, &AS0);
  std::vector<SimLaunchShape> stage{b};
  for (int mb : {2, 1}) {
    if (mb == 1 && b.pgs_lanes != 32) continue;
    for (int sc : {S0 / 2, S0, S0 + S0 / 2})
      for (int ap : {8, 16, 32, 64}) {
        SimLaunchShape k = b;
        k.pgs_min_blocks = mb;
        k.pgs_stage_contacts = std::max(sc, 1);
        k.pgs_stage_pool = ap;
        if ((mb != b.pgs_min_blocks || sc != S0 || ap != AS0) && pgs_occupancy(h, k) > 0) stage.push_back(k);
      }
  }
  const int n2 = (int)stage.size();
  if ((r = time_trials(h, stage, steps_per_trial, rounds, steps, med2, snap.p))) { restore(old_shape); return r; }
  int bs = 0;
  for (int t = 1; t < n2; ++t)
    if (med2[5 * t + 2] < med2[5 * bs + 2]) bs = t;
  b = stage[bs];
  best_ms[2] = med2[5 * bs + 2];
  float best_step = med2[5 * bs + 3];

  // phase 3: play-off of the PGS grid options (warps, persistence, lanes, LPT, heavy
  // SMs) that phase 1 ranked best, each under the phase-2 staging, replayed from a
  // CUDA graph as sim_step runs them: a phase-1 margin smaller than the step-to-step
  // spread does not decide the kernel's shape
  std::vector<int> rank(opt[2].size());
  for (int o = 0; o < (int)rank.size(); ++o) rank[o] = o;
  std::stable_sort(rank.begin(), rank.end(), [&](int x, int y) { return pgs_score[x] < pgs_score[y]; });
  std::vector<SimLaunchShape> off{b};
  for (int q = 0; q < (int)rank.size() && (int)off.size() < 4; ++q) {
    const SimLaunchShape& o = opt[2][rank[q]];
    SimLaunchShape k = b;
    k.pgs_warps = o.pgs_warps; k.pgs_persistent = o.pgs_persistent; k.pgs_lanes = o.pgs_lanes;
    k.pgs_lpt = o.pgs_lpt; k.pgs_heavy_sms = o.pgs_heavy_sms;
    if (k.pgs_lanes != 32 && k.pgs_min_blocks == 1) k.pgs_min_blocks = 2;  // 255-register build: 32 lanes only
    bool dup = false;
    for (const SimLaunchShape& x : off) dup |= memcmp(&x, &k, sizeof(k)) == 0;
    if (!dup && pgs_occupancy(h, k) > 0) off.push_back(k);
  }
  const int n3 = (int)off.size();
  std::vector<float> med3;
  if (n1 + n2 + n3 > SIM_TUNE_MAX_TRIALS) { restore(old_shape); return fail(SIM_ERR_STATE, "too many candidate shapes"); }
  h->p.use_graph = 1;
  if ((r = time_trials(h, off, steps_per_trial, rounds, steps, med3, snap.p, true))) { restore(old_shape); return r; }
  int b3 = 0;
  for (int t = 1; t < n3; ++t)
    if (med3[5 * t + 2] < med3[5 * b3 + 2]) b3 = t;
  b = off[b3];
  best_ms[2] = med3[5 * b3 + 2];
  best_step = med3[5 * b3 + 3];

  // phase 4: environment partitions on parallel branches of the step's graph (1, 2 or
  // 4), one partition with the ABA kernels in sequence, and the fused step kernel,
  // under the phase-3 shape, the whole step timed: graph replay with no events
  // inside, CUDA events around the launch; each trial captures its graph in an untimed
  // replay first
  std::vector<SimLaunchShape> parts;
  for (int P : {1, 2, 4})
    if (P <= std::max(1, h->d.E)) {
      SimLaunchShape k = b;
      k.partitions = P;
      k.aba_overlap = 1;
      k.fused = 0;
      parts.push_back(k);
    }
  {  // and the ABA kernels in sequence with the collision kernel
    SimLaunchShape k = b;
    k.partitions = 1;
    k.aba_overlap = 0;
    k.fused = 0;
    parts.push_back(k);
  }
  if (h->d.warm_mode != 2) {  // and the fused step kernel, where it fits
    SimLaunchShape k = b;
    k.partitions = 1;
    k.fused = 1;
    if (gb::fused_warp_bytes(h->d, h->max_coll, h->max_obj, h->max_arts, k.pgs_stage_contacts, k.pgs_stage_pool) > 0)
      parts.push_back(k);
  }
  const int n4 = (int)parts.size();
  if (n1 + n2 + n3 + n4 > SIM_TUNE_MAX_TRIALS) { restore(old_shape); return fail(SIM_ERR_STATE, "too many candidate shapes"); }
  std::vector<float> med4(n4, 0.f);
  {
    h->profiling = 0;
    h->p.use_graph = 1;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    std::vector<std::vector<float>> ms4(n4);
    for (int round = 0; round <= rounds && r == 0; ++round) {
      cudaError_t se = state_snapshot(h, snap.p, true);  // the round's trials start from it
      if (se != cudaSuccess) r = fail(SIM_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(se));
      for (int i = 0; i < n4 && r == 0; ++i) {
        const int t = round % 2 ? n4 - 1 - i : i;  // alternating order, as in time_trials
        if (i > 0 && (se = state_snapshot(h, snap.p, false)) != cudaSuccess) {
          r = fail(SIM_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(se));
          break;
        }
        apply_shape(h, parts[t]);
        reset_graph(h);
        if ((r = sim_step(h, steps_per_trial))) break;
        cudaEventRecord(t0, h->stream);
        if ((r = sim_step(h, steps_per_trial))) break;
        cudaEventRecord(t1, h->stream);
        cudaError_t e = cudaEventSynchronize(t1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
        if (e != cudaSuccess) r = fail(SIM_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(e));
        if (round > 0) ms4[t].push_back(ms / steps_per_trial);
      }
      steps += 2 * steps_per_trial;  // the round's last trial: its untimed and timed steps
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (r) { restore(old_shape); return r; }
    for (int t = 0; t < n4; ++t) med4[t] = median_of(ms4[t]);
  }
  int b4 = 0;
  for (int t = 1; t < n4; ++t)
    if (med4[t] < med4[b4]) b4 = t;
  b = parts[b4];
  best_step = med4[b4];

  restore(b);
  if (chosen) *chosen = b;
  if (report) {
    memset(report, 0, sizeof(*report));
    const int nt = n1 + n2 + n3 + n4;
    report->n_trials = nt;
    report->steps_taken = steps;
    for (int t = 0; t < nt; ++t) {
      report->trial[t] = t < n1 ? trials[t]
                                : (t < n1 + n2 ? stage[t - n1] : (t < n1 + n2 + n3 ? off[t - n1 - n2] : parts[t - n1 - n2 - n3]));
      if (t >= n1 + n2 + n3) {  // phase 4: the whole step only
        report->ms[t][3] = med4[t - n1 - n2 - n3];
        continue;
      }
      const float* m = t < n1 ? &med1[5 * t] : (t < n1 + n2 ? &med2[5 * (t - n1)] : &med3[5 * (t - n1 - n2)]);
      for (int k = 0; k < 5; ++k) report->ms[t][k] = m[k];
    }
    for (int k = 0; k < 3; ++k) report->chosen_ms[k] = best_ms[k];
    report->chosen_ms[3] = best_step;
    report->chosen_ms[4] = best_ms[3];
  }
  return SIM_OK;
}

int sim_launch_count(SimHandle* h, long long* count) {
  if (!h || !count) return fail(SIM_ERR_INVALID_ARG, "NULL argument");
  ON_DEVICE(h);
  *count = h->launches;
  return SIM_OK;
}

int sim_sync(SimHandle* h, uint32_t* env_status_or, uint32_t* env_status) {
  if (!h) return fail(SIM_ERR_INVALID_ARG, "handle is NULL");
  ON_DEVICE(h);
  CK(cudaStreamSynchronize(h->stream));
  std::vector<int> st(h->d.E);
  if (h->d.E) CK(cudaMemcpy(st.data(), h->d.status, sizeof(int) * h->d.E, cudaMemcpyDeviceToHost));
  uint32_t acc = 0;
  for (int e = 0; e < h->d.E; ++e) {
    acc |= (uint32_t)st[e];
    if (env_status) env_status[e] = (uint32_t)st[e];
  }
  if (env_status_or) *env_status_or = acc;
  if (h->d.E) {
    CK(cudaMemsetAsync(h->d.status, 0, sizeof(int) * h->d.E, h->stream));
    CK(cudaStreamSynchronize(h->stream));
  }
  if (acc & SIM_ENV_NUMERIC) return fail(SIM_ERR_NUMERIC, "non-finite state in some environment");
  if (acc & SIM_ENV_OVERFLOW) return fail(SIM_ERR_OVERFLOW, "contact / pair / row capacity exceeded");
  if (acc & SIM_ENV_ITER_CAP) return fail(SIM_ERR_TIMEOUT, "PGS iteration cap reached before the residual target");
  if (acc & SIM_ENV_DEVICE_WAIT) return fail(SIM_ERR_TIMEOUT, "a bounded device wait ran out (SIM_ENV_DEVICE_WAIT)");
  return SIM_OK;
}

}  // extern "C"

// copy n items of a float4 field into caller buffer dst[n*w]
static int get_f4(SimHandle* h, const float4* src, float* dst, long n, int w, int to_device) {
  if (!dst || n == 0) return SIM_OK;
  float* tgt = dst;
  if (!to_device) {
    int r = ensure_stage(h, (size_t)n * w);
    if (r) return r;
    tgt = h->stage;
  }
  k_pack<<<nblk(n, 256), 256, 0, h->stream>>>(src, tgt, n, w);
  CK(cudaGetLastError());
  if (!to_device) CK(cudaMemcpyAsync(dst, h->stage, sizeof(float) * n * w, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return SIM_OK;
}
static int set_f4(SimHandle* h, float4* dst, const float* src, long n, int w, int from_device) {
  if (!src || n == 0) return SIM_OK;
  const float* s = src;
  if (!from_device) {
    int r = ensure_stage(h, (size_t)n * w);
    if (r) return r;
    CK(cudaMemcpyAsync(h->stage, src, sizeof(float) * n * w, cudaMemcpyHostToDevice, h->stream));
    s = h->stage;
  }
  k_unpack<<<nblk(n, 256), 256, 0, h->stream>>>(s, dst, n, w);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(h->stream));
  return SIM_OK;
}
template <typename T>
static int get_plain(SimHandle* h, const T* src, T* dst, long n, int to_device) {
  if (!dst || n == 0) return SIM_OK;
  CK(cudaMemcpyAsync(dst, src, sizeof(T) * n, to_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return SIM_OK;
}
template <typename T>
static int set_plain(SimHandle* h, T* dst, const T* src, long n, int from_device) {
  if (!src || n == 0) return SIM_OK;
  CK(cudaMemcpyAsync(dst, src, sizeof(T) * n, from_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return SIM_OK;
}
static int get_i4(SimHandle* h, const int4* src, int* dst, long n, int to_device) {
  if (!dst || n == 0) return SIM_OK;
  int* tgt = dst;
  if (!to_device) {
    int r = ensure_stage(h, (size_t)n * 3);
    if (r) return r;
    tgt = reinterpret_cast<int*>(h->stage);
  }
  k_pack_i4<<<nblk(n, 256), 256, 0, h->stream>>>(src, tgt, n);
  CK(cudaGetLastError());
  if (!to_device) CK(cudaMemcpyAsync(dst, h->stage, sizeof(int) * n * 3, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return SIM_OK;
}
static int set_i4(SimHandle* h, int4* dst, const int* src, long n, int from_device) {
  if (!src || n == 0) return SIM_OK;
  const int* s = src;
  if (!from_device) {
    int r = ensure_stage(h, (size_t)n * 3);
    if (r) return r;
    CK(cudaMemcpyAsync(h->stage, src, sizeof(int) * n * 3, cudaMemcpyHostToDevice, h->stream));
    s = reinterpret_cast<const int*>(h->stage);
  }
  k_unpack_i4<<<nblk(n, 256), 256, 0, h->stream>>>(s, dst, n);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(h->stream));
  return SIM_OK;
}

extern "C" {

int sim_get_state(SimHandle* h, const SimStateView* o, int to_device) {
  if (!h || !o) return fail(SIM_ERR_INVALID_ARG, "NULL argument");
  ON_DEVICE(h);
  const Dev& d = h->d;
  long EC = (long)d.E * d.C;
  int r;
  if ((r = get_f4(h, d.obj_pos, o->obj_pos, d.NO, 3, to_device))) return r;
  if ((r = get_f4(h, d.obj_comp, o->obj_pos_comp, d.NO, 3, to_device))) return r;
  if ((r = get_f4(h, d.obj_quat, o->obj_quat, d.NO, 4, to_device))) return r;
  if ((r = get_f4(h, d.obj_vel, o->obj_vel, d.NO, 3, to_device))) return r;
  if ((r = get_f4(h, d.obj_omega, o->obj_omega, d.NO, 3, to_device))) return r;
  if ((r = get_plain(h, d.obj_awake, o->obj_awake, d.NO, to_device))) return r;
  if ((r = get_plain(h, d.obj_ctr, o->obj_ctr, d.NO, to_device))) return r;
  if ((r = get_plain(h, d.j_q, o->joint_q, d.NJ, to_device))) return r;
  if ((r = get_plain(h, d.j_qcomp, o->joint_q_comp, d.NJ, to_device))) return r;
  if ((r = get_plain(h, d.j_qd, o->joint_qd, d.NJ, to_device))) return r;
  if ((r = get_plain(h, d.j_target, o->joint_target, d.NJ, to_device))) return r;
  if ((r = get_f4(h, d.art_base_pos, o->art_base_pos, d.NA, 3, to_device))) return r;
  if ((r = get_f4(h, d.art_base_quat, o->art_base_quat, d.NA, 4, to_device))) return r;
  if ((r = get_plain(h, d.j_lim_lambda, o->joint_lim_lambda, d.NJ, to_device))) return r;
  if ((r = get_plain(h, d.j_motor_lambda, o->joint_motor_lambda, d.NJ, to_device))) return r;
  if ((r = get_plain(h, d.j_lim_side, o->joint_lim_side, d.NJ, to_device))) return r;
  if ((r = get_plain(h, d.cache_count, o->cache_count, d.E, to_device))) return r;
  if ((r = get_i4(h, d.cache_key, o->cache_key, EC, to_device))) return r;
  if ((r = get_f4(h, d.cache_p, o->cache_p, EC, 3, to_device))) return r;
  if ((r = get_f4(h, d.cache_lam, o->cache_lambda, EC, 4, to_device))) return r;
  return SIM_OK;
}

int sim_set_state(SimHandle* h, const SimStateView* in, int from_device) {
  if (!h || !in) return fail(SIM_ERR_INVALID_ARG, "NULL argument");
  ON_DEVICE(h);
  Dev& d = h->d;
  long EC = (long)d.E * d.C;
  int r;
  if ((r = set_f4(h, d.obj_pos, in->obj_pos, d.NO, 3, from_device))) return r;
  if ((r = set_f4(h, d.obj_comp, in->obj_pos_comp, d.NO, 3, from_device))) return r;
  if ((r = set_f4(h, d.obj_quat, in->obj_quat, d.NO, 4, from_device))) return r;
  if ((r = set_f4(h, d.obj_vel, in->obj_vel, d.NO, 3, from_device))) return r;
  if ((r = set_f4(h, d.obj_omega, in->obj_omega, d.NO, 3, from_device))) return r;
  if ((r = set_plain(h, d.obj_awake, in->obj_awake, d.NO, from_device))) return r;
  if ((r = set_plain(h, d.obj_ctr, in->obj_ctr, d.NO, from_device))) return r;
  if ((r = set_plain(h, d.j_q, in->joint_q, d.NJ, from_device))) return r;
  if ((r = set_plain(h, d.j_qcomp, in->joint_q_comp, d.NJ, from_device))) return r;
  if ((r = set_plain(h, d.j_qd, in->joint_qd, d.NJ, from_device))) return r;
  if ((r = set_plain(h, d.j_target, in->joint_target, d.NJ, from_device))) return r;
  if ((r = set_f4(h, d.art_base_pos, in->art_base_pos, d.NA, 3, from_device))) return r;
  if ((r = set_f4(h, d.art_base_quat, in->art_base_quat, d.NA, 4, from_device))) return r;
  if ((r = set_plain(h, d.j_lim_lambda, in->joint_lim_lambda, d.NJ, from_device))) return r;
  if ((r = set_plain(h, d.j_motor_lambda, in->joint_motor_lambda, d.NJ, from_device))) return r;
  if ((r = set_plain(h, d.j_lim_side, in->joint_lim_side, d.NJ, from_device))) return r;
  if ((r = set_plain(h, d.cache_count, in->cache_count, d.E, from_device))) return r;
  if ((r = set_i4(h, d.cache_key, in->cache_key, EC, from_device))) return r;
  if ((r = set_f4(h, d.cache_p, in->cache_p, EC, 3, from_device))) return r;
  if ((r = set_f4(h, d.cache_lam, in->cache_lambda, EC, 4, from_device))) return r;
  return SIM_OK;
}

int sim_get_env_stats(SimHandle* h, int* status, int* iters, float* resid, int* n_contacts, int* n_rows,
                      int* n_limit_rows, int* n_colours, int* fp64_used, int to_device) {
  if (!h) return fail(SIM_ERR_INVALID_ARG, "handle is NULL");
  ON_DEVICE(h);
  const Dev& d = h->d;
  int r;
  if ((r = get_plain(h, d.status, status, d.E, to_device))) return r;
  if ((r = get_plain(h, d.iters, iters, d.E, to_device))) return r;
  if ((r = get_plain(h, d.resid, resid, d.E, to_device))) return r;
  if ((r = get_plain(h, d.n_contacts, n_contacts, d.E, to_device))) return r;
  if ((r = get_plain(h, d.n_rows, n_rows, d.E, to_device))) return r;
  if ((r = get_plain(h, d.n_limit, n_limit_rows, d.E, to_device))) return r;
  if ((r = get_plain(h, d.n_colours, n_colours, d.E, to_device))) return r;
  if ((r = get_plain(h, d.fp64_used, fp64_used, d.E, to_device))) return r;
  return SIM_OK;
}

int sim_get_robot_force(SimHandle* h, float* step_force, float* accumulated, int to_device) {
  if (!h) return fail(SIM_ERR_INVALID_ARG, "handle is NULL");
  ON_DEVICE(h);
  int r;
  if ((r = get_plain(h, h->d.robot_force, step_force, h->d.E, to_device))) return r;
  if ((r = get_plain(h, h->d.robot_force_acc, accumulated, h->d.E, to_device))) return r;
  return SIM_OK;
}

__global__ void k_zero_listed(float* a, const int* ids, int n, int E, int* bad) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int e = ids[i];
  if (e < 0 || e >= E) { atomicOr(bad, 1); return; }
  a[e] = 0.f;
}

int sim_reset_robot_force(SimHandle* h, const int* env_ids, int n, int on_device) {
  if (!h) return fail(SIM_ERR_INVALID_ARG, "handle is NULL");
  ON_DEVICE(h);
  const Dev& d = h->d;
  if (!env_ids) {
    if (d.E) CK(cudaMemsetAsync(d.robot_force_acc, 0, sizeof(float) * d.E, h->stream));
    return SIM_OK;
  }
  if (n < 0) return fail(SIM_ERR_INVALID_ARG, "n < 0");
  if (n == 0) return SIM_OK;
  int r = ensure_stage(h, (size_t)n + 1);
  if (r) return r;
  int* ids = reinterpret_cast<int*>(h->stage);
  int* bad = ids + n;
  if (!on_device) {
    for (int k = 0; k < n; ++k)
      if (env_ids[k] < 0 || env_ids[k] >= d.E) return fail(SIM_ERR_INVALID_ARG, "environment index out of range");
    CK(cudaMemcpyAsync(ids, env_ids, sizeof(int) * n, cudaMemcpyHostToDevice, h->stream));
  } else {
    CK(cudaMemcpyAsync(ids, env_ids, sizeof(int) * n, cudaMemcpyDeviceToDevice, h->stream));
  }
  CK(cudaMemsetAsync(bad, 0, sizeof(int), h->stream));
  k_zero_listed<<<(n + 255) / 256, 256, 0, h->stream>>>(d.robot_force_acc, ids, n, d.E, bad);
  CK(cudaGetLastError());
  int hb = 0;
  CK(cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (hb) return fail(SIM_ERR_INVALID_ARG, "environment index out of range (entries outside [0, E) skipped)");
  return SIM_OK;
}

// one block per listed environment: its objects, joints and articulation bases
// from the template; no prior-frame contacts; robot force and limit state cleared
__global__ void k_reset_envs(Dev d, float4* t_pos, float4* t_comp, float4* t_quat, float4* t_vel, float4* t_omega,
                             int* t_awake, int* t_ctr, float* t_q, float* t_qcomp, float* t_qd, float* t_target,
                             float* t_llam, int* t_lside, float* t_mlam, float4* t_bpos, float4* t_bquat,
                             const int* ids, int n) {
  if (blockIdx.x >= (unsigned)n) return;
  const int e = ids[blockIdx.x];
  if (e < 0 || e >= d.E) return;
  for (int i = d.obj_off[e] + threadIdx.x; i < d.obj_off[e + 1]; i += blockDim.x) {
    d.obj_pos[i] = t_pos[i]; d.obj_comp[i] = t_comp[i]; d.obj_quat[i] = t_quat[i];
    d.obj_vel[i] = t_vel[i]; d.obj_omega[i] = t_omega[i]; d.obj_awake[i] = t_awake[i]; d.obj_ctr[i] = t_ctr[i];
  }
  const int a0 = d.art_off[e], a1 = d.art_off[e + 1];
  for (int j = d.joint_off[a0] + threadIdx.x; j < d.joint_off[a1]; j += blockDim.x) {
    d.j_q[j] = t_q[j]; d.j_qcomp[j] = t_qcomp[j]; d.j_qd[j] = t_qd[j]; d.j_target[j] = t_target[j];
    d.j_lim_lambda[j] = t_llam[j]; d.j_lim_side[j] = t_lside[j]; d.j_motor_lambda[j] = t_mlam[j];
  }
  for (int a = a0 + threadIdx.x; a < a1; a += blockDim.x) {
    d.art_base_pos[a] = t_bpos[a];
    d.art_base_quat[a] = t_bquat[a];
  }
  if (threadIdx.x == 0) {
    d.cache_count[e] = 0;
    d.robot_force[e] = 0.f;
    d.robot_force_acc[e] = 0.f;
  }
}

int sim_reset_envs(SimHandle* h, const int* env_ids, int n, int on_device) {
  if (!h) return fail(SIM_ERR_INVALID_ARG, "handle is NULL");
  ON_DEVICE(h);
  if (n < 0 || (n > 0 && !env_ids)) return fail(SIM_ERR_INVALID_ARG, "bad environment list");
  if (n == 0) return SIM_OK;
  const Dev& d = h->d;
  const int* ids = env_ids;
  if (!on_device) {
    for (int k = 0; k < n; ++k)
      if (env_ids[k] < 0 || env_ids[k] >= d.E) return fail(SIM_ERR_INVALID_ARG, "environment index out of range");
    int r = ensure_stage(h, (size_t)n);
    if (r) return r;
    CK(cudaMemcpyAsync(h->stage, env_ids, sizeof(int) * n, cudaMemcpyHostToDevice, h->stream));
    ids = reinterpret_cast<const int*>(h->stage);
  }
  auto& t = h->tmpl;
  k_reset_envs<<<n, 128, 0, h->stream>>>(d, t.obj_pos, t.obj_comp, t.obj_quat, t.obj_vel, t.obj_omega, t.obj_awake,
                                         t.obj_ctr, t.j_q, t.j_qcomp, t.j_qd, t.j_target, t.j_lim_lambda,
                                         t.j_lim_side, t.j_motor_lambda, t.base_pos, t.base_quat, ids, n);
  CK(cudaGetLastError());
  if (!on_device) CK(cudaStreamSynchronize(h->stream));  // the staging buffer may be reused
  return SIM_OK;
}

int sim_set_reset_state(SimHandle* h, const SimStateView* in, int from_device) {
  if (!h || !in) return fail(SIM_ERR_INVALID_ARG, "NULL argument");
  ON_DEVICE(h);
  const Dev& d = h->d;
  auto& t = h->tmpl;
  int r;
  if ((r = set_f4(h, t.obj_pos, in->obj_pos, d.NO, 3, from_device))) return r;
  if ((r = set_f4(h, t.obj_comp, in->obj_pos_comp, d.NO, 3, from_device))) return r;
  if ((r = set_f4(h, t.obj_quat, in->obj_quat, d.NO, 4, from_device))) return r;
  if ((r = set_f4(h, t.obj_vel, in->obj_vel, d.NO, 3, from_device))) return r;
  if ((r = set_f4(h, t.obj_omega, in->obj_omega, d.NO, 3, from_device))) return r;
  if ((r = set_plain(h, t.obj_awake, in->obj_awake, d.NO, from_device))) return r;
  if ((r = set_plain(h, t.obj_ctr, in->obj_ctr, d.NO, from_device))) return r;
  if ((r = set_plain(h, t.j_q, in->joint_q, d.NJ, from_device))) return r;
  if ((r = set_plain(h, t.j_qcomp, in->joint_q_comp, d.NJ, from_device))) return r;
  if ((r = set_plain(h, t.j_qd, in->joint_qd, d.NJ, from_device))) return r;
  if ((r = set_plain(h, t.j_target, in->joint_target, d.NJ, from_device))) return r;
  if ((r = set_plain(h, t.j_lim_lambda, in->joint_lim_lambda, d.NJ, from_device))) return r;
  if ((r = set_plain(h, t.j_motor_lambda, in->joint_motor_lambda, d.NJ, from_device))) return r;
  if ((r = set_plain(h, t.j_lim_side, in->joint_lim_side, d.NJ, from_device))) return r;
  if ((r = set_f4(h, t.base_pos, in->art_base_pos, d.NA, 3, from_device))) return r;
  if ((r = set_f4(h, t.base_quat, in->art_base_quat, d.NA, 4, from_device))) return r;
  return SIM_OK;
}

int sim_get_contacts(SimHandle* h, int* count, int* key, float* point, float* normal, float* sep, float* lam,
                     int to_device) {
  if (!h) return fail(SIM_ERR_INVALID_ARG, "handle is NULL");
  ON_DEVICE(h);
  const Dev& d = h->d;
  long EC = (long)d.E * d.C;
  int r;
  if ((r = get_plain(h, d.n_contacts, count, d.E, to_device))) return r;
  if ((r = get_i4(h, d.c_key, key, EC, to_device))) return r;
  if ((r = get_f4(h, d.c_p, point, EC, 3, to_device))) return r;
  if ((r = get_f4(h, d.c_n, normal, EC, 3, to_device))) return r;
  if (sep && EC) {
    float* tgt = sep;
    if (!to_device) {
      if ((r = ensure_stage(h, EC))) return r;
      tgt = h->stage;
    }
    k_pack_w<<<nblk(EC, 256), 256, 0, h->stream>>>(d.c_p, tgt, EC);
    CK(cudaGetLastError());
    if (!to_device) CK(cudaMemcpyAsync(sep, h->stage, sizeof(float) * EC, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
  }
  if ((r = get_f4(h, d.c_lam, lam, EC, 3, to_device))) return r;
  return SIM_OK;
}

int sim_get_pairs(SimHandle* h, int pair_cap, int* count, int* pairs, int to_device) {
  if (!h) return fail(SIM_ERR_INVALID_ARG, "handle is NULL");
  ON_DEVICE(h);
  if (pair_cap < 0 || pair_cap > gb::PAIR_CAP) return fail(SIM_ERR_INVALID_ARG, "pair_cap out of range");
  const Dev& d = h->d;
  int r;
  if ((r = get_plain(h, d.pair_count, count, d.E, to_device))) return r;
  long n = (long)d.E * pair_cap;
  if (pairs && n) {
    int* tgt = pairs;
    if (!to_device) {
      if ((r = ensure_stage(h, n))) return r;
      tgt = reinterpret_cast<int*>(h->stage);
    }
    k_pairs_out<<<nblk(n, 256), 256, 0, h->stream>>>(d.pairs, pair_cap, tgt, d.E);
    CK(cudaGetLastError());
    if (!to_device) CK(cudaMemcpyAsync(pairs, h->stage, sizeof(int) * n, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
  }
  return SIM_OK;
}

int sim_get_articulation(SimHandle* h, float* com, float* rot, float* qdd, float* minv, int to_device) {
  if (!h) return fail(SIM_ERR_INVALID_ARG, "handle is NULL");
  ON_DEVICE(h);
  const Dev& d = h->d;
  int r;
  if ((r = get_f4(h, d.l_com, com, d.NJ, 3, to_device))) return r;
  if (rot && d.NJ) {
    float* tgt = rot;
    if (!to_device) {
      if ((r = ensure_stage(h, (size_t)d.NJ * 9))) return r;
      tgt = h->stage;
    }
    k_pack_rot<<<nblk(d.NJ, 256), 256, 0, h->stream>>>(d.l_r0, d.l_r1, d.l_r2, tgt, d.NJ);
    CK(cudaGetLastError());
    if (!to_device) CK(cudaMemcpyAsync(rot, h->stage, sizeof(float) * 9 * d.NJ, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
  }
  if ((r = get_plain(h, d.j_qdd, qdd, d.NJ, to_device))) return r;
  if ((r = get_plain(h, d.a_minv, minv, (long)d.NA * 81, to_device))) return r;
  return SIM_OK;
}

int sim_set_mlp(SimHandle* h, const float* params, int on_device) {
  if (!h) return fail(SIM_ERR_INVALID_ARG, "handle is NULL");
  ON_DEVICE(h);
  if (h->mlp) { cudaStreamSynchronize(h->stream); gb::mlp_destroy(h->mlp); h->mlp = nullptr; }
  h->mlp_ready = 0;
  reset_graph(h);
  if (!params) return SIM_OK;
  std::string err;
  h->mlp = gb::mlp_create(params, on_device, h->stream, err);
  if (!h->mlp) return fail(SIM_ERR_CUDA, "sim_set_mlp: " + err);
  h->mlp_ready = 1;
  return SIM_OK;
}


int sim_debug_hold_async(SimHandle* h, int on) {
  if (!h) return fail(SIM_ERR_INVALID_ARG, "handle is NULL");
  ON_DEVICE(h);
  if (on != 0 && on != 1) return fail(SIM_ERR_INVALID_ARG, "on must be 0 or 1");
  h->d.hold_async = on;
  reset_graph(h);  // the kernels take the device view by value at capture
  return SIM_OK;
}

int sim_log_predictions(SimHandle* h, float* preds, int cap, int* n_out) {
  if (!h || !n_out) return fail(SIM_ERR_INVALID_ARG, "NULL argument");
  ON_DEVICE(h);
  if (!h->d.pred || !h->d.feat || h->d.warm_mode != 2) return fail(SIM_ERR_STATE, "warm_mode 2 is not set");
  if (cap < 0 || (cap > 0 && !preds)) return fail(SIM_ERR_INVALID_ARG, "bad output buffer");
  const Dev& d = h->d;
  int r;
  if ((r = ensure_stage(h, (size_t)d.E + 1))) return r;
  int* prefix = reinterpret_cast<int*>(h->stage);
  if ((r = gb::enqueue_contact_log(d, h->stream, prefix, preds, nullptr, cap, true))) return r;
  CK(cudaMemcpyAsync(n_out, prefix + d.E, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return SIM_OK;
}

int sim_log_contacts(SimHandle* h, float* feats, float* lams, int cap, int* n_out) {
  if (!h || !n_out) return fail(SIM_ERR_INVALID_ARG, "NULL argument");
  ON_DEVICE(h);
  if (!h->d.feat) return fail(SIM_ERR_STATE, "log_features was not enabled");
  if (cap < 0 || (cap > 0 && (!feats || !lams))) return fail(SIM_ERR_INVALID_ARG, "bad output buffers");
  const Dev& d = h->d;
  int r;
  if ((r = ensure_stage(h, (size_t)d.E + 1))) return r;
  int* prefix = reinterpret_cast<int*>(h->stage);
  if ((r = gb::enqueue_contact_log(d, h->stream, prefix, feats, lams, cap, false))) return r;
  CK(cudaMemcpyAsync(n_out, prefix + d.E, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return SIM_OK;
}


// Batch totals of the last step (sim_get_stats): 64-bit sums and maxima over the
// environments and objects, accumulated with one atomic per warp into acc (zeroed by
// the caller): [0] sweeps, [1] rows x sweeps, [2] contacts, [3] rows, [4] limit rows,
// [5] articulation row endpoints, [6] awake objects, [7] envs with the sweep cap,
// [8] envs with the FP64 inverse; mx: [0] max sweeps, [1] max colours, [2] max residual
// (float bits; non-negative), [3] OR of the status bits.
__global__ void k_batch_stats(Dev d, unsigned long long* acc, unsigned* mx) {
  unsigned long long a[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  unsigned m_it = 0, m_col = 0, m_res = 0, st_or = 0;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
  for (int e = tid; e < d.E; e += nth) {
    const int it = d.iters[e], nr = d.n_rows[e], stt = d.status[e];
    a[0] += (unsigned long long)it;
    a[1] += (unsigned long long)it * (unsigned long long)nr;
    a[2] += (unsigned long long)d.n_contacts[e];
    a[3] += (unsigned long long)nr;
    a[4] += (unsigned long long)d.n_limit[e];
    a[5] += (unsigned long long)d.ap_count[e];
    a[7] += (stt & gb::ST_ITER_CAP) ? 1ull : 0ull;
    a[8] += d.fp64_used[e] ? 1ull : 0ull;
    m_it = max(m_it, (unsigned)it);
    m_col = max(m_col, (unsigned)d.n_colours[e]);
    const float rs = d.resid[e];
    if (rs > 0.f) m_res = max(m_res, __float_as_uint(isfinite(rs) ? rs : 3.4e38f));
    st_or |= (unsigned)stt;
  }
  for (int i = tid; i < d.NO; i += nth) a[6] += d.obj_awake[i] ? 1ull : 0ull;
  for (int o = 16; o > 0; o >>= 1) {
    for (int k = 0; k < 9; ++k) a[k] += __shfl_down_sync(0xffffffffu, a[k], o);
    m_it = max(m_it, __shfl_down_sync(0xffffffffu, m_it, o));
    m_col = max(m_col, __shfl_down_sync(0xffffffffu, m_col, o));
    m_res = max(m_res, __shfl_down_sync(0xffffffffu, m_res, o));
    st_or |= __shfl_down_sync(0xffffffffu, st_or, o);
  }
  if ((threadIdx.x & 31) == 0) {
    for (int k = 0; k < 9; ++k)
      if (a[k]) atomicAdd(acc + k, a[k]);
    atomicMax(mx, m_it);
    atomicMax(mx + 1, m_col);
    atomicMax(mx + 2, m_res);
    atomicOr(mx + 3, st_or);
  }
}

int sim_get_stats(SimHandle* h, SimStats* out) {
  if (!h || !out) return fail(SIM_ERR_INVALID_ARG, "NULL argument");
  ON_DEVICE(h);
  const Dev& d = h->d;
  int r;
  // 9 x 8-byte sums then 4 x 4-byte maxima in the staging buffer (floats)
  if ((r = ensure_stage(h, 18 + 4))) return r;
  unsigned long long* acc = reinterpret_cast<unsigned long long*>(h->stage);
  unsigned* mx = reinterpret_cast<unsigned*>(h->stage + 18);
  CK(cudaMemsetAsync(h->stage, 0, sizeof(float) * 22, h->stream));
  const long items = std::max<long>(d.E, d.NO);
  if (items > 0) {
    const unsigned blocks = std::min<unsigned>(nblk(items, 256), 4u * (unsigned)std::max(1, h->sm_count));
    k_batch_stats<<<blocks, 256, 0, h->stream>>>(d, acc, mx);
  }
  CK(cudaGetLastError());
  unsigned long long a[9];
  unsigned m[4];
  CK(cudaMemcpyAsync(a, acc, sizeof(a), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(m, mx, sizeof(m), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  SimStats o;
  std::memset(&o, 0, sizeof(o));
  o.n_envs = d.E;
  o.max_iters = (int32_t)m[0];
  o.sum_iters = (int64_t)a[0];
  o.row_sweeps = (int64_t)a[1];
  o.n_contacts = (int64_t)a[2];
  o.n_rows = (int64_t)a[3];
  o.n_limit_rows = (int64_t)a[4];
  o.n_pool_slots = (int64_t)a[5];
  o.n_awake = (int64_t)a[6];
  o.n_iter_cap = (int32_t)a[7];
  o.n_fp64 = (int32_t)a[8];
  o.max_colours = (int32_t)m[1];
  o.status_or = m[3];
  float fr;
  std::memcpy(&fr, &m[2], sizeof(fr));
  o.max_resid = fr;
  if (d.warm_mode == 2 && d.mlp_count) {  // each partition of the last step counted its own rows
    int cnt[SIM_MAX_PARTITIONS] = {0, 0, 0, 0};
    const int P = std::max(1, std::min(h->last_parts, SIM_MAX_PARTITIONS));
    CK(cudaMemcpy(cnt, d.mlp_count, sizeof(int) * P, cudaMemcpyDeviceToHost));
    for (int p = 0; p < P; ++p) o.n_net_rows += cnt[p];
  }
  *out = o;
  return SIM_OK;
}

int sim_set_warm_start(SimHandle* h, int mode, const float* mlp_params, int on_device) {
  if (!h) return fail(SIM_ERR_INVALID_ARG, "handle is NULL");
  ON_DEVICE(h);
  if (mode < 0 || mode > 2) return fail(SIM_ERR_INVALID_ARG, "warm-start mode must be 0, 1 or 2");
  if (mode == 2 && !mlp_params && !h->mlp_ready)
    return fail(SIM_ERR_STATE, "learned warm start without a network (pass its parameters)");
  SimParams p = h->p;
  p.warm_mode = mode;
  int r = sim_set_params(h, &p);
  if (r) return r;
  if (mlp_params) return sim_set_mlp(h, mlp_params, on_device);
  return SIM_OK;
}

}  // extern "C"
