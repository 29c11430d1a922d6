/*
 * sim.h - C ABI of the GB300 batched rigid/articulated physics step.
 *
 * One physics step advances thousands of independent home-rearrangement
 * environments: the simulator transition T:(s_t, a_t) -> s_{t+1} of the paper
 * (Sec. 2, "What is a simulator?"; the agent's action a_t is a set of joint
 * PD-motor targets, Sec. 5.1 "Action space"), restricted to the physics the
 * paper localises (Sec. 4.1 "Localized Physics": kinematic robot base, object
 * sleeping, static receptacle parts).  Per environment and step:
 *   articulations: forward kinematics, Featherstone ABA with a stable PD motor
 *     folded in as joint armature, CRBA mass matrix and its inverse;
 *   free bodies: gravity;  collision: AABB broadphase, wake pass, sphere / box
 *     / plane narrowphase;  projected Gauss-Seidel on contact (normal + two
 *     friction rows) and joint-limit rows;  semi-implicit Euler + sleeping.
 *
 * Conventions for every call:
 *   - Every function returns a SimStatus; none throws, none aborts.  After a
 *     failure sim_last_error(h) describes it: the last error of a call on the
 *     handle h (valid until the handle's next failing call), or with h = NULL
 *     the last error of any call on this thread (sim_create before a handle
 *     exists, the trainer, calls given a NULL handle).
 *   - All pointers passed in are owned by the caller and only read (or written
 *     for outputs) during the call; the library copies what it keeps.  With
 *     on_device = 0 they are host pointers, with on_device = 1 device pointers
 *     of the current device.  Nothing returned needs freeing except the handle
 *     (sim_destroy).
 *   - All work is enqueued on the CUDA stream given to sim_create; calls that
 *     return data to the host synchronise that stream first.
 *   - A handle is single-threaded: one host thread at a time.
 *   - Units SI, z up, angles in radians, quaternions (w, x, y, z).
 *   - Per-environment error bits (SIM_ENV_*) are accumulated on the device and
 *     never trap; sim_sync reports them.
 */
#ifndef PAPER_2106_14405_GB300_SIM_H
#define PAPER_2106_14405_GB300_SIM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct SimHandle SimHandle;

typedef enum {
  SIM_OK = 0,
  SIM_ERR_INVALID_ARG = 1, /* malformed description, out-of-range size, NULL where required */
  SIM_ERR_CUDA = 2,        /* a CUDA runtime call failed (message in sim_last_error) */
  SIM_ERR_OOM = 3,         /* device allocation failed */
  SIM_ERR_NUMERIC = 4,     /* some environment produced a non-finite state */
  SIM_ERR_OVERFLOW = 5,    /* some environment exceeded a contact / pair / row capacity */
  SIM_ERR_TIMEOUT = 6,     /* PGS iteration cap in residual mode, or a bounded device wait ran out */
  SIM_ERR_STATE = 7        /* call not valid in the handle's current state */
} SimStatus;

/* Per-environment status bits (sim_sync, sim_get_env_stats). */
#define SIM_ENV_OVERFLOW 1u
#define SIM_ENV_NUMERIC 2u
#define SIM_ENV_ITER_CAP 4u
#define SIM_ENV_FORCE_LIMIT 8u  /* accumulated robot contact force above params.force_limit (a task signal, not an engine error) */
#define SIM_ENV_DEVICE_WAIT 16u /* a bounded device wait (tensor-core completion of the learned warm start) gave up; the env kept its previous prediction */

/* Capacities (validated by sim_create). */
#define SIM_MAX_DOF 9          /* joints per articulation */
#define SIM_MAX_OBJECTS 64     /* free objects per environment */
#define SIM_MAX_COLLIDERS 128  /* objects + links + robot bases + statics + plane per environment */
#define SIM_MAX_ARTS 8         /* articulations per environment */
#define SIM_MAX_CONTACTS 256   /* upper bound of SimParams.max_contacts */

/*
 * Batch description: flat arrays with CSR offsets (host pointers, read once by
 * sim_create).  Floats are double here and converted to float32 on upload.
 *   obj_off[E+1]          objects of env e are [obj_off[e], obj_off[e+1])
 *   obj_shape[NO]         0 sphere, 1 box
 *   obj_half[NO*3]        box half extents; sphere radius in [0]
 *   obj_mass, obj_mu, obj_rest [NO]   mass (kg), friction, restitution
 *   obj_pos[NO*3], obj_quat[NO*4], obj_vel[NO*3], obj_omega[NO*3]  initial state
 *   stat_off[E+1], stat_pos[NS*3], stat_quat[NS*4], stat_half[NS*3], stat_mu[NS]
 *                          static boxes (cabinet walls, furniture; Sec. 4.1 item 4)
 *   art_off[E+1]          articulations of env e; joint_off[NA+1] joints of art a
 *   art_base_pos[NA*3], art_base_quat[NA*4]   base pose (kinematic: moved only
 *                          by sim_set_base_pose, Sec. 4.1 item 2)
 *   art_has_base_coll[NA], art_base_coll_off[NA*3], art_base_coll_half[NA*3]
 *                          optional base box collider (offset in the base frame)
 *   art_kinematic[NA]     1 for the robot (the articulation sim_set_base_pose moves)
 *   joint_parent[NJ]      parent joint within the articulation (-1 = base);
 *                          must be smaller than the joint's own index
 *   joint_type[NJ]        0 revolute, 1 prismatic
 *   joint_axis[NJ*3]      unit axis in the joint frame
 *   joint_origin_pos[NJ*3], joint_origin_quat[NJ*4]  joint frame in the parent link frame
 *   joint_com[NJ*3]       link centre of mass in the link frame (the link's box
 *                          collider is centred there, axes of the link frame)
 *   joint_half[NJ*3], joint_mass[NJ]   link box (inertia of a solid box)
 *   joint_lo, joint_hi[NJ], joint_has_limit[NJ]  joint limits
 *   joint_kp, joint_kd[NJ] PD gains (stable PD, see sim_step)
 *   joint_mu[NJ], joint_q0[NJ], joint_qd0[NJ], joint_target[NJ]
 *   env_plane[E]          1: ground plane z = 0 present
 */
typedef struct SimBatchDesc {
  int n_envs;
  const int* obj_off; const int* obj_shape; const double* obj_half; const double* obj_mass;
  const double* obj_mu; const double* obj_rest; const double* obj_pos; const double* obj_quat;
  const double* obj_vel; const double* obj_omega;
  const int* stat_off; const double* stat_pos; const double* stat_quat; const double* stat_half;
  const double* stat_mu;
  const int* art_off; const int* joint_off; const double* art_base_pos; const double* art_base_quat;
  const int* art_has_base_coll; const double* art_base_coll_off; const double* art_base_coll_half;
  const int* art_kinematic;
  const int* joint_parent; const int* joint_type; const double* joint_axis; const double* joint_origin_pos;
  const double* joint_origin_quat; const double* joint_com; const double* joint_half; const double* joint_mass;
  const double* joint_lo; const double* joint_hi; const int* joint_has_limit; const double* joint_kp;
  const double* joint_kd; const double* joint_mu; const double* joint_q0; const double* joint_qd0;
  const double* joint_target;
  const int* env_plane;
} SimBatchDesc;

/*
 * Step parameters.
 *   dt, gravity            time step (s), gravity (m/s^2)
 *   pgs_iters              PGS sweeps when pgs_tol == 0
 *   pgs_tol, pgs_max_iters residual mode: sweep until ||λ_k - λ_{k-1}|| /
 *                          max(||λ_k||, lambda_floor) <= pgs_tol, at most pgs_max_iters
 *   baumgarte, slop        position correction below -slop penetration
 *   margin                 contact distance; AABBs are fattened by margin/2
 *   rest_thresh            restitution only for approach speeds above this
 *   sleep_lin, sleep_ang, sleep_steps, sleep_enabled   a body sleeps after
 *                          sleep_steps consecutive steps under both speed thresholds
 *   warm_mode              0 cold, 1 prior-frame impulses, 2 learned (sim_set_mlp)
 *   plane_mu, match_dist   ground friction; warm-start point-match distance
 *   max_contacts           per-env contact capacity (<= SIM_MAX_CONTACTS)
 *   fp64_cond              articulations whose ABA pivots D_i span more than this
 *                          ratio get their joint-space inverse in FP64
 *   use_graph              1: sim_step replays a captured CUDA graph of the n steps
 *   log_features           1: every step also writes the learned warm start's 32
 *                          features per contact (needed by sim_log_contacts)
 */
typedef struct SimParams {
  double dt; double gravity[3]; int pgs_iters; double pgs_tol; int pgs_max_iters;
  double baumgarte, slop, margin, rest_thresh;
  double sleep_lin, sleep_ang; int sleep_steps; int sleep_enabled; int warm_mode;
  double plane_mu, lambda_floor, match_dist; int max_contacts;
  double fp64_cond; int use_graph; int log_features;
  double force_limit;  /* N: accumulated robot contact force that sets SIM_ENV_FORCE_LIMIT; <= 0 disables */
  /* Joint motors (the paper's Sec. 5.1 "Action space": impulse-capped motors with a
   * position gain).  motor_mode 1: every joint of a kinematic-base articulation (the
   * robot) gets a PGS row on its rate with target motor_kp (q_target - q) / dt and
   * impulse within +-motor_max_impulse (N s, or N m s) per step, warm-started from
   * the previous step's motor impulse; those joints then have no implicit PD (no
   * PD torque, no armature).  0: the implicit PD of the joint gains (default). */
  int motor_mode; double motor_kp; double motor_max_impulse;
} SimParams;

/*
 * State view for sim_get_state / sim_set_state: caller-owned float32 (and
 * int32) arrays laid out like the batch description; any pointer may be NULL
 * to skip that field.  C = max_contacts.
 *   obj_pos[NO*3], obj_pos_comp[NO*3] (Kahan compensation of the position sum),
 *   obj_quat[NO*4], obj_vel[NO*3], obj_omega[NO*3], obj_awake[NO], obj_ctr[NO],
 *   joint_q[NJ], joint_q_comp[NJ], joint_qd[NJ], joint_target[NJ],
 *   art_base_pos[NA*3], art_base_quat[NA*4],
 *   joint_lim_lambda[NJ], joint_lim_side[NJ] (0 none, 1 lower, 2 upper; last step's limit rows),
 *   cache_count[E], cache_key[E*C*3] (collider a, collider b, feature), cache_p[E*C*3],
 *   cache_lambda[E*C*4] (normal impulse, friction impulse as a world vector): the
 *   prior-frame warm-start cache written by the last step;
 *   joint_motor_lambda[NJ]: last step's motor impulse per joint (motor mode).
 */
typedef struct SimStateView {
  float* obj_pos; float* obj_pos_comp; float* obj_quat; float* obj_vel; float* obj_omega;
  int* obj_awake; int* obj_ctr;
  float* joint_q; float* joint_q_comp; float* joint_qd; float* joint_target;
  float* art_base_pos; float* art_base_quat;
  float* joint_lim_lambda; int* joint_lim_side;
  int* cache_count; int* cache_key; float* cache_p; float* cache_lambda;
  float* joint_motor_lambda;
} SimStateView;

/* Create a handle for a batch of environments, each holding the state s_t of the
 * simulator transition T:(s_t, a_t) -> s_{t+1} (Sec. 2, "What is a simulator?"):
 * validates and uploads `desc` (host arrays, copied), allocates all device state
 * on the current device -- the handle's device: every later call on the handle
 * selects it for its duration and restores the caller's current device -- and
 * enqueues on `cuda_stream` (a cudaStream_t of that device; NULL = legacy default
 * stream).  On failure *out is NULL. */
int sim_create(const SimBatchDesc* desc, const SimParams* params, void* cuda_stream, SimHandle** out);

/* Free the handle and all of its device memory (synchronises its stream). */
void sim_destroy(SimHandle* h);

/* Replace the step parameters (same max_contacts as at creation). */
int sim_set_params(SimHandle* h, const SimParams* params);

/* Joint PD targets for every joint, targets[NJ] float32 in joint_off order
 * (the agent's action a_t: joint-position targets of the arm's PD motors,
 * Sec. 5.1 "Action space").  Host array (on_device = 0, copied before return) or
 * device array of the handle's device (on_device = 1, read on the stream). */
int sim_set_joint_targets(SimHandle* h, const float* targets, int on_device);

/* Kinematic base pose of every kinematic articulation (the robot), xy_yaw[E*3]:
 * base position (x, y, unchanged z) and yaw about z.  The base is moved
 * kinematically, not simulated (Sec. 4.1 "Localized Physics", item 2: the robot's
 * base follows its navigation commands without dynamics). */
int sim_set_base_pose(SimHandle* h, const float* xy_yaw, int on_device);

/* Enqueue n physics steps of dt on the handle's stream (asynchronous): n
 * applications of the transition T (Sec. 2, "What is a simulator?"); the paper's
 * simulation step is 4 such steps of 1/120 s (Sec. 4.4).  Errors of the steps are
 * reported by sim_sync.  Step order per environment: (1) FK + ABA with stable PD
 * τ = kp(q̄ - q - dt q̇) - kd q̇ and armature dt kd + dt² kp, q̇* = q̇ + dt q̈;
 * CRBA + inverse; (2) v* = v + dt g for awake objects; (3) collision at x_t;
 * (4) rows and warm start; (5) PGS; (6) x += dt v (Kahan), quaternion update,
 * q += dt q̇ (Kahan), sleeping of resting objects (Sec. 4.1 item 3). */
int sim_step(SimHandle* h, int n);

/* Wait for the stream (the completion of the transitions enqueued by sim_step,
 * Sec. 2); OR of all per-env status bits since the last sim_sync
 * into *env_status_or (if not NULL), per-env bits into env_status[E] (if not
 * NULL), then clear them.  Returns SIM_ERR_NUMERIC / OVERFLOW / TIMEOUT when
 * the corresponding bit is set anywhere (in that priority; TIMEOUT for
 * SIM_ENV_ITER_CAP or SIM_ENV_DEVICE_WAIT), else SIM_OK. */
int sim_sync(SimHandle* h, uint32_t* env_status_or, uint32_t* env_status);

/* Copy the full state s_t (Sec. 2: the simulator's state between transitions;
 * the checkpoint of an episode) out to / in from caller buffers (see
 * SimStateView); host (0) or handle-device (1) buffers per to_device /
 * from_device; NULL fields are skipped.  Synchronises the stream. */
int sim_get_state(SimHandle* h, const SimStateView* out, int to_device);
int sim_set_state(SimHandle* h, const SimStateView* in, int from_device);

/* Per-env results of the last step (any pointer may be NULL): status bits,
 * PGS sweeps run, final relative residual, #contacts, #rows, #joint-limit rows,
 * #colours of the greedy colouring, and whether the FP64 inverse path ran for
 * some articulation of the env. */
int sim_get_env_stats(SimHandle* h, int* status, int* iters, float* resid, int* n_contacts, int* n_rows,
                      int* n_limit_rows, int* n_colours, int* fp64_used, int to_device);

/* Contacts of the last step, per env up to max_contacts in (a, b, feature)
 * order: count[E], key[E*C*3], point[E*C*3], normal (from B to A)[E*C*3],
 * separation[E*C], final impulses (normal, t1, t2)[E*C*3]. */
int sim_get_contacts(SimHandle* h, int* count, int* key, float* point, float* normal, float* sep, float* lam,
                     int to_device);

/* Candidate pairs of the last step after the wake pass, packed a*4096 + b,
 * ascending, per env up to pair_cap: count[E], pairs[E*pair_cap]. */
int sim_get_pairs(SimHandle* h, int pair_cap, int* count, int* pairs, int to_device);

/* Articulation kinematics/dynamics of the last step (at q_t): link COM[NJ*3],
 * link rotation[NJ*9] (row-major), q̈[NJ], and M(q)+armature inverse per
 * articulation [NA*81] (row-major 9x9, n x n block used). */
int sim_get_articulation(SimHandle* h, float* com, float* rot, float* qdd, float* minv, int to_device);

/* Learned warm start network (warm_mode 2): 32 -> 128 -> 128 -> 128 -> 3 with
 * GELU, parameters float32 in the layout W1[128][32] b1[128] W2[128][128] b2
 * W3[128][128] b3 W4[3][128] b4[3] (37635 values), stored on the device in
 * BF16 (weights) / FP32 (biases).  The network serves the contacts without a
 * prior-frame match and the matched ones whose relative velocity before the
 * solve (features 9-11) exceeds 4 |g| dt; the other contacts keep their
 * prior-frame impulse.  For a served contact its output (each component limited
 * to +-10) times the contact's impulse unit u = m_eff,n (|g| dt + |v_rel|) is
 * added to the prior-frame impulse (zero without a match) and projected onto the
 * friction pyramid; a non-finite output falls back to the prior frame.  params
 * NULL disables it. */
int sim_set_mlp(SimHandle* h, const float* params, int on_device);

/* The solver's warm start (the contract's single call for it): mode 0 cold (zero
 * impulses), 1 prior-frame impulses, 2 learned (the network of sim_set_mlp).
 * With mlp_params not NULL the network is (re)loaded as by sim_set_mlp (host or
 * device array per on_device); mode 2 with mlp_params NULL keeps the network
 * already set.  Equivalent to sim_set_params with that warm_mode followed by
 * sim_set_mlp.  Errors: SIM_ERR_INVALID_ARG (mode outside 0..2), SIM_ERR_STATE
 * (mode 2 and no network), the errors of sim_set_mlp. */
int sim_set_warm_start(SimHandle* h, int mode, const float* mlp_params, int on_device);

/* Batch totals of the last step (the contract's solver statistics: iterations,
 * residuals, contacts, awake bodies), reduced on the device; synchronises the
 * stream.  Per-environment values come from sim_get_env_stats. */
typedef struct SimStats {
  int32_t n_envs;
  int32_t max_iters;     /* most PGS sweeps of one environment */
  int64_t sum_iters;     /* PGS sweeps summed over the environments */
  int64_t row_sweeps;    /* sum over environments of rows x sweeps: the solver's row updates */
  int64_t n_contacts, n_rows, n_limit_rows;
  int64_t n_pool_slots;  /* articulation row endpoints (J and M~^-1 J^T rows of one contact on one articulation) */
  int64_t n_awake;       /* awake free objects after the step */
  int32_t n_iter_cap;    /* environments with SIM_ENV_ITER_CAP since the last sim_sync */
  int32_t n_fp64;        /* environments whose joint-space inverse ran in FP64 */
  int32_t max_colours;   /* most colours of one environment's Gauss-Seidel order */
  uint32_t status_or;    /* OR of the per-environment status bits since the last sim_sync */
  float max_resid;       /* largest final relative PGS residual */
  int64_t n_net_rows;    /* contacts the warm-start network served in the last
                          * physics step (warm mode 2; 0 otherwise) */
} SimStats;
int sim_get_stats(SimHandle* h, SimStats* out);

/* Contact-impulse log of the last step for training the warm-start network
 * (requires log_features = 1 during that step): per contact its 32 features
 * and its final impulses minus its prior-frame impulses (features 23-25),
 * divided by its impulse unit m_eff,n (|g| dt + |v_rel|) (the learned network's
 * target), in env then contact order, into feats[cap*32], lams[cap*3] (device
 * pointers).  Logged are the contacts of environments whose solve met the
 * residual target in that step (every environment at a fixed sweep count: only
 * converged impulses are targets) and whose three targets are finite (a
 * degenerate row, m_eff,n = 0, has no unit and is left out).  *n_out = number of
 * logged contacts (may exceed cap; only the first cap are written). */
int sim_log_contacts(SimHandle* h, float* feats, float* lams, int cap, int* n_out);

/* The learned warm start's raw network outputs of the last step (warm_mode 2):
 * the 3 predicted impulse corrections in units of m_eff,n (|g| dt + |v_rel|) of
 * each row that sim_log_contacts would log for the step (same rows, same order;
 * requires log_features or warm_mode 2), into preds[cap*3] (device pointer);
 * *n_out = number of those rows (only the first cap are written).  The network
 * runs only on the contacts it serves (see sim_set_mlp); the other rows hold
 * outputs left from earlier steps.
 * For checking the tensor-core inference against a reference forward. */
int sim_log_predictions(SimHandle* h, float* preds, int cap, int* n_out);

/* Testing the device's bounded waits: with on = 1 every following step withholds
 * its asynchronous completions -- the bulk copy of each environment's row pool
 * into the PGS kernel's shared memory is not issued, the learned warm start's
 * tensor-core MMAs are not committed to their mbarrier -- so those waits run out
 * (after 0.5 s): the PGS kernel reads the pool from global memory instead (for
 * the rest of that launch, every environment of the warp that gave up does, so a
 * late completion cannot overwrite what it reads; before the warp exits it waits,
 * bounded again, for a copy still in flight), the learned warm start keeps the
 * previous step's predictions, and the affected environments get
 * SIM_ENV_DEVICE_WAIT.  The results of the step are unchanged: both pool paths
 * compute the same values.  The context stays usable; on = 0 restores normal
 * operation. */
int sim_debug_hold_async(SimHandle* h, int on);

/*
 * Contact force on the robot (the paper's episode-failure signal, Sec. 5.1
 * "Evaluation": an episode fails once the accumulated contact force on the
 * arm / body exceeds 5 kN).  Per environment, each physics step adds the sum
 * of the normal impulses of its contacts with a link or the base box of a
 * kinematic-base articulation (the robot), divided by dt; above
 * params.force_limit the env's SIM_ENV_FORCE_LIMIT bit is set (sim_sync still
 * returns SIM_OK for it).  sim_get_robot_force copies E floats each of the
 * last step's force and the accumulated force (N; either pointer may be NULL;
 * host or device buffers per to_device).  sim_reset_robot_force zeroes the
 * accumulated force of env_ids[0..n) (host or device array per on_device), or
 * of every environment when env_ids is NULL; out-of-range indices give
 * SIM_ERR_INVALID_ARG (checked on the host for a host array; a device array's
 * bad entries are skipped and reported).  Synchronises the stream.
 */
int sim_get_robot_force(SimHandle* h, float* step_force, float* accumulated, int to_device);
int sim_reset_robot_force(SimHandle* h, const int* env_ids, int n, int on_device);

/*
 * Fast reset (the per-episode reset that the paper finds to be a bottleneck of
 * the training loop, Sec. 6, done on the device instead of by reloading).  The
 * handle keeps a reset template of every environment's state, initially the
 * batch's initial state.  sim_reset_envs restores env_ids[0..n) (host or device
 * int array per on_device) from it -- object poses, velocities, Kahan
 * compensations, sleep flags and counters, joint positions, rates, targets,
 * compensations and limit state, articulation base poses -- and clears their
 * prior-frame contact cache and robot contact force; other environments are
 * untouched.  A reset environment then steps exactly as a freshly created one
 * with that state.  Host lists are checked (SIM_ERR_INVALID_ARG for an index
 * outside [0, E)) and the call synchronises; a device list is used
 * asynchronously, so the call can be captured in a stream graph, and entries
 * outside [0, E) are skipped.  sim_set_reset_state replaces the template from
 * a state view (same layout as sim_set_state; the cache fields are ignored,
 * NULL fields keep their template values) -- e.g. new episode layouts
 * uploaded once, then reset on the device as episodes end.
 */
int sim_reset_envs(SimHandle* h, const int* env_ids, int n, int on_device);
int sim_set_reset_state(SimHandle* h, const SimStateView* in, int from_device);

/* Kernel timing: with enable = 1, every following sim_step also records CUDA
 * events around each of its kernels (inside the captured graph when use_graph
 * is set); with enable = 2 only around the PGS kernel (each event node costs a
 * few microseconds of step time; the other stages then read 0 ms); 0 turns it
 * off, other values are an error.  sim_kernel_times then waits for the stream
 * and writes, for the last sim_step call, the summed device time in
 * milliseconds of each of the
 * SIM_N_STAGES stages: ms[0] ABA, [1] collision, [2] rows, [3] learned warm
 * start, [4] LPT ordering of the PGS work queue, [5] PGS (with each
 * environment's integration in its write-back), [6] integration outside PGS
 * (no kernel: kept as a stage so the array layout does not change); and
 * launches[k] = kernels of that stage in that call (arrays of SIM_N_STAGES
 * entries). */
#define SIM_N_STAGES 7
int sim_set_profiling(SimHandle* h, int enable);
int sim_kernel_times(SimHandle* h, float* ms, int* launches);

/* Number of this library's kernels enqueued by sim_step since creation
 * (graph replays count every kernel node). */
int sim_launch_count(SimHandle* h, long long* count);

/*
 * Launch shapes of the three warp-per-environment kernels (collision, row
 * build, PGS).  Every environment is processed by one warp in all shapes;
 * the shape only decides how warps are grouped into blocks and how
 * environments are handed to warps.  A step's results are bit-identical
 * under every shape at a fixed sweep count; with a residual target
 * (pgs_tol > 0) the lanes per environment change the summation order of the
 * residual, so at the tolerance's edge the sweep that meets it can differ.  This is the batching of uneven environments into one
 * launch; the paper's concluding section names the synchronisation of
 * parallel environments as a bottleneck of the whole loop, and a warp that
 * waits for its block's slowest environment is that cost on the GPU.
 *   *_warps       environments (warps) per block: 1, 2, 4 or 8, where the
 *                 block's shared memory fits the device (sim_set_launch_shape
 *                 returns SIM_ERR_INVALID_ARG otherwise);
 *   *_persistent  0: one warp per environment slot in a plain grid;
 *                 1: a persistent grid (as many blocks as stay resident)
 *                 whose warps take the next environment slot from a device
 *                 counter until none is left;
 *   pgs_lpt       1: PGS slots are handed out in descending order of the
 *                 environment's row count (longest processing time first; the
 *                 order is recomputed on the first physics step of each
 *                 sim_step call -- it schedules work only, any order gives the
 *                 same results), 0: in environment order;
 *   pgs_lanes     lanes per environment in the PGS kernel: 32 (one warp), 16
 *                 or 8 (two or four environments share a warp, each on its own
 *                 lane group; a colour of the Gauss-Seidel order rarely holds
 *                 more than a few units, so narrower groups idle fewer lanes);
 *   pgs_min_blocks  register build of the PGS kernel: 2 (up to 128 registers
 *                 per thread) or, with 32 lanes, 1 (up to 255: no spills, for
 *                 shapes whose shared memory already limits the resident
 *                 warps) or 3 (up to 85, more resident warps, some values
 *                 spilled to local memory);
 *   pgs_heavy_sms with a persistent PGS grid in LPT order: SMs 0 .. n-1 each run
 *                 a single block whose environments start with the heaviest
 *                 ones (one per environment slot of the block), so the longest
 *                 Gauss-Seidel chains -- which set the kernel's length -- do
 *                 not share their SM; 0 = off, at most the SM count (and 256);
 *   pgs_stage_contacts, pgs_stage_pool
 *                 contacts and articulation row endpoints (J and M^-1 J^T of
 *                 one contact on one articulation) of an environment held in
 *                 shared memory during PGS; the rest are read from global
 *                 memory (same results, slower).  Larger values cost shared
 *                 memory and so resident environments.  0 = default
 *                 (contacts: 4 x the batch's largest object count + 8, at
 *                 least 32, at most max_contacts; endpoints: 32, halved down
 *                 to 8 while an environment would need more than 19 KB).
 *   aba_lanes     lanes per multi-joint articulation in the ABA kernel: 32
 *                 (one per warp) or 16 (two per warp; a 9-joint chain keeps at
 *                 most 9 lanes busy in most of its phases).
 *   partitions    1 .. SIM_MAX_PARTITIONS (and at most the environments): the
 *                 batch is split into that many equal runs of environments, and
 *                 each run's kernels go to a stream of its own, forked from the
 *                 handle's stream and joined back to it at the end of sim_step
 *                 (parallel branches of the captured graph).  Environments never
 *                 interact, so one run's kernels can fill the SMs another's leave
 *                 idle at the end of each of its kernels; the heavy SMs are split
 *                 between the runs.  Results do not depend on it.  While kernel
 *                 timing is on (sim_set_profiling), steps run unpartitioned, so
 *                 each kernel is timed alone.
 *   aba_overlap   1: the ABA kernels run on a side stream (a parallel branch of
 *                 the captured graph) beside the forward-kinematics and
 *                 collision kernels, which read only the link poses at q_t,
 *                 and are joined before the row kernel; 0: in sequence.
 *                 While kernel timing is on, in sequence.  Results do not
 *                 depend on it.
 *   fused         0: one kernel per stage (the fields above); 1: the n physics
 *                 steps of a sim_step call run as ONE persistent launch of
 *                 128-thread blocks in which each warp takes an environment from
 *                 a work queue (in LPT order with pgs_lpt) and carries it through
 *                 link poses, ABA, collision, rows, PGS (32 lanes, the shape's
 *                 staging capacities) and integration of all n steps, with no
 *                 synchronisation between environments.  Needs partitions = 1
 *                 and four warps' shared memory (each the PGS layout with the
 *                 other stages' working sets below its mbarrier) within a block.
 *                 Warm mode 2 (the network's inference) and kernel timing use
 *                 the stage kernels.  Results do not depend on it.
 * Default: 4 warps per block, plain grids, LPT on, 32 lanes per environment,
 * the 128-register build, no heavy SMs, default staging, 32 ABA lanes, one
 * partition, ABA beside collision, stage kernels.
 */
#define SIM_MAX_PARTITIONS 4
typedef struct SimLaunchShape {
  int32_t collide_warps, collide_persistent;
  int32_t rows_warps, rows_persistent;
  int32_t pgs_warps, pgs_persistent, pgs_lpt, pgs_lanes, pgs_min_blocks, pgs_heavy_sms;
  int32_t pgs_stage_contacts, pgs_stage_pool;
  int32_t aba_lanes;
  int32_t partitions;
  int32_t aba_overlap;
  int32_t fused;
} SimLaunchShape;

int sim_get_launch_shape(SimHandle* h, SimLaunchShape* out);
/* Validates and applies *in (a cached autotune result, for instance); the
 * captured step graph is rebuilt on the next sim_step. */
int sim_set_launch_shape(SimHandle* h, const SimLaunchShape* in);

#define SIM_TUNE_MAX_TRIALS 96
typedef struct SimTuneReport {
  int32_t n_trials;                  /* candidate shapes timed */
  int32_t steps_taken;               /* physics steps the tuning advanced the batch by */
  SimLaunchShape trial[SIM_TUNE_MAX_TRIALS];
  float ms[SIM_TUNE_MAX_TRIALS][5];  /* median device ms per physics step of the
                                      * collision, row-build and PGS (with its LPT
                                      * ordering) kernels, of the whole step and of
                                      * the ABA kernels under trial[t] (phase-4
                                      * trials: the whole step only) */
  float chosen_ms[5];                /* the same for the chosen options: phase-1
                                      * mean for collision, rows and ABA, phase-3
                                      * PGS and whole step of the chosen shape */
} SimTuneReport;

/*
 * Autotuner.  Phase 1 times every admissible option of each kernel -- ABA
 * lanes {32, 16}; warps per block x {plain, persistent} of the collision,
 * row-build and PGS kernels, and for PGS x {LPT on, off} x lanes per
 * environment {32, 16} x heavy SMs {0, SMs/16, SMs/8, SMs/4} (32 lanes,
 * persistent, LPT) -- on the live batch: trial t runs option t mod (options
 * of that kernel) of every kernel for steps_per_trial physics steps without
 * graph capture, with CUDA events around each kernel; the trials run
 * round-robin (forward on even rounds, backward on odd ones), once untimed
 * (warm-up) and then `rounds` timed times.  For
 * each kernel the option with the lowest mean of its trials' median time is
 * kept.  Phase 2 times PGS staging capacities ({1/2, 1, 3/2} x the default
 * contacts x {8, 16, 32, 64} endpoints, the phase-1 shape among them) under
 * that shape the same way and keeps the fastest.  Phase 3 is a play-off for
 * the PGS kernel: the phase-2 shape and up to three more, which combine the
 * phase-1 runners-up's grid options (warps, persistence, lanes, LPT, heavy SMs)
 * with the phase-2 staging, run round-robin as above but each captured into a
 * CUDA graph and replayed, as sim_step runs it; the fastest PGS median wins.
 * Phase 4 times the whole step with 1, 2 and 4 partitions, with one partition and
 * the ABA kernels in sequence (aba_overlap 0), and with the fused step kernel
 * (fused 1, where it fits and the warm mode is not 2), under that shape (graph
 * replay without events inside, CUDA events around the launch; each trial first
 * replays once untimed) and keeps the fastest.
 * The result is applied (and returned in *chosen when non-NULL; *report, when
 * non-NULL, receives every trial of the four phases).  Every round of a phase
 * saves the step state on the device (bodies, joints, bases, the warm-start
 * cache, the robot's contact forces, status flags) and runs each of its trials
 * from that same state, so the trials of a round time identical steps; the
 * tuning steps are real physics steps and the batch advances by
 * report->steps_taken steps ((rounds + 1) * steps_per_trial for each of phases
 * 1-3, twice that for phase 4: per round, the last trial's steps), exactly as
 * sim_step of that many steps would advance it, because results do not depend
 * on the launch shape.  The saved state needs device memory of about the
 * state's size for the duration of the call.  Synchronises the handle's stream; the
 * caller's profiling and use_graph settings are restored.  Errors:
 * SIM_ERR_INVALID_ARG (steps_per_trial or rounds < 1), SIM_ERR_STATE (warm
 * mode 2 without network), SIM_ERR_CUDA (the previous shape is restored).
 */
int sim_autotune(SimHandle* h, int steps_per_trial, int rounds, SimLaunchShape* chosen, SimTuneReport* report);

/*
 * Warm-start network trainer (the learned warm start of sim_set_mlp).  The
 * network is trained on (features, converged impulse) pairs logged by
 * sim_log_contacts with the project's own kernels: fused BF16 tensor-core
 * forward (FP32 accumulation, activations kept per layer), BF16 GEMM backward,
 * mean-squared-error loss L = 1/(3n) sum (y - t)^2, Adam (beta 0.9 / 0.999,
 * eps 1e-8) on FP32 master weights.  Inputs are normalised inside the trainer
 * by feat_mean / feat_std (NULL: identity); mlp_get_params returns parameters
 * for raw features (normalisation folded into W1, b1) in the layout of
 * sim_set_mlp.  All X / T / Y / gradient pointers are device pointers of
 * row-major float32 arrays, X 16-byte aligned (the forward reads each row's
 * features as 16-byte vectors; any allocation of [n][32] float32 rows, or a row
 * slice of one, is); init_params is host (on_device = 0) or device.
 *   mlp_train_create   batch = largest n of any later call
 *   mlp_train_step     one Adam step on n rows; *loss_out (host, may be NULL)
 *   mlp_loss_grad      loss and gradient (device grad_out[37635]) without a step
 *   mlp_forward        Y[n][3] = network(X) with the current weights
 * Errors: SIM_ERR_INVALID_ARG for NULL pointers, an X not 16-byte aligned or n
 * outside [1, batch], SIM_ERR_OOM / SIM_ERR_CUDA as for the simulator.
 */
typedef struct MlpTrainer MlpTrainer;
/* Training-set preparation, on the device (the learned warm start's recipe):
 *   mlp_select_rows  keeps the logged rows (X[n][32], T[n][3], device) whose
 *       targets are finite and, with only_used = 1, only the rows the in-step warm
 *       start serves (feature 26 = 0, or |features 9-11| > gate_speed, which is
 *       4 |g| dt for the simulator's gravity and step); targets clipped to
 *       [-clip, clip] (clip > 0); kept rows in their order into X_out, T_out
 *       (device, n rows of room); *n_out (host) = rows kept.  Synchronises.
 *   mlp_feature_stats  per-feature mean and population standard deviation of
 *       X[n][32] (device; a deviation below 1e-6 is reported as 1), into host or
 *       device arrays of 32 per to_device -- the normalisation of mlp_train_create.
 * Both enqueue on cuda_stream and use stream-ordered scratch (cudaMallocAsync). */
int mlp_select_rows(const float* X, const float* T, int n, int only_used, float gate_speed, float clip,
                    float* X_out, float* T_out, int* n_out, void* cuda_stream);
int mlp_feature_stats(const float* X, int n, float* mean, float* std_out, int to_device, void* cuda_stream);
int mlp_train_create(const float* init_params, int on_device, int batch, const float* feat_mean,
                     const float* feat_std, void* cuda_stream, MlpTrainer** out);
void mlp_train_destroy(MlpTrainer* t);
int mlp_train_step(MlpTrainer* t, const float* X, const float* T, int n, float lr, float* loss_out);
int mlp_loss_grad(MlpTrainer* t, const float* X, const float* T, int n, float* grad_out, float* loss_out);
int mlp_forward(MlpTrainer* t, const float* X, int n, float* Y);
int mlp_get_params(MlpTrainer* t, float* params_out, int to_device);

/* Allocation-free sim_log_contacts (the paper has no counterpart; this is a
 * library service).  For callers that must not allocate device memory while
 * they run: a training loop whose framework allocator already holds the GPU's
 * memory budget, or a real-time control loop that cannot take the implicit
 * device synchronisation of cudaMalloc/cudaFree.  Same arguments, outputs,
 * errors (checked in the same order) and kernels as sim_log_contacts; its
 * per-environment counts and prefix sums live in a fixed device array of
 * SIM_NOALLOC_MAX_ENVS + 1 ints that every GPU loading the library holds until
 * the process exits, instead of a buffer the handle may allocate.
 *   - The array's device address is looked up (cudaGetSymbolAddress) on the
 *     handle's device when the handle is created, so no call does it; a handle
 *     created after a device reset looks it up afresh.
 *   - Like sim_log_contacts, the call ends by copying the count to the host and
 *     synchronising the handle's stream, so that stream must not be capturing a
 *     graph when it is called.
 *   - Handles with more than SIM_NOALLOC_MAX_ENVS environments are rejected
 *     with SIM_ERR_INVALID_ARG.
 *   - All calls share the array: calls whose work overlaps on the GPU (other
 *     streams or handles of the same device) race; serialise them.
 *   - Calls no cudaMalloc, cudaFree or allocating library routine. */
#define SIM_NOALLOC_MAX_ENVS 65536
int sim_log_contacts_noalloc(SimHandle* h, float* feats, float* lams, int cap, int* n_out);

/* FP32 throughput of the current device measured by the library's own kernel
 * (no counterpart in the paper: the denominator of the solver kernels' ALU
 * roofline): every SM filled to its resident-thread limit, each thread running 8
 * independent fused multiply-add chains of iters x 16 steps; the best of `reps`
 * launches after one warm-up, timed with CUDA events on cuda_stream.  *tflops =
 * 2 x FMAs / time in TFLOP/s; *ms_best (may be NULL) its duration.  Allocates and
 * frees a small output buffer; synchronises the stream. */
int sim_fp32_fma_peak(void* cuda_stream, int iters, int reps, double* tflops, double* ms_best);

/* Human-readable description of the last error of a call on handle h (the
 * contract's per-handle error string), or of any call on this thread when h is
 * NULL; an empty string when there was none.  The string stays valid until the
 * next failing call on h (or on this thread). */
const char* sim_last_error(const SimHandle* h);

#ifdef __cplusplus
}
#endif

#endif
