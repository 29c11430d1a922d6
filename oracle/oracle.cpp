// FP64 CPU oracle for the batched rigid/articulated physics step.
//
// TEST INFRASTRUCTURE ONLY.  This engine exists to check the CUDA engine; only
// the test suite, the package's smoke check and the benchmark's CPU-baseline leg
// may load it.  It shares no code, header, table or helper with the CUDA path:
// both implement the same published methods independently.  It is deliberately
// plain: double precision, scalar loops, one environment at a time, no blocking
// or fusion beyond what each method states.
//
// What it computes, one physics step of dt per environment (the paper's
// simulator transition T:(s_t, a_t) -> s_{t+1}, Sec. 2 "What is a simulator?";
// robot of Sec. 5.1 "Agent embodiment", PD joint motors of Sec. 5.1 "Action space";
// kinematic base, sleeping and static receptacle parts of Sec. 4.1 "Localized
// Physics"; the paper names Bullet but prints no physics equations, so each
// stage follows the textbook method named at its function):
//   1. articulations: forward kinematics, Featherstone's articulated-body
//      algorithm (ABA) with a stable (implicit) PD motor folded in as armature,
//      q̇* = q̇ + dt q̈;  CRBA mass matrix M + diag(armature) and its inverse;
//   2. free bodies: v* = v + dt g (awake only), ω* = ω (no gyroscopic term);
//   3. collision at x_t: fattened AABBs, all-pairs broadphase, wake pass,
//      sphere/box/plane narrowphase (box-box by 15-axis SAT and
//      Sutherland-Hodgman clipping), contacts in (a, b, feature) order;
//   4. rows: normal + two friction rows per contact, joint-limit rows;
//      warm start (cold / prior frame / learned);
//   5. projected Gauss-Seidel (sequential impulses) in the shared order or
//      in greedy-colour order, with the relative residual;
//   6. semi-implicit Euler integration and sleeping.
//
// Parity pins live in tests/test_oracle_pins.py (free fall closed form,
// pendulum frequency of semi-implicit Euler, ABA == CRBA dense solve, energy
// drift order, elastic momentum exchange, brute-force SAT / AABB / LCP
// enumeration, friction on inclines, sleep timing, MLP finite differences).
//
// Build: g++ -O2 -std=c++17 -shared -fPIC oracle.cpp -o liboracle.so
//        (add -DORACLE_COUNT_OPS for the op-counting variant used to state the
//        algorithmic FLOPs per env-step of each stage, or -DORACLE_FP32 for the
//        same algorithm in single precision, used to measure the FP32 floor of
//        each output when deriving parity tolerances).

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

// ---------------------------------------------------------------------------
// Scalar type: double, or a double that counts arithmetic operations.
// ---------------------------------------------------------------------------
enum { ST_ABA = 0, ST_PREDICT, ST_COLLIDE, ST_ROWS, ST_PGS, ST_INTEGRATE, ST_MLP, ST_COUNT };
static thread_local int g_stage = 0;
static thread_local uint64_t g_ops[ST_COUNT];
// counts of worker threads that have finished (each adds its own when its range ends)
static std::atomic<uint64_t> g_ops_done[ST_COUNT];
static void flush_op_counts() {
  for (int i = 0; i < ST_COUNT; ++i) {
    g_ops_done[i] += g_ops[i];
    g_ops[i] = 0;
  }
}

#ifdef ORACLE_COUNT_OPS
struct real {
  double v;
  real() : v(0) {}
  real(double x) : v(x) {}
  explicit operator double() const { return v; }
};
static inline void cnt(int k = 1) { g_ops[g_stage] += k; }
static inline real operator+(real a, real b) { cnt(); return real(a.v + b.v); }
static inline real operator-(real a, real b) { cnt(); return real(a.v - b.v); }
static inline real operator*(real a, real b) { cnt(); return real(a.v * b.v); }
static inline real operator/(real a, real b) { cnt(); return real(a.v / b.v); }
static inline real operator-(real a) { return real(-a.v); }
static inline real& operator+=(real& a, real b) { cnt(); a.v += b.v; return a; }
static inline real& operator-=(real& a, real b) { cnt(); a.v -= b.v; return a; }
static inline real& operator*=(real& a, real b) { cnt(); a.v *= b.v; return a; }
static inline real& operator/=(real& a, real b) { cnt(); a.v /= b.v; return a; }
static inline bool operator<(real a, real b) { return a.v < b.v; }
static inline bool operator>(real a, real b) { return a.v > b.v; }
static inline bool operator<=(real a, real b) { return a.v <= b.v; }
static inline bool operator>=(real a, real b) { return a.v >= b.v; }
static inline bool operator==(real a, real b) { return a.v == b.v; }
static inline bool operator!=(real a, real b) { return a.v != b.v; }
static inline real rsqrt_(real a) { cnt(); return real(std::sqrt(a.v)); }
static inline real Sqrt(real a) { cnt(); return real(std::sqrt(a.v)); }
static inline real Fabs(real a) { return real(std::fabs(a.v)); }
static inline real Sin(real a) { cnt(); return real(std::sin(a.v)); }
static inline real Cos(real a) { cnt(); return real(std::cos(a.v)); }
static inline real Erf(real a) { cnt(); return real(std::erf(a.v)); }
static inline real Exp(real a) { cnt(); return real(std::exp(a.v)); }
static inline double D(real a) { return a.v; }
static inline bool Finite(real a) { return std::isfinite(a.v); }
#elif defined(ORACLE_FP32)
// Same algorithm in single precision: measures the floor any FP32 engine meets.
typedef float real;
static inline real Sqrt(real a) { return std::sqrt(a); }
static inline real Fabs(real a) { return std::fabs(a); }
static inline real Sin(real a) { return std::sin(a); }
static inline real Cos(real a) { return std::cos(a); }
static inline real Erf(real a) { return std::erf(a); }
static inline real Exp(real a) { return std::exp(a); }
static inline double D(real a) { return a; }
static inline bool Finite(real a) { return std::isfinite(a); }
#else
typedef double real;
static inline real Sqrt(real a) { return std::sqrt(a); }
static inline real Fabs(real a) { return std::fabs(a); }
static inline real Sin(real a) { return std::sin(a); }
static inline real Cos(real a) { return std::cos(a); }
static inline real Erf(real a) { return std::erf(a); }
static inline real Exp(real a) { return std::exp(a); }
static inline double D(real a) { return a; }
static inline bool Finite(real a) { return std::isfinite(a); }
#endif

static inline real Max(real a, real b) { return a < b ? b : a; }
static inline real Min(real a, real b) { return b < a ? b : a; }

// ---------------------------------------------------------------------------
// 3-vectors, 3x3 matrices, quaternions (w, x, y, z)
// ---------------------------------------------------------------------------
struct V3 {
  real x, y, z;
  V3() : x(0), y(0), z(0) {}
  V3(real a, real b, real c) : x(a), y(b), z(c) {}
  real& operator[](int i) { return i == 0 ? x : (i == 1 ? y : z); }
  real operator[](int i) const { return i == 0 ? x : (i == 1 ? y : z); }
};
static inline V3 operator+(V3 a, V3 b) { return V3(a.x + b.x, a.y + b.y, a.z + b.z); }
static inline V3 operator-(V3 a, V3 b) { return V3(a.x - b.x, a.y - b.y, a.z - b.z); }
static inline V3 operator*(V3 a, real s) { return V3(a.x * s, a.y * s, a.z * s); }
static inline V3 operator*(real s, V3 a) { return V3(a.x * s, a.y * s, a.z * s); }
static inline V3 operator-(V3 a) { return V3(-a.x, -a.y, -a.z); }
static inline real dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static inline V3 cross(V3 a, V3 b) {
  return V3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
static inline real norm(V3 a) { return Sqrt(dot(a, a)); }

struct M3 {
  real m[3][3];
  M3() { for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) m[i][j] = 0; }
};
static inline M3 mmul(const M3& a, const M3& b) {
  M3 r;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      real s = 0;
      for (int k = 0; k < 3; ++k) s += a.m[i][k] * b.m[k][j];
      r.m[i][j] = s;
    }
  return r;
}
static inline V3 mv(const M3& a, V3 v) {
  return V3(a.m[0][0] * v.x + a.m[0][1] * v.y + a.m[0][2] * v.z,
            a.m[1][0] * v.x + a.m[1][1] * v.y + a.m[1][2] * v.z,
            a.m[2][0] * v.x + a.m[2][1] * v.y + a.m[2][2] * v.z);
}
static inline V3 mtv(const M3& a, V3 v) {  // a^T v
  return V3(a.m[0][0] * v.x + a.m[1][0] * v.y + a.m[2][0] * v.z,
            a.m[0][1] * v.x + a.m[1][1] * v.y + a.m[2][1] * v.z,
            a.m[0][2] * v.x + a.m[1][2] * v.y + a.m[2][2] * v.z);
}
static inline V3 col(const M3& a, int j) { return V3(a.m[0][j], a.m[1][j], a.m[2][j]); }

struct Quat { real w, x, y, z; };
static M3 quat_to_mat(Quat q) {
  M3 r;
  real w = q.w, x = q.x, y = q.y, z = q.z;
  r.m[0][0] = 1 - 2 * (y * y + z * z); r.m[0][1] = 2 * (x * y - w * z); r.m[0][2] = 2 * (x * z + w * y);
  r.m[1][0] = 2 * (x * y + w * z); r.m[1][1] = 1 - 2 * (x * x + z * z); r.m[1][2] = 2 * (y * z - w * x);
  r.m[2][0] = 2 * (x * z - w * y); r.m[2][1] = 2 * (y * z + w * x); r.m[2][2] = 1 - 2 * (x * x + y * y);
  return r;
}
// Rotation by angle t about unit axis u (Rodrigues' formula).
static M3 axis_angle(V3 u, real t) {
  real c = Cos(t), s = Sin(t), k = 1 - c;
  M3 r;
  r.m[0][0] = c + u.x * u.x * k;        r.m[0][1] = u.x * u.y * k - u.z * s; r.m[0][2] = u.x * u.z * k + u.y * s;
  r.m[1][0] = u.y * u.x * k + u.z * s;  r.m[1][1] = c + u.y * u.y * k;       r.m[1][2] = u.y * u.z * k - u.x * s;
  r.m[2][0] = u.z * u.x * k - u.y * s;  r.m[2][1] = u.z * u.y * k + u.x * s; r.m[2][2] = c + u.z * u.z * k;
  return r;
}
// Box inertia about its centre, principal axes = box axes (half extents h).
static V3 box_inertia(real m, V3 h) {
  return V3(m * (h.y * h.y + h.z * h.z) / 3, m * (h.x * h.x + h.z * h.z) / 3, m * (h.x * h.x + h.y * h.y) / 3);
}
// World inverse inertia R diag(d) R^T.
static M3 rot_diag(const M3& R, V3 d) {
  M3 r;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      r.m[i][j] = R.m[i][0] * d.x * R.m[j][0] + R.m[i][1] * d.y * R.m[j][1] + R.m[i][2] * d.z * R.m[j][2];
  return r;
}

// ---------------------------------------------------------------------------
// Spatial algebra (Featherstone 2008, ch. 2): motion m = (ω; v_O), force
// f = (n_O; f), all in world-aligned axes about a reference point O.
// ---------------------------------------------------------------------------
struct SV { real v[6]; SV() { for (int i = 0; i < 6; ++i) v[i] = 0; } };
struct SM { real m[6][6]; SM() { for (int i = 0; i < 6; ++i) for (int j = 0; j < 6; ++j) m[i][j] = 0; } };
static SV sv(V3 a, V3 b) { SV r; r.v[0] = a.x; r.v[1] = a.y; r.v[2] = a.z; r.v[3] = b.x; r.v[4] = b.y; r.v[5] = b.z; return r; }
static V3 ang(const SV& s) { return V3(s.v[0], s.v[1], s.v[2]); }
static V3 lin(const SV& s) { return V3(s.v[3], s.v[4], s.v[5]); }
static SV add(const SV& a, const SV& b) { SV r; for (int i = 0; i < 6; ++i) r.v[i] = a.v[i] + b.v[i]; return r; }
static SV scale(const SV& a, real s) { SV r; for (int i = 0; i < 6; ++i) r.v[i] = a.v[i] * s; return r; }
static real sdot(const SV& a, const SV& b) { real s = 0; for (int i = 0; i < 6; ++i) s += a.v[i] * b.v[i]; return s; }
static SV smv(const SM& m, const SV& a) {
  SV r;
  for (int i = 0; i < 6; ++i) { real s = 0; for (int j = 0; j < 6; ++j) s += m.m[i][j] * a.v[j]; r.v[i] = s; }
  return r;
}
static SM sadd(const SM& a, const SM& b) { SM r; for (int i = 0; i < 6; ++i) for (int j = 0; j < 6; ++j) r.m[i][j] = a.m[i][j] + b.m[i][j]; return r; }
// motion x motion
static SV crm(const SV& a, const SV& b) { return sv(cross(ang(a), ang(b)), cross(ang(a), lin(b)) + cross(lin(a), ang(b))); }
// motion x* force
static SV crf(const SV& a, const SV& f) { return sv(cross(ang(a), ang(f)) + cross(lin(a), lin(f)), cross(ang(a), lin(f))); }
// Spatial inertia about O of a body with mass m, centre c (relative to O), rotational inertia Ic about c.
static SM spatial_inertia(real m, V3 c, const M3& Ic) {
  SM r;
  // [[Ic + m cx cx^T, m cx], [m cx^T, m 1]], cx = skew(c)
  real cxm[3][3] = {{0, -c.z, c.y}, {c.z, 0, -c.x}, {-c.y, c.x, 0}};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      real s = 0;
      for (int k = 0; k < 3; ++k) s += cxm[i][k] * cxm[j][k];
      r.m[i][j] = Ic.m[i][j] + m * s;
      r.m[i][3 + j] = m * cxm[i][j];
      r.m[3 + i][j] = m * cxm[j][i];
      r.m[3 + i][3 + j] = (i == j) ? m : real(0);
    }
  return r;
}

// ---------------------------------------------------------------------------
// Public structures (the oracle's own definitions of the batch layout).
// ---------------------------------------------------------------------------
extern "C" {
typedef struct {
  int n_envs;
  const int* obj_off; const int* obj_shape; const double* obj_half; const double* obj_mass;
  const double* obj_mu; const double* obj_rest; const double* obj_pos; const double* obj_quat;
  const double* obj_vel; const double* obj_omega;
  const int* stat_off; const double* stat_pos; const double* stat_quat; const double* stat_half; const double* stat_mu;
  const int* art_off; const int* joint_off; const double* art_base_pos; const double* art_base_quat;
  const int* art_has_base_coll; const double* art_base_coll_off; const double* art_base_coll_half; const int* art_kinematic;
  const int* joint_parent; const int* joint_type; const double* joint_axis; const double* joint_origin_pos;
  const double* joint_origin_quat; const double* joint_com; const double* joint_half; const double* joint_mass;
  const double* joint_lo; const double* joint_hi; const int* joint_has_limit; const double* joint_kp;
  const double* joint_kd; const double* joint_mu; const double* joint_q0; const double* joint_qd0; const double* joint_target;
  const int* env_plane;
} OrDesc;

typedef struct {
  double dt; double gravity[3]; int pgs_iters; double pgs_tol; int pgs_max_iters;
  double baumgarte, slop, margin, rest_thresh;
  double sleep_lin, sleep_ang; int sleep_steps; int sleep_enabled; int warm_mode;
  double plane_mu, lambda_floor, match_dist; int max_contacts; int use_colouring;
  double force_limit;
  int motor_mode; double motor_kp, motor_max_impulse;
} OrParams;
}

enum { SHAPE_SPHERE = 0, SHAPE_BOX = 1, SHAPE_PLANE = 2 };
enum { JT_REV = 0, JT_PRISM = 1 };
enum { STATUS_OVERFLOW = 1, STATUS_NUMERIC = 2, STATUS_ITER_CAP = 4, STATUS_FORCE = 8 };
static const int MAXDOF = 9;

struct Obj {
  int shape; V3 half; real mass, inv_mass; V3 inv_I; real mu, rest;
  V3 x; Quat q; V3 v, w; int awake, ctr;
};
struct Stat { V3 x; Quat q; V3 half; real mu; };
struct Joint {
  int parent, type; V3 axis, opos; Quat oq; V3 com, half; real mass; real lo, hi; int has_limit; real kp, kd, mu;
  real q, qd, target; real lim_lambda; int lim_side;
  real motor_lambda;  // last step's motor impulse (motor mode)
};
struct Art {
  V3 base_x; Quat base_q; int has_bc; V3 bc_off, bc_half; int kinematic;
  int motor = 0;  // this step: joints driven by impulse-capped motor rows instead of the implicit PD
  std::vector<Joint> j;
  // per-step kinematics and dynamics (at q_t)
  M3 R[MAXDOF]; V3 o[MAXDOF], c[MAXDOF], ja[MAXDOF], jo[MAXDOF];
  real qdd[MAXDOF], qd_star[MAXDOF];
  real M[MAXDOF][MAXDOF], Minv[MAXDOF][MAXDOF];
};
struct CacheEntry { int a, b, f; V3 p; real ln; V3 lt; };
struct Contact { int a, b, f; V3 p, n; real sep; real lam[3]; };

struct Env {
  std::vector<Obj> obj;
  std::vector<Stat> st;
  std::vector<Art> art;
  int plane;
  std::vector<CacheEntry> cache;
  // results of the last step
  std::vector<Contact> contacts;
  std::vector<int> pairs;  // candidate pairs after filtering, packed a*4096+b
  int n_rows, iters, status, n_limit_rows, n_colours;
  real resid;
  // contact force on the robot: this step, and accumulated since the last reset
  real robot_force = 0, robot_force_acc = 0;
  std::vector<double> mlp_pred;  // learned warm start per contact (3), set from outside
  // colouring of the last step, per unit in unit order: colour (64: serial overflow)
  // and the two colouring nodes (-1: static)
  std::vector<int> unit_colour, unit_node_a, unit_node_b;
};

struct World {
  OrParams P;
  std::vector<Env> env;
  std::vector<int> obj_off, art_off, joint_off, stat_off;
  int n_obj, n_art, n_joint, n_stat;
  // optional learned warm-start network (FP64)
  std::vector<double> mlp_w;  // flat parameters
  int has_mlp;
};

// ---------------------------------------------------------------------------
// 1. Articulations: FK, ABA with implicit PD, RNEA, CRBA, inverse.
//    Featherstone, Rigid Body Dynamics Algorithms (2008): ABA Table 7.1 /
//    ch. 7.3 (here in world-aligned coordinates about the base origin), RNEA
//    ch. 5.3, CRBA ch. 6.2.  Implicit PD: Tan, Liu & Turk, "Stable
//    Proportional-Derivative Controllers", IEEE CG&A 2011, with the position
//    at the next step taken as q + dt q̇ + dt² q̈ (semi-implicit Euler), which
//    adds dt kd + dt² kp to each joint's D_i (joint-space armature).
// ---------------------------------------------------------------------------
static void art_fk(Art& A) {
  M3 Rb = quat_to_mat(A.base_q);
  for (size_t i = 0; i < A.j.size(); ++i) {
    const Joint& J = A.j[i];
    M3 Rp = J.parent < 0 ? Rb : A.R[J.parent];
    V3 op = J.parent < 0 ? A.base_x : A.o[J.parent];
    M3 Rj = mmul(Rp, quat_to_mat(J.oq));
    V3 oj = op + mv(Rp, J.opos);
    V3 a = mv(Rj, J.axis);
    if (J.type == JT_REV) {
      A.R[i] = mmul(Rj, axis_angle(J.axis, J.q));
      A.o[i] = oj;
    } else {
      A.R[i] = Rj;
      A.o[i] = oj + a * J.q;
    }
    A.ja[i] = a;
    A.jo[i] = oj;
    A.c[i] = A.o[i] + mv(A.R[i], J.com);
  }
}

static SV joint_S(const Art& A, int i) {
  V3 a = A.ja[i];
  if (A.j[i].type == JT_REV) return sv(a, cross(A.jo[i] - A.base_x, a));
  return sv(V3(0, 0, 0), a);
}
static SM link_inertia(const Art& A, int i) {
  const Joint& J = A.j[i];
  V3 Id = box_inertia(J.mass, J.half);
  M3 Ic = rot_diag(A.R[i], Id);
  return spatial_inertia(J.mass, A.c[i] - A.base_x, Ic);
}
static real armature(const Joint& J, real dt) { return dt * J.kd + dt * dt * J.kp; }
static real pd_tau(const Joint& J, real dt) { return J.kp * (J.target - J.q - dt * J.qd) - J.kd * J.qd; }
// the implicit PD of articulation A's joint i (none for joints driven by motor rows)
static real arm_of(const Art& A, int i, real dt) { return A.motor ? real(0) : armature(A.j[i], dt); }
static real tau_of(const Art& A, int i, real dt) { return A.motor ? real(0) : pd_tau(A.j[i], dt); }

// ABA: q̈ for joint torques tau (implicit-PD armature on D_i when dt > 0).
static void art_aba(const Art& A, V3 g, real dt, const real* tau, real* qdd) {
  int n = (int)A.j.size();
  SV vel[MAXDOF], cb[MAXDOF], pA[MAXDOF], U[MAXDOF], acc[MAXDOF], S[MAXDOF];
  SM IA[MAXDOF];
  real Dd[MAXDOF], u[MAXDOF];
  for (int i = 0; i < n; ++i) {
    S[i] = joint_S(A, i);
    SV vp = A.j[i].parent < 0 ? SV() : vel[A.j[i].parent];
    SV vJ = scale(S[i], A.j[i].qd);
    vel[i] = add(vp, vJ);
    cb[i] = crm(vel[i], vJ);
    IA[i] = link_inertia(A, i);
    pA[i] = crf(vel[i], smv(IA[i], vel[i]));
  }
  for (int i = n - 1; i >= 0; --i) {
    U[i] = smv(IA[i], S[i]);
    Dd[i] = sdot(S[i], U[i]) + arm_of(A, i, dt);
    u[i] = tau[i] - sdot(S[i], pA[i]);
    int p = A.j[i].parent;
    if (p >= 0) {
      SM Ia;
      for (int r = 0; r < 6; ++r)
        for (int c = 0; c < 6; ++c) Ia.m[r][c] = IA[i].m[r][c] - U[i].v[r] * U[i].v[c] / Dd[i];
      SV pa = add(add(pA[i], smv(Ia, cb[i])), scale(U[i], u[i] / Dd[i]));
      IA[p] = sadd(IA[p], Ia);
      pA[p] = add(pA[p], pa);
    }
  }
  SV a0 = sv(V3(0, 0, 0), -g);  // gravity as an upward acceleration of the fixed base
  for (int i = 0; i < n; ++i) {
    SV ap = A.j[i].parent < 0 ? a0 : acc[A.j[i].parent];
    SV a1 = add(ap, cb[i]);
    qdd[i] = (u[i] - sdot(U[i], a1)) / Dd[i];
    acc[i] = add(a1, scale(S[i], qdd[i]));
  }
}

// RNEA: joint forces that produce accelerations qdd (gravity included).
static void art_rnea(const Art& A, V3 g, const real* qdd, real* tau) {
  int n = (int)A.j.size();
  SV vel[MAXDOF], acc[MAXDOF], f[MAXDOF], S[MAXDOF];
  SV a0 = sv(V3(0, 0, 0), -g);
  for (int i = 0; i < n; ++i) {
    S[i] = joint_S(A, i);
    int p = A.j[i].parent;
    SV vp = p < 0 ? SV() : vel[p];
    SV ap = p < 0 ? a0 : acc[p];
    SV vJ = scale(S[i], A.j[i].qd);
    vel[i] = add(vp, vJ);
    acc[i] = add(add(ap, scale(S[i], qdd[i])), crm(vel[i], vJ));
    SM I = link_inertia(A, i);
    f[i] = add(smv(I, acc[i]), crf(vel[i], smv(I, vel[i])));
  }
  for (int i = n - 1; i >= 0; --i) {
    tau[i] = sdot(S[i], f[i]);
    if (A.j[i].parent >= 0) f[A.j[i].parent] = add(f[A.j[i].parent], f[i]);
  }
}

// CRBA: joint-space inertia M(q) (+ armature on the diagonal when dt > 0).
static void art_crba(Art& A, real dt) {
  int n = (int)A.j.size();
  SM Ic[MAXDOF];
  SV S[MAXDOF];
  for (int i = 0; i < n; ++i) { Ic[i] = link_inertia(A, i); S[i] = joint_S(A, i); }
  for (int i = n - 1; i >= 0; --i)
    if (A.j[i].parent >= 0) Ic[A.j[i].parent] = sadd(Ic[A.j[i].parent], Ic[i]);
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k) A.M[i][k] = 0;
  for (int i = 0; i < n; ++i) {
    SV F = smv(Ic[i], S[i]);
    A.M[i][i] = sdot(S[i], F) + arm_of(A, i, dt);
    for (int k = A.j[i].parent; k >= 0; k = A.j[k].parent) {
      A.M[i][k] = sdot(S[k], F);
      A.M[k][i] = A.M[i][k];
    }
  }
}

// Dense inverse of the SPD matrix M by Cholesky factorisation.
static void spd_inverse(int n, real M[MAXDOF][MAXDOF], real Minv[MAXDOF][MAXDOF]) {
  real L[MAXDOF][MAXDOF];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) L[i][j] = 0;
  for (int j = 0; j < n; ++j) {
    real s = M[j][j];
    for (int k = 0; k < j; ++k) s -= L[j][k] * L[j][k];
    L[j][j] = Sqrt(s);
    for (int i = j + 1; i < n; ++i) {
      real t = M[i][j];
      for (int k = 0; k < j; ++k) t -= L[i][k] * L[j][k];
      L[i][j] = t / L[j][j];
    }
  }
  for (int c = 0; c < n; ++c) {  // solve L L^T x = e_c
    real y[MAXDOF], x[MAXDOF];
    for (int i = 0; i < n; ++i) {
      real s = (i == c) ? real(1) : real(0);
      for (int k = 0; k < i; ++k) s -= L[i][k] * y[k];
      y[i] = s / L[i][i];
    }
    for (int i = n - 1; i >= 0; --i) {
      real s = y[i];
      for (int k = i + 1; k < n; ++k) s -= L[k][i] * x[k];
      x[i] = s / L[i][i];
    }
    for (int i = 0; i < n; ++i) Minv[i][c] = x[i];
  }
}

// ---------------------------------------------------------------------------
// 3. Collision.  Colliders of an env, in index order: free objects, articulation
//    links (articulation order, joint order), articulation base boxes, static
//    boxes, ground plane.  Dynamic colliders (objects, links) precede static
//    ones, so in a pair (a < b) a dynamic body is always A.
// ---------------------------------------------------------------------------
enum { CK_OBJ = 0, CK_LINK, CK_BASE, CK_STATIC, CK_PLANE };
struct Coll {
  int kind, shape, idx, joint;
  V3 x; M3 R; V3 half; real mu;
  int node;     // colouring node (-1 static)
  V3 lo, hi;    // AABB (unfattened)
};

static void build_colliders(Env& E, std::vector<Coll>& C, real plane_mu) {
  C.clear();
  for (size_t i = 0; i < E.obj.size(); ++i) {
    Coll c; c.kind = CK_OBJ; c.shape = E.obj[i].shape; c.idx = (int)i; c.joint = -1;
    c.x = E.obj[i].x; c.R = quat_to_mat(E.obj[i].q); c.half = E.obj[i].half; c.mu = E.obj[i].mu; c.node = (int)i;
    C.push_back(c);
  }
  for (size_t k = 0; k < E.art.size(); ++k)
    for (size_t i = 0; i < E.art[k].j.size(); ++i) {
      Coll c; c.kind = CK_LINK; c.shape = SHAPE_BOX; c.idx = (int)k; c.joint = (int)i;
      c.x = E.art[k].c[i]; c.R = E.art[k].R[i]; c.half = E.art[k].j[i].half; c.mu = E.art[k].j[i].mu;
      c.node = (int)E.obj.size() + (int)k;
      C.push_back(c);
    }
  for (size_t k = 0; k < E.art.size(); ++k)
    if (E.art[k].has_bc) {
      const Art& A = E.art[k];
      M3 Rb = quat_to_mat(A.base_q);
      Coll c; c.kind = CK_BASE; c.shape = SHAPE_BOX; c.idx = (int)k; c.joint = -1;
      c.x = A.base_x + mv(Rb, A.bc_off); c.R = Rb; c.half = A.bc_half; c.mu = 0.5; c.node = -1;
      C.push_back(c);
    }
  for (size_t s = 0; s < E.st.size(); ++s) {
    Coll c; c.kind = CK_STATIC; c.shape = SHAPE_BOX; c.idx = (int)s; c.joint = -1;
    c.x = E.st[s].x; c.R = quat_to_mat(E.st[s].q); c.half = E.st[s].half; c.mu = E.st[s].mu; c.node = -1;
    C.push_back(c);
  }
  if (E.plane) {
    Coll c; c.kind = CK_PLANE; c.shape = SHAPE_PLANE; c.idx = 0; c.joint = -1; c.mu = plane_mu; c.node = -1;
    C.push_back(c);
  }
  for (auto& c : C) {
    if (c.shape == SHAPE_SPHERE) {
      c.lo = c.x - V3(c.half.x, c.half.x, c.half.x);
      c.hi = c.x + V3(c.half.x, c.half.x, c.half.x);
    } else if (c.shape == SHAPE_BOX) {
      V3 e;
      for (int r = 0; r < 3; ++r)
        e[r] = Fabs(c.R.m[r][0]) * c.half.x + Fabs(c.R.m[r][1]) * c.half.y + Fabs(c.R.m[r][2]) * c.half.z;
      c.lo = c.x - e; c.hi = c.x + e;
    }
  }
}

static bool is_dynamic(const Coll& c) { return c.kind == CK_OBJ || c.kind == CK_LINK; }

// Candidate pair test: static-static and same-articulation pairs are never
// candidates; otherwise AABBs fattened by margin/2 on every side must overlap.
static bool aabb_candidate(const Coll& a, const Coll& b, real margin) {
  if (!is_dynamic(a) && !is_dynamic(b)) return false;
  bool a_art = a.kind == CK_LINK || a.kind == CK_BASE, b_art = b.kind == CK_LINK || b.kind == CK_BASE;
  if (a_art && b_art && a.idx == b.idx) return false;
  real h = margin / 2;
  if (b.shape == SHAPE_PLANE) return a.lo.z - h <= h;
  if (a.shape == SHAPE_PLANE) return b.lo.z - h <= h;
  for (int r = 0; r < 3; ++r)
    if (a.lo[r] - h > b.hi[r] + h || b.lo[r] - h > a.hi[r] + h) return false;
  return true;
}

struct RawContact { V3 p, n; real sep; int f; };

static V3 box_vertex(const Coll& c, int k) {
  V3 l((k & 1) ? c.half.x : -c.half.x, (k & 2) ? c.half.y : -c.half.y, (k & 4) ? c.half.z : -c.half.z);
  return c.x + mv(c.R, l);
}

// Index of the first element whose value is within tol of the best one
// (largest if maximise, smallest otherwise), skipping excluded entries.
static int first_within(const std::vector<real>& val, const std::vector<int>& excluded, real tol, bool maximise) {
  int best = -1;
  for (size_t i = 0; i < val.size(); ++i) {
    if (excluded[i]) continue;
    if (best < 0 || (maximise ? val[i] > val[best] : val[i] < val[best])) best = (int)i;
  }
  if (best < 0) return -1;
  for (size_t i = 0; i < val.size(); ++i) {
    if (excluded[i]) continue;
    if (maximise ? val[i] >= val[best] - tol : val[i] <= val[best] + tol) return (int)i;
  }
  return best;
}

// Reduce a manifold (ascending feature order) to at most four points: deepest,
// farthest from it, largest triangle, largest quadrilateral; near-ties go to
// the lower feature id.
static void reduce_manifold(std::vector<RawContact>& pts) {
  if (pts.size() <= 4) return;
  std::sort(pts.begin(), pts.end(), [](const RawContact& a, const RawContact& b) { return a.f < b.f; });
  size_t n = pts.size();
  std::vector<int> ex(n, 0);
  std::vector<real> val(n);
  for (size_t i = 0; i < n; ++i) val[i] = pts[i].sep;
  int i1 = first_within(val, ex, 1e-5, false);
  ex[i1] = 1;
  for (size_t i = 0; i < n; ++i) val[i] = norm(pts[i].p - pts[i1].p);
  int i2 = first_within(val, ex, 1e-5, true);
  ex[i2] = 1;
  V3 p1 = pts[i1].p, p2 = pts[i2].p;
  for (size_t i = 0; i < n; ++i) val[i] = norm(cross(p2 - p1, pts[i].p - p1));
  int i3 = first_within(val, ex, 1e-6, true);
  ex[i3] = 1;
  V3 p3 = pts[i3].p;
  for (size_t i = 0; i < n; ++i) {
    V3 p = pts[i].p;
    val[i] = norm(cross(p - p1, p2 - p1)) + norm(cross(p - p2, p3 - p2)) + norm(cross(p - p3, p1 - p3));
  }
  int i4 = first_within(val, ex, 1e-6, true);
  std::vector<RawContact> out;
  for (size_t i = 0; i < n; ++i)
    if ((int)i == i1 || (int)i == i2 || (int)i == i3 || (int)i == i4) out.push_back(pts[i]);
  pts = out;
}

// Sphere (centre s, radius r) against a box: normal from box to sphere,
// separation, and the witness point on the box.
static void sphere_box_raw(V3 s, real r, const Coll& box, V3& n, real& sep, V3& pbox) {
  V3 l = mtv(box.R, s - box.x);
  V3 q(Max(-box.half.x, Min(box.half.x, l.x)), Max(-box.half.y, Min(box.half.y, l.y)), Max(-box.half.z, Min(box.half.z, l.z)));
  bool inside = (q.x == l.x) && (q.y == l.y) && (q.z == l.z);
  if (!inside) {
    V3 pw = box.x + mv(box.R, q);
    V3 d = s - pw;
    real dist = norm(d);
    n = d * (real(1) / dist);
    sep = dist - r;
    pbox = pw;
  } else {
    int k = 0;
    real best = box.half[0] - Fabs(l[0]);
    for (int i = 1; i < 3; ++i) {
      real d = box.half[i] - Fabs(l[i]);
      if (d < best) { best = d; k = i; }
    }
    real sg = l[k] < 0 ? real(-1) : real(1);
    n = col(box.R, k) * sg;
    sep = -best - r;
    pbox = s + n * best;
  }
}

// SAT separation of boxes a, b along unit axis u.
static real sat_sep(const Coll& a, const Coll& b, V3 u) {
  real ra = 0, rb = 0;
  for (int k = 0; k < 3; ++k) {
    ra += a.half[k] * Fabs(dot(u, col(a.R, k)));
    rb += b.half[k] * Fabs(dot(u, col(b.R, k)));
  }
  return Fabs(dot(u, a.x - b.x)) - ra - rb;
}

struct PolyV { V3 p; int id; int carrier; };

// Box-box: 15-axis SAT (Gottschalk, Lin & Manocha, OBBTree, SIGGRAPH 1996;
// Ericson, Real-Time Collision Detection 2005, 4.4) then, for a face axis,
// Sutherland-Hodgman clipping (Sutherland & Hodgman, CACM 1974) of the
// incident face against the reference face's side planes.
static void box_box(const Coll& A, const Coll& B, real margin, std::vector<RawContact>& out) {
  // face axes: B0 B1 B2 A0 A1 A2
  real fsep[6];
  for (int k = 0; k < 3; ++k) {
    fsep[k] = sat_sep(A, B, col(B.R, k));
    fsep[3 + k] = sat_sep(A, B, col(A.R, k));
  }
  real fmax = fsep[0];
  for (int k = 1; k < 6; ++k) fmax = Max(fmax, fsep[k]);
  int face = 0;
  for (int k = 0; k < 6; ++k)
    if (fsep[k] >= fmax - real(1e-4)) { face = k; break; }
  // edge axes
  real emax = -1e30;
  int nvalid = 0;
  real esep[9];
  int evalid[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      V3 u = cross(col(A.R, i), col(B.R, j));
      real len = norm(u);
      evalid[3 * i + j] = len >= real(1e-3);
      if (!evalid[3 * i + j]) { esep[3 * i + j] = -1e30; continue; }
      esep[3 * i + j] = sat_sep(A, B, u * (real(1) / len));
      if (nvalid == 0 || esep[3 * i + j] > emax) emax = esep[3 * i + j];
      ++nvalid;
    }
  bool use_edge = nvalid > 0 && emax > fmax + real(1e-3);
  if (use_edge) {
    if (emax > margin) return;
    int e = -1;
    for (int k = 0; k < 9; ++k)
      if (evalid[k] && esep[k] >= emax - real(1e-4)) { e = k; break; }
    int i = e / 3, j = e % 3;
    V3 ua = col(A.R, i), ub = col(B.R, j);
    V3 L = cross(ua, ub);
    L = L * (real(1) / norm(L));
    if (dot(L, A.x - B.x) < 0) L = -L;
    V3 pa = A.x, pb = B.x;
    for (int k = 0; k < 3; ++k) {
      if (k != i) pa = pa + col(A.R, k) * (A.half[k] * (dot(L, col(A.R, k)) > 0 ? real(-1) : real(1)));
      if (k != j) pb = pb + col(B.R, k) * (B.half[k] * (dot(L, col(B.R, k)) < 0 ? real(-1) : real(1)));
    }
    V3 r = pa - pb;
    real bb = dot(ua, ub), c = dot(ua, r), f = dot(ub, r);
    real den = 1 - bb * bb;
    real s = (bb * f - c) / den;
    real t = f + s * bb;
    s = Max(-A.half[i], Min(A.half[i], s));
    t = Max(-B.half[j], Min(B.half[j], t));
    V3 qa = pa + ua * s, qb = pb + ub * t;
    RawContact rc;
    rc.p = (qa + qb) * real(0.5);
    rc.n = L;
    rc.sep = esep[e];
    rc.f = 1024 + e;
    out.push_back(rc);
    return;
  }
  if (fmax > margin) return;
  bool refB = face < 3;
  int k = face % 3;
  const Coll& R = refB ? B : A;
  const Coll& I = refB ? A : B;
  V3 u = col(R.R, k);
  bool neg = dot(u, I.x - R.x) < 0;
  V3 nref = neg ? -u : u;
  V3 fc = R.x + nref * R.half[k];
  int k1 = k == 0 ? 1 : 0, k2 = k == 2 ? 1 : 2;
  V3 t1 = col(R.R, k1), t2 = col(R.R, k2);
  real e1 = R.half[k1], e2 = R.half[k2];
  // incident face: axis of I most parallel to nref, facing against it
  int m = 0;
  real best = Fabs(dot(col(I.R, 0), nref));
  for (int q = 1; q < 3; ++q) {
    real d = Fabs(dot(col(I.R, q), nref));
    if (d > best) { best = d; m = q; }
  }
  real sg = dot(col(I.R, m), nref) > 0 ? real(-1) : real(1);
  V3 ic = I.x + col(I.R, m) * (sg * I.half[m]);
  int m1 = m == 0 ? 1 : 0, m2 = m == 2 ? 1 : 2;
  V3 w1 = col(I.R, m1) * I.half[m1], w2 = col(I.R, m2) * I.half[m2];
  std::vector<PolyV> poly(4);
  poly[0].p = ic - w1 - w2; poly[1].p = ic + w1 - w2; poly[2].p = ic + w1 + w2; poly[3].p = ic - w1 + w2;
  for (int v = 0; v < 4; ++v) { poly[v].id = v; poly[v].carrier = (v + 3) % 4; }
  for (int s = 0; s < 4; ++s) {
    V3 dir = (s < 2) ? t1 : t2;
    real sgn = (s % 2 == 0) ? real(1) : real(-1);
    real ext = (s < 2) ? e1 : e2;
    std::vector<PolyV> np;
    size_t cnt = poly.size();
    for (size_t q = 0; q < cnt; ++q) {
      const PolyV& P = poly[(q + cnt - 1) % cnt];
      const PolyV& Q = poly[q];
      real dP = sgn * dot(dir, P.p - fc) - ext;
      real dQ = sgn * dot(dir, Q.p - fc) - ext;
      int c = Q.carrier;
      bool pin = dP <= 0, qin = dQ <= 0;
      if (pin != qin) {
        PolyV X;
        X.p = P.p + (Q.p - P.p) * (dP / (dP - dQ));
        X.id = c < 4 ? 4 + 4 * c + s : 20 + 4 * (c - 4) + s;
        X.carrier = qin ? 4 + s : c;
        np.push_back(X);
      }
      if (qin) np.push_back(Q);
    }
    poly = np;
    if (poly.empty()) break;
  }
  int ref_code = (refB ? 0 : 6) + 2 * k + (neg ? 1 : 0);
  std::vector<RawContact> pts;
  for (auto& P : poly) {
    real sep = dot(nref, P.p - fc);
    if (sep > margin) continue;
    RawContact rc;
    rc.p = P.p - nref * (sep * real(0.5));
    rc.n = refB ? nref : -nref;
    rc.sep = sep;
    rc.f = ref_code * 64 + P.id;
    pts.push_back(rc);
  }
  reduce_manifold(pts);
  std::sort(pts.begin(), pts.end(), [](const RawContact& a, const RawContact& b) { return a.f < b.f; });
  for (auto& p : pts) out.push_back(p);
}

// Contacts of the pair (A, B), normals from B to A, ascending feature ids.
static void narrowphase(const Coll& A, const Coll& B, real margin, std::vector<RawContact>& out) {
  out.clear();
  if (B.shape == SHAPE_PLANE) {
    if (A.shape == SHAPE_SPHERE) {
      real r = A.half.x;
      real sep = A.x.z - r;
      if (sep > margin) return;
      RawContact rc; rc.p = V3(A.x.x, A.x.y, (A.x.z - r) * real(0.5)); rc.n = V3(0, 0, 1); rc.sep = sep; rc.f = 0;
      out.push_back(rc);
    } else {
      std::vector<RawContact> pts;
      for (int k = 0; k < 8; ++k) {
        V3 v = box_vertex(A, k);
        if (v.z > margin) continue;
        RawContact rc; rc.p = V3(v.x, v.y, v.z * real(0.5)); rc.n = V3(0, 0, 1); rc.sep = v.z; rc.f = k;
        pts.push_back(rc);
      }
      reduce_manifold(pts);
      for (auto& p : pts) out.push_back(p);
    }
    return;
  }
  if (A.shape == SHAPE_SPHERE && B.shape == SHAPE_SPHERE) {
    V3 d = A.x - B.x;
    real dist = norm(d);
    V3 n = dist > real(1e-12) ? d * (real(1) / dist) : V3(0, 0, 1);
    real sep = dist - A.half.x - B.half.x;
    if (sep > margin) return;
    V3 pa = A.x - n * A.half.x, pb = B.x + n * B.half.x;
    RawContact rc; rc.p = (pa + pb) * real(0.5); rc.n = n; rc.sep = sep; rc.f = 0;
    out.push_back(rc);
    return;
  }
  if (A.shape == SHAPE_SPHERE || B.shape == SHAPE_SPHERE) {
    const Coll& S = A.shape == SHAPE_SPHERE ? A : B;
    const Coll& X = A.shape == SHAPE_SPHERE ? B : A;
    V3 n; real sep; V3 pb;
    sphere_box_raw(S.x, S.half.x, X, n, sep, pb);
    if (sep > margin) return;
    V3 ps = S.x - n * S.half.x;
    RawContact rc; rc.p = (pb + ps) * real(0.5); rc.n = (A.shape == SHAPE_SPHERE) ? n : -n; rc.sep = sep; rc.f = 0;
    out.push_back(rc);
    return;
  }
  box_box(A, B, margin, out);
}

// ---------------------------------------------------------------------------
// 4-5. Rows and projected Gauss-Seidel (sequential impulses: Catto, "Iterative
//      Dynamics with Temporal Coherence", GDC 2005).
// ---------------------------------------------------------------------------
struct EndPt {
  int type;   // 0 static, 1 free object, 2 articulation
  int idx;    // object index or articulation index
  V3 r;       // free: contact point minus centre of mass
  real j[3][MAXDOF], w[3][MAXDOF];  // articulation: generalised Jacobian / M^-1 j^T for n, t1, t2
};
struct Unit {
  int is_limit;  // 0 contact, 1 joint limit, 2 joint motor
  int node_a, node_b;
  // contact
  int contact;
  EndPt ea, eb;
  V3 d[3];
  real meff[3], target, mu, lam[3];
  // limit / motor
  int art, joint; real lsign, bound;
};

struct Dyn {  // velocity state during the solve
  std::vector<V3> v, w;
  std::vector<M3> Iinv;
  std::vector<std::vector<real>> qd;
};

static real endpoint_vel(const Env& E, const Dyn& S, const EndPt& e, int row, V3 d) {
  if (e.type == 1) return dot(d, S.v[e.idx] + cross(S.w[e.idx], e.r));
  if (e.type == 2) {
    real s = 0;
    int n = (int)E.art[e.idx].j.size();
    for (int i = 0; i < n; ++i) s += e.j[row][i] * S.qd[e.idx][i];
    return s;
  }
  return 0;
}
static void endpoint_apply(const Env& E, Dyn& S, const EndPt& e, int row, V3 d, real imp) {
  if (e.type == 1) {
    const Obj& o = E.obj[e.idx];
    S.v[e.idx] = S.v[e.idx] + d * (o.inv_mass * imp);
    S.w[e.idx] = S.w[e.idx] + mv(S.Iinv[e.idx], cross(e.r, d)) * imp;
  } else if (e.type == 2) {
    int n = (int)E.art[e.idx].j.size();
    for (int i = 0; i < n; ++i) S.qd[e.idx][i] += e.w[row][i] * imp;
  }
}
static real endpoint_k(const Env& E, const Dyn& S, const EndPt& e, int row, V3 d) {
  if (e.type == 1) {
    V3 rd = cross(e.r, d);
    return E.obj[e.idx].inv_mass + dot(rd, mv(S.Iinv[e.idx], rd));
  }
  if (e.type == 2) {
    real s = 0;
    int n = (int)E.art[e.idx].j.size();
    for (int i = 0; i < n; ++i) s += e.j[row][i] * e.w[row][i];
    return s;
  }
  return 0;
}
static void endpoint_setup(const Env& E, const Dyn& S, const Coll& c, V3 p, V3 d[3], EndPt& e) {
  (void)S;
  if (c.kind == CK_OBJ) {
    e.type = 1; e.idx = c.idx; e.r = p - E.obj[c.idx].x;
  } else if (c.kind == CK_LINK) {
    e.type = 2; e.idx = c.idx;
    const Art& A = E.art[c.idx];
    int n = (int)A.j.size();
    for (int row = 0; row < 3; ++row) {
      for (int i = 0; i < n; ++i) e.j[row][i] = 0;
      // ancestors of the touched link (inclusive) move the point
      for (int i = c.joint; i >= 0; i = A.j[i].parent) {
        V3 sp = A.j[i].type == JT_REV ? cross(A.ja[i], p - A.jo[i]) : A.ja[i];
        e.j[row][i] = dot(d[row], sp);
      }
      for (int i = 0; i < n; ++i) {
        real s = 0;
        for (int k = 0; k < n; ++k) s += A.Minv[i][k] * e.j[row][k];
        e.w[row][i] = s;
      }
    }
  } else {
    e.type = 0; e.idx = -1;
  }
}

static void tangent_basis(V3 n, V3& t1, V3& t2) {
  V3 e = Fabs(n.x) < real(0.57735) ? V3(1, 0, 0) : V3(0, 1, 0);
  t1 = cross(n, e);
  t1 = t1 * (real(1) / norm(t1));
  t2 = cross(n, t1);
}

static void unit_apply(const Env& E, Dyn& S, const Unit& u, int row, real imp) {
  if (u.is_limit) {
    const Art& A = E.art[u.art];
    int n = (int)A.j.size();
    for (int i = 0; i < n; ++i) S.qd[u.art][i] += A.Minv[i][u.joint] * u.lsign * imp;
    return;
  }
  endpoint_apply(E, S, u.ea, row, u.d[row], imp);
  endpoint_apply(E, S, u.eb, row, u.d[row], -imp);
}
static real unit_vel(const Env& E, const Dyn& S, const Unit& u, int row) {
  if (u.is_limit) return u.lsign * S.qd[u.art][u.joint];
  return endpoint_vel(E, S, u.ea, row, u.d[row]) - endpoint_vel(E, S, u.eb, row, u.d[row]);
}

// ---------------------------------------------------------------------------
// Learned warm start network (FP64): 32 -> 128 -> 128 -> 128 -> 3, GELU (erf
// form).  Parameter layout: W1[128][32], b1[128], W2[128][128], b2[128],
// W3[128][128], b3[128], W4[3][128], b4[3]  (row-major, out x in).
// ---------------------------------------------------------------------------
static const int MLP_IN = 32, MLP_H = 128, MLP_OUT = 3;
// The deployed network's output is limited to the range of its training targets
// (impulse corrections clipped to +-10 units of m_eff,n |g| dt): beyond it the
// network extrapolates, and on a contact with a large effective mass an
// extrapolated correction is an impulse that a fixed number of sweeps cannot undo.
static const double MLP_OUT_LIMIT = 10.0;
// Unit of the learned warm start's impulses for one contact: its normal effective mass
// times the velocity change the step can ask of it -- the free-fall increment |g| dt
// plus the size of the contact's relative velocity before the solve (features 9-11).
// A resting contact needs about one |g| dt, an impact about its approach speed, so the
// targets stay of order one in both regimes.
static real learn_scale(const real* f, V3 g, real dt) {
  return f[18] * (norm(g) * dt + Sqrt(f[9] * f[9] + f[10] * f[10] + f[11] * f[11]));
}
// The contacts the network starts: those without a prior-frame match, and the matched
// ones whose relative velocity exceeds LEARN_GATE |g| dt (impacts, sliding, contacts
// pushed by the arm).  Persistent resting contacts keep their prior-frame impulse,
// which is already their converged value up to the step's small changes.
static const double LEARN_GATE = 4.0;
static bool learn_uses(const real* f, V3 g, real dt) {
  if (f[26] == real(0)) return true;
  return Sqrt(f[9] * f[9] + f[10] * f[10] + f[11] * f[11]) > real(LEARN_GATE) * norm(g) * dt;
}
static const int MLP_NPARAM = 128 * 32 + 128 + 128 * 128 + 128 + 128 * 128 + 128 + 3 * 128 + 3;
static real gelu(real x) { return real(0.5) * x * (real(1) + Erf(x * real(0.70710678118654752440))); }
static real gelu_grad(real x) {
  return real(0.5) * (real(1) + Erf(x * real(0.70710678118654752440))) +
         x * Exp(real(-0.5) * x * x) * real(0.39894228040143267794);
}
static void mlp_layer_offsets(int off[8]) {
  off[0] = 0;                      // W1
  off[1] = off[0] + 128 * 32;      // b1
  off[2] = off[1] + 128;           // W2
  off[3] = off[2] + 128 * 128;     // b2
  off[4] = off[3] + 128;           // W3
  off[5] = off[4] + 128 * 128;     // b3
  off[6] = off[5] + 128;           // W4
  off[7] = off[6] + 3 * 128;       // b4
}
// Forward one sample; keeps the pre-activations for backward.
static void mlp_forward1(const double* P, const real* x, real z[3][128], real h[3][128], real* y) {
  int off[8];
  mlp_layer_offsets(off);
  const real* in = x;
  int nin = MLP_IN;
  for (int l = 0; l < 3; ++l) {
    const double* W = P + off[2 * l];
    const double* b = P + off[2 * l + 1];
    for (int o = 0; o < MLP_H; ++o) {
      real s = b[o];
      for (int i = 0; i < nin; ++i) s += real(W[o * nin + i]) * in[i];
      z[l][o] = s;
      h[l][o] = gelu(s);
    }
    in = h[l];
    nin = MLP_H;
  }
  for (int o = 0; o < MLP_OUT; ++o) {
    real s = P[off[7] + o];
    for (int i = 0; i < MLP_H; ++i) s += real(P[off[6] + o * MLP_H + i]) * h[2][i];
    y[o] = s;
  }
}

// Per-contact features of the learned warm start (32 values).
static void contact_features(const Env& E, const Dyn& S, const Coll& ca, const Coll& cb, const Contact& c,
                             const Unit& u, real prev[3], int matched, V3 g, real dt, real* f) {
  int k = 0;
  f[k++] = c.n.x; f[k++] = c.n.y; f[k++] = c.n.z;
  V3 xa = ca.kind == CK_OBJ ? E.obj[ca.idx].x : ca.x;
  V3 xb = cb.kind == CK_OBJ ? E.obj[cb.idx].x : (cb.shape == SHAPE_PLANE ? V3(c.p.x, c.p.y, 0) : cb.x);
  V3 ra = c.p - xa, rb = c.p - xb;
  f[k++] = ra.x; f[k++] = ra.y; f[k++] = ra.z;
  f[k++] = rb.x; f[k++] = rb.y; f[k++] = rb.z;
  for (int r = 0; r < 3; ++r) f[k++] = unit_vel(E, S, u, r);
  V3 wa = ca.kind == CK_OBJ ? S.w[ca.idx] : V3(0, 0, 0);
  V3 wb = cb.kind == CK_OBJ ? S.w[cb.idx] : V3(0, 0, 0);
  V3 wr = wa - wb;
  f[k++] = wr.x; f[k++] = wr.y; f[k++] = wr.z;
  f[k++] = c.sep;
  f[k++] = ca.kind == CK_OBJ ? E.obj[ca.idx].inv_mass : real(0);
  f[k++] = cb.kind == CK_OBJ ? E.obj[cb.idx].inv_mass : real(0);
  for (int r = 0; r < 3; ++r) f[k++] = u.meff[r];
  f[k++] = u.mu;
  f[k++] = dot(g, c.n) * dt;
  for (int r = 0; r < 3; ++r) f[k++] = prev[r];
  f[k++] = matched ? real(1) : real(0);
  int type;  // 0 sphere-sphere, 1 sphere-plane, 2 sphere-box, 3 box-plane, 4 box-box
  if (ca.shape == SHAPE_SPHERE && cb.shape == SHAPE_SPHERE) type = 0;
  else if (cb.shape == SHAPE_PLANE) type = ca.shape == SHAPE_SPHERE ? 1 : 3;
  else if (ca.shape == SHAPE_SPHERE || cb.shape == SHAPE_SPHERE) type = 2;
  else type = 4;
  for (int t = 0; t < 5; ++t) f[k++] = t == type ? real(1) : real(0);
}

// ---------------------------------------------------------------------------
// One step of one environment.
// ---------------------------------------------------------------------------
struct StepLog {  // optional per-step log of (features, converged impulses)
  std::vector<double>* feats;
  std::vector<double>* lams;
};

static void env_step(World& W, Env& E, StepLog* log) {
  const OrParams& P = W.P;
  real dt = P.dt;
  V3 g(P.gravity[0], P.gravity[1], P.gravity[2]);
  E.status = 0;

  // 1. articulations at q_t
  g_stage = ST_ABA;
  for (auto& A : E.art) {
    int n = (int)A.j.size();
    A.motor = P.motor_mode && A.kinematic;
    art_fk(A);
    real tau[MAXDOF];
    for (int i = 0; i < n; ++i) tau[i] = tau_of(A, i, dt);
    art_aba(A, g, dt, tau, A.qdd);
    for (int i = 0; i < n; ++i) A.qd_star[i] = A.j[i].qd + dt * A.qdd[i];
    art_crba(A, dt);
    spd_inverse(n, A.M, A.Minv);
  }
  // 2. free bodies
  g_stage = ST_PREDICT;
  Dyn S;
  S.v.resize(E.obj.size()); S.w.resize(E.obj.size()); S.Iinv.resize(E.obj.size());
  for (size_t i = 0; i < E.obj.size(); ++i) {
    Obj& o = E.obj[i];
    if (o.awake) { S.v[i] = o.v + g * dt; S.w[i] = o.w; }
    else { S.v[i] = V3(0, 0, 0); S.w[i] = V3(0, 0, 0); }
    S.Iinv[i] = rot_diag(quat_to_mat(o.q), o.inv_I);
  }
  S.qd.resize(E.art.size());
  for (size_t k = 0; k < E.art.size(); ++k) {
    S.qd[k].assign(E.art[k].j.size(), 0);
    for (size_t i = 0; i < E.art[k].j.size(); ++i) S.qd[k][i] = E.art[k].qd_star[i];
  }

  // 3. collision
  g_stage = ST_COLLIDE;
  std::vector<Coll> C;
  build_colliders(E, C, P.plane_mu);
  int nc = (int)C.size();
  std::vector<std::pair<int, int>> cand;
  for (int a = 0; a < nc; ++a)
    for (int b = a + 1; b < nc; ++b)
      if (aabb_candidate(C[a], C[b], P.margin)) cand.push_back(std::make_pair(a, b));
  auto awake_dyn = [&](int c) {
    if (C[c].kind == CK_LINK) return true;
    if (C[c].kind == CK_OBJ) return E.obj[C[c].idx].awake != 0;
    return false;
  };
  if (P.sleep_enabled) {  // wake pass, ascending pair order, state updated in place
    for (auto& pr : cand) {
      int a = pr.first, b = pr.second;
      bool sa = C[a].kind == CK_OBJ && !E.obj[C[a].idx].awake;
      bool sb = C[b].kind == CK_OBJ && !E.obj[C[b].idx].awake;
      if (sa && awake_dyn(b)) { E.obj[C[a].idx].awake = 1; E.obj[C[a].idx].ctr = 0; }
      else if (sb && awake_dyn(a)) { E.obj[C[b].idx].awake = 1; E.obj[C[b].idx].ctr = 0; }
    }
  }
  E.pairs.clear();
  E.contacts.clear();
  std::vector<std::pair<int, int>> cpair;  // collider indices per contact
  std::vector<RawContact> raw;
  for (auto& pr : cand) {
    int a = pr.first, b = pr.second;
    if (!awake_dyn(a) && !awake_dyn(b)) continue;
    E.pairs.push_back(a * 4096 + b);
    narrowphase(C[a], C[b], P.margin, raw);
    for (auto& r : raw) {
      if ((int)E.contacts.size() >= P.max_contacts) { E.status |= STATUS_OVERFLOW; break; }
      Contact c; c.a = a; c.b = b; c.f = r.f; c.p = r.p; c.n = r.n; c.sep = r.sep;
      c.lam[0] = c.lam[1] = c.lam[2] = 0;
      E.contacts.push_back(c);
      cpair.push_back(pr);
    }
  }

  // 4. rows
  g_stage = ST_ROWS;
  std::vector<Unit> units;
  for (size_t ci = 0; ci < E.contacts.size(); ++ci) {
    Contact& c = E.contacts[ci];
    const Coll& ca = C[c.a];
    const Coll& cb = C[c.b];
    Unit u;
    u.is_limit = 0; u.contact = (int)ci; u.node_a = ca.node; u.node_b = cb.node;
    u.d[0] = c.n;
    tangent_basis(c.n, u.d[1], u.d[2]);
    endpoint_setup(E, S, ca, c.p, u.d, u.ea);
    endpoint_setup(E, S, cb, c.p, u.d, u.eb);
    for (int r = 0; r < 3; ++r) {  // a row that cannot change the relative velocity gets no impulse
      real K = endpoint_k(E, S, u.ea, r, u.d[r]) + endpoint_k(E, S, u.eb, r, u.d[r]);
      u.meff[r] = K > real(1e-6) ? real(1) / K : real(0);
    }
    u.mu = Sqrt(ca.mu * cb.mu);
    real vn = unit_vel(E, S, u, 0);
    real tgt;
    if (c.sep > 0) tgt = -c.sep / dt;
    else if (c.sep > -P.slop) tgt = 0;
    else tgt = -P.baumgarte * (c.sep + P.slop) / dt;
    real e = Max(ca.kind == CK_OBJ ? E.obj[ca.idx].rest : real(0), cb.kind == CK_OBJ ? E.obj[cb.idx].rest : real(0));
    if (vn < -P.rest_thresh) tgt = Max(tgt, -e * vn);
    u.target = tgt;
    u.lam[0] = u.lam[1] = u.lam[2] = 0;
    units.push_back(u);
  }
  int n_contact_units = (int)units.size();
  for (size_t k = 0; k < E.art.size(); ++k) {
    Art& A = E.art[k];
    for (size_t i = 0; i < A.j.size(); ++i) {
      Joint& J = A.j[i];
      int side = 0;
      if (J.has_limit) {
        real qp = J.q + dt * A.qd_star[i];
        if (qp < J.lo) side = 1;
        else if (qp > J.hi) side = 2;
      }
      if (!side) continue;
      Unit u;
      u.is_limit = 1; u.contact = -1; u.art = (int)k; u.joint = (int)i;
      u.node_a = (int)E.obj.size() + (int)k; u.node_b = -1;
      u.lsign = side == 1 ? real(1) : real(-1);
      u.meff[0] = real(1) / A.Minv[i][i];
      // distance to the limit: reach it exactly within the step when not yet
      // violated, push back at the Baumgarte rate when violated
      real cgap = side == 1 ? J.q - J.lo : J.hi - J.q;
      u.target = cgap >= 0 ? -cgap / dt : -P.baumgarte * cgap / dt;
      u.lam[0] = u.lam[1] = u.lam[2] = 0;
      u.mu = 0;
      units.push_back(u);
    }
  }
  // joint motors (motor mode, the paper's Sec. 5.1 "Action space"): per joint of a
  // kinematic-base articulation a row on q̇_i with target rate motor_kp (q̄ - q) / dt
  // and impulse bounded by motor_max_impulse in either direction
  for (size_t k = 0; k < E.art.size(); ++k) {
    Art& A = E.art[k];
    if (!A.motor) continue;
    for (size_t i = 0; i < A.j.size(); ++i) {
      Joint& J = A.j[i];
      Unit u;
      u.is_limit = 2; u.contact = -1; u.art = (int)k; u.joint = (int)i;
      u.node_a = (int)E.obj.size() + (int)k; u.node_b = -1;
      u.lsign = 1;
      u.meff[0] = real(1) / A.Minv[i][i];
      u.target = P.motor_kp * (J.target - J.q) / dt;
      u.bound = P.motor_max_impulse;
      u.lam[0] = u.lam[1] = u.lam[2] = 0;
      u.mu = 0;
      units.push_back(u);
    }
  }
  E.n_limit_rows = (int)units.size() - n_contact_units;
  E.n_rows = 3 * n_contact_units + E.n_limit_rows;

  // warm start
  std::vector<std::vector<real>> feats;
  if (P.warm_mode >= 1 || log) {
    for (int ui = 0; ui < n_contact_units; ++ui) {
      Unit& u = units[ui];
      const Contact& c = E.contacts[u.contact];
      real prev[3] = {0, 0, 0};
      int matched = 0;
      for (auto& ce : E.cache) {
        if (ce.a == c.a && ce.b == c.b && ce.f == c.f && norm(ce.p - c.p) < P.match_dist) {
          prev[0] = ce.ln;
          prev[1] = Max(-u.mu * ce.ln, Min(u.mu * ce.ln, dot(ce.lt, u.d[1])));
          prev[2] = Max(-u.mu * ce.ln, Min(u.mu * ce.ln, dot(ce.lt, u.d[2])));
          matched = 1;
          break;
        }
      }
      if (log || P.warm_mode == 2) {
        std::vector<real> f(MLP_IN);
        contact_features(E, S, C[c.a], C[c.b], c, u, prev, matched, g, dt, f.data());
        feats.push_back(f);
      }
      if (P.warm_mode == 1)
        for (int r = 0; r < 3; ++r) u.lam[r] = prev[r];
    }
    if (P.warm_mode == 2) {
      g_stage = ST_MLP;
      for (int ui = 0; ui < n_contact_units; ++ui) {
        Unit& u = units[ui];
        real y[3];
        bool ok = false;
        // the network predicts the correction for the contacts it serves (learn_uses);
        // the others keep their prior-frame impulse
        if (W.has_mlp && learn_uses(feats[ui].data(), g, dt)) {
          real z[3][128], h[3][128];
          mlp_forward1(W.mlp_w.data(), feats[ui].data(), z, h, y);
          ok = Finite(y[0]) && Finite(y[1]) && Finite(y[2]);
          for (int r = 0; r < 3; ++r) y[r] = Max(real(-MLP_OUT_LIMIT), Min(real(MLP_OUT_LIMIT), y[r]));
        }
        // network output (limited to +-MLP_OUT_LIMIT): correction to the prior-frame
        // impulse in units of learn_scale; the sum is projected onto the friction pyramid
        if (ok) {
          real sc = learn_scale(feats[ui].data(), g, dt);
          real ln = Max(real(0), feats[ui][23] + y[0] * sc);
          u.lam[0] = ln;
          u.lam[1] = Max(-u.mu * ln, Min(u.mu * ln, feats[ui][24] + y[1] * sc));
          u.lam[2] = Max(-u.mu * ln, Min(u.mu * ln, feats[ui][25] + y[2] * sc));
        } else {  // fall back to the prior-frame value
          for (int r = 0; r < 3; ++r) u.lam[r] = feats[ui][23 + r];
        }
      }
      g_stage = ST_ROWS;
    }
  }
  if (P.warm_mode >= 1) {  // prior-frame limit and motor impulses
    for (size_t ui = n_contact_units; ui < units.size(); ++ui) {
      Unit& u = units[ui];
      const Joint& J = E.art[u.art].j[u.joint];
      if (u.is_limit == 2) {
        u.lam[0] = J.motor_lambda;
        continue;
      }
      int side = u.lsign > 0 ? 1 : 2;
      if (J.lim_side == side) u.lam[0] = J.lim_lambda;
    }
  }
  for (auto& u : units) {
    if (u.is_limit) unit_apply(E, S, u, 0, u.lam[0]);
    else for (int r = 0; r < 3; ++r) unit_apply(E, S, u, r, u.lam[r]);
  }

  // order: shared (a, b, feature) order, or greedy colours in that order
  std::vector<int> order(units.size());
  for (size_t i = 0; i < units.size(); ++i) order[i] = (int)i;
  E.n_colours = 0;
  if (P.use_colouring) {
    int nnodes = (int)E.obj.size() + (int)E.art.size();
    std::vector<uint64_t> used(nnodes, 0);
    std::vector<int> colour(units.size());
    for (size_t i = 0; i < units.size(); ++i) {
      uint64_t m = 0;
      if (units[i].node_a >= 0) m |= used[units[i].node_a];
      if (units[i].node_b >= 0) m |= used[units[i].node_b];
      int c = 0;
      while (c < 64 && (m >> c) & 1) ++c;
      colour[i] = c;  // 64 = the serial overflow colour
      if (c < 64) {
        if (units[i].node_a >= 0) used[units[i].node_a] |= (uint64_t(1) << c);
        if (units[i].node_b >= 0) used[units[i].node_b] |= (uint64_t(1) << c);
      }
      E.n_colours = std::max(E.n_colours, c + 1);
    }
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return colour[x] < colour[y]; });
    E.unit_colour = colour;
  } else {
    E.unit_colour.clear();
  }
  E.unit_node_a.resize(units.size());
  E.unit_node_b.resize(units.size());
  for (size_t i = 0; i < units.size(); ++i) {
    E.unit_node_a[i] = units[i].node_a;
    E.unit_node_b[i] = units[i].node_b;
  }

  // 5. PGS sweeps
  g_stage = ST_PGS;
  int it = 0;
  real resid = 0;
  int max_it = P.pgs_tol > 0 ? P.pgs_max_iters : P.pgs_iters;
  if (!units.empty()) {
    for (it = 1; it <= max_it; ++it) {
      real d2 = 0, l2 = 0;
      for (int ui : order) {
        Unit& u = units[ui];
        if (u.is_limit) {
          real v = unit_vel(E, S, u, 0);
          real nl = u.is_limit == 2 ? Max(-u.bound, Min(u.bound, u.lam[0] + u.meff[0] * (u.target - v)))
                                    : Max(real(0), u.lam[0] + u.meff[0] * (u.target - v));
          real dl = nl - u.lam[0];
          unit_apply(E, S, u, 0, dl);
          u.lam[0] = nl;
          d2 += dl * dl; l2 += nl * nl;
          continue;
        }
        real v = unit_vel(E, S, u, 0);
        real nl = Max(real(0), u.lam[0] + u.meff[0] * (u.target - v));
        real dl = nl - u.lam[0];
        unit_apply(E, S, u, 0, dl);
        u.lam[0] = nl;
        d2 += dl * dl; l2 += nl * nl;
        for (int r = 1; r < 3; ++r) {
          real vt = unit_vel(E, S, u, r);
          real lim = u.mu * u.lam[0];
          real nt = Max(-lim, Min(lim, u.lam[r] - u.meff[r] * vt));
          real dt_ = nt - u.lam[r];
          unit_apply(E, S, u, r, dt_);
          u.lam[r] = nt;
          d2 += dt_ * dt_; l2 += nt * nt;
        }
      }
      resid = Sqrt(d2) / Max(Sqrt(l2), real(P.lambda_floor));
      if (P.pgs_tol > 0 && resid <= real(P.pgs_tol)) break;
    }
    if (it > max_it) {
      it = max_it;
      if (P.pgs_tol > 0) E.status |= STATUS_ITER_CAP;
    }
  } else {
    it = 0;
  }
  E.iters = it;
  E.resid = resid;

  // cache for the next step's warm start; optional training log; contact force on
  // the robot (Sec. 5.1, "Evaluation": the episode fails once the accumulated contact
  // force on the arm / body exceeds 5 kN): the normal impulses of every contact with
  // a link or the base box of a kinematic-base articulation, divided by dt
  auto robot = [&](int ci) { return (C[ci].kind == CK_LINK || C[ci].kind == CK_BASE) && E.art[C[ci].idx].kinematic; };
  real f_robot = 0;
  E.cache.clear();
  for (int ui = 0; ui < n_contact_units; ++ui) {
    Unit& u = units[ui];
    Contact& c = E.contacts[u.contact];
    for (int r = 0; r < 3; ++r) c.lam[r] = u.lam[r];
    if (robot(c.a) || robot(c.b)) f_robot += u.lam[0] / dt;
    CacheEntry ce;
    ce.a = c.a; ce.b = c.b; ce.f = c.f; ce.p = c.p; ce.ln = u.lam[0];
    ce.lt = u.d[1] * u.lam[1] + u.d[2] * u.lam[2];
    E.cache.push_back(ce);
    // logged training pair: features and (converged - prior-frame) / learn_scale, for
    // the contacts of an environment whose solve met its residual target (fixed sweep
    // counts always do) and whose targets are finite (a degenerate row has no scale)
    if (log && (P.pgs_tol <= 0 || E.resid <= real(P.pgs_tol))) {
      real sc = learn_scale(feats[ui].data(), g, dt);
      real t[3];
      bool fin = sc > real(0);
      for (int r = 0; r < 3; ++r) {
        t[r] = (u.lam[r] - feats[ui][23 + r]) / sc;
        fin = fin && Finite(t[r]);
      }
      if (fin) {
        for (int k = 0; k < MLP_IN; ++k) log->feats->push_back(D(feats[ui][k]));
        for (int r = 0; r < 3; ++r) log->lams->push_back(D(t[r]));
      }
    }
  }
  E.robot_force = f_robot;
  E.robot_force_acc += f_robot;
  if (P.force_limit > 0 && E.robot_force_acc > P.force_limit) E.status |= STATUS_FORCE;
  for (auto& A : E.art)
    for (auto& J : A.j) { J.lim_side = 0; J.lim_lambda = 0; J.motor_lambda = 0; }
  for (size_t ui = n_contact_units; ui < units.size(); ++ui) {
    Unit& u = units[ui];
    Joint& J = E.art[u.art].j[u.joint];
    if (u.is_limit == 2) {
      J.motor_lambda = u.lam[0];
      continue;
    }
    J.lim_side = u.lsign > 0 ? 1 : 2;
    J.lim_lambda = u.lam[0];
  }

  // 6. integrate and sleep
  g_stage = ST_INTEGRATE;
  for (size_t i = 0; i < E.obj.size(); ++i) {
    Obj& o = E.obj[i];
    if (!o.awake) continue;
    o.v = S.v[i];
    o.w = S.w[i];
    o.x = o.x + o.v * dt;
    real hw = real(0.5) * dt;
    Quat q = o.q;
    Quat dq;  // (0, w) (x) q
    dq.w = -(o.w.x * q.x + o.w.y * q.y + o.w.z * q.z);
    dq.x = q.w * o.w.x + (o.w.y * q.z - o.w.z * q.y);
    dq.y = q.w * o.w.y + (o.w.z * q.x - o.w.x * q.z);
    dq.z = q.w * o.w.z + (o.w.x * q.y - o.w.y * q.x);
    q.w = q.w + hw * dq.w; q.x = q.x + hw * dq.x; q.y = q.y + hw * dq.y; q.z = q.z + hw * dq.z;
    real qn = Sqrt(q.w * q.w + q.x * q.x + q.y * q.y + q.z * q.z);
    o.q.w = q.w / qn; o.q.x = q.x / qn; o.q.y = q.y / qn; o.q.z = q.z / qn;
    if (P.sleep_enabled) {
      if (norm(o.v) < real(P.sleep_lin) && norm(o.w) < real(P.sleep_ang)) o.ctr += 1;
      else o.ctr = 0;
      if (o.ctr >= P.sleep_steps) { o.awake = 0; o.v = V3(0, 0, 0); o.w = V3(0, 0, 0); }
    }
  }
  for (size_t k = 0; k < E.art.size(); ++k) {
    Art& A = E.art[k];
    for (size_t i = 0; i < A.j.size(); ++i) {
      A.j[i].qd = S.qd[k][i];
      A.j[i].q = A.j[i].q + dt * A.j[i].qd;
    }
  }
  bool bad = false;
  for (auto& o : E.obj)
    bad |= !(Finite(o.x.x) && Finite(o.x.y) && Finite(o.x.z) && Finite(o.v.x) && Finite(o.v.y) && Finite(o.v.z) &&
             Finite(o.w.x) && Finite(o.w.y) && Finite(o.w.z));
  for (auto& A : E.art)
    for (auto& J : A.j) bad |= !(Finite(J.q) && Finite(J.qd));
  if (bad) E.status |= STATUS_NUMERIC;
}

// ---------------------------------------------------------------------------
// C interface
// ---------------------------------------------------------------------------
static V3 v3(const double* p) { return V3(p[0], p[1], p[2]); }
static Quat qt(const double* p) { Quat q; q.w = p[0]; q.x = p[1]; q.y = p[2]; q.z = p[3]; return q; }

extern "C" {

typedef struct {
  double* obj_pos; double* obj_quat; double* obj_vel; double* obj_omega; int* obj_awake; int* obj_ctr;
  double* joint_q; double* joint_qd; double* joint_target; double* art_base_pos; double* art_base_quat;
  double* joint_lim_lambda; int* joint_lim_side;
  int* cache_count; int* cache_key; double* cache_p; double* cache_lambda;  // [E], [E*C*3], [E*C*3], [E*C*4]
  double* joint_motor_lambda;  // [NJ], may be NULL
} OrState;

void* oracle_create(const OrDesc* d, const OrParams* p) {
  World* W = new World();
  W->P = *p;
  W->has_mlp = 0;
  int E = d->n_envs;
  W->env.resize(E);
  W->obj_off.assign(d->obj_off, d->obj_off + E + 1);
  W->stat_off.assign(d->stat_off, d->stat_off + E + 1);
  W->art_off.assign(d->art_off, d->art_off + E + 1);
  W->n_obj = d->obj_off[E]; W->n_stat = d->stat_off[E]; W->n_art = d->art_off[E];
  W->joint_off.assign(d->joint_off, d->joint_off + W->n_art + 1);
  W->n_joint = d->joint_off[W->n_art];
  for (int e = 0; e < E; ++e) {
    Env& en = W->env[e];
    en.plane = d->env_plane[e];
    en.n_rows = en.iters = en.status = en.n_limit_rows = en.n_colours = 0;
    en.resid = 0;
    for (int i = d->obj_off[e]; i < d->obj_off[e + 1]; ++i) {
      Obj o;
      o.shape = d->obj_shape[i]; o.half = v3(d->obj_half + 3 * i); o.mass = d->obj_mass[i];
      o.inv_mass = real(1) / o.mass;
      if (o.shape == SHAPE_SPHERE) {
        real I = real(0.4) * o.mass * o.half.x * o.half.x;
        o.inv_I = V3(real(1) / I, real(1) / I, real(1) / I);
      } else {
        V3 I = box_inertia(o.mass, o.half);
        o.inv_I = V3(real(1) / I.x, real(1) / I.y, real(1) / I.z);
      }
      o.mu = d->obj_mu[i]; o.rest = d->obj_rest[i];
      o.x = v3(d->obj_pos + 3 * i); o.q = qt(d->obj_quat + 4 * i);
      o.v = v3(d->obj_vel + 3 * i); o.w = v3(d->obj_omega + 3 * i);
      o.awake = 1; o.ctr = 0;
      en.obj.push_back(o);
    }
    for (int s = d->stat_off[e]; s < d->stat_off[e + 1]; ++s) {
      Stat st; st.x = v3(d->stat_pos + 3 * s); st.q = qt(d->stat_quat + 4 * s); st.half = v3(d->stat_half + 3 * s);
      st.mu = d->stat_mu[s];
      en.st.push_back(st);
    }
    for (int a = d->art_off[e]; a < d->art_off[e + 1]; ++a) {
      Art A;
      A.base_x = v3(d->art_base_pos + 3 * a); A.base_q = qt(d->art_base_quat + 4 * a);
      A.has_bc = d->art_has_base_coll[a]; A.bc_off = v3(d->art_base_coll_off + 3 * a);
      A.bc_half = v3(d->art_base_coll_half + 3 * a); A.kinematic = d->art_kinematic[a];
      for (int j = d->joint_off[a]; j < d->joint_off[a + 1]; ++j) {
        Joint J;
        J.parent = d->joint_parent[j]; J.type = d->joint_type[j]; J.axis = v3(d->joint_axis + 3 * j);
        J.opos = v3(d->joint_origin_pos + 3 * j); J.oq = qt(d->joint_origin_quat + 4 * j);
        J.com = v3(d->joint_com + 3 * j); J.half = v3(d->joint_half + 3 * j); J.mass = d->joint_mass[j];
        J.lo = d->joint_lo[j]; J.hi = d->joint_hi[j]; J.has_limit = d->joint_has_limit[j];
        J.kp = d->joint_kp[j]; J.kd = d->joint_kd[j]; J.mu = d->joint_mu[j];
        J.q = d->joint_q0[j]; J.qd = d->joint_qd0[j]; J.target = d->joint_target[j];
        J.lim_lambda = 0; J.lim_side = 0; J.motor_lambda = 0;
        A.j.push_back(J);
      }
      en.art.push_back(A);
    }
  }
  return W;
}

void oracle_destroy(void* h) { delete (World*)h; }

static void step_range(World* W, int e0, int e1, int n) {
  for (int e = e0; e < e1; ++e)
    for (int s = 0; s < n; ++s) env_step(*W, W->env[e], nullptr);
  flush_op_counts();
}

// Advance every environment by n steps using up to `threads` host threads
// (static contiguous partition of the environments).
int oracle_step(void* h, int n, int threads) {
  World* W = (World*)h;
  int E = (int)W->env.size();
  if (threads <= 1 || E < 2) {
    step_range(W, 0, E, n);
  } else {
    std::vector<std::thread> th;
    int T = std::min(threads, E);
    for (int t = 0; t < T; ++t) {
      int e0 = (int)((long long)E * t / T), e1 = (int)((long long)E * (t + 1) / T);
      th.emplace_back(step_range, W, e0, e1, n);
    }
    for (auto& t : th) t.join();
  }
  int st = 0;
  for (auto& en : W->env) st |= en.status;
  return st;
}

// One step while logging (features, normalised impulse corrections) of every contact.
int oracle_step_logged(void* h, double* feats, double* lams, int cap, int* n_out) {
  World* W = (World*)h;
  std::vector<double> f, l;
  StepLog lg; lg.feats = &f; lg.lams = &l;
  int st = 0;
  for (auto& en : W->env) { env_step(*W, en, &lg); st |= en.status; }
  int n = (int)(l.size() / 3);
  int m = std::min(n, cap);
  std::memcpy(feats, f.data(), sizeof(double) * MLP_IN * m);
  std::memcpy(lams, l.data(), sizeof(double) * 3 * m);
  *n_out = n;
  return st;
}

void oracle_set_params(void* h, const OrParams* p) { ((World*)h)->P = *p; }

void oracle_get_state(void* h, OrState* s) {
  World* W = (World*)h;
  int C = W->P.max_contacts;
  for (size_t e = 0; e < W->env.size(); ++e) {
    Env& en = W->env[e];
    int o0 = W->obj_off[e];
    for (size_t i = 0; i < en.obj.size(); ++i) {
      const Obj& o = en.obj[i];
      int k = o0 + (int)i;
      double* p = s->obj_pos + 3 * k; p[0] = D(o.x.x); p[1] = D(o.x.y); p[2] = D(o.x.z);
      double* q = s->obj_quat + 4 * k; q[0] = D(o.q.w); q[1] = D(o.q.x); q[2] = D(o.q.y); q[3] = D(o.q.z);
      double* v = s->obj_vel + 3 * k; v[0] = D(o.v.x); v[1] = D(o.v.y); v[2] = D(o.v.z);
      double* w = s->obj_omega + 3 * k; w[0] = D(o.w.x); w[1] = D(o.w.y); w[2] = D(o.w.z);
      s->obj_awake[k] = o.awake; s->obj_ctr[k] = o.ctr;
    }
    int a0 = W->art_off[e];
    for (size_t a = 0; a < en.art.size(); ++a) {
      const Art& A = en.art[a];
      int ka = a0 + (int)a;
      double* bp = s->art_base_pos + 3 * ka; bp[0] = D(A.base_x.x); bp[1] = D(A.base_x.y); bp[2] = D(A.base_x.z);
      double* bq = s->art_base_quat + 4 * ka; bq[0] = D(A.base_q.w); bq[1] = D(A.base_q.x); bq[2] = D(A.base_q.y); bq[3] = D(A.base_q.z);
      int j0 = W->joint_off[ka];
      for (size_t j = 0; j < A.j.size(); ++j) {
        s->joint_q[j0 + j] = D(A.j[j].q); s->joint_qd[j0 + j] = D(A.j[j].qd); s->joint_target[j0 + j] = D(A.j[j].target);
        s->joint_lim_lambda[j0 + j] = D(A.j[j].lim_lambda); s->joint_lim_side[j0 + j] = A.j[j].lim_side;
        if (s->joint_motor_lambda) s->joint_motor_lambda[j0 + j] = D(A.j[j].motor_lambda);
      }
    }
    int n = std::min((int)en.cache.size(), C);
    s->cache_count[e] = n;
    for (int i = 0; i < n; ++i) {
      const CacheEntry& ce = en.cache[i];
      size_t b = (size_t)e * C + i;
      s->cache_key[3 * b] = ce.a; s->cache_key[3 * b + 1] = ce.b; s->cache_key[3 * b + 2] = ce.f;
      s->cache_p[3 * b] = D(ce.p.x); s->cache_p[3 * b + 1] = D(ce.p.y); s->cache_p[3 * b + 2] = D(ce.p.z);
      s->cache_lambda[4 * b] = D(ce.ln); s->cache_lambda[4 * b + 1] = D(ce.lt.x);
      s->cache_lambda[4 * b + 2] = D(ce.lt.y); s->cache_lambda[4 * b + 3] = D(ce.lt.z);
    }
  }
}

void oracle_set_state(void* h, const OrState* s) {
  World* W = (World*)h;
  int C = W->P.max_contacts;
  for (size_t e = 0; e < W->env.size(); ++e) {
    Env& en = W->env[e];
    int o0 = W->obj_off[e];
    for (size_t i = 0; i < en.obj.size(); ++i) {
      Obj& o = en.obj[i];
      int k = o0 + (int)i;
      o.x = v3(s->obj_pos + 3 * k); o.q = qt(s->obj_quat + 4 * k); o.v = v3(s->obj_vel + 3 * k);
      o.w = v3(s->obj_omega + 3 * k); o.awake = s->obj_awake[k]; o.ctr = s->obj_ctr[k];
    }
    int a0 = W->art_off[e];
    for (size_t a = 0; a < en.art.size(); ++a) {
      Art& A = en.art[a];
      int ka = a0 + (int)a;
      A.base_x = v3(s->art_base_pos + 3 * ka); A.base_q = qt(s->art_base_quat + 4 * ka);
      int j0 = W->joint_off[ka];
      for (size_t j = 0; j < A.j.size(); ++j) {
        A.j[j].q = s->joint_q[j0 + j]; A.j[j].qd = s->joint_qd[j0 + j]; A.j[j].target = s->joint_target[j0 + j];
        A.j[j].lim_lambda = s->joint_lim_lambda[j0 + j]; A.j[j].lim_side = s->joint_lim_side[j0 + j];
        if (s->joint_motor_lambda) A.j[j].motor_lambda = s->joint_motor_lambda[j0 + j];
      }
    }
    en.cache.clear();
    int n = std::min(s->cache_count[e], C);
    for (int i = 0; i < n; ++i) {
      size_t b = (size_t)e * C + i;
      CacheEntry ce;
      ce.a = s->cache_key[3 * b]; ce.b = s->cache_key[3 * b + 1]; ce.f = s->cache_key[3 * b + 2];
      ce.p = v3(s->cache_p + 3 * b);
      ce.ln = s->cache_lambda[4 * b];
      ce.lt = V3(s->cache_lambda[4 * b + 1], s->cache_lambda[4 * b + 2], s->cache_lambda[4 * b + 3]);
      en.cache.push_back(ce);
    }
  }
}

// Per-env results of the last step: status, PGS sweeps, residual, #contacts, #rows, #limit rows, #colours.
void oracle_get_stats(void* h, int* status, int* iters, double* resid, int* n_contacts, int* n_rows,
                      int* n_limit_rows, int* n_colours) {
  World* W = (World*)h;
  for (size_t e = 0; e < W->env.size(); ++e) {
    const Env& en = W->env[e];
    status[e] = en.status; iters[e] = en.iters; resid[e] = D(en.resid);
    n_contacts[e] = (int)en.contacts.size(); n_rows[e] = en.n_rows; n_limit_rows[e] = en.n_limit_rows;
    n_colours[e] = en.n_colours;
  }
}

// Contact force on the robot (N): this step's and the accumulated value per env.
void oracle_get_robot_force(void* h, double* step, double* acc) {
  World* W = (World*)h;
  for (size_t e = 0; e < W->env.size(); ++e) {
    if (step) step[e] = D(W->env[e].robot_force);
    if (acc) acc[e] = D(W->env[e].robot_force_acc);
  }
}

// Zero the accumulated robot contact force of the listed envs (all when ids is NULL).
void oracle_reset_robot_force(void* h, const int* ids, int n) {
  World* W = (World*)h;
  if (!ids) {
    for (auto& E : W->env) E.robot_force_acc = 0;
    return;
  }
  for (int k = 0; k < n; ++k) W->env[ids[k]].robot_force_acc = 0;
}

// Contacts of env e from the last step: key (a, b, f), point, normal, sep, final impulses.
int oracle_get_contacts(void* h, int e, int cap, int* key, double* p, double* n, double* sep, double* lam) {
  World* W = (World*)h;
  const Env& en = W->env[e];
  int m = std::min(cap, (int)en.contacts.size());
  for (int i = 0; i < m; ++i) {
    const Contact& c = en.contacts[i];
    key[3 * i] = c.a; key[3 * i + 1] = c.b; key[3 * i + 2] = c.f;
    p[3 * i] = D(c.p.x); p[3 * i + 1] = D(c.p.y); p[3 * i + 2] = D(c.p.z);
    n[3 * i] = D(c.n.x); n[3 * i + 1] = D(c.n.y); n[3 * i + 2] = D(c.n.z);
    sep[i] = D(c.sep);
    lam[3 * i] = D(c.lam[0]); lam[3 * i + 1] = D(c.lam[1]); lam[3 * i + 2] = D(c.lam[2]);
  }
  return (int)en.contacts.size();
}

// Candidate pairs (after the wake pass) of env e from the last step, packed a*4096+b.
// Colouring of env e's units at the last step (unit order): colour, node A, node B.
// Returns the number of units (0 colours written when colouring is off).
int oracle_get_colouring(void* h, int e, int cap, int* colour, int* node_a, int* node_b) {
  const Env& E = static_cast<World*>(h)->env[e];
  const int n = (int)E.unit_node_a.size();
  for (int i = 0; i < n && i < cap; ++i) {
    colour[i] = i < (int)E.unit_colour.size() ? E.unit_colour[i] : -1;
    node_a[i] = E.unit_node_a[i];
    node_b[i] = E.unit_node_b[i];
  }
  return n;
}

int oracle_get_pairs(void* h, int e, int cap, int* out) {
  World* W = (World*)h;
  const Env& en = W->env[e];
  int m = std::min(cap, (int)en.pairs.size());
  for (int i = 0; i < m; ++i) out[i] = en.pairs[i];
  return (int)en.pairs.size();
}

// Articulation a of env e at its current state: link poses (world COM, 3x3
// rotation), q̈ from ABA (implicit PD armature with the world's dt), M + armature
// and its inverse (n x n row-major).
int oracle_articulation(void* h, int e, int a, double* com, double* rot, double* qdd, double* M, double* Minv) {
  World* W = (World*)h;
  Art& A = W->env[e].art[a];
  int n = (int)A.j.size();
  real dt = W->P.dt;
  V3 g(W->P.gravity[0], W->P.gravity[1], W->P.gravity[2]);
  art_fk(A);
  real tau[MAXDOF], q2[MAXDOF];
  for (int i = 0; i < n; ++i) tau[i] = pd_tau(A.j[i], dt);
  art_aba(A, g, dt, tau, q2);
  art_crba(A, dt);
  spd_inverse(n, A.M, A.Minv);
  for (int i = 0; i < n; ++i) {
    qdd[i] = D(q2[i]);
    com[3 * i] = D(A.c[i].x); com[3 * i + 1] = D(A.c[i].y); com[3 * i + 2] = D(A.c[i].z);
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) rot[9 * i + 3 * r + c] = D(A.R[i].m[r][c]);
    for (int k = 0; k < n; ++k) { M[n * i + k] = D(A.M[i][k]); Minv[n * i + k] = D(A.Minv[i][k]); }
  }
  return n;
}

// Textbook cross-checks on articulation a of env e (no armature, given q̇):
// ABA q̈ for joint forces tau, RNEA forces for accelerations, CRBA M(q).
void oracle_dynamics_check(void* h, int e, int a, const double* tau, double* qdd_aba, const double* qdd_in,
                           double* tau_rnea, double* M) {
  World* W = (World*)h;
  Art& A = W->env[e].art[a];
  int n = (int)A.j.size();
  V3 g(W->P.gravity[0], W->P.gravity[1], W->P.gravity[2]);
  art_fk(A);
  real t[MAXDOF], q2[MAXDOF], qi[MAXDOF], tr[MAXDOF];
  for (int i = 0; i < n; ++i) { t[i] = tau[i]; qi[i] = qdd_in[i]; }
  art_aba(A, g, 0, t, q2);
  art_rnea(A, g, qi, tr);
  art_crba(A, 0);
  for (int i = 0; i < n; ++i) {
    qdd_aba[i] = D(q2[i]); tau_rnea[i] = D(tr[i]);
    for (int k = 0; k < n; ++k) M[n * i + k] = D(A.M[i][k]);
  }
}

// Narrowphase on two standalone shapes (tests): shape 0 sphere, 1 box, 2 plane
// (z = 0); B must not precede A in collider order.  Returns the contact count.
int oracle_narrowphase(int shape_a, const double* xa, const double* qa, const double* ha, int shape_b,
                       const double* xb, const double* qb, const double* hb, double margin, double* p, double* n,
                       double* sep, int* feat, int cap) {
  Coll A, B;
  A.kind = CK_OBJ; A.shape = shape_a; A.x = v3(xa); A.R = quat_to_mat(qt(qa)); A.half = v3(ha);
  B.kind = shape_b == SHAPE_PLANE ? CK_PLANE : CK_STATIC; B.shape = shape_b;
  if (shape_b != SHAPE_PLANE) { B.x = v3(xb); B.R = quat_to_mat(qt(qb)); B.half = v3(hb); }
  std::vector<RawContact> out;
  narrowphase(A, B, margin, out);
  int m = std::min(cap, (int)out.size());
  for (int i = 0; i < m; ++i) {
    p[3 * i] = D(out[i].p.x); p[3 * i + 1] = D(out[i].p.y); p[3 * i + 2] = D(out[i].p.z);
    n[3 * i] = D(out[i].n.x); n[3 * i + 1] = D(out[i].n.y); n[3 * i + 2] = D(out[i].n.z);
    sep[i] = D(out[i].sep); feat[i] = out[i].f;
  }
  return (int)out.size();
}

// ---- learned warm start: parameters, forward, backward (FP64) ----
int oracle_mlp_nparam() { return MLP_NPARAM; }

void oracle_set_mlp(void* h, const double* params) {
  World* W = (World*)h;
  if (!params) { W->has_mlp = 0; return; }
  W->mlp_w.assign(params, params + MLP_NPARAM);
  W->has_mlp = 1;
}

// Forward a batch X[n][32] -> Y[n][3].
void oracle_mlp_forward(const double* params, int n, const double* X, double* Y) {
  g_stage = ST_MLP;
  for (int s = 0; s < n; ++s) {
    real x[MLP_IN], z[3][128], h[3][128], y[3];
    for (int i = 0; i < MLP_IN; ++i) x[i] = X[s * MLP_IN + i];
    mlp_forward1(params, x, z, h, y);
    for (int o = 0; o < 3; ++o) Y[s * 3 + o] = D(y[o]);
  }
}

// Mean-squared-error loss L = (1/(3n)) sum (Y - T)^2 and its gradient w.r.t.
// every parameter (same layout as params), by backpropagation.
double oracle_mlp_loss_grad(const double* params, int n, const double* X, const double* T, double* grad) {
  int off[8];
  mlp_layer_offsets(off);
  std::vector<real> G(MLP_NPARAM, real(0));
  real loss = 0;
  for (int s = 0; s < n; ++s) {
    real x[MLP_IN], z[3][128], h[3][128], y[3];
    for (int i = 0; i < MLP_IN; ++i) x[i] = X[s * MLP_IN + i];
    mlp_forward1(params, x, z, h, y);
    real dy[3];
    for (int o = 0; o < 3; ++o) {
      real d = y[o] - real(T[s * 3 + o]);
      loss += d * d;
      dy[o] = real(2) * d / real(3 * n);
    }
    // layer 4
    real dh[128], dz[128];
    for (int i = 0; i < MLP_H; ++i) dh[i] = 0;
    for (int o = 0; o < 3; ++o) {
      G[off[7] + o] += dy[o];
      for (int i = 0; i < MLP_H; ++i) {
        G[off[6] + o * MLP_H + i] += dy[o] * h[2][i];
        dh[i] += real(params[off[6] + o * MLP_H + i]) * dy[o];
      }
    }
    for (int l = 2; l >= 0; --l) {
      for (int i = 0; i < MLP_H; ++i) dz[i] = dh[i] * gelu_grad(z[l][i]);
      int nin = l == 0 ? MLP_IN : MLP_H;
      const real* in = l == 0 ? x : h[l - 1];
      real dprev[128];
      for (int i = 0; i < nin; ++i) dprev[i] = 0;
      for (int o = 0; o < MLP_H; ++o) {
        G[off[2 * l + 1] + o] += dz[o];
        for (int i = 0; i < nin; ++i) {
          G[off[2 * l] + o * nin + i] += dz[o] * in[i];
          dprev[i] += real(params[off[2 * l] + o * nin + i]) * dz[o];
        }
      }
      for (int i = 0; i < nin; ++i) dh[i] = dprev[i];
    }
  }
  for (int i = 0; i < MLP_NPARAM; ++i) grad[i] = D(G[i]);
  return D(loss / real(3 * n));
}

// Features of every contact of the last step are not kept; this recomputes
// them for a fresh step without advancing: returns the number of contacts.
// (Used by tests on tiny scenes through oracle_step_logged instead.)

// Op counts per stage (op-counting build only): every thread's, since the last reset.
void oracle_get_op_counts(unsigned long long* out) {
  for (int i = 0; i < ST_COUNT; ++i) out[i] = g_ops_done[i].load() + g_ops[i];
}
void oracle_reset_op_counts() {
  for (int i = 0; i < ST_COUNT; ++i) {
    g_ops[i] = 0;
    g_ops_done[i] = 0;
  }
}

}  // extern "C"
