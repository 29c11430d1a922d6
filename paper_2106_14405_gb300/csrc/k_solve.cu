// Constraint rows, projected Gauss-Seidel and integration.
//
// k_rows (one warp per environment, lanes over contacts):
//   per contact a normal row and two friction rows on the tangent basis
//   t1 = normalize(n x e) (e = x unless |n_x| >= 0.57735, then y), t2 = n x t1;
//   endpoint A is the contact's first collider, B the second; a free object
//   contributes inv_m + (r x d)^T I_w^-1 (r x d) to the row's inverse effective
//   mass, an articulation link j^T M^-1 j with j the generalised Jacobian of the
//   contact point (stored with w = M^-1 j in a per-environment pool); the
//   normal row's target velocity is -sep/dt for a speculative contact (sep > 0),
//   0 inside the slop band, beta (-sep - slop)/dt deeper, raised to the
//   restitution bounce e |v_n| above the rest threshold; a row whose inverse
//   effective mass is below 1e-6 gets none.  Joint-limit rows are added where
//   q + dt q̇* leaves [lo, hi], targeting the limit within the step (or pushing
//   back at the Baumgarte rate once violated).  Warm start: the prior frame's
//   impulse of the contact with the same (a, b, feature) key whose point moved
//   less than match_dist, friction re-projected on the new basis and clamped.
//   Optional 32 features per contact for the learned warm start.
// k_pgs (one warp per environment; sequential impulses after Catto, GDC 2005):
//   the environment's body velocities and impulses live in shared memory;
//   constraint units (a contact's three rows, or a limit row) get greedy
//   colours in (a, b, feature) order -- an articulation is one node, statics
//   are none -- so units of one colour touch disjoint bodies and the lanes
//   update them in parallel with exactly the arithmetic of a sequential sweep
//   in colour order.  Friction is clamped to mu times the contact's current
//   normal impulse.  Relative residual ||Δλ|| / max(||λ||, floor) per sweep by
//   warp reduction.
// k_integrate (one thread per object or joint): semi-implicit Euler with
//   Kahan-compensated position sums, quaternion update, sleeping.
#include <math.h>

#include "sim_internal.cuh"

namespace gb {

struct EnvInfo {
  int o0, nobj, a0, narts, l0, nlink, s0;
};

__device__ __forceinline__ EnvInfo env_info(const Dev& d, int e) {
  EnvInfo r;
  r.o0 = d.obj_off[e];
  r.nobj = d.obj_off[e + 1] - r.o0;
  r.a0 = d.art_off[e];
  r.narts = d.art_off[e + 1] - r.a0;
  r.l0 = d.joint_off[r.a0];
  r.nlink = d.joint_off[r.a0 + r.narts] - r.l0;
  r.s0 = d.stat_off[e];
  return r;
}

__device__ __forceinline__ M3 inv_inertia_world(float4 q, float4 inv) {
  M3 R = quat_mat(q);
  M3 r;
  V3 c0 = v3(R.r0.x, R.r1.x, R.r2.x), c1 = v3(R.r0.y, R.r1.y, R.r2.y), c2 = v3(R.r0.z, R.r1.z, R.r2.z);
  // R diag(inv) R^T, entry (i, j) = sum_k R_ik inv_k R_jk
  V3 rows[3] = {R.r0, R.r1, R.r2};
  float m[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      m[3 * i + j] = rows[i].x * inv.y * rows[j].x + rows[i].y * inv.z * rows[j].y + rows[i].z * inv.w * rows[j].z;
  (void)c0; (void)c1; (void)c2;
  r.r0 = v3(m[0], m[1], m[2]);
  r.r1 = v3(m[3], m[4], m[5]);
  r.r2 = v3(m[6], m[7], m[8]);
  return r;
}

__device__ __forceinline__ void tangents(V3 n, V3& t1, V3& t2) {
  V3 e = fabsf(n.x) < 0.57735f ? v3(1.f, 0.f, 0.f) : v3(0.f, 1.f, 0.f);
  t1 = cross(n, e);
  t1 = t1 * (1.f / norm(t1));
  t2 = cross(n, t1);
}

// ---------------------------------------------------------------------------
// k_rows
// ---------------------------------------------------------------------------
struct EndRow {
  int code;        // -1 static, object local index, or ART_TAG | art << 8 | slot
  V3 r;            // object: contact point minus COM
  float k[3];      // contribution to the inverse effective mass per row
  float vel[3];    // contribution to J v* per row (sign not applied)
  float mu, rest, inv_m;
  V3 w;            // object angular velocity (features)
  V3 x;            // reference position (features)
};

__device__ void endpoint_rows(const Dev& d, const EnvInfo& ei, int e, int c, V3 p, const V3* dir, int slot,
                              EndRow& o) {
  o.inv_m = 0.f;
  o.rest = 0.f;
  o.w = v3(0.f, 0.f, 0.f);
  o.r = v3(0.f, 0.f, 0.f);
  for (int r = 0; r < 3; ++r) { o.k[r] = 0.f; o.vel[r] = 0.f; }
  if (c < ei.nobj) {
    int k = ei.o0 + c;
    float4 q = d.obj_quat[k], inv = d.obj_inv[k];
    float2 mat = d.obj_mat[k];
    V3 x = v3(d.obj_pos[k]);
    V3 v = v3(d.obj_vstar[k]), w = v3(d.obj_wstar[k]);
    M3 Ii = inv_inertia_world(q, inv);
    o.code = c;
    o.r = p - x;
    o.x = x;
    o.w = w;
    o.mu = mat.x;
    o.rest = mat.y;
    o.inv_m = inv.x;
    for (int r = 0; r < 3; ++r) {
      V3 rd = cross(o.r, dir[r]);
      o.k[r] = inv.x + dot(rd, mv(Ii, rd));
      o.vel[r] = dot(dir[r], v + cross(w, o.r));
    }
    return;
  }
  if (c < ei.nobj + ei.nlink) {
    int jg = ei.l0 + (c - ei.nobj);
    int art = d.j_art[jg];
    int jb = d.joint_off[art];
    int n = d.joint_off[art + 1] - jb;
    int jl = jg - jb;
    o.code = ART_TAG | ((art - ei.a0) << 8) | slot;
    o.x = v3(d.l_com[jg]);
    o.mu = d.j_half[jg].w;
    float* J = d.ap_j + ((size_t)e * APOOL + slot) * 27;
    float* W = d.ap_w + ((size_t)e * APOOL + slot) * 27;
    const float* Mi = d.a_minv + (size_t)art * 81;
    float jv[3][MAX_DOF];
    for (int r = 0; r < 3; ++r)
      for (int i = 0; i < MAX_DOF; ++i) jv[r][i] = 0.f;
    for (int i = jl; i >= 0; i = d.j_parent[jb + i]) {
      float4 a4 = d.l_ja[jb + i];
      V3 a = v3(a4);
      V3 sp = a4.w == 0.f ? cross(a, p - v3(d.l_jo[jb + i])) : a;
      for (int r = 0; r < 3; ++r) jv[r][i] = dot(dir[r], sp);
    }
    for (int r = 0; r < 3; ++r) {
      float kk = 0.f, vv = 0.f;
      for (int i = 0; i < MAX_DOF; ++i) {  // zero beyond n: the solver sums all MAX_DOF entries
        float s = 0.f;
        if (i < n) {
          for (int k = 0; k < n; ++k) s += Mi[9 * i + k] * jv[r][k];
          kk += jv[r][i] * s;
          vv += jv[r][i] * d.j_qdstar[jb + i];
        }
        J[9 * r + i] = i < n ? jv[r][i] : 0.f;
        W[9 * r + i] = s;
      }
      o.k[r] = kk;
      o.vel[r] = vv;
    }
    return;
  }
  o.code = -1;
  // static colliders: robot base boxes, static boxes, plane
  int nb = d.base_off[e + 1] - d.base_off[e];
  int cs = c - ei.nobj - ei.nlink;
  if (cs < nb) {
    int art = d.base_art[d.base_off[e] + cs];
    M3 R = quat_mat(d.art_base_quat[art]);
    o.x = v3(d.art_base_pos[art]) + mv(R, v3(d.art_bc_off[art]));
    o.mu = 0.5f;
  } else if (cs - nb < d.stat_off[e + 1] - ei.s0) {
    float4 sp = d.stat_pos[ei.s0 + cs - nb];
    o.x = v3(sp);
    o.mu = sp.w;
  } else {
    o.x = v3(p.x, p.y, 0.f);
    o.mu = d.plane_mu;
  }
}

__global__ void __launch_bounds__(128) k_rows(Dev d) {
  const int lane = threadIdx.x & 31;
  const int e = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (e >= d.E) return;
  const EnvInfo ei = env_info(d, e);
  const int C = d.C;
  const int nct = d.n_contacts[e];
  const float dt = d.dt;
  const V3 g = v3(d.gx, d.gy, d.gz);
  const float gdt = norm(g) * dt;
  const bool want_feat = d.log_features || d.warm_mode == 2;
  const int ncache = d.cache_count[e];
  unsigned status = 0;
  int pool = 0;
  for (int i0 = 0; i0 < nct; i0 += 32) {
    int i = i0 + lane;
    bool valid = i < nct;
    size_t gi = (size_t)e * C + (valid ? i : 0);
    int4 key = valid ? d.c_key[gi] : make_int4(0, 0, 0, 0);
    int need = valid ? ((key.x >= ei.nobj && key.x < ei.nobj + ei.nlink) ? 1 : 0) +
                           ((key.y >= ei.nobj && key.y < ei.nobj + ei.nlink) ? 1 : 0)
                     : 0;
    int incl = need;
    for (int o = 1; o < 32; o <<= 1) {
      int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    int total = __shfl_sync(0xffffffffu, incl, 31);
    int slot = pool + incl - need;
    pool += total;
    if (!valid) continue;
    float4 p4 = d.c_p[gi], n4 = d.c_n[gi];
    V3 p = v3(p4), n = v3(n4);
    float sep = p4.w;
    V3 dir[3];
    dir[0] = n;
    tangents(n, dir[1], dir[2]);
    if (slot + need > APOOL) {  // articulation row pool exhausted: drop the contact's response
      status |= ST_OVERFLOW;
      slot = 0;
    }
    EndRow A, B;
    int sa = slot, sb = slot + ((key.x >= ei.nobj && key.x < ei.nobj + ei.nlink) ? 1 : 0);
    endpoint_rows(d, ei, e, key.x, p, dir, sa, A);
    endpoint_rows(d, ei, e, key.y, p, dir, sb, B);
    float meff[3];
    for (int r = 0; r < 3; ++r) {  // a row that cannot change the relative velocity gets no impulse
      float K = A.k[r] + B.k[r];
      meff[r] = K > 1e-6f ? 1.f / K : 0.f;
    }
    float mu = sqrtf(A.mu * B.mu);
    float vn = A.vel[0] - B.vel[0];
    float tgt;
    if (sep > 0.f) tgt = -sep / dt;
    else if (sep > -d.slop) tgt = 0.f;
    else tgt = -d.baumgarte * (sep + d.slop) / dt;
    float rest = fmaxf(A.rest, B.rest);
    if (vn < -d.rest_thresh) tgt = fmaxf(tgt, -rest * vn);
    // prior-frame match: cache is in (a, b, feature) order
    float prev[3] = {0.f, 0.f, 0.f};
    int matched = 0;
    {
      int lo = 0, hi = ncache - 1, found = -1;
      while (lo <= hi) {
        int mid = (lo + hi) >> 1;
        int4 k = d.cache_key[(size_t)e * C + mid];
        bool less = k.x < key.x || (k.x == key.x && (k.y < key.y || (k.y == key.y && k.z < key.z)));
        bool eq = k.x == key.x && k.y == key.y && k.z == key.z;
        if (eq) { found = mid; break; }
        if (less) lo = mid + 1; else hi = mid - 1;
      }
      if (found >= 0) {
        float4 cp = d.cache_p[(size_t)e * C + found];
        if (norm(v3(cp) - p) < d.match_dist) {
          float4 cl = d.cache_lam[(size_t)e * C + found];
          V3 lt = v3(cl.y, cl.z, cl.w);
          float lim = mu * cl.x;
          prev[0] = cl.x;
          prev[1] = fmaxf(-lim, fminf(lim, dot(lt, dir[1])));
          prev[2] = fmaxf(-lim, fminf(lim, dot(lt, dir[2])));
          matched = 1;
        }
      }
    }
    d.r_t1[gi] = f4(dir[1], mu);
    d.r_meff[gi] = make_float4(meff[0], meff[1], meff[2], tgt);
    d.r_lam[gi] = d.warm_mode >= 1 ? make_float4(prev[0], prev[1], prev[2], 0.f) : make_float4(0.f, 0.f, 0.f, 0.f);
    d.r_ra[gi] = f4(A.r, 0.f);
    d.r_rb[gi] = f4(B.r, 0.f);
    d.r_ends[gi] = make_int2(A.code, B.code);
    if (want_feat) {
      float* f = d.feat + gi * NFEAT;
      V3 ra = p - A.x, rb = p - B.x;
      V3 wr = A.w - B.w;
      f[0] = n.x; f[1] = n.y; f[2] = n.z;
      f[3] = ra.x; f[4] = ra.y; f[5] = ra.z;
      f[6] = rb.x; f[7] = rb.y; f[8] = rb.z;
      for (int r = 0; r < 3; ++r) f[9 + r] = A.vel[r] - B.vel[r];
      f[12] = wr.x; f[13] = wr.y; f[14] = wr.z;
      f[15] = sep;
      f[16] = A.inv_m; f[17] = B.inv_m;
      f[18] = meff[0]; f[19] = meff[1]; f[20] = meff[2];
      f[21] = mu;
      f[22] = dot(g, n) * dt;
      f[23] = prev[0]; f[24] = prev[1]; f[25] = prev[2];
      f[26] = (float)matched;
      // pair type: 0 sphere-sphere, 1 sphere-plane, 2 sphere-box, 3 box-plane, 4 box-box
      bool sphA = key.x < ei.nobj && d.obj_half[ei.o0 + key.x].w == 0.f;
      bool sphB = key.y < ei.nobj && d.obj_half[ei.o0 + key.y].w == 0.f;
      bool plane = d.env_plane[e] &&
                   key.y == ei.nobj + ei.nlink + (d.base_off[e + 1] - d.base_off[e]) + (d.stat_off[e + 1] - ei.s0);
      int type = (sphA && sphB) ? 0 : (plane ? (sphA ? 1 : 3) : ((sphA || sphB) ? 2 : 4));
      for (int t = 0; t < 5; ++t) f[27 + t] = t == type ? 1.f : 0.f;
    }
    (void)gdt;
  }
  // joint-limit rows, (articulation, joint) order
  int nlim = 0;
  for (int t0 = 0; t0 < ei.nlink; t0 += 32) {
    int t = t0 + lane;
    int side = 0;
    int jg = ei.l0 + t;
    if (t < ei.nlink) {
      float4 lim = d.j_lim[jg];
      if (lim.z != 0.f) {
        float qp = d.j_q[jg] + dt * d.j_qdstar[jg];
        if (qp < lim.x) side = 1;
        else if (qp > lim.y) side = 2;
      }
    }
    unsigned m = __ballot_sync(0xffffffffu, side != 0);
    if (side) {
      int pos = nlim + __popc(m & ((1u << lane) - 1u));
      if (pos < LCAP) {
        int art = d.j_art[jg];
        int jb = d.joint_off[art];
        int n = d.joint_off[art + 1] - jb;
        int jl = jg - jb;
        const float* Mi = d.a_minv + (size_t)art * 81;
        float sgn = side == 1 ? 1.f : -1.f;
        float4 lim = d.j_lim[jg];
        float q = d.j_q[jg];
        // reach the limit within the step when not yet violated, push back at the Baumgarte rate when violated
        float cgap = side == 1 ? q - lim.x : lim.y - q;
        float tgt = cgap >= 0.f ? -cgap / dt : -d.baumgarte * cgap / dt;
        float lam0 = (d.warm_mode >= 1 && d.j_lim_side[jg] == side) ? d.j_lim_lambda[jg] : 0.f;
        size_t li = (size_t)e * LCAP + pos;
        d.lr_info[li] = make_int4(art - ei.a0, jl, side == 1 ? 1 : -1, jg);
        d.lr_data[li] = make_float4(1.f / Mi[9 * jl + jl], tgt, lam0, 0.f);
        for (int i = 0; i < MAX_DOF; ++i) d.lr_w[li * MAX_DOF + i] = i < n ? Mi[9 * i + jl] * sgn : 0.f;
      }
    }
    nlim += __popc(m);
  }
  if (nlim > LCAP) { status |= ST_OVERFLOW; nlim = LCAP; }
  status = __reduce_or_sync(0xffffffffu, status);
  if (lane == 0) {
    d.n_limit[e] = nlim;
    d.n_rows[e] = 3 * nct + nlim;
    if (status) atomicOr(&d.status[e], (int)status);
  }
}

// ---------------------------------------------------------------------------
// k_pgs
// ---------------------------------------------------------------------------
struct PgsLayout {
  int C;
  __host__ __device__ int units() const { return C + LCAP; }
  // floats: bodies 64*13, art q̇ 8*9, lambda units*3; ints: colour, order units*2, counts 66, used 72*2
  __host__ __device__ size_t bytes() const {
    size_t b = sizeof(float) * (MAX_OBJ * 13 + MAX_ARTS * MAX_DOF + (size_t)units() * 3) +
               sizeof(int) * ((size_t)units() * 2 + 66) + sizeof(unsigned long long) * (MAX_OBJ + MAX_ARTS);
    return (b + 15) & ~(size_t)15;
  }
};

struct PgsSh {
  float *v, *w, *im, *Ii, *qd, *lam;
  int *colour, *order, *cstart;
  unsigned long long* used;
};

__device__ __forceinline__ PgsSh pgs_carve(unsigned char* base, const PgsLayout& L) {
  PgsSh s;
  unsigned long long* u = reinterpret_cast<unsigned long long*>(base);
  s.used = u;
  float* f = reinterpret_cast<float*>(u + MAX_OBJ + MAX_ARTS);
  s.v = f; f += MAX_OBJ * 3;
  s.w = f; f += MAX_OBJ * 3;
  s.im = f; f += MAX_OBJ;
  s.Ii = f; f += MAX_OBJ * 6;
  s.qd = f; f += MAX_ARTS * MAX_DOF;
  s.lam = f; f += (size_t)L.units() * 3;
  int* ip = reinterpret_cast<int*>(f);
  s.colour = ip; ip += L.units();
  s.order = ip; ip += L.units();
  s.cstart = ip;
  return s;
}

struct PgsCtx {
  const Dev* d;
  PgsSh s;
  int e, C, nobj, nct;
};

// J v of one endpoint along direction d (row r), velocities from shared memory
__device__ __forceinline__ float end_vel(const PgsCtx& X, int code, V3 r, int row, V3 dv, size_t apbase) {
  if (code < 0) return 0.f;
  if (code < ART_TAG) {
    V3 v = v3(X.s.v[3 * code], X.s.v[3 * code + 1], X.s.v[3 * code + 2]);
    V3 w = v3(X.s.w[3 * code], X.s.w[3 * code + 1], X.s.w[3 * code + 2]);
    return dot(dv, v + cross(w, r));
  }
  int art = (code >> 8) & 0xff, slot = code & 0xff;
  const float* J = X.d->ap_j + (apbase + slot) * 27 + 9 * row;
  const float* qd = X.s.qd + art * MAX_DOF;
  float s = 0.f;
  for (int i = 0; i < MAX_DOF; ++i) s += J[i] * qd[i];
  return s;
}

__device__ __forceinline__ void end_apply(const PgsCtx& X, int code, V3 r, int row, V3 dv, float imp, size_t apbase) {
  if (code < 0) return;
  if (code < ART_TAG) {
    float im = X.s.im[code];
    const float* I = X.s.Ii + 6 * code;  // symmetric: xx xy xz yy yz zz
    V3 rd = cross(r, dv);
    V3 dw = v3(I[0] * rd.x + I[1] * rd.y + I[2] * rd.z, I[1] * rd.x + I[3] * rd.y + I[4] * rd.z,
               I[2] * rd.x + I[4] * rd.y + I[5] * rd.z);
    X.s.v[3 * code] += dv.x * (im * imp);
    X.s.v[3 * code + 1] += dv.y * (im * imp);
    X.s.v[3 * code + 2] += dv.z * (im * imp);
    X.s.w[3 * code] += dw.x * imp;
    X.s.w[3 * code + 1] += dw.y * imp;
    X.s.w[3 * code + 2] += dw.z * imp;
    return;
  }
  int art = (code >> 8) & 0xff, slot = code & 0xff;
  const float* W = X.d->ap_w + (apbase + slot) * 27 + 9 * row;
  float* qd = X.s.qd + art * MAX_DOF;
  for (int i = 0; i < MAX_DOF; ++i) qd[i] += W[i] * imp;
}

// One unit: either the three rows of contact u (< nct), or limit row u - nct.
// mode 0: sweep (returns squared change / squared value sums); mode 1: apply the warm start.
__device__ void do_unit(const PgsCtx& X, int u, int mode, float& d2, float& l2) {
  const Dev& d = *X.d;
  const size_t apbase = (size_t)X.e * APOOL;
  float* lam = X.s.lam + 3 * u;
  if (u >= X.nct) {
    size_t li = (size_t)X.e * LCAP + (u - X.nct);
    int4 info = d.lr_info[li];
    float4 ld = d.lr_data[li];
    const float* W = d.lr_w + li * MAX_DOF;
    float* qd = X.s.qd + info.x * MAX_DOF;
    if (mode == 1) {
      for (int i = 0; i < MAX_DOF; ++i) qd[i] += W[i] * lam[0];
      return;
    }
    float v = (float)info.z * qd[info.y];
    float nl = fmaxf(0.f, lam[0] + ld.x * (ld.y - v));
    float dl = nl - lam[0];
    for (int i = 0; i < MAX_DOF; ++i) qd[i] += W[i] * dl;
    lam[0] = nl;
    d2 += dl * dl;
    l2 += nl * nl;
    return;
  }
  size_t g = (size_t)X.e * X.C + u;
  V3 n = v3(d.c_n[g]);
  float4 t1m = d.r_t1[g];
  V3 t1 = v3(t1m);
  V3 t2 = cross(n, t1);
  float4 me = d.r_meff[g];
  V3 ra = v3(d.r_ra[g]), rb = v3(d.r_rb[g]);
  int2 ends = d.r_ends[g];
  V3 dirs[3] = {n, t1, t2};
  if (mode == 1) {
    for (int r = 0; r < 3; ++r) {
      end_apply(X, ends.x, ra, r, dirs[r], lam[r], apbase);
      end_apply(X, ends.y, rb, r, dirs[r], -lam[r], apbase);
    }
    return;
  }
  float vn = end_vel(X, ends.x, ra, 0, n, apbase) - end_vel(X, ends.y, rb, 0, n, apbase);
  float nl = fmaxf(0.f, lam[0] + me.x * (me.w - vn));
  float dl = nl - lam[0];
  end_apply(X, ends.x, ra, 0, n, dl, apbase);
  end_apply(X, ends.y, rb, 0, n, -dl, apbase);
  lam[0] = nl;
  d2 += dl * dl;
  l2 += nl * nl;
  float meff_t[2] = {me.y, me.z};
  for (int r = 1; r < 3; ++r) {
    V3 dv = dirs[r];
    float vt = end_vel(X, ends.x, ra, r, dv, apbase) - end_vel(X, ends.y, rb, r, dv, apbase);
    float lim = t1m.w * lam[0];
    float nt = fmaxf(-lim, fminf(lim, lam[r] - meff_t[r - 1] * vt));
    float dtl = nt - lam[r];
    end_apply(X, ends.x, ra, r, dv, dtl, apbase);
    end_apply(X, ends.y, rb, r, dv, -dtl, apbase);
    lam[r] = nt;
    d2 += dtl * dtl;
    l2 += nt * nt;
  }
}

__device__ __forceinline__ int unit_node(const EnvInfo& ei, int code) {
  if (code < 0) return -1;
  if (code < ART_TAG) return code;
  return ei.nobj + ((code >> 8) & 0xff);
}

__global__ void __launch_bounds__(128) k_pgs(Dev d, PgsLayout L) {
  extern __shared__ __align__(16) unsigned char smp[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int e = blockIdx.x * (blockDim.x >> 5) + wib;
  if (e >= d.E) return;
  PgsCtx X;
  X.d = &d;
  X.s = pgs_carve(smp + (size_t)wib * L.bytes(), L);
  X.e = e;
  X.C = d.C;
  const EnvInfo ei = env_info(d, e);
  X.nobj = ei.nobj;
  const int nct = d.n_contacts[e];
  X.nct = nct;
  const int nlim = d.n_limit[e];
  const int nu = nct + nlim;
  const float dt = d.dt;

  // ---- stage bodies
  for (int c = lane; c < ei.nobj; c += 32) {
    int k = ei.o0 + c;
    float4 v = d.obj_vstar[k], w = d.obj_wstar[k];
    X.s.v[3 * c] = v.x; X.s.v[3 * c + 1] = v.y; X.s.v[3 * c + 2] = v.z;
    X.s.w[3 * c] = w.x; X.s.w[3 * c + 1] = w.y; X.s.w[3 * c + 2] = w.z;
    float4 inv = d.obj_inv[k];
    M3 I = inv_inertia_world(d.obj_quat[k], inv);
    X.s.im[c] = inv.x;
    float* Ii = X.s.Ii + 6 * c;
    Ii[0] = I.r0.x; Ii[1] = I.r0.y; Ii[2] = I.r0.z; Ii[3] = I.r1.y; Ii[4] = I.r1.z; Ii[5] = I.r2.z;
  }
  for (int t = lane; t < ei.narts * MAX_DOF; t += 32) X.s.qd[t] = 0.f;
  __syncwarp();
  for (int t = lane; t < ei.nlink; t += 32) {
    int jg = ei.l0 + t;
    int art = d.j_art[jg];
    X.s.qd[(art - ei.a0) * MAX_DOF + (jg - d.joint_off[art])] = d.j_qdstar[jg];
  }
  // ---- impulses: warm start (prior frame in r_lam; learned network output if present)
  for (int u = lane; u < nu; u += 32) {
    float* lam = X.s.lam + 3 * u;
    if (u < nct) {
      size_t g = (size_t)e * X.C + u;
      float4 l0 = d.r_lam[g];
      if (d.warm_mode == 2) {
        float4 y = d.pred[g];
        if (isfinite(y.x) && isfinite(y.y) && isfinite(y.z)) {
          float4 me = d.r_meff[g];
          float mu = d.r_t1[g].w;
          float sc = me.x * sqrtf(d.gx * d.gx + d.gy * d.gy + d.gz * d.gz) * dt;
          float ln = fmaxf(0.f, y.x * sc);
          l0 = make_float4(ln, fmaxf(-mu * ln, fminf(mu * ln, y.y * sc)), fmaxf(-mu * ln, fminf(mu * ln, y.z * sc)), 0.f);
        }
      }
      lam[0] = l0.x; lam[1] = l0.y; lam[2] = l0.z;
    } else {
      lam[0] = d.lr_data[(size_t)e * LCAP + (u - nct)].z;
      lam[1] = lam[2] = 0.f;
    }
  }
  // ---- greedy colouring in unit order (lane 0), counting sort by colour
  const int nnodes = ei.nobj + ei.narts;
  for (int t = lane; t < nnodes; t += 32) X.s.used[t] = 0ull;
  __syncwarp();
  int ncol = 0;
  if (lane == 0) {
    int counts[66];
    for (int c = 0; c < 66; ++c) counts[c] = 0;
    for (int u = 0; u < nu; ++u) {
      int na, nb;
      if (u < nct) {
        int2 ends = d.r_ends[(size_t)e * X.C + u];
        na = unit_node(ei, ends.x);
        nb = unit_node(ei, ends.y);
      } else {
        na = ei.nobj + d.lr_info[(size_t)e * LCAP + (u - nct)].x;
        nb = -1;
      }
      unsigned long long m = (na >= 0 ? X.s.used[na] : 0ull) | (nb >= 0 ? X.s.used[nb] : 0ull);
      int c = (~m == 0ull) ? 64 : __ffsll((long long)~m) - 1;
      if (c < 64) {
        if (na >= 0) X.s.used[na] |= 1ull << c;
        if (nb >= 0) X.s.used[nb] |= 1ull << c;
      }
      X.s.colour[u] = c;
      counts[c]++;
      ncol = max(ncol, c + 1);
    }
    int acc = 0;
    for (int c = 0; c < ncol; ++c) { X.s.cstart[c] = acc; acc += counts[c]; counts[c] = X.s.cstart[c]; }
    X.s.cstart[ncol] = acc;
    for (int u = 0; u < nu; ++u) X.s.order[counts[X.s.colour[u]]++] = u;
  }
  ncol = __shfl_sync(0xffffffffu, ncol, 0);
  __syncwarp();
  float dummy0 = 0.f, dummy1 = 0.f;
  // apply the warm start colour by colour
  for (int c = 0; c < ncol; ++c) {
    int b = X.s.cstart[c], en = X.s.cstart[c + 1];
    if (c == 64) {
      if (lane == 0)
        for (int k = b; k < en; ++k) do_unit(X, X.s.order[k], 1, dummy0, dummy1);
    } else {
      for (int k = b + lane; k < en; k += 32) do_unit(X, X.s.order[k], 1, dummy0, dummy1);
    }
    __syncwarp();
  }
  // ---- sweeps
  const int max_it = d.pgs_tol > 0.f ? d.pgs_max_iters : d.pgs_iters;
  int it = 0;
  float resid = 0.f;
  unsigned status = 0;
  if (nu > 0) {
    for (it = 1; it <= max_it; ++it) {
      float d2 = 0.f, l2 = 0.f;
      for (int c = 0; c < ncol; ++c) {
        int b = X.s.cstart[c], en = X.s.cstart[c + 1];
        if (c == 64) {
          if (lane == 0)
            for (int k = b; k < en; ++k) do_unit(X, X.s.order[k], 0, d2, l2);
        } else {
          for (int k = b + lane; k < en; k += 32) do_unit(X, X.s.order[k], 0, d2, l2);
        }
        __syncwarp();
      }
      d2 = warp_sum(d2);
      l2 = warp_sum(l2);
      resid = sqrtf(d2) / fmaxf(sqrtf(l2), d.lambda_floor);
      if (d.pgs_tol > 0.f && resid <= d.pgs_tol) break;
    }
    if (it > max_it) {
      it = max_it;
      if (d.pgs_tol > 0.f) status |= ST_ITER_CAP;
    }
  }
  __syncwarp();
  // ---- write back velocities, impulses, warm-start cache, limit impulses
  for (int c = lane; c < ei.nobj; c += 32) {
    int k = ei.o0 + c;
    d.obj_vel[k] = make_float4(X.s.v[3 * c], X.s.v[3 * c + 1], X.s.v[3 * c + 2], 0.f);
    d.obj_omega[k] = make_float4(X.s.w[3 * c], X.s.w[3 * c + 1], X.s.w[3 * c + 2], 0.f);
  }
  for (int t = lane; t < ei.nlink; t += 32) {
    int jg = ei.l0 + t;
    int art = d.j_art[jg];
    d.j_qd[jg] = X.s.qd[(art - ei.a0) * MAX_DOF + (jg - d.joint_off[art])];
    d.j_lim_side[jg] = 0;
    d.j_lim_lambda[jg] = 0.f;
  }
  for (int u = lane; u < nct; u += 32) {
    size_t g = (size_t)e * X.C + u;
    const float* lam = X.s.lam + 3 * u;
    V3 n = v3(d.c_n[g]);
    V3 t1 = v3(d.r_t1[g]);
    V3 t2 = cross(n, t1);
    V3 lt = t1 * lam[1] + t2 * lam[2];
    d.c_lam[g] = make_float4(lam[0], lam[1], lam[2], 0.f);
    d.cache_key[g] = d.c_key[g];
    d.cache_p[g] = d.c_p[g];
    d.cache_lam[g] = make_float4(lam[0], lt.x, lt.y, lt.z);
  }
  __syncwarp();
  for (int l = lane; l < nlim; l += 32) {
    int4 info = d.lr_info[(size_t)e * LCAP + l];
    d.j_lim_side[info.w] = info.z > 0 ? 1 : 2;
    d.j_lim_lambda[info.w] = X.s.lam[3 * (nct + l)];
  }
  if (lane == 0) {
    d.cache_count[e] = nct;
    d.iters[e] = it;
    d.resid[e] = resid;
    d.n_colours[e] = ncol;
    if (status) atomicOr(&d.status[e], (int)status);
  }
}

// ---------------------------------------------------------------------------
// k_integrate
// ---------------------------------------------------------------------------
__global__ void k_integrate(Dev d) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  const float dt = d.dt;
  if (i < d.NO) {
    if (!d.obj_awake[i]) return;
    float4 x = d.obj_pos[i], c = d.obj_comp[i], v = d.obj_vel[i], w = d.obj_omega[i], q = d.obj_quat[i];
    // Kahan-compensated x += dt v
    float xs[3] = {x.x, x.y, x.z}, cs[3] = {c.x, c.y, c.z}, vs[3] = {v.x, v.y, v.z};
    for (int k = 0; k < 3; ++k) {
      float y = __fsub_rn(__fmul_rn(dt, vs[k]), cs[k]);
      float t = __fadd_rn(xs[k], y);
      cs[k] = __fsub_rn(__fsub_rn(t, xs[k]), y);
      xs[k] = t;
    }
    d.obj_pos[i] = make_float4(xs[0], xs[1], xs[2], 0.f);
    d.obj_comp[i] = make_float4(cs[0], cs[1], cs[2], 0.f);
    // q <- normalize(q + dt/2 (0, w) q)
    float hw = 0.5f * dt;
    float qw = q.x, qx = q.y, qy = q.z, qz = q.w;
    float dw = -(w.x * qx + w.y * qy + w.z * qz);
    float dx = qw * w.x + (w.y * qz - w.z * qy);
    float dy = qw * w.y + (w.z * qx - w.x * qz);
    float dz = qw * w.z + (w.x * qy - w.y * qx);
    qw = qw + hw * dw; qx = qx + hw * dx; qy = qy + hw * dy; qz = qz + hw * dz;
    float qn = sqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
    d.obj_quat[i] = make_float4(qw / qn, qx / qn, qy / qn, qz / qn);
    bool bad = !(isfinite(xs[0]) && isfinite(xs[1]) && isfinite(xs[2]) && isfinite(v.x) && isfinite(v.y) &&
                 isfinite(v.z) && isfinite(w.x) && isfinite(w.y) && isfinite(w.z));
    if (d.sleep_enabled) {
      float vn = sqrtf(v.x * v.x + v.y * v.y + v.z * v.z), wn = sqrtf(w.x * w.x + w.y * w.y + w.z * w.z);
      int ctr = (vn < d.sleep_lin && wn < d.sleep_ang) ? d.obj_ctr[i] + 1 : 0;
      d.obj_ctr[i] = ctr;
      if (ctr >= d.sleep_steps) {
        d.obj_awake[i] = 0;
        d.obj_vel[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        d.obj_omega[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    if (bad) atomicOr(&d.status[d.obj_env[i]], ST_NUMERIC);
    return;
  }
  int j = i - d.NO;
  if (j < d.NJ) {
    float q = d.j_q[j], c = d.j_qcomp[j], qd = d.j_qd[j];
    float y = __fsub_rn(__fmul_rn(dt, qd), c);
    float t = __fadd_rn(q, y);
    d.j_qcomp[j] = __fsub_rn(__fsub_rn(t, q), y);
    d.j_q[j] = t;
    if (!(isfinite(t) && isfinite(qd))) atomicOr(&d.status[d.j_env[j]], ST_NUMERIC);
  }
}

void launch_rows(const Dev& d, cudaStream_t st) {
  if (d.E == 0) return;
  k_rows<<<(d.E + 3) / 4, 128, 0, st>>>(d);
}

void configure_pgs(int C) {
  PgsLayout L{C};
  cudaFuncSetAttribute(k_pgs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(L.bytes() * 4));
}

void launch_pgs(const Dev& d, cudaStream_t st) {
  if (d.E == 0) return;
  PgsLayout L{d.C};
  const int warps = 4;
  k_pgs<<<(d.E + warps - 1) / warps, 32 * warps, L.bytes() * warps, st>>>(d, L);
}

void launch_integrate(const Dev& d, cudaStream_t st) {
  int n = d.NO + d.NJ;
  if (n == 0) return;
  k_integrate<<<(n + 255) / 256, 256, 0, st>>>(d);
}

}  // namespace gb
