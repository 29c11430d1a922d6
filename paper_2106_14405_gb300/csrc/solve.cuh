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
//   the environment's bodies, rows and impulses live in shared memory;
//   constraint units (a contact's three rows, or a limit row) get greedy
//   colours in (a, b, feature) order -- an articulation is one node, statics
//   are none -- so units of one colour touch disjoint bodies and the lanes
//   update them in parallel with exactly the arithmetic of a sequential sweep
//   in colour order.  Friction is clamped to mu times the contact's current
//   normal impulse.  Relative residual ||Δλ|| / max(||λ||, floor) per sweep by
//   warp reduction.
// Integration, in the same warp at the end of an environment's solve (one lane
//   per object or joint): semi-implicit Euler with Kahan-compensated position
//   sums, quaternion update, sleeping.
#pragma once
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

__device__ __forceinline__ void endpoint_rows(const Dev& d, const EnvInfo& ei, int e, int c, V3 p, const V3* dir, int slot,
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
    o.code = ART_TAG | ((art - ei.a0) << 8) | slot;
    o.x = v3(d.l_com[jg]);
    o.mu = d.j_half[jg].w;
    float* J = d.ap + ((size_t)e * APOOL + slot) * APS;  // rows at 0, 12, 24
    float* W = J + 36;                                  // rows at 36, 48, 60
    const float* Mi = d.a_minv + (size_t)art * 81;
    // the link's ancestors (itself included) as a bit set; then one row at a time:
    // J_r over the joints (zero off the path) and W_r = M^-1 J_r, unrolled so the
    // row stays in registers (the link data and M^-1 come from L1 after the first row)
    const unsigned anc = d.j_anc[jg];
    // (the row loop stays rolled to bound the code size; the row's direction and its
    //  results are selected with constant indices so that nothing lands in local memory)
#pragma unroll 1
    for (int r = 0; r < 3; ++r) {
      const V3 dr = r == 0 ? dir[0] : (r == 1 ? dir[1] : dir[2]);
      float jv[MAX_DOF];
#pragma unroll
      for (int i = 0; i < MAX_DOF; ++i) {
        V3 sp = v3(0.f, 0.f, 0.f);
        if ((anc >> i) & 1u) {
          const float4 a4 = d.l_ja[jb + i];
          const V3 a = v3(a4);
          sp = a4.w == 0.f ? cross(a, p - v3(d.l_jo[jb + i])) : a;
        }
        jv[i] = dot(dr, sp);
      }
      // both rows as three 16-byte stores each (the padding entries 9-11 written as
      // zeros: the solver stages its own values there)
      float4* J4 = reinterpret_cast<float4*>(J + 12 * r);
      float4* W4 = reinterpret_cast<float4*>(W + 12 * r);
      J4[0] = make_float4(0 < n ? jv[0] : 0.f, 1 < n ? jv[1] : 0.f, 2 < n ? jv[2] : 0.f, 3 < n ? jv[3] : 0.f);
      J4[1] = make_float4(4 < n ? jv[4] : 0.f, 5 < n ? jv[5] : 0.f, 6 < n ? jv[6] : 0.f, 7 < n ? jv[7] : 0.f);
      J4[2] = make_float4(8 < n ? jv[8] : 0.f, 0.f, 0.f, 0.f);
      float kk = 0.f, vv = 0.f;
      float wq[4];
#pragma unroll
      for (int i = 0; i < MAX_DOF; ++i) {  // zero beyond n: the solver sums all MAX_DOF entries
        float w = 0.f;
        if (i < n) {
#pragma unroll
          for (int k = 0; k < MAX_DOF; ++k)
            if (k < n) w += Mi[9 * i + k] * jv[k];
          kk += jv[i] * w;
          vv += jv[i] * d.j_qdstar[jb + i];
        }
        wq[i & 3] = w;
        if ((i & 3) == 3) W4[i >> 2] = make_float4(wq[0], wq[1], wq[2], wq[3]);
      }
      static_assert(MAX_DOF == 9, "three 16-byte stores per row");
      W4[2] = make_float4(wq[0], 0.f, 0.f, 0.f);
      if (r == 0) { o.k[0] = kk; o.vel[0] = vv; }
      else if (r == 1) { o.k[1] = kk; o.vel[1] = vv; }
      else { o.k[2] = kk; o.vel[2] = vv; }
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

__device__ __forceinline__ void rows_env(const Dev& d, const int e, const int lane) {
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
      // the contact set changes little between steps: probe the same index first,
      // then bisect the side it leaves
      int lo = 0, hi = ncache - 1, found = -1;
      if (ncache > 0) {
        const int g = min(i, ncache - 1);
        int4 k = d.cache_key[(size_t)e * C + g];
        bool less = k.x < key.x || (k.x == key.x && (k.y < key.y || (k.y == key.y && k.z < key.z)));
        bool eq = k.x == key.x && k.y == key.y && k.z == key.z;
        if (eq) found = g;
        else if (less) lo = g + 1;
        else hi = g - 1;
      }
      while (found < 0 && lo <= hi) {
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
    // learned warm start: the network serves the contacts without a prior-frame match and
    // the matched ones moving faster than LEARN_GATE |g| dt relative to each other; they
    // are listed for the inference kernel and flagged in the warm start's w lane
    bool use_net = false;
    if (d.warm_mode == 2) {
      const float vr2 = (A.vel[0] - B.vel[0]) * (A.vel[0] - B.vel[0]) + (A.vel[1] - B.vel[1]) * (A.vel[1] - B.vel[1]) +
                        (A.vel[2] - B.vel[2]) * (A.vel[2] - B.vel[2]);
      use_net = !matched || sqrtf(vr2) > LEARN_GATE * gdt;
      const unsigned am = __activemask();
      const unsigned bal = __ballot_sync(am, use_net);
      if (bal) {
        const int leader = __ffs(am) - 1;
        int base = 0;
        if (lane == leader) base = atomicAdd(d.mlp_count, __popc(bal));
        base = __shfl_sync(am, base, leader);
        if (use_net) d.mlp_rows[base + __popc(bal & ((1u << lane) - 1u))] = (int)gi;
      }
    }
    d.r_t1[gi] = f4(dir[1], mu);
    d.r_meff[gi] = make_float4(meff[0], meff[1], meff[2], tgt);
    d.r_lam[gi] = d.warm_mode >= 1 ? make_float4(prev[0], prev[1], prev[2], use_net ? 1.f : 0.f)
                                   : make_float4(0.f, 0.f, 0.f, 0.f);
    d.r_ra[gi] = f4(A.r, 0.f);
    d.r_rb[gi] = f4(B.r, 0.f);
    d.r_ends[gi] = make_int2(A.code, B.code);
    // the features: for the contact log (every contact), else only for the rows the
    // network serves (nothing else reads them)
    if (want_feat && (d.log_features || use_net)) {
      // (32 values in the order n, r_a, r_b, v_rel, w_rel, separation, inverse masses,
      // effective masses, mu, (g . n) dt, prior impulses, matched, pair type one-hot;
      // eight 16-byte stores)
      float4* f = reinterpret_cast<float4*>(d.feat + gi * NFEAT);
      const V3 ra = p - A.x, rb = p - B.x;
      const V3 wr = A.w - B.w;
      // pair type: 0 sphere-sphere, 1 sphere-plane, 2 sphere-box, 3 box-plane, 4 box-box
      const bool sphA = key.x < ei.nobj && d.obj_half[ei.o0 + key.x].w == 0.f;
      const bool sphB = key.y < ei.nobj && d.obj_half[ei.o0 + key.y].w == 0.f;
      const bool plane = d.env_plane[e] &&
                         key.y == ei.nobj + ei.nlink + (d.base_off[e + 1] - d.base_off[e]) + (d.stat_off[e + 1] - ei.s0);
      const int type = (sphA && sphB) ? 0 : (plane ? (sphA ? 1 : 3) : ((sphA || sphB) ? 2 : 4));
      auto hot = [&](int t) { return t == type ? 1.f : 0.f; };
      f[0] = make_float4(n.x, n.y, n.z, ra.x);
      f[1] = make_float4(ra.y, ra.z, rb.x, rb.y);
      f[2] = make_float4(rb.z, A.vel[0] - B.vel[0], A.vel[1] - B.vel[1], A.vel[2] - B.vel[2]);
      f[3] = make_float4(wr.x, wr.y, wr.z, sep);
      f[4] = make_float4(A.inv_m, B.inv_m, meff[0], meff[1]);
      f[5] = make_float4(meff[2], mu, dot(g, n) * dt, prev[0]);
      f[6] = make_float4(prev[1], prev[2], (float)matched, hot(0));
      f[7] = make_float4(hot(1), hot(2), hot(3), hot(4));
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
  // joint motors (motor mode, the paper's Sec. 5.1 "Action space"): a row on q̇ of every
  // joint of a kinematic-base articulation, target rate motor_kp (q̄ - q) / dt, impulse
  // within +-motor_max_impulse; after the limit rows, (articulation, joint) order
  if (d.motor_mode)
    for (int t0 = 0; t0 < ei.nlink; t0 += 32) {
      const int t = t0 + lane;
      const int jg = ei.l0 + t;
      const bool on = t < ei.nlink && d.art_kin[d.j_art[jg]] != 0;
      const unsigned m = __ballot_sync(0xffffffffu, on);
      if (on) {
        const int pos = nlim + __popc(m & ((1u << lane) - 1u));
        if (pos < LCAP) {
          const int art = d.j_art[jg];
          const int jb = d.joint_off[art];
          const int n = d.joint_off[art + 1] - jb;
          const int jl = jg - jb;
          const float* Mi = d.a_minv + (size_t)art * 81;
          const float tgt = d.motor_kp * (d.j_target[jg] - d.j_q[jg]) / dt;
          const float lam0 = d.warm_mode >= 1 ? d.j_motor_lambda[jg] : 0.f;
          const size_t li = (size_t)e * LCAP + pos;
          d.lr_info[li] = make_int4(art - ei.a0, jl, 0, jg);
          d.lr_data[li] = make_float4(1.f / Mi[9 * jl + jl], tgt, lam0, d.motor_max_impulse);
          for (int i = 0; i < MAX_DOF; ++i) d.lr_w[li * MAX_DOF + i] = i < n ? Mi[9 * i + jl] : 0.f;
        }
      }
      nlim += __popc(m);
    }
  if (nlim > LCAP) { status |= ST_OVERFLOW; nlim = LCAP; }
  status = __reduce_or_sync(0xffffffffu, status);
  if (lane == 0) {
    d.ap_count[e] = min(pool, APOOL);
    d.n_limit[e] = nlim;
    d.n_rows[e] = 3 * nct + nlim;
    if (status) atomicOr(&d.status[e], (int)status);
  }
}


// ---------------------------------------------------------------------------
// k_pgs
//
// Shared memory per warp (one environment), capacities fixed per launch from
// the batch: bodies, articulation rates, the first S contact units' rows and
// impulses, the first LS limit rows, the first AS articulation row endpoints
// (J and M^-1 J), colours and the colour-sorted order.  Units beyond the staged
// capacities are read from the global row buffers (same arithmetic).
// A unit is one contact (its normal and two friction rows) or one joint-limit
// row.  Units are coloured greedily in unit order so that the units of one
// colour touch disjoint bodies and articulations; within a colour the lanes
// take one unit each (an articulation's nine joint rates sit in the lane's
// registers for the unit), and the overflow colour runs on one lane in unit
// order.  Colours run in ascending order, which is the Gauss-Seidel order the
// oracle implements.
// ---------------------------------------------------------------------------
constexpr int CREC = 20;  // n(3) t1(3) ra(3) rb(3) meff(3) target mu ends a, b (int) pad: five float4
constexpr int BREC = 16;  // body: v(3) 1/m | w(3) I_xx | I_xy I_xz I_yy I_yz | I_zz pad(3): world inverse inertia
constexpr int QS = 12;    // joint rates of one articulation, padded to three float4
// one articulation row endpoint: APS floats, J rows at 0, 12, 24 (J M^-1 J^T below the
// diagonal in the rows' padding once staged), M^-1 J^T rows at 36, 48, 60
constexpr int LREC = 16;  // w(9) meff target lambda info(int) bound pad(2)
constexpr int ART_FLAG = 1 << 15;

struct PgsLayout {
  int C, S, nobj, narts, LS, AS;
  int bar_floor;  // lowest offset of the mbarrier: 0, or above the other stages' working
                  // sets where the fused step kernel shares the memory among the stages
  __host__ __device__ int units() const { return C + LCAP; }
  __host__ __device__ size_t off_used() const { return 0; }
  __host__ __device__ size_t off_body() const { return al(off_used() + 8 * (size_t)(nobj + narts)); }
  __host__ __device__ size_t off_qd() const { return al(off_body() + 4 * (size_t)BREC * nobj); }
  __host__ __device__ size_t off_crec() const { return al(off_qd() + 4 * (size_t)QS * narts); }
  __host__ __device__ size_t off_clam() const { return al(off_crec() + 4 * (size_t)CREC * S); }
  __host__ __device__ size_t off_lrec() const { return al(off_clam() + 16 * (size_t)S); }
  __host__ __device__ size_t off_ap() const { return al(off_lrec() + 4 * (size_t)LREC * LS); }
  __host__ __device__ size_t off_colour() const { return al(off_ap() + 4 * (size_t)APS * AS); }
  __host__ __device__ size_t off_order() const { return al(off_colour() + (size_t)units()); }
  __host__ __device__ size_t off_cstart() const { return al(off_order() + 2 * (size_t)units()); }
  __host__ __device__ size_t off_bar() const {  // after the colour starts, then counts
    const size_t b = al(off_cstart() + 4 * 132);
    return b > (size_t)bar_floor ? b : al((size_t)bar_floor);
  }
  __host__ __device__ size_t bytes() const { return al(off_bar() + 8); }  // mbarrier of the pool's bulk copy
  __host__ __device__ static size_t al(size_t x) { return (x + 15) & ~(size_t)15; }
};

PgsLayout pgs_layout(const Dev& d, int max_obj, int max_arts, int stage_contacts, int stage_pool);

struct PgsCtx {
  const Dev* d;
  PgsLayout L;
  unsigned long long* used;  // colour masks per node
  float *body, *qd, *crec, *clam, *lrec, *ap;
  unsigned char* colour;
  unsigned short* order;
  int* cstart;
  int e, nct, nlim, S, LS, AS;
  size_t gbase;  // e * C
};

// 16-byte shared-memory accesses (every record above starts on a 16-byte boundary)
__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }

struct Body {
  V3 v, w;
  float im, I[6];  // inverse mass, world inverse inertia as xx xy xz yy yz zz
};
__device__ __forceinline__ void body_load(const PgsCtx& X, int b, Body& B) {
  const float* p = X.body + BREC * b;
  const float4 a = ld4(p), c = ld4(p + 4), e = ld4(p + 8), f = ld4(p + 12);
  B.v = v3(a.x, a.y, a.z);
  B.im = a.w;
  B.w = v3(c.x, c.y, c.z);
  B.I[0] = c.w; B.I[1] = e.x; B.I[2] = e.y; B.I[3] = e.z; B.I[4] = e.w; B.I[5] = f.x;
}
__device__ __forceinline__ void body_store(const PgsCtx& X, int b, const Body& B) {
  float* p = X.body + BREC * b;
  st4(p, make_float4(B.v.x, B.v.y, B.v.z, B.im));
  st4(p + 4, make_float4(B.w.x, B.w.y, B.w.z, B.I[0]));
}
__device__ __forceinline__ V3 sym_mv(const float* I, V3 a) {  // symmetric 3x3 as xx xy xz yy yz zz
  return v3(I[0] * a.x + I[1] * a.y + I[2] * a.z, I[1] * a.x + I[3] * a.y + I[4] * a.z,
            I[2] * a.x + I[4] * a.y + I[5] * a.z);
}

struct ContactRow {
  V3 n, t1, ra, rb;
  float meff[3], tgt, mu;
  int ea, eb;
};

template <bool SMALL>
__device__ __forceinline__ void contact_load(const PgsCtx& X, int u, ContactRow& c, float* lam) {
  if (SMALL || u < X.S) {
    const float* r = X.crec + CREC * u;
    const float4 a = ld4(r), b = ld4(r + 4), q = ld4(r + 8), m = ld4(r + 12), z = ld4(r + 16);
    c.n = v3(a.x, a.y, a.z); c.t1 = v3(a.w, b.x, b.y);
    c.ra = v3(b.z, b.w, q.x); c.rb = v3(q.y, q.z, q.w);
    c.meff[0] = m.x; c.meff[1] = m.y; c.meff[2] = m.z; c.tgt = m.w; c.mu = z.x;
    c.ea = __float_as_int(z.y);
    c.eb = __float_as_int(z.z);
    const float4 l = ld4(X.clam + 4 * u);
    lam[0] = l.x; lam[1] = l.y; lam[2] = l.z;
  } else {
    const Dev& d = *X.d;
    size_t g = X.gbase + u;
    c.n = v3(d.c_n[g]);
    float4 t = d.r_t1[g];
    c.t1 = v3(t); c.mu = t.w;
    float4 me = d.r_meff[g];
    c.meff[0] = me.x; c.meff[1] = me.y; c.meff[2] = me.z; c.tgt = me.w;
    c.ra = v3(d.r_ra[g]); c.rb = v3(d.r_rb[g]);
    int2 en = d.r_ends[g];
    c.ea = en.x; c.eb = en.y;
    float4 l = d.r_lam[g];
    lam[0] = l.x; lam[1] = l.y; lam[2] = l.z;
  }
}
template <bool SMALL>
__device__ __forceinline__ void contact_store_lam(const PgsCtx& X, int u, const float* lam) {
  if (SMALL || u < X.S) st4(X.clam + 4 * u, make_float4(lam[0], lam[1], lam[2], 0.f));
  else X.d->r_lam[X.gbase + u] = make_float4(lam[0], lam[1], lam[2], 0.f);
}

// Contact between objects and/or statics, one lane: one Gauss-Seidel update.
// SMALL: every row of the environment is staged in shared memory.
// Gauss-Seidel over the three rows (n, t1, t2) needs each row's relative velocity
// after the earlier rows' impulses.  With c_r = r x d_r and u_r = I^-1 c_r per body,
// that is v_r(0) + sum_{s<r} K[r][s] imp_s, K[r][s] = u_s . c_r summed over the
// two bodies (the linear terms d_r . d_s vanish: the directions are orthonormal),
// so each row is a few scalar operations and the bodies are updated once at the
// end, in the same order as row by row.
template <bool SMALL>
__device__ __forceinline__ void object_unit(const PgsCtx& X, int u, float& d2, float& l2) {
  ContactRow c;
  float lam[3];
  contact_load<SMALL>(X, u, c, lam);
  const V3 dirs[3] = {c.n, c.t1, cross(c.n, c.t1)};
  const bool ha = c.ea >= 0, hb = c.eb >= 0;
  // per body: velocity along the rows at the start, couplings, and u_r = I^-1 c_r
  V3 ua[3], ub[3], va, wa, vb, wb;
  float ima = 0.f, imb = 0.f;
  float v0[3] = {0.f, 0.f, 0.f}, k10 = 0.f, k20 = 0.f, k21 = 0.f;
  if (ha) {
    Body A;
    body_load(X, c.ea, A);
    va = A.v; wa = A.w; ima = A.im;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const V3 cr = cross(c.ra, dirs[r]);
      ua[r] = sym_mv(A.I, cr);
      v0[r] = dot(dirs[r], va) + dot(wa, cr);
      if (r >= 1) k10 = r == 1 ? dot(ua[0], cr) : k10;
      if (r == 2) { k20 = dot(ua[0], cr); k21 = dot(ua[1], cr); }
    }
  }
  if (hb) {
    Body B;
    body_load(X, c.eb, B);
    vb = B.v; wb = B.w; imb = B.im;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const V3 cr = cross(c.rb, dirs[r]);
      ub[r] = sym_mv(B.I, cr);
      v0[r] -= dot(dirs[r], vb) + dot(wb, cr);
      if (r == 1) k10 += dot(ub[0], cr);
      if (r == 2) { k20 += dot(ub[0], cr); k21 += dot(ub[1], cr); }
    }
  }
  float imp[3];
  const float n0 = fmaxf(0.f, lam[0] + c.meff[0] * (c.tgt - v0[0]));
  imp[0] = n0 - lam[0];
  const float lim = c.mu * n0;
  const float n1 = fmaxf(-lim, fminf(lim, lam[1] - c.meff[1] * (v0[1] + k10 * imp[0])));
  imp[1] = n1 - lam[1];
  const float n2 = fmaxf(-lim, fminf(lim, lam[2] - c.meff[2] * (v0[2] + k20 * imp[0] + k21 * imp[1])));
  imp[2] = n2 - lam[2];
  lam[0] = n0; lam[1] = n1; lam[2] = n2;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    d2 += imp[r] * imp[r];
    l2 += lam[r] * lam[r];
  }
  if (ha) {
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      va = va + dirs[r] * (ima * imp[r]);
      wa = wa + ua[r] * imp[r];
    }
    float* p = X.body + BREC * c.ea;
    p[0] = va.x; p[1] = va.y; p[2] = va.z;
    p[4] = wa.x; p[5] = wa.y; p[6] = wa.z;
  }
  if (hb) {
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      vb = vb + dirs[r] * (imb * -imp[r]);
      wb = wb + ub[r] * -imp[r];
    }
    float* p = X.body + BREC * c.eb;
    p[0] = vb.x; p[1] = vb.y; p[2] = vb.z;
    p[4] = wb.x; p[5] = wb.y; p[6] = wb.z;
  }
  contact_store_lam<SMALL>(X, u, lam);
}

// row `which` (0-2: J, 3-5: M^-1 J^T) of articulation row endpoint `slot`
template <bool SMALL>
__device__ __forceinline__ void pool_row(const PgsCtx& X, int slot, int which, float* out) {
  if (SMALL || slot < X.AS) {
    const float* p = X.ap + APS * slot + 12 * which;
    const float4 a = ld4(p), b = ld4(p + 4), c = ld4(p + 8);
    out[0] = a.x; out[1] = a.y; out[2] = a.z; out[3] = a.w;
    out[4] = b.x; out[5] = b.y; out[6] = b.z; out[7] = b.w; out[8] = c.x;
  } else {
    const Dev& d = *X.d;
    const float* g = d.ap + ((size_t)X.e * APOOL + slot) * APS + 12 * which;
#pragma unroll
    for (int i = 0; i < MAX_DOF; ++i) out[i] = g[i];
  }
}
__device__ __forceinline__ void rates_load(const PgsCtx& X, int art, float* q) {
  const float* p = X.qd + QS * art;
  const float4 a = ld4(p), b = ld4(p + 4), c = ld4(p + 8);
  q[0] = a.x; q[1] = a.y; q[2] = a.z; q[3] = a.w; q[4] = b.x; q[5] = b.y; q[6] = b.z; q[7] = b.w; q[8] = c.x;
}
__device__ __forceinline__ void rates_store(const PgsCtx& X, int art, const float* q) {
  float* p = X.qd + QS * art;
  st4(p, make_float4(q[0], q[1], q[2], q[3]));
  st4(p + 4, make_float4(q[4], q[5], q[6], q[7]));
  p[8] = q[8];
}

// Joint-limit row, one lane: q̇ += sign * column of M^-1 * Δλ.
template <bool SMALL>
__device__ __forceinline__ void limit_unit(const PgsCtx& X, int l, float& d2, float& l2) {
  float w[MAX_DOF];
  float meff, tgt, lam0, bound;
  int info;
  if (SMALL || l < X.LS) {
    const float* r = X.lrec + LREC * l;
    const float4 a = ld4(r), b = ld4(r + 4), c = ld4(r + 8), z = ld4(r + 12);
    w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w; w[4] = b.x; w[5] = b.y; w[6] = b.z; w[7] = b.w; w[8] = c.x;
    meff = c.y; tgt = c.z; lam0 = c.w;
    info = __float_as_int(z.x);
    bound = z.y;
  } else {
    size_t li = (size_t)X.e * LCAP + l;
    int4 in4 = X.d->lr_info[li];
    float4 ld = X.d->lr_data[li];
    const float* wg = X.d->lr_w + li * MAX_DOF;
#pragma unroll
    for (int i = 0; i < MAX_DOF; ++i) w[i] = wg[i];
    meff = ld.x; tgt = ld.y; lam0 = ld.z;
    info = in4.x | (in4.y << 8) | ((in4.z > 0 ? 1 : 0) << 16) | ((in4.z == 0 ? 1 : 0) << 17);
    bound = ld.w;
  }
  const bool motor = (info >> 17) & 1;
  const int art = info & 0xff, joint = (info >> 8) & 0xff;
  const float sgn = ((info >> 16) & 1) || motor ? 1.f : -1.f;
  float q[MAX_DOF];
  rates_load(X, art, q);
  float imp;
  float qj = q[0];
#pragma unroll
  for (int i = 1; i < MAX_DOF; ++i) qj = joint == i ? q[i] : qj;
  float v = sgn * qj;
  float nl = motor ? fmaxf(-bound, fminf(bound, lam0 + meff * (tgt - v))) : fmaxf(0.f, lam0 + meff * (tgt - v));
  imp = nl - lam0;
  d2 += imp * imp;
  l2 += nl * nl;
  if (SMALL || l < X.LS) X.lrec[LREC * l + 11] = nl;
  else X.d->lr_data[(size_t)X.e * LCAP + l].z = nl;
#pragma unroll
  for (int i = 0; i < MAX_DOF; ++i) q[i] += w[i] * imp;
  rates_store(X, art, q);
}

// Contact unit with an articulation endpoint, one lane.  The rows' articulation
// terms come from the pool: J (3 x 9), W = M^-1 J^T (3 x 9) and the 3 x 3 block
// JW = J M^-1 J^T (staged in the J rows' padding).  Gauss-Seidel over the three
// rows needs J_r q after the earlier rows' impulses, which is J_r q0 + sum_{s<r}
// JW[r][s] e_s (e_s the impulse with the endpoint's sign); the other endpoint, an
// object, adds its velocity along the row at the start plus sum_{s<r} K[r][s]
// imp_s as in object_unit.  The three starting velocities are independent dot
// products, each row is then a few scalar operations, and q += sum_r W_r e_r
// (and the object's update) once at the end -- the same sweep as updating the
// bodies after every row, with the dependent chain cut to scalars.
// the three entries of JW below the diagonal: JW[1][0], JW[2][0], JW[2][1]
template <bool SMALL>
__device__ __forceinline__ void jw_lower(const PgsCtx& X, int slot, float* jw) {
  if (SMALL || slot < X.AS) {
    const float* p = X.ap + APS * slot;
    jw[0] = p[12 + 9];
    jw[1] = p[24 + 9];
    jw[2] = p[24 + 10];
  } else {  // endpoint beyond the staged pool: form them from global memory
    float J[MAX_DOF], W[MAX_DOF];
    const int rs[3][2] = {{1, 0}, {2, 0}, {2, 1}};
    for (int k = 0; k < 3; ++k) {
      pool_row<SMALL>(X, slot, rs[k][0], J);
      pool_row<SMALL>(X, slot, 3 + rs[k][1], W);
      float acc = 0.f;
#pragma unroll
      for (int i = 0; i < MAX_DOF; ++i) acc += J[i] * W[i];
      jw[k] = acc;
    }
  }
}

template <bool SMALL>
__device__ __forceinline__ void art_unit(const PgsCtx& X, int u, float& d2, float& l2) {
  ContactRow c;
  float lam[3];
  contact_load<SMALL>(X, u, c, lam);
  const V3 dirs[3] = {c.n, c.t1, cross(c.n, c.t1)};
  const bool aa = c.ea >= ART_TAG, ba = c.eb >= ART_TAG;
  // at most one endpoint is read through each of these (the other endpoint may be an object or static)
  const int ecode = aa ? c.ea : c.eb;             // the articulation endpoint handled with registers
  const float esgn = aa ? 1.f : -1.f;
  const int ocode = aa ? c.eb : c.ea;             // the other endpoint
  const float osgn = aa ? -1.f : 1.f;
  const V3 orr = aa ? c.rb : c.ra;
  const bool other_art = aa && ba;
  const int slot = ecode & 0xff, art = (ecode >> 8) & 0xff;
  const int slot2 = c.eb & 0xff, art2 = (c.eb >> 8) & 0xff;  // rare: robot and a door or drawer
  float q[MAX_DOF];
  rates_load(X, art, q);
  const bool oobj = ocode >= 0 && ocode < ART_TAG;
  Body O;
  V3 uo[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) uo[r] = v3(0.f, 0.f, 0.f);
  // velocity along each row at the start (times the endpoint's sign convention
  // below) and the coupling K[r][s] (s < r) of row r to the impulse of row s
  float v0[3] = {0.f, 0.f, 0.f}, k10 = 0.f, k20 = 0.f, k21 = 0.f;
  if (oobj) {
    body_load(X, ocode, O);
    V3 co[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      co[r] = cross(orr, dirs[r]);
      uo[r] = sym_mv(O.I, co[r]);
      v0[r] = osgn * (dot(dirs[r], O.v) + dot(O.w, co[r]));
    }
    k10 = dot(uo[0], co[1]);
    k20 = dot(uo[0], co[2]);
    k21 = dot(uo[1], co[2]);
  }
  float imp[3];
  // J_r q0 of the endpoint(s) and the JW blocks
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    float J[MAX_DOF];
    pool_row<SMALL>(X, slot, r, J);
    float s0 = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll
    for (int i = 0; i < MAX_DOF; i += 3) {
      s0 += J[i] * q[i];
      s1 += J[i + 1] * q[i + 1];
      s2 += J[i + 2] * q[i + 2];
    }
    v0[r] += esgn * ((s0 + s1) + s2);
  }
  float jw[3];
  jw_lower<SMALL>(X, slot, jw);
  k10 += jw[0];
  k20 += jw[1];
  k21 += jw[2];
  if (other_art) {  // second articulation (endpoint B): -J_r q2 - sum_{s<r} JW2[r][s] (-imp_s)
    const float* q2 = X.qd + QS * art2;
    for (int r = 0; r < 3; ++r) {
      float J[MAX_DOF];
      pool_row<SMALL>(X, slot2, r, J);
      float t = 0.f;
      for (int i = 0; i < MAX_DOF; ++i) t += J[i] * q2[i];
      v0[r] -= t;
    }
    float jw2[3];
    jw_lower<SMALL>(X, slot2, jw2);
    k10 += jw2[0];
    k20 += jw2[1];
    k21 += jw2[2];
  }
  const float n0 = fmaxf(0.f, lam[0] + c.meff[0] * (c.tgt - v0[0]));
  imp[0] = n0 - lam[0];
  const float lim = c.mu * n0;
  const float n1 = fmaxf(-lim, fminf(lim, lam[1] - c.meff[1] * (v0[1] + k10 * imp[0])));
  imp[1] = n1 - lam[1];
  const float n2 = fmaxf(-lim, fminf(lim, lam[2] - c.meff[2] * (v0[2] + k20 * imp[0] + k21 * imp[1])));
  imp[2] = n2 - lam[2];
  lam[0] = n0; lam[1] = n1; lam[2] = n2;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    d2 += imp[r] * imp[r];
    l2 += lam[r] * lam[r];
  }
  // q += sum_r W_r e_r with e_r = esgn imp_r (and the second articulation's share)
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    float W[MAX_DOF];
    pool_row<SMALL>(X, slot, 3 + r, W);
    const float e = esgn * imp[r];
#pragma unroll
    for (int i = 0; i < MAX_DOF; ++i) q[i] += W[i] * e;
  }
  rates_store(X, art, q);
  if (other_art) {
    float* q2 = X.qd + QS * art2;
    for (int r = 0; r < 3; ++r) {
      float W[MAX_DOF];
      pool_row<SMALL>(X, slot2, 3 + r, W);
      for (int i = 0; i < MAX_DOF; ++i) q2[i] += W[i] * -imp[r];
    }
  }
  if (oobj) {
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const float oi = osgn * imp[r];
      O.v = O.v + dirs[r] * (O.im * oi);
      O.w = O.w + uo[r] * oi;
    }
    body_store(X, ocode, O);
  }
  contact_store_lam<SMALL>(X, u, lam);
}

// Endpoint codes and warm-start impulses of contact unit u.
template <bool SMALL>
__device__ __forceinline__ void unit_ends(const PgsCtx& X, int u, int& ea, int& eb) {
  if (SMALL || u < X.S) {
    const int* r = reinterpret_cast<const int*>(X.crec + CREC * u);
    ea = r[17];
    eb = r[18];
  } else {
    const int2 en = X.d->r_ends[X.gbase + u];
    ea = en.x;
    eb = en.y;
  }
}
template <bool SMALL>
__device__ __forceinline__ float4 unit_lam(const PgsCtx& X, int u) {
  return (SMALL || u < X.S) ? ld4(X.clam + 4 * u) : X.d->r_lam[X.gbase + u];
}

// The warm start (the pass before the sweeps): every unit's starting impulses enter
// its bodies and articulations at once.  Their sum does not depend on the order of
// the units, so instead of a pass per colour each value gets one owner lane that
// adds its units' shares in unit order -- an object: F = n l0 + t1 l1 + t2 l2 with
// sign s = +1 on endpoint A and -1 on B, v += s F / m, w += s I^-1 (r x F); a joint
// rate: s W_r l_r of the contact units on its articulation, then w l0 of its limit
// and motor rows.  Per chunk of G units, a match over the endpoints gives each object
// and articulation the bit mask of its units (kept in the colouring's scratch, free
// by now), so an owner visits only its own units.  One owner and a fixed order per
// value keep the result the same under every launch shape.
template <int G, bool SMALL>
__device__ __forceinline__ void warm_start_gather(const Dev& d, const PgsCtx& X, const EnvInfo& ei, const int gl,
                                                  const unsigned gm) {
  unsigned* mobj = reinterpret_cast<unsigned*>(X.used);  // [2 nobj]: units with the object as endpoint A, B
  unsigned* mart = mobj + 2 * ei.nobj;                   // [2 narts]: the same per articulation
  const int nm = 2 * (ei.nobj + ei.narts);
  const int sh = __ffs(gm) - 1;  // the group's first lane: bit k of a mask is unit u0 + k
  for (int u0 = 0; u0 < X.nct; u0 += G) {
    for (int t = gl; t < nm; t += G) mobj[t] = 0u;
    __syncwarp(gm);
    const int u = u0 + gl;
    int ea = -1, eb = -1;
    if (u < X.nct) unit_ends<SMALL>(X, u, ea, eb);
    const int oa = ea >= 0 && ea < ART_TAG ? ea : -1, ob = eb >= 0 && eb < ART_TAG ? eb : -1;
    const int aa = ea >= ART_TAG ? (ea >> 8) & 0xff : -1, ab = eb >= ART_TAG ? (eb >> 8) & 0xff : -1;
    const unsigned moa = __match_any_sync(gm, oa) >> sh, mob = __match_any_sync(gm, ob) >> sh;
    const unsigned maa = __match_any_sync(gm, aa) >> sh, mab = __match_any_sync(gm, ab) >> sh;
    if (oa >= 0) mobj[2 * oa] = moa;  // lanes sharing an endpoint store the same mask
    if (ob >= 0) mobj[2 * ob + 1] = mob;
    if (aa >= 0) mart[2 * aa] = maa;
    if (ab >= 0) mart[2 * ab + 1] = mab;
    __syncwarp(gm);
    for (int b = gl; b < ei.nobj; b += G) {
      const unsigned ma = mobj[2 * b];
      unsigned m = ma | mobj[2 * b + 1];
      if (!m) continue;
      Body B;
      body_load(X, b, B);
      do {
        const int k = __ffs(m) - 1;
        m &= m - 1;
        ContactRow c;
        float lam[3];
        contact_load<SMALL>(X, u0 + k, c, lam);
        const V3 F = c.n * lam[0] + c.t1 * lam[1] + cross(c.n, c.t1) * lam[2];
        const bool on_a = (ma >> k) & 1u;
        const float s = on_a ? 1.f : -1.f;
        B.v = B.v + F * (s * B.im);
        B.w = B.w + sym_mv(B.I, cross(on_a ? c.ra : c.rb, F)) * s;
      } while (m);
      body_store(X, b, B);
    }
    for (int t = gl; t < ei.nlink; t += G) {
      const int jg = ei.l0 + t;
      const int art = d.j_art[jg];
      const int a = art - ei.a0, i = jg - d.joint_off[art];
      const unsigned ma = mart[2 * a];
      unsigned m = ma | mart[2 * a + 1];
      if (!m) continue;
      float q = X.qd[QS * a + i];
      do {
        const int k = __ffs(m) - 1;
        m &= m - 1;
        int e0, e1;
        unit_ends<SMALL>(X, u0 + k, e0, e1);
        const float4 l = unit_lam<SMALL>(X, u0 + k);
        const float lam[3] = {l.x, l.y, l.z};
        // a contact between two links of one articulation has both endpoints on it
        const bool on[2] = {((ma >> k) & 1u) != 0u, e1 >= ART_TAG && ((e1 >> 8) & 0xff) == a};
#pragma unroll
        for (int side = 0; side < 2; ++side) {
          if (!on[side]) continue;
          const int slot = (side == 0 ? e0 : e1) & 0xff;
          const float sg = side == 0 ? 1.f : -1.f;
          const float* p = (SMALL || slot < X.AS) ? X.ap + APS * slot
                                                 : d.ap + ((size_t)X.e * APOOL + slot) * APS;
#pragma unroll
          for (int r = 0; r < 3; ++r) q += p[12 * (3 + r) + i] * (sg * lam[r]);
        }
      } while (m);
      X.qd[QS * a + i] = q;
    }
    __syncwarp(gm);
  }
  for (int t = gl; t < ei.nlink; t += G) {
    const int jg = ei.l0 + t;
    const int art = d.j_art[jg];
    const int a = art - ei.a0, i = jg - d.joint_off[art];
    float q = X.qd[QS * a + i];
    for (int l = 0; l < X.nlim; ++l) {
      int la;
      float w, l0;
      if (SMALL || l < X.LS) {
        const float* r = X.lrec + LREC * l;
        la = __float_as_int(r[12]) & 0xff;
        w = r[i];
        l0 = r[11];
      } else {
        const size_t li = (size_t)X.e * LCAP + l;
        la = d.lr_info[li].x;
        w = d.lr_w[li * MAX_DOF + i];
        l0 = d.lr_data[li].z;
      }
      if (la == a) q += w * l0;
    }
    X.qd[QS * a + i] = q;
  }
  __syncwarp(gm);
}

__device__ __forceinline__ int node_of(const EnvInfo& ei, int code) {
  if (code < 0) return -1;
  if (code < ART_TAG) return code;
  return ei.nobj + ((code >> 8) & 0xff);
}

// The warm start (a gather), then the sweeps, each unit routine instantiated once
// per SMALL.  Units of a colour touch disjoint bodies, so lanes take one unit
// each; the overflow colour (64) runs on one lane in unit order.  With `one_lane` (colours holding about one unit
// each) one lane runs every unit in colour order without a pass per colour: the
// same sweep, as units of a colour share no body.  Returns whether the residual
// target was met.
template <int G, bool SMALL>
__device__ __forceinline__ bool pgs_sweeps(const Dev& d, const PgsCtx& X, const EnvInfo& ei, const int ncol,
                                           const int max_it, const bool one_lane, const int gl, const unsigned gm,
                                           int& it, float& resid) {
  const int npass = one_lane ? 1 : ncol;
  warm_start_gather<G, SMALL>(d, X, ei, gl, gm);
  for (int sweep = 1; sweep <= max_it; ++sweep) {
    float d2 = 0.f, l2 = 0.f;
    for (int c = 0; c < npass; ++c) {
      const int b = one_lane ? 0 : X.cstart[c], en = X.cstart[one_lane ? ncol : c + 1];
      const bool serial = one_lane || c == 64;
      const int start = serial ? (gl == 0 ? b : en) : b + gl;
      const int stride = serial ? 1 : G;
      for (int k = start; k < en; k += stride) {
        const int ou = X.order[k];
        const int u = ou & (ART_FLAG - 1);
        if (!(ou & ART_FLAG)) object_unit<SMALL>(X, u, d2, l2);
        else if (u >= X.nct) limit_unit<SMALL>(X, u - X.nct, d2, l2);
        else art_unit<SMALL>(X, u, d2, l2);
      }
      __syncwarp(gm);
    }
    it = sweep;
    // the residual: after every sweep in residual mode, after the last one (for the
    // statistics) at a fixed sweep count
    if (d.pgs_tol > 0.f || sweep == max_it) {
      d2 = group_sum<G>(d2, gm);
      l2 = group_sum<G>(l2, gm);
      resid = sqrtf(d2) / fmaxf(sqrtf(l2), d.lambda_floor);
      if (d.pgs_tol > 0.f && resid <= d.pgs_tol) return true;
    }
  }
  return false;
}

// One free object: Kahan-compensated x += dt v, quaternion update, sleep counter.
__device__ __forceinline__ void integrate_object(const Dev& d, const int i) {
  const float dt = d.dt;
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
  if (bad) atomicOr(&d.status[d.obj_env[i] - d.env0], ST_NUMERIC);
}

// One joint: Kahan-compensated q += dt q̇.
__device__ __forceinline__ void integrate_joint(const Dev& d, const int j) {
  const float dt = d.dt;
  float q = d.j_q[j], c = d.j_qcomp[j], qd = d.j_qd[j];
  float y = __fsub_rn(__fmul_rn(dt, qd), c);
  float t = __fadd_rn(q, y);
  d.j_qcomp[j] = __fsub_rn(__fsub_rn(t, q), y);
  d.j_q[j] = t;
  if (!(isfinite(t) && isfinite(qd))) atomicOr(&d.status[d.j_env[j] - d.env0], ST_NUMERIC);
}

// Bulk copy (TMA engine) global -> shared memory completing on an mbarrier, and
// its bounded wait (0.5 s, then the caller falls back to plain loads).
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
  unsigned long long t0, t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  for (int it = 0; it < (1 << 26); ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (t - t0 > 500000000ull) return false;
  }
  return false;
}

template <int G>
__device__ __forceinline__ void pgs_env(const Dev& d, const PgsLayout& L, unsigned char* base, const int e,
                                        const int gl, const unsigned gm, const int g0, uint32_t& bar_phase,
                                        int& pending) {
  PgsCtx X;
  X.d = &d;
  X.L = L;
  X.used = reinterpret_cast<unsigned long long*>(base + L.off_used());
  X.body = reinterpret_cast<float*>(base + L.off_body());
  X.qd = reinterpret_cast<float*>(base + L.off_qd());
  X.crec = reinterpret_cast<float*>(base + L.off_crec());
  X.clam = reinterpret_cast<float*>(base + L.off_clam());
  X.lrec = reinterpret_cast<float*>(base + L.off_lrec());
  X.ap = reinterpret_cast<float*>(base + L.off_ap());
  X.colour = base + L.off_colour();
  X.order = reinterpret_cast<unsigned short*>(base + L.off_order());
  X.cstart = reinterpret_cast<int*>(base + L.off_cstart());
  const EnvInfo ei = env_info(d, e);
  X.e = e;
  X.nct = d.n_contacts[e];
  X.nlim = d.n_limit[e];
  X.S = L.S;
  X.LS = L.LS;
  // a group whose pool wait ran out earlier reads every pool row from global memory: a
  // late completion of the copy it gave up on could still land in its shared memory
  X.AS = bar_phase == 2u ? 0 : L.AS;
  X.gbase = (size_t)e * d.C;
  const int nct = X.nct, nlim = X.nlim, nu = nct + nlim;
  const float dt = d.dt;

  // ---- the articulation row pool: one bulk copy into shared memory (the global pool
  //      is kept in this layout), overlapping the rest of the staging
  unsigned status = 0;
  const int napool = min(d.ap_count[e], X.AS);
  const uint32_t ubar = (uint32_t)__cvta_generic_to_shared(base + L.off_bar());
  // (bar_phase 2: an earlier wait of this group ran out -- its barrier is retired and the
  //  group reads the pool from global memory; hold_async withholds the copy, for testing
  //  that path)
  if (napool > 0 && gl == 0 && bar_phase != 2u && !d.hold_async)
    bulk_copy_g2s(X.ap, d.ap + (size_t)e * APOOL * APS, (uint32_t)(napool * APS * 4), ubar);
  // ---- stage bodies, articulation rates, rows, limit rows
  for (int c = gl; c < ei.nobj; c += G) {
    int k = ei.o0 + c;
    float4 v = d.obj_vstar[k], w = d.obj_wstar[k];
    float4 inv = d.obj_inv[k];
    M3 I = inv_inertia_world(d.obj_quat[k], inv);
    float* p = X.body + BREC * c;
    st4(p, make_float4(v.x, v.y, v.z, inv.x));
    st4(p + 4, make_float4(w.x, w.y, w.z, I.r0.x));
    st4(p + 8, make_float4(I.r0.y, I.r0.z, I.r1.y, I.r1.z));
    st4(p + 12, make_float4(I.r2.z, 0.f, 0.f, 0.f));
  }
  for (int t = gl; t < ei.narts * QS; t += G) X.qd[t] = 0.f;
  __syncwarp(gm);
  for (int t = gl; t < ei.nlink; t += G) {
    int jg = ei.l0 + t;
    int art = d.j_art[jg];
    X.qd[(art - ei.a0) * QS + (jg - d.joint_off[art])] = d.j_qdstar[jg];
  }
  const float gnorm = sqrtf(d.gx * d.gx + d.gy * d.gy + d.gz * d.gz);
  const int ns = min(nct, X.S);
  for (int u = gl; u < ns; u += G) {
    size_t g = X.gbase + u;
    float* r = X.crec + CREC * u;
    float4 n = d.c_n[g], t = d.r_t1[g], me = d.r_meff[g], ra = d.r_ra[g], rb = d.r_rb[g];
    int2 en = d.r_ends[g];
    st4(r, make_float4(n.x, n.y, n.z, t.x));
    st4(r + 4, make_float4(t.y, t.z, ra.x, ra.y));
    st4(r + 8, make_float4(ra.z, rb.x, rb.y, rb.z));
    st4(r + 12, me);
    st4(r + 16, make_float4(t.w, __int_as_float(en.x), __int_as_float(en.y), 0.f));
  }
  // warm start (prior frame in r_lam; learned network output for the rows the row
  // kernel flagged in the w lane)
  for (int u = gl; u < nct; u += G) {
    size_t g = X.gbase + u;
    float4 l0 = d.r_lam[g];
    if (d.warm_mode == 2 && l0.w != 0.f) {
      float4 y = d.pred[g];
      if (isfinite(y.x) && isfinite(y.y) && isfinite(y.z)) {
        float4 me = d.r_meff[g];
        float mu = d.r_t1[g].w;
        // network output: correction to the prior-frame impulse (l0) in units of learn_scale
        float sc = learn_scale(me.x, d.feat + g * NFEAT, gnorm * dt);
        float ln = fmaxf(0.f, l0.x + y.x * sc);
        l0 = make_float4(ln, fmaxf(-mu * ln, fminf(mu * ln, l0.y + y.y * sc)),
                         fmaxf(-mu * ln, fminf(mu * ln, l0.z + y.z * sc)), 0.f);
      }
    }
    if (u < X.S) {
      st4(X.clam + 4 * u, make_float4(l0.x, l0.y, l0.z, 0.f));
    } else {
      d.r_lam[g] = make_float4(l0.x, l0.y, l0.z, 0.f);  // (unchanged unless learned)
    }
  }
  int nstaged = napool;
  if (napool > 0) {
    bool done = false;
    if (bar_phase != 2u) {
      done = __all_sync(gm, mbar_wait_bounded(ubar, bar_phase));
      if (!done && !d.hold_async) pending = (int)bar_phase;  // the copy may still be in flight
      bar_phase = done ? bar_phase ^ 1u : 2u;
    }
    if (!done) {  // the copy did not complete in time: flag the env, read the pool from global memory
      status |= ST_DEVICE_WAIT;
      X.AS = 0;
      nstaged = 0;
    }
  }
  __syncwarp(gm);
  for (int t = gl; t < nstaged * 9; t += G) {  // JW = J M^-1 J^T into the J rows' padding
    const int slot = t / 9, r = (t % 9) / 3, s2 = t % 3;
    const float* J = X.ap + APS * slot + 12 * r;
    const float* W = X.ap + APS * slot + 36 + 12 * s2;
    float acc = 0.f;
#pragma unroll
    for (int i = 0; i < MAX_DOF; ++i) acc += J[i] * W[i];
    X.ap[APS * slot + 12 * r + 9 + s2] = acc;
  }
  const int nls = min(nlim, X.LS);
  for (int t = gl; t < nls * LREC; t += G) {
    int l = t / LREC, k = t % LREC;
    size_t li = (size_t)e * LCAP + l;
    float val = 0.f;
    if (k < MAX_DOF) val = d.lr_w[li * MAX_DOF + k];
    else if (k == 9) val = d.lr_data[li].x;
    else if (k == 10) val = d.lr_data[li].y;
    else if (k == 11) val = d.lr_data[li].z;
    else if (k == 12) {
      int4 in4 = d.lr_info[li];
      val = __int_as_float(in4.x | (in4.y << 8) | ((in4.z > 0 ? 1 : 0) << 16) | ((in4.z == 0 ? 1 : 0) << 17));
    } else if (k == 13) {
      val = d.lr_data[li].w;
    }
    X.lrec[t] = val;
  }
  // ---- greedy colouring in unit order (lane 0) on the units' nodes, found by all lanes
  //      first (packed into the order array, free until the sort); then a stable
  //      counting sort by colour: per-colour counts, scan, scatter, with lanes of equal
  //      colour ranked by match_any.  Units touching an articulation are flagged.
  const int nnodes = ei.nobj + ei.narts;
  for (int t = gl; t < nnodes; t += G) X.used[t] = 0ull;
  for (int u = gl; u < nu; u += G) {
    int na, nb;
    if (u < nct) {
      int2 en;
      if (u < X.S) en = make_int2(__float_as_int(X.crec[CREC * u + 17]), __float_as_int(X.crec[CREC * u + 18]));
      else en = d.r_ends[X.gbase + u];
      na = node_of(ei, en.x);
      nb = node_of(ei, en.y);
    } else {
      na = ei.nobj + d.lr_info[(size_t)e * LCAP + (u - nct)].x;
      nb = -1;
    }
    X.order[u] = (unsigned short)((na + 1) | ((nb + 1) << 8));
  }
  __syncwarp(gm);
  int ncol = 0;
  if (gl == 0) {
    for (int u = 0; u < nu; ++u) {
      const int pk = X.order[u];
      const int na = (pk & 0xff) - 1, nb = (pk >> 8) - 1;
      unsigned long long m = (na >= 0 ? X.used[na] : 0ull) | (nb >= 0 ? X.used[nb] : 0ull);
      int c = (~m == 0ull) ? 64 : __ffsll((long long)~m) - 1;
      if (c < 64) {
        if (na >= 0) X.used[na] |= 1ull << c;
        if (nb >= 0) X.used[nb] |= 1ull << c;
      }
      const bool art = u >= nct || na >= ei.nobj || nb >= ei.nobj;
      X.colour[u] = (unsigned char)(c | (art ? 128 : 0));
      ncol = max(ncol, c + 1);
    }
  }
  ncol = __shfl_sync(gm, ncol, g0);
  int* run = X.cstart + 66;  // per-colour counts, then running positions
  for (int t = gl; t < 66; t += G) run[t] = 0;
  __syncwarp(gm);
  const unsigned lane_bit = 1u << (threadIdx.x & 31);
  for (int u0 = 0; u0 < nu; u0 += G) {
    const int u = u0 + gl;
    const int c = u < nu ? (X.colour[u] & 127) : -1;
    const unsigned same = __match_any_sync(gm, c);
    if (u < nu && (same & (lane_bit - 1u)) == 0u) run[c] += __popc(same);  // one lane per colour present
    __syncwarp(gm);
  }
  {  // exclusive scan of the counts over colours 0 .. ncol-1
    int carry = 0;
    for (int c0 = 0; c0 < ncol; c0 += G) {
      const int c = c0 + gl;
      const int k = c < ncol ? run[c] : 0;
      int incl = k;
      for (int o = 1; o < G; o <<= 1) {
        const int v = __shfl_up_sync(gm, incl, o, G);
        if (gl >= o) incl += v;
      }
      if (c < ncol) {
        X.cstart[c] = carry + incl - k;
        run[c] = carry + incl - k;
      }
      carry += __shfl_sync(gm, incl, G - 1, G);
    }
    if (gl == 0) X.cstart[ncol] = carry;
  }
  __syncwarp(gm);
  for (int u0 = 0; u0 < nu; u0 += G) {
    const int u = u0 + gl;
    const int cc = u < nu ? X.colour[u] : 0;
    const int c = u < nu ? (cc & 127) : -1;
    const unsigned same = __match_any_sync(gm, c);
    if (u < nu) X.order[run[c] + __popc(same & (lane_bit - 1u))] = (unsigned short)(u | ((cc & 128) ? ART_FLAG : 0));
    __syncwarp(gm);
    if (u < nu && (same & (lane_bit - 1u)) == 0u) run[c] += __popc(same);
    __syncwarp(gm);
  }

  __syncwarp(gm);
  // ---- the warm-start gather, then the sweeps.  Units of a colour touch disjoint
  //      bodies, so lanes take one unit each; the overflow colour (64) runs on one
  //      lane in unit order.
  const int max_it = d.pgs_tol > 0.f ? d.pgs_max_iters : d.pgs_iters;
  int it = 0;
  float resid = 0.f;
  if (nu > 0) {
    bool converged;
    // colours of about one unit each (an arm pressed into clutter: every unit on the
    // arm's node) run on one lane; environments whose rows all sit in shared memory
    // take the loop without global fallbacks
    const bool one_lane = 2 * nu <= 3 * ncol;
    if (nct <= X.S && nlim <= X.LS && d.ap_count[e] <= X.AS)
      converged = pgs_sweeps<G, true>(d, X, ei, ncol, max_it, one_lane, gl, gm, it, resid);
    else
      converged = pgs_sweeps<G, false>(d, X, ei, ncol, max_it, one_lane, gl, gm, it, resid);
    if (!converged && d.pgs_tol > 0.f) status |= ST_ITER_CAP;
  }
  __syncwarp(gm);
  // ---- write back velocities, impulses, warm-start cache, limit impulses; the lane
  //      that writes an object's or a joint's velocity integrates it (semi-implicit
  //      Euler, sleeping) -- the environment's step ends here
  for (int c = gl; c < ei.nobj; c += G) {
    int k = ei.o0 + c;
    const float4 v = ld4(X.body + BREC * c), w = ld4(X.body + BREC * c + 4);
    d.obj_vel[k] = make_float4(v.x, v.y, v.z, 0.f);
    d.obj_omega[k] = make_float4(w.x, w.y, w.z, 0.f);
    integrate_object(d, k);
  }
  for (int t = gl; t < ei.nlink; t += G) {
    int jg = ei.l0 + t;
    int art = d.j_art[jg];
    d.j_qd[jg] = X.qd[(art - ei.a0) * QS + (jg - d.joint_off[art])];
    d.j_lim_side[jg] = 0;
    d.j_lim_lambda[jg] = 0.f;
    d.j_motor_lambda[jg] = 0.f;
    integrate_joint(d, jg);
  }
  // contact force on the robot: normal impulses of the contacts with a link or the base
  // box of a kinematic-base articulation, over dt
  float f_robot = 0.f;
  const int b0 = d.base_off[e], nbase = d.base_off[e + 1] - b0;
  for (int u = gl; u < nct; u += G) {
    size_t g = X.gbase + u;
    float lam[3];
    if (u < X.S) {
      const float4 l = ld4(X.clam + 4 * u);
      lam[0] = l.x; lam[1] = l.y; lam[2] = l.z;
    } else {
      float4 l = d.r_lam[g];
      lam[0] = l.x; lam[1] = l.y; lam[2] = l.z;
    }
    V3 n = v3(d.c_n[g]);
    V3 t1 = v3(d.r_t1[g]);
    V3 t2 = cross(n, t1);
    V3 lt = t1 * lam[1] + t2 * lam[2];
    d.c_lam[g] = make_float4(lam[0], lam[1], lam[2], 0.f);
    const int4 key = d.c_key[g];
    bool robot = false;
#pragma unroll
    for (int s2 = 0; s2 < 2; ++s2) {
      const int c = s2 == 0 ? key.x : key.y;
      if (c >= ei.nobj && c < ei.nobj + ei.nlink) robot |= d.art_kin[d.j_art[ei.l0 + c - ei.nobj]] != 0;
      else if (c >= ei.nobj + ei.nlink && c < ei.nobj + ei.nlink + nbase)
        robot |= d.art_kin[d.base_art[b0 + c - ei.nobj - ei.nlink]] != 0;
    }
    if (robot) f_robot += lam[0] / dt;
    d.cache_key[g] = key;
    d.cache_p[g] = d.c_p[g];
    d.cache_lam[g] = make_float4(lam[0], lt.x, lt.y, lt.z);
  }
  __syncwarp(gm);
  for (int l = gl; l < nlim; l += G) {
    size_t li = (size_t)e * LCAP + l;
    int4 info = d.lr_info[li];
    const float lam = l < X.LS ? X.lrec[LREC * l + 11] : d.lr_data[li].z;
    if (info.z == 0) {
      d.j_motor_lambda[info.w] = lam;
    } else {
      d.j_lim_side[info.w] = info.z > 0 ? 1 : 2;
      d.j_lim_lambda[info.w] = lam;
    }
  }
  f_robot = group_sum<G>(f_robot, gm);
  if (gl == 0) {
    const float acc = d.robot_force_acc[e] + f_robot;
    d.robot_force[e] = f_robot;
    d.robot_force_acc[e] = acc;
    if (d.force_limit > 0.f && acc > d.force_limit) status |= ST_FORCE;
    d.cache_count[e] = nct;
    d.iters[e] = it;
    d.resid[e] = resid;
    d.n_colours[e] = ncol;
    if (status) atomicOr(&d.status[e], (int)status);
  }
}

// Environment schedule of the PGS kernel.  Plain grid: one slot per group.
// Persistent grid: groups take slots from a device counter.  Persistent grid
// with heavy SMs (SMs 0 .. heavy_sms - 1): the first block to start on each of
// those SMs keeps the SM to itself (later blocks there leave at once) and its
// groups first take the heaviest environments (the first H slots of the LPT
// order, one per group), then help with the rest; every other group takes the
// remaining slots first and the heavy ones last, so every slot is taken
// whichever blocks run where.  A Gauss-Seidel chain is serial, so the heaviest
// environments set the kernel's length; on an SM of their own they do not
// share issue slots, shared-memory bandwidth or instruction cache.
struct PgsSched {
  int* ctr;      // {next light slot, groups finished, next heavy slot}
  int* sm_rank;  // blocks started on each heavy SM, zero between launches
  int heavy_sms;
  int persistent;
  int pass, role;  // per group: queue pass (0, 1, 2 = done); role 0 normal, 1 heavy block, 2 idle
  int H, E, first;

  // next slot of this group in LPT order, or -1
  template <int G>
  __device__ __forceinline__ int next(int gl, unsigned gm, int g0) {
    if (!persistent) {
      const int s = first;
      first = 0x7fffffff;
      return s < E ? s : -1;
    }
    while (pass < 2) {
      const bool heavy = (pass == 0) == (role == 1);
      int s = 0;
      if (gl == 0) s = atomicAdd(heavy ? ctr + 2 : ctr, 1);
      s = __shfl_sync(gm, s, g0);
      if (s < (heavy ? H : E - H)) return heavy ? s : H + s;
      ++pass;
    }
    return -1;
  }
};

}  // namespace gb
