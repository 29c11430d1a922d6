// Articulated-body dynamics: one warp per articulation.
//
// Per articulation (n <= 9 joints, a tree with parent < child):
//   forward kinematics at q_t (link rotation, COM, joint axis and origin);
//   Featherstone's articulated-body algorithm (Rigid Body Dynamics Algorithms,
//   2008, ch. 7) with every link's spatial quantities expressed in world-aligned
//   axes about the link's own joint origin, so that moving between a link and
//   its parent is a pure translation by the link offset (2.8: translation-only
//   Plücker transforms) -- lever arms stay link-sized and FP32 cancellation in
//   the articulated inertias stays small -- with the stable PD motor of Tan,
//   Liu & Turk (2011) folded in:
//     tau_i = kp (q̄ - q - dt q̇) - kd q̇,  D_i = S_i^T I^A_i S_i + dt kd + dt² kp;
//   q̇* = q̇ + dt q̈;
//   joint-space inertia by the composite-rigid-body algorithm (ch. 6) plus the
//   same armature, and its inverse by Cholesky factorisation -- in FP64 when the
//   ABA pivots D_i span more than fp64_cond (ill-conditioned chain).
// Single-joint articulations (doors, drawers) take a thread-per-articulation
// kernel with the same recursion written out for one link (k_aba1).  The links'
// world COM and rotation come from a forward-kinematics kernel of their own
// (k_fk, a thread per link) at the start of the step.
// The inverse serves the contact and joint-limit rows of the solver
// (generalised response M^-1 J^T).
//
// Parallel layout: lane i owns link i for the per-link work (FK by walking its
// ancestor path, spatial inertias, velocities); the leaf-to-root and
// root-to-leaf recursions run link by link with lanes over the 36 entries of
// the 6x6 articulated inertia; the inverse runs one right-hand side per lane.
#pragma once
#include "sim_internal.cuh"

namespace gb {


struct AbaSh {
  int n, parent[MAX_DOF], type[MAX_DOF];
  float axis[MAX_DOF][3], com[MAX_DOF][3], half[MAX_DOF][3], mass[MAX_DOF];
  float q[MAX_DOF], qd[MAX_DOF], tau[MAX_DOF], arm[MAX_DOF];
  float T[MAX_DOF][9];      // local rotation: origin rotation x joint rotation
  float t[MAX_DOF][3];      // local translation of the link frame
  float al[MAX_DOF][3];     // joint axis in the parent link frame
  float op[MAX_DOF][3];     // joint origin in the parent link frame
  float R[MAX_DOF][9];      // world rotation of each link (row-major)
  float c[MAX_DOF][3];      // COM relative to the base origin
  float r[MAX_DOF][3];      // joint origin minus parent joint origin (base origin for roots)
  float ja[MAX_DOF][3], jo[MAX_DOF][3];
  float S[MAX_DOF][6], cb[MAX_DOF][6], pA[MAX_DOF][6], U[MAX_DOF][6], acc[MAX_DOF][6];
  union {  // articulated inertias (passes 1-2), composite inertias (CRBA), then the FP64
           // factorisation workspace
    float IA[MAX_DOF][36];
    float Ic[MAX_DOF][36];
    struct { double Md[MAX_DOF][MAX_DOF], Ld[MAX_DOF][MAX_DOF]; } f64;
  };
  float D[MAX_DOF], invD[MAX_DOF], u[MAX_DOF], qdd[MAX_DOF];
  float invL[MAX_DOF];      // reciprocals of the Cholesky pivots
  float M[MAX_DOF][MAX_DOF], L[MAX_DOF][MAX_DOF];
};

__device__ __forceinline__ void mat3_from_quat(float4 q, float* m) {
  float w = q.x, x = q.y, y = q.z, z = q.w;
  m[0] = 1.f - 2.f * (y * y + z * z); m[1] = 2.f * (x * y - w * z); m[2] = 2.f * (x * z + w * y);
  m[3] = 2.f * (x * y + w * z); m[4] = 1.f - 2.f * (x * x + z * z); m[5] = 2.f * (y * z - w * x);
  m[6] = 2.f * (x * z - w * y); m[7] = 2.f * (y * z + w * x); m[8] = 1.f - 2.f * (x * x + y * y);
}
__device__ __forceinline__ void mat3_mul(const float* a, const float* b, float* r) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) r[3 * i + j] = a[3 * i] * b[j] + a[3 * i + 1] * b[3 + j] + a[3 * i + 2] * b[6 + j];
}
__device__ __forceinline__ void mat3_vec(const float* a, const float* v, float* r) {
  for (int i = 0; i < 3; ++i) r[i] = a[3 * i] * v[0] + a[3 * i + 1] * v[1] + a[3 * i + 2] * v[2];
}

// Local transform of a joint at coordinate q: rotation T of the link frame in its
// parent's (origin rotation x joint rotation; Rodrigues' formula about the axis for
// a revolute joint), translation t of the link frame, joint axis al in the parent frame.
__device__ __forceinline__ void joint_local(const float4 ax, const float4 opos, const float4 oq, const int type,
                                            const float q, float* T, float* t, float* al) {
  float Ro[9];
  mat3_from_quat(oq, Ro);
  float axv[3] = {ax.x, ax.y, ax.z};
  mat3_vec(Ro, axv, al);
  if (type == 0) {
    float c = cosf(q), sn = sinf(q), k = 1.f - c;
    float ux = ax.x, uy = ax.y, uz = ax.z;
    float J[9] = {c + ux * ux * k, ux * uy * k - uz * sn, ux * uz * k + uy * sn,
                  uy * ux * k + uz * sn, c + uy * uy * k, uy * uz * k - ux * sn,
                  uz * ux * k - uy * sn, uz * uy * k + ux * sn, c + uz * uz * k};
    mat3_mul(Ro, J, T);
    t[0] = opos.x; t[1] = opos.y; t[2] = opos.z;
  } else {
    for (int k = 0; k < 9; ++k) T[k] = Ro[k];
    t[0] = opos.x + al[0] * q; t[1] = opos.y + al[1] * q; t[2] = opos.z + al[2] * q;
  }
}

// spatial motion x motion and motion x* force (Featherstone 2008, 2.9 / 2.10)
__device__ __forceinline__ void crm(const float* a, const float* b, float* r) {
  r[0] = a[1] * b[2] - a[2] * b[1]; r[1] = a[2] * b[0] - a[0] * b[2]; r[2] = a[0] * b[1] - a[1] * b[0];
  r[3] = (a[1] * b[5] - a[2] * b[4]) + (a[4] * b[2] - a[5] * b[1]);
  r[4] = (a[2] * b[3] - a[0] * b[5]) + (a[5] * b[0] - a[3] * b[2]);
  r[5] = (a[0] * b[4] - a[1] * b[3]) + (a[3] * b[1] - a[4] * b[0]);
}
__device__ __forceinline__ void crf(const float* a, const float* f, float* r) {
  r[0] = (a[1] * f[2] - a[2] * f[1]) + (a[4] * f[5] - a[5] * f[4]);
  r[1] = (a[2] * f[0] - a[0] * f[2]) + (a[5] * f[3] - a[3] * f[5]);
  r[2] = (a[0] * f[1] - a[1] * f[0]) + (a[3] * f[4] - a[4] * f[3]);
  r[3] = a[1] * f[5] - a[2] * f[4]; r[4] = a[2] * f[3] - a[0] * f[5]; r[5] = a[0] * f[4] - a[1] * f[3];
}

// 6x6 spatial inertia about the link's joint origin of a solid box link:
// [[Ic + m cx cx^T, m cx], [m cx^T, m 1]] with Ic = R diag(I) R^T.
__device__ __forceinline__ void spatial_inertia(const AbaSh& s, int i, float* I) {
  float m = s.mass[i];
  float hx = s.half[i][0], hy = s.half[i][1], hz = s.half[i][2];
  float d0 = m * (hy * hy + hz * hz) / 3.f, d1 = m * (hx * hx + hz * hz) / 3.f, d2 = m * (hx * hx + hy * hy) / 3.f;
  const float* R = s.R[i];
  float cx = s.c[i][0] - s.jo[i][0], cy = s.c[i][1] - s.jo[i][1], cz = s.c[i][2] - s.jo[i][2];
  float X[9] = {0.f, -cz, cy, cz, 0.f, -cx, -cy, cx, 0.f};
  for (int r = 0; r < 3; ++r)
    for (int k = 0; k < 3; ++k) {
      float ic = R[3 * r] * d0 * R[3 * k] + R[3 * r + 1] * d1 * R[3 * k + 1] + R[3 * r + 2] * d2 * R[3 * k + 2];
      float xx = X[3 * r] * X[3 * k] + X[3 * r + 1] * X[3 * k + 1] + X[3 * r + 2] * X[3 * k + 2];
      I[6 * r + k] = ic + m * xx;
      I[6 * r + 3 + k] = m * X[3 * r + k];
      I[6 * (3 + r) + k] = m * X[3 * k + r];
      I[6 * (3 + r) + 3 + k] = (r == k) ? m : 0.f;
    }
}

__device__ __forceinline__ void smv6(const float* I, const float* v, float* r) {
  for (int a = 0; a < 6; ++a) {
    float s = 0.f;
    for (int b = 0; b < 6; ++b) s += I[6 * a + b] * v[b];
    r[a] = s;
  }
}

// Entry e (0..20) of the upper triangle of a symmetric 6x6, in row order.
__device__ __forceinline__ void sym6_index(int e, int& row, int& col) {
  row = (int)((0x591b692449240000ull >> (3 * e)) & 7ull);
  col = (int)((0x5b2c76356346c688ull >> (3 * e)) & 7ull);
}

// Entry (row, col) of a symmetric 6x6 spatial inertia I carried to the frame
// offset by -r (the parent's): T I T^T with T = [[1, X], [0, 1]], X = r x; with
// x_row the row of X for row < 3 (zero below),
//   I'[row][col] = I[row][col] + x_row . I[3..5][col] + I[row][3..5] . x_col
//                  + x_row^T I[3..5][3..5] x_col,
// one formula for every block (no branch on the block of the entry).
__device__ __forceinline__ float shift_entry(const float* I, const float* r, int row, int col) {
  const float zr = row < 3 ? 1.f : 0.f, zc = col < 3 ? 1.f : 0.f;
  const int ir = row < 3 ? row : 0, ic = col < 3 ? col : 0;
  // rows of X = r x: (0, -r2, r1), (r2, 0, -r0), (-r1, r0, 0)
  const float xr0 = zr * (ir == 0 ? 0.f : (ir == 1 ? r[2] : -r[1]));
  const float xr1 = zr * (ir == 0 ? -r[2] : (ir == 1 ? 0.f : r[0]));
  const float xr2 = zr * (ir == 0 ? r[1] : (ir == 1 ? -r[0] : 0.f));
  const float xc0 = zc * (ic == 0 ? 0.f : (ic == 1 ? r[2] : -r[1]));
  const float xc1 = zc * (ic == 0 ? -r[2] : (ic == 1 ? 0.f : r[0]));
  const float xc2 = zc * (ic == 0 ? r[1] : (ic == 1 ? -r[0] : 0.f));
  float t = I[6 * row + col];
  t += xr0 * I[18 + col] + xr1 * I[24 + col] + xr2 * I[30 + col];
  t += I[6 * row + 3] * xc0 + I[6 * row + 4] * xc1 + I[6 * row + 5] * xc2;
  const float c0 = I[21] * xc0 + I[22] * xc1 + I[23] * xc2;
  const float c1 = I[27] * xc0 + I[28] * xc1 + I[29] * xc2;
  const float c2 = I[33] * xc0 + I[34] * xc1 + I[35] * xc2;
  return t + (xr0 * c0 + xr1 * c1 + xr2 * c2);
}

// Multi-joint articulation a on a group of G lanes (32: a warp; 16: two
// articulations per warp); gl = lane within the group (= joint for the per-link
// work), gm = the group's lane mask.
template <int G>
__device__ __forceinline__ void aba_multi(const Dev& d, const int a, const int gl, const unsigned gm, AbaSh& s) {
  const int j0 = d.joint_off[a];
  const int n = d.joint_off[a + 1] - j0;
  const float dt = d.dt;
  const float4 bq = d.art_base_quat[a];
  const float4 bp = d.art_base_pos[a];

  // ---- load constants, local transforms (lane = joint)
  if (gl < n) {
    int j = j0 + gl;
    s.parent[gl] = d.j_parent[j];
    s.type[gl] = d.j_type[j];
    float4 ax = d.j_axis[j], opos = d.j_opos[j], oq = d.j_oquat[j], cm = d.j_com[j], hf = d.j_half[j];
    float2 gain = d.j_gain[j];
    if (d.motor_mode && d.art_kin[a]) gain = make_float2(0.f, 0.f);  // motor rows replace the implicit PD
    float q = d.j_q[j], qd = d.j_qd[j];
    s.axis[gl][0] = ax.x; s.axis[gl][1] = ax.y; s.axis[gl][2] = ax.z;
    s.com[gl][0] = cm.x; s.com[gl][1] = cm.y; s.com[gl][2] = cm.z; s.mass[gl] = cm.w;
    s.half[gl][0] = hf.x; s.half[gl][1] = hf.y; s.half[gl][2] = hf.z;
    s.q[gl] = q; s.qd[gl] = qd;
    s.tau[gl] = gain.x * (d.j_target[j] - q - dt * qd) - gain.y * qd;
    s.arm[gl] = dt * gain.y + dt * dt * gain.x;
    float al[3];
    joint_local(ax, opos, oq, s.type[gl], q, s.T[gl], s.t[gl], al);
    s.al[gl][0] = al[0]; s.al[gl][1] = al[1]; s.al[gl][2] = al[2];
    s.op[gl][0] = opos.x; s.op[gl][1] = opos.y; s.op[gl][2] = opos.z;
  }
  if (gl == 0) s.n = n;
  __syncwarp(gm);

  // ---- forward kinematics: lane i composes its ancestor path from the base
  if (gl < n) {
    // ancestors of this link (itself included) as a bit set; parent < child, so
    // ascending bit order walks the path from the root down
    unsigned anc = 0;
    for (int k = gl; k >= 0; k = s.parent[k]) anc |= 1u << k;
    float R[9], Rn[9];
    mat3_from_quat(bq, R);
    float o[3] = {0.f, 0.f, 0.f};  // relative to the base origin
    float jo[3] = {0.f, 0.f, 0.f}, ja[3] = {0.f, 0.f, 0.f};
#pragma unroll 1
    for (int k = 0; k <= gl; ++k) {
      if (!((anc >> k) & 1u)) continue;
      float tw[3], aw[3], ow[3];
      mat3_vec(R, s.op[k], ow);
      mat3_vec(R, s.al[k], aw);
      if (k == gl) {
        jo[0] = o[0] + ow[0]; jo[1] = o[1] + ow[1]; jo[2] = o[2] + ow[2];
        ja[0] = aw[0]; ja[1] = aw[1]; ja[2] = aw[2];
      }
      mat3_vec(R, s.t[k], tw);
      o[0] += tw[0]; o[1] += tw[1]; o[2] += tw[2];
      mat3_mul(R, s.T[k], Rn);
      for (int e = 0; e < 9; ++e) R[e] = Rn[e];
    }
    for (int e = 0; e < 9; ++e) s.R[gl][e] = R[e];
    float cw[3];
    mat3_vec(R, s.com[gl], cw);
    s.c[gl][0] = o[0] + cw[0]; s.c[gl][1] = o[1] + cw[1]; s.c[gl][2] = o[2] + cw[2];
    for (int e = 0; e < 3; ++e) { s.ja[gl][e] = ja[e]; s.jo[gl][e] = jo[e]; }
    // motion subspace about the link's own joint origin
    if (s.type[gl] == 0) {
      s.S[gl][0] = ja[0]; s.S[gl][1] = ja[1]; s.S[gl][2] = ja[2];
      s.S[gl][3] = 0.f; s.S[gl][4] = 0.f; s.S[gl][5] = 0.f;
    } else {
      s.S[gl][0] = 0.f; s.S[gl][1] = 0.f; s.S[gl][2] = 0.f;
      s.S[gl][3] = ja[0]; s.S[gl][4] = ja[1]; s.S[gl][5] = ja[2];
    }
  }
  __syncwarp(gm);
  if (gl < n) {  // offset of this link's frame from its parent's (base origin for a root link)
    int p = s.parent[gl];
    for (int e = 0; e < 3; ++e) s.r[gl][e] = s.jo[gl][e] - (p < 0 ? 0.f : s.jo[p][e]);
  }
  __syncwarp(gm);

  // ---- pass 1: velocities (parent velocity translated to this frame plus the joint's), bias terms
  if (gl < n) {
    unsigned anc = 0;
    for (int k = gl; k >= 0; k = s.parent[k]) anc |= 1u << k;
    float v[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll 1
    for (int k = 0; k <= gl; ++k) {
      if (!((anc >> k) & 1u)) continue;
      const float* r = s.r[k];
      // translate to frame k: v_lin -= r x w, then add the joint velocity
      float lx = v[3] - (r[1] * v[2] - r[2] * v[1]);
      float ly = v[4] - (r[2] * v[0] - r[0] * v[2]);
      float lz = v[5] - (r[0] * v[1] - r[1] * v[0]);
      v[3] = lx; v[4] = ly; v[5] = lz;
      for (int e = 0; e < 6; ++e) v[e] = v[e] + s.S[k][e] * s.qd[k];
    }
    float vJ[6];
    for (int e = 0; e < 6; ++e) vJ[e] = s.S[gl][e] * s.qd[gl];
    crm(v, vJ, s.cb[gl]);
    spatial_inertia(s, gl, s.IA[gl]);  // built in place (a 36-float local array would live in local memory)
    float Iv[6];
    smv6(s.IA[gl], v, Iv);
    crf(v, Iv, s.pA[gl]);
  }
  __syncwarp(gm);

  // ---- pass 2: articulated inertias, leaf to root.  Per link: lanes 0-5 form
  //      U = IA S and IA cb, shuffle sums give D, S^T pA and U^T cb, and
  //      pa = pA + Ia cb + U u / D (Ia = IA - U U^T / D, so Ia cb = IA cb - U (U^T cb) / D)
  //      is carried to the parent frame by shuffles; then Ia in place; then the
  //      inertia shift to the parent frame, added to the parent's.
  for (int i = n - 1; i >= 0; --i) {
    float Ue = 0.f, ce = 0.f, Se = 0.f, pAe = 0.f, cbe = 0.f;
    if (gl < 6) {
#pragma unroll
      for (int b = 0; b < 6; ++b) {
        Ue += s.IA[i][6 * gl + b] * s.S[i][b];
        ce += s.IA[i][6 * gl + b] * s.cb[i][b];
      }
      Se = s.S[i][gl];
      pAe = s.pA[i][gl];
      cbe = s.cb[i][gl];
      s.U[i][gl] = Ue;
    }
    float Dv = Se * Ue, sp = Se * pAe, ucb = Ue * cbe;
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) {  // lanes 0-7 of the group hold the terms (6, 7 hold zeros)
      Dv += __shfl_xor_sync(gm, Dv, o);
      sp += __shfl_xor_sync(gm, sp, o);
      ucb += __shfl_xor_sync(gm, ucb, o);
    }
    const int g0 = (threadIdx.x & 31) & ~(G - 1);
    Dv = __shfl_sync(gm, Dv, g0);
    sp = __shfl_sync(gm, sp, g0);
    ucb = __shfl_sync(gm, ucb, g0);
    const float Di = Dv + s.arm[i];
    const float invDi = 1.f / Di;
    const float ui = s.tau[i] - sp;
    if (gl == 0) {
      s.D[i] = Di;
      s.invD[i] = invDi;
      s.u[i] = ui;
    }
    int p = s.parent[i];
    // pa in frame i, then to the parent frame: n_p = n_i + r x f
    float pa = (pAe + (ce - Ue * (ucb * invDi))) + Ue * (ui * invDi);
    const float f3 = __shfl_sync(gm, pa, g0 + 3), f4 = __shfl_sync(gm, pa, g0 + 4), f5 = __shfl_sync(gm, pa, g0 + 5);
    __syncwarp(gm);
    if (p >= 0) {
      const float* r = s.r[i];
      if (gl == 0) pa = pa + (r[1] * f5 - r[2] * f4);
      if (gl == 1) pa = pa + (r[2] * f3 - r[0] * f5);
      if (gl == 2) pa = pa + (r[0] * f4 - r[1] * f3);
      // Ia = IA - U U^T / D (symmetric: the 21 entries of the upper triangle, mirrored)
      for (int e = gl; e < 21; e += G) {
        int rr, cc;
        sym6_index(e, rr, cc);
        const float v = s.IA[i][6 * rr + cc] - s.U[i][rr] * (s.U[i][cc] * invDi);
        s.IA[i][6 * rr + cc] = v;
        s.IA[i][6 * cc + rr] = v;
      }
      __syncwarp(gm);
      // inertia to the parent frame, added to the parent's (each lane reads and
      // writes only its own entry pair of the parent)
      for (int e = gl; e < 21; e += G) {
        int rr, cc;
        sym6_index(e, rr, cc);
        const float v = s.IA[p][6 * rr + cc] + shift_entry(s.IA[i], s.r[i], rr, cc);
        s.IA[p][6 * rr + cc] = v;
        s.IA[p][6 * cc + rr] = v;
      }
      if (gl < 6) s.pA[p][gl] = s.pA[p][gl] + pa;
      __syncwarp(gm);
    }
  }

  // ---- pass 3: accelerations, root to leaf (gravity as an upward base acceleration)
  if (gl == 0) {
    for (int i = 0; i < n; ++i) {
      int p = s.parent[i];
      float ap[6];
      if (p < 0) {
        ap[0] = ap[1] = ap[2] = 0.f;
        ap[3] = -d.gx; ap[4] = -d.gy; ap[5] = -d.gz;
      } else {
        const float* r = s.r[i];
        const float* q = s.acc[p];
        ap[0] = q[0]; ap[1] = q[1]; ap[2] = q[2];
        ap[3] = q[3] - (r[1] * q[2] - r[2] * q[1]);
        ap[4] = q[4] - (r[2] * q[0] - r[0] * q[2]);
        ap[5] = q[5] - (r[0] * q[1] - r[1] * q[0]);
      }
      float a1[6];
      for (int e = 0; e < 6; ++e) a1[e] = ap[e] + s.cb[i][e];
      float ua = 0.f;
      for (int e = 0; e < 6; ++e) ua += s.U[i][e] * a1[e];
      float qdd = (s.u[i] - ua) * s.invD[i];
      s.qdd[i] = qdd;
      for (int e = 0; e < 6; ++e) s.acc[i][e] = a1[e] + s.S[i][e] * qdd;
    }
  }
  __syncwarp(gm);

  // ---- CRBA: composite inertias leaf to root (translated to the parent frame),
  //      then M_ik = S_k^T F with F = Ic_i S_i carried up to frame k; the composite
  //      inertias start from the link inertias again, in the articulated inertias'
  //      storage (dead after pass 3)
  if (gl < n) spatial_inertia(s, gl, s.Ic[gl]);
  __syncwarp(gm);
  for (int i = n - 1; i >= 0; --i) {
    int p = s.parent[i];
    if (p >= 0) {
      for (int e = gl; e < 21; e += G) {  // symmetric: upper triangle, mirrored
        int rr, cc;
        sym6_index(e, rr, cc);
        const float v = s.Ic[p][6 * rr + cc] + shift_entry(s.Ic[i], s.r[i], rr, cc);
        s.Ic[p][6 * rr + cc] = v;
        s.Ic[p][6 * cc + rr] = v;
      }
    }
    __syncwarp(gm);
  }
  if (gl < n) {
    int i = gl;
    float F[6];
    smv6(s.Ic[i], s.S[i], F);
    float mii = 0.f;
    for (int e = 0; e < 6; ++e) mii += s.S[i][e] * F[e];
    for (int k = 0; k < n; ++k) s.M[i][k] = 0.f;
    s.M[i][i] = mii + s.arm[i];
    for (int k = i; s.parent[k] >= 0; k = s.parent[k]) {
      const float* r = s.r[k];  // carry F from frame k to frame parent(k)
      float n0 = F[0] + (r[1] * F[5] - r[2] * F[4]);
      float n1 = F[1] + (r[2] * F[3] - r[0] * F[5]);
      float n2 = F[2] + (r[0] * F[4] - r[1] * F[3]);
      F[0] = n0; F[1] = n1; F[2] = n2;
      int pk = s.parent[k];
      float mik = 0.f;
      for (int e = 0; e < 6; ++e) mik += s.S[pk][e] * F[e];
      s.M[i][pk] = mik;
    }
  }
  __syncwarp(gm);
  if (gl < n)
    for (int k = gl + 1; k < n; ++k) s.M[gl][k] = s.M[k][gl];
  __syncwarp(gm);

  // ---- conditioning estimate from the ABA pivots; Cholesky and inverse
  float dmax = 0.f, dmin = 3.4e38f;
  for (int i = 0; i < n; ++i) { dmax = fmaxf(dmax, s.D[i]); dmin = fminf(dmin, s.D[i]); }
  const bool use64 = dmax > d.fp64_cond * dmin;
  float* minv = d.a_minv + (size_t)a * 81;
  if (!use64) {
    for (int j = 0; j < n; ++j) {
      if (gl == 0) {
        float sj = s.M[j][j];
        for (int k = 0; k < j; ++k) sj -= s.L[j][k] * s.L[j][k];
        s.L[j][j] = sqrtf(sj);
        s.invL[j] = 1.f / s.L[j][j];
      }
      __syncwarp(gm);
      int i = j + 1 + gl;
      if (i < n) {
        float t = s.M[i][j];
        for (int k = 0; k < j; ++k) t -= s.L[i][k] * s.L[j][k];
        s.L[i][j] = t * s.invL[j];
      }
      __syncwarp(gm);
    }
    if (gl < n) {  // column `gl` of the inverse: L L^T x = e_gl, unrolled so y and x stay in registers
      float y[MAX_DOF], x[MAX_DOF];
#pragma unroll
      for (int i = 0; i < MAX_DOF; ++i) {
        float sv = (i == gl) ? 1.f : 0.f;
#pragma unroll
        for (int k = 0; k < i; ++k) sv -= s.L[i][k] * y[k];
        y[i] = i < n ? sv * s.invL[i] : 0.f;
      }
#pragma unroll
      for (int i = MAX_DOF - 1; i >= 0; --i) {
        float sv = y[i];
#pragma unroll
        for (int k = i + 1; k < MAX_DOF; ++k)
          if (k < n) sv -= s.L[k][i] * x[k];
        x[i] = i < n ? sv * s.invL[i] : 0.f;
      }
#pragma unroll
      for (int i = 0; i < MAX_DOF; ++i)
        if (i < n) minv[9 * i + gl] = x[i];
    }
  } else {
    for (int i = gl; i < n * n; i += G) s.f64.Md[i / n][i % n] = (double)s.M[i / n][i % n];
    __syncwarp(gm);
    for (int j = 0; j < n; ++j) {
      if (gl == 0) {
        double sj = s.f64.Md[j][j];
        for (int k = 0; k < j; ++k) sj -= s.f64.Ld[j][k] * s.f64.Ld[j][k];
        s.f64.Ld[j][j] = sqrt(sj);
      }
      __syncwarp(gm);
      int i = j + 1 + gl;
      if (i < n) {
        double t = s.f64.Md[i][j];
        for (int k = 0; k < j; ++k) t -= s.f64.Ld[i][k] * s.f64.Ld[j][k];
        s.f64.Ld[i][j] = t / s.f64.Ld[j][j];
      }
      __syncwarp(gm);
    }
    if (gl < n) {  // (rare path: kept rolled, registers stay low for the common path)
      double y[MAX_DOF], x[MAX_DOF];
      for (int i = 0; i < n; ++i) {
        double sv = (i == gl) ? 1.0 : 0.0;
        for (int k = 0; k < i; ++k) sv -= s.f64.Ld[i][k] * y[k];
        y[i] = sv / s.f64.Ld[i][i];
      }
      for (int i = n - 1; i >= 0; --i) {
        double sv = y[i];
        for (int k = i + 1; k < n; ++k) sv -= s.f64.Ld[k][i] * x[k];
        x[i] = sv / s.f64.Ld[i][i];
      }
      for (int i = 0; i < n; ++i) minv[9 * i + gl] = (float)x[i];
    }
    if (gl == 0) {
      int lo = 0, hi = d.E - 1;  // environment of this articulation: art_off[e] <= a < art_off[e + 1]
      while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (d.art_off[mid] <= a) lo = mid; else hi = mid - 1;
      }
      atomicOr(&d.fp64_used[lo], 1);
    }
  }

  // ---- outputs (world positions = base origin + relative)
  if (gl < n) {
    int j = j0 + gl;
    d.l_ja[j] = make_float4(s.ja[gl][0], s.ja[gl][1], s.ja[gl][2], (float)s.type[gl]);
    d.l_jo[j] = make_float4(bp.x + s.jo[gl][0], bp.y + s.jo[gl][1], bp.z + s.jo[gl][2], 0.f);
    d.j_qdd[j] = s.qdd[gl];
    d.j_qdstar[j] = s.qd[gl] + dt * s.qdd[gl];
  }
}

// Single-joint articulations (doors, drawers), one thread each: the same
// articulated-body recursion collapses to q̈ = (τ - S^T p - U^T a_0) / D with
// U = I S, D = S^T I S + armature, and M = D, M^-1 = 1 / D.
__device__ __forceinline__ void aba_single(const Dev& d, const int a) {
  const int j = d.joint_off[a];
  const float dt = d.dt;
  const float4 bq = d.art_base_quat[a], bp = d.art_base_pos[a];
  const float4 ax = d.j_axis[j], opos = d.j_opos[j], oq = d.j_oquat[j], cm = d.j_com[j], hf = d.j_half[j];
  const float2 gain = d.motor_mode && d.art_kin[a] ? make_float2(0.f, 0.f) : d.j_gain[j];
  const int type = d.j_type[j];
  const float q = d.j_q[j], qd = d.j_qd[j];
  const float tau = gain.x * (d.j_target[j] - q - dt * qd) - gain.y * qd;
  const float arm = dt * gain.y + dt * dt * gain.x;
  float Rb[9], T[9], R[9], al[3], tt[3];
  mat3_from_quat(bq, Rb);
  joint_local(ax, opos, oq, type, q, T, tt, al);
  float op3[3] = {opos.x, opos.y, opos.z}, jo[3], ja[3], o[3], cw[3], com[3] = {cm.x, cm.y, cm.z};
  mat3_vec(Rb, op3, jo);
  mat3_vec(Rb, al, ja);
  mat3_vec(Rb, tt, o);
  mat3_mul(Rb, T, R);
  mat3_vec(R, com, cw);
  float c[3] = {o[0] + cw[0], o[1] + cw[1], o[2] + cw[2]};  // relative to the base origin
  // spatial inertia about the joint origin
  const float m = cm.w;
  const float hx = hf.x, hy = hf.y, hz = hf.z;
  const float d0 = m * (hy * hy + hz * hz) / 3.f, d1 = m * (hx * hx + hz * hz) / 3.f, d2 = m * (hx * hx + hy * hy) / 3.f;
  const float cx = c[0] - jo[0], cy = c[1] - jo[1], cz = c[2] - jo[2];
  const float X[9] = {0.f, -cz, cy, cz, 0.f, -cx, -cy, cx, 0.f};
  float I[36];
  for (int r = 0; r < 3; ++r)
    for (int k = 0; k < 3; ++k) {
      float ic = R[3 * r] * d0 * R[3 * k] + R[3 * r + 1] * d1 * R[3 * k + 1] + R[3 * r + 2] * d2 * R[3 * k + 2];
      float xx = X[3 * r] * X[3 * k] + X[3 * r + 1] * X[3 * k + 1] + X[3 * r + 2] * X[3 * k + 2];
      I[6 * r + k] = ic + m * xx;
      I[6 * r + 3 + k] = m * X[3 * r + k];
      I[6 * (3 + r) + k] = m * X[3 * k + r];
      I[6 * (3 + r) + 3 + k] = (r == k) ? m : 0.f;
    }
  float S[6];
  if (type == 0) { S[0] = ja[0]; S[1] = ja[1]; S[2] = ja[2]; S[3] = S[4] = S[5] = 0.f; }
  else { S[0] = S[1] = S[2] = 0.f; S[3] = ja[0]; S[4] = ja[1]; S[5] = ja[2]; }
  float v[6], Iv[6], pA[6], U[6];
  for (int e = 0; e < 6; ++e) v[e] = S[e] * qd;
  smv6(I, v, Iv);
  crf(v, Iv, pA);
  smv6(I, S, U);
  float Dv = 0.f, sp = 0.f;
  for (int e = 0; e < 6; ++e) { Dv += S[e] * U[e]; sp += S[e] * pA[e]; }
  const float D = Dv + arm;
  const float u = tau - sp;
  const float a0[6] = {0.f, 0.f, 0.f, -d.gx, -d.gy, -d.gz};
  float ua = 0.f;
  for (int e = 0; e < 6; ++e) ua += U[e] * a0[e];
  const float qdd = (u - ua) / D;
  d.a_minv[(size_t)a * 81] = 1.f / D;
  d.l_ja[j] = make_float4(ja[0], ja[1], ja[2], (float)type);
  d.l_jo[j] = make_float4(bp.x + jo[0], bp.y + jo[1], bp.z + jo[2], 0.f);
  d.j_qdd[j] = qdd;
  d.j_qdstar[j] = qd + dt * qdd;
}

// Forward kinematics at q_t for the links' world COM and rotation (what collision
// detection and the contact rows read), by the same composition of local transforms
// along each link's ancestor path from the base as in aba_multi.  It runs in a kernel
// of its own at the start of the step, so the collision kernel does not wait for the
// articulated-body kernel.  Multi-joint articulation a on a group of G lanes (lane =
// joint): local transforms to shared memory, then each lane composes its path.
struct FkSh {
  int parent[MAX_DOF];
  float T[MAX_DOF][9], t[MAX_DOF][3];
};

__device__ __forceinline__ void fk_out(const Dev& d, const int j, const float4 bp, const float* R, const float* o) {
  const float4 cm = d.j_com[j];
  float com[3] = {cm.x, cm.y, cm.z}, cw[3];
  mat3_vec(R, com, cw);
  d.l_com[j] = make_float4(bp.x + (o[0] + cw[0]), bp.y + (o[1] + cw[1]), bp.z + (o[2] + cw[2]), 0.f);
  d.l_r0[j] = make_float4(R[0], R[1], R[2], 0.f);
  d.l_r1[j] = make_float4(R[3], R[4], R[5], 0.f);
  d.l_r2[j] = make_float4(R[6], R[7], R[8], 0.f);
}

template <int G>
__device__ __forceinline__ void fk_multi(const Dev& d, const int a, const int gl, const unsigned gm, FkSh& s) {
  const int j0 = d.joint_off[a];
  const int n = d.joint_off[a + 1] - j0;
  if (gl < n) {
    const int j = j0 + gl;
    s.parent[gl] = d.j_parent[j];
    float al[3];
    joint_local(d.j_axis[j], d.j_opos[j], d.j_oquat[j], d.j_type[j], d.j_q[j], s.T[gl], s.t[gl], al);
  }
  __syncwarp(gm);
  if (gl < n) {
    unsigned anc = 0;  // ancestors of this link (itself included); parent < child
    for (int k = gl; k >= 0; k = s.parent[k]) anc |= 1u << k;
    const float4 bq = d.art_base_quat[a], bp = d.art_base_pos[a];
    float R[9], Rn[9];
    mat3_from_quat(bq, R);
    float o[3] = {0.f, 0.f, 0.f};  // relative to the base origin
#pragma unroll 1
    for (int k = 0; k <= gl; ++k) {
      if (!((anc >> k) & 1u)) continue;
      float tw[3];
      mat3_vec(R, s.t[k], tw);
      o[0] += tw[0]; o[1] += tw[1]; o[2] += tw[2];
      mat3_mul(R, s.T[k], Rn);
      for (int e = 0; e < 9; ++e) R[e] = Rn[e];
    }
    fk_out(d, j0 + gl, bp, R, o);
  }
}

// single-joint articulation a, one thread
__device__ __forceinline__ void fk_single(const Dev& d, const int a) {
  const int j = d.joint_off[a];
  float Rb[9], T[9], R[9], t[3], al[3], o[3];
  mat3_from_quat(d.art_base_quat[a], Rb);
  joint_local(d.j_axis[j], d.j_opos[j], d.j_oquat[j], d.j_type[j], d.j_q[j], T, t, al);
  mat3_vec(Rb, t, o);
  mat3_mul(Rb, T, R);
  fk_out(d, j, d.art_base_pos[a], R, o);
}

}  // namespace gb
