// Collision detection: one warp per environment.
//
// Colliders of an environment, in index order: free objects, articulation
// links (articulation order, joint order), articulation base boxes, static
// boxes, ground plane -- dynamic colliders first, so in a pair (a < b) body A
// is dynamic and the normal points from B to A.
//
//   1. stage every collider's pose, half extents and AABB in shared memory;
//   2. broadphase: all pairs a < b in ascending order (lanes over the dynamic
//      colliders a, a bit mask of candidate b per lane, ordered output by a
//      warp prefix sum); static-static and same-articulation pairs are never
//      candidates; AABBs fattened by margin/2 must overlap;
//   3. wake pass (Sec. 4.1 "sleeping"): in ascending pair order, a sleeping
//      object paired with an awake dynamic collider wakes;
//   4. pairs with no awake dynamic collider are dropped;
//   5. narrowphase, one pair per lane: sphere-sphere, sphere-plane, sphere-box,
//      box-plane (vertex enumeration), box-box (15-axis SAT from C = A^T B; face
//      contacts from the incident face clipped to the reference face -- its vertices
//      enumerated directly: incident vertices, edge-plane crossings, reference
//      corners, with the labels of Sutherland-Hodgman clipping -- edge contacts by
//      the closest points of the two edges' lines, each clamped to its edge);
//      manifolds above four points reduced
//      (deepest, farthest, largest triangle, largest quadrilateral); candidate
//      points in a per-lane shared-memory scratch;
//   6. contacts written in (a, b, feature) order with a warp prefix sum.
#pragma once
#include "sim_internal.cuh"

namespace gb {


struct Coll {  // one collider, read from shared memory
  V3 x;
  M3 R;
  V3 h;
  int shape;
};

// Per-lane scratch in shared memory for the narrowphase's candidate points (kept out
// of local memory: the clipping and the manifold reduction index their points at run
// time).  Column layout, word w of lane l at w * 32 + l, so every access of a warp is
// free of bank conflicts.  Slots 0..7: candidate point x, y, z, separation, feature id
// (5 words each); words 40..42: the contact normal of the pair.
constexpr int NP_SLOTS = 8, NP_WORDS = 44;
struct Cand {
  float* c;  // this lane's column: word w at c[32 * w]
  __device__ __forceinline__ float& w(int i) const { return c[32 * i]; }
  __device__ __forceinline__ V3 p(int k) const { return v3(w(5 * k), w(5 * k + 1), w(5 * k + 2)); }
  __device__ __forceinline__ float sep(int k) const { return w(5 * k + 3); }
  __device__ __forceinline__ int f(int k) const { return __float_as_int(w(5 * k + 4)); }
  __device__ __forceinline__ void put(int k, V3 p, float sep, int f) const {
    w(5 * k) = p.x; w(5 * k + 1) = p.y; w(5 * k + 2) = p.z; w(5 * k + 3) = sep; w(5 * k + 4) = __int_as_float(f);
  }
  __device__ __forceinline__ void copy(int dst, int src) const {
#pragma unroll
    for (int i = 0; i < 5; ++i) w(5 * dst + i) = w(5 * src + i);
  }
  __device__ __forceinline__ V3 n() const { return v3(w(40), w(41), w(42)); }
  __device__ __forceinline__ void set_n(V3 n) const { w(40) = n.x; w(41) = n.y; w(42) = n.z; }
};

// index of the first candidate within tol of the extreme of val(i) (largest if
// maximise), skipping those flagged in `ex`
template <class Val>
static __device__ int first_within(int n, unsigned ex, float tol, bool maximise, Val val) {
  int best = -1;
  float bv = 0.f;
  for (int i = 0; i < n; ++i) {
    if (ex >> i & 1) continue;
    const float v = val(i);
    if (best < 0 || (maximise ? v > bv : v < bv)) { best = i; bv = v; }
  }
  if (best < 0) return -1;
  for (int i = 0; i < n; ++i) {
    if (ex >> i & 1) continue;
    const float v = val(i);
    if (maximise ? v >= bv - tol : v <= bv + tol) return i;
  }
  return best;
}

// candidates sorted by feature id; keeps at most four (deepest, farthest from it,
// largest triangle, largest quadrilateral), ascending feature order, in slots 0..3
static __device__ int reduce4(const Cand& c, int n) {
  if (n <= 4) return n;
  unsigned ex = 0;
  const int i1 = first_within(n, ex, 1e-5f, false, [&](int i) { return c.sep(i); });
  ex |= 1u << i1;
  const V3 p1 = c.p(i1);
  const int i2 = first_within(n, ex, 1e-5f, true, [&](int i) { return norm(c.p(i) - p1); });
  ex |= 1u << i2;
  const V3 p2 = c.p(i2);
  const int i3 = first_within(n, ex, 1e-6f, true, [&](int i) { return norm(cross(p2 - p1, c.p(i) - p1)); });
  ex |= 1u << i3;
  const V3 p3 = c.p(i3);
  const int i4 = first_within(n, ex, 1e-6f, true, [&](int i) {
    const V3 p = c.p(i);
    return norm(cross(p - p1, p2 - p1)) + norm(cross(p - p2, p3 - p2)) + norm(cross(p - p3, p1 - p3));
  });
  ex |= 1u << i4;
  int m = 0;
  for (int i = 0; i < n; ++i)
    if (ex >> i & 1) c.copy(m++, i);
  return m;
}

static __device__ int box_box(const Coll& A, const Coll& B, float margin, const Cand& out) {
  // SAT over the 15 axes from C = A^T B (C[i][j] = a_i . b_j) and the centre offset
  // D = x_A - x_B in both frames: the separation along an axis u is
  // |u . D| - sum_k hA_k |u . a_k| - sum_k hB_k |u . b_k|, and every projection of a
  // face or edge axis is a C entry (a_i x b_j . a_k, . b_k and its length
  // |a_i x b_j| = sqrt(C[i1][j]^2 + C[i2][j]^2) from the other two components).
  float Cm[3][3], Ca[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      Cm[i][j] = dot(mcol(A.R, i), mcol(B.R, j));
      Ca[i][j] = fabsf(Cm[i][j]);
    }
  const V3 D = A.x - B.x;
  float tA[3], tB[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    tA[k] = dot(mcol(A.R, k), D);
    tB[k] = dot(mcol(B.R, k), D);
  }
  float fsep[6];
#pragma unroll
  for (int k = 0; k < 3; ++k) {  // face axes b_k, then a_k
    fsep[k] = fabsf(tB[k]) - (comp(A.h, 0) * Ca[0][k] + comp(A.h, 1) * Ca[1][k] + comp(A.h, 2) * Ca[2][k]) -
              comp(B.h, k);
    fsep[3 + k] = fabsf(tA[k]) - comp(A.h, k) -
                  (comp(B.h, 0) * Ca[k][0] + comp(B.h, 1) * Ca[k][1] + comp(B.h, 2) * Ca[k][2]);
  }
  float fmax = fsep[0];
#pragma unroll
  for (int k = 1; k < 6; ++k) fmax = fmaxf(fmax, fsep[k]);
  int face = 5;
#pragma unroll
  for (int k = 5; k >= 0; --k)  // the first face axis within 1e-4 m of the largest separation
    if (fsep[k] >= fmax - 1e-4f) face = k;
  float esep[9];
  float emax = -1e30f;
  int nvalid = 0;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const int i1 = (i + 1) % 3, i2 = (i + 2) % 3;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int j1 = (j + 1) % 3, j2 = (j + 2) % 3;
      // u = a_i x b_j = C[i1][j] a_i2 - C[i2][j] a_i1 in A's frame
      const float len = sqrtf(Cm[i1][j] * Cm[i1][j] + Cm[i2][j] * Cm[i2][j]);
      if (len < 1e-3f) { esep[3 * i + j] = -1e30f; continue; }
      const float ud = Cm[i1][j] * tA[i2] - Cm[i2][j] * tA[i1];
      const float ra = comp(A.h, i1) * Ca[i2][j] + comp(A.h, i2) * Ca[i1][j];
      const float rb = comp(B.h, j1) * Ca[i][j2] + comp(B.h, j2) * Ca[i][j1];
      esep[3 * i + j] = (fabsf(ud) - ra - rb) / len;
      if (nvalid == 0 || esep[3 * i + j] > emax) emax = esep[3 * i + j];
      ++nvalid;
    }
  }
  if (nvalid > 0 && emax > fmax + 1e-3f) {
    if (emax > margin) return 0;
    int e = 0;
    float es = esep[0];
#pragma unroll
    for (int k = 8; k >= 0; --k)  // the first edge axis within 1e-4 m of the largest separation
      if (esep[k] > -1e29f && esep[k] >= emax - 1e-4f) { e = k; es = esep[k]; }
    int i = e / 3, j = e % 3;
    V3 ua = mcol(A.R, i), ub = mcol(B.R, j);
    V3 L = cross(ua, ub);
    L = L * (1.f / norm(L));
    if (dot(L, A.x - B.x) < 0.f) L = -L;
    V3 pa = A.x, pb = B.x;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      if (k != i) pa = pa + mcol(A.R, k) * (comp(A.h, k) * (dot(L, mcol(A.R, k)) > 0.f ? -1.f : 1.f));
      if (k != j) pb = pb + mcol(B.R, k) * (comp(B.h, k) * (dot(L, mcol(B.R, k)) < 0.f ? -1.f : 1.f));
    }
    V3 r = pa - pb;
    float bb = dot(ua, ub), c = dot(ua, r), f = dot(ub, r);
    float den = 1.f - bb * bb;
    float sa = (bb * f - c) / den;
    float tb = f + sa * bb;
    sa = fmaxf(-comp(A.h, i), fminf(comp(A.h, i), sa));
    tb = fmaxf(-comp(B.h, j), fminf(comp(B.h, j), tb));
    V3 qa = pa + ua * sa, qb = pb + ub * tb;
    out.put(0, (qa + qb) * 0.5f, es, 1024 + e);
    out.set_n(L);
    return 1;
  }
  if (fmax > margin) return 0;
  const bool refB = face < 3;
  const int k = face % 3;
  const Coll& R = refB ? B : A;
  const Coll& I = refB ? A : B;
  V3 u = mcol(R.R, k);
  const bool neg = dot(u, I.x - R.x) < 0.f;
  V3 nref = neg ? -u : u;
  V3 fc = R.x + nref * comp(R.h, k);
  const int k1 = k == 0 ? 1 : 0, k2 = k == 2 ? 1 : 2;
  V3 t1 = mcol(R.R, k1), t2 = mcol(R.R, k2);
  float e1 = comp(R.h, k1), e2 = comp(R.h, k2);
  int m = 0;
  float best = fabsf(dot(mcol(I.R, 0), nref));
#pragma unroll
  for (int q = 1; q < 3; ++q) {
    float dq = fabsf(dot(mcol(I.R, q), nref));
    if (dq > best) { best = dq; m = q; }
  }
  float sg = dot(mcol(I.R, m), nref) > 0.f ? -1.f : 1.f;
  V3 ic = I.x + mcol(I.R, m) * (sg * comp(I.h, m));
  const int m1 = m == 0 ? 1 : 0, m2 = m == 2 ? 1 : 2;
  V3 w1 = mcol(I.R, m1) * comp(I.h, m1), w2 = mcol(I.R, m2) * comp(I.h, m2);
  // The incident face (vertices V0..V3, edge c from V_c to V_c+1) clipped to the
  // reference face's four side planes s (0, 1: +-t1 at e1; 2, 3: +-t2 at e2; a point is
  // inside plane s where its distance d_s <= 0).  The clipped polygon's vertices are
  //   - the incident vertices inside all four planes (feature label k),
  //   - the crossings of incident edge c with plane s that lie inside the other three
  //     (label 4 + 4c + s),
  //   - the reference face's corners, where planes s < s2 meet, that lie on the incident
  //     face (label 20 + 4s + s2),
  // the same points and labels as clipping the face plane by plane (Sutherland-Hodgman);
  // produced here directly in ascending label order, i.e. sorted by feature.
  const int ref_code = (refB ? 0 : 6) + 2 * k + (neg ? 1 : 0);
  const V3 V[4] = {ic - w1 - w2, ic + w1 - w2, ic + w1 + w2, ic - w1 + w2};
  float pu[4], pv[4];  // coordinates along t1, t2 relative to the face centre
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    pu[v] = dot(t1, V[v] - fc);
    pv[v] = dot(t2, V[v] - fc);
  }
  auto dist = [&](int s, float uu, float vv) {
    return s == 0 ? uu - e1 : (s == 1 ? -uu - e1 : (s == 2 ? vv - e2 : -vv - e2));
  };
  int np = 0;
  auto emit = [&](V3 P, int label) {
    const float sep = dot(nref, P - fc);
    if (sep > margin || np >= NP_SLOTS) return;
    out.put(np, P - nref * (sep * 0.5f), sep, ref_code * 64 + label);
    ++np;
  };
#pragma unroll
  for (int v = 0; v < 4; ++v)
    if (dist(0, pu[v], pv[v]) <= 0.f && dist(1, pu[v], pv[v]) <= 0.f && dist(2, pu[v], pv[v]) <= 0.f &&
        dist(3, pu[v], pv[v]) <= 0.f)
      emit(V[v], v);
  // (the edge loop stays rolled to bound the code size: an edge's end vertices are
  //  selected by its index and their face coordinates formed again, the same values
  //  as pu, pv)
  auto vert = [&](int v) { return v == 0 ? V[0] : (v == 1 ? V[1] : (v == 2 ? V[2] : V[3])); };
#pragma unroll 1
  for (int c = 0; c < 4; ++c) {
    const int c2 = (c + 1) & 3;
    const V3 Vc = vert(c), Vc2 = vert(c2);
    const float puc = dot(t1, Vc - fc), pvc = dot(t2, Vc - fc);
    const float puc2 = dot(t1, Vc2 - fc), pvc2 = dot(t2, Vc2 - fc);
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const float dP = dist(s, puc, pvc), dQ = dist(s, puc2, pvc2);
      if ((dP <= 0.f) == (dQ <= 0.f)) continue;
      const V3 X = Vc + (Vc2 - Vc) * (dP / (dP - dQ));
      const float xu = dot(t1, X - fc), xv = dot(t2, X - fc);
      bool in = true;
#pragma unroll
      for (int s2 = 0; s2 < 4; ++s2)
        if (s2 != s) in = in && dist(s2, xu, xv) <= 0.f;
      if (in) emit(X, 4 + 4 * c + s);
    }
  }
  // corners: planes (s, s2) with s in {0, 1} (t1) and s2 in {2, 3} (t2); the point on
  // the incident face's plane above or below the corner, kept where it lies on the face
  const V3 nI = cross(w1, w2);
  const float nn = dot(nI, nref);
  const float w11 = dot(w1, w1), w22 = dot(w2, w2);
#pragma unroll
  for (int s = 0; s < 2; ++s) {
#pragma unroll
    for (int s2 = 2; s2 < 4; ++s2) {
      const V3 K = fc + t1 * (s == 0 ? e1 : -e1) + t2 * (s2 == 2 ? e2 : -e2);
      if (fabsf(nn) < 1e-12f) continue;
      const V3 X = K + nref * (dot(nI, ic - K) / nn);
      const V3 r = X - ic;
      if (fabsf(dot(r, w1)) <= w11 && fabsf(dot(r, w2)) <= w22) emit(X, 20 + 4 * s + s2);
    }
  }
  np = reduce4(out, np);
  out.set_n(refB ? nref : -nref);
  return np;
}

static __device__ int narrowphase(const Coll& A, const Coll& B, float margin, const Cand& out) {
  if (B.shape == SHAPE_PLANE) {
    if (A.shape == SHAPE_SPHERE) {
      float r = A.h.x;
      float sep = A.x.z - r;
      if (sep > margin) return 0;
      out.put(0, v3(A.x.x, A.x.y, (A.x.z - r) * 0.5f), sep, 0);
      out.set_n(v3(0.f, 0.f, 1.f));
      return 1;
    }
    int np = 0;
#pragma unroll 1
    for (int k = 0; k < 8; ++k) {
      V3 l = v3((k & 1) ? A.h.x : -A.h.x, (k & 2) ? A.h.y : -A.h.y, (k & 4) ? A.h.z : -A.h.z);
      V3 v = A.x + mv(A.R, l);
      if (v.z > margin) continue;
      out.put(np, v3(v.x, v.y, v.z * 0.5f), v.z, k);
      ++np;
    }
    np = reduce4(out, np);
    out.set_n(v3(0.f, 0.f, 1.f));
    return np;
  }
  if (A.shape == SHAPE_SPHERE && B.shape == SHAPE_SPHERE) {
    V3 d = A.x - B.x;
    float dist = norm(d);
    V3 n = dist > 1e-12f ? d * (1.f / dist) : v3(0.f, 0.f, 1.f);
    float sep = dist - A.h.x - B.h.x;
    if (sep > margin) return 0;
    V3 pa = A.x - n * A.h.x, pb = B.x + n * B.h.x;
    out.put(0, (pa + pb) * 0.5f, sep, 0);
    out.set_n(n);
    return 1;
  }
  if (A.shape == SHAPE_SPHERE || B.shape == SHAPE_SPHERE) {
    const Coll& S = A.shape == SHAPE_SPHERE ? A : B;
    const Coll& X = A.shape == SHAPE_SPHERE ? B : A;
    float r = S.h.x;
    V3 l = mtv(X.R, S.x - X.x);
    V3 q = v3(fmaxf(-X.h.x, fminf(X.h.x, l.x)), fmaxf(-X.h.y, fminf(X.h.y, l.y)), fmaxf(-X.h.z, fminf(X.h.z, l.z)));
    bool inside = (q.x == l.x) && (q.y == l.y) && (q.z == l.z);
    V3 n, pb;
    float sep;
    if (!inside) {
      V3 pw = X.x + mv(X.R, q);
      V3 dd = S.x - pw;
      float dist = norm(dd);
      n = dd * (1.f / dist);
      sep = dist - r;
      pb = pw;
    } else {
      int k = 0;
      float bst = X.h.x - fabsf(l.x);
#pragma unroll
      for (int i = 1; i < 3; ++i) {
        float dd = comp(X.h, i) - fabsf(comp(l, i));
        if (dd < bst) { bst = dd; k = i; }
      }
      float sg = comp(l, k) < 0.f ? -1.f : 1.f;
      n = mcol(X.R, k) * sg;
      sep = -bst - r;
      pb = S.x + n * bst;
    }
    if (sep > margin) return 0;
    V3 ps = S.x - n * r;
    out.put(0, (pb + ps) * 0.5f, sep, 0);
    out.set_n(A.shape == SHAPE_SPHERE ? n : -n);
    return 1;
  }
  return box_box(A, B, margin, out);
}

// per-warp shared memory, NC = colliders capacity of the launch
struct CollLayout {
  int NC;
  // staged colliders, the pair list, the narrowphase's candidate scratch
  __device__ __host__ size_t floats() const { return (size_t)NC * 25 + PAIR_CAP / 2 + 32 * NP_WORDS; }
};

__device__ __forceinline__ void collide_env(const Dev& d, const int NC, float* base, const int e, const int lane) {
  // AABBs fattened by margin/2 as two float4 per collider: (lo, info bits), (hi, 0)
  float4* sbox = reinterpret_cast<float4*>(base);  // [NC*2]
  float* sx = base + NC * 8;    // [NC*3]
  float* sR = sx + NC * 3;      // [NC*9]
  float* sh = sR + NC * 9;      // [NC*3]
  int* sinfo = reinterpret_cast<int*>(sh + NC * 3);  // [NC]: shape | kind << 4 | local index << 8
  unsigned short* spairs = reinterpret_cast<unsigned short*>(sinfo + NC);  // [PAIR_CAP]: a << 8 | b
  const Cand cand{base + NC * 25 + PAIR_CAP / 2 + lane};                   // [NP_WORDS][32]

  const int o0 = d.obj_off[e], nobj = d.obj_off[e + 1] - o0;
  const int a0 = d.art_off[e], a1 = d.art_off[e + 1];
  const int l0 = d.joint_off[a0], nlink = d.joint_off[a1] - l0;
  const int b0 = d.base_off[e], nbase = d.base_off[e + 1] - b0;
  const int s0 = d.stat_off[e], nstat = d.stat_off[e + 1] - s0;
  const int plane = d.env_plane[e];
  const int nc = nobj + nlink + nbase + nstat + plane;
  const float h = d.margin * 0.5f;
  unsigned status = 0;

  // ---- 1. stage colliders
  for (int c = lane; c < nc; c += 32) {
    V3 x = v3(0.f, 0.f, 0.f), hf = v3(0.f, 0.f, 0.f);
    M3 R;
    R.r0 = v3(1.f, 0.f, 0.f); R.r1 = v3(0.f, 1.f, 0.f); R.r2 = v3(0.f, 0.f, 1.f);
    int shape = SHAPE_BOX, kind, idx;
    if (c < nobj) {
      int k = o0 + c;
      x = v3(d.obj_pos[k]);
      R = quat_mat(d.obj_quat[k]);
      float4 hh = d.obj_half[k];
      hf = v3(hh);
      shape = (int)hh.w;
      kind = CK_OBJ; idx = c;
    } else if (c < nobj + nlink) {
      int j = l0 + (c - nobj);
      x = v3(d.l_com[j]);
      R.r0 = v3(d.l_r0[j]); R.r1 = v3(d.l_r1[j]); R.r2 = v3(d.l_r2[j]);
      hf = v3(d.j_half[j]);
      kind = CK_LINK; idx = d.j_art[j] - a0;
    } else if (c < nobj + nlink + nbase) {
      int art = d.base_art[b0 + (c - nobj - nlink)];
      R = quat_mat(d.art_base_quat[art]);
      x = v3(d.art_base_pos[art]) + mv(R, v3(d.art_bc_off[art]));
      hf = v3(d.art_bc_half[art]);
      kind = CK_BASE; idx = art - a0;
    } else if (c < nobj + nlink + nbase + nstat) {
      int k = s0 + (c - nobj - nlink - nbase);
      x = v3(d.stat_pos[k]);
      R = quat_mat(d.stat_quat[k]);
      hf = v3(d.stat_half[k]);
      kind = CK_STATIC; idx = k - s0;
    } else {
      shape = SHAPE_PLANE; kind = CK_PLANE; idx = 0;
    }
    sx[3 * c] = x.x; sx[3 * c + 1] = x.y; sx[3 * c + 2] = x.z;
    sR[9 * c + 0] = R.r0.x; sR[9 * c + 1] = R.r0.y; sR[9 * c + 2] = R.r0.z;
    sR[9 * c + 3] = R.r1.x; sR[9 * c + 4] = R.r1.y; sR[9 * c + 5] = R.r1.z;
    sR[9 * c + 6] = R.r2.x; sR[9 * c + 7] = R.r2.y; sR[9 * c + 8] = R.r2.z;
    sh[3 * c] = hf.x; sh[3 * c + 1] = hf.y; sh[3 * c + 2] = hf.z;
    V3 ext;
    if (shape == SHAPE_SPHERE) {
      ext = v3(hf.x, hf.x, hf.x);
    } else {
      ext.x = fabsf(R.r0.x) * hf.x + fabsf(R.r0.y) * hf.y + fabsf(R.r0.z) * hf.z;
      ext.y = fabsf(R.r1.x) * hf.x + fabsf(R.r1.y) * hf.y + fabsf(R.r1.z) * hf.z;
      ext.z = fabsf(R.r2.x) * hf.x + fabsf(R.r2.y) * hf.y + fabsf(R.r2.z) * hf.z;
    }
    const int info = shape | (kind << 4) | (idx << 8);
    // broadphase group: the articulation's index for its links and base, a value of
    // its own (negative) for every other collider -- a pair within a group is skipped
    const int group = (kind == CK_LINK || kind == CK_BASE) ? idx : -1 - c;
    sbox[2 * c] = make_float4((x.x - ext.x) - h, (x.y - ext.y) - h, (x.z - ext.z) - h, __int_as_float(info));
    sbox[2 * c + 1] = make_float4((x.x + ext.x) + h, (x.y + ext.y) + h, (x.z + ext.z) + h, __int_as_float(group));
    sinfo[c] = info;
  }
  // awake mask of the objects (bit per local object index)
  unsigned long long awake = 0ull;
  for (int c0 = 0; c0 < nobj; c0 += 32) {
    int c = c0 + lane;
    bool aw = c < nobj && d.obj_awake[o0 + c] != 0;
    if (c < nobj) {  // v* = v + dt g for awake objects (before the wake pass), zero while asleep
      float4 v = d.obj_vel[o0 + c], w = d.obj_omega[o0 + c];
      d.obj_vstar[o0 + c] = aw ? make_float4(v.x + d.gx * d.dt, v.y + d.gy * d.dt, v.z + d.gz * d.dt, 0.f)
                               : make_float4(0.f, 0.f, 0.f, 0.f);
      d.obj_wstar[o0 + c] = aw ? make_float4(w.x, w.y, w.z, 0.f) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    unsigned b = __ballot_sync(0xffffffffu, aw);
    awake |= (unsigned long long)b << c0;
  }
  __syncwarp();

  // ---- 2. broadphase, ascending (a, b).  Every candidate pair has a dynamic
  //      collider (object or link), and those come first, so a runs over the
  //      dynamic colliders, one per lane; b sweeps all colliders in order for the
  //      whole warp (its data is a shared-memory broadcast) and each lane keeps a
  //      bit per candidate b; a prefix sum then writes the pairs in (a, b) order.
  const int ndyn = nobj + nlink;
  const int plane_b = plane ? nc - 1 : -1;  // the plane is the last collider
  int npairs = 0;
  for (int abase = 0; abase < ndyn; abase += 32) {
    const int a = abase + lane;
    unsigned long long m0 = 0ull, m1 = 0ull;  // candidate b < 64, b >= 64 (at most 128 colliders)
    const bool on = a < ndyn;
    const float4 la = sbox[2 * (on ? a : 0)], ua = sbox[2 * (on ? a : 0) + 1];
    const int ga = __float_as_int(ua.w);
    const bool below = la.z <= h;
#pragma unroll 4
    for (int b = abase + 1; b < nc; ++b) {
      const float4 lb = sbox[2 * b], ub = sbox[2 * b + 1];  // same address on every lane: broadcast
      bool cand = on && b > a && __float_as_int(ub.w) != ga;
      if (b == plane_b) cand = cand && below;
      else cand = cand && !(la.x > ub.x || lb.x > ua.x || la.y > ub.y || lb.y > ua.y || la.z > ub.z || lb.z > ua.z);
      if (cand) {
        if (b < 64) m0 |= 1ull << b;
        else m1 |= 1ull << (b - 64);
      }
    }
    const int cnt = __popcll(m0) + __popcll(m1);
    int incl = cnt;
    for (int o = 1; o < 32; o <<= 1) {
      int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    int pos = npairs + incl - cnt;
    while (m0) {
      const int bb = __ffsll((long long)m0) - 1;
      m0 &= m0 - 1ull;
      if (pos < PAIR_CAP) spairs[pos] = (unsigned short)((a << 8) | bb);
      ++pos;
    }
    while (m1) {
      const int bb = 64 + __ffsll((long long)m1) - 1;
      m1 &= m1 - 1ull;
      if (pos < PAIR_CAP) spairs[pos] = (unsigned short)((a << 8) | bb);
      ++pos;
    }
    npairs += total;
  }
  if (npairs > PAIR_CAP) { status |= ST_OVERFLOW; npairs = PAIR_CAP; }
  __syncwarp();

  // ---- 3. wake pass (sequential in pair order; only when some object sleeps).  Only
  //      a pair of two objects or links with an object asleep at the start of the
  //      pass can wake anything (awake flags only grow): the lanes flag those 32 pairs
  //      at a time and the warp applies the rule to the flagged ones in pair order.
  const unsigned long long all_obj = nobj >= 64 ? ~0ull : ((1ull << nobj) - 1ull);
  if (d.sleep_enabled && (awake & all_obj) != all_obj) {
    const unsigned long long before = awake;
    for (int i0 = 0; i0 < npairs; i0 += 32) {
      const int i = i0 + lane;
      int a = 0, b = 0, ka = 0, kb = 0;
      bool rel = false;
      if (i < npairs) {
        a = spairs[i] >> 8;
        b = spairs[i] & 0xff;
        ka = (sinfo[a] >> 4) & 15;
        kb = (sinfo[b] >> 4) & 15;
        const bool sleepy = (ka == CK_OBJ && !((before >> a) & 1ull)) || (kb == CK_OBJ && !((before >> b) & 1ull));
        rel = sleepy && (ka == CK_OBJ || ka == CK_LINK) && (kb == CK_OBJ || kb == CK_LINK);
      }
      unsigned m = __ballot_sync(0xffffffffu, rel);
      while (m) {  // warp-uniform
        const int l = __ffs(m) - 1;
        m &= m - 1u;
        const int pa = __shfl_sync(0xffffffffu, a, l), pb = __shfl_sync(0xffffffffu, b, l);
        const int pka = __shfl_sync(0xffffffffu, ka, l), pkb = __shfl_sync(0xffffffffu, kb, l);
        const bool sa = pka == CK_OBJ && !((awake >> pa) & 1ull);
        const bool sb = pkb == CK_OBJ && !((awake >> pb) & 1ull);
        const bool dyn_b = pkb == CK_LINK || (pkb == CK_OBJ && ((awake >> pb) & 1ull));
        const bool dyn_a = pka == CK_LINK || (pka == CK_OBJ && ((awake >> pa) & 1ull));
        if (sa && dyn_b) awake |= 1ull << pa;
        else if (sb && dyn_a) awake |= 1ull << pb;
      }
    }
    if (lane == 0) {
      unsigned long long woke = awake & ~before;
      while (woke) {
        int c = __ffsll((long long)woke) - 1;
        woke &= woke - 1;
        d.obj_awake[o0 + c] = 1;
        d.obj_ctr[o0 + c] = 0;
      }
    }
  }

  // ---- 4. keep pairs with an awake dynamic collider (in place, order kept)
  int nact = 0;
  for (int i0 = 0; i0 < npairs; i0 += 32) {
    int i = i0 + lane;
    int pr = i < npairs ? spairs[i] : 0;
    bool keep = false;
    if (i < npairs) {
      int a = pr >> 8, b = pr & 0xff;
      int ka = (sinfo[a] >> 4) & 15, kb = (sinfo[b] >> 4) & 15;
      bool dyn_a = ka == CK_LINK || (ka == CK_OBJ && ((awake >> a) & 1ull));
      bool dyn_b = kb == CK_LINK || (kb == CK_OBJ && ((awake >> b) & 1ull));
      keep = dyn_a || dyn_b;
    }
    unsigned m = __ballot_sync(0xffffffffu, keep);
    if (keep) {
      int pos = nact + __popc(m & ((1u << lane) - 1u));
      spairs[pos] = (unsigned short)pr;
      d.pairs[(size_t)e * PAIR_CAP + pos] = (pr >> 8) * 4096 + (pr & 0xff);
    }
    nact += __popc(m);
    __syncwarp();
  }
  if (lane == 0) d.pair_count[e] = nact;

  // ---- 5-6. narrowphase, one pair per lane, ordered output
  const int C = d.C;
  int ncontact = 0;
  for (int i0 = 0; i0 < nact; i0 += 32) {
    int i = i0 + lane;
    int cnt = 0;
    int a = 0, b = 0;
    if (i < nact) {
      a = spairs[i] >> 8;
      b = spairs[i] & 0xff;
      Coll A, B;
      A.shape = sinfo[a] & 15;
      B.shape = sinfo[b] & 15;
      A.x = v3(sx[3 * a], sx[3 * a + 1], sx[3 * a + 2]);
      B.x = v3(sx[3 * b], sx[3 * b + 1], sx[3 * b + 2]);
      A.R.r0 = v3(sR[9 * a], sR[9 * a + 1], sR[9 * a + 2]);
      A.R.r1 = v3(sR[9 * a + 3], sR[9 * a + 4], sR[9 * a + 5]);
      A.R.r2 = v3(sR[9 * a + 6], sR[9 * a + 7], sR[9 * a + 8]);
      B.R.r0 = v3(sR[9 * b], sR[9 * b + 1], sR[9 * b + 2]);
      B.R.r1 = v3(sR[9 * b + 3], sR[9 * b + 4], sR[9 * b + 5]);
      B.R.r2 = v3(sR[9 * b + 6], sR[9 * b + 7], sR[9 * b + 8]);
      A.h = v3(sh[3 * a], sh[3 * a + 1], sh[3 * a + 2]);
      B.h = v3(sh[3 * b], sh[3 * b + 1], sh[3 * b + 2]);
      cnt = narrowphase(A, B, d.margin, cand);
    }
    // exclusive prefix sum of the counts across the warp
    int incl = cnt;
    for (int o = 1; o < 32; o <<= 1) {
      int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    int total = __shfl_sync(0xffffffffu, incl, 31);
    int pos = ncontact + incl - cnt;
    const V3 nrm = cnt > 0 ? cand.n() : v3(0.f, 0.f, 0.f);
    for (int q = 0; q < cnt; ++q) {
      int slot = pos + q;
      if (slot < C) {
        size_t g = (size_t)e * C + slot;
        d.c_key[g] = make_int4(a, b, cand.f(q), 0);
        d.c_p[g] = f4(cand.p(q), cand.sep(q));
        d.c_n[g] = f4(nrm, 0.f);
      }
    }
    ncontact += total;
  }
  if (ncontact > C) { status |= ST_OVERFLOW; ncontact = C; }
  if (lane == 0) {
    d.n_contacts[e] = ncontact;
    if (status) atomicOr(&d.status[e], (int)status);
  }
}

}  // namespace gb
