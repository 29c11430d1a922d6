"""Planted mistakes in the oracle, on the CPU: each mutant is a copy of the oracle's
source with one plausible mistake (a sign, a dropped term, an explicit instead of a
semi-implicit update, a wrong approximation, an off-by-one, a missing guard), in
every stage of the step, built into its own
library and run against the pin suite, which must fail for every mutant.  The
unmodified source, built and run the same way, must pass (the control), so that a
broken harness cannot pass as caught mutants.  Mutants that change nothing
(for example a pair filter that a later filter subsumes) are not listed.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.cpp")

MUTANTS = [
    ("gravity sign in the free-body predict",
     "if (o.awake) { S.v[i] = o.v + g * dt; S.w[i] = o.w; }", "if (o.awake) { S.v[i] = o.v - g * dt; S.w[i] = o.w; }"),
    ("positions advanced with the old velocity (explicit Euler)",
     "    o.v = S.v[i];\n    o.w = S.w[i];\n    o.x = o.x + o.v * dt;", "    o.x = o.x + o.v * dt;\n    o.v = S.v[i];\n    o.w = S.w[i];"),
    ("normal impulse allowed to pull",
     "real nl = Max(real(0), u.lam[0] + u.meff[0] * (u.target - v));", "real nl = u.lam[0] + u.meff[0] * (u.target - v);"),
    ("friction bound without the coefficient",
     "real lim = u.mu * u.lam[0];", "real lim = u.lam[0];"),
    ("ABA: articulated inertia passed to the parent without the projection",
     "Ia.m[r][c] = IA[i].m[r][c] - U[i].v[r] * U[i].v[c] / Dd[i];", "Ia.m[r][c] = IA[i].m[r][c];"),
    ("ABA: implicit-PD armature dropped",
     "Dd[i] = sdot(S[i], U[i]) + arm_of(A, i, dt);", "Dd[i] = sdot(S[i], U[i]);"),
    ("box-box SAT without the edge-edge axes",
     "bool use_edge = nvalid > 0 && emax > fmax + real(1e-3);", "bool use_edge = false;"),
    ("GELU by the tanh approximation",
     "static real gelu(real x) { return real(0.5) * x * (real(1) + Erf(x * real(0.70710678118654752440))); }",
     "static real gelu(real x) { return real(0.5) * x * (real(1) + std::tanh(real(0.7978845608028654) * (x + real(0.044715) * x * x * x))); }"),
    ("colouring starts at colour 1", "int c = 0;\n      while (c < 64", "int c = 1;\n      while (c < 64"),
    ("restitution ignored",
     "real e = Max(ca.kind == CK_OBJ", "real e = real(0) * Max(ca.kind == CK_OBJ"),
    ("Baumgarte correction with the wrong sign",
     "else tgt = -P.baumgarte * (c.sep + P.slop) / dt;", "else tgt = P.baumgarte * (c.sep + P.slop) / dt;"),
    ("sleep counter never reset", "else o.ctr = 0;", "else o.ctr = o.ctr;"),
    ("wake pass repeated to a fixed point (a closure over the contact graph)",
     "  if (P.sleep_enabled) {  // wake pass, ascending pair order, state updated in place",
     "  if (P.sleep_enabled) for (int rep = 0; rep < 64; ++rep) {  // wake pass, ascending pair order, state updated in place"),
    ("wake pass in descending pair order",
     "    for (auto& pr : cand) {\n      int a = pr.first, b = pr.second;\n      bool sa",
     "    for (auto it = cand.rbegin(); it != cand.rend(); ++it) {\n      auto& pr = *it;\n      int a = pr.first, b = pr.second;\n      bool sa"),
    ("quaternion update with the full angle", "real hw = real(0.5) * dt;", "real hw = dt;"),
    ("joint positions advanced with the old rate",
     "      A.j[i].qd = S.qd[k][i];\n      A.j[i].q = A.j[i].q + dt * A.j[i].qd;",
     "      A.j[i].q = A.j[i].q + dt * A.j[i].qd;\n      A.j[i].qd = S.qd[k][i];"),
    ("contact features: effective masses in reverse order",
     "for (int r = 0; r < 3; ++r) f[k++] = u.meff[r];", "for (int r = 0; r < 3; ++r) f[k++] = u.meff[2 - r];"),
    ("broadphase without the fattening margin", "real h = margin / 2;", "real h = 0;"),
    ("sphere-box normal pointing into the box", "    n = d * (real(1) / dist);\n    sep = dist - r;\n    pbox = pw;",
     "    n = d * (real(-1) / dist);\n    sep = dist - r;\n    pbox = pw;"),
    ("sphere inside a box pushed out along the deepest axis", "      if (d < best) { best = d; k = i; }",
     "      if (d > best) { best = d; k = i; }"),
    ("joint-limit rows with the side's sign swapped", "u.lsign = side == 1 ? real(1) : real(-1);",
     "u.lsign = side == 1 ? real(-1) : real(1);"),
    ("joint-limit effective mass from the inverse diagonal itself",
     "      u.meff[0] = real(1) / A.Minv[i][i];\n      // distance to the limit",
     "      u.meff[0] = A.Minv[i][i];\n      // distance to the limit"),
    ("motor impulse not capped",
     "real nl = u.is_limit == 2 ? Max(-u.bound, Min(u.bound, u.lam[0] + u.meff[0] * (u.target - v)))",
     "real nl = u.is_limit == 2 ? (u.lam[0] + u.meff[0] * (u.target - v))"),
    ("robot contact force as an impulse (no division by dt)", "f_robot += u.lam[0] / dt;", "f_robot += u.lam[0];"),
    ("prior-frame match ignores the distance", "ce.f == c.f && norm(ce.p - c.p) < P.match_dist) {", "ce.f == c.f) {"),
    ("ABA gravity with the wrong sign",
     "SV a0 = sv(V3(0, 0, 0), -g);  // gravity as an upward acceleration of the fixed base",
     "SV a0 = sv(V3(0, 0, 0), g);  // gravity as an upward acceleration of the fixed base"),
    ("restitution applied below the threshold speed", "if (vn < -P.rest_thresh) tgt = Max(tgt, -e * vn);",
     "if (vn > -P.rest_thresh) tgt = Max(tgt, -e * vn);"),
    ("no speculative contact target", "if (c.sep > 0) tgt = -c.sep / dt;", "if (c.sep > 0) tgt = 0;"),
    ("motor target without the division by dt", "u.target = P.motor_kp * (J.target - J.q) / dt;",
     "u.target = P.motor_kp * (J.target - J.q);"),
    ("world inverse inertia with the rotation transposed",
     "r.m[i][j] = R.m[i][0] * d.x * R.m[j][0] + R.m[i][1] * d.y * R.m[j][1] + R.m[i][2] * d.z * R.m[j][2];",
     "r.m[i][j] = R.m[0][i] * d.x * R.m[0][j] + R.m[1][i] * d.y * R.m[1][j] + R.m[2][i] * d.z * R.m[2][j];"),
    ("residual without the normalisation", "resid = Sqrt(d2) / Max(Sqrt(l2), real(P.lambda_floor));", "resid = Sqrt(d2);"),
    ("solid sphere inertia as a shell", "real I = real(0.4) * o.mass * o.half.x * o.half.x;",
     "real I = real(2.0 / 3.0) * o.mass * o.half.x * o.half.x;"),
    ("box-plane vertices kept beyond the margin", "        if (v.z > margin) continue;", "        if (v.z > 1e30) continue;"),
    ("normal impulse not accumulated across sweeps",
     "        unit_apply(E, S, u, 0, dl);\n        u.lam[0] = nl;\n        d2 += dl * dl; l2 += nl * nl;\n        for (int r = 1; r < 3; ++r) {",
     "        unit_apply(E, S, u, 0, dl);\n        d2 += dl * dl; l2 += nl * nl;\n        for (int r = 1; r < 3; ++r) {"),
    ("box-box contact normal not flipped for a reference face on A", "rc.n = refB ? nref : -nref;", "rc.n = nref;"),
    ("cached tangential impulse stored along t1 only", "ce.lt = u.d[1] * u.lam[1] + u.d[2] * u.lam[2];",
     "ce.lt = u.d[1] * u.lam[1];"),
    ("logged training target not normalised",
     "        t[r] = (u.lam[r] - feats[ui][23 + r]) / sc;", "        t[r] = u.lam[r] - feats[ui][23 + r];"),
    ("logged pairs include solves that missed the residual target",
     "    if (log && (P.pgs_tol <= 0 || E.resid <= real(P.pgs_tol))) {", "    if (log) {"),
    ("learned scale without the contact's relative velocity",
     "  return f[18] * (norm(g) * dt + Sqrt(f[9] * f[9] + f[10] * f[10] + f[11] * f[11]));",
     "  return f[18] * norm(g) * dt;"),
    ("learned gate closed for fast matched contacts",
     "  return Sqrt(f[9] * f[9] + f[10] * f[10] + f[11] * f[11]) > real(LEARN_GATE) * norm(g) * dt;",
     "  return false;"),
    ("learned gate open for every matched contact",
     "  return Sqrt(f[9] * f[9] + f[10] * f[10] + f[11] * f[11]) > real(LEARN_GATE) * norm(g) * dt;",
     "  return true;"),
    ("manifold reduction keeps the shallowest point first", "  int i1 = first_within(val, ex, 1e-5, false);",
     "  int i1 = first_within(val, ex, 1e-5, true);"),
    ("violated joint limit pushed back by the whole gap in one step",
     "u.target = cgap >= 0 ? -cgap / dt : -P.baumgarte * cgap / dt;", "u.target = -cgap / dt;"),
    ("clipped contact point on the incident face instead of midway", "    rc.p = P.p - nref * (sep * real(0.5));",
     "    rc.p = P.p;"),
    ("learned warm start scaled by the tangential effective mass",
     "  return f[18] * (norm(g) * dt + Sqrt(f[9] * f[9] + f[10] * f[10] + f[11] * f[11]));",
     "  return f[19] * (norm(g) * dt + Sqrt(f[9] * f[9] + f[10] * f[10] + f[11] * f[11]));"),
    ("learned tangential warm start not projected onto the pyramid",
     "          u.lam[1] = Max(-u.mu * ln, Min(u.mu * ln, feats[ui][24] + y[1] * sc));",
     "          u.lam[1] = feats[ui][24] + y[1] * sc;"),
    ("ABA without the velocity-product bias", "    pA[i] = crf(vel[i], smv(IA[i], vel[i]));",
     "    pA[i] = sv(V3(0, 0, 0), V3(0, 0, 0));"),
    ("robot force counted for every articulation",
     "auto robot = [&](int ci) { return (C[ci].kind == CK_LINK || C[ci].kind == CK_BASE) && E.art[C[ci].idx].kinematic; };",
     "auto robot = [&](int ci) { return (C[ci].kind == CK_LINK || C[ci].kind == CK_BASE); };"),
    ("prior friction clamped by mu alone",
     "          prev[1] = Max(-u.mu * ce.ln, Min(u.mu * ce.ln, dot(ce.lt, u.d[1])));",
     "          prev[1] = Max(-u.mu, Min(u.mu, dot(ce.lt, u.d[1])));"),
    ("box-plane contact point at the vertex instead of midway",
     "RawContact rc; rc.p = V3(v.x, v.y, v.z * real(0.5)); rc.n = V3(0, 0, 1); rc.sep = v.z; rc.f = k;",
     "RawContact rc; rc.p = V3(v.x, v.y, v.z); rc.n = V3(0, 0, 1); rc.sep = v.z; rc.f = k;"),
    ("articulation self-pairs not filtered", "  if (a_art && b_art && a.idx == b.idx) return false;\n", ""),
    ("a body put to sleep keeps its velocity", "{ o.awake = 0; o.v = V3(0, 0, 0); o.w = V3(0, 0, 0); }",
     "{ o.awake = 0; }"),
    ("contact capacity off by one",
     "if ((int)E.contacts.size() >= P.max_contacts) { E.status |= STATUS_OVERFLOW; break; }",
     "if ((int)E.contacts.size() > P.max_contacts) { E.status |= STATUS_OVERFLOW; break; }"),
    ("contact overflow not flagged",
     "if ((int)E.contacts.size() >= P.max_contacts) { E.status |= STATUS_OVERFLOW; break; }",
     "if ((int)E.contacts.size() >= P.max_contacts) { break; }"),
    ("prismatic joint's motion subspace taken as an angular axis",
     "  return sv(V3(0, 0, 0), a);\n}\nstatic SM link_inertia",
     "  return sv(a, V3(0, 0, 0));\n}\nstatic SM link_inertia"),
    ("contact unit's normal impulse applied after its friction rows",
     "        unit_apply(E, S, u, 0, dl);\n        u.lam[0] = nl;\n        d2 += dl * dl; l2 += nl * nl;\n        for (int r = 1; r < 3; ++r) {\n          real vt = unit_vel(E, S, u, r);\n          real lim = u.mu * u.lam[0];\n          real nt = Max(-lim, Min(lim, u.lam[r] - u.meff[r] * vt));\n          real dt_ = nt - u.lam[r];\n          unit_apply(E, S, u, r, dt_);\n          u.lam[r] = nt;\n          d2 += dt_ * dt_; l2 += nt * nt;\n        }",
     "        u.lam[0] = nl;\n        d2 += dl * dl; l2 += nl * nl;\n        for (int r = 1; r < 3; ++r) {\n          real vt = unit_vel(E, S, u, r);\n          real lim = u.mu * u.lam[0];\n          real nt = Max(-lim, Min(lim, u.lam[r] - u.meff[r] * vt));\n          real dt_ = nt - u.lam[r];\n          unit_apply(E, S, u, r, dt_);\n          u.lam[r] = nt;\n          d2 += dt_ * dt_; l2 += nt * nt;\n        }\n        unit_apply(E, S, u, 0, dl);"),
    ("joint-space inverse: back substitution with L instead of its transpose",
     "      for (int k = i + 1; k < n; ++k) s -= L[k][i] * x[k];",
     "      for (int k = i + 1; k < n; ++k) s -= L[i][k] * x[k];"),
    ("FK: joint rotation composed on the wrong side",
     "      A.R[i] = mmul(Rj, axis_angle(J.axis, J.q));",
     "      A.R[i] = mmul(axis_angle(J.axis, J.q), Rj);"),
    ("FK: joint origin offset not rotated by the parent",
     "    V3 oj = op + mv(Rp, J.opos);",
     "    V3 oj = op + J.opos;"),
    ("FK: link COM offset not rotated",
     "    A.c[i] = A.o[i] + mv(A.R[i], J.com);",
     "    A.c[i] = A.o[i] + J.com;"),
    ("FK: prismatic joint moves along its unrotated axis",
     "      A.o[i] = oj + a * J.q;",
     "      A.o[i] = oj + J.axis * J.q;"),
    ("spatial inertia: parallel-axis term with the wrong sign",
     "      r.m[i][j] = Ic.m[i][j] + m * s;",
     "      r.m[i][j] = Ic.m[i][j] - m * s;"),
    ("incident face: the least aligned axis",
     "    if (d > best) { best = d; m = q; }",
     "    if (d < best) { best = d; m = q; }"),
    ("incident face on the side facing the reference",
     "  real sg = dot(col(I.R, m), nref) > 0 ? real(-1) : real(1);",
     "  real sg = dot(col(I.R, m), nref) > 0 ? real(1) : real(-1);"),
    ("link contact Jacobian with the lever arm reversed",
     "        V3 sp = A.j[i].type == JT_REV ? cross(A.ja[i], p - A.jo[i]) : A.ja[i];",
     "        V3 sp = A.j[i].type == JT_REV ? cross(p - A.jo[i], A.ja[i]) : A.ja[i];"),
    ("limit rows left out of the colouring's nodes",
     "      u.node_a = (int)E.obj.size() + (int)k; u.node_b = -1;\n      u.lsign = side == 1",
     "      u.node_a = -1; u.node_b = -1;\n      u.lsign = side == 1"),
    ("manifold: second pick the nearest point",
     "  int i2 = first_within(val, ex, 1e-5, true);",
     "  int i2 = first_within(val, ex, 1e-5, false);"),
    ("manifold: third pick the smallest triangle",
     "  int i3 = first_within(val, ex, 1e-6, true);",
     "  int i3 = first_within(val, ex, 1e-6, false);"),
    ("manifold: fourth pick the smallest quadrilateral",
     "  int i4 = first_within(val, ex, 1e-6, true);",
     "  int i4 = first_within(val, ex, 1e-6, false);"),
    ("edge-edge contact point on edge A only",
     "    rc.p = (qa + qb) * real(0.5);",
     "    rc.p = qa;"),
    ("edge-edge closest points without clamping to the edges",
     "    s = Max(-A.half[i], Min(A.half[i], s));",
     "    s = s;"),
    ("features: relative angular velocity reversed",
     "  V3 wr = wa - wb;",
     "  V3 wr = wb - wa;"),
    ("features: plane endpoint at the contact point itself",
     "(cb.shape == SHAPE_PLANE ? V3(c.p.x, c.p.y, 0) : cb.x);",
     "(cb.shape == SHAPE_PLANE ? c.p : cb.x);"),
    ("features: pair type sphere-box read as box-box",
     "  else if (ca.shape == SHAPE_SPHERE || cb.shape == SHAPE_SPHERE) type = 2;",
     "  else if (ca.shape == SHAPE_SPHERE || cb.shape == SHAPE_SPHERE) type = 4;"),
    ("features: gravity term without dt",
     "  f[k++] = dot(g, c.n) * dt;",
     "  f[k++] = dot(g, c.n);"),
    ("pair restitution by the smaller coefficient",
     "    real e = Max(ca.kind == CK_OBJ ? E.obj[ca.idx].rest : real(0), cb.kind == CK_OBJ ? E.obj[cb.idx].rest : real(0));",
     "    real e = Min(ca.kind == CK_OBJ ? E.obj[ca.idx].rest : real(0), cb.kind == CK_OBJ ? E.obj[cb.idx].rest : real(0));"),
]


def test_every_planted_mistake_fails_a_pin(tmp_path):
    src = open(SRC).read()
    cases = [("control (unmodified)", None, None)] + MUTANTS
    builds = []
    for i, (name, old, new) in enumerate(cases):
        d = tmp_path / f"m{i}"
        d.mkdir()
        if old is not None:
            assert src.count(old) == 1, f"mutation site not found once: {name}"
        (d / "oracle.cpp").write_text(src if old is None else src.replace(old, new))
        builds.append(subprocess.Popen(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", str(d / "oracle.cpp"),
                                        "-o", str(d / "liboracle.so"), "-lpthread"]))
    assert all(b.wait() == 0 for b in builds)
    runs = []
    for i, (name, _, _) in enumerate(cases):
        env = dict(os.environ, ORACLE_LIBDIR=str(tmp_path / f"m{i}"))
        runs.append((name, subprocess.Popen([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                                             "-x", "-q", "-p", "no:cacheprovider"], cwd=ROOT, env=env,
                                            stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)))
    results = {}
    for name, p in runs:
        out = p.communicate(timeout=600)[0]
        results[name] = (p.returncode, out)
    rc, out = results.pop("control (unmodified)")
    assert rc == 0, out[-2000:]
    survivors = [name for name, (rc, _) in results.items() if rc == 0]
    assert not survivors, f"mutants no pin caught: {survivors}"
