// Central-difference check of the per-operation adjoint rules the kernels use
// (csrc/spatial.cuh, csrc/aba_step.cuh), compiled for the host in double
// precision.  For each rule a scalar L(x) = <ybar, f(x)> is differentiated along
// random directions by central differences and compared with <xbar, dx> from the
// rule.  Symmetric 6x6 quantities pair by the full-matrix Frobenius product (the
// kernels' convention), so a symmetric perturbation's off-diagonal entries count
// twice.  Rotation arguments are perturbed in their tangent space (dE = E skew(k)),
// the only directions the kernels differentiate along.  Also checks that the
// closed forms for a joint about e_z equal the general formulas at a = e_z.
// Prints one line per check: name, max relative error.
#include <cmath>
#include <cstdio>
#include <functional>
#include <random>
#include <vector>

#include "../paper_2109_07719_gb300/csrc/aba_step.cuh"

using namespace abasim;
using D = double;
using Vec = std::vector<D>;

static std::mt19937_64 rng(20210915);
static D U() { return std::uniform_real_distribution<D>(-1.0, 1.0)(rng); }

// flat parameter vector <-> structured values
struct Rd {
  const D* p;
  int i = 0;
  D s() { return p[i++]; }
  V3<D> v3() { const D a = s(), b = s(), c = s(); return {a, b, c}; }
  M3<D> m3() { M3<D> m; for (auto& x : m.a) x = s(); return m; }
  S3<D> s3() { S3<D> m; m.xx = s(); m.yy = s(); m.zz = s(); m.xy = s(); m.xz = s(); m.yz = s(); return m; }
  SV<D> sv() { const V3<D> w = v3(), v = v3(); return {w, v}; }
  SI<D> si() { const S3<D> A = s3(); const M3<D> B = m3(); const S3<D> C = s3(); return {A, B, C}; }
};
struct Wr {
  Vec v;
  void s(D x) { v.push_back(x); }
  void v3(V3<D> a) { s(a.x); s(a.y); s(a.z); }
  void m3(const M3<D>& m) { for (D x : m.a) s(x); }
  // gradient of a symmetric 3x3 under the full pairing: off-diagonals twice
  void s3g(const S3<D>& m) { s(m.xx); s(m.yy); s(m.zz); s(2 * m.xy); s(2 * m.xz); s(2 * m.yz); }
  void sv(SV<D> a) { v3(a.w); v3(a.v); }
  void sig(const SI<D>& m) { s3g(m.A); for (D x : m.B.a) s(2 * x); s3g(m.C); }
};

static M3<D> rand_rot() {  // orthonormal, det +1, from a random unit quaternion
  D q[4], n = 0;
  for (D& x : q) { x = U(); n += x * x; }
  n = std::sqrt(n);
  return quat_R(q[0] / n, q[1] / n, q[2] / n, q[3] / n);
}
static Vec rnd(int n) { Vec v(n); for (D& x : v) x = U(); return v; }

// max relative error over trials of the directional derivative.  x0: base point,
// dir(x0): a perturbation direction, L: the scalar, grad(x0): the rule's gradient
static D fd_check(const std::function<Vec()>& base, const std::function<Vec(const Vec&)>& dir,
                  const std::function<D(const Vec&)>& L, const std::function<Vec(const Vec&)>& grad,
                  int trials = 20) {
  D worst = 0;
  const D h = 1e-6;
  for (int t = 0; t < trials; ++t) {
    const Vec x = base();
    const Vec d = dir(x);
    Vec xp = x, xm = x;
    for (size_t i = 0; i < x.size(); ++i) { xp[i] += h * d[i]; xm[i] -= h * d[i]; }
    const D fd = (L(xp) - L(xm)) / (2 * h);
    const Vec g = grad(x);
    D an = 0;
    for (size_t i = 0; i < x.size(); ++i) an += g[i] * d[i];
    worst = std::fmax(worst, std::fabs(fd - an) / std::fmax(1.0, std::fabs(an)));
  }
  return worst;
}
static Vec any_dir(const Vec& x) { return rnd((int)x.size()); }
// direction with the first 9 entries (a rotation E) in the tangent space E skew(k)
static Vec rot_dir(const Vec& x) {
  Vec d = rnd((int)x.size());
  Rd r{x.data()};
  const M3<D> E = r.m3();
  const M3<D> dE = mm(E, skew(V3<D>{U(), U(), U()}));
  for (int i = 0; i < 9; ++i) d[i] = dE.a[i];
  return d;
}
static void report(const char* name, D err) { std::printf("%s %.3e\n", name, err); }

int main() {
  // crossm: y = m x n
  {
    const SV<D> yb{{U(), U(), U()}, {U(), U(), U()}};
    report("crossm_adj", fd_check([] { return rnd(12); }, any_dir,
        [&](const Vec& x) { Rd r{x.data()}; const SV<D> m = r.sv(), n = r.sv(); return dot(yb, crossm(m, n)); },
        [&](const Vec& x) {
          Rd r{x.data()}; const SV<D> m = r.sv(), n = r.sv();
          SV<D> mb = zeroSV<D>(), nb = zeroSV<D>();
          crossm_adj(m, n, yb, mb, nb);
          Wr w; w.sv(mb); w.sv(nb); return w.v; }));
  }
  // crossf: y = m x* f
  {
    const SV<D> yb{{U(), U(), U()}, {U(), U(), U()}};
    report("crossf_adj", fd_check([] { return rnd(12); }, any_dir,
        [&](const Vec& x) { Rd r{x.data()}; const SV<D> m = r.sv(), f = r.sv(); return dot(yb, crossf(m, f)); },
        [&](const Vec& x) {
          Rd r{x.data()}; const SV<D> m = r.sv(), f = r.sv();
          SV<D> mb = zeroSV<D>(), fb = zeroSV<D>();
          crossf_adj(m, f, yb, mb, fb);
          Wr w; w.sv(mb); w.sv(fb); return w.v; }));
  }
  // apply / applyT: y = X x, y = X^T x with X = (E, r)
  auto xf_base = [] { Wr w; w.m3(rand_rot()); for (int i = 0; i < 9; ++i) w.s(U()); return w.v; };
  for (int tr = 0; tr < 2; ++tr) {
    const SV<D> yb{{U(), U(), U()}, {U(), U(), U()}};
    auto f = [&](const XF<D>& X, SV<D> x) { return tr == 0 ? apply(X, x) : applyT(X, x); };
    report(tr == 0 ? "apply_adj" : "applyT_adj", fd_check(xf_base, rot_dir,
        [&](const Vec& v) { Rd r{v.data()}; const M3<D> E = r.m3(); const V3<D> rr = r.v3(); const SV<D> x = r.sv();
                            return dot(yb, f(XF<D>{E, rr}, x)); },
        [&](const Vec& v) {
          Rd r{v.data()}; const M3<D> E = r.m3(); const V3<D> rr = r.v3(); const SV<D> x = r.sv();
          M3<D> Eb = zeroM3<D>(); V3<D> rb = zero3<D>(); SV<D> xb = zeroSV<D>();
          if (tr == 0) apply_adj(XF<D>{E, rr}, x, yb, Eb, rb, &xb);
          else applyT_adj(XF<D>{E, rr}, x, yb, Eb, rb, &xb);
          Wr w; w.m3(Eb); w.v3(rb); w.sv(xb); return w.v; }));
  }
  // congruence: Y = X^T I X
  {
    Rd ry{nullptr};
    const Vec yv = rnd(21);
    ry.p = yv.data();
    const SI<D> Yb = ry.si();
    report("congruence_adj", fd_check([] { Wr w; w.m3(rand_rot()); for (int i = 0; i < 3 + 21; ++i) w.s(U()); return w.v; },
        rot_dir,
        [&](const Vec& v) { Rd r{v.data()}; const M3<D> E = r.m3(); const V3<D> rr = r.v3(); const SI<D> I = r.si();
                            return frob(Yb, congruence(XF<D>{E, rr}, I)); },
        [&](const Vec& v) {
          Rd r{v.data()}; const M3<D> E = r.m3(); const V3<D> rr = r.v3(); const SI<D> I = r.si();
          SI<D> Ib = zeroSI<D>(); M3<D> Eb = zeroM3<D>(); V3<D> rb = zero3<D>();
          congruence_adj(XF<D>{E, rr}, I, Yb, Ib, Eb, rb);
          Wr w; w.m3(Eb); w.v3(rb); w.sig(Ib); return w.v; }));
  }
  // mass derivatives of the rigid-body inertia (c and Ic fixed)
  {
    const V3<D> c{U(), U(), U()};
    const S3<D> Ic{0.3, 0.2, 0.4, 0.01, -0.02, 0.03};
    const Vec mv = rnd(21);
    Rd rm{mv.data()};
    const SI<D> Mb = rm.si();
    report("rbi_dmass", fd_check([] { return Vec{1.0 + 0.5 * U()}; }, any_dir,
        [&](const Vec& v) { return frob(Mb, rbi(v[0], c, Ic)); },
        [&](const Vec&) { return Vec{rbi_dmass(Mb, c)}; }));
    const SV<D> z{{U(), U(), U()}, {U(), U(), U()}}, x{{U(), U(), U()}, {U(), U(), U()}};
    report("rbi_dmass_bilinear", fd_check([] { return Vec{1.0 + 0.5 * U()}; }, any_dir,
        [&](const Vec& v) { return dot(z, mul(rbi(v[0], c, Ic), x)); },
        [&](const Vec&) { return Vec{rbi_dmass_bilinear(z, x, c)}; }));
  }
  // joint rotation derivatives: general axis and the closed form about e_z
  {
    D a[3] = {U(), U(), U()};
    const D n = std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    const V3<D> ax{a[0] / n, a[1] / n, a[2] / n};
    M3<D> Gb = zeroM3<D>(), Et = rand_rot(), Eb = zeroM3<D>();
    for (D& g : Gb.a) g = U();
    for (D& g : Eb.a) g = U();
    report("rot_axis_T_dq", fd_check([] { return Vec{3 * U()}; }, any_dir,
        [&](const Vec& v) { return frob(Gb, rot_axis_T(ax, std::sin(v[0]), std::cos(v[0]))); },
        [&](const Vec& v) { return Vec{rot_axis_T_dq(ax, std::sin(v[0]), std::cos(v[0]), Gb)}; }));
    report("rotz_T_dq", fd_check([] { return Vec{3 * U()}; }, any_dir,
        [&](const Vec& v) { return frob(Eb, rotz_T_mm(std::sin(v[0]), std::cos(v[0]), Et)); },
        [&](const Vec& v) { return Vec{rotz_T_dq(std::sin(v[0]), std::cos(v[0]), Eb, Et)}; }));
    // closed forms against the general formulas at a = e_z
    D worst = 0, worst_dq = 0;
    for (int t = 0; t < 20; ++t) {
      const D q = 3 * U(), s = std::sin(q), c = std::cos(q);
      const M3<D> g = mm(rot_axis_T(zaxis<D>(), s, c), Et), z = rotz_T_mm(s, c, Et);
      for (int i = 0; i < 9; ++i) worst = std::fmax(worst, std::fabs(g.a[i] - z.a[i]));
      worst_dq = std::fmax(worst_dq, std::fabs(rot_axis_T_dq(zaxis<D>(), s, c, mmT(Eb, Et)) - rotz_T_dq(s, c, Eb, Et)));
    }
    report("rotz_T_mm_equals_general", worst);
    report("rotz_T_dq_equals_general", worst_dq);
  }
  // the velocity-product term of a joint about e_z and its adjoint
  {
    const SV<D> yb{{U(), U(), U()}, {U(), U(), U()}};
    report("crossm_z_adj", fd_check([] { return rnd(7); }, any_dir,
        [&](const Vec& x) { Rd r{x.data()}; const SV<D> m = r.sv(); return dot(yb, crossm_z(m, r.s())); },
        [&](const Vec& x) {
          Rd r{x.data()}; const SV<D> m = r.sv(); const D qd = r.s();
          SV<D> mb = zeroSV<D>();
          const D qdb = crossm_z_adj(m, qd, yb, mb);
          Wr w; w.sv(mb); w.s(qdb); return w.v; }));
    D worst = 0;
    for (int t = 0; t < 20; ++t) {
      const Vec x = rnd(7);
      Rd r{x.data()};
      const SV<D> m = r.sv();
      const D qd = r.s();
      const SV<D> n{{0, 0, qd}, {0, 0, 0}};
      const SV<D> a = crossm(m, n), b = crossm_z(m, qd);
      worst = std::fmax(worst, std::fabs(dot(a - b, a - b)));
      const Vec iv = rnd(21);
      Rd ri{iv.data()};
      const SI<D> I = ri.si();
      const SV<D> u1 = col_z(I), u2{mul(I.A, zaxis<D>()), mulT(I.B, zaxis<D>())};
      worst = std::fmax(worst, std::fabs(dot(u1 - u2, u1 - u2)));
    }
    report("crossm_z_col_z_equal_general", worst);
  }
  // rotation matrix of a quaternion
  {
    M3<D> Rb = zeroM3<D>();
    for (D& g : Rb.a) g = U();
    report("quat_R_adj", fd_check([] { return rnd(4); }, any_dir,
        [&](const Vec& v) { return frob(Rb, quat_R(v[0], v[1], v[2], v[3])); },
        [&](const Vec& v) { D qb[4] = {0, 0, 0, 0}; quat_R_adj(v[0], v[1], v[2], v[3], Rb, qb); return Vec(qb, qb + 4); }));
  }
  // a = (I^A)^-1 u of a free joint: ubar = (I^A)^-1 abar, I^A bar = -sym(ubar a^T)
  {
    const SV<D> yb{{U(), U(), U()}, {U(), U(), U()}};
    auto spd = [](const Vec& v) {  // I^A = G G^T + 1 from the first 21 entries (kept symmetric)
      Rd r{v.data()};
      SI<D> I = r.si();
      I.A.xx += 4; I.A.yy += 4; I.A.zz += 4; I.C.xx += 4; I.C.yy += 4; I.C.zz += 4;
      return I;
    };
    report("spd_solve_adj", fd_check([] { return rnd(27); }, any_dir,
        [&](const Vec& v) { Rd r{v.data() + 21}; return dot(yb, spd_solve<D, D>(spd(v), r.sv())); },
        [&](const Vec& v) {
          Rd r{v.data() + 21};
          const SV<D> u = r.sv();
          const SI<D> I = spd(v);
          const SV<D> a = spd_solve<D, D>(I, u), ub = spd_solve<D, D>(I, yb);
          Wr w; w.sig(scale(D(-1), sym_outer(ub, a))); w.sv(ub); return w.v; }));
  }
  return 0;
}
