// Central-difference check of the kernels' constrained step, built for the host
// in FP64 from csrc/aba_step.cuh and csrc/contact.cuh: the forward step with
// sphere-ground contacts and joint-limit rows (the MLCP solved by projected
// Gauss-Seidel, its impulse folded into the integrator) and its adjoint in the
// order the adjoint kernels run it (integrator adjoint of every link with the
// constraint terms, the solver's adjoint, then the ABA adjoint with the
// constraint tape).  Model: a floating base with four two-link legs, a sphere on
// every foot, the base lowered until all four spheres penetrate the ground, and
// two knees past a limit.  Away from a change of active set or of a Gauss-Seidel
// projection the step is smooth, so L = <qbar', q'> + <qdbar', qd'> is
// differentiated along random directions by central differences and compared
// with the adjoint's gradient in q, qd, tau and the link masses.  Prints: case
// name, max relative error, and the number of active rows seen.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>
#include <vector>

#include "../paper_2109_07719_gb300/csrc/contact.cuh"

using namespace abasim;
using D = double;

static std::mt19937_64 rng(20210916);
static D U(D lo = -1, D hi = 1) { return std::uniform_real_distribution<D>(lo, hi)(rng); }

constexpr int NLINK = 9;
static D prm[NLINK * NPRM * LANES], tape[NLINK * NTAPE * LANES], adjw[NLINK * NADJ * LANES];
static D ct[NLINK * NCT * LANES], cs[NCS * LANES];
static int meta[NLINK * LANES];
static const int parent[NLINK] = {-1, 0, 1, 0, 3, 0, 5, 0, 7};
static int nq = 0, nv = 0;
static const V3<D> kGrav{0, 0, -9.81};
static const D kDt = 1e-3;
static const ContactParams<D> kCp{0.8, 0.2, 20};
static int g_rows = 0;

static M3<D> rand_rot(D spread) {
  D q[4] = {spread * U(), spread * U(), spread * U(), 1.0}, n = 0;
  for (D x : q) n += x * x;
  n = std::sqrt(n);
  return quat_R(q[0] / n, q[1] / n, q[2] / n, q[3] / n);
}

static void build() {
  std::memset(prm, 0, sizeof prm);
  int qo = 0, vo = 0;
  for (int l = 0; l < NLINK; ++l) {
    auto P = [&](int f) -> D& { return prm[(l * NPRM + f) * LANES]; };
    const bool base = l == 0, foot = l > 0 && l % 2 == 0;
    const M3<D> E = base ? rand_rot(0.0) : rand_rot(1.0);
    for (int i = 0; i < 9; ++i) P(P_E + i) = E.a[i];
    const V3<D> r = base ? V3<D>{0, 0, 0} : (l % 2 == 1 ? V3<D>{U(0.1, 0.2), U(0.1, 0.2), U(-0.1, 0.0)}
                                                         : V3<D>{U(-0.1, 0.1), U(-0.1, 0.1), U(-0.3, -0.2)});
    P(P_R) = r.x; P(P_R + 1) = r.y; P(P_R + 2) = r.z;
    for (int i = 0; i < 3; ++i) P(P_C + i) = U(-0.05, 0.05);
    P(P_AX + 2) = base ? 0 : 1;
    P(P_M) = base ? 5.0 : U(0.5, 1.5);
    const D ic[6] = {U(0.02, 0.1), U(0.02, 0.1), U(0.02, 0.1), U(-0.005, 0.005), U(-0.005, 0.005), U(-0.005, 0.005)};
    for (int i = 0; i < 6; ++i) P(P_IC + i) = ic[i];
    P(P_DAMP) = base ? 0.0 : 0.1;
    P(P_CR) = foot ? 0.03 : -1.0;
    if (foot)
      for (int i = 0; i < 3; ++i) P(P_CP + i) = U(-0.05, 0.05);
    P(P_LO) = -INFINITY;
    P(P_HI) = INFINITY;
    bool treechild = false;
    for (int c = l + 2; c < NLINK; ++c)
      if (parent[c] == l) treechild = true;
    meta[l * LANES] = make_meta(parent[l], base ? J_FREE : J_REVOLUTE, treechild, qo, vo);
    qo += base ? 7 : 1;
    vo += base ? 6 : 1;
  }
  nq = qo;
  nv = vo;
}

static Sys<D> sys() { return Sys<D>{prm, meta, tape, adjw, NLINK}; }
static CView<D> cview() { return CView<D>{ct, cs}; }
static void set_masses(const D* m) {
  for (int l = 0; l < NLINK; ++l) prm[(l * NPRM + P_M) * LANES] = m[l];
}

// x = [q (nq), qd (nv), tau (nv), m (links)]
static std::vector<D> base_point(int tr) {
  std::vector<D> x;
  for (int i = 0; i < 3; ++i) x.push_back(i == 2 ? 0.0 : U(-0.1, 0.1));
  D qv[4] = {0.1 * U(), 0.1 * U(), 0.1 * U(), 1.0}, n = 0;
  for (D v : qv) n += v * v;
  for (D v : qv) x.push_back(v / std::sqrt(n));
  for (int l = 1; l < NLINK; ++l) x.push_back(U(-0.3, 0.3));
  for (int i = 0; i < nv; ++i) x.push_back(0.3 * U());
  for (int i = 0; i < nv; ++i) x.push_back(i < 6 ? 0.0 : U());
  for (int l = 0; l < NLINK; ++l) x.push_back(prm[(l * NPRM + P_M) * LANES]);
  // lower the base until every foot sphere is at least 5 mm into the ground
  Sys<D> s = sys();
  aba_forward<D, D, false>(s, Col<const D>{x.data(), 1}, Col<const D>{x.data() + nq, 1},
                           Col<const D>{x.data() + nq + nv, 1}, kGrav);
  world_poses(s, cview());
  D worst = -1e9;
  for (int l = 2; l < NLINK; l += 2) {
    const V3<D> p = s.pv3(l, P_CP);
    const V3<D> y = cget3(cview(), l, C_OW) + mulT(cgetm(cview(), l, C_EW), p);
    worst = std::fmax(worst, y.z - s.P(l, P_CR));
  }
  x[2] = -worst - 0.005 - 0.01 * (tr % 3);
  // two knees past a limit by at least 0.05 rad (one above its range, one below)
  const int k1 = 7 + (2 - 1), k2 = 7 + (6 - 1);  // joint coordinates of links 2 and 6 (after the base's 7)
  prm[(2 * NPRM + P_HI) * LANES] = x[k1] - 0.05 - 0.02 * U(0, 1);
  prm[(2 * NPRM + P_LO) * LANES] = -INFINITY;
  prm[(6 * NPRM + P_LO) * LANES] = x[k2] + 0.05 + 0.02 * U(0, 1);
  prm[(6 * NPRM + P_HI) * LANES] = INFINITY;
  return x;
}

static D loss(const std::vector<D>& x, const std::vector<D>& wq, const std::vector<D>& wqd, int integ) {
  std::vector<D> q(x.begin(), x.begin() + nq), qd(x.begin() + nq, x.begin() + nq + nv);
  set_masses(x.data() + nq + 2 * nv);
  Sys<D> s = sys();
  const Col<const D> qc{q.data(), 1}, qdc{qd.data(), 1};
  aba_forward<D, D, false>(s, qc, qdc, Col<const D>{x.data() + nq + nv, 1}, kGrav);
  const int nr = contact_forward<D, D, D>(s, cview(), qc, qdc, kDt, kCp);
  g_rows = (int)cs[S_NC * LANES] * 3 + (int)cs[S_NL * LANES];
  std::vector<D> q2 = q, qd2 = qd;
  integrate<D>(s, Col<D>{q2.data(), 1}, Col<D>{qd2.data(), 1}, kDt, integ, nr > 0 ? (const D*)ct : nullptr);
  D L = 0;
  for (int i = 0; i < nq; ++i) L += wq[i] * q2[i];
  for (int i = 0; i < nv; ++i) L += wqd[i] * qd2[i];
  return L;
}

static std::vector<D> gradient(const std::vector<D>& x, const std::vector<D>& wq, const std::vector<D>& wqd,
                               int integ) {
  std::vector<D> q(x.begin(), x.begin() + nq), qd(x.begin() + nq, x.begin() + nq + nv);
  set_masses(x.data() + nq + 2 * nv);
  std::memset(adjw, 0, sizeof adjw);
  Sys<D> s = sys();
  const CView<D> cv = cview();
  const Col<const D> qc{q.data(), 1}, qdc{qd.data(), 1};
  std::vector<D> gq = wq, gqd = wqd, gtau(nv, 0.0), gm(NLINK, 0.0);
  const Col<D> gqc{gq.data(), 1}, gqdc{gqd.data(), 1};
  aba_forward<D, D, true>(s, qc, qdc, Col<const D>{x.data() + nq + nv, 1}, kGrav);
  const int nr = contact_forward<D, D, D>(s, cv, qc, qdc, kDt, kCp);
  if (nr > 0) {
    for (int l = 0; l < NLINK; ++l) {
      const int mt = s.M(l);
      D qb[6] = {0, 0, 0, 0, 0, 0};
      integrator_adjoint(s, l, meta_jtype(mt), meta_qoff(mt), meta_voff(mt), qc, qdc, gqc, gqdc, kDt, integ, qb,
                         (const D*)ct);
      for (int i = 0; i < 6; ++i) cv.L(l, C_QDDB + i) = qb[i];
    }
    contact_adjoint<D, D, D>(s, cv, kDt, kCp);
    step_adjoint<D, D>(s, qc, qdc, gqc, gqdc, Col<D>{gtau.data(), 1}, Col<D>{gm.data(), 1}, kGrav, kDt, integ,
                       (const D*)ct);
  } else {
    step_adjoint<D, D>(s, qc, qdc, gqc, gqdc, Col<D>{gtau.data(), 1}, Col<D>{gm.data(), 1}, kGrav, kDt, integ);
  }
  std::vector<D> g = gq;
  g.insert(g.end(), gqd.begin(), gqd.end());
  g.insert(g.end(), gtau.begin(), gtau.end());
  g.insert(g.end(), gm.begin(), gm.end());
  return g;
}

int main() {
  build();
  for (int integ : {I_SEMI_IMPLICIT, I_EXPLICIT}) {
    D worst = 0;
    int min_rows = 1 << 20;
    const D h = 1e-6;
    for (int t = 0; t < 12; ++t) {
      const std::vector<D> x = base_point(t);
      std::vector<D> wq(nq), wqd(nv), d(x.size());
      for (D& v : wq) v = U();
      for (D& v : wqd) v = U();
      for (D& v : d) v = U();
      for (int i = 0; i < 6; ++i) d[nq + nv + i] = 0;  // the base is unactuated
      std::vector<D> xp = x, xm = x;
      for (size_t i = 0; i < x.size(); ++i) { xp[i] += h * d[i]; xm[i] -= h * d[i]; }
      const D fd = (loss(xp, wq, wqd, integ) - loss(xm, wq, wqd, integ)) / (2 * h);
      loss(x, wq, wqd, integ);
      min_rows = std::min(min_rows, g_rows);
      const std::vector<D> g = gradient(x, wq, wqd, integ);
      D an = 0;
      for (size_t i = 0; i < x.size(); ++i) an += g[i] * d[i];
      worst = std::fmax(worst, std::fabs(fd - an) / std::fmax(1.0, std::fabs(an)));
    }
    std::printf("%s %.3e %d\n", integ == I_SEMI_IMPLICIT ? "contacts_limits_semi_implicit" : "contacts_limits_explicit",
                worst, min_rows);
  }
  return 0;
}
