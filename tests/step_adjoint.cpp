// Central-difference check of the kernels' whole adjoint step, built for the
// host in FP64 from csrc/aba_step.cuh: the forward step (jcalc, the three ABA
// passes, the integrator) maps (q, qd, tau, m) to (q', qd'); step_adjoint pulls
// (qbar', qdbar') back to (qbar, qdbar, taubar, mbar).  For random models -- a
// floating base carrying a branched tree of revolute joints, a damped revolute
// chain, and the explicit integrator -- the directional derivative of
// L = <qbar', q'> + <qdbar', qd'> along random directions is compared with the
// rule's gradient.  Revolute joints turn about their link's z axis (the frame
// the library chooses for every revolute link).  Prints: case name, max
// relative error.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>
#include <vector>

#include "../paper_2109_07719_gb300/csrc/aba_step.cuh"

using namespace abasim;
using D = double;

static std::mt19937_64 rng(2109077190);
static D U(D lo = -1, D hi = 1) { return std::uniform_real_distribution<D>(lo, hi)(rng); }

constexpr int MAXL = 8;
static D prm[MAXL * NPRM * LANES], tape[MAXL * NTAPE * LANES], adjw[MAXL * NADJ * LANES];
static int meta[MAXL * LANES];

struct Model {
  int n = 0, nq = 0, nv = 0, integ = I_SEMI_IMPLICIT;
  std::vector<int> parent, jt;
};

static void build(Model& md, const std::vector<int>& parent, const std::vector<int>& jt, bool damping) {
  md.parent = parent;
  md.jt = jt;
  md.n = (int)parent.size();
  std::memset(prm, 0, sizeof prm);
  int qo = 0, vo = 0;
  for (int l = 0; l < md.n; ++l) {
    auto P = [&](int f) -> D& { return prm[(l * NPRM + f) * LANES]; };
    D q4[4], nn = 0;
    for (D& x : q4) { x = U(); nn += x * x; }
    nn = std::sqrt(nn);
    const M3<D> E = quat_R(q4[0] / nn, q4[1] / nn, q4[2] / nn, q4[3] / nn);
    for (int i = 0; i < 9; ++i) P(P_E + i) = E.a[i];
    for (int i = 0; i < 3; ++i) {
      P(P_R + i) = U(-0.3, 0.3);
      P(P_C + i) = U(-0.2, 0.2);
    }
    P(P_AX + 2) = jt[l] == J_REVOLUTE ? 1 : 0;
    P(P_M) = U(0.5, 2.0);
    const D ic[6] = {U(0.05, 0.15), U(0.05, 0.15), U(0.05, 0.15), U(-0.01, 0.01), U(-0.01, 0.01), U(-0.01, 0.01)};
    for (int i = 0; i < 6; ++i) P(P_IC + i) = ic[i];
    P(P_DAMP) = (damping && jt[l] == J_REVOLUTE) ? U(0.0, 0.5) : 0.0;
    bool treechild = false;
    for (int c = l + 2; c < md.n; ++c)
      if (parent[c] == l) treechild = true;
    meta[l * LANES] = make_meta(parent[l], jt[l], treechild, qo, vo);
    qo += jt[l] == J_FREE ? 7 : 1;
    vo += jt[l] == J_FREE ? 6 : 1;
  }
  md.nq = qo;
  md.nv = vo;
}

// x = [q (nq), qd (nv), tau (nv), m (n)]
static std::vector<D> base_point(const Model& md) {
  std::vector<D> x;
  for (int l = 0; l < md.n; ++l) {
    if (md.jt[l] == J_FREE) {
      for (int i = 0; i < 3; ++i) x.push_back(U());
      D q4[4], nn = 0;
      for (D& v : q4) { v = U(); nn += v * v; }
      for (D v : q4) x.push_back(v / std::sqrt(nn));
    } else {
      x.push_back(U());
    }
  }
  for (int i = 0; i < md.nv; ++i) x.push_back(U());
  for (int i = 0; i < md.nv; ++i) x.push_back(3 * U());
  for (int l = 0; l < md.n; ++l) x.push_back(U(0.5, 2.0));
  return x;
}

static const V3<D> kGrav{0, 0, -9.81};
static const D kDt = 1e-3;

static D loss(const Model& md, const std::vector<D>& x, const std::vector<D>& wq, const std::vector<D>& wqd) {
  std::vector<D> q(x.begin(), x.begin() + md.nq), qd(x.begin() + md.nq, x.begin() + md.nq + md.nv);
  const D* tau = x.data() + md.nq + md.nv;
  for (int l = 0; l < md.n; ++l) prm[(l * NPRM + P_M) * LANES] = x[md.nq + 2 * md.nv + l];
  Sys<D> s{prm, meta, tape, adjw, md.n};
  aba_forward<D, D, false>(s, Col<const D>{q.data(), 1}, Col<const D>{qd.data(), 1}, Col<const D>{tau, 1}, kGrav);
  integrate<D>(s, Col<D>{q.data(), 1}, Col<D>{qd.data(), 1}, kDt, md.integ);
  D L = 0;
  for (int i = 0; i < md.nq; ++i) L += wq[i] * q[i];
  for (int i = 0; i < md.nv; ++i) L += wqd[i] * qd[i];
  return L;
}

static std::vector<D> gradient(const Model& md, const std::vector<D>& x, const std::vector<D>& wq,
                               const std::vector<D>& wqd) {
  std::vector<D> q(x.begin(), x.begin() + md.nq), qd(x.begin() + md.nq, x.begin() + md.nq + md.nv);
  const D* tau = x.data() + md.nq + md.nv;
  for (int l = 0; l < md.n; ++l) prm[(l * NPRM + P_M) * LANES] = x[md.nq + 2 * md.nv + l];
  std::memset(adjw, 0, sizeof adjw);
  Sys<D> s{prm, meta, tape, adjw, md.n};
  std::vector<D> gq = wq, gqd = wqd, gtau(md.nv, 0.0), gm(md.n, 0.0);
  aba_forward<D, D, true>(s, Col<const D>{q.data(), 1}, Col<const D>{qd.data(), 1}, Col<const D>{tau, 1}, kGrav);
  step_adjoint<D, D>(s, Col<const D>{q.data(), 1}, Col<const D>{qd.data(), 1}, Col<D>{gq.data(), 1},
                     Col<D>{gqd.data(), 1}, Col<D>{gtau.data(), 1}, Col<D>{gm.data(), 1}, kGrav, kDt, md.integ);
  std::vector<D> g = gq;
  g.insert(g.end(), gqd.begin(), gqd.end());
  g.insert(g.end(), gtau.begin(), gtau.end());
  g.insert(g.end(), gm.begin(), gm.end());
  return g;
}

static D check(const Model& md, int trials = 12) {
  D worst = 0;
  const D h = 1e-6;
  for (int t = 0; t < trials; ++t) {
    const std::vector<D> x = base_point(md);
    std::vector<D> wq(md.nq), wqd(md.nv), d(x.size());
    for (D& v : wq) v = U();
    for (D& v : wqd) v = U();
    for (D& v : d) v = U();
    std::vector<D> xp = x, xm = x;
    for (size_t i = 0; i < x.size(); ++i) { xp[i] += h * d[i]; xm[i] -= h * d[i]; }
    const D fd = (loss(md, xp, wq, wqd) - loss(md, xm, wq, wqd)) / (2 * h);
    const std::vector<D> g = gradient(md, x, wq, wqd);
    D an = 0;
    for (size_t i = 0; i < x.size(); ++i) an += g[i] * d[i];
    worst = std::fmax(worst, std::fabs(fd - an) / std::fmax(1.0, std::fabs(an)));
  }
  return worst;
}

int main() {
  Model a;  // floating base, two branches of revolute joints (link 4 is a second child of the base)
  build(a, {-1, 0, 1, 2, 0, 4, 5}, {J_FREE, J_REVOLUTE, J_REVOLUTE, J_REVOLUTE, J_REVOLUTE, J_REVOLUTE, J_REVOLUTE},
        false);
  std::printf("floating_base_tree %.3e\n", check(a));
  Model b;  // damped revolute chain
  build(b, {-1, 0, 1, 2, 3}, {J_REVOLUTE, J_REVOLUTE, J_REVOLUTE, J_REVOLUTE, J_REVOLUTE}, true);
  std::printf("damped_chain %.3e\n", check(b));
  Model c;  // revolute tree with two children at the root, explicit Euler
  build(c, {-1, 0, 1, 0, 3, 3}, {J_REVOLUTE, J_REVOLUTE, J_REVOLUTE, J_REVOLUTE, J_REVOLUTE, J_REVOLUTE}, true);
  c.integ = I_EXPLICIT;
  std::printf("revolute_tree_explicit %.3e\n", check(c));
  Model e;  // floating base alone, explicit Euler
  build(e, {-1}, {J_FREE}, false);
  e.integ = I_EXPLICIT;
  std::printf("free_body_explicit %.3e\n", check(e));
  return 0;
}
