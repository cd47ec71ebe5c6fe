// Host FP64 checks of the world-aligned step (csrc/wstep.cuh) without the oracle:
// (1) its joint accelerations equal those of the link-frame step
//     (csrc/aba_step.cuh, aba_forward) on the same packed model -- two
//     formulations of the same recursions, so they agree to rounding;
// (2) its adjoint (wstep_adjoint) against central differences of its own
//     forward step (with the integrator) in q, qd, tau and the link masses,
//     for serial chains, branched trees, damping and both integrators.
// Prints: case name, max relative error.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>
#include <vector>

#include "../paper_2109_07719_gb300/csrc/wstep.cuh"

using namespace abasim;
using D = double;

static std::mt19937_64 rng(2109077191);
static D U(D lo = -1, D hi = 1) { return std::uniform_real_distribution<D>(lo, hi)(rng); }

constexpr int MAXL = 12;
static D prm[MAXL * NPRM * LANES], tape[MAXL * NTAPE * LANES], adjw[MAXL * NADJ * LANES];
static D wtape[MAXL * NWT * LANES], wadj[MAXL * NWA * LANES];
static int meta[MAXL * LANES];

struct Model {
  int n = 0, integ = I_SEMI_IMPLICIT;
  std::vector<int> parent;
};

static void build(Model& md, const std::vector<int>& parent, bool damping) {
  md.parent = parent;
  md.n = (int)parent.size();
  std::memset(prm, 0, sizeof prm);
  for (int l = 0; l < md.n; ++l) {
    auto P = [&](int f) -> D& { return prm[(l * NPRM + f) * LANES]; };
    D q4[4], nn = 0;
    for (D& x : q4) { x = U(); nn += x * x; }
    nn = std::sqrt(nn);
    const M3<D> E = quat_R(q4[0] / nn, q4[1] / nn, q4[2] / nn, q4[3] / nn);
    for (int i = 0; i < 9; ++i) P(P_E + i) = E.a[i];
    for (int i = 0; i < 3; ++i) {
      P(P_R + i) = U(-0.4, 0.4);
      P(P_C + i) = U(-0.2, 0.2);
    }
    P(P_AX + 2) = 1;
    P(P_M) = U(0.5, 2.0);
    const D ic[6] = {U(0.05, 0.15), U(0.05, 0.15), U(0.05, 0.15), U(-0.01, 0.01), U(-0.01, 0.01), U(-0.01, 0.01)};
    for (int i = 0; i < 6; ++i) P(P_IC + i) = ic[i];
    P(P_DAMP) = damping ? U(0.0, 0.5) : 0.0;
    bool treechild = false;
    for (int c = l + 2; c < md.n; ++c)
      if (parent[c] == l) treechild = true;
    meta[l * LANES] = make_meta(parent[l], J_REVOLUTE, treechild, l, l);
  }
}

static const V3<D> kGrav{0, 0, -9.81};
static const D kDt = 1e-3;

static WSys<D> wsys(const Model& md) { return WSys<D>{prm, meta, wtape, wadj, md.n}; }

// (1) joint accelerations of both formulations from random states
static D forward_agreement(const Model& md, int trials = 8) {
  D worst = 0;
  for (int t = 0; t < trials; ++t) {
    std::vector<D> q(md.n), qd(md.n), tau(md.n);
    for (int i = 0; i < md.n; ++i) { q[i] = 2 * U(); qd[i] = 3 * U(); tau[i] = U(); }
    Sys<D> s{prm, meta, tape, adjw, md.n};
    aba_forward<D, D, true>(s, Col<const D>{q.data(), 1}, Col<const D>{qd.data(), 1}, Col<const D>{tau.data(), 1},
                            kGrav);
    std::vector<D> q2 = q, qd2 = qd;
    wstep_forward<D, D, true, false>(wsys(md), Col<const D>{q.data(), 1}, Col<const D>{qd.data(), 1},
                                     Col<const D>{tau.data(), 1}, kGrav, kDt, md.integ, Col<D>{q2.data(), 1},
                                     Col<D>{qd2.data(), 1});
    D mx = 0, err = 0;
    for (int l = 0; l < md.n; ++l) {
      const D a = tape[(l * NTAPE + T_QDD) * LANES], b = wtape[(l * NWT + W_QDD) * LANES];
      mx = std::fmax(mx, std::fabs(a));
      err = std::fmax(err, std::fabs(a - b));
    }
    worst = std::fmax(worst, err / std::fmax(mx, 1e-300));
  }
  return worst;
}

// x = [q (n), qd (n), tau (n), m (n)]
static D loss(const Model& md, const std::vector<D>& x, const std::vector<D>& wq, const std::vector<D>& wqd) {
  const int n = md.n;
  std::vector<D> q(x.begin(), x.begin() + n), qd(x.begin() + n, x.begin() + 2 * n);
  const D* tau = x.data() + 2 * n;
  for (int l = 0; l < n; ++l) prm[(l * NPRM + P_M) * LANES] = x[3 * n + l];
  wstep_forward<D, D, false, true>(wsys(md), Col<const D>{q.data(), 1}, Col<const D>{qd.data(), 1},
                                   Col<const D>{tau, 1}, kGrav, kDt, md.integ, Col<D>{q.data(), 1},
                                   Col<D>{qd.data(), 1});
  D L = 0;
  for (int i = 0; i < n; ++i) L += wq[i] * q[i] + wqd[i] * qd[i];
  return L;
}

static std::vector<D> gradient(const Model& md, const std::vector<D>& x, const std::vector<D>& wq,
                               const std::vector<D>& wqd) {
  const int n = md.n;
  std::vector<D> q(x.begin(), x.begin() + n), qd(x.begin() + n, x.begin() + 2 * n);
  const D* tau = x.data() + 2 * n;
  for (int l = 0; l < n; ++l) prm[(l * NPRM + P_M) * LANES] = x[3 * n + l];
  for (D& v : wadj) v = std::nan("");  // every adjoint word is written before it is read
  std::vector<D> gq = wq, gqd = wqd, gtau(n, 0.0), gm(n, 0.0), q2 = q, qd2 = qd;
  wstep_forward<D, D, true, false>(wsys(md), Col<const D>{q.data(), 1}, Col<const D>{qd.data(), 1},
                                   Col<const D>{tau, 1}, kGrav, kDt, md.integ, Col<D>{q2.data(), 1},
                                   Col<D>{qd2.data(), 1});
  wstep_adjoint<D, D>(wsys(md), Col<const D>{q.data(), 1}, Col<const D>{qd.data(), 1}, Col<D>{gq.data(), 1},
                      Col<D>{gqd.data(), 1}, Col<D>{gtau.data(), 1}, Col<D>{gm.data(), 1}, kDt, md.integ);
  std::vector<D> g = gq;
  g.insert(g.end(), gqd.begin(), gqd.end());
  g.insert(g.end(), gtau.begin(), gtau.end());
  g.insert(g.end(), gm.begin(), gm.end());
  return g;
}

// (2) directional derivatives along random directions, and along each block alone
static D adjoint_check(const Model& md, int trials = 12) {
  D worst = 0;
  const D h = 1e-6;
  const int n = md.n;
  for (int t = 0; t < trials; ++t) {
    std::vector<D> x;
    for (int i = 0; i < n; ++i) x.push_back(2 * U());
    for (int i = 0; i < n; ++i) x.push_back(3 * U());
    for (int i = 0; i < n; ++i) x.push_back(U());
    for (int i = 0; i < n; ++i) x.push_back(U(0.5, 2.0));
    std::vector<D> wq(n), wqd(n);
    for (D& v : wq) v = U();
    for (D& v : wqd) v = U();
    const std::vector<D> g = gradient(md, x, wq, wqd);
    for (int block = -1; block < 4; ++block) {
      std::vector<D> d(x.size(), 0.0);
      for (size_t i = 0; i < x.size(); ++i)
        if (block < 0 || (int)i / n == block) d[i] = U();
      std::vector<D> xp = x, xm = x;
      for (size_t i = 0; i < x.size(); ++i) { xp[i] += h * d[i]; xm[i] -= h * d[i]; }
      const D fd = (loss(md, xp, wq, wqd) - loss(md, xm, wq, wqd)) / (2 * h);
      D an = 0;
      for (size_t i = 0; i < x.size(); ++i) an += g[i] * d[i];
      worst = std::fmax(worst, std::fabs(fd - an) / std::fmax(1.0, std::fabs(an)));
    }
  }
  return worst;
}

int main() {
  struct Case { const char* name; std::vector<int> parent; bool damping; int integ; };
  const Case cases[] = {
      {"chain", {-1, 0, 1, 2, 3, 4, 5}, false, I_SEMI_IMPLICIT},
      {"damped_chain", {-1, 0, 1, 2, 3}, true, I_SEMI_IMPLICIT},
      {"branched_tree", {-1, 0, 1, 0, 3, 3, 1, 6, 2}, false, I_SEMI_IMPLICIT},
      {"tree_explicit", {-1, 0, 0, 1, 1, 2, 2}, true, I_EXPLICIT},
      {"single_link", {-1}, true, I_SEMI_IMPLICIT},
  };
  for (const Case& c : cases) {
    Model md;
    build(md, c.parent, c.damping);
    md.integ = c.integ;
    std::printf("forward_%s %.3e\n", c.name, forward_agreement(md));
    std::printf("adjoint_%s %.3e\n", c.name, adjoint_check(md));
  }
  return 0;
}
