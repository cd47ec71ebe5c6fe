// Host FP64 checks of the world-aligned step (csrc/wstep.cuh) without the oracle:
// (1) its joint accelerations equal those of the link-frame step
//     (csrc/aba_step.cuh, aba_forward) on the same packed model -- two
//     formulations of the same recursions, so they agree to rounding;
// (2) its adjoint (wstep_adjoint) against central differences of its own
//     forward step (with the integrator) in q, qd, tau and the link masses,
//     for serial chains, branched trees, damping and both integrators.
// Models are stored as the library stores them: links in depth-first preorder
// (csrc/tree_order.h), the branching flags in the meta words and a stack of
// parent values exactly as deep as the order needs, with NaN guard entries after
// it (a pass that overran the stack would read them back).
// Prints: case name, max relative error.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>
#include <vector>

#include "../paper_2109_07719_gb300/csrc/tree_order.h"
#include "../paper_2109_07719_gb300/csrc/wstep.cuh"

using namespace abasim;
using D = double;

static std::mt19937_64 rng(2109077191);
static D U(D lo = -1, D hi = 1) { return std::uniform_real_distribution<D>(lo, hi)(rng); }

constexpr int MAXL = 40;
static D prm[MAXL * NPRM * LANES], tape[MAXL * NTAPE * LANES], adjw[MAXL * NADJ * LANES];
static D wtape[MAXL * NWT * LANES], wadj[MAXL * NWA * LANES];
static int meta[MAXL * LANES];
static std::vector<D> wstk;  // depth + 2 guard entries, [entry][WSW][LANES]

struct Model {
  int n = 0, integ = I_SEMI_IMPLICIT, depth = 0;
  std::vector<int> parent;  // in stored (preorder) numbering
};

static void build(Model& md, const std::vector<int>& model_parent, bool damping) {
  const TreeOrder to = tree_order(model_parent.data(), (int)model_parent.size());
  md.parent = to.parent;
  md.n = (int)model_parent.size();
  md.depth = to.depth;
  wstk.assign((size_t)(md.depth + 2) * WSW * LANES, std::nan(""));
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
    meta[l * LANES] = make_meta(to.parent[l], J_REVOLUTE, to.branch[l], l, l, to.lastsib[l]);
  }
}

// the stack guard entries still NaN: no pass went past the depth the order gives
static bool guards_intact(const Model& md) {
  for (size_t i = (size_t)md.depth * WSW * LANES; i < wstk.size(); ++i)
    if (!std::isnan(wstk[i])) return false;
  return true;
}

static const V3<D> kGrav{0, 0, -9.81};
static const D kDt = 1e-3;
static V3<D> kGravD() { return kGrav; }
static D kDtD() { return kDt; }

// the adjoint's interleaved loop order (two links' independent work in one loop
// body, the kernels' choice with an FP32 global tape) or the plain one
static bool g_ilp = false;
template <bool ADJ, bool INTEG>
static void wfwd(const WSys<D>& s, const D* q, const D* qd, const D* tau, D* qo, D* qdo, int integ) {
  wstep_forward<D, D, ADJ, INTEG>(s, Col<const D>{q, 1}, Col<const D>{qd, 1}, Col<const D>{tau, 1}, kGravD(), kDtD(),
                                  integ, Col<D>{qo, 1}, Col<D>{qdo, 1});
}
static void wadjoint(const WSys<D>& s, D* gq, D* gqd, D* gtau, D* gm, int integ) {
  if (g_ilp)
    wstep_adjoint<D, D, true>(s, Col<D>{gq, 1}, Col<D>{gqd, 1}, Col<D>{gtau, 1}, Col<D>{gm, 1}, kDtD(), integ);
  else
    wstep_adjoint<D, D, false>(s, Col<D>{gq, 1}, Col<D>{gqd, 1}, Col<D>{gtau, 1}, Col<D>{gm, 1}, kDtD(), integ);
}

static WSys<D> wsys(const Model& md) {
  WSys<D> s{prm, meta, wtape, wadj, md.n};
  s.stk = wstk.data();
  return s;
}

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
    wfwd<true, false>(wsys(md), q.data(), qd.data(), tau.data(), q2.data(), qd2.data(), md.integ);
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
  wfwd<false, true>(wsys(md), q.data(), qd.data(), tau, q.data(), qd.data(), md.integ);
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
  wfwd<true, false>(wsys(md), q.data(), qd.data(), tau, q2.data(), qd2.data(), md.integ);
  wadjoint(wsys(md), gq.data(), gqd.data(), gtau.data(), gm.data(), md.integ);
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

// a random tree: each new link attaches to a uniformly drawn earlier link that has
// fewer than bf children
static std::vector<int> random_tree(int n, int bf) {
  std::vector<int> parent{-1}, kids(n, 0), open{0};
  for (int i = 1; i < n; ++i) {
    const int j = std::min((int)(U(0, 1) * open.size()), (int)open.size() - 1);
    const int p = open[j];
    parent.push_back(p);
    if (++kids[p] >= bf) open.erase(open.begin() + j);
    open.push_back(i);
  }
  return parent;
}

// the order's invariants on random trees and forests of 1..64 links: parents
// before children, contiguous subtrees, a link's first child at l + 1, and stack
// traffic that never pops an empty stack nor reads a missing top, ends empty and
// peaks at the depth the order reports, in both directions
static bool order_invariants() {
  for (int trial = 0; trial < 300; ++trial) {
    const int n = 1 + trial % 64, bf = 1 + trial % 3;
    std::vector<int> parent = random_tree(n, bf);
    if (trial % 7 == 0)
      for (int l = 1; l < n; l += 5) parent[l] = -1;  // a forest
    const TreeOrder t = tree_order(parent.data(), n);
    std::vector<int> seen(n, 0), size(n, 1);
    for (int l = 0; l < n; ++l) {
      if (t.pos[t.perm[l]] != l || seen[t.perm[l]]++) return false;
      const int p = t.parent[l];
      if (p >= l || (p >= 0 && parent[t.perm[l]] != t.perm[p]) || (p < 0 && parent[t.perm[l]] >= 0)) return false;
    }
    for (int l = n - 1; l > 0; --l)
      if (t.parent[l] >= 0) size[t.parent[l]] += size[l];
    for (int l = 0; l < n; ++l) {
      int kids = 0;
      for (int c = l + 1; c < n; ++c) {
        const bool inside = c < l + size[l];
        int a = c;
        while (a > l) a = t.parent[a];
        if ((a == l) != inside) return false;  // the subtree of l is exactly [l, l + size)
        if (t.parent[c] == l) {
          if (kids++ == 0 && c != l + 1) return false;
        }
      }
      if ((kids > 1) != (bool)t.branch[l]) return false;
    }
    int sp = 0, peak = 0;
    for (int l = 0; l < n; ++l) {  // outward: read (and on the last child pop) the top, then push
      const int p = t.parent[l];
      if (p >= 0 && p != l - 1 && sp == 0) return false;
      if (t.lastsib[l]) --sp;
      if (t.branch[l]) peak = std::max(peak, ++sp);
    }
    if (sp != 0 || peak != t.depth) return false;
    peak = 0;
    for (int l = n - 1; l >= 0; --l) {  // inward: pop the own entry, then push or add for the parent
      if (t.branch[l] && sp-- == 0) return false;
      const int p = t.parent[l];
      if (p >= 0 && p != l - 1) {
        if (t.lastsib[l]) peak = std::max(peak, ++sp);
        else if (sp == 0) return false;
      }
    }
    if (sp != 0 || peak != t.depth) return false;
  }
  return true;
}

int main() {
  std::printf("order_invariants %d\n", order_invariants() ? 1 : 0);
  struct Case { const char* name; std::vector<int> parent; bool damping; int integ; };
  // a caterpillar: spine links 0..8, then a leaf on each; a spine link's first
  // child continues the spine and its leaf comes later, so the stack grows with
  // the spine (depth 8)
  std::vector<int> cat{-1};
  for (int i = 1; i < 9; ++i) cat.push_back(i - 1);
  for (int i = 0; i < 9; ++i) cat.push_back(i);
  const Case cases[] = {
      {"chain", {-1, 0, 1, 2, 3, 4, 5}, false, I_SEMI_IMPLICIT},
      {"damped_chain", {-1, 0, 1, 2, 3}, true, I_SEMI_IMPLICIT},
      {"branched_tree", {-1, 0, 1, 0, 3, 3, 1, 6, 2}, false, I_SEMI_IMPLICIT},
      {"tree_explicit", {-1, 0, 0, 1, 1, 2, 2}, true, I_EXPLICIT},
      {"single_link", {-1}, true, I_SEMI_IMPLICIT},
      {"two_roots", {-1, 0, -1, 2, 2, 0}, true, I_SEMI_IMPLICIT},
      {"random_tree_bf2", random_tree(24, 2), false, I_SEMI_IMPLICIT},
      {"random_tree_bf3", random_tree(32, 3), true, I_SEMI_IMPLICIT},
      {"star", {-1, 0, 0, 0, 0, 0, 0}, false, I_EXPLICIT},
      {"caterpillar", cat, true, I_SEMI_IMPLICIT},
  };
  for (const Case& c : cases) {
    Model md;
    build(md, c.parent, c.damping);
    md.integ = c.integ;
    // both loop orders: the worse of the two against the references, and the two
    // against each other on one gradient
    D fw = 0, aj = 0;
    for (int ilp = 0; ilp < 2; ++ilp) {
      g_ilp = ilp;
      fw = std::fmax(fw, forward_agreement(md));
      aj = std::fmax(aj, adjoint_check(md));
    }
    std::printf("forward_%s %.3e\n", c.name, fw);
    std::printf("adjoint_%s %.3e\n", c.name, aj);
    {
      const int n = md.n;
      std::vector<D> x, wq(n), wqd(n);
      for (int i = 0; i < 4 * n; ++i) x.push_back(i >= 3 * n ? U(0.5, 2.0) : U());
      for (D& v : wq) v = U();
      for (D& v : wqd) v = U();
      g_ilp = false;
      const std::vector<D> g0 = gradient(md, x, wq, wqd);
      g_ilp = true;
      const std::vector<D> g1 = gradient(md, x, wq, wqd);
      D mx = 0, err = 0;
      for (size_t i = 0; i < g0.size(); ++i) {
        mx = std::fmax(mx, std::fabs(g0[i]));
        err = std::fmax(err, std::fabs(g0[i] - g1[i]));
      }
      std::printf("ilp_%s %.3e\n", c.name, err / std::fmax(mx, 1e-300));
    }
    std::printf("depth_%s %d\n", c.name, md.depth);
    std::printf("guards_%s %d\n", c.name, guards_intact(md) ? 1 : 0);
  }
  return 0;
}
