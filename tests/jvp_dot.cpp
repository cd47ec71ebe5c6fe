// Dot-product test of the kernels' two derivatives of one step, built for the
// host in FP64: the forward-mode JVP (the step run on dual numbers, as the JVP
// kernel does) and the reverse-mode step_adjoint must be transposes of each
// other, <ybar, J xdot> = <J^T ybar, xdot> for random xdot = (qdot, qddot, taudot)
// and ybar = (qbar', qdbar'), to round-off -- no finite-difference error enters.
// Models: a floating base carrying a branched revolute tree, and a damped
// revolute chain under both integrators.  Prints: case name, max relative gap.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>
#include <vector>

#include "../paper_2109_07719_gb300/csrc/dual.cuh"

using namespace abasim;
using D = double;
using DD = Dual<double>;

static std::mt19937_64 rng(7190);
static D U(D lo = -1, D hi = 1) { return std::uniform_real_distribution<D>(lo, hi)(rng); }

constexpr int NL = 7;
static D prm[NL * NPRM * LANES], tape[NL * NTAPE * LANES], adjw[NL * NADJ * LANES];
static DD tape_d[NL * NTAPE * LANES];
static int meta[NL * LANES];

struct Model {
  int n, nq, nv, integ;
  std::vector<int> jt;
};

static Model build(const std::vector<int>& parent, const std::vector<int>& jt, bool damping, int integ) {
  Model md{(int)parent.size(), 0, 0, integ, jt};
  std::memset(prm, 0, sizeof prm);
  int qo = 0, vo = 0;
  for (int l = 0; l < md.n; ++l) {
    auto P = [&](int f) -> D& { return prm[(l * NPRM + f) * LANES]; };
    D qv[4], nn = 0;
    for (D& v : qv) { v = U(); nn += v * v; }
    nn = std::sqrt(nn);
    const M3<D> E = quat_R(qv[0] / nn, qv[1] / nn, qv[2] / nn, qv[3] / nn);
    for (int i = 0; i < 9; ++i) P(P_E + i) = E.a[i];
    for (int i = 0; i < 3; ++i) { P(P_R + i) = U(-0.3, 0.3); P(P_C + i) = U(-0.2, 0.2); }
    P(P_AX + 2) = jt[l] == J_REVOLUTE ? 1 : 0;
    P(P_M) = U(0.5, 2.0);
    P(P_IC) = U(0.05, 0.15); P(P_IC + 1) = U(0.05, 0.15); P(P_IC + 2) = U(0.05, 0.15);
    P(P_IC + 3) = U(-0.01, 0.01); P(P_IC + 4) = U(-0.01, 0.01); P(P_IC + 5) = U(-0.01, 0.01);
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
  return md;
}

static D gap(const Model& md) {
  const V3<D> g{0, 0, -9.81};
  const D dt = 1e-3;
  std::vector<D> q, qd(md.nv), tau(md.nv), dq(md.nq), dqd(md.nv), dtau(md.nv), wq(md.nq), wqd(md.nv);
  for (int l = 0; l < md.n; ++l) {
    if (md.jt[l] == J_FREE) {
      for (int i = 0; i < 3; ++i) q.push_back(U());
      D qv[4], nn = 0;
      for (D& v : qv) { v = U(); nn += v * v; }
      for (D v : qv) q.push_back(v / std::sqrt(nn));
    } else {
      q.push_back(U());
    }
  }
  for (D& v : qd) v = U();
  for (D& v : tau) v = 3 * U();
  for (D& v : dq) v = U();
  for (D& v : dqd) v = U();
  for (D& v : dtau) v = U();
  for (D& v : wq) v = U();
  for (D& v : wqd) v = U();
  // forward mode: the step on dual numbers
  std::vector<DD> xq(md.nq), xqd(md.nv), xt(md.nv);
  for (int i = 0; i < md.nq; ++i) xq[i] = DD(q[i], dq[i]);
  for (int i = 0; i < md.nv; ++i) { xqd[i] = DD(qd[i], dqd[i]); xt[i] = DD(tau[i], dtau[i]); }
  Sys<DD, D> sd{prm, meta, tape_d, nullptr, md.n};
  const V3<DD> gd{DD(g.x), DD(g.y), DD(g.z)};
  aba_forward<DD, DD, false>(sd, Col<const DD>{xq.data(), 1}, Col<const DD>{xqd.data(), 1},
                             Col<const DD>{xt.data(), 1}, gd);
  integrate<DD>(sd, Col<DD>{xq.data(), 1}, Col<DD>{xqd.data(), 1}, DD(dt), md.integ);
  D lhs = 0;
  for (int i = 0; i < md.nq; ++i) lhs += wq[i] * xq[i].d;
  for (int i = 0; i < md.nv; ++i) lhs += wqd[i] * xqd[i].d;
  // reverse mode: step_adjoint
  std::memset(adjw, 0, sizeof adjw);
  Sys<D> s{prm, meta, tape, adjw, md.n};
  std::vector<D> gq = wq, gqd = wqd, gtau(md.nv, 0.0), gm(md.n, 0.0);
  aba_forward<D, D, true>(s, Col<const D>{q.data(), 1}, Col<const D>{qd.data(), 1}, Col<const D>{tau.data(), 1}, g);
  step_adjoint<D, D>(s, Col<const D>{q.data(), 1}, Col<const D>{qd.data(), 1}, Col<D>{gq.data(), 1},
                     Col<D>{gqd.data(), 1}, Col<D>{gtau.data(), 1}, Col<D>{gm.data(), 1}, g, dt, md.integ);
  D rhs = 0;
  for (int i = 0; i < md.nq; ++i) rhs += gq[i] * dq[i];
  for (int i = 0; i < md.nv; ++i) rhs += gqd[i] * dqd[i] + gtau[i] * dtau[i];
  return std::fabs(lhs - rhs) / std::fmax(1.0, std::fabs(lhs));
}

int main() {
  const std::vector<int> tree_parent{-1, 0, 1, 2, 0, 4, 5};
  const std::vector<int> tree_jt{J_FREE, J_REVOLUTE, J_REVOLUTE, J_REVOLUTE, J_REVOLUTE, J_REVOLUTE, J_REVOLUTE};
  const std::vector<int> chain_parent{-1, 0, 1, 2, 3, 4};
  const std::vector<int> chain_jt(6, J_REVOLUTE);
  struct Case { const char* name; const std::vector<int>* p; const std::vector<int>* j; bool damp; int integ; };
  const Case cases[] = {{"floating_base_tree_semi_implicit", &tree_parent, &tree_jt, false, I_SEMI_IMPLICIT},
                        {"floating_base_tree_explicit", &tree_parent, &tree_jt, false, I_EXPLICIT},
                        {"damped_chain_semi_implicit", &chain_parent, &chain_jt, true, I_SEMI_IMPLICIT},
                        {"damped_chain_explicit", &chain_parent, &chain_jt, true, I_EXPLICIT}};
  for (const Case& c : cases) {
    D worst = 0;
    for (int t = 0; t < 10; ++t) {
      const Model md = build(*c.p, *c.j, c.damp, c.integ);
      worst = std::fmax(worst, gap(md));
    }
    std::printf("%s %.3e\n", c.name, worst);
  }
  return 0;
}
