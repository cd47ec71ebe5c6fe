// Host check (FP64) of what the two-warp pipelined kernels compute differently
// from the one-warp kernels, on serial chains of 1 to 7 revolute links:
//  * the adjoint step on the compact tapes (the producer's LAY_PROD tape read
//    through the consumer's LAY_CONS adjoint layout) equals the adjoint step on
//    the full layout bit for bit, and no field a compact layout lacks is touched
//    (ABASIM_HOST_CHECKS aborts if one is);
//  * the split forward step (the inertia recursion, then the bias passes and the
//    integrator, as the inertia and bias warps run them) equals aba_forward +
//    integrate bit for bit, with one hand-off per link and per step.
// Prints one line per chain; exits non-zero on the first mismatch.
#define ABASIM_HOST_CHECKS 1
#include <cmath>
#include <cstdio>
#include <random>
#include <vector>

#include "../paper_2109_07719_gb300/csrc/aba_step.cuh"

using namespace abasim;
using D = double;

static std::mt19937_64 rng(9077190);
static D U(D lo = -1, D hi = 1) { return std::uniform_real_distribution<D>(lo, hi)(rng); }

int main() {
  const V3<D> g{0, 0, -9.81};
  for (int trial = 0; trial < 21; ++trial) {
    const int nl = 1 + trial % 7;
    const int integ = trial % 3 == 0 ? I_EXPLICIT : I_SEMI_IMPLICIT;
    std::vector<D> prm(nl * NPRM * LANES, 0.0);
    std::vector<int> meta(nl * LANES, 0);
    for (int l = 0; l < nl; ++l) {
      auto P = [&](int f) -> D& { return prm[(l * NPRM + f) * LANES]; };
      D qv[4], n = 0;
      for (D& v : qv) { v = U(); n += v * v; }
      n = std::sqrt(n);
      const M3<D> E = quat_R(qv[0] / n, qv[1] / n, qv[2] / n, qv[3] / n);
      for (int i = 0; i < 9; ++i) P(P_E + i) = E.a[i];
      for (int i = 0; i < 3; ++i) P(P_R + i) = l ? U(-0.3, 0.3) : 0.0;
      P(P_AX + 2) = 1.0;
      P(P_M) = U(0.5, 2.0);
      for (int i = 0; i < 3; ++i) P(P_C + i) = U(-0.1, 0.1);
      P(P_IC) = U(0.01, 0.1); P(P_IC + 1) = U(0.01, 0.1); P(P_IC + 2) = U(0.01, 0.1);
      P(P_IC + 3) = U(-0.003, 0.003); P(P_IC + 4) = U(-0.003, 0.003); P(P_IC + 5) = U(-0.003, 0.003);
      P(P_DAMP) = trial % 2 ? U(0.0, 0.1) : 0.0;
      meta[l * LANES] = make_meta(l - 1, J_REVOLUTE, false, l, l);
    }
    std::vector<D> q(nl), qd(nl), tau(nl), gq0(nl), gqd0(nl);
    for (int i = 0; i < nl; ++i) { q[i] = U(); qd[i] = U(-0.5, 0.5); tau[i] = U(); gq0[i] = U(); gqd0[i] = U(); }
    const Col<const D> qc{q.data(), 1}, qdc{qd.data(), 1}, tauc{tau.data(), 1};
    // adjoint step, full layout
    std::vector<D> tF(nl * NTAPE * LANES), aF(nl * NADJ * LANES);
    Sys<D> sf{prm.data(), meta.data(), tF.data(), aF.data(), nl, 1};
    std::vector<D> gqF = gq0, gqdF = gqd0, gtF(nl), gmF(nl, 0.0);
    aba_forward<D, D, true>(sf, qc, qdc, tauc, g);
    step_adjoint<D, D>(sf, qc, qdc, Col<D>{gqF.data(), 1}, Col<D>{gqdF.data(), 1}, Col<D>{gtF.data(), 1},
                       Col<D>{gmF.data(), 1}, g, 1e-3, integ);
    // adjoint step, the producer's tape read through the consumer's layout
    std::vector<D> tP(nl * NTAPE_PROD * LANES), aC(nl * NADJ_CONS * LANES);
    Sys<D, D, LAY_PROD, LAY_FULL> sp{prm.data(), meta.data(), tP.data(), nullptr, nl, 1};
    aba_forward<D, D, true>(sp, qc, qdc, tauc, g);
    Sys<D, D, LAY_PROD, LAY_CONS> sc{prm.data(), meta.data(), tP.data(), aC.data(), nl, 1};
    std::vector<D> gqC = gq0, gqdC = gqd0, gtC(nl), gmC(nl, 0.0);
    step_adjoint<D, D>(sc, qc, qdc, Col<D>{gqC.data(), 1}, Col<D>{gqdC.data(), 1}, Col<D>{gtC.data(), 1},
                       Col<D>{gmC.data(), 1}, g, 1e-3, integ);
    D e1 = 0;
    for (int i = 0; i < nl; ++i) {
      e1 = std::fmax(e1, std::fabs(gqF[i] - gqC[i]));
      e1 = std::fmax(e1, std::fabs(gqdF[i] - gqdC[i]));
      e1 = std::fmax(e1, std::fabs(gtF[i] - gtC[i]));
      e1 = std::fmax(e1, std::fabs(gmF[i] - gmC[i]));
    }
    // forward step: one pass against the inertia / bias split
    std::vector<D> qa = q, qda = qd, qb = q, qdb = qd;
    std::vector<D> tA(nl * NTAPE * LANES);
    Sys<D> sa{prm.data(), meta.data(), tA.data(), nullptr, nl, 1};
    aba_forward<D, D, false>(sa, Col<const D>{qa.data(), 1}, Col<const D>{qda.data(), 1}, tauc, g);
    integrate<D>(sa, Col<D>{qa.data(), 1}, Col<D>{qda.data(), 1}, 1e-3, integ);
    std::vector<D> ex(nl * EX_N * LANES), bs(nl * BS_N * LANES);
    Sys<D> sb{prm.data(), meta.data(), nullptr, nullptr, nl, 1};
    int readies = 0, waits = 0;
    chain_inertia<D, D>(sb, Col<const D>{qb.data(), 1}, ex.data(), [&](int) { ++readies; }, nl + 1);
    chain_bias_out(sb, Col<const D>{qb.data(), 1}, Col<const D>{qdb.data(), 1}, bs.data());
    chain_bias_in<D, D>(sb, Col<D>{qb.data(), 1}, Col<D>{qdb.data(), 1}, tauc, g, ex.data(), bs.data(),
                        [&](int) { ++waits; }, nl + 1, 1e-3, integ);
    D e2 = 0;
    for (int i = 0; i < nl; ++i) {
      e2 = std::fmax(e2, std::fabs(qa[i] - qb[i]));
      e2 = std::fmax(e2, std::fabs(qda[i] - qdb[i]));
    }
    std::printf("links %d adjoint_diff %.3g forward_diff %.3g handoffs %d/%d\n", nl, e1, e2, readies, waits);
    if (e1 != 0 || e2 != 0 || readies != nl + 1 || waits != nl + 1) return 1;
  }
  return 0;
}
