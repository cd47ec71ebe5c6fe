// Critical-path depth of one step, by compiling the step functions (csrc/aba_step.cuh)
// on the host with a scalar type that carries, besides its value, the length of the
// longest chain of dependent floating-point operations that produced it (+ - * /
// sqrt sin cos each one level; a multiply feeding an add counts two, as if no
// multiply-add were fused).  Tape words and model constants enter at depth 0, as a
// warp that has them on chip sees them.  Prints, for a serial chain of n revolute
// links, the depth and the operation count of the forward step and of the adjoint
// step (without its recompute), and the depth of the adjoint's three passes.  With
// one warp per SM sub-partition a dependent level costs at least the FP32 pipe
// latency, so depth, not operation count, bounds a latency-bound step.
//
//   g++ -O1 -std=c++17 -o depthcount depthcount.cpp && ./depthcount 7
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>

static long long g_ops = 0;

struct Dp {
  double v;
  int d;
  Dp() : v(0), d(0) {}
  Dp(double x) : v(x), d(0) {}
  Dp(double x, int dd) : v(x), d(dd) {}
  Dp& operator+=(Dp o) { ++g_ops; v += o.v; d = std::max(d, o.d) + 1; return *this; }
  Dp& operator-=(Dp o) { ++g_ops; v -= o.v; d = std::max(d, o.d) + 1; return *this; }
  Dp& operator*=(Dp o) { ++g_ops; v *= o.v; d = std::max(d, o.d) + 1; return *this; }
};
inline Dp op(double v, Dp a, Dp b) { ++g_ops; return Dp(v, std::max(a.d, b.d) + 1); }
inline Dp operator+(Dp a, Dp b) { return op(a.v + b.v, a, b); }
inline Dp operator-(Dp a, Dp b) { return op(a.v - b.v, a, b); }
inline Dp operator*(Dp a, Dp b) { return op(a.v * b.v, a, b); }
inline Dp operator/(Dp a, Dp b) { return op(a.v / b.v, a, b); }
inline Dp operator-(Dp a) { return Dp(-a.v, a.d); }
inline Dp sqrt(Dp a) { ++g_ops; return Dp(std::sqrt(a.v), a.d + 1); }

#include "csrc/aba_step.cuh"

namespace abasim {
template <> inline void sincos_t<Dp>(Dp x, Dp* s, Dp* c) {
  g_ops += 2;
  *s = Dp(std::sin(x.v), x.d + 1);
  *c = Dp(std::cos(x.v), x.d + 1);
}
}  // namespace abasim

using namespace abasim;

constexpr int MAXN = 14;
static Dp prm[MAXN * NPRM * LANES], tape[MAXN * NTAPE * LANES], adj[MAXN * NADJ * LANES];
static int meta[MAXN * LANES];

static int max_depth(const Dp* x, int n, int stride) {
  int d = 0;
  for (int i = 0; i < n; ++i) d = std::max(d, x[i * stride].d);
  return d;
}

int main(int argc, char** argv) {
  const int n = argc > 1 ? std::max(1, std::min(MAXN, std::atoi(argv[1]))) : 7;
  for (int l = 0; l < n; ++l) {
    auto P = [&](int f) -> Dp& { return prm[(l * NPRM + f) * LANES]; };
    for (int f = 0; f < NPRM; ++f) P(f) = Dp(0.01 * (f + 1));
    const double E[9] = {0.36, 0.48, -0.8, -0.8, 0.6, 0.0, 0.48, 0.64, 0.6};
    for (int f = 0; f < 9; ++f) P(P_E + f) = Dp(E[f]);
    P(P_AX) = 0; P(P_AX + 1) = 0; P(P_AX + 2) = 1;
    P(P_M) = 1.0;
    P(P_IC) = 0.1; P(P_IC + 1) = 0.12; P(P_IC + 2) = 0.08;
    meta[l * LANES] = make_meta(l - 1, J_REVOLUTE, false, l, l);
  }
  Dp q[MAXN], qd[MAXN], tau[MAXN], gq[MAXN], gqd[MAXN], gtau[MAXN], gm[MAXN];
  for (int i = 0; i < n; ++i) { q[i] = 0.1 * i; qd[i] = 0.2; tau[i] = 0.3; gq[i] = 1; gqd[i] = 1; gm[i] = 0; }
  Sys<Dp> s{prm, meta, tape, adj, n};
  const V3<Dp> g{Dp(0), Dp(0), Dp(-9.81)};
  // forward step
  g_ops = 0;
  Dp q2[MAXN], qd2[MAXN];
  aba_forward<Dp, Dp, true>(s, Col<const Dp>{q, 1}, Col<const Dp>{qd, 1}, Col<const Dp>{tau, 1}, g);
  for (int i = 0; i < n; ++i) { q2[i] = q[i]; qd2[i] = qd[i]; }
  integrate<Dp>(s, Col<Dp>{q2, 1}, Col<Dp>{qd2, 1}, Dp(1e-3), I_SEMI_IMPLICIT);
  const long long fwd_ops = g_ops;
  const int fwd_depth = std::max(max_depth(q2, n, 1), max_depth(qd2, n, 1));
  // adjoint step from an on-chip tape: every tape word at depth 0
  for (Dp& t : tape) t.d = 0;
  g_ops = 0;
  step_adjoint<Dp, Dp>(s, Col<const Dp>{q, 1}, Col<const Dp>{qd, 1}, Col<Dp>{gq, 1}, Col<Dp>{gqd, 1},
                       Col<Dp>{gtau, 1}, Col<Dp>{gm, 1}, g, Dp(1e-3), I_SEMI_IMPLICIT);
  const long long adj_ops = g_ops;
  int adj_depth = std::max({max_depth(gq, n, 1), max_depth(gqd, n, 1), max_depth(gtau, n, 1), max_depth(gm, n, 1)});
  // depth reached at the end of pass 3 (the U, D and c adjoints), pass 2 (the p^A adjoints and
  // the inertia adjoint accumulators) and pass 1 (the outputs)
  int d3 = 0, d2 = 0;
  for (int l = 0; l < n; ++l) {
    d3 = std::max({d3, s.ad(l, G_D).d, s.ad(l, G_u).d});
    for (int i = 0; i < 6; ++i) d2 = std::max(d2, s.ad(l, G_PA + i).d);
    d2 = std::max(d2, s.ad(l, G_M).d);
  }
  std::printf("{\"links\": %d, \"forward\": {\"ops\": %lld, \"depth\": %d}, "
              "\"adjoint\": {\"ops\": %lld, \"depth\": %d, \"depth_after_pass3\": %d, \"depth_after_pass2\": %d}}\n",
              n, fwd_ops, fwd_depth, adj_ops, adj_depth, d3, d2);
  return 0;
}
