// Counts the floating-point operations of one forward step and one adjoint step
// of the kernels' formulations, by compiling the step functions (aba_step.cuh:
// link frames; wstep.cuh: world-aligned frames) on the host with a scalar type
// that counts +, -, *, / (each one FLOP; an FMA is two) and sqrt, sin, cos (one
// each).  Writes the per-link table to flops.json, which the throughput benchmark
// uses as the algorithmic FLOP count: "fwd" / "adj" for the link-frame step,
// "wfwd" (the rollout's step with the integrator), "wrec" (the adjoint's
// recompute, storing the tape) and "wadj" (the adjoint step) for the
// world-aligned one.
//
//   g++ -O1 -std=c++17 -o /tmp/flopcount flopcount.cpp && /tmp/flopcount > flops.json
#include <cmath>
#include <cstdio>

static long long g_flops = 0;

struct F {
  double v;
  F() : v(0) {}
  F(double x) : v(x) {}
  F& operator+=(F o) { ++g_flops; v += o.v; return *this; }
  F& operator-=(F o) { ++g_flops; v -= o.v; return *this; }
  F& operator*=(F o) { ++g_flops; v *= o.v; return *this; }
};
inline F operator+(F a, F b) { ++g_flops; return F(a.v + b.v); }
inline F operator-(F a, F b) { ++g_flops; return F(a.v - b.v); }
inline F operator*(F a, F b) { ++g_flops; return F(a.v * b.v); }
inline F operator/(F a, F b) { ++g_flops; return F(a.v / b.v); }
inline F operator-(F a) { return F(-a.v); }
inline F sqrt(F a) { ++g_flops; return F(std::sqrt(a.v)); }

#include "csrc/wstep.cuh"

namespace abasim {
template <> inline void sincos_t<F>(F x, F* s, F* c) { g_flops += 2; *s = F(std::sin(x.v)); *c = F(std::cos(x.v)); }
}  // namespace abasim

using namespace abasim;

struct Counts { long long fwd, adj; };

// one system of n links: link 0 is free or revolute, links 1.. revolute children of 0
static Counts count(int n, bool free_root) {
  const int B = 1;
  static F prm[8 * NPRM * LANES], tape[8 * NTAPE * LANES], adj[8 * NADJ * LANES];
  static int meta[8 * LANES];
  F q[64], qd[64], tau[64], gq[64], gqd[64], gtau[64], gm[8];
  int qo = 0, vo = 0;
  for (int l = 0; l < n; ++l) {
    const bool fr = free_root && l == 0;
    auto P = [&](int f) -> F& { return prm[(l * NPRM + f) * LANES]; };
    for (int f = 0; f < NPRM; ++f) P(f) = F(0.1 * (f + 1));
    for (int f = 0; f < 9; ++f) P(P_E + f) = F(f % 4 == 0 ? 1.0 : 0.0);
    P(P_AX) = 0; P(P_AX + 1) = 0; P(P_AX + 2) = 1;
    P(P_M) = 1;
    meta[l * LANES] = make_meta(l == 0 ? -1 : 0, fr ? J_FREE : J_REVOLUTE, false, qo, vo);
    qo += fr ? 7 : 1;
    vo += fr ? 6 : 1;
  }
  for (int i = 0; i < 64; ++i) { q[i] = F(0.1 * i); qd[i] = F(0.2); tau[i] = F(0.3); gq[i] = F(1); gqd[i] = F(1); gm[i % 8] = F(0); }
  if (free_root) { q[3] = 0; q[4] = 0; q[5] = 0; q[6] = 1; }
  Sys<F> s{prm, meta, tape, adj, n};
  V3<F> g{F(0), F(0), F(-9.81)};
  g_flops = 0;
  aba_forward<F, F>(s, Col<const F>{q, B}, Col<const F>{qd, B}, Col<const F>{tau, B}, g);
  F q2[64], qd2[64];
  for (int i = 0; i < 64; ++i) { q2[i] = q[i]; qd2[i] = qd[i]; }
  integrate<F>(s, Col<F>{q2, B}, Col<F>{qd2, B}, F(1e-3), I_SEMI_IMPLICIT);
  Counts c;
  c.fwd = g_flops;
  g_flops = 0;
  step_adjoint<F, F>(s, Col<const F>{q, B}, Col<const F>{qd, B}, Col<F>{gq, B}, Col<F>{gqd, B},
                  Col<F>{gtau, B}, Col<F>{gm, B}, g, F(1e-3), I_SEMI_IMPLICIT);
  c.adj = g_flops;
  return c;
}

struct WCounts { long long fwd, rec, adj; };

// the world-aligned step of a revolute chain of n links
static WCounts wcount(int n) {
  const int B = 1;
  static F prm[8 * NPRM * LANES], tape[8 * NWT * LANES], adj[8 * NWA * LANES];
  static int meta[8 * LANES];
  F q[64], qd[64], tau[64], gq[64], gqd[64], gtau[64], gm[8], q2[64], qd2[64];
  for (int l = 0; l < n; ++l) {
    auto P = [&](int f) -> F& { return prm[(l * NPRM + f) * LANES]; };
    for (int f = 0; f < NPRM; ++f) P(f) = F(0.1 * (f + 1));
    for (int f = 0; f < 9; ++f) P(P_E + f) = F(f % 4 == 0 ? 1.0 : 0.0);
    P(P_M) = 1;
    meta[l * LANES] = make_meta(l - 1, J_REVOLUTE, false, l, l);
  }
  for (int i = 0; i < 64; ++i) { q[i] = F(0.1 * i); qd[i] = F(0.2); tau[i] = F(0.3); gq[i] = F(1); gqd[i] = F(1); q2[i] = q[i]; qd2[i] = qd[i]; }
  for (int i = 0; i < 8; ++i) gm[i] = F(0);
  WSys<F> s{prm, meta, tape, adj, n};
  const V3<F> g{F(0), F(0), F(-9.81)};
  WCounts c;
  g_flops = 0;
  wstep_forward<F, F, false, true>(s, Col<const F>{q, B}, Col<const F>{qd, B}, Col<const F>{tau, B}, g, F(1e-3),
                                   I_SEMI_IMPLICIT, Col<F>{q2, B}, Col<F>{qd2, B});
  c.fwd = g_flops;
  g_flops = 0;
  wstep_forward<F, F, true, false>(s, Col<const F>{q, B}, Col<const F>{qd, B}, Col<const F>{tau, B}, g, F(1e-3),
                                   I_SEMI_IMPLICIT, Col<F>{q2, B}, Col<F>{qd2, B});
  c.rec = g_flops;
  g_flops = 0;
  wstep_adjoint<F, F>(s, Col<F>{gq, B}, Col<F>{gqd, B}, Col<F>{gtau, B},
                      Col<F>{gm, B}, F(1e-3), I_SEMI_IMPLICIT);
  c.adj = g_flops;
  return c;
}

int main() {
  Counts r1 = count(1, false), r2 = count(2, false), f1 = count(1, true);
  WCounts w1 = wcount(1), w2 = wcount(2);
  printf("{\n  \"convention\": \"+ - * / sqrt sin cos each count 1 FLOP (an FMA counts 2)\",\n");
  printf("  \"fwd\": {\"rev_root\": %lld, \"rev\": %lld, \"free_root\": %lld},\n", r1.fwd, r2.fwd - r1.fwd, f1.fwd);
  printf("  \"adj\": {\"rev_root\": %lld, \"rev\": %lld, \"free_root\": %lld},\n", r1.adj, r2.adj - r1.adj, f1.adj);
  printf("  \"wfwd\": {\"rev_root\": %lld, \"rev\": %lld},\n", w1.fwd, w2.fwd - w1.fwd);
  printf("  \"wrec\": {\"rev_root\": %lld, \"rev\": %lld},\n", w1.rec, w2.rec - w1.rec);
  printf("  \"wadj\": {\"rev_root\": %lld, \"rev\": %lld}\n}\n", w1.adj, w2.adj - w1.adj);
  return 0;
}
