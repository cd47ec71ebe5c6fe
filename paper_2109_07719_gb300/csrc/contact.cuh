// Contact and joint-limit resolution of one system (sphere contacts against the
// ground plane, revolute joint position limits) and its reverse-mode adjoint.
//
// Sec. 3.1 ("collision resolution", Eq. 8) poses the contact impulses as a mixed
// LCP  a = A x + b,  0 <= a _|_ x >= 0 on the normal rows, boxed friction rows,
// solved by projected Gauss-Seidel (the supplement's Alg. 1).  Here, per system
// and step, after the unconstrained ABA step:
//   * every contact sphere (centre p in its link's frame, radius r) is tested
//     against z = 0: gap phi = y_z - r, y = world centre; active when phi < 0;
//   * every limited revolute joint is tested against [lo, hi]: below the range
//     it gives a row J = +e_j with gap q - lo, above it J = -e_j with gap hi - q;
//     a limit row's impulse is >= 0, like a normal row;
//   * A = J M^-1 J^T of the active rows, J = world velocity Jacobian of the
//     sphere centres, then the limit rows.  Column j is one "test pass":
//     Featherstone's ABA run with zero velocity and gravity and row j's unit
//     impulse (a world force on its contact point, or a joint impulse), reusing
//     the step's articulated quantities (U, 1/D, X and the free root's
//     articulated inertia), so no mass matrix is formed;
//   * b = J v* + (erp/dt) phi on the normal and limit rows, v* = qd + dt qdd
//     (the velocity after the unconstrained step);
//   * a fixed number of Gauss-Seidel sweeps from lambda = 0: over the active
//     contacts, normal row first (projected onto lambda_n >= 0), then the x and
//     y friction rows (boxed by +-mu lambda_n with the current lambda_n), then
//     over the active limit rows (projected onto lambda >= 0);
//   * the velocity change M^-1 J^T lambda is one more test pass with all the
//     impulses applied at once; the integrator adds it to qd'.
// The adjoint reverses these steps exactly for a fixed active set: the final
// test pass, the Gauss-Seidel updates (from a tape of the impulse each update
// overwrote), the test passes of A's columns, b and the world kinematics.  It
// hands the step adjoint the adjoints of U, 1/D, the free root's articulated
// inertia, the link transforms, the unconstrained qdd, qd and (through the limit
// gaps) q (the B_* fields).
#pragma once

#include "../../include/abasim.h"
#include "aba_step.cuh"

#ifdef __CUDACC__
#define CD __host__ __device__ __noinline__
#else
#define CD inline
#endif

namespace abasim {

constexpr int MAXC = SIM_MAX_CONTACTS;         // contact spheres per system
constexpr int MAXL = SIM_MAX_LIMITS;           // limited joints per system
constexpr int NROW = 3 * MAXC + MAXL;          // impulse rows: world x, y, z per contact, then limits
constexpr int MAXPGS = SIM_MAX_PGS_ITERATIONS;  // Gauss-Seidel sweeps

// per-system contact record, [field][system]
enum : int {
  S_A = 0,                       // A of the active contacts, [row][col]
  S_B = S_A + NROW * NROW,       // b
  S_LAM = S_B + NROW,            // the impulse each Gauss-Seidel update overwrote, [sweep][row]
  S_LF = S_LAM + MAXPGS * NROW,  // lambda (final after the forward solve)
  S_PHI = S_LF + NROW,           // gap of each active contact [MAXC], then of each active limit [MAXL]
  S_LINK = S_PHI + MAXC + MAXL,  // link of each active contact, then of each active limit
  S_SGN = S_LINK + MAXC + MAXL,  // sign s of each active limit row (J = s e_j)
  S_NC = S_SGN + MAXL,           // number of active contacts
  S_NL = S_NC + 1,               // number of active limit rows
  S_AB = S_NL + 1,               // adjoint of A
  S_BB = S_AB + NROW * NROW,     // adjoint of b
  S_LB = S_BB + NROW,            // adjoint of lambda
  NCS = S_LB + NROW
};

template <class T> struct CView {
  T* ct;  // per-link contact tape of this system: [link][NCT][LANES] at its lane
  T* cs;  // per-system contact record: [NCS][LANES] at its lane
  SD T& L(int l, int f) const { return ct[(l * NCT + f) * LANES]; }
  SD T& S(int f) const { return cs[f * LANES]; }
};

template <class T> struct ContactParams {
  T mu;    // friction coefficient
  T erp;   // penetration correction rate
  int iters;  // Gauss-Seidel sweeps
};

// ------------------------------------------------------------------ field helpers
template <class T> SD V3<T> cget3(const CView<T>& c, int l, int f) { return {c.L(l, f), c.L(l, f + 1), c.L(l, f + 2)}; }
template <class T> SD void cput3(const CView<T>& c, int l, int f, V3<T> v) {
  c.L(l, f) = v.x; c.L(l, f + 1) = v.y; c.L(l, f + 2) = v.z;
}
template <class T> SD void cadd3(const CView<T>& c, int l, int f, V3<T> v) {
  c.L(l, f) += v.x; c.L(l, f + 1) += v.y; c.L(l, f + 2) += v.z;
}
template <class T> SD SV<T> cgetv(const CView<T>& c, int l, int f) { return {cget3(c, l, f), cget3(c, l, f + 3)}; }
template <class T> SD void cputv(const CView<T>& c, int l, int f, SV<T> v) { cput3(c, l, f, v.w); cput3(c, l, f + 3, v.v); }
template <class T> SD void caddv(const CView<T>& c, int l, int f, SV<T> v) { cadd3(c, l, f, v.w); cadd3(c, l, f + 3, v.v); }
template <class T> SD M3<T> cgetm(const CView<T>& c, int l, int f) {
  M3<T> m;
  for (int i = 0; i < 9; ++i) m.a[i] = c.L(l, f + i);
  return m;
}
template <class T> SD void cputm(const CView<T>& c, int l, int f, const M3<T>& m) {
  for (int i = 0; i < 9; ++i) c.L(l, f + i) = m.a[i];
}
template <class T> SD void caddm(const CView<T>& c, int l, int f, const M3<T>& m) {
  for (int i = 0; i < 9; ++i) c.L(l, f + i) += m.a[i];
}
template <class T> SD void caddsi(const CView<T>& c, int l, int f, const SI<T>& I) {
  const T a[6] = {I.A.xx, I.A.yy, I.A.zz, I.A.xy, I.A.xz, I.A.yz};
  const T b[6] = {I.C.xx, I.C.yy, I.C.zz, I.C.xy, I.C.xz, I.C.yz};
  for (int i = 0; i < 6; ++i) c.L(l, f + i) += a[i];
  for (int i = 0; i < 9; ++i) c.L(l, f + 6 + i) += I.B.a[i];
  for (int i = 0; i < 6; ++i) c.L(l, f + 15 + i) += b[i];
}

// ------------------------------------------------------------------ world kinematics
// E_w (world -> link rotation) and o (link origin in world coordinates) of every
// link: E_w = E E_w(parent), o = o(parent) + E_w(parent)^T r.
template <class T, class PT> SD void world_poses(const Sys<T, PT>& s, const CView<T>& cv) {
  for (int l = 0; l < s.nl; ++l) {
    const int par = meta_parent(s.M(l));
    const XF<T> X = tp_xf(s, l, T_E);
    if (par < 0) {
      cputm(cv, l, C_EW, X.E);
      cput3(cv, l, C_OW, X.r);
    } else {
      const M3<T> Ep = cgetm(cv, par, C_EW);
      cputm(cv, l, C_EW, mm(X.E, Ep));
      cput3(cv, l, C_OW, cget3(cv, par, C_OW) + mulT(Ep, X.r));
    }
  }
}

// ------------------------------------------------------------------ test pass
// Response of the articulated system at rest (no velocity or gravity) to
// external spatial forces fv[i] (link coordinates, at the link origin) on links
// fl[i] and joint impulses jv[i] on revolute joints jl[i]: the ABA's bias-force
// pass and acceleration pass with the step's U, 1/D, X and root articulated
// inertia.  Leaves the articulated bias forces (C_TP), joint forces (C_TU) and
// link accelerations (C_TA) on the contact tape, and the joint accelerations
// M^-1 (sum J_i^T f_i + sum e_j jv) in field qf (if qf >= 0).
template <class T, class DT, class PT>
CD void test_pass(Sys<T, PT> s, CView<T> cv, const int* fl, const SV<T>* fv, int nf, const int* jl, const T* jv,
                  int nj, int qf) {
  const int nl = s.nl;
  for (int l = 0; l < nl; ++l) cputv(cv, l, C_TP, zeroSV<T>());
  for (int l = nl - 1; l >= 0; --l) {
    const int m = s.M(l);
    const int par = meta_parent(m);
    SV<T> pA = cgetv(cv, l, C_TP);
    for (int i = 0; i < nf; ++i)
      if (fl[i] == l) pA -= fv[i];
    cputv(cv, l, C_TP, pA);
    if (meta_jtype(m) == J_REVOLUTE) {
      const V3<T> ax = s.pv3(l, P_AX);
      T u = -dot(ax, pA.w);
      for (int i = 0; i < nj; ++i)
        if (jl[i] == l) u += jv[i];
      cv.L(l, C_TU) = u;
      if (par >= 0) {
        const DT Di = get_di<T, DT, PT>(s, l);
        const SV<T> pa = pA + (T)((DT)u * Di) * tp_sv(s, l, T_U);
        caddv(cv, par, C_TP, applyT(tp_xf(s, l, T_E), pa));
      }
    } else {
      cputv(cv, l, C_TU, zeroSV<T>() - pA);
    }
  }
  for (int l = 0; l < nl; ++l) {
    const int m = s.M(l);
    const int par = meta_parent(m);
    SV<T> a;
    if (meta_jtype(m) == J_REVOLUTE) {
      const V3<T> ax = s.pv3(l, P_AX);
      const SV<T> ap = par >= 0 ? apply(tp_xf(s, l, T_E), cgetv(cv, par, C_TA)) : zeroSV<T>();
      const DT Di = get_di<T, DT, PT>(s, l);
      const T qdd = (T)(((DT)cv.L(l, C_TU) - (DT)dot(tp_sv(s, l, T_U), ap)) * Di);
      a = ap;
      a.w += qdd * ax;
      if (qf >= 0) cv.L(l, qf) = qdd;
    } else {  // free root: a = (I^A)^-1 u, qdd = a (its parent acceleration is 0)
      a = spd_solve<T, DT>(tp_si(s, l, T_IA), cgetv(cv, l, C_TU));
      if (qf >= 0) cputv(cv, l, qf, a);
    }
    cputv(cv, l, C_TA, a);
  }
}

// Reverse of test_pass (which must have just run with the same inputs): the
// caller has put the adjoints of the link accelerations in C_TAB; field qbf
// (scaled by qbs; qbf < 0: none) holds the adjoint of the joint accelerations.
// Adds the adjoints of U, 1/D, X and the root articulated inertia to B_U, B_DI,
// B_E / B_R and B_IA, returns the adjoint of each applied force in fvb and
// leaves the adjoint of each revolute joint's force (that of a joint impulse on
// it) in C_TUB.
template <class T, class DT, class PT>
CD void test_pass_reverse(Sys<T, PT> s, CView<T> cv, int qbf, T qbs, const int* fl, int nf, SV<T>* fvb) {
  const int nl = s.nl;
  for (int l = nl - 1; l >= 0; --l) {  // acceleration pass, leaves -> root
    const int m = s.M(l);
    const int par = meta_parent(m);
    const XF<T> X = tp_xf(s, l, T_E);
    const SV<T> ab = cgetv(cv, l, C_TAB);
    const SV<T> apar = par >= 0 ? cgetv(cv, par, C_TA) : zeroSV<T>();
    SV<T> apb;
    if (meta_jtype(m) == J_REVOLUTE) {
      const V3<T> ax = s.pv3(l, P_AX);
      const SV<T> U = tp_sv(s, l, T_U);
      const DT Di = get_di<T, DT, PT>(s, l);
      const T u = cv.L(l, C_TU);
      const SV<T> ap = par >= 0 ? apply(X, apar) : zeroSV<T>();
      T qb = dot(ax, ab.w);
      if (qbf >= 0) qb += qbs * cv.L(l, qbf);
      const T w = (T)((DT)qb * Di);  // qdd = (u - U.ap) / D
      cv.L(l, C_TUB) = w;
      caddv(cv, l, B_U, zeroSV<T>() - w * ap);
      cv.L(l, B_DI) += (T)((DT)qb * ((DT)u - (DT)dot(U, ap)));
      apb = ab - w * U;
    } else {
      SV<T> qb = zeroSV<T>();
      if (qbf >= 0) qb = qbs * cgetv(cv, l, qbf);
      const SV<T> a = cgetv(cv, l, C_TA);
      const SV<T> ub = spd_solve<T, DT>(tp_si(s, l, T_IA), ab + qb);
      cputv(cv, l, C_TUB, ub);
      caddsi(cv, l, B_IA, scale(T(-1), sym_outer(ub, a)));
      apb = zeroSV<T>() - qb;
    }
    if (par >= 0) {
      M3<T> Eb = zeroM3<T>();
      V3<T> rb = zero3<T>();
      SV<T> aparb = zeroSV<T>();
      apply_adj(X, apar, apb, Eb, rb, &aparb);
      caddm(cv, l, B_E, Eb);
      cadd3(cv, l, B_R, rb);
      caddv(cv, par, C_TAB, aparb);
    }
  }
  for (int l = 0; l < nl; ++l) {  // bias-force pass, root -> leaves
    const int m = s.M(l);
    const int par = meta_parent(m);
    SV<T> pAb = zeroSV<T>();
    if (meta_jtype(m) == J_REVOLUTE) {
      const V3<T> ax = s.pv3(l, P_AX);
      T ub = cv.L(l, C_TUB);
      if (par >= 0) {
        const XF<T> X = tp_xf(s, l, T_E);
        const SV<T> U = tp_sv(s, l, T_U);
        const DT Di = get_di<T, DT, PT>(s, l);
        const T u = cv.L(l, C_TU);
        const T uDi = (T)((DT)u * Di);
        const SV<T> pa = cgetv(cv, l, C_TP) + uDi * U;
        M3<T> Eb = zeroM3<T>();
        V3<T> rb = zero3<T>();
        SV<T> pab = zeroSV<T>();
        applyT_adj(X, pa, cgetv(cv, par, C_TPB), Eb, rb, &pab);
        caddm(cv, l, B_E, Eb);
        cadd3(cv, l, B_R, rb);
        pAb += pab;  // pa = pA + U (u / D)
        caddv(cv, l, B_U, uDi * pab);
        const T gb = dot(U, pab);
        ub += (T)((DT)gb * Di);
        cv.L(l, B_DI) += (T)((DT)gb * (DT)u);
      }
      pAb.w -= ub * ax;  // u = -a . pA_w (+ joint impulse)
      cv.L(l, C_TUB) = ub;
    } else {
      pAb = zeroSV<T>() - cgetv(cv, l, C_TUB);  // u = -pA
    }
    cputv(cv, l, C_TPB, pAb);
  }
  for (int i = 0; i < nf; ++i) fvb[i] = zeroSV<T>() - cgetv(cv, fl[i], C_TPB);  // pA = (children) - f
}

// ------------------------------------------------------------------ forward
// Gauss-Seidel row order within a sweep: row q of contact c (q = 0 normal, 1 x,
// 2 y) is impulse index 3c + 2, 3c, 3c + 1.
SD int contact_row(int c, int q) { return q == 0 ? 3 * c + 2 : 3 * c + q - 1; }

// One Gauss-Seidel update of row r: lambda_r <- project(lambda_r - (A_r . lambda + b_r) / A_rr),
// onto [lo, hi] (box) or [0, inf) (box false).
template <class T>
SD void gs_update(const CView<T>& cv, int r, int nr, bool box, T hi) {
  const T lr = cv.S(S_LF + r);
  T res = cv.S(S_B + r);
  for (int k = 0; k < nr; ++k) res += cv.S(S_A + r * NROW + k) * cv.S(S_LF + k);
  const T sv = lr - res / cv.S(S_A + r * NROW + r);
  T ln;
  if (!box) {
    ln = sv > T(0) ? sv : T(0);
  } else {
    ln = sv < hi ? sv : hi;
    ln = ln > -hi ? ln : -hi;
  }
  cv.S(S_LF + r) = ln;
}

// Contact and limit impulses of one step; requires aba_forward to have filled the
// tape (unconstrained qdd included).  Leaves the velocity change in C_DV of every
// link and returns the number of active rows (0: C_DV is not written and the step
// has no constraint term).
template <class T, class DT, class PT>
CD int contact_forward(Sys<T, PT> s, CView<T> cv, Col<const T> q, Col<const T> qd, T dt, ContactParams<T> cp) {
  const int nl = s.nl;
  world_poses(s, cv);
  int nc = 0;
  int link[MAXC];
  V3<T> pc[MAXC];
  for (int l = 0; l < nl && nc < MAXC; ++l) {
    const T r = s.P(l, P_CR);
    if (!(r >= T(0))) continue;
    const V3<T> p = s.pv3(l, P_CP);
    const V3<T> y = cget3(cv, l, C_OW) + mulT(cgetm(cv, l, C_EW), p);
    const T phi = y.z - r;
    if (phi < T(0)) {
      link[nc] = l;
      pc[nc] = p;
      cv.S(S_LINK + nc) = (T)l;
      cv.S(S_PHI + nc) = phi;
      ++nc;
    }
  }
  int nlr = 0;
  int llink[MAXL];
  T lsg[MAXL];
  for (int l = 0; l < nl && nlr < MAXL; ++l) {
    const int m = s.M(l);
    if (meta_jtype(m) != J_REVOLUTE) continue;
    const T ql = q[meta_qoff(m)];
    const T below = ql - s.P(l, P_LO), above = s.P(l, P_HI) - ql;
    T sg, phi;
    if (below < T(0)) {
      sg = T(1);
      phi = below;
    } else if (above < T(0)) {
      sg = T(-1);
      phi = above;
    } else {
      continue;
    }
    llink[nlr] = l;
    lsg[nlr] = sg;
    cv.S(S_LINK + MAXC + nlr) = (T)l;
    cv.S(S_PHI + MAXC + nlr) = phi;
    cv.S(S_SGN + nlr) = sg;
    ++nlr;
  }
  cv.S(S_NC) = (T)nc;
  cv.S(S_NL) = (T)nlr;
  const int nr = 3 * nc + nlr;
  if (nr == 0) return 0;
  // link velocities for v* = qd + dt qdd
  for (int l = 0; l < nl; ++l) {
    const int m = s.M(l);
    const int par = meta_parent(m), vo = meta_voff(m);
    SV<T> vJ;
    if (meta_jtype(m) == J_REVOLUTE) {
      vJ = SV<T>{(qd[vo] + dt * s.tp(l, T_QDD)) * s.pv3(l, P_AX), zero3<T>()};
    } else {
      T w[6];
      for (int i = 0; i < 6; ++i) w[i] = qd[vo + i] + dt * s.tp(l, T_QDD + i);
      vJ = SV<T>{{w[0], w[1], w[2]}, {w[3], w[4], w[5]}};
    }
    SV<T> V = vJ;
    if (par >= 0) V = apply(tp_xf(s, l, T_E), cgetv(cv, par, C_VS)) + vJ;
    cputv(cv, l, C_VS, V);
  }
  const T kphi = cp.erp / dt;
  for (int c = 0; c < nc; ++c) {
    const int l = link[c];
    const SV<T> V = cgetv(cv, l, C_VS);
    const V3<T> pv = mulT(cgetm(cv, l, C_EW), V.v + cross(V.w, pc[c]));
    cv.S(S_B + 3 * c) = pv.x;
    cv.S(S_B + 3 * c + 1) = pv.y;
    cv.S(S_B + 3 * c + 2) = pv.z + kphi * cv.S(S_PHI + c);
  }
  for (int k = 0; k < nlr; ++k) {
    const int l = llink[k];
    const T vstar = qd[meta_voff(s.M(l))] + dt * s.tp(l, T_QDD);
    cv.S(S_B + 3 * nc + k) = lsg[k] * vstar + kphi * cv.S(S_PHI + MAXC + k);
  }
  // A, one column per active row
  for (int j = 0; j < nr; ++j) {
    if (j < 3 * nc) {
      const int c = j / 3, k = j % 3;
      const M3<T> Ew = cgetm(cv, link[c], C_EW);
      const V3<T> f{Ew.a[k], Ew.a[3 + k], Ew.a[6 + k]};  // E_w e_k
      const SV<T> fv{cross(pc[c], f), f};
      test_pass<T, DT, PT>(s, cv, &link[c], &fv, 1, nullptr, nullptr, 0, C_TQ);
    } else {
      const int k = j - 3 * nc;
      test_pass<T, DT, PT>(s, cv, nullptr, nullptr, 0, &llink[k], &lsg[k], 1, C_TQ);
    }
    for (int c2 = 0; c2 < nc; ++c2) {
      const SV<T> a = cgetv(cv, link[c2], C_TA);
      const V3<T> pa = mulT(cgetm(cv, link[c2], C_EW), a.v + cross(a.w, pc[c2]));
      cv.S(S_A + (3 * c2) * NROW + j) = pa.x;
      cv.S(S_A + (3 * c2 + 1) * NROW + j) = pa.y;
      cv.S(S_A + (3 * c2 + 2) * NROW + j) = pa.z;
    }
    for (int k2 = 0; k2 < nlr; ++k2) cv.S(S_A + (3 * nc + k2) * NROW + j) = lsg[k2] * cv.L(llink[k2], C_TQ);
  }
  // projected Gauss-Seidel
  for (int r = 0; r < nr; ++r) cv.S(S_LF + r) = T(0);
  for (int it = 0; it < cp.iters; ++it) {
    for (int c = 0; c < nc; ++c) {
      for (int qq = 0; qq < 3; ++qq) {
        const int r = contact_row(c, qq);
        cv.S(S_LAM + it * NROW + r) = cv.S(S_LF + r);
        gs_update(cv, r, nr, qq != 0, cp.mu * cv.S(S_LF + 3 * c + 2));
      }
    }
    for (int k = 0; k < nlr; ++k) {
      const int r = 3 * nc + k;
      cv.S(S_LAM + it * NROW + r) = cv.S(S_LF + r);
      gs_update(cv, r, nr, false, T(0));
    }
  }
  // velocity change M^-1 J^T lambda
  SV<T> fv[MAXC];
  for (int c = 0; c < nc; ++c) {
    const V3<T> lam{cv.S(S_LF + 3 * c), cv.S(S_LF + 3 * c + 1), cv.S(S_LF + 3 * c + 2)};
    const V3<T> f = mul(cgetm(cv, link[c], C_EW), lam);
    fv[c] = SV<T>{cross(pc[c], f), f};
  }
  T jv[MAXL];
  for (int k = 0; k < nlr; ++k) jv[k] = lsg[k] * cv.S(S_LF + 3 * nc + k);
  test_pass<T, DT, PT>(s, cv, link, fv, nc, llink, jv, nlr, C_DV);
  return nr;
}

// ------------------------------------------------------------------ adjoint
// Reverse of one Gauss-Seidel update of row r (the vector in S_LF is the one
// after it; the overwritten value comes from the tape): moves the adjoint of the
// new lambda_r in S_LB onto lambda (S_LB), A (S_AB) and b (S_BB).  For a box row
// the bound's adjoint goes to the normal impulse of contact c.
template <class T>
SD void gs_update_reverse(const CView<T>& cv, int it, int r, int nr, bool box, int rn, T mu) {
  const T lnb = cv.S(S_LB + r);
  const T lr = cv.S(S_LAM + it * NROW + r);
  cv.S(S_LF + r) = lr;  // the vector as the update saw it
  cv.S(S_LB + r) = T(0);
  const T Arr = cv.S(S_A + r * NROW + r);
  T res = cv.S(S_B + r);
  for (int k = 0; k < nr; ++k) res += cv.S(S_A + r * NROW + k) * cv.S(S_LF + k);
  const T sv = lr - res / Arr;
  T sb = T(0);
  if (!box) {
    if (sv >= T(0)) sb = lnb;
  } else {
    const T hi = mu * cv.S(S_LF + rn);
    T hb = T(0);
    if (sv > hi) hb = lnb;
    else if (sv < -hi) hb = -lnb;
    else sb = lnb;
    cv.S(S_LB + rn) += mu * hb;
  }
  if (sb != T(0)) {  // sv = lambda_r - (A_r . lambda + b_r) / A_rr
    cv.S(S_LB + r) += sb;
    const T g = sb / Arr;
    for (int k = 0; k < nr; ++k) {
      cv.S(S_LB + k) -= g * cv.S(S_A + r * NROW + k);
      cv.S(S_AB + r * NROW + k) -= g * cv.S(S_LF + k);
    }
    cv.S(S_BB + r) -= g;
    cv.S(S_AB + r * NROW + r) += g * res / Arr;
  }
}

// Requires aba_forward and contact_forward (with active rows) of the same step,
// and the adjoint of the unconstrained-plus-constraint qdd from the integrator
// adjoint in C_QDDB (dt times the adjoint of qd').  Fills the B_* fields.
template <class T, class DT, class PT>
CD void contact_adjoint(Sys<T, PT> s, CView<T> cv, T dt, ContactParams<T> cp) {
  const int nl = s.nl;
  const int nc = (int)cv.S(S_NC);
  const int nlr = (int)cv.S(S_NL);
  const int nr = 3 * nc + nlr;
  for (int l = 0; l < nl; ++l)
    for (int f = B_U; f < B_END; ++f) cv.L(l, f) = T(0);
  int link[MAXC];
  V3<T> pc[MAXC];
  for (int c = 0; c < nc; ++c) {
    link[c] = (int)cv.S(S_LINK + c);
    pc[c] = s.pv3(link[c], P_CP);
  }
  int llink[MAXL];
  T lsg[MAXL];
  for (int k = 0; k < nlr; ++k) {
    llink[k] = (int)cv.S(S_LINK + MAXC + k);
    lsg[k] = cv.S(S_SGN + k);
  }
  // 1. the velocity change dv = M^-1 J^T lambda; dv enters qd' directly
  {
    SV<T> fv[MAXC], fvb[MAXC];
    V3<T> lam[MAXC];
    T jv[MAXL];
    for (int c = 0; c < nc; ++c) {
      lam[c] = V3<T>{cv.S(S_LF + 3 * c), cv.S(S_LF + 3 * c + 1), cv.S(S_LF + 3 * c + 2)};
      const V3<T> f = mul(cgetm(cv, link[c], C_EW), lam[c]);
      fv[c] = SV<T>{cross(pc[c], f), f};
    }
    for (int k = 0; k < nlr; ++k) jv[k] = lsg[k] * cv.S(S_LF + 3 * nc + k);
    test_pass<T, DT, PT>(s, cv, link, fv, nc, llink, jv, nlr, -1);
    for (int l = 0; l < nl; ++l) cputv(cv, l, C_TAB, zeroSV<T>());
    test_pass_reverse<T, DT, PT>(s, cv, C_QDDB, T(1) / dt, link, nc, fvb);
    for (int c = 0; c < nc; ++c) {
      const V3<T> flb = fvb[c].v + cross(fvb[c].w, pc[c]);  // f = E_w lambda, n = p x f
      const V3<T> lb = mulT(cgetm(cv, link[c], C_EW), flb);
      cv.S(S_LB + 3 * c) = lb.x;
      cv.S(S_LB + 3 * c + 1) = lb.y;
      cv.S(S_LB + 3 * c + 2) = lb.z;
      caddm(cv, link[c], B_EW, outer(flb, lam[c]));
    }
    for (int k = 0; k < nlr; ++k) cv.S(S_LB + 3 * nc + k) = lsg[k] * cv.L(llink[k], C_TUB);
  }
  // 2. the Gauss-Seidel sweeps, last update first
  for (int r = 0; r < nr; ++r) {
    cv.S(S_BB + r) = T(0);
    for (int k = 0; k < nr; ++k) cv.S(S_AB + r * NROW + k) = T(0);
  }
  for (int it = cp.iters - 1; it >= 0; --it) {
    for (int k = nlr - 1; k >= 0; --k) gs_update_reverse(cv, it, 3 * nc + k, nr, false, 0, cp.mu);
    for (int c = nc - 1; c >= 0; --c)
      for (int qq = 2; qq >= 0; --qq) gs_update_reverse(cv, it, contact_row(c, qq), nr, qq != 0, 3 * c + 2, cp.mu);
  }
  // 3. the columns of A
  for (int j = 0; j < nr; ++j) {
    const bool is_contact = j < 3 * nc;
    const int c = j / 3, k = j % 3;
    SV<T> fv;
    if (is_contact) {
      const M3<T> Ew = cgetm(cv, link[c], C_EW);
      const V3<T> f{Ew.a[k], Ew.a[3 + k], Ew.a[6 + k]};
      fv = SV<T>{cross(pc[c], f), f};
      test_pass<T, DT, PT>(s, cv, &link[c], &fv, 1, nullptr, nullptr, 0, -1);
    } else {
      test_pass<T, DT, PT>(s, cv, nullptr, nullptr, 0, &llink[j - 3 * nc], &lsg[j - 3 * nc], 1, -1);
    }
    for (int l = 0; l < nl; ++l) {
      cputv(cv, l, C_TAB, zeroSV<T>());
      cputv(cv, l, C_TQB, zeroSV<T>());
    }
    for (int c2 = 0; c2 < nc; ++c2) {  // A_{., j} = E_w^T (a_v + a_w x p)
      const int l2 = link[c2];
      const V3<T> yb{cv.S(S_AB + (3 * c2) * NROW + j), cv.S(S_AB + (3 * c2 + 1) * NROW + j),
                     cv.S(S_AB + (3 * c2 + 2) * NROW + j)};
      const SV<T> a = cgetv(cv, l2, C_TA);
      const V3<T> z = a.v + cross(a.w, pc[c2]);
      caddm(cv, l2, B_EW, outer(z, yb));
      const V3<T> zb = mul(cgetm(cv, l2, C_EW), yb);
      caddv(cv, l2, C_TAB, SV<T>{cross(pc[c2], zb), zb});
    }
    for (int k2 = 0; k2 < nlr; ++k2)  // A_{limit k2, j} = s qdd_j
      cv.L(llink[k2], C_TQB) += lsg[k2] * cv.S(S_AB + (3 * nc + k2) * NROW + j);
    SV<T> fvb;
    test_pass_reverse<T, DT, PT>(s, cv, C_TQB, T(1), is_contact ? &link[c] : link, is_contact ? 1 : 0, &fvb);
    if (is_contact) {
      const V3<T> flb = fvb.v + cross(fvb.w, pc[c]);  // f = E_w e_k
      V3<T> ek = zero3<T>();
      if (k == 0) ek.x = T(1);
      else if (k == 1) ek.y = T(1);
      else ek.z = T(1);
      caddm(cv, link[c], B_EW, outer(flb, ek));
    }
  }
  // 4. b = E_w^T (V*_v + V*_w x p) + (erp / dt) phi e_z on contacts, s v*_j + (erp / dt) phi on limits
  for (int l = 0; l < nl; ++l) cputv(cv, l, B_VS, zeroSV<T>());
  const T kphi = cp.erp / dt;
  for (int c = 0; c < nc; ++c) {
    const int l = link[c];
    const V3<T> bb{cv.S(S_BB + 3 * c), cv.S(S_BB + 3 * c + 1), cv.S(S_BB + 3 * c + 2)};
    const SV<T> V = cgetv(cv, l, C_VS);
    const V3<T> z = V.v + cross(V.w, pc[c]);
    caddm(cv, l, B_EW, outer(z, bb));
    const V3<T> zb = mul(cgetm(cv, l, C_EW), bb);
    caddv(cv, l, B_VS, SV<T>{cross(pc[c], zb), zb});
    // phi = (o + E_w^T p)_z - r
    const V3<T> yb{T(0), T(0), kphi * bb.z};
    cadd3(cv, l, B_OW, yb);
    caddm(cv, l, B_EW, outer(pc[c], yb));
  }
  for (int k = 0; k < nlr; ++k) {  // phi = s (q - limit), v* = qd + dt qdd
    const int l = llink[k];
    const T bb = cv.S(S_BB + 3 * nc + k);
    const T vb = lsg[k] * bb;
    cv.L(l, B_QD) += vb;
    cv.L(l, B_QDD) += dt * vb;
    cv.L(l, B_Q) += lsg[k] * (kphi * bb);
  }
  // 5. the link velocities of v* = qd + dt qdd, leaves -> root
  for (int l = nl - 1; l >= 0; --l) {
    const int m = s.M(l);
    const int par = meta_parent(m);
    const SV<T> Vb = cgetv(cv, l, B_VS);
    if (meta_jtype(m) == J_REVOLUTE) {
      const T vb = dot(s.pv3(l, P_AX), Vb.w);
      cv.L(l, B_QD) += vb;
      cv.L(l, B_QDD) += dt * vb;
    } else {
      const T vb[6] = {Vb.w.x, Vb.w.y, Vb.w.z, Vb.v.x, Vb.v.y, Vb.v.z};
      for (int i = 0; i < 6; ++i) {
        cv.L(l, B_QD + i) += vb[i];
        cv.L(l, B_QDD + i) += dt * vb[i];
      }
    }
    if (par >= 0) {
      M3<T> Eb = zeroM3<T>();
      V3<T> rb = zero3<T>();
      SV<T> Vpb = zeroSV<T>();
      apply_adj(tp_xf(s, l, T_E), cgetv(cv, par, C_VS), Vb, Eb, rb, &Vpb);
      caddm(cv, l, B_E, Eb);
      cadd3(cv, l, B_R, rb);
      caddv(cv, par, B_VS, Vpb);
    }
  }
  // 6. world kinematics, leaves -> root
  for (int l = nl - 1; l >= 0; --l) {
    const int par = meta_parent(s.M(l));
    const M3<T> Ewb = cgetm(cv, l, B_EW);
    const V3<T> ob = cget3(cv, l, B_OW);
    const XF<T> X = tp_xf(s, l, T_E);
    if (par < 0) {
      caddm(cv, l, B_E, Ewb);
      cadd3(cv, l, B_R, ob);
    } else {
      const M3<T> Ep = cgetm(cv, par, C_EW);
      caddm(cv, l, B_E, mmT(Ewb, Ep));                         // E_w = E E_w(parent)
      cadd3(cv, l, B_R, mul(Ep, ob));                          // o = o(parent) + E_w(parent)^T r
      caddm(cv, par, B_EW, mTm(X.E, Ewb) + outer(X.r, ob));
      cadd3(cv, par, B_OW, ob);
    }
  }
}

}  // namespace abasim

#undef CD
