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
// Inputs of a test pass: n entries, each a spatial force (link coordinates, at
// the link origin) on a link or an impulse on a revolute joint (f.w.x), for one
// of the pass's right-hand sides.
constexpr int MAXIN = MAXC + MAXL;
template <class T> struct TPIn {
  int n = 0;
  int link[MAXIN];
  int rhs[MAXIN];
  bool joint[MAXIN];
  SV<T> f[MAXIN];
  SD void force(int l, int r, SV<T> v) { link[n] = l; rhs[n] = r; joint[n] = false; f[n++] = v; }
  SD void impulse(int l, int r, T v) {
    link[n] = l; rhs[n] = r; joint[n] = true;
    f[n++] = SV<T>{{v, T(0), T(0)}, zero3<T>()};
  }
};

// Free-root solves of several right-hand sides sharing one Cholesky factor (the
// same operations as spd_solve).
template <class T, class DT, int NR>
SD void spd_solve_n(const SI<T>& IA, const SV<T>* b, SV<T>* x) {
  DT L[21];
  chol6(si_cast<DT>(IA), L);
  for (int r = 0; r < NR; ++r) {
    const SV<DT> y = chol6_solve(L, sv_cast<DT>(b[r]));
    x[r] = SV<T>{{(T)y.w.x, (T)y.w.y, (T)y.w.z}, {(T)y.v.x, (T)y.v.y, (T)y.v.z}};
  }
}

// Response of the articulated system at rest (no velocity or gravity) to the
// inputs, for NR right-hand sides at once: the ABA's bias-force pass and
// acceleration pass with the step's U, 1/D, X and root articulated inertia.
// Leaves, per right-hand side r (fields + 6 r), the articulated bias forces
// (C_TP), joint forces (C_TU) and link accelerations (C_TA) on the contact tape,
// and the joint accelerations M^-1 (sum J_i^T f_i + sum e_j impulse) in field
// qf + 6 r (if qf >= 0).
template <class T, class DT, class PT, int NR>
CD void test_pass(Sys<T, PT> s, CView<T> cv, TPIn<T> in, int qf) {
  const int nl = s.nl;
  for (int l = 0; l < nl; ++l)
    for (int r = 0; r < NR; ++r) cputv(cv, l, C_TP + 6 * r, zeroSV<T>());
  for (int l = nl - 1; l >= 0; --l) {
    const int m = s.M(l);
    const int par = meta_parent(m);
    SV<T> pA[NR];
    T jadd[NR];
    for (int r = 0; r < NR; ++r) {
      pA[r] = cgetv(cv, l, C_TP + 6 * r);
      jadd[r] = T(0);
    }
    for (int i = 0; i < in.n; ++i)
      if (in.link[i] == l) {
        for (int r = 0; r < NR; ++r)
          if (in.rhs[i] == r) {
            if (in.joint[i]) jadd[r] += in.f[i].w.x;
            else pA[r] -= in.f[i];
          }
      }
    for (int r = 0; r < NR; ++r) cputv(cv, l, C_TP + 6 * r, pA[r]);
    if (meta_jtype(m) == J_REVOLUTE) {
      const V3<T> ax = zaxis<T>();
      T u[NR];
      for (int r = 0; r < NR; ++r) {
        u[r] = -dot(ax, pA[r].w) + jadd[r];
        cv.L(l, C_TU + 6 * r) = u[r];
      }
      if (par >= 0) {
        const DT Di = get_di<T, DT, PT>(s, l);
        const SV<T> U = tp_sv(s, l, T_U);
        const XF<T> X = tp_xf(s, l, T_E);
        for (int r = 0; r < NR; ++r) {
          const SV<T> pa = pA[r] + (T)((DT)u[r] * Di) * U;
          caddv(cv, par, C_TP + 6 * r, applyT(X, pa));
        }
      }
    } else {
      for (int r = 0; r < NR; ++r) cputv(cv, l, C_TU + 6 * r, zeroSV<T>() - pA[r]);
    }
  }
  for (int l = 0; l < nl; ++l) {
    const int m = s.M(l);
    const int par = meta_parent(m);
    const XF<T> X = tp_xf(s, l, T_E);
    if (meta_jtype(m) == J_REVOLUTE) {
      const V3<T> ax = zaxis<T>();
      const DT Di = get_di<T, DT, PT>(s, l);
      const SV<T> U = tp_sv(s, l, T_U);
      for (int r = 0; r < NR; ++r) {
        const SV<T> ap = par >= 0 ? apply(X, cgetv(cv, par, C_TA + 6 * r)) : zeroSV<T>();
        const T qdd = (T)(((DT)cv.L(l, C_TU + 6 * r) - (DT)dot(U, ap)) * Di);
        SV<T> a = ap;
        a.w += qdd * ax;
        if (qf >= 0) cv.L(l, qf + 6 * r) = qdd;
        cputv(cv, l, C_TA + 6 * r, a);
      }
    } else {  // free root: a = (I^A)^-1 u, qdd = a (its parent acceleration is 0)
      SV<T> u[NR], a[NR];
      for (int r = 0; r < NR; ++r) u[r] = cgetv(cv, l, C_TU + 6 * r);
      spd_solve_n<T, DT, NR>(tp_si(s, l, T_IA), u, a);
      for (int r = 0; r < NR; ++r) {
        if (qf >= 0) cputv(cv, l, qf + 6 * r, a[r]);
        cputv(cv, l, C_TA + 6 * r, a[r]);
      }
    }
  }
}

// Reverse of test_pass (which must have just run with the same inputs): the
// caller has put the adjoints of the link accelerations in C_TAB + 6 r; field
// qbf + 6 r (scaled by qbs; qbf < 0: none) holds the adjoint of the joint
// accelerations.  Adds the adjoints of U, 1/D, X and the root articulated
// inertia to B_U, B_DI, B_E / B_R and B_IA and returns the adjoint of each input
// in fvb (a force's spatial adjoint; a joint impulse's adjoint in w.x).
template <class T, class DT, class PT, int NR>
CD void test_pass_reverse(Sys<T, PT> s, CView<T> cv, int qbf, T qbs, TPIn<T> in, SV<T>* fvb) {
  const int nl = s.nl;
  for (int l = nl - 1; l >= 0; --l) {  // acceleration pass, leaves -> root
    const int m = s.M(l);
    const int par = meta_parent(m);
    const XF<T> X = tp_xf(s, l, T_E);
    SV<T> apb[NR], apar[NR];
    for (int r = 0; r < NR; ++r) apar[r] = par >= 0 ? cgetv(cv, par, C_TA + 6 * r) : zeroSV<T>();
    if (meta_jtype(m) == J_REVOLUTE) {
      const V3<T> ax = zaxis<T>();
      const SV<T> U = tp_sv(s, l, T_U);
      const DT Di = get_di<T, DT, PT>(s, l);
      SV<T> Ub = zeroSV<T>();
      T Dib = T(0);
      for (int r = 0; r < NR; ++r) {
        const SV<T> ab = cgetv(cv, l, C_TAB + 6 * r);
        const T u = cv.L(l, C_TU + 6 * r);
        const SV<T> ap = par >= 0 ? apply(X, apar[r]) : zeroSV<T>();
        T qb = dot(ax, ab.w);
        if (qbf >= 0) qb += qbs * cv.L(l, qbf + 6 * r);
        const T w = (T)((DT)qb * Di);  // qdd = (u - U.ap) / D
        cv.L(l, C_TUB + 6 * r) = w;
        Ub -= w * ap;
        Dib += (T)((DT)qb * ((DT)u - (DT)dot(U, ap)));
        apb[r] = ab - w * U;
      }
      caddv(cv, l, B_U, Ub);
      cv.L(l, B_DI) += Dib;
    } else {
      SV<T> rhs[NR], ub[NR];
      for (int r = 0; r < NR; ++r) {
        SV<T> qb = zeroSV<T>();
        if (qbf >= 0) qb = qbs * cgetv(cv, l, qbf + 6 * r);
        rhs[r] = cgetv(cv, l, C_TAB + 6 * r) + qb;
        apb[r] = zeroSV<T>() - qb;
      }
      spd_solve_n<T, DT, NR>(tp_si(s, l, T_IA), rhs, ub);
      for (int r = 0; r < NR; ++r) {
        cputv(cv, l, C_TUB + 6 * r, ub[r]);
        caddsi(cv, l, B_IA, scale(T(-1), sym_outer(ub[r], cgetv(cv, l, C_TA + 6 * r))));
      }
    }
    if (par >= 0) {
      M3<T> Eb = zeroM3<T>();
      V3<T> rb = zero3<T>();
      for (int r = 0; r < NR; ++r) {
        SV<T> aparb = zeroSV<T>();
        apply_adj(X, apar[r], apb[r], Eb, rb, &aparb);
        caddv(cv, par, C_TAB + 6 * r, aparb);
      }
      caddm(cv, l, B_E, Eb);
      cadd3(cv, l, B_R, rb);
    }
  }
  for (int l = 0; l < nl; ++l) {  // bias-force pass, root -> leaves
    const int m = s.M(l);
    const int par = meta_parent(m);
    if (meta_jtype(m) == J_REVOLUTE) {
      const V3<T> ax = zaxis<T>();
      if (par >= 0) {
        const XF<T> X = tp_xf(s, l, T_E);
        const SV<T> U = tp_sv(s, l, T_U);
        const DT Di = get_di<T, DT, PT>(s, l);
        M3<T> Eb = zeroM3<T>();
        V3<T> rb = zero3<T>();
        SV<T> Ub = zeroSV<T>();
        T Dib = T(0);
        for (int r = 0; r < NR; ++r) {
          T ub = cv.L(l, C_TUB + 6 * r);
          const T u = cv.L(l, C_TU + 6 * r);
          const T uDi = (T)((DT)u * Di);
          const SV<T> pa = cgetv(cv, l, C_TP + 6 * r) + uDi * U;
          SV<T> pab = zeroSV<T>();
          applyT_adj(X, pa, cgetv(cv, par, C_TPB + 6 * r), Eb, rb, &pab);
          SV<T> pAb = pab;  // pa = pA + U (u / D)
          Ub += uDi * pab;
          const T gb = dot(U, pab);
          ub += (T)((DT)gb * Di);
          Dib += (T)((DT)gb * (DT)u);
          pAb.w -= ub * ax;  // u = -a . pA_w (+ joint impulse)
          cv.L(l, C_TUB + 6 * r) = ub;
          cputv(cv, l, C_TPB + 6 * r, pAb);
        }
        caddm(cv, l, B_E, Eb);
        cadd3(cv, l, B_R, rb);
        caddv(cv, l, B_U, Ub);
        cv.L(l, B_DI) += Dib;
      } else {
        for (int r = 0; r < NR; ++r) {
          const T ub = cv.L(l, C_TUB + 6 * r);
          SV<T> pAb = zeroSV<T>();
          pAb.w -= ub * ax;
          cputv(cv, l, C_TPB + 6 * r, pAb);
        }
      }
    } else {
      for (int r = 0; r < NR; ++r) cputv(cv, l, C_TPB + 6 * r, zeroSV<T>() - cgetv(cv, l, C_TUB + 6 * r));  // u = -pA
    }
  }
  for (int i = 0; i < in.n; ++i) {
    const int l = in.link[i], r = in.rhs[i];
    if (in.joint[i]) fvb[i] = SV<T>{{cv.L(l, C_TUB + 6 * r), T(0), T(0)}, zero3<T>()};
    else fvb[i] = zeroSV<T>() - cgetv(cv, l, C_TPB + 6 * r);  // pA = (children) - f
  }
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

// Test-pass inputs of rows j0, j0 + 1, j0 + 2 (one right-hand side each): the unit
// world force E_w e_k at a contact point (rows 3c + k) or the unit impulse s on a
// limited joint (rows 3 nc + k).
template <class T>
SD TPIn<T> unit_inputs(const CView<T>& cv, int nc, int nr, int j0, const int* link, const V3<T>* pc,
                       const int* llink, const T* lsg) {
  TPIn<T> in;
  for (int r = 0; r < 3 && j0 + r < nr; ++r) {
    const int j = j0 + r;
    if (j < 3 * nc) {
      const int c = j / 3, k = j % 3;
      const M3<T> Ew = cgetm(cv, link[c], C_EW);
      const V3<T> f{Ew.a[k], Ew.a[3 + k], Ew.a[6 + k]};
      in.force(link[c], r, SV<T>{cross(pc[c], f), f});
    } else {
      in.impulse(llink[j - 3 * nc], r, lsg[j - 3 * nc]);
    }
  }
  return in;
}

// Test-pass inputs of the impulses lambda (one right-hand side): f = E_w lambda_c
// at each contact point, s lambda on each limited joint.
template <class T>
SD TPIn<T> impulse_inputs(const CView<T>& cv, int nc, int nlr, const int* link, const V3<T>* pc,
                          const int* llink, const T* lsg) {
  TPIn<T> in;
  for (int c = 0; c < nc; ++c) {
    const V3<T> lam{cv.S(S_LF + 3 * c), cv.S(S_LF + 3 * c + 1), cv.S(S_LF + 3 * c + 2)};
    const V3<T> f = mul(cgetm(cv, link[c], C_EW), lam);
    in.force(link[c], 0, SV<T>{cross(pc[c], f), f});
  }
  for (int k = 0; k < nlr; ++k) in.impulse(llink[k], 0, lsg[k] * cv.S(S_LF + 3 * nc + k));
  return in;
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
      vJ = SV<T>{(qd[vo] + dt * s.tp(l, T_QDD)) * zaxis<T>(), zero3<T>()};
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
  // A, three columns (right-hand sides) per test pass
  for (int j0 = 0; j0 < nr; j0 += 3) {
    const TPIn<T> in = unit_inputs(cv, nc, nr, j0, link, pc, llink, lsg);
    test_pass<T, DT, PT, 3>(s, cv, in, C_TQ);
    for (int r = 0; r < 3 && j0 + r < nr; ++r) {
      const int j = j0 + r;
      for (int c2 = 0; c2 < nc; ++c2) {
        const SV<T> a = cgetv(cv, link[c2], C_TA + 6 * r);
        const V3<T> pa = mulT(cgetm(cv, link[c2], C_EW), a.v + cross(a.w, pc[c2]));
        cv.S(S_A + (3 * c2) * NROW + j) = pa.x;
        cv.S(S_A + (3 * c2 + 1) * NROW + j) = pa.y;
        cv.S(S_A + (3 * c2 + 2) * NROW + j) = pa.z;
      }
      for (int k2 = 0; k2 < nlr; ++k2)
        cv.S(S_A + (3 * nc + k2) * NROW + j) = lsg[k2] * cv.L(llink[k2], C_TQ + 6 * r);
    }
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
  test_pass<T, DT, PT, 1>(s, cv, impulse_inputs(cv, nc, nlr, link, pc, llink, lsg), C_DV);
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
    const TPIn<T> in = impulse_inputs(cv, nc, nlr, link, pc, llink, lsg);
    SV<T> fvb[MAXIN];
    test_pass<T, DT, PT, 1>(s, cv, in, -1);
    for (int l = 0; l < nl; ++l) cputv(cv, l, C_TAB, zeroSV<T>());
    test_pass_reverse<T, DT, PT, 1>(s, cv, C_QDDB, T(1) / dt, in, fvb);
    for (int c = 0; c < nc; ++c) {  // entries 0 .. nc - 1 are the contact forces
      const V3<T> lam{cv.S(S_LF + 3 * c), cv.S(S_LF + 3 * c + 1), cv.S(S_LF + 3 * c + 2)};
      const V3<T> flb = fvb[c].v + cross(fvb[c].w, pc[c]);  // f = E_w lambda, n = p x f
      const V3<T> lb = mulT(cgetm(cv, link[c], C_EW), flb);
      cv.S(S_LB + 3 * c) = lb.x;
      cv.S(S_LB + 3 * c + 1) = lb.y;
      cv.S(S_LB + 3 * c + 2) = lb.z;
      caddm(cv, link[c], B_EW, outer(flb, lam));
    }
    for (int k = 0; k < nlr; ++k) cv.S(S_LB + 3 * nc + k) = lsg[k] * fvb[nc + k].w.x;  // then the impulses
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
  // 3. the columns of A, three per test pass
  for (int j0 = 0; j0 < nr; j0 += 3) {
    const TPIn<T> in = unit_inputs(cv, nc, nr, j0, link, pc, llink, lsg);
    test_pass<T, DT, PT, 3>(s, cv, in, -1);
    for (int l = 0; l < nl; ++l)
      for (int r = 0; r < 3; ++r) {
        cputv(cv, l, C_TAB + 6 * r, zeroSV<T>());
        cputv(cv, l, C_TQB + 6 * r, zeroSV<T>());
      }
    for (int r = 0; r < 3 && j0 + r < nr; ++r) {
      const int j = j0 + r;
      for (int c2 = 0; c2 < nc; ++c2) {  // A_{., j} = E_w^T (a_v + a_w x p)
        const int l2 = link[c2];
        const V3<T> yb{cv.S(S_AB + (3 * c2) * NROW + j), cv.S(S_AB + (3 * c2 + 1) * NROW + j),
                       cv.S(S_AB + (3 * c2 + 2) * NROW + j)};
        const SV<T> a = cgetv(cv, l2, C_TA + 6 * r);
        const V3<T> z = a.v + cross(a.w, pc[c2]);
        caddm(cv, l2, B_EW, outer(z, yb));
        const V3<T> zb = mul(cgetm(cv, l2, C_EW), yb);
        caddv(cv, l2, C_TAB + 6 * r, SV<T>{cross(pc[c2], zb), zb});
      }
      for (int k2 = 0; k2 < nlr; ++k2)  // A_{limit k2, j} = s qdd_j
        cv.L(llink[k2], C_TQB + 6 * r) += lsg[k2] * cv.S(S_AB + (3 * nc + k2) * NROW + j);
    }
    SV<T> fvb[MAXIN];
    test_pass_reverse<T, DT, PT, 3>(s, cv, C_TQB, T(1), in, fvb);
    for (int i = 0; i < in.n; ++i) {
      const int j = j0 + in.rhs[i];
      if (in.joint[i] || j >= 3 * nc) continue;  // a unit impulse is a constant
      const int c = j / 3, k = j % 3;
      const V3<T> flb = fvb[i].v + cross(fvb[i].w, pc[c]);  // f = E_w e_k
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
      const T vb = dot(zaxis<T>(), Vb.w);
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
