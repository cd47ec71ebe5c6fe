// One simulation step of one articulated system and its reverse-mode adjoint.
//
// Forward (Sec. 3.1, Fig. 1): joint transforms, then the Articulated Body
// Algorithm's three tree passes (root->leaves kinematics/velocities, leaves->root
// articulated inertias and bias forces, root->leaves accelerations), then time
// integration.  Adjoint: the same modules in reverse order (Sec. 3.1), each
// spatial operator replaced by its adjoint (Eq. 6 and the supplement's rules,
// re-derived in the standard dPhi/dE convention).  The adjoint step is run after
// a recompute of the forward intermediates from the step's initial state
// (Sec. 3.2, Eq. 7): the per-link intermediates Z^k live in a per-step tape that
// is overwritten every step, never kept across steps.
//
// Joint models: revolute about a unit axis a (S = [a; 0], E_J = R(a, q)^T) and a
// free root joint (q = world position p and unit quaternion (x, y, z, w),
// qd = body-frame spatial velocity, S = 1_6, E_J = R(quat)^T, r_J = p).
// Integrator: semi-implicit Euler (qd' = qd + dt qdd, q' = q + dt qd') or
// explicit Euler (q' = q + dt qd); the free joint integrates p' = p + dt R v and
// quat' = normalize(quat + dt/2 quat (x) (w, 0)).
#pragma once

#if defined(ABASIM_HOST_CHECKS)
#include <cstdlib>
#endif

#include "spatial.cuh"

namespace abasim {

enum JointType : int { J_REVOLUTE = 0, J_FREE = 1 };
enum Integrator : int { I_SEMI_IMPLICIT = 0, I_EXPLICIT = 1 };

// per-link model parameters, [link][field][system], in the frames sim_create
// chooses (a revolute link's z axis is its joint axis, so P_AX is e_z there and
// the kernels use S = [e_z; 0] without reading it); P_CP / P_CR: contact sphere
// centre (link frame) and radius (< 0: the link has none); P_LO / P_HI: revolute
// joint position limits (-inf / +inf: none)
enum : int {
  P_E = 0, P_R = 9, P_AX = 12, P_M = 15, P_C = 16, P_IC = 19, P_DAMP = 25, P_CP = 26, P_CR = 29, P_LO = 30,
  P_HI = 31, NPRM = 32
};
// per-link forward tape
enum : int {
  T_E = 0, T_R = 9, T_V = 12, T_C = 18, T_H = 24, T_IA = 30, T_PA = 51, T_U = 57, T_D = 63,
  T_DI = 64, T_u = 65, T_Ia = 71, T_pa = 92, T_AP = 98, T_A = 104, T_QDD = 110, T_SC = 116,
  T_DI2 = 118, NTAPE = 119
};
// per-link adjoint accumulators
enum : int {
  G_A = 0, G_C = 6, G_E = 12, G_R = 21, G_U = 24, G_D = 30, G_u = 31, G_IA = 37, G_PA = 58,
  G_V = 64, G_M = 70, NADJ = 71
};

// per-link contact tape (models with contact spheres or joint limits only),
// [link][field][system]: world pose of the link (C_EW rotation world -> link,
// C_OW origin), link velocities for the velocity after the unconstrained step
// (C_VS), the constraint velocity change per coordinate (C_DV), the adjoint of
// the unconstrained qdd from the integrator (C_QDDB), the adjoints the
// constraint solve hands to the step adjoint (B_*: U, 1/D, the free root's
// articulated inertia, the link transform E and r, world pose, unconstrained
// qdd, qd and, for limited joints, q), then a test pass's bias forces, link
// accelerations, joint forces, their adjoints and its joint accelerations and
// their adjoint, 6 words per right-hand side for up to 3 right-hand sides.
enum : int {
  C_EW = 0, C_OW = 9, C_VS = 12, C_DV = 18, C_QDDB = 24, B_U = 30, B_DI = 36, B_IA = 37, B_E = 58, B_R = 67,
  B_EW = 70, B_OW = 79, B_VS = 82, B_QDD = 88, B_QD = 94, B_Q = 100, B_END = 101, C_TP = 101, C_TA = 119,
  C_TU = 137, C_TAB = 155, C_TPB = 173, C_TUB = 191, C_TQ = 209, C_TQB = 227, NCT = 245
};

// meta word per link: parent+1 (8 bits) | joint type (1) | "has a child other than
// link l+1" (1) | q offset (10) | v offset (10) | "last of several children" (1).
// Chains never set the flags: their parent/child values are carried in registers
// from one loop iteration to the next.  Links are numbered in depth-first preorder
// (children in ascending order of the model's numbering), so a link with children
// has link l+1 as its first child, and the flags say when a world-aligned pass
// pushes or pops its stack of parent values: a link with a child other than l+1
// pushes (or, in the passes that run leaves -> root, pops) one entry, and the last
// child of such a link, which is never link parent+1, pops it (or pushes it).
SD int meta_parent(int m) { return (m & 0xff) - 1; }
SD int meta_jtype(int m) { return (m >> 8) & 0x1; }
SD bool meta_treechild(int m) { return (m >> 9) & 0x1; }
SD int meta_qoff(int m) { return (m >> 10) & 0x3ff; }
SD int meta_voff(int m) { return (m >> 20) & 0x3ff; }
SD bool meta_lastsib(int m) { return (m >> 30) & 0x1; }
SD int make_meta(int parent, int jt, bool treechild, int qo, int vo, bool lastsib = false) {
  return (parent + 1) | (jt << 8) | ((treechild ? 1 : 0) << 9) | (qo << 10) | (vo << 20) | ((lastsib ? 1 : 0) << 30);
}

template <class T> SD void sincos_t(T x, T* s, T* c);
template <> SD void sincos_t<float>(float x, float* s, float* c) {
#ifdef __CUDA_ARCH__
  sincosf(x, s, c);
#else
  *s = sinf(x); *c = cosf(x);
#endif
}
template <> SD void sincos_t<double>(double x, double* s, double* c) {
#ifdef __CUDA_ARCH__
  sincos(x, s, c);
#else
  *s = sin(x); *c = cos(x);
#endif
}
template <class T> SD T sqrt_t(T x) { return sqrt(x); }

// Tape and adjoint layouts.  LAY_FULL holds every field (any tree, any joint).
// The pipelined adjoint of serial chains of revolute joints uses two compact
// layouts: LAY_CONS, the 81 tape fields and 33 adjoint fields the adjoint step
// reads for such links, and LAY_PROD, the same 81 tape fields at the same places
// (so the adjoint reads a LAY_PROD tape directly) followed by the forward pass's
// own scratch, the bias force T_PA (in LAY_PROD the inward pass recomputes each
// link's rigid-body inertia from the model constants instead of storing it).
// Fields a compact
// layout lacks are never touched for chain links; host builds with
// ABASIM_HOST_CHECKS abort if one is.
enum : int { LAY_FULL = 0, LAY_PROD = 1, LAY_CONS = 2 };
constexpr int NTAPE_CONS = 81, NTAPE_PROD = 87, NADJ_CONS = 33;
SD constexpr int cons_field(int f) {
  return f < T_IA                      ? f
         : f >= T_U && f < T_U + 6     ? 30 + (f - T_U)
         : f == T_DI                   ? 36
         : f == T_DI2                  ? 37
         : f == T_u                    ? 38
         : f >= T_Ia && f < T_Ia + 21  ? 39 + (f - T_Ia)
         : f >= T_pa && f < T_pa + 6   ? 60 + (f - T_pa)
         : f >= T_AP && f < T_AP + 6   ? 66 + (f - T_AP)
         : f >= T_A && f < T_A + 6     ? 72 + (f - T_A)
         : f == T_QDD                  ? 78
         : f >= T_SC && f < T_SC + 2   ? 79 + (f - T_SC)
                                       : -1;
}
SD constexpr int prod_field(int f) {
  return cons_field(f) >= 0            ? cons_field(f)
         : f >= T_PA && f < T_PA + 6   ? 81 + (f - T_PA)
                                       : -1;
}
SD constexpr int cons_adj(int f) {
  return f >= G_C && f < G_C + 6       ? f - G_C
         : f >= G_E && f < G_E + 9     ? 6 + (f - G_E)
         : f >= G_R && f < G_R + 3     ? 15 + (f - G_R)
         : f >= G_U && f < G_U + 6     ? 18 + (f - G_U)
         : f == G_D                    ? 24
         : f == G_u                    ? 25
         : f >= G_PA && f < G_PA + 6   ? 26 + (f - G_PA)
         : f == G_M                    ? 32
                                       : -1;
}
template <int TL> SD constexpr int tape_stride() { return TL == LAY_FULL ? NTAPE : TL == LAY_PROD ? NTAPE_PROD : NTAPE_CONS; }
template <int AL> SD constexpr int adj_stride() { return AL == LAY_CONS ? NADJ_CONS : NADJ; }
SD int lay_checked(int i) {
#if defined(ABASIM_HOST_CHECKS) && !defined(__CUDA_ARCH__)
  if (i < 0) abort();
#endif
  return i < 0 ? 0 : i;
}
template <int TL> SD int tape_field(int f) {
  return TL == LAY_FULL ? f : lay_checked(TL == LAY_PROD ? prod_field(f) : cons_field(f));
}
template <int AL> SD int adj_field(int f) { return AL == LAY_CONS ? lay_checked(cons_adj(f)) : f; }

// Strided column of one system: element d lives at p[d * B].
template <class T> struct Col {
  T* p;
  long long B;
  SD T& operator[](int d) const { return p[(long long)d * B]; }
};

// Model constants and tapes are stored tile-major: tiles of LANES consecutive
// slots, [tile][link][field][lane], so a warp's 32 systems touch 32 consecutive
// words and every field offset is a compile-time multiple of LANES.
constexpr int LANES = 32;

// contact-tape word of link l, field f (ct points at this system's lane)
template <class T> SD T& ctw(T* ct, int l, int f) { return ct[(l * NCT + f) * LANES]; }
template <class T> SD T ctr(const T* ct, int l, int f) { return ct[(l * NCT + f) * LANES]; }

// The per-system view used by the step functions (pointers at this system's lane).
// T is the arithmetic scalar, PT the stored type of the model constants (they
// differ when T carries derivatives, e.g. a dual number for forward mode).
template <class T, class PT = T, int TL = LAY_FULL, int AL = LAY_FULL> struct Sys {
  const PT* prm;    // [maxL][NPRM][LANES] of this tile
  const int* meta;  // [maxL][LANES] (ints spaced mstride apart)
  T* tape;          // [maxL][tape_stride<TL>][LANES]
  T* adj;           // [maxL][adj_stride<AL>][LANES]
  int nl;
  int mstride = 1;
  SD T P(int l, int f) const { return T(prm[(l * NPRM + f) * LANES]); }
  SD int M(int l) const { return meta[l * LANES * mstride]; }
  SD T& tp(int l, int f) const { return tape[(l * tape_stride<TL>() + tape_field<TL>(f)) * LANES]; }
  SD T& ad(int l, int f) const { return adj[(l * adj_stride<AL>() + adj_field<AL>(f)) * LANES]; }

  // ---- field helpers
  SD V3<T> pv3(int l, int f) const { return {P(l, f), P(l, f + 1), P(l, f + 2)}; }
  SD M3<T> pm3(int l, int f) const { M3<T> m; for (int i = 0; i < 9; ++i) m.a[i] = P(l, f + i); return m; }
  SD S3<T> ps3(int l, int f) const { return {P(l, f), P(l, f + 1), P(l, f + 2), P(l, f + 3), P(l, f + 4), P(l, f + 5)}; }
};

#define ABASIM_FIELD_IO(NAME, ACC)                                                                   \
  template <class T, class PT, int TL, int AL> SD V3<T> NAME##_v3(const Sys<T, PT, TL, AL>& s, int l, int f) {                              \
    return {s.ACC(l, f), s.ACC(l, f + 1), s.ACC(l, f + 2)};                                           \
  }                                                                                                  \
  template <class T, class PT, int TL, int AL> SD void NAME##_v3(const Sys<T, PT, TL, AL>& s, int l, int f, V3<T> v) {                      \
    s.ACC(l, f) = v.x; s.ACC(l, f + 1) = v.y; s.ACC(l, f + 2) = v.z;                                  \
  }                                                                                                  \
  template <class T, class PT, int TL, int AL> SD SV<T> NAME##_sv(const Sys<T, PT, TL, AL>& s, int l, int f) {                              \
    return {NAME##_v3(s, l, f), NAME##_v3(s, l, f + 3)};                                              \
  }                                                                                                  \
  template <class T, class PT, int TL, int AL> SD void NAME##_sv(const Sys<T, PT, TL, AL>& s, int l, int f, SV<T> v) {                      \
    NAME##_v3(s, l, f, v.w); NAME##_v3(s, l, f + 3, v.v);                                             \
  }                                                                                                  \
  template <class T, class PT, int TL, int AL> SD M3<T> NAME##_m3(const Sys<T, PT, TL, AL>& s, int l, int f) {                              \
    M3<T> m; for (int i = 0; i < 9; ++i) m.a[i] = s.ACC(l, f + i); return m;                          \
  }                                                                                                  \
  template <class T, class PT, int TL, int AL> SD void NAME##_m3(const Sys<T, PT, TL, AL>& s, int l, int f, const M3<T>& m) {               \
    for (int i = 0; i < 9; ++i) s.ACC(l, f + i) = m.a[i];                                             \
  }                                                                                                  \
  template <class T, class PT, int TL, int AL> SD S3<T> NAME##_s3(const Sys<T, PT, TL, AL>& s, int l, int f) {                              \
    return {s.ACC(l, f), s.ACC(l, f + 1), s.ACC(l, f + 2), s.ACC(l, f + 3), s.ACC(l, f + 4), s.ACC(l, f + 5)}; \
  }                                                                                                  \
  template <class T, class PT, int TL, int AL> SD void NAME##_s3(const Sys<T, PT, TL, AL>& s, int l, int f, const S3<T>& v) {               \
    s.ACC(l, f) = v.xx; s.ACC(l, f + 1) = v.yy; s.ACC(l, f + 2) = v.zz;                               \
    s.ACC(l, f + 3) = v.xy; s.ACC(l, f + 4) = v.xz; s.ACC(l, f + 5) = v.yz;                           \
  }                                                                                                  \
  template <class T, class PT, int TL, int AL> SD SI<T> NAME##_si(const Sys<T, PT, TL, AL>& s, int l, int f) {                              \
    return {NAME##_s3(s, l, f), NAME##_m3(s, l, f + 6), NAME##_s3(s, l, f + 15)};                     \
  }                                                                                                  \
  template <class T, class PT, int TL, int AL> SD void NAME##_si(const Sys<T, PT, TL, AL>& s, int l, int f, const SI<T>& v) {               \
    NAME##_s3(s, l, f, v.A); NAME##_m3(s, l, f + 6, v.B); NAME##_s3(s, l, f + 15, v.C);               \
  }                                                                                                  \
  template <class T, class PT, int TL, int AL> SD XF<T> NAME##_xf(const Sys<T, PT, TL, AL>& s, int l, int f) {                              \
    return {NAME##_m3(s, l, f), NAME##_v3(s, l, f + 9)};                                              \
  }                                                                                                  \
  template <class T, class PT, int TL, int AL> SD void NAME##_xf(const Sys<T, PT, TL, AL>& s, int l, int f, const XF<T>& v) {               \
    NAME##_m3(s, l, f, v.E); NAME##_v3(s, l, f + 9, v.r);                                             \
  }

ABASIM_FIELD_IO(tp, tp)
ABASIM_FIELD_IO(ad, ad)
#undef ABASIM_FIELD_IO

// ------------------------------------------------------------------ 6x6 SPD solve
// Cholesky of a symmetric 6x6 given in block form; L stored row-major lower
// triangle (21 numbers).  Used for the free root's D = S^T I^A S = I^A.
template <class T> SD void si_full(const SI<T>& I, T* F) {  // 36, row major
  M3<T> A = full(I.A), C = full(I.C);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      F[i * 6 + j] = A.a[3 * i + j];
      F[i * 6 + 3 + j] = I.B.a[3 * i + j];
      F[(3 + i) * 6 + j] = I.B.a[3 * j + i];
      F[(3 + i) * 6 + 3 + j] = C.a[3 * i + j];
    }
}
template <class T> SD void chol6(const SI<T>& I, T* L) {
  T F[36];
  si_full(I, F);
  for (int i = 0; i < 6; ++i) {
    for (int j = 0; j <= i; ++j) {
      T s = F[i * 6 + j];
      for (int k = 0; k < j; ++k) s -= L[i * (i + 1) / 2 + k] * L[j * (j + 1) / 2 + k];
      if (i == j) L[i * (i + 1) / 2 + i] = sqrt_t(s);
      else L[i * (i + 1) / 2 + j] = s / L[j * (j + 1) / 2 + j];
    }
  }
}
template <class T> SD SV<T> chol6_solve(const T* L, SV<T> b) {
  T x[6] = {b.w.x, b.w.y, b.w.z, b.v.x, b.v.y, b.v.z};
  for (int i = 0; i < 6; ++i) {
    T s = x[i];
    for (int k = 0; k < i; ++k) s -= L[i * (i + 1) / 2 + k] * x[k];
    x[i] = s / L[i * (i + 1) / 2 + i];
  }
  for (int i = 5; i >= 0; --i) {
    T s = x[i];
    for (int k = i + 1; k < 6; ++k) s -= L[k * (k + 1) / 2 + i] * x[k];
    x[i] = s / L[i * (i + 1) / 2 + i];
  }
  return {{x[0], x[1], x[2]}, {x[3], x[4], x[5]}};
}

// ------------------------------------------------------------------ D-solve scalar
// The articulated-inertia solves (D = S^T I^A S, 1/D, U D^-1 U^T, the free root's
// 6x6 solve) run in the scalar DT: the storage type T, or double in the mixed
// FP32 + FP64 mode.  1/D is kept on the tape as a hi/lo pair of T words.
template <class T, class DT, class PT, int TL, int AL> SD void put_di(const Sys<T, PT, TL, AL>& s, int l, DT di) {
  const T hi = (T)di;
  s.tp(l, T_DI) = hi;
  s.tp(l, T_DI2) = (T)(di - (DT)hi);
}
template <class T, class DT, class PT, int TL, int AL> SD DT get_di(const Sys<T, PT, TL, AL>& s, int l) {
  return (DT)s.tp(l, T_DI) + (DT)s.tp(l, T_DI2);
}
template <class DT, class T> SD SI<DT> si_cast(const SI<T>& I) {
  SI<DT> o;
  o.A = S3<DT>{(DT)I.A.xx, (DT)I.A.yy, (DT)I.A.zz, (DT)I.A.xy, (DT)I.A.xz, (DT)I.A.yz};
  o.C = S3<DT>{(DT)I.C.xx, (DT)I.C.yy, (DT)I.C.zz, (DT)I.C.xy, (DT)I.C.xz, (DT)I.C.yz};
  for (int i = 0; i < 9; ++i) o.B.a[i] = (DT)I.B.a[i];
  return o;
}
template <class DT, class T> SD SV<DT> sv_cast(const SV<T>& v) {
  return SV<DT>{{(DT)v.w.x, (DT)v.w.y, (DT)v.w.z}, {(DT)v.v.x, (DT)v.v.y, (DT)v.v.z}};
}
// I - di u u^T formed in DT, rounded to T
template <class T, class DT> SD SI<T> minus_scaled_outer(const SI<T>& I, DT di, SV<T> u) {
  const SI<DT> Id = si_cast<DT>(I);
  const SV<DT> ud = sv_cast<DT>(u);
  const SI<DT> r = Id - scale(di, sym_outer(ud, ud));
  SI<T> o;
  o.A = S3<T>{(T)r.A.xx, (T)r.A.yy, (T)r.A.zz, (T)r.A.xy, (T)r.A.xz, (T)r.A.yz};
  o.C = S3<T>{(T)r.C.xx, (T)r.C.yy, (T)r.C.zz, (T)r.C.xy, (T)r.C.xz, (T)r.C.yz};
  for (int i = 0; i < 9; ++i) o.B.a[i] = (T)r.B.a[i];
  return o;
}
// the free root's solve I^A x = b, Cholesky in DT
template <class T, class DT> SD SV<T> spd_solve(const SI<T>& IA, SV<T> b) {
  DT L[21];
  chol6(si_cast<DT>(IA), L);
  const SV<DT> x = chol6_solve(L, sv_cast<DT>(b));
  return SV<T>{{(T)x.w.x, (T)x.w.y, (T)x.w.z}, {(T)x.v.x, (T)x.v.y, (T)x.v.z}};
}

// ------------------------------------------------------------------ forward
// Runs jcalc and the three ABA passes for the state (q, qd) and joint force tau,
// leaving qdd on the tape; with ADJ set, also every intermediate the adjoint
// step reads (a forward-only rollout skips those stores).  Values passed between a
// link and its parent ride in registers when the parent is the previous link (the
// whole of a serial chain); other parents go through the tape.  Each iteration
// loads what it needs before it stores anything, so the loads overlap.
template <class T, class DT, bool ADJ = true, class PT, int TL, int AL>
SD void aba_forward(const Sys<T, PT, TL, AL>& s, Col<const T> q, Col<const T> qd, Col<const T> tau, V3<T> grav) {
  const int nl = s.nl;
  // jcalc + pass 1 (root -> leaves)
  SV<T> v_prev = zeroSV<T>();
  for (int l = 0; l < nl; ++l) {
    const int m = s.M(l);
    const int par = meta_parent(m), jt = meta_jtype(m), qo = meta_qoff(m), vo = meta_voff(m);
    const M3<T> Et = s.pm3(l, P_E);
    const V3<T> rt = s.pv3(l, P_R);
    const T mass = s.P(l, P_M);
    const V3<T> com = s.pv3(l, P_C);
    const S3<T> Ic = s.ps3(l, P_IC);
    SV<T> vpar = zeroSV<T>();
    if (par >= 0) vpar = (par == l - 1) ? v_prev : tp_sv(s, par, T_V);
    XF<T> X;
    SV<T> v, c;
    T sn = 0, cs = 1;
    if (jt == J_REVOLUTE) {  // about the link's z axis: vJ = [qd e_z; 0]
      const T ql = q[qo], vl = qd[vo];
      sincos_t(ql, &sn, &cs);
      X = XF<T>{rotz_T_mm(sn, cs, Et), rt};
      if (par >= 0) {
        v = apply(X, vpar);
        v.w.z += vl;
      } else {
        v = SV<T>{{T(0), T(0), vl}, zero3<T>()};
      }
      c = crossm_z(v, vl);
    } else {
      const V3<T> p{q[qo], q[qo + 1], q[qo + 2]};
      const M3<T> EJ = transpose(quat_R(q[qo + 3], q[qo + 4], q[qo + 5], q[qo + 6]));
      X = compose(EJ, p, Et, rt);
      const SV<T> vJ{{qd[vo], qd[vo + 1], qd[vo + 2]}, {qd[vo + 3], qd[vo + 4], qd[vo + 5]}};
      v = vJ;
      if (par >= 0) v += apply(X, vpar);
      c = crossm(v, vJ);
    }
    const SI<T> I = rbi(mass, com, Ic);
    const SV<T> h = mul(I, v);
    tp_xf(s, l, T_E, X);
    tp_sv(s, l, T_V, v);
    tp_sv(s, l, T_C, c);
    if (ADJ) tp_sv(s, l, T_H, h);
    if (TL != LAY_PROD) tp_si(s, l, T_IA, I);
    tp_sv(s, l, T_PA, crossf(v, h));
    if (ADJ && jt == J_REVOLUTE) {
      s.tp(l, T_SC) = sn;
      s.tp(l, T_SC + 1) = cs;
    }
    v_prev = v;
  }
  // pass 2 (leaves -> root)
  SI<T> cI = zeroSI<T>();
  SV<T> cp = zeroSV<T>();
  bool carry = false;
  for (int l = nl - 1; l >= 0; --l) {
    const int m = s.M(l);
    const int par = meta_parent(m), jt = meta_jtype(m), vo = meta_voff(m);
    SI<T> IA = TL == LAY_PROD ? rbi(s.P(l, P_M), s.pv3(l, P_C), s.ps3(l, P_IC)) : tp_si(s, l, T_IA);
    SV<T> pA = tp_sv(s, l, T_PA);
    if (carry) {
      IA += cI;
      pA += cp;
    }
    carry = false;
    if (jt == J_REVOLUTE) {
      const T tl = tau[vo] - s.P(l, P_DAMP) * qd[vo];  // viscous damping: joint force -b qd
      SV<T> c = zeroSV<T>();
      XF<T> X;
      if (par >= 0) {
        c = tp_sv(s, l, T_C);
        X = tp_xf(s, l, T_E);
      }
      const SV<T> U = col_z(IA);  // U = I^A S, D = S^T U, u = tau - S^T p^A with S = [e_z; 0]
      const DT Di = DT(1) / (DT)U.w.z;
      const T u = tl - pA.w.z;
      tp_sv(s, l, T_U, U);
      put_di<T, DT, PT>(s, l, Di);
      s.tp(l, T_u) = u;
      if (par >= 0) {
        const SI<T> Ia = minus_scaled_outer<T, DT>(IA, Di, U);
        const SV<T> pa = pA + mul(Ia, c) + (T)((DT)u * Di) * U;
        if (ADJ) {
          tp_si(s, l, T_Ia, Ia);
          tp_sv(s, l, T_pa, pa);
        }
        const SI<T> Cn = congruence(X, Ia);
        const SV<T> pn = applyT(X, pa);
        if (par == l - 1) {
          cI = Cn;
          cp = pn;
          carry = true;
        } else {
          tp_si(s, par, T_IA, tp_si(s, par, T_IA) + Cn);
          tp_sv(s, par, T_PA, tp_sv(s, par, T_PA) + pn);
        }
      }
    } else {  // free root: D = I^A (kept on the tape), u = tau - p^A
      SV<T> u{{tau[vo], tau[vo + 1], tau[vo + 2]}, {tau[vo + 3], tau[vo + 4], tau[vo + 5]}};
      u -= pA;
      tp_si(s, l, T_IA, IA);
      tp_sv(s, l, T_u, u);
    }
  }
  // pass 3 (root -> leaves)
  const SV<T> a0{zero3<T>(), -grav};
  SV<T> a_prev = a0;
  for (int l = 0; l < nl; ++l) {
    const int m = s.M(l);
    const int par = meta_parent(m), jt = meta_jtype(m);
    const XF<T> X = tp_xf(s, l, T_E);
    const SV<T> c = tp_sv(s, l, T_C);
    SV<T> apar = a0;
    if (par >= 0) apar = (par == l - 1) ? a_prev : tp_sv(s, par, T_A);
    SV<T> a;
    if (jt == J_REVOLUTE) {
      const SV<T> U = tp_sv(s, l, T_U);
      const T u = s.tp(l, T_u);
      const DT Di = get_di<T, DT, PT>(s, l);
      const SV<T> ap = apply(X, apar) + c;
      const T qdd = (T)(((DT)u - (DT)dot(U, ap)) * Di);
      s.tp(l, T_QDD) = qdd;
      a = ap;
      a.w.z += qdd;
      if (ADJ) tp_sv(s, l, T_AP, ap);
    } else {
      const SI<T> IA = tp_si(s, l, T_IA);
      const SV<T> u = tp_sv(s, l, T_u);
      const SV<T> ap = apply(X, apar) + c;
      a = spd_solve<T, DT>(IA, u);
      tp_sv(s, l, T_QDD, a - ap);
      if (ADJ) tp_sv(s, l, T_AP, ap);
    }
    tp_sv(s, l, T_A, a);
    a_prev = a;
  }
}

// ------------------------------------------------------------------ split forward
// The ABA forward of a serial chain of revolute joints (parent of link l is
// l - 1) split into the part that depends on q alone (the articulated-inertia
// recursion) and the rest (velocities, bias forces, accelerations), so two
// warps can run them side by side.  Same formulas and operation order as
// aba_forward.  Exchange record per link, [link][EX_N][LANES]: U, 1/D (hi/lo
// pair) and I^a; the bias half's own scratch, [link][BS_N][LANES]: X, c, p^A, u.
enum : int { EX_U = 0, EX_DI = 6, EX_Ia = 8, EX_N = 29 };
enum : int { BS_E = 0, BS_C = 12, BS_PA = 18, BS_u = 24, BS_N = 25 };

template <class T> SD T& exw(T* base, int l, int f) { return base[(l * EX_N + f) * LANES]; }
template <class T> SD T& bsw(T* base, int l, int f) { return base[(l * BS_N + f) * LANES]; }

// Inertia half, leaves -> root; ready(l) runs after link l's record is written.
template <class T, class DT, class PT, class F>
SD void chain_inertia(const Sys<T, PT>& s, Col<const T> q, T* ex, F&& ready, int links) {
  SI<T> cI = zeroSI<T>();
  for (int l = links - 1; l >= 0; --l) {
    if (l < s.nl) {
      const int m = s.M(l);
      T sn, cs;
      sincos_t(q[meta_qoff(m)], &sn, &cs);
      const XF<T> X{rotz_T_mm(sn, cs, s.pm3(l, P_E)), s.pv3(l, P_R)};
      SI<T> IA = rbi(s.P(l, P_M), s.pv3(l, P_C), s.ps3(l, P_IC));
      if (l < s.nl - 1) IA += cI;
      const SV<T> U = col_z(IA);
      const DT Di = DT(1) / (DT)U.w.z;
      const T hi = (T)Di;
      const T u6[6] = {U.w.x, U.w.y, U.w.z, U.v.x, U.v.y, U.v.z};
      for (int i = 0; i < 6; ++i) exw(ex, l, EX_U + i) = u6[i];
      exw(ex, l, EX_DI) = hi;
      exw(ex, l, EX_DI + 1) = (T)(Di - (DT)hi);
      if (l > 0) {
        const SI<T> Ia = minus_scaled_outer<T, DT>(IA, Di, U);
        const T ia[21] = {Ia.A.xx, Ia.A.yy, Ia.A.zz, Ia.A.xy, Ia.A.xz, Ia.A.yz, Ia.B.a[0], Ia.B.a[1], Ia.B.a[2],
                          Ia.B.a[3], Ia.B.a[4], Ia.B.a[5], Ia.B.a[6], Ia.B.a[7], Ia.B.a[8], Ia.C.xx, Ia.C.yy,
                          Ia.C.zz, Ia.C.xy, Ia.C.xz, Ia.C.yz};
        for (int i = 0; i < 21; ++i) exw(ex, l, EX_Ia + i) = ia[i];
        cI = congruence(X, Ia);
      }
    }
    ready(l);
  }
}

// Bias half, pass 1 (root -> leaves): X, v, c, p^A into the scratch.
template <class T, class PT>
SD void chain_bias_out(const Sys<T, PT>& s, Col<const T> q, Col<const T> qd, T* bs) {
  SV<T> v_prev = zeroSV<T>();
  for (int l = 0; l < s.nl; ++l) {
    const int m = s.M(l);
    T sn, cs;
    sincos_t(q[meta_qoff(m)], &sn, &cs);
    const XF<T> X{rotz_T_mm(sn, cs, s.pm3(l, P_E)), s.pv3(l, P_R)};
    const T vl = qd[meta_voff(m)];
    SV<T> v{{T(0), T(0), vl}, zero3<T>()};
    if (l > 0) {
      v = apply(X, v_prev);
      v.w.z += vl;
    }
    const SV<T> c = crossm_z(v, vl);
    const SV<T> h = mul(rbi(s.P(l, P_M), s.pv3(l, P_C), s.ps3(l, P_IC)), v);
    const SV<T> pA = crossf(v, h);
    for (int i = 0; i < 9; ++i) bsw(bs, l, BS_E + i) = X.E.a[i];
    bsw(bs, l, BS_E + 9) = X.r.x;
    bsw(bs, l, BS_E + 10) = X.r.y;
    bsw(bs, l, BS_E + 11) = X.r.z;
    const T cc[6] = {c.w.x, c.w.y, c.w.z, c.v.x, c.v.y, c.v.z};
    const T pp[6] = {pA.w.x, pA.w.y, pA.w.z, pA.v.x, pA.v.y, pA.v.z};
    for (int i = 0; i < 6; ++i) {
      bsw(bs, l, BS_C + i) = cc[i];
      bsw(bs, l, BS_PA + i) = pp[i];
    }
    v_prev = v;
  }
}

template <class T> SD XF<T> bs_xf(T* bs, int l) {
  XF<T> X;
  for (int i = 0; i < 9; ++i) X.E.a[i] = bsw(bs, l, BS_E + i);
  X.r = V3<T>{bsw(bs, l, BS_E + 9), bsw(bs, l, BS_E + 10), bsw(bs, l, BS_E + 11)};
  return X;
}
template <class T> SD SV<T> rd_sv(T* base, int l, int f, int n) {
  return SV<T>{{base[(l * n + f) * LANES], base[(l * n + f + 1) * LANES], base[(l * n + f + 2) * LANES]},
               {base[(l * n + f + 3) * LANES], base[(l * n + f + 4) * LANES], base[(l * n + f + 5) * LANES]}};
}

// Bias half, pass 2 (leaves -> root) and pass 3 (root -> leaves), then the
// integrator: wait(l) runs before link l's exchange record is read.
template <class T, class DT, class PT, class F>
SD void chain_bias_in(const Sys<T, PT>& s, Col<T> q, Col<T> qd, Col<const T> tau, V3<T> grav, T* ex, T* bs,
                      F&& wait, int links, T dt, int integ) {
  SV<T> cp = zeroSV<T>();
  for (int l = links - 1; l >= 0; --l) {
    wait(l);
    if (l >= s.nl) continue;
    const int m = s.M(l);
    const int vo = meta_voff(m);
    SV<T> pA = rd_sv(bs, l, BS_PA, BS_N);
    if (l < s.nl - 1) pA += cp;
    const T tl = tau[vo] - s.P(l, P_DAMP) * qd[vo];
    const T u = tl - pA.w.z;
    bsw(bs, l, BS_u) = u;
    if (l > 0) {
      const SV<T> U = rd_sv(ex, l, EX_U, EX_N);
      const DT Di = (DT)exw(ex, l, EX_DI) + (DT)exw(ex, l, EX_DI + 1);
      SI<T> Ia;
      Ia.A = S3<T>{exw(ex, l, EX_Ia), exw(ex, l, EX_Ia + 1), exw(ex, l, EX_Ia + 2), exw(ex, l, EX_Ia + 3),
                   exw(ex, l, EX_Ia + 4), exw(ex, l, EX_Ia + 5)};
      for (int i = 0; i < 9; ++i) Ia.B.a[i] = exw(ex, l, EX_Ia + 6 + i);
      Ia.C = S3<T>{exw(ex, l, EX_Ia + 15), exw(ex, l, EX_Ia + 16), exw(ex, l, EX_Ia + 17),
                   exw(ex, l, EX_Ia + 18), exw(ex, l, EX_Ia + 19), exw(ex, l, EX_Ia + 20)};
      const SV<T> c = rd_sv(bs, l, BS_C, BS_N);
      const SV<T> pa = pA + mul(Ia, c) + (T)((DT)u * Di) * U;
      cp = applyT(bs_xf(bs, l), pa);
    }
  }
  const SV<T> a0{zero3<T>(), -grav};
  SV<T> a_prev = a0;
  for (int l = 0; l < s.nl; ++l) {
    const int m = s.M(l);
    const SV<T> U = rd_sv(ex, l, EX_U, EX_N);
    const DT Di = (DT)exw(ex, l, EX_DI) + (DT)exw(ex, l, EX_DI + 1);
    const SV<T> ap = apply(bs_xf(bs, l), a_prev) + rd_sv(bs, l, BS_C, BS_N);
    const T qdd = (T)(((DT)bsw(bs, l, BS_u) - (DT)dot(U, ap)) * Di);
    SV<T> a = ap;
    a.w.z += qdd;
    a_prev = a;
    const int qo = meta_qoff(m), vo = meta_voff(m);
    const T v0 = qd[vo];
    const T v1 = v0 + dt * qdd;
    qd[vo] = v1;
    q[qo] = q[qo] + dt * (integ == I_SEMI_IMPLICIT ? v1 : v0);
  }
}

// Integrates x -> x' in place from the qdd on the tape, plus the contact
// velocity change C_DV of the contact tape ct when given.  The state columns may
// be wider than the step's scalar (A = double with T = float: the running state
// accumulated in FP64 while the dynamics run in FP32).
template <class A, class T, class PT, int TL, int AL>
SD void integrate_in(const Sys<T, PT, TL, AL>& s, Col<A> q, Col<A> qd, A dt, int integ, const T* ct) {
  for (int l = 0; l < s.nl; ++l) {
    const int m = s.M(l);
    const int jt = meta_jtype(m), qo = meta_qoff(m), vo = meta_voff(m);
    if (jt == J_REVOLUTE) {
      A v0 = qd[vo];
      A v1 = v0 + dt * (A)s.tp(l, T_QDD);
      if (ct) v1 += (A)ctr(ct, l, C_DV);
      qd[vo] = v1;
      q[qo] = q[qo] + dt * (integ == I_SEMI_IMPLICIT ? v1 : v0);
    } else {
      A nu[6];
      for (int i = 0; i < 6; ++i) {
        A v0 = qd[vo + i];
        A v1 = v0 + dt * (A)s.tp(l, T_QDD + i);
        if (ct) v1 += (A)ctr(ct, l, C_DV + i);
        qd[vo + i] = v1;
        nu[i] = integ == I_SEMI_IMPLICIT ? v1 : v0;
      }
      A qt[4] = {q[qo + 3], q[qo + 4], q[qo + 5], q[qo + 6]};
      V3<A> dp = mul(quat_R(qt[0], qt[1], qt[2], qt[3]), V3<A>{nu[3], nu[4], nu[5]});
      q[qo] = q[qo] + dt * dp.x;
      q[qo + 1] = q[qo + 1] + dt * dp.y;
      q[qo + 2] = q[qo + 2] + dt * dp.z;
      A wq[4] = {nu[0], nu[1], nu[2], A(0)};
      A r[4];
      quat_mul(qt, wq, r);
      A raw[4];
      for (int i = 0; i < 4; ++i) raw[i] = qt[i] + A(0.5) * dt * r[i];
      A n = sqrt_t(raw[0] * raw[0] + raw[1] * raw[1] + raw[2] * raw[2] + raw[3] * raw[3]);
      for (int i = 0; i < 4; ++i) q[qo + 3 + i] = raw[i] / n;
    }
  }
}
template <class T, class PT, int TL, int AL>
SD void integrate(const Sys<T, PT, TL, AL>& s, Col<T> q, Col<T> qd, T dt, int integ, const T* ct = nullptr) {
  integrate_in<T>(s, q, qd, dt, integ, ct);
}

// ------------------------------------------------------------------ adjoint
// Integrator adjoint of one link (folded into the pass-3 adjoint loop): turns the
// adjoint of x^{k+1} held in (gq, gqd) into the direct part of the adjoint of x^k
// for this link's coordinates and returns the adjoint of its qdd in qddb[0..nv).
template <class T, class PT, int TL, int AL>
SD void integrator_adjoint(const Sys<T, PT, TL, AL>& s, int l, int jt, int qo, int vo, Col<const T> q,
                           Col<const T> qd, Col<T> gq, Col<T> gqd, T dt, int integ, T* qddb,
                           const T* ct = nullptr) {
  const T half = T(0.5);
  if (jt == J_REVOLUTE) {
    const T qb = gq[qo], vb = gqd[vo];
    if (integ == I_SEMI_IMPLICIT) {
      const T vt = vb + dt * qb;
      gqd[vo] = vt;
      qddb[0] = dt * vt;
    } else {
      gqd[vo] = vb + dt * qb;
      qddb[0] = dt * vb;
    }
    return;
  }
  T nu[6], nub[6];
  for (int i = 0; i < 6; ++i) {
    const T v0 = qd[vo + i];
    T v1 = v0 + dt * s.tp(l, T_QDD + i);
    if (ct) v1 += ctr(ct, l, C_DV + i);
    nu[i] = integ == I_SEMI_IMPLICIT ? v1 : v0;
    nub[i] = gqd[vo + i];
  }
  const T qt[4] = {q[qo + 3], q[qo + 4], q[qo + 5], q[qo + 6]};
  const T wq[4] = {nu[0], nu[1], nu[2], T(0)};
  T r[4], raw[4];
  quat_mul(qt, wq, r);
  for (int i = 0; i < 4; ++i) raw[i] = qt[i] + half * dt * r[i];
  const T n = sqrt_t(raw[0] * raw[0] + raw[1] * raw[1] + raw[2] * raw[2] + raw[3] * raw[3]);
  T qn[4], qnb[4], rawb[4];
  T d = 0;
  for (int i = 0; i < 4; ++i) {
    qn[i] = raw[i] / n;
    qnb[i] = gq[qo + 3 + i];
    d += qn[i] * qnb[i];
  }
  for (int i = 0; i < 4; ++i) rawb[i] = (qnb[i] - qn[i] * d) / n;
  // raw = quat + dt/2 quat (x) (w, 0):  quat_bar += rawb (x) (w, 0)^*,  w_bar = vec(quat^* (x) rawb)
  T qb[4] = {rawb[0], rawb[1], rawb[2], rawb[3]};
  const T wconj[4] = {-nu[0], -nu[1], -nu[2], T(0)};
  T t1[4];
  quat_mul(rawb, wconj, t1);
  for (int i = 0; i < 4; ++i) qb[i] += half * dt * t1[i];
  const T qconj[4] = {-qt[0], -qt[1], -qt[2], qt[3]};
  T t2[4];
  quat_mul(qconj, rawb, t2);
  T velb[6] = {half * dt * t2[0], half * dt * t2[1], half * dt * t2[2], 0, 0, 0};
  // p' = p + dt R(quat) v
  const V3<T> pb{gq[qo], gq[qo + 1], gq[qo + 2]};
  const M3<T> R = quat_R(qt[0], qt[1], qt[2], qt[3]);
  const V3<T> vvb = dt * mulT(R, pb);
  velb[3] = vvb.x;
  velb[4] = vvb.y;
  velb[5] = vvb.z;
  quat_R_adj(qt[0], qt[1], qt[2], qt[3], scale(dt, outer(pb, V3<T>{nu[3], nu[4], nu[5]})), qb);
  for (int i = 0; i < 4; ++i) gq[qo + 3 + i] = qb[i];
  for (int i = 0; i < 6; ++i) {
    if (integ == I_SEMI_IMPLICIT) {
      const T tot = nub[i] + velb[i];
      gqd[vo + i] = tot;
      qddb[i] = dt * tot;
    } else {
      gqd[vo + i] = nub[i] + velb[i];
      qddb[i] = dt * nub[i];
    }
  }
}

// Requires aba_forward(q, qd, tau) to have filled the tape.  On entry gq, gqd hold
// the adjoint of x^{k+1}; on exit they hold the adjoint of x^k.  Writes the
// adjoint of tau into gtau and adds dPhi/dm of every link into gm[l * B].
// Adjoints flowing between a link and its parent ride in registers when the
// parent is the previous link; accumulators in the adjoint tape serve the other
// (tree) children and are zeroed first only for links that have such children.
// With a contact tape ct, the integrator adjoint has already run (its qdd
// adjoint is in C_QDDB) and the contact adjoint's B_* terms are added in.
template <class T, class DT, class PT, int TL, int AL>
SD void step_adjoint(const Sys<T, PT, TL, AL>& s, Col<const T> q, Col<const T> qd, Col<T> gq, Col<T> gqd,
                     Col<T> gtau, Col<T> gm, V3<T> grav, T dt, int integ, const T* ct = nullptr) {
  const int nl = s.nl;
  const T half = T(0.5);
  if (ct) {
    for (int l = 0; l < nl; ++l) {
      const int m = s.M(l);
      const bool rev = meta_jtype(m) == J_REVOLUTE;
      for (int i = 0; i < (rev ? 1 : 6); ++i) gqd[meta_voff(m) + i] += ctr(ct, l, B_QD + i);
      if (rev) gq[meta_qoff(m)] += ctr(ct, l, B_Q);
    }
  }
  for (int l = 0; l < nl; ++l) {
    if (meta_treechild(s.M(l))) {
      ad_sv(s, l, G_A, zeroSV<T>());
      ad_sv(s, l, G_V, zeroSV<T>());
    }
  }
  const SV<T> a0{zero3<T>(), -grav};
  // integrator adjoint + pass 3 adjoint (leaves -> root)
  {
    SV<T> cab = zeroSV<T>();
    bool carry = false;
    for (int l = nl - 1; l >= 0; --l) {
      const int m = s.M(l);
      const int par = meta_parent(m), jt = meta_jtype(m), qo = meta_qoff(m), vo = meta_voff(m);
      const XF<T> X = tp_xf(s, l, T_E);
      SV<T> apar = a0;
      if (par >= 0) apar = tp_sv(s, par, T_A);
      SV<T> ab = meta_treechild(m) ? ad_sv(s, l, G_A) : zeroSV<T>();
      if (carry) ab += cab;
      carry = false;
      T qddb[6];
      if (ct) {
        for (int i = 0; i < 6; ++i) qddb[i] = ctr(ct, l, C_QDDB + i) + ctr(ct, l, B_QDD + i);
      } else {
        integrator_adjoint(s, l, jt, qo, vo, q, qd, gq, gqd, dt, integ, qddb);
      }
      SV<T> apb;
      if (jt == J_REVOLUTE) {
        const SV<T> U = tp_sv(s, l, T_U);
        const SV<T> ap = tp_sv(s, l, T_AP);
        const DT Di = get_di<T, DT, PT>(s, l);
        const T qdd = s.tp(l, T_QDD);
        const T qb = qddb[0] + ab.w.z;
        const T wb = (T)((DT)qb * Di);
        apb = ab - wb * U;
        SV<T> Ub = zeroSV<T>() - wb * ap;
        T Db = -wb * qdd;
        if (ct) {  // contact solve: U and 1/D adjoints (dD = -D^-2 d(1/D))
          Ub += SV<T>{{ctr(ct, l, B_U), ctr(ct, l, B_U + 1), ctr(ct, l, B_U + 2)},
                      {ctr(ct, l, B_U + 3), ctr(ct, l, B_U + 4), ctr(ct, l, B_U + 5)}};
          Db -= (T)((DT)ctr(ct, l, B_DI) * Di * Di);
        }
        ad_sv(s, l, G_U, Ub);
        s.ad(l, G_D) = Db;
        s.ad(l, G_u) = wb;
      } else {
        const SV<T> qb{{qddb[0], qddb[1], qddb[2]}, {qddb[3], qddb[4], qddb[5]}};
        const SV<T> a = tp_sv(s, l, T_A);
        const SV<T> ub = spd_solve<T, DT>(tp_si(s, l, T_IA), ab + qb);
        apb = zeroSV<T>() - qb;
        ad_sv(s, l, G_u, ub);
        SI<T> IAb = scale(T(-1), sym_outer(ub, a));
        if (ct) {
          S3<T> A{ctr(ct, l, B_IA), ctr(ct, l, B_IA + 1), ctr(ct, l, B_IA + 2), ctr(ct, l, B_IA + 3),
                  ctr(ct, l, B_IA + 4), ctr(ct, l, B_IA + 5)};
          M3<T> Bm;
          for (int i = 0; i < 9; ++i) Bm.a[i] = ctr(ct, l, B_IA + 6 + i);
          S3<T> C{ctr(ct, l, B_IA + 15), ctr(ct, l, B_IA + 16), ctr(ct, l, B_IA + 17), ctr(ct, l, B_IA + 18),
                  ctr(ct, l, B_IA + 19), ctr(ct, l, B_IA + 20)};
          IAb += SI<T>{A, Bm, C};
        }
        ad_si(s, l, G_IA, IAb);
      }
      ad_sv(s, l, G_C, apb);
      M3<T> Eb = zeroM3<T>();
      V3<T> rb = zero3<T>();
      if (ct) {
        for (int i = 0; i < 9; ++i) Eb.a[i] = ctr(ct, l, B_E + i);
        rb = V3<T>{ctr(ct, l, B_R), ctr(ct, l, B_R + 1), ctr(ct, l, B_R + 2)};
      }
      SV<T> apar_b = zeroSV<T>();
      apply_adj(X, apar, apb, Eb, rb, par >= 0 ? &apar_b : (SV<T>*)nullptr);
      ad_m3(s, l, G_E, Eb);
      ad_v3(s, l, G_R, rb);
      if (par >= 0) {
        if (par == l - 1) {
          cab = apar_b;
          carry = true;
        } else {
          ad_sv(s, par, G_A, ad_sv(s, par, G_A) + apar_b);
        }
      }
    }
  }
  // pass 2 adjoint (root -> leaves)
  {
    SI<T> cIAb = zeroSI<T>();
    SV<T> cpAb = zeroSV<T>();
    for (int l = 0; l < nl; ++l) {
      const int m = s.M(l);
      const int par = meta_parent(m), jt = meta_jtype(m), vo = meta_voff(m);
      SV<T> pAb = zeroSV<T>();
      SI<T> IAb;
      if (jt == J_REVOLUTE) {
        SV<T> Ub = ad_sv(s, l, G_U);
        T Db = s.ad(l, G_D);
        T ub = s.ad(l, G_u);
        const DT Di = get_di<T, DT, PT>(s, l);
        const T u = s.tp(l, T_u);
        const SV<T> U = tp_sv(s, l, T_U);
        IAb = zeroSI<T>();
        if (par >= 0) {
          const XF<T> X = tp_xf(s, l, T_E);
          const SI<T> Ia = tp_si(s, l, T_Ia);
          const SV<T> pa = tp_sv(s, l, T_pa);
          const SV<T> c = tp_sv(s, l, T_C);
          SV<T> cb = ad_sv(s, l, G_C);
          M3<T> Eb = ad_m3(s, l, G_E);
          V3<T> rb = ad_v3(s, l, G_R);
          SI<T> IAbp;
          SV<T> pAbp;
          if (par == l - 1) {
            IAbp = cIAb;
            pAbp = cpAb;
          } else {
            IAbp = ad_si(s, par, G_IA);
            pAbp = ad_sv(s, par, G_PA);
          }
          SV<T> pab = zeroSV<T>();
          SI<T> Iab = zeroSI<T>();
          applyT_adj(X, pa, pAbp, Eb, rb, &pab);
          congruence_adj(X, Ia, IAbp, Iab, Eb, rb);
          ad_m3(s, l, G_E, Eb);
          ad_v3(s, l, G_R, rb);
          // pa = pA + Ia c + U (u / D)
          pAb += pab;
          Iab += sym_outer(pab, c);
          cb += mul(Ia, pab);
          ad_sv(s, l, G_C, cb);
          Ub += (T)((DT)u * Di) * pab;
          const T gb = dot(U, pab);
          ub += (T)((DT)gb * Di);
          Db -= (T)((DT)gb * (DT)u * Di * Di);
          // Ia = IA - U U^T / D
          IAb += Iab;
          const SV<T> IbU = mul(Iab, U);
          Ub -= (T)(DT(2) * Di) * IbU;
          Db += (T)(Di * Di * (DT)dot(U, IbU));
        }
        // u = tau - b qd - S^T pA,  D = S^T U,  U = IA S with S = [e_z; 0]:
        // IAb += sym_outer(Ub.w, e_z) and outer(e_z, Ub.v) / 2 (third column / row)
        gtau[vo] = ub;
        gqd[vo] -= s.P(l, P_DAMP) * ub;
        pAb.w.z -= ub;
        Ub.w.z += Db;
        IAb.A.zz += Ub.w.z;
        IAb.A.xz += half * Ub.w.x;
        IAb.A.yz += half * Ub.w.y;
        IAb.B.a[6] += half * Ub.v.x;
        IAb.B.a[7] += half * Ub.v.y;
        IAb.B.a[8] += half * Ub.v.z;
      } else {
        const SV<T> ub = ad_sv(s, l, G_u);
        IAb = ad_si(s, l, G_IA);
        gtau[vo] = ub.w.x;
        gtau[vo + 1] = ub.w.y;
        gtau[vo + 2] = ub.w.z;
        gtau[vo + 3] = ub.v.x;
        gtau[vo + 4] = ub.v.y;
        gtau[vo + 5] = ub.v.z;
        pAb -= ub;
      }
      if (meta_treechild(m)) ad_si(s, l, G_IA, IAb);
      ad_sv(s, l, G_PA, pAb);
      s.ad(l, G_M) = rbi_dmass(IAb, s.pv3(l, P_C));
      cIAb = IAb;
      cpAb = pAb;
    }
  }
  // pass 1 adjoint + jcalc adjoint (leaves -> root)
  {
    SV<T> cvb = zeroSV<T>();
    bool carry = false;
    for (int l = nl - 1; l >= 0; --l) {
      const int m = s.M(l);
      const int par = meta_parent(m), jt = meta_jtype(m), qo = meta_qoff(m), vo = meta_voff(m);
      const SV<T> v = tp_sv(s, l, T_V);
      const SV<T> h = tp_sv(s, l, T_H);
      const SV<T> pAb = ad_sv(s, l, G_PA);
      const SV<T> cb = ad_sv(s, l, G_C);
      const XF<T> X = tp_xf(s, l, T_E);
      M3<T> Eb = ad_m3(s, l, G_E);
      V3<T> rb = ad_v3(s, l, G_R);
      SV<T> vpar = zeroSV<T>();
      if (par >= 0) vpar = tp_sv(s, par, T_V);
      const V3<T> com = s.pv3(l, P_C);
      const T mass = s.P(l, P_M);
      const S3<T> Ic = s.ps3(l, P_IC);
      const M3<T> Et = s.pm3(l, P_E);
      T gml = s.ad(l, G_M);
      SV<T> vb = meta_treechild(m) ? ad_sv(s, l, G_V) : zeroSV<T>();
      if (carry) vb += cvb;
      carry = false;
      SV<T> hb = zeroSV<T>();
      crossf_adj(v, h, pAb, vb, hb);
      const SI<T> I = rbi(mass, com, Ic);
      gml += rbi_dmass_bilinear(hb, v, com);
      vb += mul(I, hb);
      SV<T> vJb = zeroSV<T>();
      T qdb = T(0);  // revolute: the qd adjoint through c = v x [qd e_z; 0]
      if (jt == J_REVOLUTE) {
        qdb = crossm_z_adj(v, qd[vo], cb, vb);
      } else {
        const SV<T> vJ{{qd[vo], qd[vo + 1], qd[vo + 2]}, {qd[vo + 3], qd[vo + 4], qd[vo + 5]}};
        crossm_adj(v, vJ, cb, vb, vJb);
      }
      vJb += vb;
      if (par >= 0) {
        SV<T> vpb = zeroSV<T>();
        apply_adj(X, vpar, vb, Eb, rb, &vpb);
        if (par == l - 1) {
          cvb = vpb;
          carry = true;
        } else {
          ad_sv(s, par, G_V, ad_sv(s, par, G_V) + vpb);
        }
      }
      if (jt == J_REVOLUTE) {
        gqd[vo] += qdb + vJb.w.z;
        gq[qo] += rotz_T_dq(s.tp(l, T_SC), s.tp(l, T_SC + 1), Eb, Et);  // E = E_J E_t
      } else {
        const M3<T> EJb = mmT(Eb, Et);
        const T vv[6] = {vJb.w.x, vJb.w.y, vJb.w.z, vJb.v.x, vJb.v.y, vJb.v.z};
        for (int i = 0; i < 6; ++i) gqd[vo + i] += vv[i];
        const V3<T> pb = mul(Et, rb);  // r = r_t + E_t^T p
        gq[qo] += pb.x;
        gq[qo + 1] += pb.y;
        gq[qo + 2] += pb.z;
        T qb[4] = {0, 0, 0, 0};
        quat_R_adj(q[qo + 3], q[qo + 4], q[qo + 5], q[qo + 6], transpose(EJb), qb);
        for (int i = 0; i < 4; ++i) gq[qo + 3 + i] += qb[i];
      }
      gm[l] += gml;
    }
  }
}

}  // namespace abasim
