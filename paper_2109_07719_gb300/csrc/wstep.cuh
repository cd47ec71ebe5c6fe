// The ABA step and its adjoint for trees of revolute joints, written in
// world-aligned link frames: link i's spatial quantities are expressed in a
// frame with the world's orientation whose origin is joint i.
//
// The Articulated Body Algorithm holds in any choice of link frames (Sec. 3.1
// takes Featherstone's recursions as given; they only need the transforms
// between neighbouring frames and each joint's motion subspace in its link's
// frame).  Here the transform from a parent's frame to its child's is a pure
// translation by d = R_p r (r: the joint origin in parent coordinates, R_p: the
// parent's orientation), X = (1, d), and the joint's motion subspace is
// S = [s; 0] with s the joint axis in world coordinates (the third column of the
// link's orientation R, since every revolute link turns about its own z axis).
// The price is a rotation of each body's inertia into world axes; the gain is
// that the inward recursion on the articulated inertias (the serial chain of the
// step, Fig. 1) shifts by d instead of rotating and shifting, and the rotation
// moves out of that chain into per-link work.  Same results as the link-frame
// step up to rounding; the adjoint below is derived for this formulation with
// the same operator rules (Eq. 6 and the supplement's, in the standard
// dPhi/dE convention) and is checked against central differences.
//
// Forward step, per link l with parent p (p = -1: the world, R_p = 1):
//   E   = R(e_z, q)^T E_tree                 (parent -> link coordinates)
//   R   = R_p E^T,  d = R_p r_tree,  s = R e_z
//   v   = [v_p.w + s qd; v_p.v - d x v_p.w]  (root: [s qd; 0])
//   c   = v x [s qd; 0]
//   I^W = [R A_j R^T, skew(m R com); -skew(m R com), m 1]
//         with A_j = I_com + m (|com|^2 1 - com com^T) (inertia about the joint)
//   p^A = v x* (I^W v)
//   inward: I^A = I^W + sum_c shift(I^a_c, d_c), p^A += sum_c [p^a_c.w + d_c x p^a_c.v; p^a_c.v]
//           U = I^A S = [A s; B^T s], D = s.U_w, u = tau - b qd - s.p^A_w
//           I^a = I^A - U U^T / D,  p^a = p^A + I^a c + U u / D
//   outward: a' = [a_p.w; a_p.v - d x a_p.w] + c   (a_world = [0; -g])
//            qdd = (u - U.a') / D,  a = a' + [s qdd; 0]
// shift(I, d) = X^T I X with X = (1, d): the congruence by a pure translation.
//
// Tree data flow.  Links are numbered in depth-first preorder, so a link's first
// child is link l + 1 and its values pass to it in registers; the values a link
// with several children hands to its later children (outward passes), or collects
// from them (leaves -> root passes), live on a per-system stack whose depth is the
// nesting of branchings, not the link count: a branching link pushes, its later
// children read (or add to) the top, and its last child pops (mirrored in the
// passes that run leaves -> root).  No pass reads another link's tape words.
#pragma once

#include "aba_step.cuh"

namespace abasim {

// Per-link tape of the world-aligned step, [link][field][lane]: orientation R,
// velocity v, velocity-product term c, U, 1/D (hi/lo pair), u, the articulated
// inertia I^a = I^A - U U^T / D handed to the parent, p^a's linear and p^A's
// angular part (what the adjoint reads of the bias forces), a' and qdd, the
// joint's sin/cos, the joint offset d and the joint rate qd (so that the adjoint
// reads every per-link value from its own tape words and recomputes none of the
// articulated quantities).
enum : int {
  W_R = 0, W_V = 9, W_C = 15, W_U = 21, W_DI = 27, W_u = 29, W_IA = 30, W_PA = 51, W_AP = 57, W_QDD = 63,
  W_SC = 64, W_D = 66, W_QD = 69, NWT = 70
};
// Per-link adjoint record, [link][field][lane]: from the acceleration pass's
// adjoint, the adjoints of U, D, u and c; the adjoints of s and d (completed by
// the later passes).  The inward adjoint pass leaves each link's v and R adjoints
// in its (by then dead) tape words W_IA..W_IA+14.
enum : int { WA_U = 0, WA_D = 6, WA_u = 7, WA_C = 8, WA_S = 14, WA_DD = 17, NWA = 20 };
// One entry of the stack of parent values, [entry][field][lane]: (R, v) or a in
// the outward passes, (shift(I^a, d), p^a) in the inward one; in the adjoint the
// adjoints of a, (I^A, p^A) and (v, R).
constexpr int WSW = 27;
// model constants a world-aligned kernel reads: fields [0, NPRM_W) of the
// link's record (E_tree, r_tree, the axis slot, mass, COM, I_com, damping)
constexpr int NPRM_W = P_DAMP + 1;

// View of one system for the world-aligned step (pointers at this system's lane).
template <class T> struct WSys {
  const T* prm;     // [maxL][pstride][LANES]
  const int* meta;  // [maxL][LANES] ints, mstride apart
  T* tape;          // [maxL][NWT][LANES]
  T* adj;           // [maxL][NWA][LANES]
  int nl;
  int mstride = 1;
  int pstride = NPRM;
  int pf = 0;  // prm, meta, tape and adj in global memory: prefetch this many links ahead (0: none)
  T* stk = nullptr;  // [entry][WSW][LANES]: the stack of parent values (see the tree data flow above)
  SD T P(int l, int f) const { return prm[(l * pstride + f) * LANES]; }
  SD int M(int l) const { return meta[l * LANES * mstride]; }
  SD T& tp(int l, int f) const { return tape[(l * NWT + f) * LANES]; }
  SD T& ad(int l, int f) const { return adj[(l * NWA + f) * LANES]; }
};

// Prefetch into L1 of the cache lines holding fields [f0, f0 + n) of link l of a
// [link][stride][LANES] global array (a warp's 32 lanes share each line).  The
// passes run one thread per system through its links in a fixed order and
// touch the same fields of every link, so they ask for link l +- pf's lines while
// link l computes (pf from sim_set_prefetch, 2 by default): with a global tape, a
// warp then waits for memory once per pass instead of once per link.
SD void pf_line(const void* p) {
#ifdef __CUDA_ARCH__
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
#endif
}
template <class T> SD void pf_fields(const T* base, int stride, int l, int f0, int n) {
  for (int i = 0; i < n; ++i) pf_line(base + (l * stride + f0 + i) * LANES);
}
template <class T> SD void pf_meta(const WSys<T>& s, int l) { pf_line(s.meta + l * LANES * s.mstride); }

template <class T> SD V3<T> wv3(T* base, int stride, int l, int f) {
  const T* p = base + (l * stride + f) * LANES;
  return {p[0], p[LANES], p[2 * LANES]};
}
template <class T> SD void wv3(T* base, int stride, int l, int f, V3<T> v) {
  T* p = base + (l * stride + f) * LANES;
  p[0] = v.x; p[LANES] = v.y; p[2 * LANES] = v.z;
}
template <class T> SD SV<T> wsv(T* base, int stride, int l, int f) {
  return {wv3(base, stride, l, f), wv3(base, stride, l, f + 3)};
}
template <class T> SD void wsv(T* base, int stride, int l, int f, SV<T> v) {
  wv3(base, stride, l, f, v.w);
  wv3(base, stride, l, f + 3, v.v);
}
template <class T> SD M3<T> wm3(T* base, int stride, int l, int f) {
  M3<T> m;
  const T* p = base + (l * stride + f) * LANES;
  for (int i = 0; i < 9; ++i) m.a[i] = p[i * LANES];
  return m;
}
template <class T> SD void wm3(T* base, int stride, int l, int f, const M3<T>& m) {
  T* p = base + (l * stride + f) * LANES;
  for (int i = 0; i < 9; ++i) p[i * LANES] = m.a[i];
}
template <class T> SD S3<T> ws3(T* base, int stride, int l, int f) {
  const T* p = base + (l * stride + f) * LANES;
  return {p[0], p[LANES], p[2 * LANES], p[3 * LANES], p[4 * LANES], p[5 * LANES]};
}
template <class T> SD void ws3(T* base, int stride, int l, int f, const S3<T>& v) {
  T* p = base + (l * stride + f) * LANES;
  p[0] = v.xx; p[LANES] = v.yy; p[2 * LANES] = v.zz; p[3 * LANES] = v.xy; p[4 * LANES] = v.xz; p[5 * LANES] = v.yz;
}
template <class T> SD SI<T> wsi(T* base, int stride, int l, int f) {
  return {ws3(base, stride, l, f), wm3(base, stride, l, f + 6), ws3(base, stride, l, f + 15)};
}
template <class T> SD void wsi(T* base, int stride, int l, int f, const SI<T>& v) {
  ws3(base, stride, l, f, v.A);
  wm3(base, stride, l, f + 6, v.B);
  ws3(base, stride, l, f + 15, v.C);
}

// ------------------------------------------------------------------ operators
// third column of a rotation (the joint axis of a link turning about its z axis)
template <class T> SD V3<T> col2(const M3<T>& R) { return {R.a[2], R.a[5], R.a[8]}; }
// R S R^T for symmetric S
template <class T> SD S3<T> rot_sym(const M3<T>& R, const S3<T>& S) {
  const M3<T> F = full(S);
  M3<T> RS;  // R S
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      RS.a[3 * i + j] = R.a[3 * i] * F.a[j] + R.a[3 * i + 1] * F.a[3 + j] + R.a[3 * i + 2] * F.a[6 + j];
  auto e = [&](int i, int j) {
    return RS.a[3 * i] * R.a[3 * j] + RS.a[3 * i + 1] * R.a[3 * j + 1] + RS.a[3 * i + 2] * R.a[3 * j + 2];
  };
  return S3<T>{e(0, 0), e(1, 1), e(2, 2), e(0, 1), e(0, 2), e(1, 2)};
}
// rows of M crossed with d: M skew(d)
template <class T> SD M3<T> mskew(const M3<T>& M, V3<T> d) {
  M3<T> o;
  for (int i = 0; i < 3; ++i) {
    const V3<T> r = cross(V3<T>{M.a[3 * i], M.a[3 * i + 1], M.a[3 * i + 2]}, d);
    o.a[3 * i] = r.x; o.a[3 * i + 1] = r.y; o.a[3 * i + 2] = r.z;
  }
  return o;
}
// skew(d) M: columns of M crossed by d
template <class T> SD M3<T> skewm(V3<T> d, const M3<T>& M) {
  M3<T> o;
  for (int j = 0; j < 3; ++j) {
    const V3<T> c = cross(d, V3<T>{M.a[j], M.a[3 + j], M.a[6 + j]});
    o.a[j] = c.x; o.a[3 + j] = c.y; o.a[6 + j] = c.z;
  }
  return o;
}
// shift(I, d) = X^T I X, X = (1, d): Y_A = A - B K - (B K)^T - K C K, Y_B = B + K C,
// Y_C = C with K = skew(d)
template <class T> SD SI<T> shift(const SI<T>& I, V3<T> d) {
  const M3<T> BK = mskew(I.B, d);
  const M3<T> KC = skewm(d, full(I.C));
  const M3<T> KCK = mskew(KC, d);
  S3<T> A;
  A.xx = I.A.xx - T(2) * BK.a[0] - KCK.a[0];
  A.yy = I.A.yy - T(2) * BK.a[4] - KCK.a[4];
  A.zz = I.A.zz - T(2) * BK.a[8] - KCK.a[8];
  A.xy = I.A.xy - BK.a[1] - BK.a[3] - KCK.a[1];
  A.xz = I.A.xz - BK.a[2] - BK.a[6] - KCK.a[2];
  A.yz = I.A.yz - BK.a[5] - BK.a[7] - KCK.a[5];
  return SI<T>{A, I.B + KC, I.C};
}
// adjoint of Y = shift(I, d): given Ybar (symmetric), accumulate Ibar and dbar.
// Ibar += T Ybar T^T with T = [1 0; -K 1]; dbar from <Ybar, dY/dK>.
template <class T> SD void shift_adj(const SI<T>& I, V3<T> d, const SI<T>& Yb, SI<T>& Ib, V3<T>& db) {
  const M3<T> YbA = full(Yb.A);
  const M3<T> KYB = skewm(d, Yb.B);
  const M3<T> KYAK = mskew(skewm(d, YbA), d);
  Ib.A += Yb.A;
  Ib.B += mskew(YbA, d) + Yb.B;
  Ib.C.xx += Yb.C.xx - T(2) * KYB.a[0] - KYAK.a[0];
  Ib.C.yy += Yb.C.yy - T(2) * KYB.a[4] - KYAK.a[4];
  Ib.C.zz += Yb.C.zz - T(2) * KYB.a[8] - KYAK.a[8];
  Ib.C.xy += Yb.C.xy - KYB.a[1] - KYB.a[3] - KYAK.a[1];
  Ib.C.xz += Yb.C.xz - KYB.a[2] - KYB.a[6] - KYAK.a[2];
  Ib.C.yz += Yb.C.yz - KYB.a[5] - KYB.a[7] - KYAK.a[5];
  // dPhi/dK = -2 [ (B^T - C K) Ybar_A + C Ybar_B^T ]  (K = skew(d))
  const M3<T> FC = full(I.C);
  const M3<T> G = mm(transpose(I.B) - mm(FC, skew(d)), YbA) + mmT(FC, Yb.B);
  db -= T(2) * unskew_grad(G);
}
template <class T> SD T trace(const M3<T>& m) { return m.a[0] + m.a[4] + m.a[8]; }

// inertia of body l about its joint in link coordinates: A_j and m com
template <class T> SD S3<T> body_A(T m, V3<T> c, const S3<T>& Ic) {
  S3<T> A = Ic;
  const T cc = dot(c, c);
  A.xx += m * (cc - c.x * c.x); A.yy += m * (cc - c.y * c.y); A.zz += m * (cc - c.z * c.z);
  A.xy -= m * c.x * c.y; A.xz -= m * c.x * c.z; A.yz -= m * c.y * c.z;
  return A;
}
// I^W v for I^W = [AW, skew(g); -skew(g), m 1]
template <class T> SD SV<T> mul_iw(const S3<T>& AW, V3<T> g, T m, SV<T> v) {
  return {mul(AW, v.w) + cross(g, v.v), cross(v.w, g) + m * v.v};
}

// ------------------------------------------------------------------ forward
// One step for the state (q, qd) and joint force tau.  ADJ: also store what the
// adjoint reads (I^A, p^A, a', qdd, sin/cos).  INTEG: integrate into (qo, qdo) in
// the acceleration pass (they may alias q, qd: a link's own coordinates are read
// before they are written, and no pass after it reads the state).
template <class T, class DT, bool ADJ, bool INTEG>
SD void wstep_forward(const WSys<T>& s, Col<const T> q, Col<const T> qd, Col<const T> tau, V3<T> grav, T dt,
                      int integ, Col<T> qo, Col<T> qdo) {
  T* tp = s.tape;
  const int nl = s.nl;
  // outward: orientation, joint offset, axis, velocity (a root takes R_p = 1,
  // v_p = 0, which gives its values exactly)
  struct OwnOut {
    M3<T> E;
    V3<T> r;
    T sn, cs, vl;
    int m;
  };
  auto joint_terms = [&](int l) -> OwnOut {
    const int m = s.M(l);
    T sn, cs;
    sincos_t(q[meta_qoff(m)], &sn, &cs);
    M3<T> Et;
    for (int i = 0; i < 9; ++i) Et.a[i] = s.P(l, P_E + i);
    return OwnOut{rotz_T_mm(sn, cs, Et), V3<T>{s.P(l, P_R), s.P(l, P_R + 1), s.P(l, P_R + 2)}, sn, cs,
                  qd[meta_voff(m)], m};
  };
  M3<T> R_prev = eye3<T>();
  SV<T> v_prev = zeroSV<T>();
  int sp = 0;  // entries on the stack
  auto chain_step = [&](int l, const OwnOut& o, M3<T> Rp, SV<T> vp) {
    const int par = meta_parent(o.m);
    if (par < 0) {
      Rp = eye3<T>();
      vp = zeroSV<T>();
    }
    const V3<T> d = mul(Rp, o.r);
    const M3<T> R = mmT(Rp, o.E);
    const SV<T> v{vp.w + o.vl * col2(R), vp.v - cross(d, vp.w)};
    wv3(tp, NWT, l, W_D, d);
    wm3(tp, NWT, l, W_R, R);
    wsv(tp, NWT, l, W_V, v);
    if (ADJ) {
      s.tp(l, W_SC) = o.sn;
      s.tp(l, W_SC + 1) = o.cs;
      s.tp(l, W_QD) = o.vl;
    }
    if (meta_treechild(o.m)) {
      wm3(s.stk, WSW, sp, 0, R);
      wsv(s.stk, WSW, sp, 9, v);
      ++sp;
    }
    R_prev = R;
    v_prev = v;
  };
  {
    for (int l = 0; l < nl; ++l) {
      if (s.pf > 0 && l + s.pf < nl) {
        pf_meta(s, l + s.pf);
        pf_fields(s.prm, s.pstride, l + s.pf, P_E, 12);
      }
      const OwnOut cur = joint_terms(l);
      const int par = meta_parent(cur.m);
      M3<T> Rp = R_prev;
      SV<T> vp = v_prev;
      if (par >= 0 && par != l - 1) {
        Rp = wm3(s.stk, WSW, sp - 1, 0);
        vp = wsv(s.stk, WSW, sp - 1, 9);
        if (meta_lastsib(cur.m)) --sp;
      }
      chain_step(l, cur, Rp, vp);
    }
  }
  // inward: articulated inertias and bias forces, from each link's own terms (its
  // inertia in world axes, velocity-product and bias terms) and its children's
  // contributions
  struct Own {
    SI<T> IA;
    SV<T> pA, c;
    V3<T> sx;
    T tl;
    int m;
  };
  auto own_terms = [&](int l) -> Own {
    const int m = s.M(l);
    const int vo = meta_voff(m);
    const M3<T> R = wm3(tp, NWT, l, W_R);
    const SV<T> v = wsv(tp, NWT, l, W_V);
    const V3<T> sx = col2(R);
    const T vl = qd[vo];
    const T tl = tau[vo] - s.P(l, P_DAMP) * vl;
    const V3<T> sq = vl * sx;
    const SV<T> c{cross(v.w, sq), cross(v.v, sq)};
    const T mass = s.P(l, P_M);
    const V3<T> com{s.P(l, P_C), s.P(l, P_C + 1), s.P(l, P_C + 2)};
    const S3<T> Ic{s.P(l, P_IC), s.P(l, P_IC + 1), s.P(l, P_IC + 2), s.P(l, P_IC + 3), s.P(l, P_IC + 4),
                   s.P(l, P_IC + 5)};
    const S3<T> AW = rot_sym(R, body_A(mass, com, Ic));
    const V3<T> g = mass * mul(R, com);
    const SV<T> pA = crossf(v, mul_iw(AW, g, mass, v));
    return Own{SI<T>{AW, skew(g), S3<T>{mass, mass, mass, T(0), T(0), T(0)}}, pA, c, sx, tl, m};
  };
  SI<T> cI = zeroSI<T>();  // link l + 1's contribution when l is its parent
  SV<T> cp = zeroSV<T>();
  bool carry = false;
  // the recursion step of link l from its own terms o, to which its children's
  // contributions have been added
  auto recursion = [&](int l, const Own& o) {
    const int m = o.m;
    const int par = meta_parent(m);
    const V3<T> sx = o.sx;
    const SI<T>& IA = o.IA;
    const SV<T>& pA = o.pA;
    const SV<T> U{mul(IA.A, sx), mulT(IA.B, sx)};
    const DT Di = DT(1) / (DT)dot(sx, U.w);
    const T u = o.tl - dot(sx, pA.w);
    wsv(tp, NWT, l, W_U, U);
    {
      const T hi = (T)Di;
      s.tp(l, W_DI) = hi;
      s.tp(l, W_DI + 1) = (T)(Di - (DT)hi);
    }
    s.tp(l, W_u) = u;
    wsv(tp, NWT, l, W_C, o.c);
    // the contribution to the parent (computed for a root too, with d = 0, and dropped)
    V3<T> d = wv3(tp, NWT, l, W_D);
    if (par < 0) d = zero3<T>();
    const SI<T> Ia = minus_scaled_outer<T, DT>(IA, Di, U);
    const SV<T> pa = pA + mul(Ia, o.c) + (T)((DT)u * Di) * U;
    if (ADJ) {  // what the adjoint reads of them: I^a, p^a's linear part and p^A's angular part
      wsi(tp, NWT, l, W_IA, Ia);
      wv3(tp, NWT, l, W_PA, pa.v);
      wv3(tp, NWT, l, W_PA + 3, pA.w);
    }
    const SI<T> Y = shift(Ia, d);
    const SV<T> pn{pa.w + cross(d, pa.v), pa.v};
    carry = par == l - 1 && par >= 0;
    if (carry) {
      cI = Y;
      cp = pn;
    } else if (par >= 0 && meta_lastsib(m)) {
      wsi(s.stk, WSW, sp, 0, Y);
      wsv(s.stk, WSW, sp, 21, pn);
      ++sp;
    } else if (par >= 0) {
      wsi(s.stk, WSW, sp - 1, 0, wsi(s.stk, WSW, sp - 1, 0) + Y);
      wsv(s.stk, WSW, sp - 1, 21, wsv(s.stk, WSW, sp - 1, 21) + pn);
    }
  };
  {
    for (int l = nl - 1; l >= 0; --l) {
      if (s.pf > 0 && l - s.pf >= 0) {
        pf_fields(tp, NWT, l - s.pf, W_R, 15);
        pf_fields(tp, NWT, l - s.pf, W_D, 3);
        pf_fields(s.prm, s.pstride, l - s.pf, P_M, NPRM_W - P_M);
      }
      Own cur = own_terms(l);
      if (carry) {
        cur.IA += cI;
        cur.pA += cp;
      }
      if (meta_treechild(cur.m)) {
        --sp;
        cur.IA += wsi(s.stk, WSW, sp, 0);
        cur.pA += wsv(s.stk, WSW, sp, 21);
      }
      recursion(l, cur);
    }
  }
  // outward: accelerations (and the integrator)
  const SV<T> a0{zero3<T>(), -grav};
  SV<T> a_prev = a0;
  for (int l = 0; l < nl; ++l) {
    if (s.pf > 0 && l + s.pf < nl) {
      pf_fields(tp, NWT, l + s.pf, W_R, 9);
      pf_fields(tp, NWT, l + s.pf, W_C, W_IA - W_C);
      pf_fields(tp, NWT, l + s.pf, W_D, 3);
    }
    const int m = s.M(l);
    const int par = meta_parent(m);
    const M3<T> R = wm3(tp, NWT, l, W_R);
    const SV<T> c = wsv(tp, NWT, l, W_C);
    const SV<T> U = wsv(tp, NWT, l, W_U);
    const DT Di = (DT)s.tp(l, W_DI) + (DT)s.tp(l, W_DI + 1);
    const T u = s.tp(l, W_u);
    SV<T> ap;
    if (par < 0) {
      ap = a0 + c;
    } else {
      SV<T> apar = a_prev;
      if (par != l - 1) {
        apar = wsv(s.stk, WSW, sp - 1, 0);
        if (meta_lastsib(m)) --sp;
      }
      const V3<T> d = wv3(tp, NWT, l, W_D);
      ap = SV<T>{apar.w + c.w, apar.v - cross(d, apar.w) + c.v};
    }
    const T qdd = (T)(((DT)u - (DT)dot(U, ap)) * Di);
    const SV<T> a{ap.w + qdd * col2(R), ap.v};
    if (ADJ) {
      wsv(tp, NWT, l, W_AP, ap);
      s.tp(l, W_QDD) = qdd;
    }
    if (meta_treechild(m)) {
      wsv(s.stk, WSW, sp, 0, a);
      ++sp;
    }
    if (INTEG) {
      const int qi = meta_qoff(m), vi = meta_voff(m);
      const T v0 = qd[vi];
      const T v1 = v0 + dt * qdd;
      const T q1 = q[qi] + dt * (integ == I_SEMI_IMPLICIT ? v1 : v0);
      qdo[vi] = v1;
      qo[qi] = q1;
    }
    a_prev = a;
  }
}

// ------------------------------------------------------------------ adjoint
// Requires wstep_forward<ADJ = true>(q, qd, tau) to have filled the tape.  On entry
// (gq, gqd) hold the adjoint of x^{k+1}; on exit that of x^k.  Writes the adjoint
// of tau into gtau and adds dPhi/dm of every link into gm.  Three passes: the
// integrator and acceleration adjoint (leaves -> root), the articulated-inertia
// adjoint with the per-link inertia and velocity-product adjoints (root -> leaves),
// the velocity and orientation adjoint and the joint angles' (leaves -> root).
template <class T, class DT, bool ILP = false>
SD void wstep_adjoint(const WSys<T>& s, Col<T> gq, Col<T> gqd, Col<T> gtau,
                      Col<T> gm, T dt, int integ) {
  T* tp = s.tape;
  T* ad = s.adj;
  const int nl = s.nl;
  const T half = T(0.5);
  // integrator + acceleration pass adjoint (leaves -> root)
  {
    SV<T> cab = zeroSV<T>();
    bool carry = false;
    int sp = 0;
    for (int l = nl - 1; l >= 0; --l) {
      if (s.pf > 0 && l - s.pf >= 0) {
        pf_fields(tp, NWT, l - s.pf, W_R, 9);
        pf_fields(tp, NWT, l - s.pf, W_C, 3);
        pf_fields(tp, NWT, l - s.pf, W_U, W_u - W_U);
        pf_fields(tp, NWT, l - s.pf, W_AP, W_SC - W_AP);
        pf_fields(tp, NWT, l - s.pf, W_D, 3);
      }
      const int m = s.M(l);
      const int par = meta_parent(m), qi = meta_qoff(m), vi = meta_voff(m);
      T qddb;
      {
        const T qb = gq[qi], vb = gqd[vi];
        if (integ == I_SEMI_IMPLICIT) {
          const T vt = vb + dt * qb;
          gqd[vi] = vt;
          qddb = dt * vt;
        } else {
          gqd[vi] = vb + dt * qb;
          qddb = dt * vb;
        }
      }
      SV<T> ab = carry ? cab : zeroSV<T>();
      carry = false;
      if (meta_treechild(m)) {
        --sp;
        ab += wsv(s.stk, WSW, sp, 0);
      }
      const V3<T> sx = col2(wm3(tp, NWT, l, W_R));
      const T qdd = s.tp(l, W_QDD);
      const SV<T> ap = wsv(tp, NWT, l, W_AP);
      const SV<T> U = wsv(tp, NWT, l, W_U);
      const DT Di = (DT)s.tp(l, W_DI) + (DT)s.tp(l, W_DI + 1);
      const T qb_tot = qddb + dot(sx, ab.w);
      const T wb = (T)((DT)qb_tot * Di);
      const SV<T> apb = ab - wb * U;
      wsv(ad, NWA, l, WA_U, zeroSV<T>() - wb * ap);
      s.ad(l, WA_D) = -wb * qdd;
      s.ad(l, WA_u) = wb;
      wsv(ad, NWA, l, WA_C, apb);
      wv3(ad, NWA, l, WA_S, qdd * ab.w);
      V3<T> db = zero3<T>();
      if (par >= 0) {
        const V3<T> d = wv3(tp, NWT, l, W_D);
        const V3<T> apw = ap.w - wv3(tp, NWT, l, W_C);  // the parent's angular acceleration: a'.w = a_p.w + c.w
        const SV<T> aparb{apb.w + cross(d, apb.v), apb.v};
        db = cross(apb.v, apw);
        if (par == l - 1) {
          cab = aparb;
          carry = true;
        } else if (meta_lastsib(m)) {
          wsv(s.stk, WSW, sp, 0, aparb);
          ++sp;
        } else {
          wsv(s.stk, WSW, sp - 1, 0, wsv(s.stk, WSW, sp - 1, 0) + aparb);
        }
      }
      wv3(ad, NWA, l, WA_DD, db);
    }
  }
  // articulated-inertia adjoint (root -> leaves) with each link's inertia,
  // bias-force and velocity-product adjoints.  Each link's work has a part on the
  // chain (from its parent's adjoints of I^A and p^A to its own, which its children
  // need) and a per-link part that nothing downstream in this pass waits for; with
  // ILP the loop runs link l's chain part beside link l - 1's per-link part, so
  // that one thread has two independent instruction streams (the same arithmetic
  // in the same order per link as running the two parts back to back).  It pays
  // where the tape is in global memory and the registers suffice (FP32 storage);
  // on chip the longer code costs more in instruction fetch than it gains.
  {
    SI<T> cIAb = zeroSI<T>();
    SV<T> cpAb = zeroSV<T>();
    int sp = 0;
    struct Chain {  // a link's state between its two parts
      SI<T> IAb;
      SV<T> pAb, cb, v;
      V3<T> sb, db;
      M3<T> R;
      int vi;
      bool tc;
    };
    auto chain_part = [&](int l) -> Chain {
      if (s.pf > 0 && l + s.pf < nl) {
        pf_fields(tp, NWT, l + s.pf, W_R, W_AP - W_R);
        pf_fields(tp, NWT, l + s.pf, W_D, 4);
        pf_fields(ad, NWA, l + s.pf, WA_U, NWA - WA_U);
        pf_fields(s.prm, s.pstride, l + s.pf, P_M, NPRM_W - P_M);
      }
      const int m = s.M(l);
      const int par = meta_parent(m), vi = meta_voff(m);
      const SI<T> Ia = wsi(tp, NWT, l, W_IA);
      const V3<T> pav = wv3(tp, NWT, l, W_PA), pAw = wv3(tp, NWT, l, W_PA + 3);
      const SV<T> U = wsv(tp, NWT, l, W_U);
      const DT Di = (DT)s.tp(l, W_DI) + (DT)s.tp(l, W_DI + 1);
      const T u = s.tp(l, W_u);
      const SV<T> c = wsv(tp, NWT, l, W_C);
      const M3<T> R = wm3(tp, NWT, l, W_R);
      const SV<T> v = wsv(tp, NWT, l, W_V);
      const V3<T> sx = col2(R);
      SV<T> Ub = wsv(ad, NWA, l, WA_U);
      T Db = s.ad(l, WA_D);
      T ub = s.ad(l, WA_u);
      SV<T> cb = wsv(ad, NWA, l, WA_C);
      V3<T> sb = wv3(ad, NWA, l, WA_S);
      V3<T> db = wv3(ad, NWA, l, WA_DD);
      // the parent's adjoints (zero for a root, whose terms below then add zeros)
      SI<T> IAbp = cIAb;
      SV<T> pAbp = cpAb;
      if (par >= 0 && par != l - 1) {
        IAbp = wsi(s.stk, WSW, sp - 1, 0);
        pAbp = wsv(s.stk, WSW, sp - 1, 21);
        if (meta_lastsib(m)) --sp;
      }
      V3<T> d = wv3(tp, NWT, l, W_D);
      if (par < 0) {
        IAbp = zeroSI<T>();
        pAbp = zeroSV<T>();
        d = zero3<T>();
      }
      SI<T> Iab = zeroSI<T>();
      shift_adj(Ia, d, IAbp, Iab, db);
      const SV<T> pab{pAbp.w, pAbp.v + cross(pAbp.w, d)};
      db += cross(pav, pAbp.w);
      // p^a = p^A + I^a c + U u / D
      SV<T> pAb = pab;
      Iab += sym_outer(pab, c);
      cb += mul(Ia, pab);
      Ub += (T)((DT)u * Di) * pab;
      const T gb = dot(U, pab);
      ub += (T)((DT)gb * Di);
      Db -= (T)((DT)gb * (DT)u * Di * Di);
      // I^a = I^A - U U^T / D
      SI<T> IAb = Iab;
      const SV<T> IbU = mul(Iab, U);
      Ub -= (T)(DT(2) * Di) * IbU;
      Db += (T)(Di * Di * (DT)dot(U, IbU));
      // u = tau - b qd - s.p^A_w,  D = s.U_w,  U = [A s; B^T s]
      gtau[vi] = ub;
      gqd[vi] -= s.P(l, P_DAMP) * ub;
      sb -= ub * pAw;
      pAb.w -= ub * sx;
      sb += Db * U.w;
      Ub.w += Db * sx;
      IAb.A += sym_outer(Ub.w, sx);
      IAb.B += scale(half, outer(sx, Ub.v));
      // the top rows of I^A Ub, with I^A = I^a + U U^T / D
      sb += mul(Ia.A, Ub.w) + mul(Ia.B, Ub.v) + (T)(Di * (DT)dot(U, Ub)) * U.w;
      cIAb = IAb;
      cpAb = pAb;
      return Chain{IAb, pAb, cb, v, sb, db, R, vi, meta_treechild(m)};
    };
    auto push = [&](const Chain& k) {  // hand a branching link's adjoints to its later children
      if (k.tc) {
        wsi(s.stk, WSW, sp, 0, k.IAb);
        wsv(s.stk, WSW, sp, 21, k.pAb);
        ++sp;
      }
    };
    auto per_link_part = [&](int l, const Chain& k) {
      SV<T> cb = k.cb;
      V3<T> sb = k.sb;
      const M3<T>& R = k.R;
      const SV<T>& v = k.v;
      const V3<T> sx = col2(R);
      // p^A0 = v x* h, h = I^W v: I^W enters I^A additively, p^A0 enters p^A
      const T mass = s.P(l, P_M);
      const V3<T> com{s.P(l, P_C), s.P(l, P_C + 1), s.P(l, P_C + 2)};
      const S3<T> Ic{s.P(l, P_IC), s.P(l, P_IC + 1), s.P(l, P_IC + 2), s.P(l, P_IC + 3), s.P(l, P_IC + 4),
                     s.P(l, P_IC + 5)};
      const S3<T> Aj = body_A(mass, com, Ic);
      const S3<T> AW = rot_sym(R, Aj);
      const V3<T> rw = mul(R, com);
      const V3<T> g = mass * rw;
      const SV<T> h = mul_iw(AW, g, mass, v);
      SV<T> vb = zeroSV<T>(), hb = zeroSV<T>();
      crossf_adj(v, h, k.pAb, vb, hb);
      SI<T> IWb = k.IAb;
      IWb += sym_outer(hb, v);
      vb += mul_iw(AW, g, mass, hb);
      const V3<T> gb = T(2) * unskew_grad(IWb.B);
      const M3<T> AWb = full(IWb.A);
      // A^W = R A_j R^T, g = m R com
      M3<T> Rb = scale(T(2), mm(mm(AWb, R), full(Aj)));
      Rb += outer(gb, mass * com);
      T mb = IWb.C.xx + IWb.C.yy + IWb.C.zz;
      mb += dot(com, com) * trace(AWb) - dot(rw, mul(AWb, rw)) + dot(rw, gb);
      gm[l] += mb;
      // c = [v_w x s qd; v_v x s qd]
      const T vl = s.tp(l, W_QD);
      const V3<T> sq = vl * sx;
      vb.w += cross(sq, cb.w);
      vb.v += cross(sq, cb.v);
      const V3<T> sqb = cross(cb.w, v.w) + cross(cb.v, v.v);
      sb += vl * sqb;
      gqd[k.vi] += dot(sx, sqb);
      wv3(ad, NWA, l, WA_S, sb);
      wv3(ad, NWA, l, WA_DD, k.db);
      wsv(tp, NWT, l, W_IA, vb);  // the tape's I^A words are dead from here on
      wm3(tp, NWT, l, W_IA + 6, Rb);
    };
    if (!ILP) {
      for (int l = 0; l < nl; ++l) {
        const Chain k = chain_part(l);
        push(k);
        per_link_part(l, k);
      }
    } else if (nl > 0) {
      Chain prev = chain_part(0);
      push(prev);
      for (int l = 1; l < nl; ++l) {
        const Chain cur = chain_part(l);
        per_link_part(l - 1, prev);
        push(cur);
        prev = cur;
      }
      per_link_part(nl - 1, prev);
    }
  }
  // velocity, orientation and joint-angle adjoint (leaves -> root)
  {
    SV<T> cvb = zeroSV<T>();
    M3<T> cRb = zeroM3<T>();
    bool carry = false;
    int sp = 0;
    for (int l = nl - 1; l >= 0; --l) {
      if (s.pf > 0 && l - s.pf >= 0) {
        pf_fields(tp, NWT, l - s.pf, W_R, 15);
        pf_fields(tp, NWT, l - s.pf, W_IA, 15);
        pf_fields(tp, NWT, l - s.pf, W_SC, 6);
        pf_fields(ad, NWA, l - s.pf, WA_S, 6);
        pf_fields(s.prm, s.pstride, l - s.pf, P_E, 12);
      }
      const int m = s.M(l);
      const int par = meta_parent(m), qi = meta_qoff(m), vi = meta_voff(m);
      SV<T> vb = wsv(tp, NWT, l, W_IA);
      M3<T> Rb = wm3(tp, NWT, l, W_IA + 6);
      V3<T> sb = wv3(ad, NWA, l, WA_S);
      V3<T> db = wv3(ad, NWA, l, WA_DD);
      if (carry) {
        vb += cvb;
        Rb += cRb;
      }
      carry = false;
      if (meta_treechild(m)) {
        --sp;
        vb += wsv(s.stk, WSW, sp, 0);
        Rb += wm3(s.stk, WSW, sp, 6);
      }
      const M3<T> R = wm3(tp, NWT, l, W_R);
      const V3<T> sx = col2(R);
      const T vl = s.tp(l, W_QD);
      // v = [v_p.w + s qd; v_p.v - d x v_p.w]
      sb += vl * vb.w;
      gqd[vi] += dot(sx, vb.w);
      // s = R e_z
      Rb.a[2] += sb.x;
      Rb.a[5] += sb.y;
      Rb.a[8] += sb.z;
      const T sn = s.tp(l, W_SC), cs = s.tp(l, W_SC + 1);
      M3<T> Et;
      for (int i = 0; i < 9; ++i) Et.a[i] = s.P(l, P_E + i);
      M3<T> Eb;
      if (par >= 0) {
        // R = R_p E^T, d = R_p r; the parent's orientation and angular velocity
        // from the link's own: R_p = R E, v_p.w = v.w - s qd
        const M3<T> E = rotz_T_mm(sn, cs, Et);
        const M3<T> Rp = mm(R, E);
        const V3<T> vpw = wv3(tp, NWT, l, W_V) - vl * sx;
        const V3<T> rt{s.P(l, P_R), s.P(l, P_R + 1), s.P(l, P_R + 2)};
        const V3<T> d = wv3(tp, NWT, l, W_D);
        const SV<T> vpb{vb.w + cross(d, vb.v), vb.v};
        db += cross(vb.v, vpw);
        M3<T> Rpb = mm(Rb, E);
        Rpb += outer(db, rt);
        Eb = mTm(Rb, Rp);
        if (par == l - 1) {
          cvb = vpb;
          cRb = Rpb;
          carry = true;
        } else if (meta_lastsib(m)) {
          wsv(s.stk, WSW, sp, 0, vpb);
          wm3(s.stk, WSW, sp, 6, Rpb);
          ++sp;
        } else {
          wsv(s.stk, WSW, sp - 1, 0, wsv(s.stk, WSW, sp - 1, 0) + vpb);
          wm3(s.stk, WSW, sp - 1, 6, wm3(s.stk, WSW, sp - 1, 6) + Rpb);
        }
      } else {
        Eb = transpose(Rb);
      }
      gq[qi] += rotz_T_dq(sn, cs, Eb, Et);
    }
  }
}

}  // namespace abasim
