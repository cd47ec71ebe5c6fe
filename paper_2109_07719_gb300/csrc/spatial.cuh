// Spatial algebra for the articulated-body kernels: 3-vectors, 3x3 matrices,
// spatial (6D) vectors, coordinate transforms (E, r) and symmetric 6x6 spatial
// inertias, with the reverse-mode adjoint of every operator the ABA step uses.
//
// Conventions (Sec. 3.1 Eq. 5 and the supplement's spatial-transform / spatial-
// motion / spatial-dyad operators):
//   spatial vector      [w; v]                       (angular first)
//   transform (E, r)    motion:  X m  = [E w; E (v - r x w)]          (st_apply)
//                       force^T: X^T f = [E^T n + r x (E^T f); E^T f] (st_apply_trans)
//   inertia congruence  X^T I X  (the supplement's shift = A^T B A of st2sd)
//   cross products      v x m  = [w x mw; w x mv + v x mw]            (sm_crossm)
//                       v x* f = [w x fn + v x ff; w x ff]            (sm_crossf, Eq. 5)
// Adjoints use the standard convention Ebar_ij = dPhi/dE_ij.  A symmetric 6x6
// [A B; B^T C] is stored as A, C (6 each: xx yy zz xy xz yz) and B (9, row
// major); its adjoint is the symmetric full-matrix gradient stored the same way,
// so  dPhi = <Abar, dA> + 2 <Bbar, dB> + <Cbar, dC>.
#pragma once

#ifdef __CUDACC__
#define SD __host__ __device__ __forceinline__
#else
#define SD inline
#endif

namespace abasim {

template <class T> struct V3 { T x, y, z; };
template <class T> struct M3 { T a[9]; };          // row major
template <class T> struct S3 { T xx, yy, zz, xy, xz, yz; };
template <class T> struct SV { V3<T> w, v; };
template <class T> struct XF { M3<T> E; V3<T> r; };
template <class T> struct SI { S3<T> A; M3<T> B; S3<T> C; };

// ------------------------------------------------------------------ 3-vectors
template <class T> SD V3<T> v3(T x, T y, T z) { return V3<T>{x, y, z}; }
template <class T> SD V3<T> zero3() { return V3<T>{T(0), T(0), T(0)}; }
template <class T> SD V3<T> operator+(V3<T> a, V3<T> b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
template <class T> SD V3<T> operator-(V3<T> a, V3<T> b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <class T> SD V3<T> operator-(V3<T> a) { return {-a.x, -a.y, -a.z}; }
template <class T> SD V3<T> operator*(T s, V3<T> a) { return {s * a.x, s * a.y, s * a.z}; }
template <class T> SD V3<T>& operator+=(V3<T>& a, V3<T> b) { a.x += b.x; a.y += b.y; a.z += b.z; return a; }
template <class T> SD V3<T>& operator-=(V3<T>& a, V3<T> b) { a.x -= b.x; a.y -= b.y; a.z -= b.z; return a; }
template <class T> SD T dot(V3<T> a, V3<T> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <class T> SD V3<T> cross(V3<T> a, V3<T> b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

// ------------------------------------------------------------------ 3x3
template <class T> SD M3<T> eye3() { return M3<T>{{T(1), 0, 0, 0, T(1), 0, 0, 0, T(1)}}; }
template <class T> SD M3<T> zeroM3() { M3<T> m; for (int i = 0; i < 9; ++i) m.a[i] = T(0); return m; }
template <class T> SD V3<T> mul(const M3<T>& m, V3<T> v) {
  return {m.a[0] * v.x + m.a[1] * v.y + m.a[2] * v.z,
          m.a[3] * v.x + m.a[4] * v.y + m.a[5] * v.z,
          m.a[6] * v.x + m.a[7] * v.y + m.a[8] * v.z};
}
template <class T> SD V3<T> mulT(const M3<T>& m, V3<T> v) {  // m^T v
  return {m.a[0] * v.x + m.a[3] * v.y + m.a[6] * v.z,
          m.a[1] * v.x + m.a[4] * v.y + m.a[7] * v.z,
          m.a[2] * v.x + m.a[5] * v.y + m.a[8] * v.z};
}
template <class T> SD M3<T> mm(const M3<T>& p, const M3<T>& q) {  // p q
  M3<T> o;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      o.a[3 * i + j] = p.a[3 * i] * q.a[j] + p.a[3 * i + 1] * q.a[3 + j] + p.a[3 * i + 2] * q.a[6 + j];
  return o;
}
template <class T> SD M3<T> mTm(const M3<T>& p, const M3<T>& q) {  // p^T q
  M3<T> o;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      o.a[3 * i + j] = p.a[i] * q.a[j] + p.a[3 + i] * q.a[3 + j] + p.a[6 + i] * q.a[6 + j];
  return o;
}
template <class T> SD M3<T> mmT(const M3<T>& p, const M3<T>& q) {  // p q^T
  M3<T> o;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      o.a[3 * i + j] = p.a[3 * i] * q.a[3 * j] + p.a[3 * i + 1] * q.a[3 * j + 1] + p.a[3 * i + 2] * q.a[3 * j + 2];
  return o;
}
template <class T> SD M3<T> transpose(const M3<T>& m) {
  return M3<T>{{m.a[0], m.a[3], m.a[6], m.a[1], m.a[4], m.a[7], m.a[2], m.a[5], m.a[8]}};
}
template <class T> SD M3<T> operator+(const M3<T>& p, const M3<T>& q) { M3<T> o; for (int i = 0; i < 9; ++i) o.a[i] = p.a[i] + q.a[i]; return o; }
template <class T> SD M3<T> operator-(const M3<T>& p, const M3<T>& q) { M3<T> o; for (int i = 0; i < 9; ++i) o.a[i] = p.a[i] - q.a[i]; return o; }
template <class T> SD M3<T>& operator+=(M3<T>& p, const M3<T>& q) { for (int i = 0; i < 9; ++i) p.a[i] += q.a[i]; return p; }
template <class T> SD M3<T> scale(T s, const M3<T>& p) { M3<T> o; for (int i = 0; i < 9; ++i) o.a[i] = s * p.a[i]; return o; }
template <class T> SD M3<T> outer(V3<T> a, V3<T> b) {  // a b^T
  return M3<T>{{a.x * b.x, a.x * b.y, a.x * b.z, a.y * b.x, a.y * b.y, a.y * b.z, a.z * b.x, a.z * b.y, a.z * b.z}};
}
template <class T> SD M3<T> skew(V3<T> v) {  // skew(a) b = a x b
  return M3<T>{{T(0), -v.z, v.y, v.z, T(0), -v.x, -v.y, v.x, T(0)}};
}
// gradient of <G, skew(r)> with respect to r
template <class T> SD V3<T> unskew_grad(const M3<T>& g) {
  return {g.a[7] - g.a[5], g.a[2] - g.a[6], g.a[3] - g.a[1]};
}
template <class T> SD T frob(const M3<T>& p, const M3<T>& q) { T s = 0; for (int i = 0; i < 9; ++i) s += p.a[i] * q.a[i]; return s; }

// symmetric 3x3
template <class T> SD M3<T> full(const S3<T>& s) {
  return M3<T>{{s.xx, s.xy, s.xz, s.xy, s.yy, s.yz, s.xz, s.yz, s.zz}};
}
template <class T> SD S3<T> symof(const M3<T>& m) {  // (m + m^T) / 2
  const T h = T(0.5);
  return S3<T>{m.a[0], m.a[4], m.a[8], h * (m.a[1] + m.a[3]), h * (m.a[2] + m.a[6]), h * (m.a[5] + m.a[7])};
}
template <class T> SD S3<T> zeroS3() { return S3<T>{0, 0, 0, 0, 0, 0}; }
template <class T> SD V3<T> mul(const S3<T>& s, V3<T> v) {
  return {s.xx * v.x + s.xy * v.y + s.xz * v.z, s.xy * v.x + s.yy * v.y + s.yz * v.z,
          s.xz * v.x + s.yz * v.y + s.zz * v.z};
}
template <class T> SD S3<T> operator+(const S3<T>& a, const S3<T>& b) { return {a.xx + b.xx, a.yy + b.yy, a.zz + b.zz, a.xy + b.xy, a.xz + b.xz, a.yz + b.yz}; }
template <class T> SD S3<T> operator-(const S3<T>& a, const S3<T>& b) { return {a.xx - b.xx, a.yy - b.yy, a.zz - b.zz, a.xy - b.xy, a.xz - b.xz, a.yz - b.yz}; }
template <class T> SD S3<T>& operator+=(S3<T>& a, const S3<T>& b) { a.xx += b.xx; a.yy += b.yy; a.zz += b.zz; a.xy += b.xy; a.xz += b.xz; a.yz += b.yz; return a; }
// <s, m> Frobenius with s expanded to a full symmetric matrix
template <class T> SD T frob(const S3<T>& s, const M3<T>& m) {
  return s.xx * m.a[0] + s.yy * m.a[4] + s.zz * m.a[8] + s.xy * (m.a[1] + m.a[3]) + s.xz * (m.a[2] + m.a[6]) + s.yz * (m.a[5] + m.a[7]);
}
template <class T> SD S3<T> sym_outer(V3<T> a, V3<T> b) {  // (a b^T + b a^T) / 2
  const T h = T(0.5);
  return {a.x * b.x, a.y * b.y, a.z * b.z, h * (a.x * b.y + a.y * b.x), h * (a.x * b.z + a.z * b.x), h * (a.y * b.z + a.z * b.y)};
}
template <class T> SD S3<T> congr(const M3<T>& E, const S3<T>& s) {  // E^T s E
  return symof(mTm(E, mm(full(s), E)));
}
template <class T> SD S3<T> congrT(const M3<T>& E, const S3<T>& s) {  // E s E^T
  return symof(mm(E, mmT(full(s), E)));
}

// ------------------------------------------------------------------ spatial vectors
template <class T> SD SV<T> zeroSV() { return SV<T>{zero3<T>(), zero3<T>()}; }
template <class T> SD SV<T> operator+(SV<T> a, SV<T> b) { return {a.w + b.w, a.v + b.v}; }
template <class T> SD SV<T> operator-(SV<T> a, SV<T> b) { return {a.w - b.w, a.v - b.v}; }
template <class T> SD SV<T> operator*(T s, SV<T> a) { return {s * a.w, s * a.v}; }
template <class T> SD SV<T>& operator+=(SV<T>& a, SV<T> b) { a.w += b.w; a.v += b.v; return a; }
template <class T> SD SV<T>& operator-=(SV<T>& a, SV<T> b) { a.w -= b.w; a.v -= b.v; return a; }
template <class T> SD T dot(SV<T> a, SV<T> b) { return dot(a.w, b.w) + dot(a.v, b.v); }

template <class T> SD SV<T> crossm(SV<T> m, SV<T> n) {  // m x n (motion)
  return {cross(m.w, n.w), cross(m.w, n.v) + cross(m.v, n.w)};
}
template <class T> SD SV<T> crossf(SV<T> m, SV<T> f) {  // m x* f (force)
  return {cross(m.w, f.w) + cross(m.v, f.v), cross(m.w, f.v)};
}
// adjoints of y = m x n:  mbar += ..., nbar += ...
template <class T> SD void crossm_adj(SV<T> m, SV<T> n, SV<T> yb, SV<T>& mb, SV<T>& nb) {
  mb.w += cross(n.w, yb.w) + cross(n.v, yb.v);
  mb.v += cross(n.w, yb.v);
  nb.w += cross(yb.w, m.w) + cross(yb.v, m.v);
  nb.v += cross(yb.v, m.w);
}
// adjoints of y = m x* f (the worked example of Sec. 3.1, Eq. 6)
template <class T> SD void crossf_adj(SV<T> m, SV<T> f, SV<T> yb, SV<T>& mb, SV<T>& fb) {
  mb.w += cross(f.w, yb.w) + cross(f.v, yb.v);
  mb.v += cross(f.v, yb.w);
  fb.w += cross(yb.w, m.w);
  fb.v += cross(yb.w, m.v) + cross(yb.v, m.w);
}

// ------------------------------------------------------------------ transforms
template <class T> SD SV<T> apply(const XF<T>& X, SV<T> m) {          // X m
  return {mul(X.E, m.w), mul(X.E, m.v - cross(X.r, m.w))};
}
template <class T> SD SV<T> applyT(const XF<T>& X, SV<T> f) {         // X^T f
  V3<T> z = mulT(X.E, f.v);
  return {mulT(X.E, f.w) + cross(X.r, z), z};
}
// y = X x: accumulate Ebar, rbar, xbar from ybar
template <class T> SD void apply_adj(const XF<T>& X, SV<T> x, SV<T> yb, M3<T>& Eb, V3<T>& rb, SV<T>* xb) {
  V3<T> t = x.v - cross(X.r, x.w);
  Eb += outer(yb.w, x.w);
  Eb += outer(yb.v, t);
  V3<T> Etyv = mulT(X.E, yb.v);
  rb += cross(Etyv, x.w);
  if (xb) {
    xb->w += mulT(X.E, yb.w) + cross(X.r, Etyv);
    xb->v += Etyv;
  }
}
// y = X^T x: accumulate Ebar, rbar, xbar from ybar
template <class T> SD void applyT_adj(const XF<T>& X, SV<T> x, SV<T> yb, M3<T>& Eb, V3<T>& rb, SV<T>* xb) {
  V3<T> zb = cross(yb.w, X.r) + yb.v;
  V3<T> z = mulT(X.E, x.v);
  Eb += outer(x.w, yb.w);
  Eb += outer(x.v, zb);
  rb += cross(z, yb.w);
  if (xb) {
    xb->w += mul(X.E, yb.w);
    xb->v += mul(X.E, zb);
  }
}
// composition X = X_J X_tree for X_J = (EJ, rJ): E = EJ Et, r = rt + Et^T rJ
template <class T> SD XF<T> compose(const M3<T>& EJ, V3<T> rJ, const M3<T>& Et, V3<T> rt) {
  return XF<T>{mm(EJ, Et), rt + mulT(Et, rJ)};
}

// ------------------------------------------------------------------ symmetric 6x6
template <class T> SD SI<T> zeroSI() { return SI<T>{zeroS3<T>(), zeroM3<T>(), zeroS3<T>()}; }
template <class T> SD SV<T> mul(const SI<T>& I, SV<T> x) {
  return {mul(I.A, x.w) + mul(I.B, x.v), mulT(I.B, x.w) + mul(I.C, x.v)};
}
template <class T> SD SI<T> operator+(const SI<T>& p, const SI<T>& q) { return {p.A + q.A, p.B + q.B, p.C + q.C}; }
template <class T> SD SI<T> operator-(const SI<T>& p, const SI<T>& q) { return {p.A - q.A, p.B - q.B, p.C - q.C}; }
template <class T> SD SI<T>& operator+=(SI<T>& p, const SI<T>& q) { p.A += q.A; p.B += q.B; p.C += q.C; return p; }
// sym(a b^T) as a symmetric 6x6 in block form
template <class T> SD SI<T> sym_outer(SV<T> a, SV<T> b) {
  const T h = T(0.5);
  return SI<T>{sym_outer(a.w, b.w), scale(h, outer(a.w, b.v) + outer(b.w, a.v)), sym_outer(a.v, b.v)};
}
template <class T> SD SI<T> scale(T s, const SI<T>& p) {
  return SI<T>{S3<T>{s * p.A.xx, s * p.A.yy, s * p.A.zz, s * p.A.xy, s * p.A.xz, s * p.A.yz}, scale(s, p.B),
               S3<T>{s * p.C.xx, s * p.C.yy, s * p.C.zz, s * p.C.xy, s * p.C.xz, s * p.C.yz}};
}
// full-matrix Frobenius product of two symmetric 6x6
template <class T> SD T frob(const SI<T>& p, const SI<T>& q) {
  return frob(p.A, full(q.A)) + T(2) * frob(p.B, q.B) + frob(p.C, full(q.C));
}

// spatial inertia of a body: [Ic + m cx cx^T, m cx; m cx^T, m 1]
template <class T> SD SI<T> rbi(T m, V3<T> c, const S3<T>& Ic) {
  S3<T> A = Ic;
  // cx cx^T = (c.c) 1 - c c^T
  T cc = dot(c, c);
  A.xx += m * (cc - c.x * c.x); A.yy += m * (cc - c.y * c.y); A.zz += m * (cc - c.z * c.z);
  A.xy -= m * c.x * c.y; A.xz -= m * c.x * c.z; A.yz -= m * c.y * c.z;
  return SI<T>{A, scale(m, skew(c)), S3<T>{m, m, m, 0, 0, 0}};
}
// <Mbar, dI/dm> for the body above with c and Ic held fixed
template <class T> SD T rbi_dmass(const SI<T>& Mb, V3<T> c) {
  T cc = dot(c, c);
  S3<T> D{cc - c.x * c.x, cc - c.y * c.y, cc - c.z * c.z, -c.x * c.y, -c.x * c.z, -c.y * c.z};
  return frob(Mb.A, full(D)) + T(2) * frob(Mb.B, skew(c)) + (Mb.C.xx + Mb.C.yy + Mb.C.zz);
}
// z^T (dI/dm) x
template <class T> SD T rbi_dmass_bilinear(SV<T> z, SV<T> x, V3<T> c) {
  return dot(cross(z.w, c), cross(x.w, c)) + dot(z.w, cross(c, x.v)) - dot(z.v, cross(c, x.w)) + dot(z.v, x.v);
}

// congruence Y = X^T I X (inertia of a child expressed in its parent's frame):
// rotate  I~ = diag(E^T, E^T) I diag(E, E), then shift by r:
//   Y_A = A~ - B~ R + R B~^T - R C~ R,  Y_B = B~ + R C~,  Y_C = C~,   R = skew(r)
template <class T> SD SI<T> congruence(const XF<T>& X, const SI<T>& I) {
  M3<T> At = mTm(X.E, mm(full(I.A), X.E));
  M3<T> Bt = mTm(X.E, mm(I.B, X.E));
  M3<T> Ct = mTm(X.E, mm(full(I.C), X.E));
  M3<T> R = skew(X.r);
  M3<T> BR = mm(Bt, R);
  M3<T> RCR = mm(R, mm(Ct, R));
  M3<T> YA = At - BR - transpose(BR) - RCR;   // R B~^T = -(B~ R)^T
  return SI<T>{symof(YA), Bt + mm(R, Ct), symof(Ct)};
}
// adjoint of the congruence: given Ybar (symmetric), accumulate Ibar, Ebar, rbar
template <class T> SD void congruence_adj(const XF<T>& X, const SI<T>& I, const SI<T>& Yb,
                                          SI<T>& Ib, M3<T>& Eb, V3<T>& rb) {
  M3<T> R = skew(X.r);
  M3<T> YbA = full(Yb.A), YbC = full(Yb.C);
  // shift adjoint: I~bar = T Ybar T^T with T = [1 0; -R 1]
  M3<T> tA = YbA;
  M3<T> tB = mm(YbA, R) + Yb.B;
  M3<T> RYB = mm(R, Yb.B);
  M3<T> tC = YbC - RYB - transpose(RYB) - mm(R, mm(YbA, R));
  // R bar = -2 [ (B~^T - C~ R) YbA + C~ YbB^T ]
  M3<T> Bt = mTm(X.E, mm(I.B, X.E));
  M3<T> Ct = mTm(X.E, mm(full(I.C), X.E));
  M3<T> G = mm(transpose(Bt) - mm(Ct, R), YbA) + mmT(Ct, Yb.B);
  V3<T> rg = unskew_grad(G);
  rb -= T(2) * rg;
  // rotation adjoint: Mbar_blk = E tbar_blk E^T;  Ebar = 2 [A E tA + B E tB^T + B^T E tB + C E tC]
  M3<T> FA = full(I.A), FC = full(I.C);
  M3<T> EtA = mm(X.E, tA), EtB = mm(X.E, tB), EtC = mm(X.E, tC);
  Eb += scale(T(2), mm(FA, EtA) + mmT(mm(I.B, X.E), tB) + mTm(I.B, EtB) + mm(FC, EtC));
  Ib.A += symof(mmT(EtA, X.E));
  Ib.B += mmT(EtB, X.E);
  Ib.C += symof(mmT(EtC, X.E));
}

// ------------------------------------------------------------------ rotations
// E_J of a revolute joint about unit axis a by angle q: R(a, q)^T with Rodrigues'
// R = 1 + s K + (1 - c) K^2, K = skew(a); for a unit axis K^2 = a a^T - 1, so
// E_J = c 1 - s K + (1 - c) a a^T
template <class T> SD M3<T> rot_axis_T(V3<T> a, T s, T c) {
  const T k = T(1) - c;
  const T xy = k * a.x * a.y, xz = k * a.x * a.z, yz = k * a.y * a.z;
  return M3<T>{{c + k * a.x * a.x, xy + s * a.z, xz - s * a.y,
                xy - s * a.z, c + k * a.y * a.y, yz + s * a.x,
                xz + s * a.y, yz - s * a.x, c + k * a.z * a.z}};
}
// <Gb, dE_J/dq> with dE_J/dq = -s 1 - c K + s a a^T
template <class T> SD T rot_axis_T_dq(V3<T> a, T s, T c, const M3<T>& Gb) {
  const T* g = Gb.a;
  const T tr = g[0] + g[4] + g[8];
  // <G, K> = a.x (g7 - g5) + a.y (g2 - g6) + a.z (g3 - g1)
  const T gk = a.x * (g[7] - g[5]) + a.y * (g[2] - g[6]) + a.z * (g[3] - g[1]);
  const V3<T> Ga = mul(Gb, a);
  return -s * tr - c * gk + s * dot(a, Ga);
}
// ------------------------------------------------------------------ revolute joints about z
// sim_create expresses every revolute link in a frame whose z axis is the joint
// axis, so S = [e_z; 0] and E_J = R(e_z, q)^T.  The helpers below are the general
// formulas above with a = e_z written out: without fast-math the compiler keeps
// products with constant zeros, so the saving has to be spelled out.
template <class T> SD V3<T> zaxis() { return V3<T>{T(0), T(0), T(1)}; }
// R(e_z, q)^T Et: rows 0 and 1 of Et rotated, row 2 kept
template <class T> SD M3<T> rotz_T_mm(T s, T c, const M3<T>& Et) {
  const T* e = Et.a;
  return M3<T>{{c * e[0] + s * e[3], c * e[1] + s * e[4], c * e[2] + s * e[5],
                c * e[3] - s * e[0], c * e[4] - s * e[1], c * e[5] - s * e[2], e[6], e[7], e[8]}};
}
// <Eb Et^T, dE_J/dq> for E = E_J Et (rot_axis_T_dq at a = e_z: -s (g0 + g4) - c (g3 - g1)
// with G = Eb Et^T; only those four entries are formed)
template <class T> SD T rotz_T_dq(T s, T c, const M3<T>& Eb, const M3<T>& Et) {
  const T* b = Eb.a;
  const T* e = Et.a;
  const T g0 = b[0] * e[0] + b[1] * e[1] + b[2] * e[2];
  const T g1 = b[0] * e[3] + b[1] * e[4] + b[2] * e[5];
  const T g3 = b[3] * e[0] + b[4] * e[1] + b[5] * e[2];
  const T g4 = b[3] * e[3] + b[4] * e[4] + b[5] * e[5];
  return -s * (g0 + g4) - c * (g3 - g1);
}
// I [e_z; 0]: the third column of a symmetric 6x6 (U = I^A S of a revolute link)
template <class T> SD SV<T> col_z(const SI<T>& I) {
  return SV<T>{{I.A.xz, I.A.yz, I.A.zz}, {I.B.a[6], I.B.a[7], I.B.a[8]}};
}
// m x [qd e_z; 0] (the velocity-product term c of a revolute link)
template <class T> SD SV<T> crossm_z(SV<T> m, T qd) {
  return SV<T>{{m.w.y * qd, -m.w.x * qd, T(0)}, {m.v.y * qd, -m.v.x * qd, T(0)}};
}
// adjoint of y = m x [qd e_z; 0]: mb += ..., returns the qd adjoint
template <class T> SD T crossm_z_adj(SV<T> m, T qd, SV<T> yb, SV<T>& mb) {
  mb.w.x -= qd * yb.w.y;
  mb.w.y += qd * yb.w.x;
  mb.v.x -= qd * yb.v.y;
  mb.v.y += qd * yb.v.x;
  return yb.w.x * m.w.y - yb.w.y * m.w.x + yb.v.x * m.v.y - yb.v.y * m.v.x;
}

// body -> world rotation of the unit quaternion (x, y, z, w)
template <class T> SD M3<T> quat_R(T x, T y, T z, T w) {
  return M3<T>{{T(1) - T(2) * (y * y + z * z), T(2) * (x * y - z * w), T(2) * (x * z + y * w),
                T(2) * (x * y + z * w), T(1) - T(2) * (x * x + z * z), T(2) * (y * z - x * w),
                T(2) * (x * z - y * w), T(2) * (y * z + x * w), T(1) - T(2) * (x * x + y * y)}};
}
// gradient of <Rbar, quat_R(q)> with respect to (x, y, z, w)
template <class T> SD void quat_R_adj(T x, T y, T z, T w, const M3<T>& Rb, T* qb) {
  const T* g = Rb.a;
  qb[0] += T(2) * (y * (g[1] + g[3]) + z * (g[2] + g[6]) + w * (g[7] - g[5])) - T(4) * x * (g[4] + g[8]);
  qb[1] += T(2) * (x * (g[1] + g[3]) + z * (g[5] + g[7]) + w * (g[2] - g[6])) - T(4) * y * (g[0] + g[8]);
  qb[2] += T(2) * (x * (g[2] + g[6]) + y * (g[5] + g[7]) + w * (g[3] - g[1])) - T(4) * z * (g[0] + g[4]);
  qb[3] += T(2) * (x * (g[7] - g[5]) + y * (g[2] - g[6]) + z * (g[3] - g[1]));
}
// Hamilton product a (x) b, quaternions stored (x, y, z, w)
template <class T> SD void quat_mul(const T* a, const T* b, T* o) {
  V3<T> av{a[0], a[1], a[2]}, bv{b[0], b[1], b[2]};
  V3<T> v = a[3] * bv + b[3] * av + cross(av, bv);
  o[0] = v.x; o[1] = v.y; o[2] = v.z;
  o[3] = a[3] * b[3] - dot(av, bv);
}

}  // namespace abasim
