// Dual numbers v + d eps (eps^2 = 0): running the step functions on this scalar
// carries a tangent through them, i.e. forward-mode differentiation of one
// simulation step (the Jacobian-vector product d x^{k+1} = J dx^k + J_u du^k).
#pragma once

#include <type_traits>

#include "aba_step.cuh"

namespace abasim {

template <class T> struct Dual {
  T v, d;
  SD Dual() : v(0), d(0) {}
  SD Dual(T x, T dx) : v(x), d(dx) {}
  template <class U, class = typename std::enable_if<std::is_arithmetic<U>::value>::type>
  SD Dual(U x) : v(T(x)), d(0) {}
  SD Dual& operator+=(Dual o) { v += o.v; d += o.d; return *this; }
  SD Dual& operator-=(Dual o) { v -= o.v; d -= o.d; return *this; }
  SD Dual& operator*=(Dual o) { d = d * o.v + v * o.d; v *= o.v; return *this; }
};
template <class T> SD Dual<T> operator+(Dual<T> a, Dual<T> b) { return Dual<T>(a.v + b.v, a.d + b.d); }
template <class T> SD Dual<T> operator-(Dual<T> a, Dual<T> b) { return Dual<T>(a.v - b.v, a.d - b.d); }
template <class T> SD Dual<T> operator-(Dual<T> a) { return Dual<T>(-a.v, -a.d); }
template <class T> SD Dual<T> operator*(Dual<T> a, Dual<T> b) { return Dual<T>(a.v * b.v, a.d * b.v + a.v * b.d); }
template <class T> SD Dual<T> operator/(Dual<T> a, Dual<T> b) {
  const T q = a.v / b.v;
  return Dual<T>(q, (a.d - q * b.d) / b.v);
}
template <class T> SD Dual<T> sqrt(Dual<T> a) {
  const T r = ::sqrt(a.v);
  return Dual<T>(r, a.d / (T(2) * r));
}

template <> SD void sincos_t<Dual<float>>(Dual<float> x, Dual<float>* s, Dual<float>* c) {
  float sv, cv;
  sincos_t<float>(x.v, &sv, &cv);
  *s = Dual<float>(sv, cv * x.d);
  *c = Dual<float>(cv, -sv * x.d);
}
template <> SD void sincos_t<Dual<double>>(Dual<double> x, Dual<double>* s, Dual<double>* c) {
  double sv, cv;
  sincos_t<double>(x.v, &sv, &cv);
  *s = Dual<double>(sv, cv * x.d);
  *c = Dual<double>(cv, -sv * x.d);
}

}  // namespace abasim
