/*
 * Scalar helpers of the CPU oracle (test infrastructure only): the plain
 * double type, and a forward-mode dual number Dual<N> carrying N tangent
 * directions, so that the oracle's own arithmetic, unchanged, also yields
 * exact directional derivatives (used as the CPU reference gradient for the
 * discrete adjoint).  Branches compare values only.
 */
#ifndef MPMC_ORACLE_SCALAR_HPP
#define MPMC_ORACLE_SCALAR_HPP
#include <cmath>
#include <type_traits>

namespace orc {

using std::cosh;
using std::fabs;
using std::log;
using std::sqrt;
using std::tanh;

inline double val(double x) { return x; }

template <class R>
struct is_dual : std::false_type {};

template <int N>
struct Dual {
  double v;
  double d[N];
  Dual() : v(0.0) {
    for (int i = 0; i < N; ++i) d[i] = 0.0;
  }
  Dual(double x) : v(x) {  // NOLINT: implicit from constants
    for (int i = 0; i < N; ++i) d[i] = 0.0;
  }
};

template <int N>
struct is_dual<Dual<N>> : std::true_type {};

template <int N> inline double val(const Dual<N>& x) { return x.v; }

template <int N> inline Dual<N> operator+(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r; r.v = a.v + b.v;
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
template <int N> inline Dual<N> operator-(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r; r.v = a.v - b.v;
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
template <int N> inline Dual<N> operator-(const Dual<N>& a) {
  Dual<N> r; r.v = -a.v;
  for (int i = 0; i < N; ++i) r.d[i] = -a.d[i];
  return r;
}
template <int N> inline Dual<N> operator*(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r; r.v = a.v * b.v;
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
  return r;
}
template <int N> inline Dual<N> operator/(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r; r.v = a.v / b.v;
  for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) / b.v;
  return r;
}
template <int N> inline Dual<N> operator+(double a, const Dual<N>& b) { return Dual<N>(a) + b; }
template <int N> inline Dual<N> operator+(const Dual<N>& a, double b) { return a + Dual<N>(b); }
template <int N> inline Dual<N> operator-(double a, const Dual<N>& b) { return Dual<N>(a) - b; }
template <int N> inline Dual<N> operator-(const Dual<N>& a, double b) { return a - Dual<N>(b); }
template <int N> inline Dual<N> operator*(double a, const Dual<N>& b) {
  Dual<N> r; r.v = a * b.v;
  for (int i = 0; i < N; ++i) r.d[i] = a * b.d[i];
  return r;
}
template <int N> inline Dual<N> operator*(const Dual<N>& a, double b) { return b * a; }
template <int N> inline Dual<N> operator/(const Dual<N>& a, double b) { return a / Dual<N>(b); }
template <int N> inline Dual<N> operator/(double a, const Dual<N>& b) { return Dual<N>(a) / b; }

template <int N> inline Dual<N> sqrt(const Dual<N>& a) {
  Dual<N> r; r.v = std::sqrt(a.v);
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] / (2.0 * r.v);
  return r;
}
template <int N> inline Dual<N> log(const Dual<N>& a) {
  Dual<N> r; r.v = std::log(a.v);
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] / a.v;
  return r;
}
template <int N> inline Dual<N> tanh(const Dual<N>& a) {
  Dual<N> r; r.v = std::tanh(a.v);
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * (1.0 - r.v * r.v);
  return r;
}
template <int N> inline Dual<N> cosh(const Dual<N>& a) {
  Dual<N> r; r.v = std::cosh(a.v);
  const double sh = std::sinh(a.v);
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * sh;
  return r;
}
template <int N> inline Dual<N> fabs(const Dual<N>& a) { return a.v < 0.0 ? -a : a; }

/* x with its value replaced by v and its tangent kept */
inline double with_value(double, double v) { return v; }
template <int N> inline Dual<N> with_value(const Dual<N>& x, double v) {
  Dual<N> r = x;
  r.v = v;
  return r;
}

/* value-based min / max that keep the chosen operand (and its tangent) */
template <class R> inline R rmin(const R& a, const R& b) { return val(b) < val(a) ? b : a; }
template <class R> inline R rmax(const R& a, const R& b) { return val(b) > val(a) ? b : a; }

}  // namespace orc
#endif
