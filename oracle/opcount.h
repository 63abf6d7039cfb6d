/*
 * opcount.h -- counting build of the oracle (C++ only).
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  opcount.cpp compiles rtw_oracle.c as C++ with this
 * header in front of it: `double` becomes a value type that counts every floating-point operation
 * it executes, and the complex type of the oracle (cplx) is built on it.  The oracle's sources
 * are otherwise unchanged (rtw_oracle.c takes cplx from here when OR_OPCOUNT is defined), so the
 * count is that of the oracle's own arithmetic: the algorithmic operation count of one ray
 * interaction that the throughput of the trace kernels is measured in.
 *
 * Counted: additions and subtractions, multiplications, divisions, square roots, and calls of
 * elementary functions (sin, cos, atan2, acos, asin, exp, pow, hypot, cbrt, tanh, log).  Not
 * counted: negation, comparisons, fabs, fmin, fmax, copysign, floor, ceil, conversions, and the
 * multiplication of a real number by the imaginary unit (it only places a value).
 */
#ifndef OR_OPCOUNT_H
#define OR_OPCOUNT_H

#ifndef __cplusplus
#error "opcount.h is the C++ counting build of the oracle"
#endif

/* every header the oracle includes, before double is redefined */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <cmath>
#include <type_traits>

struct or_opcount {
    unsigned long long add, mul, div, sqrt, fn;
};
/* the counters (single-threaded: the counting build runs without OpenMP) */
extern or_opcount g_or_opcount;

struct or_cdbl {
    double v;
    or_cdbl() = default;
    template <typename T, typename std::enable_if<std::is_arithmetic<T>::value, int>::type = 0>
    constexpr or_cdbl(T x) : v((double)x) {}
    template <typename T, typename std::enable_if<std::is_arithmetic<T>::value, int>::type = 0>
    explicit constexpr operator T() const { return (T)v; }
    or_cdbl& operator+=(or_cdbl o) { ++g_or_opcount.add; v += o.v; return *this; }
    or_cdbl& operator-=(or_cdbl o) { ++g_or_opcount.add; v -= o.v; return *this; }
    or_cdbl& operator*=(or_cdbl o) { ++g_or_opcount.mul; v *= o.v; return *this; }
    or_cdbl& operator/=(or_cdbl o) { ++g_or_opcount.div; v /= o.v; return *this; }
    or_cdbl operator-() const { return or_cdbl(-v); }
    or_cdbl operator+() const { return *this; }
};
static_assert(sizeof(or_cdbl) == sizeof(double), "or_cdbl is laid out as a double");

inline or_cdbl operator+(or_cdbl a, or_cdbl b) { ++g_or_opcount.add; return a.v + b.v; }
inline or_cdbl operator-(or_cdbl a, or_cdbl b) { ++g_or_opcount.add; return a.v - b.v; }
inline or_cdbl operator*(or_cdbl a, or_cdbl b) { ++g_or_opcount.mul; return a.v * b.v; }
inline or_cdbl operator/(or_cdbl a, or_cdbl b) { ++g_or_opcount.div; return a.v / b.v; }
inline bool operator==(or_cdbl a, or_cdbl b) { return a.v == b.v; }
inline bool operator!=(or_cdbl a, or_cdbl b) { return a.v != b.v; }
inline bool operator<(or_cdbl a, or_cdbl b) { return a.v < b.v; }
inline bool operator>(or_cdbl a, or_cdbl b) { return a.v > b.v; }
inline bool operator<=(or_cdbl a, or_cdbl b) { return a.v <= b.v; }
inline bool operator>=(or_cdbl a, or_cdbl b) { return a.v >= b.v; }
inline bool operator!(or_cdbl a) { return !a.v; }

#define OR_FN1(name, counter)                                                   \
    inline or_cdbl name(or_cdbl x) { counter; return std::name(x.v); }
OR_FN1(sqrt, ++g_or_opcount.sqrt)
OR_FN1(sin, ++g_or_opcount.fn)
OR_FN1(cos, ++g_or_opcount.fn)
OR_FN1(acos, ++g_or_opcount.fn)
OR_FN1(asin, ++g_or_opcount.fn)
OR_FN1(exp, ++g_or_opcount.fn)
OR_FN1(log, ++g_or_opcount.fn)
OR_FN1(cbrt, ++g_or_opcount.fn)
OR_FN1(tanh, ++g_or_opcount.fn)
OR_FN1(fabs, (void)0)
OR_FN1(floor, (void)0)
OR_FN1(ceil, (void)0)
#undef OR_FN1
inline or_cdbl atan2(or_cdbl y, or_cdbl x) { ++g_or_opcount.fn; return std::atan2(y.v, x.v); }
inline or_cdbl pow(or_cdbl x, or_cdbl y) { ++g_or_opcount.fn; return std::pow(x.v, y.v); }
inline or_cdbl hypot(or_cdbl x, or_cdbl y) { ++g_or_opcount.fn; return std::hypot(x.v, y.v); }
inline or_cdbl fmin(or_cdbl x, or_cdbl y) { return std::fmin(x.v, y.v); }
inline or_cdbl fmax(or_cdbl x, or_cdbl y) { return std::fmax(x.v, y.v); }
inline or_cdbl copysign(or_cdbl x, or_cdbl y) { return std::copysign(x.v, y.v); }
inline bool isfinite(or_cdbl x) { return std::isfinite(x.v); }

/* the oracle's complex type on counted doubles.  Its operators are templates whose operand types
 * must match exactly, so that a real operand never reaches them through a conversion and a
 * real-times-complex product is counted as the two multiplications it takes. */
struct or_imag_unit {};
struct cplx {
    or_cdbl re, im;
    cplx() = default;
    constexpr cplx(or_cdbl r, or_cdbl i) : re(r), im(i) {}
    template <typename T, typename std::enable_if<std::is_arithmetic<T>::value, int>::type = 0>
    constexpr cplx(T r) : re(r), im(0.0) {}
    constexpr cplx(or_cdbl r) : re(r), im(0.0) {}
    constexpr cplx(or_imag_unit) : re(0.0), im(1.0) {}
    cplx operator-() const { return cplx(-re, -im); }
};
template <typename T>
struct or_is_real : std::integral_constant<bool, std::is_arithmetic<T>::value || std::is_same<T, or_cdbl>::value> {};
template <typename T>
struct or_is_cplx : std::is_same<T, cplx> {};
#define OR_CC typename std::enable_if<or_is_cplx<A>::value && or_is_cplx<B>::value, int>::type = 0
#define OR_RC typename std::enable_if<or_is_real<A>::value && or_is_cplx<B>::value, int>::type = 0
#define OR_CR typename std::enable_if<or_is_cplx<A>::value && or_is_real<B>::value, int>::type = 0
template <typename A, typename B, OR_CC> inline cplx operator+(A a, B b) { return cplx(a.re + b.re, a.im + b.im); }
template <typename A, typename B, OR_CC> inline cplx operator-(A a, B b) { return cplx(a.re - b.re, a.im - b.im); }
template <typename A, typename B, OR_CC> inline cplx operator*(A a, B b)
{
    return cplx(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename A, typename B, OR_CC> inline cplx operator/(A a, B b)
{
    const or_cdbl d = b.re * b.re + b.im * b.im;
    return cplx((a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d);
}
template <typename A, typename B, OR_RC> inline cplx operator*(A a, B b) { return cplx(a * b.re, a * b.im); }
template <typename A, typename B, OR_CR> inline cplx operator*(A a, B b) { return cplx(a.re * b, a.im * b); }
template <typename A, typename B, OR_CR> inline cplx operator/(A a, B b) { return cplx(a.re / b, a.im / b); }
template <typename A, typename B, OR_RC> inline cplx operator/(A a, B b) { return cplx(a) / b; }
template <typename A, typename B, OR_RC> inline cplx operator+(A a, B b) { return cplx(a + b.re, b.im); }
template <typename A, typename B, OR_CR> inline cplx operator+(A a, B b) { return cplx(a.re + b, a.im); }
template <typename A, typename B, OR_RC> inline cplx operator-(A a, B b) { return cplx(a - b.re, -b.im); }
template <typename A, typename B, OR_CR> inline cplx operator-(A a, B b) { return cplx(a.re - b, a.im); }
#undef OR_CC
#undef OR_RC
#undef OR_CR
template <typename B> inline cplx& operator+=(cplx& a, B b) { a = a + b; return a; }
template <typename B> inline cplx& operator-=(cplx& a, B b) { a = a - b; return a; }
template <typename B> inline cplx& operator*=(cplx& a, B b) { a = a * b; return a; }
/* the imaginary unit only places a value */
template <typename R, typename std::enable_if<or_is_real<R>::value, int>::type = 0>
inline cplx operator*(or_imag_unit, R x) { return cplx(0.0, or_cdbl(x)); }
template <typename R, typename std::enable_if<or_is_real<R>::value, int>::type = 0>
inline cplx operator*(R x, or_imag_unit) { return cplx(0.0, or_cdbl(x)); }
inline cplx operator-(or_imag_unit) { return cplx(0.0, -1.0); }
inline or_cdbl creal(cplx z) { return z.re; }
inline or_cdbl cimag(cplx z) { return z.im; }
inline cplx conj(cplx z) { return cplx(z.re, -z.im); }
inline cplx cexp(cplx z)
{
    if (z.re.v == 0.0) return cplx(cos(z.im), sin(z.im));  /* e^{i y}: a cosine and a sine */
    const or_cdbl e = exp(z.re);
    return cplx(e * cos(z.im), e * sin(z.im));
}
#define I (or_imag_unit{})

/* from here on the oracle's double is the counted type */
#define double or_cdbl

#endif
