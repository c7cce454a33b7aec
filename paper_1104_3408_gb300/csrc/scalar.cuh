// Scalar types for the pointwise kernels: plain double (FP64 path) and a
// double-float "ff" (FP32 pair, hi + lo) for the mixed path.
//
// ff arithmetic uses the error-free transformations TwoSum (Knuth, TAOCP
// vol. 2, 4.2.2) and TwoProd via a fused multiply-add (Dekker 1971; FMA form
// as in Muller et al., Handbook of Floating-Point Arithmetic, 2nd ed., 4.4),
// with the "sloppy" double-word addition and the double-word times
// double-word product of Joldes, Muller and Popescu, "Tight and rigorous
// error bounds for basic building blocks of double-word arithmetic", ACM TOMS
// 44 (2017), Algorithms 5 and 11 (FMA variant).  Division and square root take
// one Newton correction of the FP32 quotient / root computed by CUDA's own
// operators.  The relative error of one operation is O(2^-44) except under
// cancellation in the sloppy addition, whose absolute error stays O(2^-44)
// times the operands' magnitude: the quantity the pointwise kernels are
// checked against.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace cffyn {

struct ff {
  float hi, lo;
};

__device__ __forceinline__ ff ff_from_float(float a) { return ff{a, 0.0f}; }

// v * 2^sc as a double (round to nearest, integer operations only); v != 0
// handled, v == 0 gives 0.  Used where the FP64 / conversion pipes of this part
// would be the bottleneck.
__device__ __forceinline__ double u64_scaled_to_double(unsigned long long v, int sc, bool neg) {
  if (v == 0) return 0.0;
  const int nb = 64 - __clzll((long long)v);
  int ex = nb - 1 + sc;
  unsigned long long m;
  if (nb > 53) {
    const int sh = nb - 53;
    m = (v + (1ull << (sh - 1))) >> sh;
    if (m >> 53) {
      m >>= 1;
      ex += 1;
    }
  } else {
    m = v << (53 - nb);
  }
  if (ex + 1023 <= 0) return 0.0;
  if (ex + 1023 >= 2047) return neg ? -__longlong_as_double(0x7ff0000000000000ll)
                                    : __longlong_as_double(0x7ff0000000000000ll);
  const unsigned long long bits = (neg ? 0x8000000000000000ull : 0ull) |
                                  ((unsigned long long)(ex + 1023) << 52) |
                                  (m & 0x000fffffffffffffull);
  return __longlong_as_double((long long)bits);
}

// v * 2^sc as a float (truncating), integer operations only.
__device__ __forceinline__ float u64_scaled_to_float(unsigned long long v, int sc, bool neg) {
  if (v == 0) return 0.0f;
  const int nb = 64 - __clzll((long long)v);
  int ex = nb - 1 + sc;
  unsigned int m = nb > 24 ? (unsigned int)(v >> (nb - 24)) : (unsigned int)(v << (24 - nb));
  if (ex + 127 <= 0) return 0.0f;  // below the normal range: flushed
  const unsigned int bits = (neg ? 0x80000000u : 0u) | ((unsigned int)(ex + 127) << 23) | (m & 0x7fffffu);
  return __uint_as_float(bits);
}

// Split an FP64 value into hi + lo with integer operations only: hi keeps the
// leading 24 significand bits (truncated), lo the next 24 (truncated), so
// |x - hi - lo| <= 2^-47 |x|.  Values outside the FP32 normal range are
// flushed to 0 / +-Inf; NaN stays NaN.
__device__ __forceinline__ ff ff_from_double(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const bool neg = (b >> 63) != 0;
  const int e = (int)((b >> 52) & 0x7ff);
  if (e == 0) return ff{0.0f, 0.0f};
  if (e == 0x7ff) return ff{(float)x, 0.0f};   // Inf / NaN: rare, conversion is fine
  const int E = e - 1023;
  if (E > 127) return ff{neg ? -__int_as_float(0x7f800000) : __int_as_float(0x7f800000), 0.0f};
  if (E < -126) return ff{0.0f, 0.0f};
  const unsigned long long m = b & 0x000fffffffffffffull;
  const unsigned int hbits = (neg ? 0x80000000u : 0u) | ((unsigned int)(E + 127) << 23) |
                             (unsigned int)(m >> 29);
  const float hi = __uint_as_float(hbits);
  const float lo = u64_scaled_to_float(m & ((1ull << 29) - 1), E - 52, neg);
  return ff{hi, lo};
}

// hi + lo as a double with integer operations only.
__device__ __forceinline__ double ff_to_double(ff a) {
  const unsigned int uh = __float_as_uint(a.hi), ul = __float_as_uint(a.lo);
  const int eh = (int)((uh >> 23) & 0xff), el = (int)((ul >> 23) & 0xff);
  if (eh == 0xff) return (double)a.hi;         // Inf / NaN
  if (eh == 0) {                                // hi zero (or FP32 denormal): lo alone
    if (el == 0) return 0.0;
    return u64_scaled_to_double((ul & 0x7fffffu) | 0x800000u, el - 150, (ul >> 31) != 0);
  }
  const long long Mh = (long long)((uh & 0x7fffffu) | 0x800000u) << 29;  // unit 2^(eh-127-52)
  long long V = (uh >> 31) ? -Mh : Mh;
  if (el != 0) {
    const long long Ml = (long long)((ul & 0x7fffffu) | 0x800000u);
    const int sh = el - eh + 29;                  // lo relative to the unit
    long long Lv = 0;
    if (sh >= 0) Lv = Ml << sh;
    else if (sh > -40) Lv = Ml >> (-sh);
    V += (ul >> 31) ? -Lv : Lv;
  }
  const bool neg = V < 0;
  return u64_scaled_to_double(neg ? (unsigned long long)(-V) : (unsigned long long)V, eh - 127 - 52, neg);
}

// All additions and products inside the error-free transformations use the
// _rn intrinsics: the compiler never contracts those into fused multiply-adds,
// which would silently break the exactness of TwoSum / TwoProd.
__device__ __forceinline__ float fa(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fs(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fm(float a, float b) { return __fmul_rn(a, b); }

__device__ __forceinline__ ff two_sum(float a, float b) {
  const float s = fa(a, b);
  const float bb = fs(s, a);
  const float e = fa(fs(a, fs(s, bb)), fs(b, bb));
  return ff{s, e};
}
__device__ __forceinline__ ff fast_two_sum(float a, float b) {
  const float s = fa(a, b);
  const float e = fs(b, fs(s, a));
  return ff{s, e};
}
__device__ __forceinline__ ff operator+(ff x, ff y) {
  const ff s = two_sum(x.hi, y.hi);
  const float v = fa(s.lo, fa(x.lo, y.lo));
  return fast_two_sum(s.hi, v);
}
__device__ __forceinline__ ff operator-(ff x) { return ff{-x.hi, -x.lo}; }
__device__ __forceinline__ ff operator-(ff x, ff y) { return x + (-y); }
__device__ __forceinline__ ff operator*(ff x, ff y) {
  const float p = fm(x.hi, y.hi);
  const float e = fmaf(x.hi, y.hi, -p);
  const float t = fmaf(x.hi, y.lo, fm(x.lo, y.hi));
  return fast_two_sum(p, fa(e, t));
}
__device__ __forceinline__ ff operator*(ff x, float c) {
  const float p = fm(x.hi, c);
  const float e = fmaf(x.hi, c, -p);
  return fast_two_sum(p, fmaf(x.lo, c, e));
}
__device__ __forceinline__ ff operator*(float c, ff x) { return x * c; }
__device__ __forceinline__ ff operator/(ff x, ff y) {
  const float q = __fdiv_rn(x.hi, y.hi);
  const ff r = x - y * q;  // residual
  const float q2 = __fdiv_rn(r.hi, y.hi);
  return fast_two_sum(q, q2);
}
__device__ __forceinline__ ff& operator+=(ff& a, ff b) { a = a + b; return a; }
__device__ __forceinline__ ff& operator-=(ff& a, ff b) { a = a - b; return a; }
__device__ __forceinline__ ff sqrt_s(ff x) {
  if (x.hi <= 0.0f) return ff{__fsqrt_rn(x.hi), 0.0f};
  const float s = __fsqrt_rn(x.hi);
  const ff ss = ff{s, 0.0f} * ff{s, 0.0f};
  const ff r = x - ss;
  return fast_two_sum(s, __fdiv_rn(r.hi, fm(2.0f, s)));
}
__device__ __forceinline__ double sqrt_s(double x) { return sqrt(x); }

// Dot-product accumulator.  double: plain FMA.  ff: the compensated dot
// product "Dot2" of Ogita, Rump and Oishi ("Accurate sum and dot product",
// SIAM J. Sci. Comput. 26 (2005)): every product is split exactly by TwoProd
// (with the cross terms of the low parts folded in), the running sum by
// TwoSum, and all error terms collect in one FP32 word that is added back at
// the end.
template <class T> struct Acc;
template <> struct Acc<double> {
  double s = 0.0;
  __device__ __forceinline__ void fma_(double a, double b) { s = fma(a, b, s); }
  __device__ __forceinline__ void add(double a) { s += a; }
  __device__ __forceinline__ double get() const { return s; }
};
template <> struct Acc<ff> {
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void fma_(ff a, ff b) {
    const float p = fm(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    const float t = fa(s, p);
    const float bb = fs(t, s);
    const float err = fa(fs(s, fs(t, bb)), fs(p, bb));
    s = t;
    c = fa(c, fa(err, e));
  }
  __device__ __forceinline__ void add(ff a) {
    const float t = fa(s, a.hi);
    const float bb = fs(t, s);
    const float err = fa(fs(s, fs(t, bb)), fs(a.hi, bb));
    s = t;
    c = fa(c, fa(err, a.lo));
  }
  __device__ __forceinline__ ff get() const { return two_sum(s, c); }
};

// Finiteness from the bit patterns (no FP64 instruction).
__device__ __forceinline__ bool finite_s(double x) {
  return ((__double_as_longlong(x) >> 52) & 0x7ff) != 0x7ff;
}
__device__ __forceinline__ bool finite_s(ff x) {
  return ((__float_as_uint(x.hi) >> 23) & 0xff) != 0xff;
}

// Uniform helpers so that templated code reads the same for both types.
template <class T> struct S;
template <> struct S<double> {
  static __device__ __forceinline__ double c(double v) { return v; }
  static __device__ __forceinline__ double load(const double* p) { return *p; }
  static __device__ __forceinline__ double to_double(double v) { return v; }
};
template <> struct S<ff> {
  static __device__ __forceinline__ ff c(double v) { return ff_from_double(v); }
  static __device__ __forceinline__ ff load(const double* p) { return ff_from_double(__ldg(p)); }
  static __device__ __forceinline__ double to_double(ff v) { return ff_to_double(v); }
};

// Storage of an array: FP64 words (FF = false) or double-float pairs stored
// as float2 (FF = true); both are 8 bytes per value.  Internal buffers of the
// mixed path use the pair form, so that its pointwise kernels load and store
// without any conversion.
template <class T, bool FF> struct Store;
template <> struct Store<double, false> {
  static __device__ __forceinline__ double ld(const double* b, long long i) { return b[i]; }
  static __device__ __forceinline__ void st(double* b, long long i, double v) { b[i] = v; }
};
template <> struct Store<ff, false> {
  static __device__ __forceinline__ ff ld(const double* b, long long i) { return ff_from_double(__ldg(b + i)); }
  static __device__ __forceinline__ void st(double* b, long long i, ff v) { b[i] = ff_to_double(v); }
};
template <> struct Store<ff, true> {
  static __device__ __forceinline__ ff ld(const double* b, long long i) {
    const float2 v = __ldg(reinterpret_cast<const float2*>(b) + i);
    return ff{v.x, v.y};
  }
  static __device__ __forceinline__ void st(double* b, long long i, ff v) {
    reinterpret_cast<float2*>(b)[i] = make_float2(v.hi, v.lo);
  }
};
template <> struct Store<double, true> {  // FP64 access to a pair-stored buffer (setup paths)
  static __device__ __forceinline__ double ld(const double* b, long long i) {
    const float2 v = reinterpret_cast<const float2*>(b)[i];
    return ff_to_double(ff{v.x, v.y});
  }
  static __device__ __forceinline__ void st(double* b, long long i, double v) {
    const ff f = ff_from_double(v);
    reinterpret_cast<float2*>(b)[i] = make_float2(f.hi, f.lo);
  }
};

}  // namespace cffyn
