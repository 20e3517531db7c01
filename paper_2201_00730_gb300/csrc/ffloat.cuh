// Float-float ("double-single") arithmetic for the half-step epilogues.
//
// FP64 runs at a small fraction of the FP32 rate on this GPU, so the per-row
// work of the epilogues (softmin in cost units, aprox, translation, residual,
// the mass terms of the TI update) is carried as unevaluated sums hi + lo of
// two floats, about 44 significant bits, enough for results rounded to FP32
// and for mass sums accurate to ~1e-11 relative.
//
// Building blocks: error-free transformations (Knuth's TwoSum, Dekker's
// FastTwoSum, TwoProduct via FMA) and a table-driven exp2 in the manner of
// Tang (ACM TOMS 15(2), 1989): 2^y = 2^n * 2^(j/64) * e^(r ln 2) with n an
// integer, j in [-32, 32], |r| <= 1/128, the table entries 2^(j/64) held as
// float pairs and e^p for |p| <= 0.0055 summed to fourth order.
//
// Nothing here may be compiled with reassociating fast-math flags.
#pragma once

#include <cuda_runtime.h>

namespace uot {
namespace ffl {

struct ff {
  float hi, lo;
};

__device__ __forceinline__ ff two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return ff{s, e};
}

// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ ff fast_two_sum(float a, float b) {
  const float s = a + b;
  return ff{s, b - (s - a)};
}

__device__ __forceinline__ ff add(ff a, ff b) {
  ff s = two_sum(a.hi, b.hi);
  const ff t = two_sum(a.lo, b.lo);
  s = fast_two_sum(s.hi, s.lo + t.hi);
  return fast_two_sum(s.hi, s.lo + t.lo);
}

__device__ __forceinline__ ff add(ff a, float b) {
  ff s = two_sum(a.hi, b);
  return fast_two_sum(s.hi, s.lo + a.lo);
}

__device__ __forceinline__ ff neg(ff a) { return ff{-a.hi, -a.lo}; }

__device__ __forceinline__ ff mul(ff a, ff b) {
  const float p = a.hi * b.hi;
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
  return fast_two_sum(p, e);
}

__device__ __forceinline__ ff mul(ff a, float b) {
  const float p = a.hi * b;
  const float e = __fmaf_rn(a.hi, b, -p);
  return fast_two_sum(p, __fmaf_rn(a.lo, b, e));
}

// double -> float pair (FP64: one conversion, one subtraction, one conversion)
__device__ __forceinline__ ff from_double(double d) {
  const float hi = (float)d;
  return ff{hi, (float)(d - (double)hi)};
}

__host__ __device__ __forceinline__ double to_double(ff a) { return (double)a.hi + (double)a.lo; }

// ---- table of 2^(j/64), j = -32..32, as float pairs (built at compile time)

constexpr double cx_sqrt(double x) {
  double r = x > 1.0 ? x : 1.0;
  for (int i = 0; i < 80; ++i) r = 0.5 * (r + x / r);
  return r;
}

struct Exp2Table {
  float hi[65];
  float lo[65];
};

constexpr Exp2Table make_exp2_table() {
  Exp2Table t{};
  double c = 2.0;
  for (int k = 0; k < 6; ++k) c = cx_sqrt(c);  // 2^(1/64)
  double up = 1.0, dn = 1.0;
  const double ci = 1.0 / c;
  for (int j = 0; j <= 32; ++j) {
    const float uh = (float)up, dh = (float)dn;
    t.hi[32 + j] = uh;
    t.lo[32 + j] = (float)(up - (double)uh);
    t.hi[32 - j] = dh;
    t.lo[32 - j] = (float)(dn - (double)dh);
    up *= c;
    dn *= ci;
  }
  return t;
}

__device__ const Exp2Table kExp2Tab = make_exp2_table();

// 2^k as a float for integer k in [-126, 127] (built from the exponent bits).
__device__ __forceinline__ float pow2f(int k) { return __int_as_float((k + 127) << 23); }

constexpr double kLn2d = 0.69314718055994530942;
constexpr float kLn2Hi = (float)kLn2d;
constexpr float kLn2Lo = (float)(kLn2d - (double)(float)kLn2d);

// 2^y for a float pair y with y.hi <= 64; returns 0 below 2^-126.  T: the
// table (the global one, or a copy in shared memory).
__device__ __forceinline__ ff exp2(ff y, const Exp2Table& T = kExp2Tab) {
  if (!(y.hi > -126.f)) return ff{0.f, 0.f};
  const float n = rintf(y.hi);
  const float d = y.hi - n;               // exact, |d| <= 1/2
  const float jf = rintf(d * 64.f);       // j in [-32, 32]
  const float rh = (d * 64.f - jf) * (1.f / 64.f);  // exact, |rh| <= 1/128
  const ff r = two_sum(rh, y.lo);
  // p = r ln 2
  const float ph = r.hi * kLn2Hi;
  const float pl = __fmaf_rn(r.hi, kLn2Hi, -ph) + __fmaf_rn(r.hi, kLn2Lo, r.lo * kLn2Hi);
  // e^p = 1 + p + p^2/2 + p^3/6 + p^4/24 (|p| <= 0.0055: next term < 5e-14)
  const float q = __fmaf_rn(ph * ph, __fmaf_rn(ph, __fmaf_rn(ph, 1.f / 24.f, 1.f / 6.f), 0.5f), __fmaf_rn(ph, pl, pl));
  ff E = fast_two_sum(1.f, ph);
  E = fast_two_sum(E.hi, E.lo + q);
  const int j = (int)jf + 32;
  ff v = mul(ff{T.hi[j], T.lo[j]}, E);
  const float sc = pow2f((int)n);  // n in [-126, 64]
  v.hi *= sc;
  v.lo *= sc;
  return v;
}

constexpr ff kLn2ff{kLn2Hi, kLn2Lo};

// Natural log of a positive float pair: y0 = log2(hi) from the hardware
// approximation, then one Newton correction ln(1 + r) ~ r with r = a 2^-y0 - 1
// evaluated on pairs (|r| ~ 1e-7, so r^2/2 is below 1e-14).
__device__ __forceinline__ ff log_ff(ff a, const Exp2Table& T = kExp2Tab) {
  const float y0 = __log2f(a.hi);
  const ff e = exp2(ff{-y0, 0.f}, T);
  const ff r = add(mul(a, e), -1.f);
  return add(mul(kLn2ff, y0), r);
}

// The same, returned in FP64.
__device__ __forceinline__ double log(ff a) { return to_double(log_ff(a)); }

// An integer as an exact float pair (|k| < 2^31).
__device__ __forceinline__ ff from_int(int k) {
  const float hi = (float)k;
  return ff{hi, (float)(k - (int)hi)};
}

}  // namespace ffl
}  // namespace uot
