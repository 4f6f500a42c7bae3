// Double-float arithmetic: a real number as the unevaluated sum hi + lo of two
// floats (|lo| <= ulp(hi) / 2), about 48 significant bits.  GB300 executes FP64
// instructions at a small fraction of its FP32 rate, so the high-precision
// parts of the method (reliable updates, HP source preparation and
// reconstruction, the HPE remainder and the contractions of HP solutions) run
// on this type: every operation is a short sequence of FP32 additions and
// fused multiply-adds.
//
// The algorithms are the error-free transformations of Knuth (two-sum), Dekker
// (fast two-sum) and the FMA-based exact product, combined as in the
// double-double arithmetic of Hida, Li & Bailey (2001): the "accurate" sum and
// the product with the cross terms added before renormalisation.
#pragma once

#ifdef __CUDACC__
#define DF_HD __host__ __device__ __forceinline__
#else
#include <cmath>
#define DF_HD inline
#endif

struct dfloat {
  float hi, lo;
  DF_HD dfloat() {}
  DF_HD dfloat(float h, float l) : hi(h), lo(l) {}
  DF_HD dfloat(int v) : hi((float)v), lo(0.f) {}
  DF_HD dfloat(float v) : hi(v), lo(0.f) {}
  // split a double (rounds away its last ~5 bits); uses FP64 instructions
  DF_HD explicit dfloat(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
  DF_HD explicit operator double() const { return (double)hi + (double)lo; }
  DF_HD explicit operator float() const { return hi + lo; }
};

DF_HD float df_fma(float a, float b, float c) {
#ifdef __CUDA_ARCH__
  return __fmaf_rn(a, b, c);
#else
  return std::fma(a, b, c);
#endif
}

// s + e = a + b exactly (Knuth)
DF_HD void df_two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
// s + e = a + b exactly, for |a| >= |b| (Dekker)
DF_HD void df_fast_two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  e = b - (s - a);
}

DF_HD dfloat operator+(const dfloat& a, const dfloat& b) {
  float s, e, t, f;
  df_two_sum(a.hi, b.hi, s, e);
  df_two_sum(a.lo, b.lo, t, f);
  e += t;
  df_fast_two_sum(s, e, s, e);
  e += f;
  df_fast_two_sum(s, e, s, e);
  return dfloat(s, e);
}
DF_HD dfloat operator-(const dfloat& a) { return dfloat(-a.hi, -a.lo); }
DF_HD dfloat operator-(const dfloat& a, const dfloat& b) { return a + (-b); }
DF_HD dfloat operator*(const dfloat& a, const dfloat& b) {
  const float p = a.hi * b.hi;
  float e = df_fma(a.hi, b.hi, -p);  // exact error of the leading product
  e = df_fma(a.hi, b.lo, e);
  e = df_fma(a.lo, b.hi, e);
  float s;
  df_fast_two_sum(p, e, s, e);
  return dfloat(s, e);
}
DF_HD dfloat& operator+=(dfloat& a, const dfloat& b) {
  a = a + b;
  return a;
}
DF_HD dfloat& operator-=(dfloat& a, const dfloat& b) {
  a = a - b;
  return a;
}
DF_HD dfloat& operator*=(dfloat& a, const dfloat& b) {
  a = a * b;
  return a;
}

// Lazy accumulation (sums of many terms, e.g. the stencil's SU(3) products and its
// sum over hops): the running sum is kept as an unnormalised pair (hi, lo) whose hi
// part is updated by an exact two-sum and whose lo part collects the two-sum errors
// and the terms' own low parts in FP32; df_normalize makes it a dfloat again.  Each
// FP32 addition into lo errs by at most 2^-24 |lo| ~ 2^-48 of the sum's scale, so the
// result keeps the double-float accuracy of the terms (absolute error ~2^-47 times
// the sum of their magnitudes) at about half the operations of repeated dfloat adds.
DF_HD void df_acc(dfloat& s, const dfloat& t) {  // s += t
  float h, e;
  df_two_sum(s.hi, t.hi, h, e);
  s.lo = s.lo + (t.lo + e);
  s.hi = h;
}
// s += a * b, the product's leading part exact (FMA) and both cross terms added to lo
// (a.lo * b.lo, below 2^-48 of the product, is dropped)
DF_HD void df_acc_mul(dfloat& s, const dfloat& a, const dfloat& b) {
  const float p = a.hi * b.hi;
  float c = df_fma(a.hi, b.hi, -p);
  c = df_fma(a.hi, b.lo, c);
  c = df_fma(a.lo, b.hi, c);
  float h, e;
  df_two_sum(s.hi, p, h, e);
  s.lo = s.lo + (c + e);
  s.hi = h;
}
// the first term of a lazy sum: s = a * b
DF_HD dfloat df_mul_lazy(const dfloat& a, const dfloat& b) {
  const float p = a.hi * b.hi;
  float c = df_fma(a.hi, b.hi, -p);
  c = df_fma(a.hi, b.lo, c);
  c = df_fma(a.lo, b.hi, c);
  return dfloat(p, c);
}
// a + b and a - b as unnormalised pairs (exact two-sum of the hi parts)
DF_HD dfloat df_add_lazy(const dfloat& a, const dfloat& b) {
  float h, e;
  df_two_sum(a.hi, b.hi, h, e);
  return dfloat(h, (a.lo + b.lo) + e);
}
// (a full two-sum: after cancellation in the hi parts |lo| may exceed |hi|)
DF_HD dfloat df_normalize(const dfloat& s) {
  float h, e;
  df_two_sum(s.hi, s.lo, h, e);
  return dfloat(h, e);
}
