// Double-float arithmetic: a value is the unevaluated sum hi + lo of two FP32
// numbers with |lo| <= ulp(hi) / 2, about 48 significant bits.  Used for the
// FP64-accuracy operator of the mixed-precision solvers (their true residuals),
// which on this GPU runs several times faster on the FP32 pipes than in FP64.
//
// Built from two error-free transformations:
//   TwoSum (Knuth, TAOCP vol. 2, 4.2.2):  s + e = a + b exactly, s = fl(a + b);
//   TwoProduct (Dekker 1971, with a fused multiply-add):  p + e = a * b exactly,
//                                                          p = fl(a * b).
// Every FP32 operation here is an explicitly rounded one (no contraction into
// fused multiply-adds other than the written ones), which the error-free
// transformations need.  The header compiles as CUDA device/host code and as
// plain C++ (host tests build it with -ffp-contract=off).
#pragma once

#include <math.h>

#ifdef __CUDACC__
#define LQ_DF_FN __host__ __device__ __forceinline__
#else
#define LQ_DF_FN inline
#endif

namespace lq {

#if defined(__CUDA_ARCH__)
LQ_DF_FN float df_add_rn(float a, float b) { return __fadd_rn(a, b); }
LQ_DF_FN float df_sub_rn(float a, float b) { return __fsub_rn(a, b); }
LQ_DF_FN float df_mul_rn(float a, float b) { return __fmul_rn(a, b); }
LQ_DF_FN float df_fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
#else
LQ_DF_FN float df_add_rn(float a, float b) { return a + b; }
LQ_DF_FN float df_sub_rn(float a, float b) { return a - b; }
LQ_DF_FN float df_mul_rn(float a, float b) { return a * b; }
LQ_DF_FN float df_fma_rn(float a, float b, float c) { return fmaf(a, b, c); }
#endif

// s + e = a + b exactly (any a, b)
LQ_DF_FN void two_sum(float a, float b, float& s, float& e) {
  s = df_add_rn(a, b);
  const float bb = df_sub_rn(s, a);
  e = df_add_rn(df_sub_rn(a, df_sub_rn(s, bb)), df_sub_rn(b, bb));
}
// s + e = a + b exactly when |a| >= |b| (or a = 0)
LQ_DF_FN void fast_two_sum(float a, float b, float& s, float& e) {
  s = df_add_rn(a, b);
  e = df_sub_rn(b, df_sub_rn(s, a));
}
// p + e = a * b exactly (barring underflow)
LQ_DF_FN void two_prod(float a, float b, float& p, float& e) {
  p = df_mul_rn(a, b);
  e = df_fma_rn(a, b, -p);
}

// The operators are friends defined in the class, so that only argument-
// dependent lookup finds them: they never hide the standard fma() or
// arithmetic of float and double.
struct dfloat {
  float hi, lo;
  dfloat() = default;
  LQ_DF_FN dfloat(float h, float l) : hi(h), lo(l) {}
  // nearest double-float of a double: hi = fl32(x), lo = fl32(x - hi)
  LQ_DF_FN dfloat(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
  LQ_DF_FN dfloat(float x) : hi(x), lo(0.f) {}
  LQ_DF_FN dfloat(int x) : hi((float)x), lo(0.f) {}
  LQ_DF_FN double to_double() const { return (double)hi + (double)lo; }

  friend LQ_DF_FN dfloat operator+(dfloat a, dfloat b) {
    float s, e, t, f;
    two_sum(a.hi, b.hi, s, e);
    two_sum(a.lo, b.lo, t, f);
    e = df_add_rn(e, t);
    fast_two_sum(s, e, s, e);
    e = df_add_rn(e, f);
    fast_two_sum(s, e, s, e);
    return dfloat(s, e);
  }
  friend LQ_DF_FN dfloat operator-(dfloat a) { return dfloat(-a.hi, -a.lo); }
  friend LQ_DF_FN dfloat operator-(dfloat a, dfloat b) { return a + dfloat(-b.hi, -b.lo); }
  friend LQ_DF_FN dfloat operator*(dfloat a, dfloat b) {
    float p, e;
    two_prod(a.hi, b.hi, p, e);
    e = df_fma_rn(a.hi, b.lo, e);
    e = df_fma_rn(a.lo, b.hi, e);
    fast_two_sum(p, e, p, e);
    return dfloat(p, e);
  }
  friend LQ_DF_FN dfloat& operator+=(dfloat& a, dfloat b) {
    a = a + b;
    return a;
  }
  friend LQ_DF_FN dfloat fma(dfloat a, dfloat b, dfloat c) { return a * b + c; }
};

}  // namespace lq
