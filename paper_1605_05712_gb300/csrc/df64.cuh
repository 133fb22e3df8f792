// df64.cuh -- double-float arithmetic: a real number carried as the unevaluated sum hi + lo of two
// binary32 values, |lo| <= ulp(hi) / 2, about 48 significant bits.
//
// GB300 issues binary64 at 1/64 of the binary32 instruction rate.  The binary64-accurate solve
// (precision LAT_DF64) runs its FFT, Green operator, polarization and update on these pairs, on the
// binary32 pipes.  The error-free transformations are the textbook ones: Knuth's TwoSum, Dekker's
// FastTwoSum and the FMA-based exact product.  Every operation that must round exactly once uses the
// __f*_rn intrinsics, which the compiler never contracts into fused multiply-adds.
//
// Accuracy: addition is the "sloppy" pair sum (error <= about 2^-47 (|a| + |b|)), multiplication
// about 2^-46 |a b|, division two Newton-corrected quotients.  An FFT of length N then carries errors of
// order log2(N) 2^-47 relative to the input norm, four orders of magnitude below the 1e-10 tolerance
// against the binary64 reference.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

struct __align__(8) dfloat {
  float hi, lo;
  dfloat() = default;
  __host__ __device__ constexpr dfloat(float h, float l) : hi(h), lo(l) {}
  // integers: exact for |v| < 2^48 (frequencies here stay below 2^31)
  template <typename I, typename std::enable_if<std::is_integral<I>::value, int>::type = 0>
  __host__ __device__ constexpr dfloat(I v) : hi((float)v), lo((float)(v - (I)(float)v)) {}
  __host__ __device__ constexpr dfloat(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

struct __align__(16) dcplx {
  dfloat x, y;
};

#ifdef __CUDACC__  // the arithmetic is device code; host translation units see the types only

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// s + e = a + b exactly when |a| >= |b| (Dekker)
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ dfloat operator+(dfloat a, dfloat b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  dfloat r;
  fast_two_sum(s, e, r.hi, r.lo);
  return r;
}
__device__ __forceinline__ dfloat operator-(dfloat a) { return dfloat(-a.hi, -a.lo); }
__device__ __forceinline__ dfloat operator-(dfloat a, dfloat b) { return a + (-b); }
__device__ __forceinline__ dfloat operator*(dfloat a, dfloat b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);  // exact error of the product
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  dfloat r;
  fast_two_sum(p, e, r.hi, r.lo);
  return r;
}
__device__ __forceinline__ dfloat operator/(dfloat a, dfloat b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  const dfloat r = a - b * dfloat(q1, 0.f);
  const float q2 = __fdiv_rn(r.hi, b.hi);
  const dfloat r2 = r - b * dfloat(q2, 0.f);
  const float q3 = __fdiv_rn(r2.hi, b.hi);
  dfloat q;
  fast_two_sum(q1, q2, q.hi, q.lo);
  return q + dfloat(q3, 0.f);
}
__device__ __forceinline__ dfloat& operator+=(dfloat& a, dfloat b) { return a = a + b; }
__device__ __forceinline__ dfloat& operator-=(dfloat& a, dfloat b) { return a = a - b; }
__device__ __forceinline__ dfloat& operator*=(dfloat& a, dfloat b) { return a = a * b; }

// loads through the read-only path
__device__ __forceinline__ dfloat ldg_df(const dfloat* p) {
  const float2 v = __ldg((const float2*)p);
  return dfloat(v.x, v.y);
}
__device__ __forceinline__ dcplx ldg_dc(const dcplx* p) {
  const float4 v = __ldg((const float4*)p);
  dcplx r;
  r.x = dfloat(v.x, v.y);
  r.y = dfloat(v.z, v.w);
  return r;
}

// sum of squares accumulated as a pair: acc += x^2 for a pair x
__device__ __forceinline__ void df_acc_sq(dfloat& acc, dfloat x) { acc = acc + x * x; }
#endif  // __CUDACC__
