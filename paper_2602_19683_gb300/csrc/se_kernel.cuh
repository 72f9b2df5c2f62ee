// Squared-exponential covariance entries k(x, x') = v exp(-|x - x'|^2 / (2 l^2)) (Eq. 1) at FP64
// accuracy with little FP64 issue. On GB300 the FP64 pipe issues two operations per clock per SM, and
// the textbook evaluation (2D FP64 operations for the distance, about twenty for the exponential) makes
// every assembly-type kernel FP64-issue bound. Here:
//
//  * the squared distance is exact integer arithmetic on the integer pipe: coordinates are quantised
//    once to a common fixed point q = round(x 2^F) with |q| < 2^58, and sum_d (q_d - q'_d)^2 is formed
//    exactly in 128 bits and rounded once to FP64 (integer operations only). The quantisation step
//    2^-F <= 2^-57 S (S = the largest |coordinate|) perturbs r^2 by at most 2 |x - x'|_1 2^-F, far
//    below the FP64 evaluation's own rounding whenever S is within 2^6 lengthscales (FxScale::usable);
//    other inputs take the FP64 distance;
//  * the exponential of the non-positive argument is a table-driven evaluation after Tang (ACM TOMS
//    15(2), 1989): x = (1024 m + j) ln2/1024 + r with |r| <= ln2/2048, exp(x) = 2^m 2^(j/1024) exp(r),
//    2^(j/1024) from a head/tail table (exp_table.cuh, written by gen_exp_table.py), exp(r) - 1 by a
//    degree-4 polynomial (truncation below 2^-60), 2^m applied to the exponent field with integer
//    operations. About ten FP64 operations; results within one ulp of exp (checked against CUDA's exp in
//    tests/test_gpu_se_kernel.py).
#pragma once
#include <string.h>

#include "common.cuh"
#include "exp_table.cuh"

namespace gpk {

// exp(x) for x <= 0 (or NaN): NaN -> NaN, x < -745.2 -> +0, subnormal results rounded once.
__device__ __forceinline__ double exp_neg(double x) {
  if (!(x > -745.2)) return x != x ? x : 0.0;
  const double t = x * kExpInvLn2xN;
  const double kN = t + 0x1.8p52;  // round t to an integer N held in the low mantissa bits
  const int N = __double2loint(kN);
  const double Nd = kN - 0x1.8p52;
  double r = fma(-Nd, kExpLn2byNHi, x);  // exact: Nd * head has at most 53 significant bits
  r = fma(-Nd, kExpLn2byNLo, r);
  // exp(r) - 1 = r + r^2 (1/2 + r/6 + r^2/24), |r| <= ln2/2048: the omitted r^5/120 term is < 2^-62
  double q = fma(r, 1.0 / 24.0, 1.0 / 6.0);
  q = fma(q, r, 0.5);
  const double p = fma(q, r * r, r);
  const int j = N & ((1 << kExpTableBits) - 1), m = N >> kExpTableBits;  // floor division
  const double h = __ldg(kExp2Head + j);
  const double res = h + fma(h, p, __ldg(kExp2Tail + j));  // in [1 - 2^-11, 2)
  if (m >= -1021)
    return __hiloint2double(__double2hiint(res) + m * (1 << 20), __double2loint(res));
  // subnormal result: scale to a normal number, then one rounding multiplication
  return __hiloint2double(__double2hiint(res) + (m + 600) * (1 << 20), __double2loint(res)) * 0x1p-600;
}

struct U128 {
  unsigned long long lo, hi;
};

// High 64 bits of u * u and leading zeros of a nonzero word, on the device and on the host (the host
// build serves the exactness test of these routines).
__host__ __device__ __forceinline__ unsigned long long fx_mulhi(unsigned long long u) {
#ifdef __CUDA_ARCH__
  return __umul64hi(u, u);
#else
  return (unsigned long long)(((unsigned __int128)u * u) >> 64);
#endif
}
__host__ __device__ __forceinline__ int fx_clz(unsigned long long x) {
#ifdef __CUDA_ARCH__
  return __clzll((long long)x);
#else
  return __builtin_clzll(x);
#endif
}

// s += (qa - qb)^2 exactly (|qa|, |qb| < 2^58, so the square is below 2^118 and D <= 256 terms fit).
__host__ __device__ __forceinline__ void fx_add_sq(U128& s, long long qa, long long qb) {
  const long long t = qa - qb;
  const unsigned long long u = (unsigned long long)(t < 0 ? -t : t);
  const unsigned long long lo = u * u, hi = fx_mulhi(u);
  s.lo += lo;
  s.hi += hi + (s.lo < lo ? 1ull : 0ull);
}

// s 2^(-twoF) rounded to nearest-even FP64, with integer operations (the result is assumed normal or
// zero: twoF <= 1022 and s < 2^128).
__host__ __device__ __forceinline__ double fx_to_double(U128 s, int twoF) {
  if ((s.hi | s.lo) == 0ull) return 0.0;
  const int lz = s.hi ? fx_clz(s.hi) : 64 + fx_clz(s.lo);
  unsigned long long h, l;  // s << lz: the leading one at bit 127
  if (lz == 0) {
    h = s.hi;
    l = s.lo;
  } else if (lz < 64) {
    h = (s.hi << lz) | (s.lo >> (64 - lz));
    l = s.lo << lz;
  } else {
    h = s.lo << (lz - 64);
    l = 0ull;
  }
  unsigned long long mant = h >> 11;  // 53 bits, leading one included
  const unsigned long long rem = h & 0x7FFull;
  if (rem > 0x400ull || (rem == 0x400ull && (l != 0ull || (mant & 1ull)))) ++mant;
  int e = (127 - lz) - twoF;  // value = mant 2^(e - 52)
  if (mant >> 53) {
    mant >>= 1;
    ++e;
  }
  const unsigned long long bits = ((unsigned long long)(e + 1023) << 52) | (mant & 0xFFFFFFFFFFFFFull);
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)bits);
#else
  double r;
  memcpy(&r, &bits, sizeof(r));
  return r;
#endif
}

}  // namespace gpk
