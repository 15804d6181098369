// Double-single arithmetic: a value held as the unevaluated sum h + l of two
// floats (48 significant bits), built from the error-free transformations of
// Dekker (1971, "A floating-point technique for extending the available
// precision") and Knuth (TAOCP vol. 2, 4.2.2, the two-sum).  Used by the
// combination kernels, where FP64 work per target value would bound the
// kernel by the FP64 pipe (1/64 of the FP32 rate on this device), not by the
// HBM writes.  Host and device: the host copies serve the CPU tests.
#pragma once
#include <cmath>
#include <cstdint>
#include <cstring>
#include <cuda_runtime.h>

namespace st {

struct alignas(8) ds {
  float h, l;
};

// Rounded float operations that the compiler may not contract or reorder.
__host__ __device__ __forceinline__ float f_add(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fadd_rn(a, b);
#else
  volatile float r = a + b;
  return r;
#endif
}
__host__ __device__ __forceinline__ float f_sub(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fsub_rn(a, b);
#else
  volatile float r = a - b;
  return r;
#endif
}
__host__ __device__ __forceinline__ float f_mul(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fmul_rn(a, b);
#else
  volatile float r = a * b;
  return r;
#endif
}
__host__ __device__ __forceinline__ float f_fma(float a, float b, float c) {
#ifdef __CUDA_ARCH__
  return __fmaf_rn(a, b, c);
#else
  return std::fma(a, b, c);
#endif
}

// s + e = a + b exactly, s = fl(a + b) (Knuth's two-sum, no ordering needed).
__host__ __device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = f_add(a, b);
  const float bb = f_sub(s, a);
  e = f_add(f_sub(a, f_sub(s, bb)), f_sub(b, bb));
}

// x + y without renormalisation (|l| may grow to a few units of h's last place).
__host__ __device__ __forceinline__ ds ds_add(ds x, ds y) {
  float s, e;
  two_sum(x.h, y.h, s, e);
  return ds{s, f_add(e, f_add(x.l, y.l))};
}

// Renormalised pair: h = fl(h + l), |l| <= half an ulp of h.
__host__ __device__ __forceinline__ ds ds_norm(ds x) {
  ds r;
  two_sum(x.h, x.l, r.h, r.l);
  return r;
}

// x * 2^k for k = -1, -2 (exact unless the pair underflows).
__host__ __device__ __forceinline__ ds ds_scale(ds x, float p2) { return ds{f_mul(x.h, p2), f_mul(x.l, p2)}; }

// acc (S + lo) += w * c, with w a float (an exact dyadic B-spline weight) and
// c a pair: w c.h = p + pe exactly (FMA residual), p enters S by two-sum, the
// rest (two-sum error, pe, w c.l) accumulates in lo.
__host__ __device__ __forceinline__ void ds_axpy(float w, ds c, float& S, float& lo) {
  const float p = f_mul(w, c.h);
  const float pe = f_fma(w, c.h, -p);
  float se;
  two_sum(S, p, S, se);
  lo = f_add(lo, f_add(se, f_fma(w, c.l, pe)));
}

// Nearest pair of a double: h = fl32(v), l = fl32(v - h).
__host__ __device__ __forceinline__ ds ds_from_double(double v) {
  const float h = (float)v;
  return ds{h, (float)(v - (double)h)};
}

__host__ __device__ __forceinline__ uint32_t f_bits(float x) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(x);
#else
  uint32_t u;
  std::memcpy(&u, &x, 4);
  return u;
#endif
}
__host__ __device__ __forceinline__ float bits_f(uint32_t u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float x;
  std::memcpy(&x, &u, 4);
  return x;
#endif
}
__host__ __device__ __forceinline__ int f2i_rn(float x) {
#ifdef __CUDA_ARCH__
  return __float2int_rn(x);
#else
  return (int)std::nearbyint(x);
#endif
}
__host__ __device__ __forceinline__ double ll_bits_d(uint64_t u) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)u);
#else
  double x;
  std::memcpy(&x, &u, 8);
  return x;
#endif
}

// The double nearest (to within one unit in its last place) to h + l for a
// renormalised pair (|l| <= half an ulp of h), formed with integer and float
// operations only: the exact double of |h| (its exponent re-biased, its
// significand shifted into place), plus l counted in units of the last place
// of that double, k = round(l sign(h) 2^(52 - e_h)), |k| <= 2^28, then h's sign.
// When h is a power of two and l points towards zero, the result lies in the
// binade below, whose unit is half as large, so k is doubled.  For
// |h| < 2^-74 the scale 2^(52 - e) is beyond the float range and is applied in
// two factors (2^64 first).  h = 0 or subnormal gives a signed zero;
// infinities and NaN give NaN.
__host__ __device__ __forceinline__ double ds_to_double(ds x) {
  const uint32_t hb = f_bits(x.h);
  const uint32_t sgn = hb & 0x80000000u;
  const uint32_t mag = hb & 0x7fffffffu;
  const uint32_t e8 = mag >> 23;
  if (e8 == 0u || e8 == 0xffu) return ll_bits_d(((uint64_t)sgn << 32) | (e8 == 0u ? 0ull : 0x7ff8000000000000ull));
  const uint32_t hw = (mag >> 3) + 0x38000000u;
  const uint32_t lw = mag << 29;
  const bool small = e8 < 53u;
  const uint32_t fe = small ? 242u - e8 : 306u - e8;  // float exponent field of 2^(52 - e) (/ 2^64 if small)
  float lm = bits_f(f_bits(x.l) ^ sgn);               // l relative to the sign of h
  if (small) lm = f_mul(lm, 18446744073709551616.0f);
  int k = f2i_rn(f_mul(lm, bits_f(fe << 23)));
  if ((mag & 0x007fffffu) == 0u && k < 0) k *= 2;
  const uint64_t r = ((((uint64_t)hw << 32) | (uint64_t)lw) + (uint64_t)(int64_t)k) | ((uint64_t)sgn << 32);
  return ll_bits_d(r);
}

}  // namespace st
