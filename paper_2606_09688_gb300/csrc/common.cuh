// Device-side types shared by the kernels of the space-time solver.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace st {

// Interleaved complex number; 16-byte (double) or 8-byte (float) aligned so
// that one element moves with one vector load.
template <typename R> struct alignas(2 * sizeof(R)) cx {
  R re, im;
};

template <typename R> __host__ __device__ __forceinline__ cx<R> mk(R a, R b) { return cx<R>{a, b}; }
template <typename R> __host__ __device__ __forceinline__ cx<R> operator+(cx<R> a, cx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <typename R> __host__ __device__ __forceinline__ cx<R> operator-(cx<R> a, cx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <typename R> __host__ __device__ __forceinline__ cx<R> operator*(cx<R> a, cx<R> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename R> __host__ __device__ __forceinline__ cx<R> operator*(R s, cx<R> a) { return {s * a.re, s * a.im}; }
template <typename R> __host__ __device__ __forceinline__ cx<R> cdiv(cx<R> a, cx<R> b) {
  const R den = b.re * b.re + b.im * b.im;
  return {(a.re * b.re + a.im * b.im) / den, (a.im * b.re - a.re * b.im) / den};
}
// a + s * b with real s
template <typename R> __host__ __device__ __forceinline__ cx<R> fma_s(R s, cx<R> b, cx<R> a) {
  return {fma(s, b.re, a.re), fma(s, b.im, a.im)};
}
// a + c * b with complex c
template <typename R> __host__ __device__ __forceinline__ cx<R> fma_c(cx<R> c, cx<R> b, cx<R> a) {
  return {fma(c.re, b.re, fma(-c.im, b.im, a.re)), fma(c.re, b.im, fma(c.im, b.re, a.im))};
}

// Division of a 32-bit unsigned a < 2^31 by a fixed divisor d >= 1 with one
// high multiply (Granlund and Montgomery, 1994): l = ceil(log2 d),
// m = floor(2^32 (2^l - d) / d) + 1, a / d = (umulhi(a, m) + a) >> l.
struct FastDiv {
  unsigned d, m, l;
};
inline FastDiv make_fastdiv(unsigned d) {
  FastDiv f;
  f.d = d;
  f.l = 0;
  while ((1ull << f.l) < d) ++f.l;
  f.m = (unsigned)((((1ull << 32) * ((1ull << f.l) - d)) / d) + 1ull);
  return f;
}
__device__ __forceinline__ unsigned fdiv(unsigned a, const FastDiv& f) { return (__umulhi(a, f.m) + a) >> f.l; }

// Uniform tensor grid of one spatial level: N = 2^j cells per direction, the
// interior nodes (Dirichlet unknowns) number n = N - 1 per direction and are
// ordered lexicographically with the first coordinate fastest.
struct Geo {
  int d;
  int N;              // cells per direction
  int n;              // interior nodes per direction
  int64_t nnodes;     // n^d
  int64_t ncells;     // N^d
  FastDiv dn;         // division by n
};

// Q1 stencil of a node with its 3^d neighbours (offset delta in {-1,0,1}^d,
// index sum_k (delta_k + 1) 3^k).  For the stiffness, the entry between a
// node and its neighbour is (sum of c^2 over the cells that hold both) x ke,
// since the element matrix entry only depends on delta; the mass entry is
// the assembled constant mtot (cell count included).
template <typename R> struct StencilCoefT {
  R ke[27];
  R mtot[27];
  // damped inverse diagonal omega / (K + lam_q M)_aa per mode and node of a
  // multigrid level (mode-major, the level's vector stride), used by the FP64
  // Jacobi sweeps when set; null = formed on the fly
  const cx<R>* dinv = nullptr;
};
using StencilCoef = StencilCoefT<double>;
inline StencilCoefT<float> to_float(const StencilCoef& s) {
  StencilCoefT<float> f;
  for (int i = 0; i < 27; ++i) {
    f.ke[i] = (float)s.ke[i];
    f.mtot[i] = (float)s.mtot[i];
  }
  return f;
}

__host__ __device__ constexpr int ipow3(int d) { return d == 0 ? 1 : 3 * ipow3(d - 1); }

}  // namespace st
