// Quadratic B-splines on the open uniform knot vector of N intervals of
// (0,T): values and derivatives of the three functions that are non-zero on
// one interval (host and device).  Used by the setup (time matrices) and by
// the combination kernel (evaluation of the time factor at target times).
#pragma once
#include <cuda_runtime.h>

namespace st {

// Knot t_i of the vector 0,0,0,h,2h,...,T,T,T (i = 0..N+4).
__host__ __device__ inline double bs_knot(int N, double T, int i) {
  if (i <= 2) return 0.0;
  if (i >= N + 2) return T;
  return (double)(i - 2) * (T / N);
}

// On interval k (knot span s = k + 2) the non-zero degree-2 functions are
// B_{s-2}, B_{s-1}, B_s.  Degree-1 functions B_{s-1,1}, B_{s,1} are the only
// non-zero ones of degree 1; degree 2 and its derivatives follow from the
// two-term recursion and B'_{i,p} = p/(t_{i+p}-t_i) B_{i,p-1} - p/(t_{i+p+1}-t_{i+1}) B_{i+1,p-1}.
__host__ __device__ inline void bs_local(int N, double T, int k, double t, double val[3], double d1[3],
                                         double d2[3]) {
  const int s = k + 2;
  const double ks = bs_knot(N, T, s), ks1 = bs_knot(N, T, s + 1);
  const double len = ks1 - ks;
  // degree-1 values/derivatives of B_{s-1,1} and B_{s,1}
  const double b1m = (ks1 - t) / len, b1s = (t - ks) / len;
  const double db1m = -1.0 / len, db1s = 1.0 / len;
  for (int a = 0; a < 3; ++a) {
    const int i = s - 2 + a;
    const double l1 = bs_knot(N, T, i + 2) - bs_knot(N, T, i);
    const double l2 = bs_knot(N, T, i + 3) - bs_knot(N, T, i + 1);
    // B_{i,1} and B_{i+1,1} on this span
    const double bi = (i == s - 1) ? b1m : (i == s ? b1s : 0.0);
    const double bi1 = (i + 1 == s - 1) ? b1m : (i + 1 == s ? b1s : 0.0);
    const double dbi = (i == s - 1) ? db1m : (i == s ? db1s : 0.0);
    const double dbi1 = (i + 1 == s - 1) ? db1m : (i + 1 == s ? db1s : 0.0);
    double v = 0.0, dv = 0.0, ddv = 0.0;
    if (l1 > 0) {
      v += (t - bs_knot(N, T, i)) / l1 * bi;
      dv += 2.0 / l1 * bi;
      ddv += 2.0 / l1 * dbi;
    }
    if (l2 > 0) {
      v += (bs_knot(N, T, i + 3) - t) / l2 * bi1;
      dv -= 2.0 / l2 * bi1;
      ddv -= 2.0 / l2 * dbi1;
    }
    val[a] = v;
    d1[a] = dv;
    d2[a] = ddv;
  }
}

}  // namespace st
