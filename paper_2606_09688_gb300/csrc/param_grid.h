// Nodal parameter fields on the uniform grid of one level of the box (the
// parameters of the receiver-misfit gradient): the multilinear weights of a
// point, one definition for the forward sampling (st_setup, host) and for its
// transpose in the gradient kernels (device).
#pragma once
#include <cmath>
#include <cuda_runtime.h>

namespace st {

// Uniform grid of nodal parameters on the domain box: Np cells per direction.
struct ParamGrid {
  int d, Np;
  double lo[3], h[3];
};

// node[e], w[e] (e < 2^D): the (Np+1)^D-grid nodes (x fastest) of the cell
// holding x and their multilinear weights; points on or outside the box edge
// use the nearest cell (its local coordinate extrapolated).
template <int D>
__host__ __device__ inline void param_weights(const ParamGrid& pg, const double x[3], int node[8], double w[8]) {
  int c[3];
  double f[3];
  for (int k = 0; k < D; ++k) {
    const double t = (x[k] - pg.lo[k]) / pg.h[k];
    int ci = (int)floor(t);
    ci = ci < 0 ? 0 : (ci > pg.Np - 1 ? pg.Np - 1 : ci);
    c[k] = ci;
    f[k] = t - ci;
  }
  for (int e = 0; e < (1 << D); ++e) {
    double ww = 1.0;
    int idx = 0, st = 1;
    for (int k = 0; k < D; ++k) {
      const int b = (e >> k) & 1;
      ww *= b ? f[k] : 1.0 - f[k];
      idx += (c[k] + b) * st;
      st *= pg.Np + 1;
    }
    node[e] = idx;
    w[e] = ww;
  }
}

// The interpolant's value at x: sum_e w[e] vals[node[e]].
template <int D> __host__ __device__ inline double param_eval(const ParamGrid& pg, const double* vals, const double x[3]) {
  int node[8];
  double w[8];
  param_weights<D>(pg, x, node, w);
  double v = 0.0;
  for (int e = 0; e < (1 << D); ++e) v += w[e] * vals[node[e]];
  return v;
}

}  // namespace st
