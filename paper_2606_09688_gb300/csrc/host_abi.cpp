// Host-only entry points of include/st_host.h.
#include <vector>

#include "../../include/st_host.h"
#include "host_math.h"

using namespace st;

extern "C" {

st_status st_host_time_matrices(int jt, double T, double* A, double* B, double* g1, double* d0) {
  if (jt < 0 || jt > 14 || !(T > 0) || !A || !B) return ST_ERR_ARG;
  TimeLevel tl;
  build_time_level(jt, T, tl);
  for (size_t e = 0; e < tl.A.size(); ++e) {
    A[e] = tl.A[e];
    B[e] = tl.B[e];
  }
  for (int i = 0; i < tl.nt; ++i) {
    if (g1) g1[i] = tl.g1[i];
    if (d0) d0[i] = tl.d0[i];
  }
  return ST_OK;
}

st_status st_host_time_matrices_p(int jt, double T, int p, double* A, double* B, double* g1, double* d0) {
  if (jt < 0 || jt > 14 || !(T > 0) || p < 2 || p > 4 || !A || !B) return ST_ERR_ARG;
  TimeLevel tl;
  build_time_level_p(jt, T, p, tl);
  for (size_t e = 0; e < tl.A.size(); ++e) {
    A[e] = tl.A[e];
    B[e] = tl.B[e];
  }
  for (int i = 0; i < tl.nt; ++i) {
    if (g1) g1[i] = tl.g1[i];
    if (d0) d0[i] = tl.d0[i];
  }
  return ST_OK;
}

st_status st_host_time_eig(int jt, double T, int* nsel, double* lam, double* cond_est, double* resid) {
  if (jt < 0 || jt > 10 || !(T > 0) || !nsel || !lam) return ST_ERR_ARG;
  TimeLevel tl;
  build_time_level(jt, T, tl);
  TimeEig e;
  if (!time_eig(tl, e)) return ST_ERR_NUMERIC;
  *nsel = e.nsel;
  for (int q = 0; q < e.nsel; ++q) {
    lam[2 * q] = e.lam[q].real();
    lam[2 * q + 1] = e.lam[q].imag();
  }
  if (cond_est) *cond_est = e.cond_est;
  if (resid) *resid = e.resid;
  return ST_OK;
}

st_status st_host_time_eig_p(int jt, double T, int p, int* nsel, double* lam, double* cond_est, double* resid) {
  if (jt < 0 || jt > 10 || !(T > 0) || p < 2 || p > 4 || !nsel || !lam) return ST_ERR_ARG;
  TimeLevel tl;
  build_time_level_p(jt, T, p, tl);
  TimeEig e;
  if (!time_eig(tl, e)) return ST_ERR_NUMERIC;
  *nsel = e.nsel;
  for (int q = 0; q < e.nsel; ++q) {
    lam[2 * q] = e.lam[q].real();
    lam[2 * q + 1] = e.lam[q].imag();
  }
  if (cond_est) *cond_est = e.cond_est;
  if (resid) *resid = e.resid;
  return ST_OK;
}

st_status st_host_components(int J, int mx, int mt, int* out) {
  if (J < 0 || !out) return ST_ERR_ARG;
  int k = 0;
  for (int a = 0; a <= J; ++a, ++k) {
    out[3 * k] = mx + a;
    out[3 * k + 1] = mt + J - a;
    out[3 * k + 2] = 1;
  }
  for (int a = 1; a <= J; ++a, ++k) {
    out[3 * k] = mx + a - 1;
    out[3 * k + 1] = mt + J - a;
    out[3 * k + 2] = -1;
  }
  return ST_OK;
}

st_status st_host_sym_gen_eig(int n, const double* K, const double* M, double* mu, double* Phi) {
  if (n <= 0 || n > 4096 || !K || !M || !mu || !Phi) return ST_ERR_ARG;
  std::vector<double> Kv(K, K + (size_t)n * n), Mv(M, M + (size_t)n * n), m, P;
  if (!sym_gen_eig(n, Kv, Mv, m, P)) return ST_ERR_NUMERIC;
  for (int i = 0; i < n; ++i) mu[i] = m[i];
  for (size_t e = 0; e < P.size(); ++e) Phi[e] = P[e];
  return ST_OK;
}

}  // extern "C"
