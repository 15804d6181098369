/*
 * st_host.h -- host-only building blocks of st_setup (no GPU needed).
 *
 * They expose the FP64 setup math of the library so that it can be checked on
 * a machine without a GPU.  All arrays are caller-owned host memory, row-major.
 * Every call returns ST_OK or ST_ERR_ARG (bad sizes) / ST_ERR_NUMERIC.
 */
#ifndef ST_HOST_H_
#define ST_HOST_H_

#include "st.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Time matrices of level jt on (0,T) (proof of Prop. 1, Section 4.1):
 * A[i][j] = (psi_j'', psi_i')_e + psi_j'(0) psi_i'(0), B[i][j] = (psi_j, psi_i')_e,
 * g1[i] = (1, psi_i')_e, d0[i] = psi_i'(0); n_t = 2^jt + 1. */
st_status st_host_time_matrices(int jt, double T, double* A, double* B, double* g1, double* d0);
/* The same matrices for time splines of degree p = 2, 3 or 4 with maximal
 * regularity C^{p-1} (the spaces of Table "validity": proven for p = 2,
 * conjectured for 3 and 4; dimension n_t = 2^jt + p - 1 by the formula of
 * Section 3.2).  A and B: caller-owned host arrays of n_t x n_t doubles
 * (row-major, row = test index); g1, d0: n_t doubles or NULL.  ST_ERR_ARG for
 * jt outside 0..14, T <= 0, p outside 2..4 or a NULL A or B.  Host set-up
 * math only: the solves of the library use p = 2. */
st_status st_host_time_matrices_p(int jt, double T, int p, double* A, double* B, double* g1, double* d0);

/* Eigen-decomposition of B^{-1} A used by the time eigenbasis method: the
 * kept eigenvalues (one of each conjugate pair, Im > 0, and the real ones),
 * as interleaved (re, im) pairs in lam[2 * nsel] (caller provides 2 * n_t),
 * the 1-norm condition estimate of the eigenvector matrix and the relative
 * eigen-residual. */
st_status st_host_time_eig(int jt, double T, int* nsel, double* lam, double* cond_est, double* resid);
/* The same eigen-decomposition for time splines of degree p = 2, 3 or 4
 * (n_t = 2^jt + p - 1; lam holds 2 n_t doubles).  ST_ERR_ARG for jt outside
 * 0..10, T <= 0, p outside 2..4 or NULL nsel / lam; ST_ERR_NUMERIC when the
 * QR iteration does not converge.  Host set-up math only. */
st_status st_host_time_eig_p(int jt, double T, int p, int* nsel, double* lam, double* cond_est, double* resid);

/* Component list of Eq. (19): out[3k .. 3k+2] = (j_x, j_t, coefficient), k < 2J+1. */
st_status st_host_components(int J, int mx, int mt, int* out);

/* Symmetric-definite K v = mu M v (n x n dense): mu[n], Phi[n x n] (columns
 * are M-orthonormal eigenvectors). */
st_status st_host_sym_gen_eig(int n, const double* K, const double* M, double* mu, double* Phi);

/* The FP64 value the combination kernels write for a double-single pair
 * (h[i], l[i]) (a float pair whose unevaluated sum carries 48 significant
 * bits, |l| at most half an ulp of h): out[i] = h + l to within one unit in
 * the last place, formed with integer and float operations only, the same
 * routine the device runs.  ST_ERR_ARG for n < 0 or null arrays. */
st_status st_host_ds_to_double(const float* h, const float* l, int64_t n, double* out);

#ifdef __cplusplus
}
#endif
#endif /* ST_HOST_H_ */
