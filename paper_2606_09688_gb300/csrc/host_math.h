// Host-side FP64 building blocks of the setup phase (no GPU needed).
//
// Time direction (Section 2.2 and the proof of Prop. 1, Section 4.1):
//   psi_i = B_i, i = 1..N+1, quadratic B-splines on the open uniform knot
//   vector of N intervals of (0,T), B_0 removed so that w(0) = 0;
//   A[i][j] = (psi_j'', psi_i')_e + psi_j'(0) psi_i'(0),
//   B[i][j] = (psi_j,   psi_i')_e,  (u,v)_e = int_0^T u v exp(-t/T) dt.
// The time system is diagonalised through the eigenpairs of B^{-1} A (Eq. (30)
// with the time basis changed to eigenvectors).
#pragma once
#include <complex>
#include <cstdint>
#include <vector>

namespace st {

using cplx = std::complex<double>;

// n-point Gauss-Legendre rule on [-1,1] (Newton iteration on P_n).
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w);

// Values, first and second derivatives of the three quadratic B-splines that
// are non-zero on interval k of the uniform open knot vector with N intervals
// on (0,T).  Global indices of the three functions are k, k+1, k+2 (B_0 first).
void bspline_local(int N, double T, int k, double t, double val[3], double d1[3], double d2[3]);
// Interval holding t (the last interval is closed).
int bspline_span(int N, double T, double t);

struct TimeLevel {
  int jt = 0, N = 0, nt = 0;       // N = 2^jt intervals, nt = N + 1 unknowns
  double T = 1.0;
  std::vector<double> A, B;        // nt x nt, row-major, row = test index
  std::vector<double> qt, qw;      // quadrature times and weights (8 per interval)
  std::vector<double> Q;           // nt x nq: w_q exp(-t_q/T) psi_i'(t_q)
  std::vector<double> g1;          // (1, psi_i')_e
  std::vector<double> d0;          // psi_i'(0)
};
void build_time_level(int jt, double T, TimeLevel& tl);

// Splines of degree p (2..4) with maximal regularity C^{p-1}: the p + 1
// B-splines non-zero on interval k of the open uniform knot vector (p + 1
// copies of 0 and of T) have global indices k .. k + p (B_0 first); their
// values and first and second derivatives at t, by the Cox-de Boor recursion
// on that interval.
void bspline_local_p(int N, double T, int p, int k, double t, double* val, double* d1, double* d2);
// The time level with splines of degree p (nt = N + p - 1; p = 2 gives the
// quadratic level of build_time_level up to rounding).
void build_time_level_p(int jt, double T, int p, TimeLevel& tl);

// Eigen-decomposition of C = B^{-1} A (real, nt x nt).  Keeps one eigenvalue
// of each complex-conjugate pair (Im > 0) and every real one; V holds the
// matching eigenvectors (real ones scaled to be real), W the matching rows of
// V^{-1} B^{-1}, where V is the full eigenvector matrix with each kept complex
// column followed by its conjugate.  Then
//   U = sum_real V_q (W_q F) + 2 Re sum_complex V_q (W_q F)  solves the
// time-diagonalised system.  Returns false on failure (no convergence).
struct TimeEig {
  int nt = 0, nsel = 0;
  std::vector<cplx> lam;           // nsel
  std::vector<cplx> V;             // nt x nsel, column q = eigenvector of lam[q]
  std::vector<cplx> W;             // nsel x nt
  std::vector<double> weight;      // 1 (real) or 2 (complex pair)
  double cond_est = 0.0;           // ||V||_1 ||V^{-1}||_1 of the full V
  double resid = 0.0;              // ||C V - V Lam||_F / (||C||_F ||V||_F)
};
bool time_eig(const TimeLevel& tl, TimeEig& out);

// Dense real linear algebra helpers.
bool lu_solve_real(int n, std::vector<double> A, std::vector<double>& B, int nrhs);  // B <- A^{-1} B
bool lu_inverse_cplx(int n, std::vector<cplx> A, std::vector<cplx>& Ainv);

// Complex Schur form of an upper Hessenberg matrix by shifted QR; H is
// overwritten by the triangular factor, Z accumulates the unitary transform.
bool complex_schur(int n, std::vector<cplx>& H, std::vector<cplx>& Z);

// Symmetric-definite generalized eigenproblem K v = mu M v (dense, n x n):
// Phi (n x n, row-major, column a = eigenvector a) with Phi^T M Phi = I.
bool sym_gen_eig(int n, const std::vector<double>& K, const std::vector<double>& M,
                 std::vector<double>& mu, std::vector<double>& Phi);

// Banded LU with partial pivoting of an n x n matrix with kl sub- and ku
// super-diagonals (LAPACK gbtrf layout: ab has ldab = 2 kl + ku + 1 rows,
// column-major, entry (i,j) at ab[(kl + ku + i - j) + j * ldab]).
bool band_lu(int n, int kl, int ku, std::vector<double>& ab, std::vector<int>& piv);

}  // namespace st
