// Launch wrappers of the space-time solver kernels (kernels.cu).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"
#include "dsfloat.h"
#include "param_grid.h"

namespace st {

enum StencilOp { OP_APPLY = 0, OP_RESID = 1, OP_JACOBI = 2, OP_JACOBI_ZERO = 3 };

// Per-mode state of the batched COCG iteration (device memory).
struct CocgScal {
  double rho_re, rho_im;     // r . z  (bilinear)
  double alpha_re, alpha_im;
  double beta_re, beta_im;
  double rr, bb;             // ||r||^2, ||b||^2
  float alpha_f[2], beta_f[2];  // the same step lengths for FP32 kernels (no per-thread conversion)
  int active, iters, status, pad;
};

// y_q = op((K(c2) + lam_q M) x_q) for every active mode q of a level.
template <typename R>
void launch_stencil(int op, const Geo& g, const StencilCoefT<R>& sc, const R* c2, const cx<R>* x,
                    const cx<R>* b, cx<R>* y, const cx<R>* lam, const CocgScal* scal, int nmodes,
                    int64_t stride, double omega, cudaStream_t s);

// dinv_q = omega / diag(K(c2) + lam_q M) of a level for every mode (mode-major,
// vectors at q * stride), for the Jacobi sweeps through StencilCoefT::dinv.
template <typename R>
void launch_jacobi_dinv(const Geo& g, const StencilCoefT<R>& sc, const R* c2, const cx<R>* lam, double omega,
                        int nmodes, int64_t stride, cx<R>* dinv, cudaStream_t s);

// Multigrid transfers between level gf (fine) and gc = coarse (N/2).
template <typename R>
void launch_restrict(const Geo& gf, const Geo& gc, const cx<R>* rf, cx<R>* bc, const CocgScal* scal, int nmodes,
                     int64_t sf, int64_t scs, cudaStream_t s);
template <typename R>
void launch_prolong_add(const Geo& gf, const Geo& gc, const cx<R>* xc, cx<R>* xf, const CocgScal* scal, int nmodes,
                        int64_t sf, int64_t scs, cudaStream_t s);

// COCG vector steps with deterministic two-pass reductions.
template <typename R>
void launch_cocg_init(const cx<R>* b, cx<R>* x, cx<R>* r, CocgScal* scal, double* part, int nmodes, int64_t n,
                      int64_t stride, cudaStream_t s);
template <typename R>
void launch_dot(int which, const cx<R>* a, const cx<R>* b, CocgScal* scal, double* part, int nmodes, int64_t n,
                int64_t stride, double tol, int max_iter, cudaStream_t s);
template <typename R>
// The convergence test rr <= tol^2 bb takes tol from tolp[0] (device) when tolp is set.
void launch_update_xr(cx<R>* x, cx<R>* r, const cx<R>* p, const cx<R>* w, CocgScal* scal, double* part,
                      int nmodes, int64_t n, int64_t stride, double tol, int max_iter, cudaStream_t s,
                      const double* tolp = nullptr);
void launch_set_scalar(double* p, double v, cudaStream_t s);

// Inner (COCG) tolerance of the refinement sweeps.  The first sweep solves to
// `base`; with FP64 inner solves a later sweep only has to reduce the
// space-time backward error eta by target / eta, and a relative modal
// residual eps changes the space-time residual by at most amp eps (amp from
// the conditioning of the time eigenbasis), so it solves to
// eps = 0.05 target / (eta amp), kept within [base, 1e-2].
__host__ __device__ inline double next_inner_tol(double base, double target, double eta, double amp) {
  if (!(eta > 0.0) || !(eta < 1e300)) return base;
  const double t = 0.05 * target / (eta * amp);
  return fmin(1e-2, fmax(base, t));
}
struct InnerTol {
  double* tol;    // device scalar read by the COCG convergence test (null: fixed tolerance)
  double base;    // tolerance of the first sweep
  double amp;     // residual amplification bound of the transforms
  int adaptive;   // 0: every sweep solves to base
};
template <typename R>
void launch_update_p(cx<R>* p, const cx<R>* z, const CocgScal* scal, int nmodes, int64_t n, int64_t stride,
                     int first, cudaStream_t s);
void launch_cocg_activate(CocgScal* scal, int nmodes, cudaStream_t s);
// Sets the condition of a graph WHILE node: non-zero while any mode is active;
// bodies (device, may be null) counts the calls.
void launch_cocg_continue(const CocgScal* scal, int nmodes, cudaGraphConditionalHandle handle, int* bodies,
                          cudaStream_t s);

// Record of a component solve that runs entirely on the device: one CUDA
// graph whose WHILE node runs the refinement sweeps (each with its COCG loop in
// a nested WHILE node) and whose stopping test is taken by k_refine_decide.
struct RefineRec {
  double eta, rel, eta_prev;  // backward error and relative residual of the last sweep; the sweep before
  int sweeps, status, max_iters, inner_bodies;
};
enum { RR_OK = 0, RR_NUMERIC = 1, RR_ITER_LIMIT = 2, RR_TIMEOUT = 3 };
// Clears the record; the sweep loop runs when ||F||^2 (fn2[0]) is positive.
void launch_refine_init(RefineRec* rec, const double* fn2, cudaGraphConditionalHandle h, InnerTol it,
                        cudaStream_t s);
// After a sweep: nrm2 = (||R||^2, ||U||^2), fn2 = ||F||^2.  Stops on
// eta = ||R|| / (snorm ||U|| + ||F||) <= tol, when eta no longer halves, after
// max_sweeps, on a COCG status word (scal may be null), a copy timeout
// (cerr[0] != 0, may be null) or a non-finite residual.
void launch_refine_decide(RefineRec* rec, const double* nrm2, const double* fn2, double snorm, double tol,
                          int max_sweeps, const CocgScal* scal, int nsel, const int* cerr,
                          cudaGraphConditionalHandle h, InnerTol it, cudaStream_t s);

// Time transforms of the eigenbasis method (FP64 matrices):
// G[q][a] = sum_i W[q][i] R[i][a];  U[i][a] += sum_q w_q Re(V[i][q] X[q][a]).
template <typename R>
void launch_fwd_transform(const cx<double>* W, const double* Rt, cx<R>* G, int nsel, int nt, int64_t nx,
                          cudaStream_t s);
template <typename R>
void launch_back_transform(const cx<double>* V, const double* wq, const cx<R>* X, double* U, int nsel, int nt,
                           int64_t nx, cudaStream_t s);

// FP64 space-time residual R = F - (A (x) M + B (x) K) U (banded time factors).
void launch_residual(const Geo& g, const StencilCoef& sc, const double* c2, const double* U, const double* F,
                     const double* Aband, const double* Bband, double* KU, double* MU, double* Rout, int nt,
                     cudaStream_t s);
// Sum of squares of a real vector (deterministic), result to out[0] (device).
void launch_norm2(const double* v, int64_t n, double* part, double* out, cudaStream_t s);

// Loads of Q1-interpolated data: out = alphaK K_load x + alphaM M_load x with x on ALL nodes.
void launch_load(const Geo& g, const StencilCoef& sc, const double* c2, const double* xall, double* out,
                 double alphaK, double alphaM, int accumulate, cudaStream_t s);
// F[i][a] = sum_r coef[r][i] L[r][a]  (rank-nterm assembly)
void launch_rhs_assemble(const double* coef, const double* L, double* F, int nterm, int nt, int64_t nx,
                         cudaStream_t s);

// Space eigenbasis method: Y = X Phi (trans = 0) or Y = X Phi^T (trans = 1),
// X nt x nx, Phi nx x nx; then banded time solves per spatial mode.
void launch_gemm_right(const double* X, const double* Phi, double* Y, int nt, int64_t nx, int trans, int accumulate,
                       cudaStream_t s);
// Band LU factors per spatial mode a: ab[a][j][0..6] = column j of the band
// (LAPACK band layout, kl = ku = 2, row i of column j at 4 + i - j), the
// diagonal entry replaced by its reciprocal; piv[a][j].  Returns false (and
// launches nothing) when the mode's factor does not fit in shared memory
// (time_band_smem(nt) > kTimeBandMaxSmem) or the bandwidths differ.
constexpr size_t kTimeBandMaxSmem = 200 * 1024;
size_t time_band_smem(int nt);
bool launch_time_band_solve(const double* ab, const int* piv, double* Y, int nt, int64_t nx, int kl, int ku,
                            cudaStream_t s);

// Combination kernel (Eq. (19)) on a nodal target grid.
struct CombComp {
  const double* U;     // nt x nx interior coefficients (FP64)
  const double* lift;  // u0 on all nodes of level jx, or nullptr
  int jx, jt, coef, pad;
};
// One level of the hierarchical combination: Y = P Yprev + sum over
// components c0..c1-1 (all at spatial level >= j, listed in comps) of
// coef * u_k(., t_s) on the (2^j+1)^d nodes of level j, for every target time.
// tbv[c][s][0..2]: the three B-spline values of component c at target time s,
// tspan[c][s] their interval.  Yprev (level j-1, all nodes x nts) may be null.
void launch_comb_level(int d, int j, const double* Yprev, const CombComp* comps, int c0, int c1, const double* tbv,
                       const int* tspan, int nts, double* Y, cudaStream_t s);
// The same level in double-single arithmetic (combine_ds.cu): Yprev and, below
// the target level, Y hold float pairs (8 bytes per value); the target level
// (final_level) is written as FP64.  comps: per component its coefficient
// pairs with the coefficient's sign applied and u0 folded in, and coef u0 on
// all nodes of its level (from launch_comb_prep_ds).  tbw: the B-spline
// weights as floats, exact (the caller checks that every weight is
// representable).  L: target times per chunk, from comb_ds_chunk (comp_jt:
// time levels of the level's components, in table order).
struct CombCompDS {
  const ds* U;     // nt x nx interior pairs: coef (U + u0)
  const ds* lift;  // coef u0 on all nodes of level jx, or nullptr
  int jx, jt;
};
void launch_comb_prep_ds(int d, const double* U, const double* lift, int coef, int jx, int nt, ds* Uds, ds* Lds,
                         cudaStream_t s);
void launch_comb_level_ds(int d, int j, const void* Yprev, const CombCompDS* comps, int c0, int c1, const float* tbw,
                          const int* tspan, int nts, int L, void* Y, bool final_level, cudaStream_t s);
int comb_ds_chunk(int d, int j, int jt_star, const int* comp_jt, int ncomp_level);

// Coarsest multigrid level by an explicit inverse (grids of at most a few
// thousand unknowns): x_q = Ainv_q b_q for every active mode, Ainv_q the
// n x n inverse of mode q at q * n * n (row r contiguous).
template <typename R>
void launch_dense_coarse(const cx<R>* Ainv, int64_t n, const cx<R>* b, cx<R>* x, const CocgScal* scal, int nmodes,
                         int64_t vstride, cudaStream_t s);
// I (n x n identity, column j at j * n): right-hand sides of the inversion.
template <typename R> void launch_identity(cx<R>* I, int64_t n, cudaStream_t s);

// ------------------------------------------------ receiver misfit gradient
// Corner of the cell holding a receiver at one component's level: interior
// node index (-1 on the boundary), all-node index, multilinear weight.
struct RecCorner {
  int interior;
  int all;
  double w;
};
// ParamGrid: the uniform grid of nodal parameters (param_grid.h).
// Element stiffness of one cell with c^2 = 1 (2^d x 2^d, local corner c has
// bit k set at the upper end in direction k).
struct ElemK {
  double k[64];
};
// out[s][r] = sum_c coef_c u_c(x_r, t_s) for all target times s (nts) and receivers r.
void launch_receiver_eval(const CombComp* comps, int ncomp, const RecCorner* rc, int nrec, int ncorner,
                          const double* tbv, const int* tspan, int nts, double* out, cudaStream_t s);
// wm[s][r] = w_s (vals - dobs)[s][r] with trapezoid weights on [0, T]; J = 1/2 sum w_s e^2 -> Jout[0].
void launch_misfit(const double* vals, const double* dobs, int nts, int nrec, double T, double* wm, double* Jout,
                   cudaStream_t s);
// G (nt x nx) += coef sum_s sum_r psi_i(t_s) phi_a(x_r) wm[s][r] for one component (G zeroed by the caller).
void launch_adjoint_rhs(const double* wm, int nts, int nrec, const double* tb, const int* tspan, int nt,
                        const RecCorner* rc, int ncorner, double coef, int64_t nx, double* ehat, double* G,
                        cudaStream_t s);
// dc2 (param nodes) += P^T g with g_e = -sum_ij B[i][j] L_i^T K_e U_j per cell e of the level.
void launch_grad_c2(const Geo& g, const double* lo, int nt, const double* Bband, const double* U, const double* L,
                    const ElemK& ke, const ParamGrid& pg, double* dc2, cudaStream_t s);
// dg (param nodes) += Q^T M_load^T sum_i b[i] L_i (v: scratch of nx doubles).
void launch_grad_g(const Geo& g, const double* lo, const StencilCoef& sc, int nt, const double* b, const double* L,
                   double* v, const ParamGrid& pg, double* dg, cudaStream_t s);

// Energy of Section 6.3 per time: out[b] = 1/2 sum_e (z_e^T Me z_e + c2_e y_e^T Ke y_e) over
// the N^d cells of a level (y, z on all (N+1)^d nodes, ntimes rows of nall); part:
// scratch of ntimes x ceil(N^d / 256) doubles.
void launch_energy_cells(int d, int N, const double* c2, const double* y, const double* z, int64_t nall, int ntimes,
                         const ElemK& me, const ElemK& ke, double* part, double* out, cudaStream_t s);

// Stencil autotuner: times the launch shapes of one stencil operation on the
// given buffers (synchronises the stream) and keeps the fastest for later
// launch_stencil calls with the same operation, dimension, precision, grid
// size and mode count.  Returns the chosen time in ms, 0 if already tuned, < 0
// on failure.
template <typename R>
float tune_stencil(int op, const Geo& g, const StencilCoefT<R>& sc, const R* c2, const cx<R>* x, const cx<R>* b,
                   cx<R>* y, const cx<R>* lam, int nmodes, int64_t stride, double omega, cudaStream_t s);
// The tuned shapes: 7 ints per entry (op, d, element size, nodes, modes, modes per thread, block); returns the count.
int tuned_stencil_shapes(int* out, int max_entries);
// Pin one shape (same fields); false if the shape is not a valid candidate.
bool set_stencil_shape(int op, int d, int rsize, int64_t nnodes, int nmodes, int mq, int block);

// Kernels launched by this process through the wrappers above.
int64_t kernel_launch_count();
void note_launches(int k);

}  // namespace st
