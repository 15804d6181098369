// Banded complex-symmetric LDL^T of K + lam M (see band.cu).
//
// No pivoting is needed: for Im lam != 0 the matrix -i (K + lam M) has the
// positive definite Hermitian part Im(lam) M, and for real lam > 0 the matrix
// K + lam M is symmetric positive definite, so every leading principal minor
// is non-singular.  The eigenvalues of B^{-1} A are either non-real or real
// and positive (checked in setup).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"

namespace st {

struct BandLayout {
  int64_t nrow;     // unknowns of the grid
  int bw;           // half bandwidth: 1 (1D), n+1 (2D), n^2+n+1 (3D)
  int ld;           // row length in elements: bw + 1 rounded up to even
  int64_t mstride;  // elements per mode (multiple of 32)
  long long wait;   // cycle budget of the single-warp solve's copy waits (0 = 2^31)
  int stall;        // fault injection (tests): the single-warp solve withholds its first copy
  int pad;
};

BandLayout band_layout(int64_t nrow, int bw);
int band_chunk_rows(const BandLayout& L, size_t elem);

template <typename R>
void launch_band_form(const double* Kb, const double* Mb, const cx<double>* lam, cx<R>* F, const BandLayout& L,
                      int nmodes, cudaStream_t s);
// LDL^T of every mode's F in place, then G (rows of L) from F.  err[0] = 1 on a zero pivot.
template <typename R>
void launch_band_factor(cx<R>* F, cx<R>* G, const BandLayout& L, int nmodes, int* err, cudaStream_t s);
// x_q = (L D L^T)^{-1} b_q for every active mode (vectors at q * vstride);
// x may alias nothing but itself.  err[0] = 2 if a copy wait timed out.
// Returns false when bw exceeds 1024 (not supported).
template <typename R>
bool launch_band_solve(const cx<R>* F, const cx<R>* G, const BandLayout& L, const cx<R>* b, cx<R>* x,
                       const CocgScal* scal, int nmodes, int64_t vstride, int* err, cudaStream_t s);

// Blocked solve for half bandwidths up to 128 (2D grids up to 127^2, 3D up
// to 7^3).  Rows are grouped into blocks of s = 32 rt >= bw rows, so L is
// block lower bidiagonal: y_i = L_ii^{-1} (b_i - L_{i,i-1} y_{i-1}) forward and
// x_i = L_ii^{-T} (D_i^{-1} y_i - L_{i+1,i}^T x_{i+1}) backward.  The inverses
// X_i = L_ii^{-1} are formed once (FP64 arithmetic), and every operand of the
// two sweeps is laid out as a stream of 32 x 32 tiles in the order the solve
// consumes them (per block and phase the triangle's off-diagonal tiles, then
// its diagonal tiles), which the solve copies into shared memory ahead of use.
struct BlkLayout {
  int rt;           // 32-row tiles per block
  int s;            // rows per block (32 rt)
  int nb;           // blocks: ceil(nrow / s)
  int pad;
  int64_t tstride;  // elements per mode: 4 nb (tiles per phase) 1024
};
// Layout for L, or rt = 0 when the bandwidth is too wide for the blocked solve.
BlkLayout blk_layout(const BandLayout& L);
// Tile streams S (nmodes x tstride) from the factors F of launch_band_factor.
template <typename R>
void launch_band_blk_prepare(const cx<R>* F, const BandLayout& L, const BlkLayout& B, cx<R>* S, int nmodes,
                             cudaStream_t s);
// x_q = (L D L^T)^{-1} b_q for every active mode with the blocked solve;
// x may alias nothing.  err[0] = 2 if a copy wait timed out.
template <typename R>
void launch_band_solve_blk(const cx<R>* F, const BandLayout& L, const BlkLayout& B, const cx<R>* S, const cx<R>* b,
                           cx<R>* x, const CocgScal* scal, int nmodes, int64_t vstride, int* err, cudaStream_t s);

}  // namespace st
