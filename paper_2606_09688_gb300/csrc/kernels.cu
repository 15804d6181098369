// CUDA kernels of the space-time sparse-grid wave solver (sm_103a).
//
// Every kernel works on the uniform Q1 grids of one spatial level (see Geo
// in common.cuh).  Complex vectors of the time eigenbasis are stored
// mode-major: element (q, a) at q * stride + a.
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <atomic>
#include <cstdio>

#include "bspline.h"
#include "kernels.h"
#include "param_grid.h"

namespace st {

namespace {

constexpr int kBlock = 256;
constexpr int kRedBlocks = 304;  // two CTAs per SM for the reduction passes

inline unsigned blocks_for(int64_t n, int per = kBlock) { return (unsigned)((n + per - 1) / per); }

std::atomic<int64_t> g_launches{0};
inline void count(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

// Interior node index -> coordinates (node counts stay below 2^31).
template <int D> __device__ __forceinline__ void decode(int64_t a64, const Geo& g, int i[3]) {
  const unsigned a = (unsigned)a64;
  const unsigned q1 = fdiv(a, g.dn);
  i[0] = (int)(a - q1 * (unsigned)g.n);
  if (D > 1) {
    const unsigned q2 = fdiv(q1, g.dn);
    i[1] = (int)(q1 - q2 * (unsigned)g.n);
    if (D > 2) i[2] = (int)q2;
  }
}

// Sums of c^2 over the cells shared by a node and each of its 3^D neighbours.
// The 2^D cells around interior node i are i + e, e in {0,1}^D (cell
// coordinates); neighbour delta shares cell e iff, per direction, delta = +1
// needs e = 1, delta = -1 needs e = 0 and delta = 0 takes both.
template <int D, typename R>
__device__ __forceinline__ void cell_sums(const R* __restrict__ c2, int N, const int i[3], R* S) {
  constexpr int NC = 1 << D, NS = ipow3(D);
  R c[NC];
#pragma unroll
  for (int e = 0; e < NC; ++e) {
    int64_t idx = 0, stride = 1;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      idx += (int64_t)(i[k] + ((e >> k) & 1)) * stride;
      stride *= N;
    }
    c[e] = __ldg(c2 + idx);
  }
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    R acc = R(0);
#pragma unroll
    for (int e = 0; e < NC; ++e) {
      bool ok = true;
      int ss = s;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const int dk = ss % 3 - 1;
        ss /= 3;
        const int ek = (e >> k) & 1;
        ok = ok && (dk == 0 || (dk == 1 && ek == 1) || (dk == -1 && ek == 0));
      }
      if (ok) acc += c[e];
    }
    S[s] = acc;
  }
}

template <int D> __device__ __forceinline__ bool neighbour(const int i[3], int s, int n, int64_t& off) {
  off = 0;
  int64_t stride = 1;
  bool ok = true;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const int dk = s % 3 - 1;
    s /= 3;
    const int j = i[k] + dk;
    ok = ok && (j >= 0) && (j < n);
    off += (int64_t)dk * stride;
    stride *= n;
  }
  return ok;
}

// ------------------------------------------------------------------ stencils
// Reciprocal for the damping of a Jacobi sweep: the fast approximate FP32
// division (2 ulp) in FP32 sweeps, whose smoothing only feeds FP64
// refinement; the correctly rounded one in FP64.
__device__ __forceinline__ float rcp_rn(float v) { return __fdividef(1.0f, v); }
__device__ __forceinline__ double rcp_rn(double v) { return __drcp_rn(v); }

// The value of the lane below / above (lane 0 and lane 31 get their own).
template <typename R> __device__ __forceinline__ cx<R> shfl_up1(cx<R> v) {
  return mk<R>(__shfl_up_sync(0xffffffffu, v.re, 1), __shfl_up_sync(0xffffffffu, v.im, 1));
}
template <typename R> __device__ __forceinline__ cx<R> shfl_down1(cx<R> v) {
  return mk<R>(__shfl_down_sync(0xffffffffu, v.re, 1), __shfl_down_sync(0xffffffffu, v.im, 1));
}

// s * a / b with one reciprocal of |b|^2 (two divisions in the textbook form).
template <typename R> __device__ __forceinline__ cx<R> scaled_div(R s, cx<R> a, cx<R> b) {
  const R w = s * rcp_rn(fma(b.re, b.re, b.im * b.im));
  return mk<R>(w * fma(a.re, b.re, a.im * b.im), w * fma(a.im, b.re, -a.re * b.im));
}

// One thread per interior node and MQ time modes: the node's row of the
// stiffness (c^2 cell sums times the element entries) and its neighbour
// offsets are formed once and applied to every mode of the group, so the
// per-mode cost is the 3^D loads and the complex FMAs.
template <int D, typename R, int OP, int MQ>
__global__ void __launch_bounds__(512) k_stencil(Geo g, StencilCoefT<R> sc, const R* __restrict__ c2,
                                                    const cx<R>* __restrict__ x, const cx<R>* __restrict__ b,
                                                    cx<R>* __restrict__ y, const cx<R>* __restrict__ lam,
                                                    const CocgScal* __restrict__ scal, int nmodes, int64_t stride,
                                                    R omega) {
  const int q0 = blockIdx.y * MQ;
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= g.nnodes) return;
  constexpr int NS = ipow3(D), CEN = (NS - 1) / 2;
  int i[3] = {0, 0, 0};
  decode<D>(a, g, i);
  R kr[NS];
  cell_sums<D, R>(c2, g.N, i, kr);
#pragma unroll
  for (int s = 0; s < NS; ++s) kr[s] *= sc.ke[s];
  int off[NS];
  unsigned valid = 0u;
  if (OP != OP_JACOBI_ZERO) {
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      int64_t o;
      if (neighbour<D>(i, s, g.n, o)) valid |= 1u << s;
      off[s] = (int)o;
    }
  }
#pragma unroll
  for (int m = 0; m < MQ; ++m) {
    const int q = q0 + m;
    if (q >= nmodes) break;
    if (scal != nullptr && !scal[q].active) continue;
    const cx<R> l = lam[q];
    const cx<R> diag = fma_s(sc.mtot[CEN], l, mk<R>(kr[CEN], R(0)));
    const int64_t base = (int64_t)q * stride + a;
    if (OP == OP_JACOBI_ZERO) {
      y[base] = (sizeof(R) == 8 && sc.dinv != nullptr) ? sc.dinv[base] * b[base] : scaled_div(omega, b[base], diag);
      continue;
    }
    cx<R> ak = mk<R>(0, 0), am = mk<R>(0, 0);
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      if ((valid >> s) & 1u) {
        const cx<R> v = x[base + off[s]];
        ak = fma_s(kr[s], v, ak);
        am = fma_s(sc.mtot[s], v, am);
      }
    }
    const cx<R> Ax = fma_c(l, am, ak);
    if (OP == OP_APPLY) {
      y[base] = Ax;
    } else if (OP == OP_RESID) {
      y[base] = b[base] - Ax;
    } else {  // OP_JACOBI
      const cx<R> xo = x[base];
      const cx<R> r = b[base] - Ax;
      y[base] = (sizeof(R) == 8 && sc.dinv != nullptr) ? fma_c(sc.dinv[base], r, xo) : xo + scaled_div(omega, r, diag);
    }
  }
}

// Damped inverse diagonal omega / (K(c2) + lam_q M)_aa of a level for every
// mode (set-up; the same diagonal as the sweeps form on the fly).
template <int D, typename R>
__global__ void k_jacobi_dinv(Geo g, StencilCoefT<R> sc, const R* __restrict__ c2, const cx<R>* __restrict__ lam,
                              R omega, int64_t stride, cx<R>* __restrict__ dinv) {
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= g.nnodes) return;
  constexpr int NS = ipow3(D), CEN = (NS - 1) / 2;
  int i[3] = {0, 0, 0};
  decode<D>(a, g, i);
  R kr[NS];
  cell_sums<D, R>(c2, g.N, i, kr);
  const int q = blockIdx.y;
  const cx<R> diag = fma_s(sc.mtot[CEN], lam[q], mk<R>(kr[CEN] * sc.ke[CEN], R(0)));
  dinv[(int64_t)q * stride + a] = cdiv(mk<R>(omega, R(0)), diag);
}

// 2D variant with the operand staged in shared memory: a CTA takes a
// 64 x 8 tile of interior nodes and MQ modes, loads the tile's x values with a
// one-node halo (zero outside the interior) and the c^2 of its 65 x 9 cells
// with coalesced row loads, then forms each node's row and applies it from
// shared memory (one global load per node and mode instead of nine).
constexpr int kTileX = 64, kTileY = 8;
template <typename R, int OP, int MQ>
__global__ void __launch_bounds__(256) k_stencil_tile2(Geo g, StencilCoefT<R> sc, const R* __restrict__ c2,
                                                       const cx<R>* __restrict__ x, const cx<R>* __restrict__ b,
                                                       cx<R>* __restrict__ y, const cx<R>* __restrict__ lam,
                                                       const CocgScal* __restrict__ scal, int nmodes,
                                                       int64_t stride, R omega) {
  __shared__ cx<R> xs[MQ][kTileY + 2][kTileX + 2];
  __shared__ R cs[kTileY + 1][kTileX + 1];
  const int x0 = blockIdx.x * kTileX, y0 = blockIdx.y * kTileY, q0 = blockIdx.z * MQ;
  const int n = g.n, N = g.N, tid = threadIdx.x;
  const cx<R> zero = mk<R>(0, 0);
  for (int e = tid; e < (kTileX + 1) * (kTileY + 1); e += blockDim.x) {
    const int hx = e % (kTileX + 1), hy = e / (kTileX + 1);
    const int cx_ = x0 + hx, cy = y0 + hy;
    cs[hy][hx] = (cx_ < N && cy < N) ? c2[(int64_t)cy * N + cx_] : R(0);
  }
#pragma unroll
  for (int m = 0; m < MQ; ++m) {
    const int q = q0 + m;
    const bool act = q < nmodes && (scal == nullptr || scal[q].active);
    const cx<R>* xq = x + (int64_t)(act ? q : 0) * stride;
    for (int e = tid; e < (kTileX + 2) * (kTileY + 2); e += blockDim.x) {
      const int hx = e % (kTileX + 2), hy = e / (kTileX + 2);
      const int gx = x0 + hx - 1, gy = y0 + hy - 1;
      xs[m][hy][hx] = (act && gx >= 0 && gx < n && gy >= 0 && gy < n) ? xq[(int64_t)gy * n + gx] : zero;
    }
  }
  __syncthreads();
  const int tx = tid % kTileX;
  for (int r = tid / kTileX; r < kTileY; r += blockDim.x / kTileX) {
    const int ix = x0 + tx, iy = y0 + r;
    if (ix >= n || iy >= n) continue;
    const R c00 = cs[r][tx], c10 = cs[r][tx + 1], c01 = cs[r + 1][tx], c11 = cs[r + 1][tx + 1];
    R kr[9];
    kr[0] = c00;
    kr[1] = c00 + c10;
    kr[2] = c10;
    kr[3] = c00 + c01;
    kr[4] = (c00 + c10) + (c01 + c11);
    kr[5] = c10 + c11;
    kr[6] = c01;
    kr[7] = c01 + c11;
    kr[8] = c11;
#pragma unroll
    for (int s2 = 0; s2 < 9; ++s2) kr[s2] *= sc.ke[s2];
    const int64_t a = (int64_t)iy * n + ix;
#pragma unroll
    for (int m = 0; m < MQ; ++m) {
      const int q = q0 + m;
      if (q >= nmodes) break;
      if (scal != nullptr && !scal[q].active) continue;
      const cx<R> l = lam[q];
      const cx<R> diag = fma_s(sc.mtot[4], l, mk<R>(kr[4], R(0)));
      const int64_t base = (int64_t)q * stride + a;
      cx<R> ak = mk<R>(0, 0), am = mk<R>(0, 0);
#pragma unroll
      for (int s2 = 0; s2 < 9; ++s2) {
        const cx<R> v = xs[m][r + s2 / 3][tx + s2 % 3];
        ak = fma_s(kr[s2], v, ak);
        am = fma_s(sc.mtot[s2], v, am);
      }
      const cx<R> Ax = fma_c(l, am, ak);
      if (OP == OP_APPLY) {
        y[base] = Ax;
      } else if (OP == OP_RESID) {
        y[base] = b[base] - Ax;
      } else {  // OP_JACOBI
        const cx<R> res = b[base] - Ax;
        y[base] = (sizeof(R) == 8 && sc.dinv != nullptr) ? fma_c(sc.dinv[base], res, xs[m][r + 1][tx + 1])
                                     : xs[m][r + 1][tx + 1] + scaled_div(omega, res, diag);
      }
    }
  }
}

// 2D variant streaming down columns: a warp owns 30 consecutive columns of
// interior nodes (its lanes 0 and 31 hold the halo columns) and walks a strip
// of `rows` rows (as many strips as fill the device once).  The x values of
// rows i-1, i, i+1 and the c^2 cells of cell rows i, i+1 roll in registers;
// the left and right neighbours of a new row come from the adjacent lanes by
// warp shuffles.  Per node and mode the kernel reads x and b once and writes y
// once (three global requests instead of nine).  The loads of x, b and c^2 run
// PF rows ahead of the row being computed, so that a warp keeps PF rows of
// requests in flight instead of waiting one load latency per row.
constexpr int kColWarps = 4, kColOut = 30;
template <typename R, int OP, int MQ>
__global__ void __launch_bounds__(32 * kColWarps, sizeof(R) == 4 && MQ == 1 ? 5 : 1) k_stencil_col2(Geo g, StencilCoefT<R> sc, const R* __restrict__ c2,
                                                                  const cx<R>* __restrict__ x,
                                                                  const cx<R>* __restrict__ b, cx<R>* __restrict__ y,
                                                                  const cx<R>* __restrict__ lam,
                                                                  const CocgScal* __restrict__ scal, int nmodes,
                                                                  int64_t stride, R omega, int rows) {
  constexpr int PF = MQ >= 4 ? 1 : (MQ >= 2 ? 2 : 4);  // rows of loads in flight ahead of the computed row
  const int n = g.n, N = g.N;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ix = (blockIdx.x * kColWarps + warp) * kColOut - 1 + lane;
  const int r0 = blockIdx.y * rows;
  const int q0 = blockIdx.z * MQ;
  const bool colok = ix >= 0 && ix < n;
  const bool cellok = ix >= 0 && ix < N;
  const bool writer = lane >= 1 && lane <= kColOut && colok;
  const cx<R> zero = mk<R>(0, 0);
  bool act[MQ];
  const cx<R>* xq[MQ];
  const cx<R>* bq[MQ];
#pragma unroll
  for (int m = 0; m < MQ; ++m) {
    const int q = q0 + m;
    act[m] = q < nmodes && (scal == nullptr || scal[q].active);
    xq[m] = x + (int64_t)(act[m] ? q : 0) * stride;
    bq[m] = b + (int64_t)(act[m] ? q : 0) * stride;
  }
  auto ldx = [&](int m, int row) -> cx<R> {
    return (act[m] && colok && row >= 0 && row < n) ? xq[m][(int64_t)row * n + ix] : zero;
  };
  auto ldb = [&](int m, int row) -> cx<R> {
    return (OP != OP_APPLY && act[m] && writer && row < n) ? bq[m][(int64_t)row * n + ix] : zero;
  };
  auto ldc = [&](int row) -> R { return (cellok && row >= 0 && row < N) ? c2[(int64_t)row * N + ix] : R(0); };
  // rows r0-1, r0, r0+1 of x, cell rows r0, r0+1, and the queues of the next PF rows
  cx<R> xa[MQ], xb[MQ], xc[MQ], xf[PF][MQ], bf[PF][MQ];
  R cf[PF];
#pragma unroll
  for (int m = 0; m < MQ; ++m) {
    xa[m] = ldx(m, r0 - 1);
    xb[m] = ldx(m, r0);
    xc[m] = ldx(m, r0 + 1);
  }
  R ca = ldc(r0), cb = ldc(r0 + 1);
#pragma unroll
  for (int f = 0; f < PF; ++f) {
#pragma unroll
    for (int m = 0; m < MQ; ++m) {
      xf[f][m] = ldx(m, r0 + 2 + f);
      bf[f][m] = ldb(m, r0 + f);
    }
    cf[f] = ldc(r0 + 2 + f);
  }
  // neighbours (left, right) of rows r0-1 and r0 from the adjacent lanes;
  // h = left + 4 centre + right of a row: the mass stencil is
  // m0 (1, 4, 1) (x) (1, 4, 1), so M x = m0 (h(i-1) + h(i+1)) + 4 m0 h(i)
  cx<R> la[MQ], ra[MQ], lb[MQ], rb[MQ], lc[MQ], rc[MQ], ha[MQ], hb[MQ];
  const R m0 = sc.mtot[0], m3 = sc.mtot[3];
  R car, cbr;  // cells of column ix + 1
  {
#pragma unroll
    for (int m = 0; m < MQ; ++m) {
      la[m] = shfl_up1(xa[m]);
      ra[m] = shfl_down1(xa[m]);
      lb[m] = shfl_up1(xb[m]);
      rb[m] = shfl_down1(xb[m]);
      ha[m] = fma_s(R(4), xa[m], la[m] + ra[m]);
      hb[m] = fma_s(R(4), xb[m], lb[m] + rb[m]);
    }
    car = __shfl_down_sync(0xffffffffu, ca, 1);
    cbr = __shfl_down_sync(0xffffffffu, cb, 1);
  }
  const int rend = min(r0 + rows, n);
  // in the row loop every access of a mode's vectors is at one 32-bit node
  // offset (row n + ix, advanced by n per row) from the mode's base
  // pointer, and the refills at fixed distances ahead of it
  bool okx[MQ], okb[MQ];
  cx<R>* yq[MQ];
  cx<R> lq[MQ];
#pragma unroll
  for (int m = 0; m < MQ; ++m) {
    okx[m] = act[m] && colok;
    okb[m] = OP != OP_APPLY && act[m] && writer;
    yq[m] = y + (int64_t)(act[m] ? q0 + m : 0) * stride;
    lq[m] = act[m] ? lam[q0 + m] : zero;
  }
  const int dx = (2 + PF) * n, dbn = PF * n;
  int oy = r0 * n + ix;
  int oc = (r0 + 2 + PF) * N + ix;
  // rows in groups of PF: queue slot f is refilled right after it is used,
  // with no register moves of loads still in flight
  for (int row0 = r0; row0 < rend; row0 += PF) {
#pragma unroll
    for (int f = 0; f < PF; ++f) {
      const int row = row0 + f;
      if (row >= rend) break;
      // neighbours of row + 1 and the right cell of its cell row
#pragma unroll
      for (int m = 0; m < MQ; ++m) {
        lc[m] = shfl_up1(xc[m]);
        rc[m] = shfl_down1(xc[m]);
      }
      const R cnr = __shfl_down_sync(0xffffffffu, cf[f], 1);
      cx<R> hc[MQ];
#pragma unroll
      for (int m = 0; m < MQ; ++m) hc[m] = fma_s(R(4), xc[m], lc[m] + rc[m]);
      if (writer) {
        // cells of the node (ix, row): (ix, row), (ix+1, row), (ix, row+1), (ix+1, row+1)
        const R c00 = ca, c10 = car, c01 = cb, c11 = cbr;
        R kr[9];
        kr[0] = c00;
        kr[1] = c00 + c10;
        kr[2] = c10;
        kr[3] = c00 + c01;
        kr[4] = (c00 + c10) + (c01 + c11);
        kr[5] = c10 + c11;
        kr[6] = c01;
        kr[7] = c01 + c11;
        kr[8] = c11;
#pragma unroll
        for (int s2 = 0; s2 < 9; ++s2) kr[s2] *= sc.ke[s2];
#pragma unroll
        for (int m = 0; m < MQ; ++m) {
          if (!act[m]) continue;
          const cx<R> l = lq[m];
          const cx<R> v[9] = {la[m], xa[m], ra[m], lb[m], xb[m], rb[m], lc[m], xc[m], rc[m]};
          // three short chains instead of one of nine (latency, not issue, bounds a row)
          const cx<R> k0 = fma_s(kr[2], v[2], fma_s(kr[1], v[1], kr[0] * v[0]));
          const cx<R> k1 = fma_s(kr[5], v[5], fma_s(kr[4], v[4], kr[3] * v[3]));
          const cx<R> k2 = fma_s(kr[8], v[8], fma_s(kr[7], v[7], kr[6] * v[6]));
          const cx<R> ak = (k0 + k1) + k2;
          const cx<R> am = fma_s(m3, hb[m], m0 * (ha[m] + hc[m]));
          const cx<R> Ax = fma_c(l, am, ak);
          if (OP == OP_APPLY) {
            yq[m][oy] = Ax;
          } else if (OP == OP_RESID) {
            yq[m][oy] = bf[f][m] - Ax;
          } else {  // OP_JACOBI
            const cx<R> res = bf[f][m] - Ax;
            if ((sizeof(R) == 8 && sc.dinv != nullptr)) {
              yq[m][oy] = fma_c(sc.dinv[(int64_t)(q0 + m) * stride + oy], res, xb[m]);
            } else {
              const cx<R> diag = fma_s(sc.mtot[4], l, mk<R>(kr[4], R(0)));
              yq[m][oy] = xb[m] + scaled_div(omega, res, diag);
            }
          }
        }
      }
      // roll the rows; refill slot f PF rows ahead
#pragma unroll
      for (int m = 0; m < MQ; ++m) {
        ha[m] = hb[m];
        hb[m] = hc[m];
        xa[m] = xb[m];
        la[m] = lb[m];
        ra[m] = rb[m];
        xb[m] = xc[m];
        lb[m] = lc[m];
        rb[m] = rc[m];
        xc[m] = xf[f][m];
        xf[f][m] = (okx[m] && row + 2 + PF < n) ? xq[m][oy + dx] : zero;
        bf[f][m] = (okb[m] && row + PF < n) ? bq[m][oy + dbn] : zero;
      }
      ca = cb;
      car = cbr;
      cb = cf[f];
      cbr = cnr;
      cf[f] = (cellok && row + 2 + PF < N) ? c2[oc] : R(0);
      oy += n;
      oc += N;
    }
  }
}

// CTAs of a column-streaming kernel resident on the whole device at once
// (resident CTAs per SM at 32 kColWarps threads x SMs), cached per kernel
// (the template arguments) and device ordinal.
template <typename R, int OP, int MQ> int resident_ctas() {
  static std::atomic<int> cache[64];
  auto kernel = k_stencil_col2<R, OP, MQ>;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
  const bool cached = dev >= 0 && dev < 64;
  int v = cached ? cache[dev].load(std::memory_order_relaxed) : 0;
  if (v > 0) return v;
  int per_sm = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 32 * kColWarps, 0) != cudaSuccess) per_sm = 1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) sms = 1;
  v = std::max(1, per_sm) * std::max(1, sms);
  if (cached) cache[dev].store(v, std::memory_order_relaxed);
  return v;
}

// Rows per strip: as many strips as fill the device's resident CTAs once
// (a second, partly filled wave of strips would cost a whole strip time),
// at least 8 rows so that the rows loaded ahead of a strip stay a small part.
inline int col_rows(int n, int col_groups, int mode_groups, int slots) {
  const int strips = std::max(1, slots / std::max(1, col_groups * mode_groups));
  return std::max(8, (n + strips - 1) / strips);
}

template <typename R, int MQ>
void stencil_col2_mq(int op, const Geo& g, const StencilCoefT<R>& sc, const R* c2, const cx<R>* x, const cx<R>* b,
                     cx<R>* y, const cx<R>* lam, const CocgScal* scal, int nmodes, int64_t stride, double omega,
                     cudaStream_t s) {
  const int warps = (g.n + kColOut - 1) / kColOut;
  const int cg = (warps + kColWarps - 1) / kColWarps, mg = (nmodes + MQ - 1) / MQ;
  auto kern = op == OP_APPLY ? k_stencil_col2<R, OP_APPLY, MQ>
                             : (op == OP_RESID ? k_stencil_col2<R, OP_RESID, MQ> : k_stencil_col2<R, OP_JACOBI, MQ>);
  const int slots = op == OP_APPLY ? resident_ctas<R, OP_APPLY, MQ>()
                                   : (op == OP_RESID ? resident_ctas<R, OP_RESID, MQ>() : resident_ctas<R, OP_JACOBI, MQ>());
  const int rows = col_rows(g.n, cg, mg, slots);
  const dim3 grid(cg, (g.n + rows - 1) / rows, mg);
  kern<<<grid, 32 * kColWarps, 0, s>>>(g, sc, c2, x, b, y, lam, scal, nmodes, stride, (R)omega, rows);
}

template <typename R, int MQ>
void stencil_tile2_mq(int op, const Geo& g, const StencilCoefT<R>& sc, const R* c2, const cx<R>* x, const cx<R>* b,
                      cx<R>* y, const cx<R>* lam, const CocgScal* scal, int nmodes, int64_t stride, double omega,
                      cudaStream_t s) {
  const dim3 grid((g.n + kTileX - 1) / kTileX, (g.n + kTileY - 1) / kTileY, (nmodes + MQ - 1) / MQ);
  const R om = (R)omega;
  if (op == OP_APPLY)
    k_stencil_tile2<R, OP_APPLY, MQ><<<grid, 256, 0, s>>>(g, sc, c2, x, b, y, lam, scal, nmodes, stride, om);
  else if (op == OP_RESID)
    k_stencil_tile2<R, OP_RESID, MQ><<<grid, 256, 0, s>>>(g, sc, c2, x, b, y, lam, scal, nmodes, stride, om);
  else
    k_stencil_tile2<R, OP_JACOBI, MQ><<<grid, 256, 0, s>>>(g, sc, c2, x, b, y, lam, scal, nmodes, stride, om);
}

template <int D, typename R, int MQ>
void stencil_dispatch_mq(int op, const Geo& g, const StencilCoefT<R>& sc, const R* c2, const cx<R>* x, const cx<R>* b,
                         cx<R>* y, const cx<R>* lam, const CocgScal* scal, int nmodes, int64_t stride, double omega,
                         int block, cudaStream_t s) {
  dim3 grid(blocks_for(g.nnodes, block), (nmodes + MQ - 1) / MQ);
  const R om = (R)omega;
  switch (op) {
    case OP_APPLY:
      k_stencil<D, R, OP_APPLY, MQ><<<grid, block, 0, s>>>(g, sc, c2, x, b, y, lam, scal, nmodes, stride, om);
      break;
    case OP_RESID:
      k_stencil<D, R, OP_RESID, MQ><<<grid, block, 0, s>>>(g, sc, c2, x, b, y, lam, scal, nmodes, stride, om);
      break;
    case OP_JACOBI:
      k_stencil<D, R, OP_JACOBI, MQ><<<grid, block, 0, s>>>(g, sc, c2, x, b, y, lam, scal, nmodes, stride, om);
      break;
    default:
      k_stencil<D, R, OP_JACOBI_ZERO, MQ><<<grid, block, 0, s>>>(g, sc, c2, x, b, y, lam, scal, nmodes, stride, om);
      break;
  }
}

// Launch shapes of the stencil kernels chosen by the autotuner, per
// (operation, dimension, precision, grid size, mode count); shapes not in
// the table follow the built-in rule below.
struct StencilShape {
  int mq, block;
};
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int64_t, int>, StencilShape> g_tune;

bool tuned_shape(int op, int d, int rsize, int64_t nnodes, int nmodes, StencilShape& out) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  auto it = g_tune.find(std::make_tuple(op, d, rsize, nnodes, nmodes));
  if (it == g_tune.end()) return false;
  out = it->second;
  return true;
}

// Built-in rule: up to four modes per thread (two for the 27-point 3D
// stencil), fewer when the grid alone would not fill the GPU twice over.
template <int D> StencilShape default_shape(int64_t nnodes, int nmodes) {
  constexpr int MQMAX = D == 3 ? 2 : 4;
  const int64_t blocks = (int64_t)blocks_for(nnodes);
  int mq = 1;
  while (mq < MQMAX && mq < nmodes && blocks * ((nmodes + 2 * mq - 1) / (2 * mq)) >= 2 * 152) mq *= 2;
  return StencilShape{mq, kBlock};
}

// The 2D mass stencil has the tensor form m0 (1, 4, 1) (x) (1, 4, 1) (Q1 on a
// uniform grid; exact in floating point, the factors being powers of two),
// which the column-streaming kernel relies on.
template <typename R> bool mass_separable(const StencilCoefT<R>& sc) {
  const R m0 = sc.mtot[0];
  const R w[3] = {R(1), R(4), R(1)};
  for (int s = 0; s < 9; ++s)
    if (sc.mtot[s] != m0 * w[s % 3] * w[s / 3]) return false;
  return true;
}

// block == 0 selects the shared-memory tile kernel, block == kColBlockCode the
// column-streaming kernel (both 2D, operations that read x).
constexpr int kColBlockCode = 64;
template <int D, typename R>
void stencil_launch_shape(int op, const Geo& g, const StencilCoefT<R>& sc, const R* c2, const cx<R>* x,
                          const cx<R>* b, cx<R>* y, const cx<R>* lam, const CocgScal* scal, int nmodes,
                          int64_t stride, double omega, StencilShape sh, cudaStream_t s) {
  if (sh.block == 0 && D == 2 && op != OP_JACOBI_ZERO) {
    if (sh.mq == 4) stencil_tile2_mq<R, 4>(op, g, sc, c2, x, b, y, lam, scal, nmodes, stride, omega, s);
    else if (sh.mq == 2) stencil_tile2_mq<R, 2>(op, g, sc, c2, x, b, y, lam, scal, nmodes, stride, omega, s);
    else stencil_tile2_mq<R, 1>(op, g, sc, c2, x, b, y, lam, scal, nmodes, stride, omega, s);
    return;
  }
  if (sh.block == kColBlockCode && D == 2 && op != OP_JACOBI_ZERO && mass_separable(sc)) {
    if (sh.mq == 4) stencil_col2_mq<R, 4>(op, g, sc, c2, x, b, y, lam, scal, nmodes, stride, omega, s);
    else if (sh.mq == 3) stencil_col2_mq<R, 3>(op, g, sc, c2, x, b, y, lam, scal, nmodes, stride, omega, s);
    else if (sh.mq == 2) stencil_col2_mq<R, 2>(op, g, sc, c2, x, b, y, lam, scal, nmodes, stride, omega, s);
    else stencil_col2_mq<R, 1>(op, g, sc, c2, x, b, y, lam, scal, nmodes, stride, omega, s);
    return;
  }
  if (sh.mq == 4 && D < 3)
    stencil_dispatch_mq<D, R, (D < 3 ? 4 : 1)>(op, g, sc, c2, x, b, y, lam, scal, nmodes, stride, omega, sh.block, s);
  else if (sh.mq >= 2)
    stencil_dispatch_mq<D, R, 2>(op, g, sc, c2, x, b, y, lam, scal, nmodes, stride, omega, sh.block, s);
  else
    stencil_dispatch_mq<D, R, 1>(op, g, sc, c2, x, b, y, lam, scal, nmodes, stride, omega, sh.block, s);
}

template <int D, typename R>
void stencil_dispatch(int op, const Geo& g, const StencilCoefT<R>& sc, const R* c2, const cx<R>* x, const cx<R>* b,
                      cx<R>* y, const cx<R>* lam, const CocgScal* scal, int nmodes, int64_t stride, double omega,
                      cudaStream_t s) {
  StencilShape sh;
  if (!tuned_shape(op, D, (int)sizeof(R), g.nnodes, nmodes, sh)) sh = default_shape<D>(g.nnodes, nmodes);
  stencil_launch_shape<D, R>(op, g, sc, c2, x, b, y, lam, scal, nmodes, stride, omega, sh, s);
}

// Autotuner: time every candidate shape (modes per thread 1, 2, 4 (1, 2 in
// 3D) x block 128, 256, 512, and in 2D the shared-memory tile and the
// column-streaming kernels, the latter also with 3 modes per thread) of one
// stencil operation on the caller's
// buffers with CUDA events, the median of three launches each after one
// untimed launch, and keep the fastest for this (operation, dimension,
// precision, grid size, mode count).  Synchronises the stream; not to be
// called during stream capture.  Returns the chosen shape's time in ms.
template <int D, typename R>
float stencil_tune(int op, const Geo& g, const StencilCoefT<R>& sc, const R* c2, const cx<R>* x, const cx<R>* b,
                   cx<R>* y, const cx<R>* lam, int nmodes, int64_t stride, double omega, cudaStream_t s) {
  const int mqs[4] = {1, 2, 3, 4};  // 3: column-streaming kernel only (three-mode components)
  const int blocks[5] = {128, 256, 512, 0, kColBlockCode};  // 0: shared-memory tiles, 64: column streaming (2D)
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return -1.f;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return -1.f;
  }
  StencilShape best{0, 0};
  float best_ms = 1e30f;
  for (int mq : mqs) {
    if (D == 3 && mq > 2) continue;
    if (mq > 1 && mq > 2 * nmodes) continue;
    for (int bk : blocks) {
      if ((bk == 0 || bk == kColBlockCode) && (D != 2 || op == OP_JACOBI_ZERO)) continue;
      if (mq == 3 && bk != kColBlockCode) continue;
      const StencilShape sh{mq, bk};
      float t[3];
      stencil_launch_shape<D, R>(op, g, sc, c2, x, b, y, lam, nullptr, nmodes, stride, omega, sh, s);
      for (int r = 0; r < 3; ++r) {
        cudaEventRecord(e0, s);
        stencil_launch_shape<D, R>(op, g, sc, c2, x, b, y, lam, nullptr, nmodes, stride, omega, sh, s);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&t[r], e0, e1);
      }
      std::sort(t, t + 3);
      if (t[1] < best_ms) {
        best_ms = t[1];
        best = sh;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (cudaGetLastError() != cudaSuccess || best.mq == 0) return -1.f;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune[std::make_tuple(op, D, (int)sizeof(R), g.nnodes, nmodes)] = best;
  return best_ms;
}

// --------------------------------------------------------- multigrid transfer
// Restriction = transpose of Q1 prolongation: coarse interior node I sits at
// fine interior 2I+1; neighbours at offset delta weigh prod_k (delta_k ? 1/2 : 1).
template <int D, typename R>
__global__ void __launch_bounds__(kBlock) k_restrict(Geo gf, Geo gc, const cx<R>* __restrict__ rf,
                                                     cx<R>* __restrict__ bc, const CocgScal* __restrict__ scal,
                                                     int64_t sf, int64_t scs) {
  const int q = blockIdx.y;
  if (scal != nullptr && !scal[q].active) return;
  const int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= gc.nnodes) return;
  int ic[3] = {0, 0, 0};
  decode<D>(I, gc, ic);
  constexpr int NS = ipow3(D);
  cx<R> acc = mk<R>(0, 0);
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    int ss = s;
    int64_t idx = 0, stride = 1;
    R w = R(1);
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const int dk = ss % 3 - 1;
      ss /= 3;
      idx += (int64_t)(2 * ic[k] + 1 + dk) * stride;
      stride *= gf.n;
      if (dk != 0) w *= R(0.5);
    }
    acc = fma_s(w, rf[(int64_t)q * sf + idx], acc);
  }
  bc[(int64_t)q * scs + I] = acc;
}

// x_f += P x_c: fine grid node g (= interior + 1) takes, per direction, the
// coarse node g/2 (g even) or the two coarse nodes (g -+ 1)/2 with weight 1/2.
template <int D, typename R>
__global__ void __launch_bounds__(kBlock) k_prolong_add(Geo gf, Geo gc, const cx<R>* __restrict__ xc,
                                                        cx<R>* __restrict__ xf, const CocgScal* __restrict__ scal,
                                                        int64_t sf, int64_t scs) {
  const int q = blockIdx.y;
  if (scal != nullptr && !scal[q].active) return;
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= gf.nnodes) return;
  int i[3] = {0, 0, 0};
  decode<D>(a, gf, i);
  cx<R> acc = mk<R>(0, 0);
#pragma unroll
  for (int e = 0; e < (1 << D); ++e) {
    bool ok = true;
    R w = R(1);
    int64_t idx = 0, stride = 1;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const int gk = i[k] + 1;
      const int bit = (e >> k) & 1;
      int G;
      if ((gk & 1) == 0) {
        ok = ok && (bit == 0);
        G = gk >> 1;
      } else {
        G = (gk - 1) / 2 + bit;
        w *= R(0.5);
      }
      const int I = G - 1;
      ok = ok && (I >= 0) && (I < gc.n);
      idx += (int64_t)I * stride;
      stride *= gc.n;
    }
    if (ok) acc = fma_s(w, xc[(int64_t)q * scs + idx], acc);
  }
  xf[(int64_t)q * sf + a] = xf[(int64_t)q * sf + a] + acc;
}

// ------------------------------------------------------------ COCG pieces
enum { RED_BB = 0, RED_ALPHA = 1, RED_RR = 2, RED_BETA = 3, RED_RHO0 = 4 };

template <typename R> __device__ __forceinline__ cx<R> step_alpha(const CocgScal& S);
template <> __device__ __forceinline__ cx<double> step_alpha<double>(const CocgScal& S) {
  return mk<double>(S.alpha_re, S.alpha_im);
}
template <> __device__ __forceinline__ cx<float> step_alpha<float>(const CocgScal& S) {
  return mk<float>(S.alpha_f[0], S.alpha_f[1]);
}
template <typename R> __device__ __forceinline__ cx<R> step_beta(const CocgScal& S);
template <> __device__ __forceinline__ cx<double> step_beta<double>(const CocgScal& S) {
  return mk<double>(S.beta_re, S.beta_im);
}
template <> __device__ __forceinline__ cx<float> step_beta<float>(const CocgScal& S) {
  return mk<float>(S.beta_f[0], S.beta_f[1]);
}

template <typename R> __device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block sum of a complex value; thread 0 receives it.
template <typename R> __device__ __forceinline__ cx<R> block_sum(cx<R> v) {
  __shared__ R sre[32], sim[32];
  v.re = warp_sum(v.re);
  v.im = warp_sum(v.im);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    sre[wid] = v.re;
    sim[wid] = v.im;
  }
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  cx<R> r = mk<R>(0, 0);
  if (wid == 0) {
    r.re = lane < nw ? sre[lane] : R(0);
    r.im = lane < nw ? sim[lane] : R(0);
    r.re = warp_sum(r.re);
    r.im = warp_sum(r.im);
  }
  return r;
}

// which = 0: bilinear sum a_i b_i ; which = 1: sum |a_i|^2 (real part).
template <typename R, int WHICH>
__global__ void __launch_bounds__(kBlock) k_reduce_partial(const cx<R>* __restrict__ a, const cx<R>* __restrict__ b,
                                                           const CocgScal* __restrict__ scal, double* __restrict__ part,
                                                           int64_t n, int64_t stride) {
  const int q = blockIdx.y;
  if (scal != nullptr && !scal[q].active) return;
  cx<R> acc = mk<R>(0, 0);
  const cx<R>* aq = a + (int64_t)q * stride;
  const cx<R>* bq = b + (int64_t)q * stride;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const cx<R> u = aq[i];
    if (WHICH == 0) {
      acc = fma_c(u, bq[i], acc);
    } else {
      acc.re = fma(u.re, u.re, fma(u.im, u.im, acc.re));
    }
  }
  const cx<R> s = block_sum(acc);
  if (threadIdx.x == 0) {
    part[((int64_t)q * gridDim.x + blockIdx.x) * 2 + 0] = (double)s.re;
    part[((int64_t)q * gridDim.x + blockIdx.x) * 2 + 1] = (double)s.im;
  }
}

template <int WHICH>
__global__ void k_reduce_final(CocgScal* __restrict__ scal, const double* __restrict__ part, int nblk, double tol,
                               int max_iter, const double* __restrict__ tolp = nullptr) {
  const int q = blockIdx.x;
  CocgScal& S = scal[q];
  if (WHICH != RED_BB && !S.active) return;
  cx<double> acc = mk<double>(0, 0);
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) {
    acc.re += part[((int64_t)q * nblk + i) * 2 + 0];
    acc.im += part[((int64_t)q * nblk + i) * 2 + 1];
  }
  const cx<double> v = block_sum(acc);
  if (threadIdx.x != 0) return;
  const bool finite = isfinite(v.re) && isfinite(v.im);
  if (WHICH == RED_BB) {
    S.bb = v.re;
    S.rr = v.re;
    S.iters = 0;
    S.status = 0;
    S.active = (v.re > 0.0) ? 1 : 0;
    if (!finite) {
      S.status = 7;
      S.active = 0;
    }
  } else if (WHICH == RED_RHO0) {
    S.rho_re = v.re;
    S.rho_im = v.im;
  } else if (WHICH == RED_ALPHA) {
    const double den = v.re * v.re + v.im * v.im;
    if (!(den > 0.0) || !finite) {
      S.status = 7;
      S.active = 0;
      return;
    }
    // alpha = rho / (p . w)
    S.alpha_re = (S.rho_re * v.re + S.rho_im * v.im) / den;
    S.alpha_im = (S.rho_im * v.re - S.rho_re * v.im) / den;
    S.alpha_f[0] = (float)S.alpha_re;
    S.alpha_f[1] = (float)S.alpha_im;
  } else if (WHICH == RED_RR) {
    S.rr = v.re;
    S.iters += 1;
    if (!finite) {
      S.status = 7;
      S.active = 0;
    } else if (v.re <= (tolp != nullptr ? tolp[0] * tolp[0] : tol * tol) * S.bb) {
      S.active = 0;
    } else if (S.iters >= max_iter) {
      S.status = 4;
      S.active = 0;
    }
  } else if (WHICH == RED_BETA) {
    const double den = S.rho_re * S.rho_re + S.rho_im * S.rho_im;
    if (!(den > 0.0) || !finite) {
      S.status = 7;
      S.active = 0;
      return;
    }
    S.beta_re = (v.re * S.rho_re + v.im * S.rho_im) / den;
    S.beta_im = (v.im * S.rho_re - v.re * S.rho_im) / den;
    S.beta_f[0] = (float)S.beta_re;
    S.beta_f[1] = (float)S.beta_im;
    S.rho_re = v.re;
    S.rho_im = v.im;
  }
}

template <typename R>
__global__ void __launch_bounds__(kBlock) k_cocg_init(const cx<R>* __restrict__ b, cx<R>* __restrict__ x,
                                                      cx<R>* __restrict__ r, int64_t n, int64_t stride) {
  const int q = blockIdx.y;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t e = (int64_t)q * stride + i;
  x[e] = mk<R>(0, 0);
  r[e] = b[e];
}

template <typename R>
__global__ void __launch_bounds__(kBlock) k_update_xr(cx<R>* __restrict__ x, cx<R>* __restrict__ r,
                                                      const cx<R>* __restrict__ p, const cx<R>* __restrict__ w,
                                                      const CocgScal* __restrict__ scal, double* __restrict__ part,
                                                      int64_t n, int64_t stride) {
  const int q = blockIdx.y;
  if (!scal[q].active) return;
  const cx<R> al = step_alpha<R>(scal[q]);
  const cx<R> nal = mk<R>(-al.re, -al.im);
  cx<R> acc = mk<R>(0, 0);
  const int64_t base = (int64_t)q * stride;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    x[base + i] = fma_c(al, p[base + i], x[base + i]);
    const cx<R> rn = fma_c(nal, w[base + i], r[base + i]);
    r[base + i] = rn;
    acc.re = fma(rn.re, rn.re, fma(rn.im, rn.im, acc.re));
  }
  const cx<R> s = block_sum(acc);
  if (threadIdx.x == 0) {
    part[((int64_t)q * gridDim.x + blockIdx.x) * 2 + 0] = (double)s.re;
    part[((int64_t)q * gridDim.x + blockIdx.x) * 2 + 1] = 0.0;
  }
}

template <typename R>
__global__ void __launch_bounds__(kBlock) k_update_p(cx<R>* __restrict__ p, const cx<R>* __restrict__ z,
                                                     const CocgScal* __restrict__ scal, int64_t n, int64_t stride,
                                                     int first) {
  const int q = blockIdx.y;
  if (!scal[q].active) return;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t e = (int64_t)q * stride + i;
  if (first) {
    p[e] = z[e];
  } else {
    const cx<R> be = step_beta<R>(scal[q]);
    p[e] = fma_c(be, p[e], z[e]);
  }
}

__global__ void k_activate(CocgScal* scal, int nmodes) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < nmodes) scal[q].active = 1;
}

// --------------------------------------------------------- time transforms
constexpr int kQB = 4;

template <typename R>
__global__ void __launch_bounds__(kBlock) k_fwd_transform(const cx<double>* __restrict__ W,
                                                          const double* __restrict__ Rt, cx<R>* __restrict__ G,
                                                          int nsel, int nt, int64_t nx) {
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= nx) return;
  const int q0 = blockIdx.y * kQB;
  cx<double> acc[kQB];
#pragma unroll
  for (int u = 0; u < kQB; ++u) acc[u] = mk<double>(0, 0);
  for (int i = 0; i < nt; ++i) {
    const double r = Rt[(int64_t)i * nx + a];
#pragma unroll
    for (int u = 0; u < kQB; ++u)
      if (q0 + u < nsel) acc[u] = fma_s(r, W[(int64_t)(q0 + u) * nt + i], acc[u]);
  }
#pragma unroll
  for (int u = 0; u < kQB; ++u)
    if (q0 + u < nsel) G[(int64_t)(q0 + u) * nx + a] = mk<R>((R)acc[u].re, (R)acc[u].im);
}

template <typename R>
__global__ void __launch_bounds__(kBlock) k_back_transform(const cx<double>* __restrict__ V,
                                                           const double* __restrict__ wq,
                                                           const cx<R>* __restrict__ X, double* __restrict__ U,
                                                           int nsel, int nt, int64_t nx) {
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= nx) return;
  const int i0 = blockIdx.y * kQB;
  double acc[kQB];
#pragma unroll
  for (int u = 0; u < kQB; ++u) acc[u] = 0.0;
  for (int q = 0; q < nsel; ++q) {
    const cx<R> xr = X[(int64_t)q * nx + a];
    const double xre = (double)xr.re, xim = (double)xr.im, w = wq[q];
#pragma unroll
    for (int u = 0; u < kQB; ++u)
      if (i0 + u < nt) {
        const cx<double> v = V[(int64_t)(i0 + u) * nsel + q];
        acc[u] = fma(w, v.re * xre - v.im * xim, acc[u]);
      }
  }
#pragma unroll
  for (int u = 0; u < kQB; ++u)
    if (i0 + u < nt) U[(int64_t)(i0 + u) * nx + a] += acc[u];
}

// ------------------------------------------------------- FP64 residual, loads
template <int D, bool ALLNODES>
__global__ void __launch_bounds__(kBlock) k_stencil_real2(Geo g, StencilCoef sc, const double* __restrict__ c2,
                                                          const double* __restrict__ x, double* __restrict__ K_out,
                                                          double* __restrict__ M_out, double alphaK, double alphaM,
                                                          int64_t xrow, int64_t orow, int accumulate) {
  const int row = blockIdx.y;
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= g.nnodes) return;
  constexpr int NS = ipow3(D);
  int i[3] = {0, 0, 0};
  decode<D>(a, g, i);
  double S[NS];
  cell_sums<D, double>(c2, g.N, i, S);
  const double* xr = x + (int64_t)row * xrow;
  double ak = 0.0, am = 0.0;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    double v;
    if (ALLNODES) {
      // all (N+1)^D nodes; interior node i sits at grid node i + 1
      int ss = s;
      int64_t idx = 0, stride = 1;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const int dk = ss % 3 - 1;
        ss /= 3;
        idx += (int64_t)(i[k] + 1 + dk) * stride;
        stride *= (g.N + 1);
      }
      v = xr[idx];
    } else {
      int64_t off;
      if (!neighbour<D>(i, s, g.n, off)) continue;
      v = xr[a + off];
    }
    ak = fma(S[s] * sc.ke[s], v, ak);
    am = fma(sc.mtot[s], v, am);
  }
  if (ALLNODES) {
    const double v = alphaK * ak + alphaM * am;
    K_out[(int64_t)row * orow + a] = accumulate ? K_out[(int64_t)row * orow + a] + v : v;
  } else {
    K_out[(int64_t)row * orow + a] = ak;
    M_out[(int64_t)row * orow + a] = am;
  }
}

// FP64 space-time residual R = F - (A (x) M + B (x) K) U in one pass: one
// thread per interior node and chunk of time rows [jb, je) forms its
// stiffness row and neighbour offsets once, then streams over the time rows
// j = jb-2 .. je+1, applying K and M to U_j and adding A(i, j) M U_j +
// B(i, j) K U_j to the five rows i = j-2 .. j+2 that row j reaches (A, B
// pentadiagonal); row j-2 is complete after step j.  Chunks (the grid's y)
// only matter for small grids with many time rows; they recompute the two
// rows of halo on either side.
template <int D>
__global__ void __launch_bounds__(kBlock) k_residual_fused(Geo g, StencilCoef sc, const double* __restrict__ c2,
                                                           const double* __restrict__ U,
                                                           const double* __restrict__ F,
                                                           const double* __restrict__ Aband,
                                                           const double* __restrict__ Bband,
                                                           double* __restrict__ Rout, int nt, int chunk) {
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= g.nnodes) return;
  const int jb = blockIdx.y * chunk, je = min(nt, jb + chunk);
  const int64_t nx = g.nnodes;
  constexpr int NS = ipow3(D);
  int i[3] = {0, 0, 0};
  decode<D>(a, g, i);
  double kr[NS];
  cell_sums<D, double>(c2, g.N, i, kr);
#pragma unroll
  for (int s = 0; s < NS; ++s) kr[s] *= sc.ke[s];
  int off[NS];
  unsigned valid = 0u;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    int64_t o;
    if (neighbour<D>(i, s, g.n, o)) valid |= 1u << s;
    off[s] = (int)o;
  }
  double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};  // rows j-2 .. j+2
  for (int j = max(0, jb - 2); j <= je + 1; ++j) {
    if (j < nt) {
      const double* uj = U + (int64_t)j * nx + a;
      double ku = 0.0, mu = 0.0;
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        if ((valid >> s) & 1u) {
          const double v = uj[off[s]];
          ku = fma(kr[s], v, ku);
          mu = fma(sc.mtot[s], v, mu);
        }
      }
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        const int r = j - 2 + k;  // A(r, j) sits at Aband[r * 5 + (j - r) + 2]
        if (r >= 0 && r < nt) {
          const int e = r * 5 + 4 - k;
          acc[k] = fma(-__ldg(Aband + e), mu, fma(-__ldg(Bband + e), ku, acc[k]));
        }
      }
    }
    const int done = j - 2;
    if (done >= jb && done < je) Rout[(int64_t)done * nx + a] = F[(int64_t)done * nx + a] + acc[0];
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[k] = acc[k + 1];
    acc[4] = 0.0;
  }
}

__global__ void __launch_bounds__(kBlock) k_norm2_partial(const double* __restrict__ v, int64_t n,
                                                          double* __restrict__ part) {
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc = fma(v[i], v[i], acc);
  const cx<double> s = block_sum(mk<double>(acc, 0.0));
  if (threadIdx.x == 0) part[blockIdx.x] = s.re;
}

__global__ void k_norm2_final(const double* __restrict__ part, int nblk, double* __restrict__ out) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) acc += part[i];
  const cx<double> s = block_sum(mk<double>(acc, 0.0));
  if (threadIdx.x == 0) out[0] = s.re;
}

__global__ void __launch_bounds__(kBlock) k_rhs_assemble(const double* __restrict__ coef,
                                                         const double* __restrict__ L, double* __restrict__ F,
                                                         int nterm, int nt, int64_t nx) {
  const int i = blockIdx.y;
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= nx) return;
  double acc = 0.0;
  for (int r = 0; r < nterm; ++r) acc = fma(coef[(int64_t)r * nt + i], L[(int64_t)r * nx + a], acc);
  F[(int64_t)i * nx + a] = acc;
}

// ---------------------------------------------------- space eigenbasis method
constexpr int kTile = 16;

// Y[i][a] (+)= sum_b X[i][b] P[b][a], P = Phi (trans 0) or its transpose stored row-major.
__global__ void k_gemm_right(const double* __restrict__ X, const double* __restrict__ P, double* __restrict__ Y,
                             int nt, int64_t nx, int accumulate) {
  __shared__ double sx[kTile][kTile + 1], sp[kTile][kTile + 1];
  const int64_t a = (int64_t)blockIdx.x * kTile + threadIdx.x;
  const int i = blockIdx.y * kTile + threadIdx.y;
  double acc = 0.0;
  for (int64_t b0 = 0; b0 < nx; b0 += kTile) {
    const int64_t bx = b0 + threadIdx.x, by = b0 + threadIdx.y;
    sx[threadIdx.y][threadIdx.x] = (i < nt && bx < nx) ? X[(int64_t)i * nx + bx] : 0.0;
    sp[threadIdx.y][threadIdx.x] = (by < nx && a < nx) ? P[by * nx + a] : 0.0;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kTile; ++k) acc = fma(sx[threadIdx.y][k], sp[k][threadIdx.x], acc);
    __syncthreads();
  }
  if (i < nt && a < nx) {
    if (accumulate) Y[(int64_t)i * nx + a] += acc;
    else Y[(int64_t)i * nx + a] = acc;
  }
}

// Banded LU solve with partial pivoting (factor layout of band_lu, spatial
// mode fastest), one thread per spatial mode, Y column a (stride nx) in place.
// Banded LU solves (A + mu_a B) y_a = r_a, one spatial mode a per CTA: the
// mode's factor (mode-major: column j of the band at j * ld, the diagonal
// stored as its reciprocal), pivots and right-hand side are staged in shared
// memory, then one thread runs the forward (row interchanges, unit lower
// factor, kl sub-diagonals) and backward (upper factor, kl + ku
// super-diagonals) recurrences on a register window of the rows in reach, so
// each step waits on two shared-memory loads and its own multiply-adds.
template <int KL, int KU>
__global__ void __launch_bounds__(128) k_time_band_solve(const double* __restrict__ ab, const int* __restrict__ piv,
                                                         double* __restrict__ Y, int nt, int64_t nx) {
  constexpr int KV = KL + KU, LD = 2 * KL + KU + 1;
  extern __shared__ __align__(16) unsigned char tb_smem[];
  double* sa = reinterpret_cast<double*>(tb_smem);  // nt x LD
  double* sy = sa + (size_t)nt * LD;                // nt
  int* sp = reinterpret_cast<int*>(sy + nt);        // nt
  const int64_t a = blockIdx.x;
  const double* aba = ab + a * (int64_t)nt * LD;
  for (int e = threadIdx.x; e < nt * LD; e += blockDim.x) sa[e] = aba[e];
  for (int j = threadIdx.x; j < nt; j += blockDim.x) {
    sp[j] = piv[a * nt + j];
    sy[j] = Y[(int64_t)j * nx + a];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // forward: window w[0..KL] = rows j .. j+KL
    double w[KL + 1];
#pragma unroll
    for (int t = 0; t <= KL; ++t) w[t] = t < nt ? sy[t] : 0.0;
    for (int j = 0; j < nt; ++j) {
      const int p = sp[j] - j;  // 0 .. KL
      double yj = w[0];
#pragma unroll
      for (int t = 1; t <= KL; ++t) {
        const double wt = w[t];
        w[t] = (p == t) ? yj : wt;
        yj = (p == t) ? wt : yj;
      }
      const double* col = sa + (size_t)j * LD + KV;  // col[i - j] = A(i, j)
#pragma unroll
      for (int t = 1; t <= KL; ++t) w[t] = (j + t < nt) ? fma(-col[t], yj, w[t]) : w[t];
      sy[j] = yj;
#pragma unroll
      for (int t = 0; t < KL; ++t) w[t] = w[t + 1];
      w[KL] = (j + KL + 1 < nt) ? sy[j + KL + 1] : 0.0;
    }
    // backward: window w[0..KV] = rows j, j-1, .., j-KV
    double v[KV + 1];
#pragma unroll
    for (int t = 0; t <= KV; ++t) v[t] = (nt - 1 - t >= 0) ? sy[nt - 1 - t] : 0.0;
    for (int j = nt - 1; j >= 0; --j) {
      const double* col = sa + (size_t)j * LD + KV;  // col[i - j] = A(i, j), col[0] = 1 / A(j, j)
      const double yj = v[0] * col[0];
      sy[j] = yj;
#pragma unroll
      for (int t = 1; t <= KV; ++t) v[t] = (j - t >= 0) ? fma(-col[-t], yj, v[t]) : v[t];
#pragma unroll
      for (int t = 0; t < KV; ++t) v[t] = v[t + 1];
      v[KV] = (j - KV - 1 >= 0) ? sy[j - KV - 1] : 0.0;
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < nt; j += blockDim.x) Y[(int64_t)j * nx + a] = sy[j];
}

// --------------------------------------------------------------- combination
// Hierarchical evaluation of Eq. (19) on a nodal target grid.  The Q1 spaces
// are nested, so a component of spatial level j < j* evaluated at the target
// nodes equals its bilinear prolongation through the levels j+1..j*.
// Level by level, Y_j = P Y_{j-1} + sum_{components at level j} c_k u_k(., t_s),
// on all nodes of level j (boundary included, for the lift by u0); a component
// finer than the target level is injected (its nodes contain the target nodes).
// Sign flip on the integer pipe: FP64 issue slots are the scarce resource of
// the combination kernel on this GPU, so neither the sign of a coefficient
// nor a power-of-two scale costs an FP64 instruction there.
__device__ __forceinline__ double with_sign(double x, unsigned sign_hi) {
  return __hiloint2double(__double2hiint(x) ^ (int)sign_hi, __double2loint(x));
}

// v + coef * (component value at level-j node P, target time s), three FP64
// FMAs per node; coef = -1 enters as a sign flip of the B-spline values.
template <int D> __device__ __forceinline__ double comp_add(const CombComp& cc, int j, const int P[3], int s,
                                                            int nts, int c, const double* __restrict__ tbv,
                                                            const int* __restrict__ tspan, bool interior, double v) {
  const int sh = cc.jx - j;  // >= 0: injection from a finer component grid
  const int N = 1 << cc.jx, n = N - 1, nt = (1 << cc.jt) + 1;
  const unsigned sg = cc.coef > 0 ? 0u : 0x80000000u;
  if (interior) {
    int64_t ii = 0, si = 1, nx = 1;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      ii += (int64_t)((P[k] << sh) - 1) * si;
      si *= n;
      nx *= n;
    }
    const int span = tspan[(int64_t)c * nts + s];
    const double* tb = tbv + ((int64_t)c * nts + s) * 3;
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      const int row = span + t - 1;
      const bool ok = row >= 0 && row < nt;
      const double u = ok ? cc.U[(int64_t)row * nx + ii] : 0.0;
      v = fma(with_sign(tb[t], sg), u, v);
    }
  }
  if (cc.lift != nullptr) {
    int64_t ia = 0, sa = 1;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      ia += (int64_t)(P[k] << sh) * sa;
      sa *= (N + 1);
    }
    v += with_sign(cc.lift[ia], sg);
  }
  return v;
}

// x / 2 for the prolongation midpoints as an exponent decrement of the high
// word (integer pipe): exact whenever the half is a normal number; a half in
// the subnormal range (|x| < 2^-1021) flushes to a signed zero, and infinities
// and NaNs pass unchanged.
__device__ __forceinline__ double half_of(double x) {
  int hi = __double2hiint(x), lo = __double2loint(x);
  const unsigned ex = ((unsigned)hi >> 20) & 0x7ffu;
  if (ex - 2u < 0x7fdu) {
    hi -= 0x100000;
  } else if (ex < 2u) {
    hi &= (int)0x80000000u;
    lo = 0;
  }
  return __hiloint2double(hi, lo);
}

// One thread per node Q of level j-1 (all nodes, boundary included): it
// produces the level-j nodes P = 2Q + e, e in {0,1}^d (those inside the grid).
// Their prolongated values are formed separably, direction by direction
// (value at the odd node = half the sum of its two coarse neighbours), so
// each fine node costs about one FP64 addition; the components of this level
// are then added node by node.  Without Yprev (the coarsest level of
// the combination) only the components are evaluated.
template <int D>
__global__ void __launch_bounds__(kBlock) k_comb_level(int j, const double* __restrict__ Yprev,
                                                       const CombComp* __restrict__ comps, int c0, int c1,
                                                       const double* __restrict__ tbv, const int* __restrict__ tspan,
                                                       int nts, double* __restrict__ Y, FastDiv dQ1) {
  const int s = blockIdx.y;
  const int Nj = 1 << j, Nc = Nj >> 1;
  int64_t ncs = 1, nsp = 1;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    ncs *= (Nc + 1);
    nsp *= (Nj + 1);
  }
  const int64_t qi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (qi >= ncs) return;
  int Q[3] = {0, 0, 0};
  {
    unsigned r = (unsigned)qi;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const unsigned qq = fdiv(r, dQ1);
      Q[k] = (int)(r - qq * (unsigned)(Nc + 1));
      r = qq;
    }
  }
  constexpr int NE = 1 << D;
  double f[NE];
#pragma unroll
  for (int e = 0; e < NE; ++e) f[e] = 0.0;
  if (Yprev != nullptr) {
    const double* Ys = Yprev + (int64_t)s * ncs;
    // coarse corners Q + e (zero outside the grid: those only feed fine nodes outside it)
#pragma unroll
    for (int e = 0; e < NE; ++e) {
      bool ok = true;
      int64_t idx = 0, st = 1;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const int b = (e >> k) & 1;
        ok = ok && (Q[k] + b <= Nc);
        idx += (int64_t)(Q[k] + b) * st;
        st *= (Nc + 1);
      }
      f[e] = ok ? Ys[idx] : 0.0;
    }
    // separable prolongation: along direction k, bit k = 1 becomes the midpoint
#pragma unroll
    for (int k = 0; k < D; ++k) {
#pragma unroll
      for (int e = 0; e < NE; ++e)
        if ((e >> k) & 1) f[e] = half_of(f[e ^ (1 << k)] + f[e]);
    }
  }
#pragma unroll
  for (int e = 0; e < NE; ++e) {
    int P[3] = {0, 0, 0};
    bool inside = true, interior = true;
    int64_t pidx = 0, st = 1;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      P[k] = 2 * Q[k] + ((e >> k) & 1);
      inside = inside && P[k] <= Nj;
      interior = interior && P[k] >= 1 && P[k] <= Nj - 1;
      pidx += (int64_t)P[k] * st;
      st *= (Nj + 1);
    }
    if (!inside) continue;
    double v = f[e];
    for (int c = c0; c < c1; ++c) v = comp_add<D>(comps[c], j, P, s, nts, c, tbv, tspan, interior, v);
    Y[(int64_t)s * nsp + pidx] = v;
  }
}

// ------------------------------------------------- dense coarse-level solve
// x_q = Ainv_q b_q: b_q staged in shared memory, one warp per row (coalesced
// row reads, lanes over columns), warp-shuffle reduction of the dot product.
// One row per warp and CTA of 8 warps: a coarse grid of 961 unknowns and a few
// modes gives several hundred CTAs, spread evenly over the SMs (with 32 rows
// per CTA the ~150 CTAs left a few SMs with two, and the FP64 launch at half
// of the FP64 rate).
constexpr int kDenseRowsPerBlock = 8;

template <typename R>
__global__ void __launch_bounds__(kBlock) k_dense_mv(const cx<R>* __restrict__ Ainv, int n,
                                                     const cx<R>* __restrict__ b, cx<R>* __restrict__ x,
                                                     const CocgScal* __restrict__ scal, int64_t vstride) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<R>* bs = reinterpret_cast<cx<R>*>(smem_raw);
  const int q = blockIdx.y;
  if (scal != nullptr && !scal[q].active) return;
  const cx<R>* bq = b + (int64_t)q * vstride;
  for (int c = threadIdx.x; c < n; c += blockDim.x) bs[c] = bq[c];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const cx<R>* Aq = Ainv + (int64_t)q * n * n;
  const int r1 = min(n, (int)(blockIdx.x + 1) * kDenseRowsPerBlock);
  for (int r = blockIdx.x * kDenseRowsPerBlock + warp; r < r1; r += kBlock / 32) {
    const cx<R>* row = Aq + (int64_t)r * n;
    // four independent partial sums: four row loads in flight per warp (one
    // load per iteration left the kernel waiting on memory latency)
    R re[4] = {R(0), R(0), R(0), R(0)}, im[4] = {R(0), R(0), R(0), R(0)};
    int c = lane;
    for (; c + 96 < n; c += 128) {
      cx<R> a[4], v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] = row[c + 32 * u];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = bs[c + 32 * u];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        re[u] = fma(a[u].re, v[u].re, fma(-a[u].im, v[u].im, re[u]));
        im[u] = fma(a[u].re, v[u].im, fma(a[u].im, v[u].re, im[u]));
      }
    }
    for (; c < n; c += 32) {
      const cx<R> a = row[c], v = bs[c];
      re[0] = fma(a.re, v.re, fma(-a.im, v.im, re[0]));
      im[0] = fma(a.re, v.im, fma(a.im, v.re, im[0]));
    }
    const R rs = warp_sum((re[0] + re[1]) + (re[2] + re[3]));
    const R is = warp_sum((im[0] + im[1]) + (im[2] + im[3]));
    if (lane == 0) x[(int64_t)q * vstride + r] = mk<R>(rs, is);
  }
}

template <typename R> __global__ void k_identity(cx<R>* __restrict__ I, int64_t n) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * n) return;
  const int64_t j = e / n, r = e - (e / n) * n;
  I[e] = mk<R>(r == j ? R(1) : R(0), R(0));
}

// ----------------------------------------------- receiver misfit gradient

__global__ void __launch_bounds__(kBlock) k_receiver_eval(const CombComp* __restrict__ comps, int ncomp,
                                                          const RecCorner* __restrict__ rc, int nrec, int ncorner,
                                                          const double* __restrict__ tbv,
                                                          const int* __restrict__ tspan, int nts,
                                                          double* __restrict__ out) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x, s = blockIdx.y;
  if (r >= nrec) return;
  double val = 0.0;
  for (int c = 0; c < ncomp; ++c) {
    const CombComp cc = comps[c];
    const int n = (1 << cc.jx) - 1, nt = (1 << cc.jt) + 1;
    int64_t nx = n;  // interior nodes of the component grid (ncorner = 2^d)
    for (int k = 2; k < ncorner; k <<= 1) nx *= n;
    const int span = tspan[(int64_t)c * nts + s];
    const double* tb = tbv + ((int64_t)c * nts + s) * 3;
    double vc = 0.0;
    for (int e = 0; e < ncorner; ++e) {
      const RecCorner q = rc[((int64_t)c * nrec + r) * ncorner + e];
      double u = 0.0;
      if (q.interior >= 0)
        for (int t = 0; t < 3; ++t) {
          const int row = span + t - 1;
          if (row >= 0 && row < nt) u = fma(tb[t], cc.U[(int64_t)row * nx + q.interior], u);
        }
      if (cc.lift != nullptr) u += cc.lift[q.all];
      vc = fma(q.w, u, vc);
    }
    val = fma((double)cc.coef, vc, val);
  }
  out[(int64_t)s * nrec + r] = val;
}

__global__ void __launch_bounds__(kBlock) k_misfit(const double* __restrict__ vals, const double* __restrict__ dobs,
                                                   int nts, int nrec, double T, double* __restrict__ wm,
                                                   double* __restrict__ Jout) {
  const double dt = T / (double)(nts - 1);
  double acc = 0.0;
  for (int e = threadIdx.x; e < nts * nrec; e += blockDim.x) {
    const int s = e / nrec;
    const double w = (s == 0 || s == nts - 1) ? 0.5 * dt : dt;
    const double m = vals[e] - dobs[e];
    wm[e] = w * m;
    acc = fma(w * m, m, acc);
  }
  const cx<double> t = block_sum(mk<double>(acc, 0.0));
  if (threadIdx.x == 0) Jout[0] = 0.5 * t.re;
}

// ehat[i][r] = sum_s psi_i(t_s) wm[s][r] (one thread per receiver, no races)
__global__ void k_adj_time_project(const double* __restrict__ wm, int nts, int nrec, const double* __restrict__ tb,
                                   const int* __restrict__ tspan, int nt, double* __restrict__ ehat) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrec) return;
  for (int i = 0; i < nt; ++i) ehat[(int64_t)i * nrec + r] = 0.0;
  for (int s = 0; s < nts; ++s) {
    const double m = wm[(int64_t)s * nrec + r];
    for (int t = 0; t < 3; ++t) {
      const int row = tspan[s] + t - 1;
      if (row >= 0 && row < nt) ehat[(int64_t)row * nrec + r] = fma(tb[s * 3 + t], m, ehat[(int64_t)row * nrec + r]);
    }
  }
}

__global__ void k_adj_scatter(const double* __restrict__ ehat, int nrec, int nt, const RecCorner* __restrict__ rc,
                              int ncorner, double coef, int64_t nx, double* __restrict__ G) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y;
  if (r >= nrec || i >= nt) return;
  const double v = coef * ehat[(int64_t)i * nrec + r];
  for (int e = 0; e < ncorner; ++e) {
    const RecCorner q = rc[(int64_t)r * ncorner + e];
    if (q.interior >= 0) atomicAdd(&G[(int64_t)i * nx + q.interior], q.w * v);
  }
}

// One thread per cell of the level: g_e = -sum_i L_i|_e^T K_ref Z_i|_e with
// Z_i = sum_j B[i][j] U_j, then P^T onto the parameter nodes.
template <int D>
__global__ void __launch_bounds__(kBlock) k_grad_c2(Geo g, double lo0, double lo1, double lo2, double h0, double h1,
                                                    double h2, int nt, const double* __restrict__ Bband,
                                                    const double* __restrict__ U, const double* __restrict__ L,
                                                    ElemK ke, ParamGrid pg, double* __restrict__ dc2) {
  constexpr int NC = 1 << D;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= g.ncells) return;
  int cidx[3] = {0, 0, 0};
  {
    int64_t r = e;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      cidx[k] = (int)(r % g.N);
      r /= g.N;
    }
  }
  int node[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    int idx = 0, st = 1;
    bool in = true;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const int p = cidx[k] + ((c >> k) & 1);  // all-node coordinate
      in = in && p >= 1 && p <= g.N - 1;
      idx += (p - 1) * st;
      st *= g.n;
    }
    node[c] = in ? idx : -1;
  }
  const int64_t nx = g.nnodes;
  double acc = 0.0;
  for (int i = 0; i < nt; ++i) {
    double Z[NC], Lv[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      double z = 0.0;
      if (node[c] >= 0)
        for (int t = -2; t <= 2; ++t) {
          const int j = i + t;
          if (j >= 0 && j < nt) z = fma(Bband[i * 5 + t + 2], U[(int64_t)j * nx + node[c]], z);
        }
      Z[c] = z;
      Lv[c] = node[c] >= 0 ? L[(int64_t)i * nx + node[c]] : 0.0;
    }
#pragma unroll
    for (int p = 0; p < NC; ++p) {
      double kz = 0.0;
#pragma unroll
      for (int q = 0; q < NC; ++q) kz = fma(ke.k[p * NC + q], Z[q], kz);
      acc = fma(Lv[p], kz, acc);
    }
  }
  const double x[3] = {lo0 + (cidx[0] + 0.5) * h0, lo1 + (cidx[1] + 0.5) * h1, lo2 + (cidx[2] + 0.5) * h2};
  int pn[8];
  double pw[8];
  param_weights<D>(pg, x, pn, pw);
#pragma unroll
  for (int c = 0; c < NC; ++c) atomicAdd(&dc2[pn[c]], -acc * pw[c]);
}

__global__ void __launch_bounds__(kBlock) k_grad_g_v(int nt, int64_t nx, const double* __restrict__ b,
                                                     const double* __restrict__ L, double* __restrict__ v) {
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= nx) return;
  double acc = 0.0;
  for (int i = 0; i < nt; ++i) acc = fma(b[i], L[(int64_t)i * nx + a], acc);
  v[a] = acc;
}

// One thread per node of the level (boundary included): (M_load^T v)(m) =
// sum over interior neighbours a of mtot[a - m] v[a], then Q^T onto the parameter nodes.
template <int D>
__global__ void __launch_bounds__(kBlock) k_grad_g(Geo g, double lo0, double lo1, double lo2, double h0, double h1,
                                                   double h2, StencilCoef sc, const double* __restrict__ v,
                                                   ParamGrid pg, double* __restrict__ dg) {
  constexpr int NS = ipow3(D);
  int64_t nall = 1;
#pragma unroll
  for (int k = 0; k < D; ++k) nall *= (g.N + 1);
  const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= nall) return;
  int P[3] = {0, 0, 0};
  {
    int64_t r = m;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      P[k] = (int)(r % (g.N + 1));
      r /= (g.N + 1);
    }
  }
  double acc = 0.0;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    int ss = s, idx = 0, st = 1;
    bool in = true;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const int q = P[k] + ss % 3 - 1;
      ss /= 3;
      in = in && q >= 1 && q <= g.N - 1;
      idx += (q - 1) * st;
      st *= g.n;
    }
    if (in) acc = fma(sc.mtot[s], v[idx], acc);
  }
  const double x[3] = {lo0 + P[0] * h0, lo1 + P[1] * h1, lo2 + P[2] * h2};
  int pn[8];
  double pw[8];
  param_weights<D>(pg, x, pn, pw);
#pragma unroll
  for (int c = 0; c < (1 << D); ++c) atomicAdd(&dg[pn[c]], acc * pw[c]);
}

}  // namespace

// ================================================================ wrappers
template <typename R>
void launch_stencil(int op, const Geo& g, const StencilCoefT<R>& sc, const R* c2, const cx<R>* x, const cx<R>* b,
                    cx<R>* y, const cx<R>* lam, const CocgScal* scal, int nmodes, int64_t stride, double omega,
                    cudaStream_t s) {
  count(1);
  if (g.d == 1) stencil_dispatch<1, R>(op, g, sc, c2, x, b, y, lam, scal, nmodes, stride, omega, s);
  else if (g.d == 2) stencil_dispatch<2, R>(op, g, sc, c2, x, b, y, lam, scal, nmodes, stride, omega, s);
  else stencil_dispatch<3, R>(op, g, sc, c2, x, b, y, lam, scal, nmodes, stride, omega, s);
}

template <typename R>
void launch_jacobi_dinv(const Geo& g, const StencilCoefT<R>& sc, const R* c2, const cx<R>* lam, double omega,
                        int nmodes, int64_t stride, cx<R>* dinv, cudaStream_t s) {
  count(1);
  StencilCoefT<R> sc0 = sc;
  sc0.dinv = nullptr;
  const dim3 grid(blocks_for(g.nnodes), nmodes);
  if (g.d == 1) k_jacobi_dinv<1, R><<<grid, kBlock, 0, s>>>(g, sc0, c2, lam, (R)omega, stride, dinv);
  else if (g.d == 2) k_jacobi_dinv<2, R><<<grid, kBlock, 0, s>>>(g, sc0, c2, lam, (R)omega, stride, dinv);
  else k_jacobi_dinv<3, R><<<grid, kBlock, 0, s>>>(g, sc0, c2, lam, (R)omega, stride, dinv);
}

template <typename R>
void launch_restrict(const Geo& gf, const Geo& gc, const cx<R>* rf, cx<R>* bc, const CocgScal* scal, int nmodes,
                     int64_t sf, int64_t scs, cudaStream_t s) {
  count(1);
  dim3 grid(blocks_for(gc.nnodes), nmodes);
  if (gf.d == 1) k_restrict<1, R><<<grid, kBlock, 0, s>>>(gf, gc, rf, bc, scal, sf, scs);
  else if (gf.d == 2) k_restrict<2, R><<<grid, kBlock, 0, s>>>(gf, gc, rf, bc, scal, sf, scs);
  else k_restrict<3, R><<<grid, kBlock, 0, s>>>(gf, gc, rf, bc, scal, sf, scs);
}

template <typename R>
void launch_prolong_add(const Geo& gf, const Geo& gc, const cx<R>* xc, cx<R>* xf, const CocgScal* scal, int nmodes,
                        int64_t sf, int64_t scs, cudaStream_t s) {
  count(1);
  dim3 grid(blocks_for(gf.nnodes), nmodes);
  if (gf.d == 1) k_prolong_add<1, R><<<grid, kBlock, 0, s>>>(gf, gc, xc, xf, scal, sf, scs);
  else if (gf.d == 2) k_prolong_add<2, R><<<grid, kBlock, 0, s>>>(gf, gc, xc, xf, scal, sf, scs);
  else k_prolong_add<3, R><<<grid, kBlock, 0, s>>>(gf, gc, xc, xf, scal, sf, scs);
}

template <typename R>
void launch_cocg_init(const cx<R>* b, cx<R>* x, cx<R>* r, CocgScal* scal, double* part, int nmodes, int64_t n,
                      int64_t stride, cudaStream_t s) {
  count(3);
  k_cocg_init<R><<<dim3(blocks_for(n), nmodes), kBlock, 0, s>>>(b, x, r, n, stride);
  k_reduce_partial<R, 1><<<dim3(kRedBlocks, nmodes), kBlock, 0, s>>>(b, b, nullptr, part, n, stride);
  k_reduce_final<RED_BB><<<nmodes, 256, 0, s>>>(scal, part, kRedBlocks, 0.0, 0);
}

template <typename R>
void launch_dot(int which, const cx<R>* a, const cx<R>* b, CocgScal* scal, double* part, int nmodes, int64_t n,
                int64_t stride, double tol, int max_iter, cudaStream_t s) {
  count(2);
  k_reduce_partial<R, 0><<<dim3(kRedBlocks, nmodes), kBlock, 0, s>>>(a, b, scal, part, n, stride);
  if (which == 0) k_reduce_final<RED_ALPHA><<<nmodes, 256, 0, s>>>(scal, part, kRedBlocks, tol, max_iter);
  else if (which == 1) k_reduce_final<RED_BETA><<<nmodes, 256, 0, s>>>(scal, part, kRedBlocks, tol, max_iter);
  else k_reduce_final<RED_RHO0><<<nmodes, 256, 0, s>>>(scal, part, kRedBlocks, tol, max_iter);
}

template <typename R>
void launch_update_xr(cx<R>* x, cx<R>* r, const cx<R>* p, const cx<R>* w, CocgScal* scal, double* part,
                      int nmodes, int64_t n, int64_t stride, double tol, int max_iter, cudaStream_t s,
                      const double* tolp) {
  count(2);
  k_update_xr<R><<<dim3(kRedBlocks, nmodes), kBlock, 0, s>>>(x, r, p, w, scal, part, n, stride);
  k_reduce_final<RED_RR><<<nmodes, 256, 0, s>>>(scal, part, kRedBlocks, tol, max_iter, tolp);
}

__global__ void k_set_scalar(double* __restrict__ p, double v) { p[0] = v; }

void launch_set_scalar(double* p, double v, cudaStream_t s) {
  count(1);
  k_set_scalar<<<1, 1, 0, s>>>(p, v);
}

template <typename R>
void launch_update_p(cx<R>* p, const cx<R>* z, const CocgScal* scal, int nmodes, int64_t n, int64_t stride,
                     int first, cudaStream_t s) {
  k_update_p<R><<<dim3(blocks_for(n), nmodes), kBlock, 0, s>>>(p, z, scal, n, stride, first);
  count(1);
}

void launch_cocg_activate(CocgScal* scal, int nmodes, cudaStream_t s) {
  count(1);
  k_activate<<<(nmodes + 127) / 128, 128, 0, s>>>(scal, nmodes);
}

template <typename R>
void launch_fwd_transform(const cx<double>* W, const double* Rt, cx<R>* G, int nsel, int nt, int64_t nx,
                          cudaStream_t s) {
  count(1);
  k_fwd_transform<R><<<dim3(blocks_for(nx), (nsel + kQB - 1) / kQB), kBlock, 0, s>>>(W, Rt, G, nsel, nt, nx);
}

template <typename R>
void launch_back_transform(const cx<double>* V, const double* wq, const cx<R>* X, double* U, int nsel, int nt,
                           int64_t nx, cudaStream_t s) {
  count(1);
  k_back_transform<R><<<dim3(blocks_for(nx), (nt + kQB - 1) / kQB), kBlock, 0, s>>>(V, wq, X, U, nsel, nt, nx);
}

void launch_residual(const Geo& g, const StencilCoef& sc, const double* c2, const double* U, const double* F,
                     const double* Aband, const double* Bband, double* KU, double* MU, double* Rout, int nt,
                     cudaStream_t s) {
  count(1);
  (void)KU;
  (void)MU;
  // time chunks of at least 8 rows, as many as it takes to give the grid
  // about two CTAs per SM
  const unsigned bx = blocks_for(g.nnodes);
  int nch = (int)std::min<int64_t>((nt + 7) / 8, (304 + (int64_t)bx - 1) / bx);
  nch = std::max(nch, 1);
  const int chunk = (nt + nch - 1) / nch;
  const dim3 grid(bx, (nt + chunk - 1) / chunk);
  if (g.d == 1) k_residual_fused<1><<<grid, kBlock, 0, s>>>(g, sc, c2, U, F, Aband, Bband, Rout, nt, chunk);
  else if (g.d == 2) k_residual_fused<2><<<grid, kBlock, 0, s>>>(g, sc, c2, U, F, Aband, Bband, Rout, nt, chunk);
  else k_residual_fused<3><<<grid, kBlock, 0, s>>>(g, sc, c2, U, F, Aband, Bband, Rout, nt, chunk);
}

void launch_norm2(const double* v, int64_t n, double* part, double* out, cudaStream_t s) {
  count(2);
  k_norm2_partial<<<kRedBlocks, kBlock, 0, s>>>(v, n, part);
  k_norm2_final<<<1, 256, 0, s>>>(part, kRedBlocks, out);
}

void launch_load(const Geo& g, const StencilCoef& sc, const double* c2, const double* xall, double* out,
                 double alphaK, double alphaM, int accumulate, cudaStream_t s) {
  count(1);
  dim3 grid(blocks_for(g.nnodes), 1);
  if (g.d == 1) k_stencil_real2<1, true><<<grid, kBlock, 0, s>>>(g, sc, c2, xall, out, nullptr, alphaK, alphaM, 0, 0, accumulate);
  else if (g.d == 2) k_stencil_real2<2, true><<<grid, kBlock, 0, s>>>(g, sc, c2, xall, out, nullptr, alphaK, alphaM, 0, 0, accumulate);
  else k_stencil_real2<3, true><<<grid, kBlock, 0, s>>>(g, sc, c2, xall, out, nullptr, alphaK, alphaM, 0, 0, accumulate);
}

void launch_rhs_assemble(const double* coef, const double* L, double* F, int nterm, int nt, int64_t nx,
                         cudaStream_t s) {
  count(1);
  k_rhs_assemble<<<dim3(blocks_for(nx), nt), kBlock, 0, s>>>(coef, L, F, nterm, nt, nx);
}

void launch_gemm_right(const double* X, const double* Phi, double* Y, int nt, int64_t nx, int trans, int accumulate,
                       cudaStream_t s) {
  count(1);
  (void)trans;  // the caller passes Phi or its stored transpose
  dim3 block(kTile, kTile), grid((unsigned)((nx + kTile - 1) / kTile), (nt + kTile - 1) / kTile);
  k_gemm_right<<<grid, block, 0, s>>>(X, Phi, Y, nt, nx, accumulate);
}

// Energy of Section 6.3 on the cells of one level: for every time b,
// part[b][block] = 1/2 sum over the block's cells e of
//   z_e^T Me z_e + c2_e y_e^T Ke y_e,
// y (values) and z (time derivatives) on all (N+1)^D nodes of the level (x
// fastest), Me / Ke the element mass and unit-coefficient stiffness (local
// corner c: bit k set at the upper end in direction k), c2 cellwise.
template <int D>
__global__ void __launch_bounds__(kBlock) k_energy_cells(int N, const double* __restrict__ c2,
                                                         const double* __restrict__ y, const double* __restrict__ z,
                                                         int64_t nall, ElemK me, ElemK ke, double* __restrict__ part) {
  constexpr int NC = 1 << D;
  const int b = blockIdx.y;
  int64_t ncell = 1;
#pragma unroll
  for (int k = 0; k < D; ++k) ncell *= N;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double acc = 0.0;
  if (e < ncell) {
    int64_t r = e, base = 0, st = 1;
    int64_t off[NC];
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const int64_t ik = r % N;
      r /= N;
      base += ik * st;
      st *= (N + 1);
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      int64_t o = 0, s2 = 1;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        o += ((c >> k) & 1) * s2;
        s2 *= (N + 1);
      }
      off[c] = base + o;
    }
    double yv[NC], zv[NC];
    const double* yb = y + (int64_t)b * nall;
    const double* zb = z + (int64_t)b * nall;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      yv[c] = yb[off[c]];
      zv[c] = zb[off[c]];
    }
    double qm = 0.0, qk = 0.0;
#pragma unroll
    for (int a = 0; a < NC; ++a) {
      double rm = 0.0, rk = 0.0;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        rm = fma(me.k[a * NC + c], zv[c], rm);
        rk = fma(ke.k[a * NC + c], yv[c], rk);
      }
      qm = fma(zv[a], rm, qm);
      qk = fma(yv[a], rk, qk);
    }
    acc = 0.5 * (qm + c2[e] * qk);
  }
  const cx<double> t = block_sum(mk<double>(acc, 0.0));
  if (threadIdx.x == 0) part[(int64_t)b * gridDim.x + blockIdx.x] = t.re;
}

__global__ void k_energy_final(const double* __restrict__ part, int nblk, double* __restrict__ out) {
  const int b = blockIdx.x;
  double acc = 0.0;
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) acc += part[(int64_t)b * nblk + i];
  const cx<double> t = block_sum(mk<double>(acc, 0.0));
  if (threadIdx.x == 0) out[b] = t.re;
}

// Condition of the device-side COCG loop (a WHILE node of a CUDA graph):
// continue while any mode is still iterating.  Every mode leaves the active
// set at convergence, at a breakdown or at its iteration limit, so the loop
// ends after at most max_iter / (iterations per body) + 1 bodies.  One thread
// sets the condition (concurrent calls would race).
__global__ void k_cocg_continue(const CocgScal* __restrict__ scal, int nmodes, cudaGraphConditionalHandle handle,
                                int* bodies) {
  int any = 0;
  for (int q = threadIdx.x; q < nmodes; q += blockDim.x) any |= scal[q].active;
  any = __syncthreads_or(any);
  if (threadIdx.x == 0) {
    if (bodies != nullptr) ++*bodies;
    cudaGraphSetConditional(handle, any ? 1u : 0u);
  }
}

__global__ void k_refine_init(RefineRec* __restrict__ rec, const double* __restrict__ fn2,
                              cudaGraphConditionalHandle h, InnerTol it) {
  if (it.tol != nullptr) it.tol[0] = it.base;
  const double f = fn2[0];
  RefineRec r{};
  r.eta_prev = 1e300;
  r.status = (f >= 0.0 && f <= 1.7e308) ? RR_OK : RR_NUMERIC;
  *rec = r;
  cudaGraphSetConditional(h, (r.status == RR_OK && f > 0.0) ? 1u : 0u);
}

// The refinement test of one sweep, as the host loop takes it (one warp).
__global__ void k_refine_decide(RefineRec* __restrict__ rec, const double* __restrict__ nrm2,
                                const double* __restrict__ fn2, double snorm, double tol, int max_sweeps,
                                const CocgScal* __restrict__ scal, int nsel, const int* __restrict__ cerr,
                                cudaGraphConditionalHandle h, InnerTol itol) {
  int it = 0, worst = 0;  // worst: 2 = an iteration limit, 1 = another non-zero status word
  if (scal != nullptr)
    for (int q = threadIdx.x; q < nsel; q += 32) {
      it = max(it, scal[q].iters);
      const int sq = scal[q].status;
      worst = max(worst, sq == 4 ? 2 : (sq != 0 ? 1 : 0));
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    it = max(it, __shfl_xor_sync(0xffffffffu, it, o));
    worst = max(worst, __shfl_xor_sync(0xffffffffu, worst, o));
  }
  if (threadIdx.x != 0) return;
  RefineRec r = *rec;
  r.sweeps += 1;
  r.max_iters = max(r.max_iters, it);
  int st = worst == 2 ? RR_ITER_LIMIT : (worst == 1 ? RR_NUMERIC : RR_OK);
  if (cerr != nullptr && cerr[0] != 0) st = RR_TIMEOUT;
  const double rn = sqrt(nrm2[0]), un = sqrt(nrm2[1]), fn = sqrt(fn2[0]);
  const double rel = rn / fn, eta = rn / (snorm * un + fn);
  if (st == RR_OK && !(fabs(rel) <= 1.7e308)) st = RR_NUMERIC;
  const bool more = st == RR_OK && !(eta <= tol || eta > 0.5 * r.eta_prev) && r.sweeps < max_sweeps;
  r.rel = rel;
  r.eta = eta;
  r.eta_prev = eta;
  r.status = st;
  *rec = r;
  if (itol.tol != nullptr && itol.adaptive) itol.tol[0] = next_inner_tol(itol.base, tol, eta, itol.amp);
  cudaGraphSetConditional(h, more ? 1u : 0u);
}

void launch_energy_cells(int d, int N, const double* c2, const double* y, const double* z, int64_t nall, int ntimes,
                         const ElemK& me, const ElemK& ke, double* part, double* out, cudaStream_t s) {
  int64_t ncell = 1;
  for (int k = 0; k < d; ++k) ncell *= N;
  const unsigned nblk = blocks_for(ncell);
  const dim3 grid(nblk, ntimes);
  if (d == 1) k_energy_cells<1><<<grid, kBlock, 0, s>>>(N, c2, y, z, nall, me, ke, part);
  else if (d == 2) k_energy_cells<2><<<grid, kBlock, 0, s>>>(N, c2, y, z, nall, me, ke, part);
  else k_energy_cells<3><<<grid, kBlock, 0, s>>>(N, c2, y, z, nall, me, ke, part);
  k_energy_final<<<ntimes, kBlock, 0, s>>>(part, (int)nblk, out);
  count(2);
}

void launch_cocg_continue(const CocgScal* scal, int nmodes, cudaGraphConditionalHandle handle, int* bodies,
                          cudaStream_t s) {
  count(1);
  k_cocg_continue<<<1, 128, 0, s>>>(scal, nmodes, handle, bodies);
}

void launch_refine_init(RefineRec* rec, const double* fn2, cudaGraphConditionalHandle h, InnerTol it,
                        cudaStream_t s) {
  count(1);
  k_refine_init<<<1, 1, 0, s>>>(rec, fn2, h, it);
}

void launch_refine_decide(RefineRec* rec, const double* nrm2, const double* fn2, double snorm, double tol,
                          int max_sweeps, const CocgScal* scal, int nsel, const int* cerr,
                          cudaGraphConditionalHandle h, InnerTol it, cudaStream_t s) {
  count(1);
  k_refine_decide<<<1, 32, 0, s>>>(rec, nrm2, fn2, snorm, tol, max_sweeps, scal, nsel, cerr, h, it);
}

size_t time_band_smem(int nt) { return (size_t)nt * (7 * sizeof(double) + sizeof(double) + sizeof(int)); }

bool launch_time_band_solve(const double* ab, const int* piv, double* Y, int nt, int64_t nx, int kl, int ku,
                            cudaStream_t s) {
  if (kl != 2 || ku != 2 || time_band_smem(nt) > kTimeBandMaxSmem) return false;
  count(1);
  // set for the current device at every launch (a host-side attribute call)
  cudaFuncSetAttribute(k_time_band_solve<2, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTimeBandMaxSmem);
  k_time_band_solve<2, 2><<<(unsigned)nx, 128, time_band_smem(nt), s>>>(ab, piv, Y, nt, nx);
  return true;
}

void launch_comb_level(int d, int j, const double* Yprev, const CombComp* comps, int c0, int c1, const double* tbv,
                       const int* tspan, int nts, double* Y, cudaStream_t s) {
  count(1);
  int64_t ncs = 1;  // one thread per node of level j-1 (each writes up to 2^d level-j nodes)
  for (int k = 0; k < d; ++k) ncs *= ((1 << j) / 2 + 1);
  dim3 grid(blocks_for(ncs), nts);
  const FastDiv f = make_fastdiv((unsigned)((1 << j) / 2 + 1));
  if (d == 1) k_comb_level<1><<<grid, kBlock, 0, s>>>(j, Yprev, comps, c0, c1, tbv, tspan, nts, Y, f);
  else if (d == 2) k_comb_level<2><<<grid, kBlock, 0, s>>>(j, Yprev, comps, c0, c1, tbv, tspan, nts, Y, f);
  else k_comb_level<3><<<grid, kBlock, 0, s>>>(j, Yprev, comps, c0, c1, tbv, tspan, nts, Y, f);
}

template <typename R>
void launch_dense_coarse(const cx<R>* Ainv, int64_t n, const cx<R>* b, cx<R>* x, const CocgScal* scal, int nmodes,
                         int64_t vstride, cudaStream_t s) {
  count(1);
  const size_t smem = (size_t)n * sizeof(cx<R>);
  if (smem > 48 * 1024) {
    static std::mutex mu;
    static size_t done = 0;
    std::lock_guard<std::mutex> lock(mu);
    if (smem > done) {
      cudaFuncSetAttribute(k_dense_mv<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      done = smem;
    }
  }
  const dim3 grid((unsigned)((n + kDenseRowsPerBlock - 1) / kDenseRowsPerBlock), nmodes);
  k_dense_mv<R><<<grid, kBlock, smem, s>>>(Ainv, (int)n, b, x, scal, vstride);
}

template <typename R> void launch_identity(cx<R>* I, int64_t n, cudaStream_t s) {
  count(1);
  k_identity<R><<<blocks_for(n * n), kBlock, 0, s>>>(I, n);
}

void launch_receiver_eval(const CombComp* comps, int ncomp, const RecCorner* rc, int nrec, int ncorner,
                          const double* tbv, const int* tspan, int nts, double* out, cudaStream_t s) {
  count(1);
  k_receiver_eval<<<dim3((nrec + kBlock - 1) / kBlock, nts), kBlock, 0, s>>>(comps, ncomp, rc, nrec, ncorner, tbv,
                                                                             tspan, nts, out);
}

void launch_misfit(const double* vals, const double* dobs, int nts, int nrec, double T, double* wm, double* Jout,
                   cudaStream_t s) {
  count(1);
  k_misfit<<<1, kBlock, 0, s>>>(vals, dobs, nts, nrec, T, wm, Jout);
}

void launch_adjoint_rhs(const double* wm, int nts, int nrec, const double* tb, const int* tspan, int nt,
                        const RecCorner* rc, int ncorner, double coef, int64_t nx, double* ehat, double* G,
                        cudaStream_t s) {
  count(2);
  k_adj_time_project<<<(nrec + 63) / 64, 64, 0, s>>>(wm, nts, nrec, tb, tspan, nt, ehat);
  k_adj_scatter<<<dim3((nrec + 63) / 64, nt), 64, 0, s>>>(ehat, nrec, nt, rc, ncorner, coef, nx, G);
}

void launch_grad_c2(const Geo& g, const double* lo, int nt, const double* Bband, const double* U, const double* L,
                    const ElemK& ke, const ParamGrid& pg, double* dc2, cudaStream_t s) {
  count(1);
  const double h0 = pg.h[0] * pg.Np / g.N, h1 = pg.h[1] * pg.Np / g.N, h2 = pg.h[2] * pg.Np / g.N;
  const unsigned grid = blocks_for(g.ncells);
  if (g.d == 1) k_grad_c2<1><<<grid, kBlock, 0, s>>>(g, lo[0], lo[1], lo[2], h0, h1, h2, nt, Bband, U, L, ke, pg, dc2);
  else if (g.d == 2) k_grad_c2<2><<<grid, kBlock, 0, s>>>(g, lo[0], lo[1], lo[2], h0, h1, h2, nt, Bband, U, L, ke, pg, dc2);
  else k_grad_c2<3><<<grid, kBlock, 0, s>>>(g, lo[0], lo[1], lo[2], h0, h1, h2, nt, Bband, U, L, ke, pg, dc2);
}

void launch_grad_g(const Geo& g, const double* lo, const StencilCoef& sc, int nt, const double* b, const double* L,
                   double* v, const ParamGrid& pg, double* dg, cudaStream_t s) {
  count(2);
  k_grad_g_v<<<blocks_for(g.nnodes), kBlock, 0, s>>>(nt, g.nnodes, b, L, v);
  const double h0 = pg.h[0] * pg.Np / g.N, h1 = pg.h[1] * pg.Np / g.N, h2 = pg.h[2] * pg.Np / g.N;
  int64_t nall = 1;
  for (int k = 0; k < g.d; ++k) nall *= (g.N + 1);
  const unsigned grid = blocks_for(nall);
  if (g.d == 1) k_grad_g<1><<<grid, kBlock, 0, s>>>(g, lo[0], lo[1], lo[2], h0, h1, h2, sc, v, pg, dg);
  else if (g.d == 2) k_grad_g<2><<<grid, kBlock, 0, s>>>(g, lo[0], lo[1], lo[2], h0, h1, h2, sc, v, pg, dg);
  else k_grad_g<3><<<grid, kBlock, 0, s>>>(g, lo[0], lo[1], lo[2], h0, h1, h2, sc, v, pg, dg);
}

template <typename R>
float tune_stencil(int op, const Geo& g, const StencilCoefT<R>& sc, const R* c2, const cx<R>* x, const cx<R>* b,
                   cx<R>* y, const cx<R>* lam, int nmodes, int64_t stride, double omega, cudaStream_t s) {
  {
    StencilShape sh;
    if (tuned_shape(op, g.d, (int)sizeof(R), g.nnodes, nmodes, sh)) return 0.f;  // tuned already
  }
  if (g.d == 1) return stencil_tune<1, R>(op, g, sc, c2, x, b, y, lam, nmodes, stride, omega, s);
  if (g.d == 2) return stencil_tune<2, R>(op, g, sc, c2, x, b, y, lam, nmodes, stride, omega, s);
  return stencil_tune<3, R>(op, g, sc, c2, x, b, y, lam, nmodes, stride, omega, s);
}

bool set_stencil_shape(int op, int d, int rsize, int64_t nnodes, int nmodes, int mq, int block) {
  if (op < 0 || op > 3 || d < 1 || d > 3 || (rsize != 4 && rsize != 8) || nnodes < 1 || nmodes < 1) return false;
  if (mq != 1 && mq != 2 && mq != 3 && mq != 4) return false;
  if (mq == 3 && block != kColBlockCode) return false;
  if (d == 3 && mq == 4) return false;
  if (block != 0 && block != kColBlockCode && block != 128 && block != 256 && block != 512) return false;
  if ((block == 0 || block == kColBlockCode) && (d != 2 || op == OP_JACOBI_ZERO)) return false;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune[std::make_tuple(op, d, rsize, nnodes, nmodes)] = StencilShape{mq, block};
  return true;
}

int tuned_stencil_shapes(int* out, int max_entries) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  int n = 0;
  for (const auto& kv : g_tune) {
    if (out && n < max_entries) {
      int* e = out + 7 * n;
      e[0] = std::get<0>(kv.first);
      e[1] = std::get<1>(kv.first);
      e[2] = std::get<2>(kv.first);
      e[3] = (int)std::get<3>(kv.first);
      e[4] = std::get<4>(kv.first);
      e[5] = kv.second.mq;
      e[6] = kv.second.block;
    }
    ++n;
  }
  return n;
}

int64_t kernel_launch_count() { return g_launches.load(); }
void note_launches(int k) { count(k); }

// explicit instantiations
#define ST_INST(R)                                                                                                   \
  template void launch_stencil<R>(int, const Geo&, const StencilCoefT<R>&, const R*, const cx<R>*, const cx<R>*, cx<R>*, \
                                  const cx<R>*, const CocgScal*, int, int64_t, double, cudaStream_t);                \
  template void launch_jacobi_dinv<R>(const Geo&, const StencilCoefT<R>&, const R*, const cx<R>*, double, int,      \
                                      int64_t, cx<R>*, cudaStream_t);                                                \
  template void launch_restrict<R>(const Geo&, const Geo&, const cx<R>*, cx<R>*, const CocgScal*, int, int64_t,      \
                                   int64_t, cudaStream_t);                                                           \
  template void launch_prolong_add<R>(const Geo&, const Geo&, const cx<R>*, cx<R>*, const CocgScal*, int, int64_t,   \
                                      int64_t, cudaStream_t);                                                        \
  template void launch_cocg_init<R>(const cx<R>*, cx<R>*, cx<R>*, CocgScal*, double*, int, int64_t, int64_t,         \
                                    cudaStream_t);                                                                   \
  template void launch_dot<R>(int, const cx<R>*, const cx<R>*, CocgScal*, double*, int, int64_t, int64_t, double,    \
                              int, cudaStream_t);                                                                    \
  template void launch_update_xr<R>(cx<R>*, cx<R>*, const cx<R>*, const cx<R>*, CocgScal*, double*, int, int64_t,    \
                                    int64_t, double, int, cudaStream_t, const double*);                              \
  template void launch_update_p<R>(cx<R>*, const cx<R>*, const CocgScal*, int, int64_t, int64_t, int, cudaStream_t);      \
  template void launch_fwd_transform<R>(const cx<double>*, const double*, cx<R>*, int, int, int64_t, cudaStream_t);  \
  template void launch_back_transform<R>(const cx<double>*, const double*, const cx<R>*, double*, int, int, int64_t, \
                                         cudaStream_t);                                                              \
  template void launch_dense_coarse<R>(const cx<R>*, int64_t, const cx<R>*, cx<R>*, const CocgScal*, int, int64_t,   \
                                       cudaStream_t);                                                                \
  template void launch_identity<R>(cx<R>*, int64_t, cudaStream_t);                                              \
  template float tune_stencil<R>(int, const Geo&, const StencilCoefT<R>&, const R*, const cx<R>*, const cx<R>*,      \
                                 cx<R>*, const cx<R>*, int, int64_t, double, cudaStream_t);
ST_INST(double)
ST_INST(float)
#undef ST_INST

}  // namespace st
