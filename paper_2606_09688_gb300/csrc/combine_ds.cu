// One level of the hierarchical combination of Eq. (19) in double-single
// arithmetic (the value of a target node held as a float pair, 48 significant
// bits), the target level written as FP64.
//
// The level-j values are Y_j = P Y_{j-1} + sum_c coef_c u_c(., t_s) on the
// (2^j+1)^d nodes of level j at every target time t_s: P is the Q1
// prolongation from level j-1 (midpoints averaged direction by direction), u_c
// the components of level j (those finer than the target at the target
// level, read by injection).  Every term is a sum of exact products: the
// B-spline weights at the target times are dyadic rationals, exact in FP32,
// and the prolongation halves; so the pair arithmetic loses only the
// rounding of its error-free transformations (relative 2^-47 per step).
//
// Work layout: one thread per node Q of level j-1, which owns the 2^d level-j
// nodes 2Q + e, e in {0,1}^d, for a chunk of consecutive target times.  Over a
// chunk every component's time span is fixed (chunks are aligned to the
// component's time intervals), so the three time coefficients of each owned
// node, with the lifting u0 folded in (the three B-splines of a span sum to
// one), stay in registers as pairs, and each target value costs three pair
// multiply-adds per component, the prolongation of its own share, and one
// 8-byte store.  The coefficients are converted to pairs once per step
// (k_comb_prep_ds), so the level kernels run no FP64 instruction.
#include "../../include/st_host.h"
#include "dsfloat.h"
#include "kernels.h"

namespace st {
namespace {

constexpr int kCombThreads = 256;
constexpr int kCombMaxChunk = 256;
constexpr int kCombRegComps = 2;  // components held in registers per level
constexpr int kCombChunk = 32;     // target times per CTA (at most kCombMaxChunk)

// comps[c]: the component's coefficient pairs, the sign of its coefficient
// applied and u0 folded in (U_ds[i][a] = coef (U[i][a] + u0(x_a))), and
// coef u0 on all nodes of its level (null when u0 = 0), from k_comb_prep_ds.
template <int D, int NR, bool FINAL>
__global__ void __launch_bounds__(kCombThreads, D == 3 ? 2 : 3)
    k_comb_ds(int j, const ds* __restrict__ Yprev, const CombCompDS* __restrict__ comps, int c0, int c1,
              const float* __restrict__ tbw, const int* __restrict__ tspan, int nts, int L, ds* __restrict__ Yp,
              double* __restrict__ Yd, FastDiv dQ1) {
  constexpr int NE = 1 << D;
  __shared__ float sw[NR > 0 ? NR : 1][kCombMaxChunk + 1][3];
  __shared__ int ssp[NR > 0 ? NR : 1][kCombMaxChunk + 1];
  const int Nj = 1 << j, Nc = Nj >> 1;
  int64_t ncs = 1, nsp = 1;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    ncs *= (Nc + 1);
    nsp *= (Nj + 1);
  }
  const int s0 = blockIdx.y * L;
  const int s1 = (s0 + L >= nts - 1) ? nts : s0 + L;  // the last chunk also takes t = T
  // this chunk's weights and spans of the register-held components
  for (int i = threadIdx.x; i < NR * (s1 - s0); i += kCombThreads) {
    const int r = i / (s1 - s0), ds_ = i - r * (s1 - s0);
    const int64_t row = (int64_t)(c0 + r) * nts + s0 + ds_;
    ssp[r][ds_] = tspan[row];
    sw[r][ds_][0] = tbw[row * 3 + 0];
    sw[r][ds_][1] = tbw[row * 3 + 1];
    sw[r][ds_][2] = tbw[row * 3 + 2];
  }
  __syncthreads();
  const int64_t qi = (int64_t)blockIdx.x * kCombThreads + threadIdx.x;
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
  // owned level-j nodes: flat index, inside the grid, interior
  int64_t pidx[NE];
  bool inside[NE], interior[NE];
#pragma unroll
  for (int e = 0; e < NE; ++e) {
    int64_t idx = 0, st = 1;
    bool in = true, it = true;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const int P = 2 * Q[k] + ((e >> k) & 1);
      in = in && P <= Nj;
      it = it && P >= 1 && P <= Nj - 1;
      idx += (int64_t)P * st;
      st *= (Nj + 1);
    }
    pidx[e] = idx;
    inside[e] = in;
    interior[e] = it;
  }
  // coarse corners Q + e of level j-1 (absent outside the grid)
  int64_t cidx[NE];
  bool cok[NE];
#pragma unroll
  for (int e = 0; e < NE; ++e) {
    int64_t idx = 0, st = 1;
    bool ok = true;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const int b = (e >> k) & 1;
      ok = ok && (Q[k] + b <= Nc);
      idx += (int64_t)(Q[k] + b) * st;
      st *= (Nc + 1);
    }
    cidx[e] = idx;
    cok[e] = ok && Yprev != nullptr;
  }
  // coefficient pair of owned node e in time row `row` of component cc (the
  // lifting alone outside the interior and for the removed first B-spline)
  auto coeff = [&](const CombCompDS& cc, int e, int row) -> ds {
    const int sh = cc.jx - j;
    const int N = 1 << cc.jx, n = N - 1, nt = (1 << cc.jt) + 1;
    int64_t ii = 0, ia = 0, nx = 1, sa = 1;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const int P = (2 * Q[k] + ((e >> k) & 1)) << sh;
      ii += (int64_t)(P - 1) * nx;
      ia += (int64_t)P * sa;
      nx *= n;
      sa *= (N + 1);
    }
    if (interior[e] && row >= 0 && row < nt) return cc.U[(int64_t)row * nx + ii];
    return (cc.lift != nullptr && inside[e]) ? cc.lift[ia] : ds{0.0f, 0.0f};
  };
  // three time coefficients of every owned node for each register-held component
  ds cf[NR > 0 ? NR : 1][NE][3];
  int cur[NR > 0 ? NR : 1];
#pragma unroll
  for (int r = 0; r < NR; ++r) cur[r] = -1;

  // level j-1 values at the chunk's first time; the next time's are loaded
  // one step ahead
  ds fn[NE];
#pragma unroll
  for (int e = 0; e < NE; ++e) fn[e] = cok[e] ? Yprev[(int64_t)s0 * ncs + cidx[e]] : ds{0.0f, 0.0f};
  for (int s = s0; s < s1; ++s) {
    ds f[NE];
#pragma unroll
    for (int e = 0; e < NE; ++e) f[e] = fn[e];
    if (s + 1 < s1) {
#pragma unroll
      for (int e = 0; e < NE; ++e)
        if (cok[e]) fn[e] = Yprev[(int64_t)(s + 1) * ncs + cidx[e]];
    }
    // prolongation: midpoints averaged direction by direction
    if (Yprev != nullptr) {
#pragma unroll
      for (int k = 0; k < D; ++k) {
#pragma unroll
        for (int e = 0; e < NE; ++e)
          if ((e >> k) & 1) f[e] = ds_scale(ds_add(f[e ^ (1 << k)], f[e]), 0.5f);
      }
    }
    float S[NE], lo[NE];
#pragma unroll
    for (int e = 0; e < NE; ++e) {
      S[e] = f[e].h;
      lo[e] = f[e].l;
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      const int sp = ssp[r][s - s0];
      if (sp != cur[r]) {
        const CombCompDS cc = comps[c0 + r];
#pragma unroll
        for (int e = 0; e < NE; ++e)
#pragma unroll
          for (int t = 0; t < 3; ++t) cf[r][e][t] = coeff(cc, e, sp + t - 1);
        cur[r] = sp;
      }
      const float w0 = sw[r][s - s0][0], w1 = sw[r][s - s0][1], w2 = sw[r][s - s0][2];
#pragma unroll
      for (int e = 0; e < NE; ++e) {
        ds_axpy(w0, cf[r][e][0], S[e], lo[e]);
        ds_axpy(w1, cf[r][e][1], S[e], lo[e]);
        ds_axpy(w2, cf[r][e][2], S[e], lo[e]);
      }
    }
    // components beyond the register-held ones (several components injected
    // into the target level): coefficients read at every time
    for (int c = c0 + NR; c < c1; ++c) {
      const CombCompDS cc = comps[c];
      const int span = tspan[(int64_t)c * nts + s];
      const float* w = tbw + ((int64_t)c * nts + s) * 3;
#pragma unroll
      for (int e = 0; e < NE; ++e)
        for (int t = 0; t < 3; ++t) ds_axpy(w[t], coeff(cc, e, span + t - 1), S[e], lo[e]);
    }
#pragma unroll
    for (int e = 0; e < NE; ++e) {
      if (!inside[e]) continue;
      const ds v = ds_norm(ds{S[e], lo[e]});
      if (FINAL) Yd[(int64_t)s * nsp + pidx[e]] = ds_to_double(v);
      else Yp[(int64_t)s * nsp + pidx[e]] = v;
    }
  }
}

// Pairs of one component for the level kernels: Uds[i][a] = coef (U[i][a] +
// u0(x_a)) on the interior nodes, Lds[b] = coef u0(x_b) on all nodes (either
// output may be null and is then skipped).
template <int D>
__global__ void __launch_bounds__(kCombThreads)
    k_comb_prep_ds(const double* __restrict__ U, const double* __restrict__ lift, int coef, int jx, int nt,
                   ds* __restrict__ Uds, ds* __restrict__ Lds) {
  const int N = 1 << jx, n = N - 1;
  int64_t nx = 1, na = 1;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    nx *= n;
    na *= (N + 1);
  }
  const int64_t e = (int64_t)blockIdx.x * kCombThreads + threadIdx.x;
  if (Uds != nullptr && e < nt * nx) {
    double v = U[e];
    if (lift != nullptr) {
      unsigned r = (unsigned)(e % nx);  // interior node (fewer than 2^31 per level)
      int64_t ia = 0, sa = 1;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const unsigned q = r / (unsigned)n;
        ia += (int64_t)(r - q * (unsigned)n + 1) * sa;
        r = q;
        sa *= (N + 1);
      }
      v += lift[ia];
    }
    Uds[e] = ds_from_double(coef > 0 ? v : -v);
  }
  if (Lds != nullptr && lift != nullptr && e < na) Lds[e] = ds_from_double(coef > 0 ? lift[e] : -lift[e]);
}

template <int D, int NR>
void launch_ds(bool final_level, dim3 grid, int j, const ds* Yprev, const CombCompDS* comps, int c0, int c1,
               const float* tbw, const int* tspan, int nts, int L, ds* Yp, double* Yd, FastDiv f, cudaStream_t s) {
  if (final_level)
    k_comb_ds<D, NR, true><<<grid, kCombThreads, 0, s>>>(j, Yprev, comps, c0, c1, tbw, tspan, nts, L, Yp, Yd, f);
  else
    k_comb_ds<D, NR, false><<<grid, kCombThreads, 0, s>>>(j, Yprev, comps, c0, c1, tbw, tspan, nts, L, Yp, Yd, f);
}

template <int D>
void launch_ds_d(int nr, bool final_level, dim3 grid, int j, const ds* Yprev, const CombCompDS* comps, int c0,
                 int c1, const float* tbw, const int* tspan, int nts, int L, ds* Yp, double* Yd, FastDiv f,
                 cudaStream_t s) {
  if (nr == 0) launch_ds<D, 0>(final_level, grid, j, Yprev, comps, c0, c1, tbw, tspan, nts, L, Yp, Yd, f, s);
  else if (nr == 1) launch_ds<D, 1>(final_level, grid, j, Yprev, comps, c0, c1, tbw, tspan, nts, L, Yp, Yd, f, s);
  else launch_ds<D, 2>(final_level, grid, j, Yprev, comps, c0, c1, tbw, tspan, nts, L, Yp, Yd, f, s);
}

}  // namespace

int comb_ds_chunk(int d, int j, int jt_star, const int* comp_jt, int ncomp_level) {
  const int nts1 = 1 << jt_star;  // target time intervals
  // chunks aligned to every register-held component's time intervals, and
  // short enough that a CTA finishes within tens of microseconds (so that
  // the solves of the next step, queued at a higher stream priority, find
  // free SM slots quickly while a level runs)
  int L = kCombChunk < nts1 ? kCombChunk : nts1;
  for (int r = 0; r < ncomp_level && r < kCombRegComps; ++r) {
    const int gap = jt_star - comp_jt[r];
    const int span_len = gap <= 0 ? 1 : (gap >= 30 ? (1 << 30) : (1 << gap));
    if (span_len < L) L = span_len;
  }
  // enough CTAs for the device: about 8 resident CTAs on each of ~150 SMs, twice over
  int64_t ncs = 1;
  for (int k = 0; k < d; ++k) ncs *= ((1 << j) / 2 + 1);
  const int64_t bx = (ncs + kCombThreads - 1) / kCombThreads;
  while (L > 4 && bx * (nts1 / L) < 2400) L >>= 1;
  return L < 1 ? 1 : L;
}

void launch_comb_prep_ds(int d, const double* U, const double* lift, int coef, int jx, int nt, ds* Uds, ds* Lds,
                         cudaStream_t s) {
  note_launches(1);
  int64_t nx = 1, na = 1;
  for (int k = 0; k < d; ++k) {
    nx *= (1 << jx) - 1;
    na *= (1 << jx) + 1;
  }
  const int64_t n = (Uds != nullptr && nt * nx > na) ? nt * nx : (Lds != nullptr ? na : nt * nx);
  const unsigned blocks = (unsigned)((n + kCombThreads - 1) / kCombThreads);
  if (d == 1) k_comb_prep_ds<1><<<blocks, kCombThreads, 0, s>>>(U, lift, coef, jx, nt, Uds, Lds);
  else if (d == 2) k_comb_prep_ds<2><<<blocks, kCombThreads, 0, s>>>(U, lift, coef, jx, nt, Uds, Lds);
  else k_comb_prep_ds<3><<<blocks, kCombThreads, 0, s>>>(U, lift, coef, jx, nt, Uds, Lds);
}

void launch_comb_level_ds(int d, int j, const void* Yprev, const CombCompDS* comps, int c0, int c1, const float* tbw,
                          const int* tspan, int nts, int L, void* Y, bool final_level, cudaStream_t s) {
  note_launches(1);
  int64_t ncs = 1;  // one thread per node of level j-1 (each writes up to 2^d level-j nodes)
  for (int k = 0; k < d; ++k) ncs *= ((1 << j) / 2 + 1);
  const int nchunks = ((nts - 1) + L - 1) / L;
  dim3 grid((unsigned)((ncs + kCombThreads - 1) / kCombThreads), (unsigned)nchunks);
  const FastDiv f = make_fastdiv((unsigned)((1 << j) / 2 + 1));
  const int nr = (c1 - c0) < kCombRegComps ? (c1 - c0) : kCombRegComps;
  const ds* Yp = static_cast<const ds*>(Yprev);
  ds* Ypair = final_level ? nullptr : static_cast<ds*>(Y);
  double* Yd = final_level ? static_cast<double*>(Y) : nullptr;
  if (d == 1) launch_ds_d<1>(nr, final_level, grid, j, Yp, comps, c0, c1, tbw, tspan, nts, L, Ypair, Yd, f, s);
  else if (d == 2) launch_ds_d<2>(nr, final_level, grid, j, Yp, comps, c0, c1, tbw, tspan, nts, L, Ypair, Yd, f, s);
  else launch_ds_d<3>(nr, final_level, grid, j, Yp, comps, c0, c1, tbw, tspan, nts, L, Ypair, Yd, f, s);
}

}  // namespace st

extern "C" st_status st_host_ds_to_double(const float* h, const float* l, int64_t n, double* out) {
  if (n < 0 || (n > 0 && (h == nullptr || l == nullptr || out == nullptr))) return ST_ERR_ARG;
  for (int64_t i = 0; i < n; ++i) out[i] = st::ds_to_double(st::ds{h[i], l[i]});
  return ST_OK;
}
