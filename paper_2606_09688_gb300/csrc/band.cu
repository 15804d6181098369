// Banded complex-symmetric LDL^T: assembly, factorisation and the solve of
// the spatial problems (K + lam_q M) x = b on grids small enough for a direct
// method (whole component grids, or the coarsest multigrid level).
//
// Storage (per mode q, at q * mstride): row k of F holds column k of L,
// F[k][t] = L_{k+t,k} (t = 1..bw) and F[k][0] = 1/d_k; row k of G holds row k of L,
// G[k][t] = L_{k,k-t}.  Rows are padded to an even length ld so that every
// row starts on a 16-byte boundary (TMA bulk copies).
//
// Solve: one warp per mode.  Forward (L y = b, column-oriented with F rows in
// increasing k) and backward (L^T x = z, column-oriented with G rows in
// decreasing k) share one routine.  The window of the bw pending
// right-hand-side rows is a shift register in registers: at step k, slot j
// (lane j mod 32, register j / 32) holds row k + j, so every lane applies the
// same band offsets at every step; row k+1 is broadcast from lane 1 right
// after its update, the window shifts down by one slot with shuffles, and the
// row entering at slot bw-1 takes a right-hand-side value staged in shared
// memory one chunk ahead.  Factor rows are streamed into shared memory in
// chunks by cp.async.bulk with mbarrier completion, two chunks in flight.
#include <atomic>
#include <cstdint>
#include <mutex>

#include <cooperative_groups.h>

#include "band.h"
#include "ptx.cuh"

namespace st {

namespace cg = cooperative_groups;

namespace {

constexpr int kBlock = 256;
inline unsigned blocks_for(int64_t n, int per = kBlock) { return (unsigned)((n + per - 1) / per); }

// ------------------------------------------------------------- assembly
template <typename R>
__global__ void k_band_form(const double* __restrict__ Kb, const double* __restrict__ Mb,
                            const cx<double>* __restrict__ lam, cx<R>* __restrict__ F, BandLayout L) {
  const int q = blockIdx.y;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int W = L.bw + 1;
  if (e >= L.nrow * L.ld) return;
  const int64_t k = e / L.ld;
  const int t = (int)(e - k * L.ld);
  cx<R> v = mk<R>(0, 0);
  if (t < W) {
    const cx<double> l = lam[q];
    const double kb = Kb[k * W + t], mb = Mb[k * W + t];
    v = mk<R>((R)(kb + l.re * mb), (R)(l.im * mb));
  }
  F[(int64_t)q * L.mstride + e] = v;
}

// Right-looking LDL^T without pivoting of a complex-symmetric band (see
// band.h for why no pivot is needed).  One CTA per mode; column k:
// a_{k+i,k+j} -= a_{k+i,k} a_{k+j,k} / d_k, then l_{k+i,k} = a_{k+i,k} / d_k.
template <typename R>
__global__ void k_band_ldlt(cx<R>* __restrict__ F, BandLayout L, int* err) {
  extern __shared__ unsigned char smem_raw[];
  cx<R>* col = reinterpret_cast<cx<R>*>(smem_raw);
  const int q = blockIdx.x;
  const int bw = L.bw, ld = L.ld;
  const int64_t nrow = L.nrow;
  cx<R>* Fq = F + (int64_t)q * L.mstride;
  for (int64_t k = 0; k < nrow; ++k) {
    __syncthreads();
    for (int t = threadIdx.x; t <= bw; t += blockDim.x) col[t] = (k + t < nrow) ? Fq[k * ld + t] : mk<R>(0, 0);
    __syncthreads();
    const cx<R> d = col[0];
    if (!(d.re * d.re + d.im * d.im > R(0))) {
      if (threadIdx.x == 0) atomicExch(err, 1);
      return;
    }
    const cx<R> dinv = cdiv(mk<R>(1, 0), d);
    const int m = (int)((nrow - 1 - k) < (int64_t)bw ? (nrow - 1 - k) : bw);
    // pairs (ii, jj) with 1 <= jj <= ii <= m, enumerated row by row of the lower triangle
    const int npairs = m * (m + 1) / 2;
    for (int p = threadIdx.x; p < npairs; p += blockDim.x) {
      int ii = (int)((sqrtf(8.0f * p + 1.0f) - 1.0f) * 0.5f);
      while (ii * (ii + 1) / 2 > p) --ii;
      while ((ii + 1) * (ii + 2) / 2 <= p) ++ii;
      const int jj = p - ii * (ii + 1) / 2;  // 0 <= jj <= ii
      const int i1 = ii + 1, j1 = jj + 1;
      cx<R>& tgt = Fq[(k + j1) * ld + (i1 - j1)];
      tgt = tgt - (col[i1] * col[j1]) * dinv;
    }
    __syncthreads();
    for (int t = threadIdx.x + 1; t <= m; t += blockDim.x) Fq[k * ld + t] = col[t] * dinv;
    if (threadIdx.x == 0) Fq[k * ld] = dinv;  // the solve multiplies by 1/d_k
  }
}

// The same factorisation with the active window in shared memory: column c
// of the trailing matrix (rows c..c+bw) lives in slot c mod P, P = bw + 1,
// entry t at win[slot * P + t].  At column k every pair 1 <= j <= i <= m
// takes a_{k+i,k+j} -= (a_{k+i,k} / d_k) a_{k+j,k}; thread (i, p) owns row
// offset i and the column offsets j = 1 + p, 1 + p + NP, ..., so a warp
// (consecutive i, one j) reads and writes consecutive words of one slot.
// Then column k leaves for global memory (as L and 1/d_k) and column k + P
// (untouched so far: no column before k + 1 reaches it) enters its slot.
template <typename R>
__global__ void k_band_ldlt_win(cx<R>* __restrict__ F, BandLayout L, int RI, int NP, int* err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<R>* win = reinterpret_cast<cx<R>*>(smem_raw);
  const int q = blockIdx.x;
  const int bw = L.bw, ld = L.ld, P = bw + 1;
  const int64_t nrow = L.nrow;
  cx<R>* Fq = F + (int64_t)q * L.mstride;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int i = 1 + tid % RI, p = tid / RI;
  const cx<R> zero = mk<R>(0, 0);
  for (int e = tid; e < P * P; e += nth) {
    const int c = e / P, t = e - (e / P) * P;
    win[e] = (c < nrow && c + t < nrow) ? Fq[(int64_t)c * ld + t] : zero;
  }
  __syncthreads();
  int slot0 = 0;  // k mod P
  for (int64_t k = 0; k < nrow; ++k) {
    const cx<R>* colk = win + slot0 * P;
    const cx<R> d = colk[0];
    if (!(d.re * d.re + d.im * d.im > R(0))) {
      if (tid == 0) atomicExch(err, 1);
      return;
    }
    const cx<R> dinv = cdiv(mk<R>(1, 0), d);
    const int m = (int)((nrow - 1 - k) < (int64_t)bw ? (nrow - 1 - k) : bw);
    if (i <= m) {
      const cx<R> u = colk[i] * dinv;
      for (int j = 1 + p; j <= i; j += NP) {
        int sj = slot0 + j;
        if (sj >= P) sj -= P;
        cx<R>& tgt = win[sj * P + (i - j)];
        const cx<R> a = colk[j];
        tgt = mk<R>(fma(-u.re, a.re, fma(u.im, a.im, tgt.re)), fma(-u.re, a.im, fma(-u.im, a.re, tgt.im)));
      }
    }
    __syncthreads();
    // column k of L (with 1/d_k in place of the unit diagonal) to global
    // memory, and column k + P into the freed slot (entry t by one thread)
    const int64_t c = k + P;
    for (int t = tid; t < P; t += nth) {
      if (t <= m) Fq[k * ld + t] = t == 0 ? dinv : colk[t] * dinv;
      win[slot0 * P + t] = (c < nrow && c + t < nrow) ? Fq[c * ld + t] : zero;
    }
    __syncthreads();
    slot0 = slot0 + 1 == P ? 0 : slot0 + 1;
  }
}

// The shared-memory window of k_band_ldlt_win spread over a cluster of NC
// CTAs, for windows that exceed one CTA's shared memory (FP64 with a half
// bandwidth of 128: 266 KB): window slot s lives in CTA s mod NC, so every
// update of a column happens in the CTA that holds it.  Per column each CTA
// copies the pivot column from its owner's shared memory (distributed shared
// memory), updates the columns it holds, and one cluster barrier orders those
// reads and updates before the owner stores column k of L and reuses the slot
// and before the next pivot column is read.  Every CTA reads the same pivot,
// so all take the same number of barriers, also on a zero pivot.  Element by
// element the same arithmetic as the single-CTA window kernel.
template <typename R, int NC>
__global__ void __cluster_dims__(NC, 1, 1) __launch_bounds__(256)
    k_band_ldlt_dsm(cx<R>* __restrict__ F, BandLayout L, int RI, int NP, int* err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int q = blockIdx.x / NC;
  const int bw = L.bw, ld = L.ld, P = bw + 1;
  const int nls = (P + NC - 1) / NC;  // window slots per CTA (slot s = ls NC + rank)
  cx<R>* win = reinterpret_cast<cx<R>*>(smem_raw);
  cx<R>* pc = win + (size_t)nls * P;  // this CTA's copy of the pivot column
  const int64_t nrow = L.nrow;
  cx<R>* Fq = F + (int64_t)q * L.mstride;
  const int tid = threadIdx.x, nth = blockDim.x;
  const cx<R> zero = mk<R>(0, 0);
  for (int e = tid; e < nls * P; e += nth) {
    const int ls = e / P, t = e - ls * P;
    const int c = ls * NC + rank;  // slot c holds column c at the start
    win[e] = (c < P && c < nrow && c + t < nrow) ? Fq[(int64_t)c * ld + t] : zero;
  }
  cluster.sync();
  int slot0 = 0;  // k mod P
  for (int64_t k = 0; k < nrow; ++k) {
    const int m = (int)((nrow - 1 - k) < (int64_t)bw ? (nrow - 1 - k) : bw);
    const int own = slot0 % NC;
    const cx<R>* src = cluster.map_shared_rank(win, own) + (size_t)(slot0 / NC) * P;
    for (int t = tid; t <= m; t += nth) pc[t] = src[t];
    __syncthreads();
    const cx<R> d = pc[0];
    if (!(d.re * d.re + d.im * d.im > R(0))) {
      if (tid == 0 && rank == 0) atomicExch(err, 1);
      cluster.sync();  // no CTA leaves while another may still read its shared memory
      return;
    }
    const cx<R> dinv = cdiv(mk<R>(1, 0), d);
    for (int i = 1 + tid % RI; i <= m; i += RI) {
      const cx<R> u = pc[i] * dinv;
      for (int ls = tid / RI; ls < nls; ls += NP) {
        const int s = ls * NC + rank;
        if (s >= P) continue;
        int j = s - slot0;
        if (j < 0) j += P;
        if (j < 1 || j > i) continue;
        cx<R>& tgt = win[(size_t)ls * P + (i - j)];
        const cx<R> a = pc[j];
        tgt = mk<R>(fma(-u.re, a.re, fma(u.im, a.im, tgt.re)), fma(-u.re, a.im, fma(-u.im, a.re, tgt.im)));
      }
    }
    cluster.sync();
    if (rank == own) {
      // column k of L (with 1/d_k in place of the unit diagonal), then column
      // k + P into the freed slot
      const int64_t c = k + P;
      cx<R>* slot = win + (size_t)(slot0 / NC) * P;
      for (int t = tid; t < P; t += nth) {
        if (t <= m) Fq[k * ld + t] = t == 0 ? dinv : pc[t] * dinv;
        slot[t] = (c < nrow && c + t < nrow) ? Fq[c * ld + t] : zero;
      }
    }
    __syncthreads();
    slot0 = slot0 + 1 == P ? 0 : slot0 + 1;
  }
}

// The global-memory factorisation spread over a cluster of kLdltCluster CTAs
// per mode (bands whose window does not fit in shared memory): every CTA
// reads column k, updates its share of the pairs (i, j) (column offsets
// j = 1 + rank, 1 + rank + kLdltCluster * NP, ...), and one cluster barrier
// (release / acquire) per column makes the updates visible before column
// k + 1 is read; rank 0 then stores column k of L (no CTA reads row k again).
// Every CTA sees the same pivot, so a zero pivot returns all of them together.
constexpr int kLdltCluster = 4;
template <typename R>
__global__ void __cluster_dims__(kLdltCluster, 1, 1) __launch_bounds__(256)
    k_band_ldlt_cl(cx<R>* __restrict__ F, BandLayout L, int RI, int NP, int* err) {
  extern __shared__ unsigned char smem_raw[];
  cx<R>* col = reinterpret_cast<cx<R>*>(smem_raw);
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int q = blockIdx.x / kLdltCluster;
  const int bw = L.bw, ld = L.ld;
  const int64_t nrow = L.nrow;
  cx<R>* Fq = F + (int64_t)q * L.mstride;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int p = tid / RI;
  const int jstep = NP * kLdltCluster;
  for (int64_t k = 0; k < nrow; ++k) {
    for (int t = tid; t <= bw; t += nth) col[t] = (k + t < nrow) ? Fq[k * ld + t] : mk<R>(0, 0);
    __syncthreads();
    const cx<R> d = col[0];
    if (!(d.re * d.re + d.im * d.im > R(0))) {
      if (tid == 0 && rank == 0) atomicExch(err, 1);
      return;
    }
    const cx<R> dinv = cdiv(mk<R>(1, 0), d);
    const int m = (int)((nrow - 1 - k) < (int64_t)bw ? (nrow - 1 - k) : bw);
    // row offsets i = 1 + tid mod RI, + RI, ... (bands wider than the CTA take several)
    for (int i = 1 + tid % RI; i <= m; i += RI) {
      const cx<R> u = col[i] * dinv;
      int j = 1 + rank + kLdltCluster * p;
      // four column offsets at a time: their four target words are loaded
      // before any is stored (distinct columns), so four requests are in flight
      for (; j + 3 * jstep <= i; j += 4 * jstep) {
        cx<R>* tg[4];
        cx<R> v[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) tg[r] = Fq + (k + j + r * jstep) * ld + (i - j - r * jstep);
#pragma unroll
        for (int r = 0; r < 4; ++r) v[r] = *tg[r];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const cx<R> a = col[j + r * jstep];
          *tg[r] = mk<R>(fma(-u.re, a.re, fma(u.im, a.im, v[r].re)), fma(-u.re, a.im, fma(-u.im, a.re, v[r].im)));
        }
      }
      for (; j <= i; j += jstep) {
        cx<R>& tgt = Fq[(k + j) * ld + (i - j)];
        const cx<R> a = col[j];
        tgt = mk<R>(fma(-u.re, a.re, fma(u.im, a.im, tgt.re)), fma(-u.re, a.im, fma(-u.im, a.re, tgt.im)));
      }
    }
    cluster.sync();
    // column k of L (1/d_k in slot 0) by rank 0, after every CTA has read it
    if (rank == 0)
      for (int t = tid; t <= m; t += nth) Fq[k * ld + t] = t == 0 ? dinv : col[t] * dinv;
    __syncthreads();
  }
}

template <typename R>
__global__ void k_band_rows(const cx<R>* __restrict__ F, cx<R>* __restrict__ G, BandLayout L) {
  const int q = blockIdx.y;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= L.nrow * L.ld) return;
  const int64_t k = e / L.ld;
  const int t = (int)(e - k * L.ld);
  cx<R> v = mk<R>(0, 0);
  if (t == 0) v = F[(int64_t)q * L.mstride + k * L.ld];
  else if (t <= L.bw && k - t >= 0) v = F[(int64_t)q * L.mstride + (k - t) * L.ld + t];
  G[(int64_t)q * L.mstride + e] = v;
}

// ----------------------------------------------------------------- solve
template <typename R, int SLOTS>
__global__ void __launch_bounds__(32) k_band_solve_w(const cx<R>* __restrict__ F, const cx<R>* __restrict__ G,
                                                     BandLayout L, int C, const cx<R>* __restrict__ b,
                                                     cx<R>* __restrict__ x, const CocgScal* __restrict__ scal,
                                                     int64_t vstride, int* err) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int q = blockIdx.x;
  if (scal != nullptr && !scal[q].active) return;
  const int lane = threadIdx.x;
  const int bw = L.bw, ld = L.ld, nrow = (int)L.nrow;
  const size_t stage_elems = (size_t)C * ld;
  cx<R>* stage0 = reinterpret_cast<cx<R>*>(smem);
  cx<R>* stage1 = stage0 + stage_elems;
  cx<R>* bin = stage1 + stage_elems;  // 2 x 32 incoming right-hand-side values
  uint64_t* bar = reinterpret_cast<uint64_t*>(bin + 64);
  if (lane == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_fence_init();
  }
  __syncwarp();
  unsigned phase[2] = {0u, 0u};
  const int nchunks = (nrow + C - 1) / C;
  const int elane = (bw - 1) & 31, eslot = (bw - 1) >> 5;  // slot bw-1: where rows enter
  cx<R>* dst = x + (int64_t)q * vstride;
  const cx<R> zero = mk<R>(0, 0);
  for (int pass = 0; pass < 2; ++pass) {
    const cx<R>* Mq = (pass == 0 ? F : G) + (int64_t)q * L.mstride;
    const cx<R>* src = pass == 0 ? b + (int64_t)q * vstride : dst;
    auto chunk = [&](int c, int& klo, int& cnt) {
      const int k0 = c * C;
      cnt = min(C, nrow - k0);
      klo = pass == 0 ? k0 : nrow - k0 - cnt;
    };
    // fault injection for the failure tests: the first copy is never issued,
    // so its bounded wait runs out (nothing is left in flight for it)
    const bool withhold0 = L.stall != 0 && pass == 0;
    auto issue = [&](int c) {
      if (withhold0 && c == 0) return;
      int klo, cnt;
      chunk(c, klo, cnt);
      cx<R>* st = (c & 1) ? stage1 : stage0;
      const unsigned bytes = (unsigned)((size_t)cnt * ld * sizeof(cx<R>));
      mbar_expect_tx(&bar[c & 1], bytes);
      bulk_g2s(st, Mq + (int64_t)klo * ld, bytes, &bar[c & 1]);
    };
    auto at = [&](int rp) -> cx<R> {  // right-hand side of pass-order row rp (zero past the end)
      if (rp >= nrow) return zero;
      return src[pass == 0 ? rp : nrow - 1 - rp];
    };
    if (lane == 0) {
      issue(0);
      if (nchunks > 1) issue(1);
    }
    // rows entering during chunk c: pass-order rows c*C + i + bw, i < C (one per lane)
    bin[lane] = lane < C ? at(lane + bw) : zero;
    cx<R> v[SLOTS];
#pragma unroll
    for (int s = 0; s < SLOTS; ++s) {
      const int j = lane + 32 * s;
      v[s] = j < bw ? at(j) : zero;
    }
    __syncwarp();
    cx<R> y;  // value of the row finished at the current step
    y.re = __shfl_sync(0xffffffffu, v[0].re, 0);
    y.im = __shfl_sync(0xffffffffu, v[0].im, 0);
    bool ok = true;
    for (int c = 0; c < nchunks; ++c) {
      // prefetch the right-hand sides entering during the next chunk
      const cx<R> pre = lane < C ? at((c + 1) * C + lane + bw) : zero;
      ok = mbar_wait_bounded(&bar[c & 1], phase[c & 1], L.wait > 0 ? L.wait : (1ll << 31));
      if (!__all_sync(0xffffffffu, ok)) {
        ok = false;
        break;
      }
      phase[c & 1] ^= 1u;
      int klo, cnt;
      chunk(c, klo, cnt);
      const cx<R>* st = (c & 1) ? stage1 : stage0;
      const cx<R>* bc = bin + (c & 1) * 32;
      for (int i = 0; i < cnt; ++i) {
        const int kp = c * C + i;
        const int k = pass == 0 ? kp : nrow - 1 - kp;
        const cx<R>* row = st + (size_t)(k - klo) * ld;
        if (lane == 0) {
          const cx<R> dinv = row[0];
          dst[k] = pass == 0 ? y * dinv : y;
        }
        // update the rows k+j (slots j >= 1) and the entering row k+bw
#pragma unroll
        for (int s = 0; s < SLOTS; ++s) {
          const int j = lane + 32 * s;
          if (j >= 1 && j < bw) {
            const cx<R> a = row[j];
            v[s] = mk<R>(v[s].re - (a.re * y.re - a.im * y.im), v[s].im - (a.re * y.im + a.im * y.re));
          }
        }
        cx<R> ent = zero;
        if (lane == elane) {
          const cx<R> a = row[bw];
          const cx<R> bi = bc[i];
          ent = mk<R>(bi.re - (a.re * y.re - a.im * y.im), bi.im - (a.re * y.im + a.im * y.re));
        }
        // row k+1 (slot 1, lane 1) is final: broadcast it, then shift the window
        // (with bw = 1 the next row is the entering one)
        const cx<R> src_next = bw > 1 ? v[0] : ent;
        cx<R> yn;
        yn.re = __shfl_sync(0xffffffffu, src_next.re, bw > 1 ? 1 : elane);
        yn.im = __shfl_sync(0xffffffffu, src_next.im, bw > 1 ? 1 : elane);
#pragma unroll
        for (int s = 0; s < SLOTS; ++s) {
          cx<R> up;
          up.re = __shfl_down_sync(0xffffffffu, v[s].re, 1);
          up.im = __shfl_down_sync(0xffffffffu, v[s].im, 1);
          if (s + 1 < SLOTS) {
            cx<R> nx;
            nx.re = __shfl_sync(0xffffffffu, v[s + 1].re, 0);
            nx.im = __shfl_sync(0xffffffffu, v[s + 1].im, 0);
            if (lane == 31) up = nx;
          }
          v[s] = up;
        }
#pragma unroll
        for (int s = 0; s < SLOTS; ++s)
          if (s == eslot && lane == elane) v[s] = ent;
        y = yn;
      }
      __syncwarp();
      bin[((c + 1) & 1) * 32 + lane] = pre;
      __syncwarp();
      if (lane == 0 && c + 2 < nchunks) issue(c + 2);
    }
    if (!ok) {
      // give the copies still in flight a bounded chance to land, then report
      if (lane == 0) {
        atomicExch(err, 2);
        for (int c2 = 0; c2 < 2; ++c2)
          if (!(withhold0 && c2 == 0)) mbar_wait_bounded(&bar[c2], phase[c2]);
      }
      return;
    }
    __syncwarp();
  }
}

// Variant for bw = 32 * SLOTS (every 2D grid: bw = 2^j): rows keep their
// register slot for their whole life (row r in lane r mod 32, register
// (r mod bw) / 32), so no data moves between lanes except the broadcast of
// the finished row.  Chunks are 32 rows, one group of 32 unrolled steps in
// which every band offset is a compile-time constant; SG = chunk mod SLOTS is
// the register that holds the rows finished during the chunk.
template <typename R, int SLOTS, int PASS, int SG>
__device__ __forceinline__ void band_group32(const cx<R>* __restrict__ st, int c, int nrow, int ld, int lane,
                                             cx<R> (&v)[SLOTS], const cx<R>& bcur, cx<R>& y,
                                             cx<R>* __restrict__ dst) {
  constexpr int bw = 32 * SLOTS;
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    const cx<R>* row = st + (size_t)(PASS == 0 ? i : 31 - i) * ld;
    if (lane == i) {
      const int kp = 32 * c + i;
      const int k = PASS == 0 ? kp : nrow - 1 - kp;
      dst[k] = PASS == 0 ? y * row[0] : y;
    }
#pragma unroll
    for (int s = 0; s < SLOTS; ++s) {
      if (s == SG) {
        // lanes after i hold rows kp + (lane - i); lanes before i already hold
        // rows entered during this chunk (t = lane - i + bw); lane i takes row kp + bw
        const int t = lane - i + (lane <= i ? bw : 0);
        const cx<R> a = row[t];
        const cx<R> base = lane == i ? bcur : v[s];
        v[s] = mk<R>(fma(-a.re, y.re, fma(a.im, y.im, base.re)), fma(-a.re, y.im, fma(-a.im, y.re, base.im)));
      } else {
        const int d = (s - SG + SLOTS) % SLOTS;
        const cx<R> a = row[lane - i + 32 * d];
        v[s] = mk<R>(fma(-a.re, y.re, fma(a.im, y.im, v[s].re)), fma(-a.re, y.im, fma(-a.im, y.re, v[s].im)));
      }
    }
    const int nslot = (i < 31) ? SG : (SG + 1) % SLOTS;
    y.re = __shfl_sync(0xffffffffu, v[nslot].re, (i + 1) & 31);
    y.im = __shfl_sync(0xffffffffu, v[nslot].im, (i + 1) & 31);
  }
}

// One step with a run-time step index (the last, partial chunk).
template <typename R, int SLOTS, int PASS>
__device__ __forceinline__ void band_step_rt(const cx<R>* __restrict__ row, int i, int sg, int c, int nrow,
                                             int lane, cx<R> (&v)[SLOTS], const cx<R>& bcur, cx<R>& y,
                                             cx<R>* __restrict__ dst) {
  constexpr int bw = 32 * SLOTS;
  if (lane == i) {
    const int kp = 32 * c + i;
    const int k = PASS == 0 ? kp : nrow - 1 - kp;
    dst[k] = PASS == 0 ? y * row[0] : y;
  }
#pragma unroll
  for (int s = 0; s < SLOTS; ++s) {
    int t;
    cx<R> base = v[s];
    if (s == sg) {
      t = lane - i + (lane <= i ? bw : 0);
      if (lane == i) base = bcur;
    } else {
      t = lane - i + 32 * ((s - sg + SLOTS) % SLOTS);
    }
    const cx<R> a = row[t];
    v[s] = mk<R>(fma(-a.re, y.re, fma(a.im, y.im, base.re)), fma(-a.re, y.im, fma(-a.im, y.re, base.im)));
  }
  const int nslot = (i < 31) ? sg : (sg + 1) % SLOTS;
  cx<R> src = v[0];
#pragma unroll
  for (int s = 1; s < SLOTS; ++s)
    if (s == nslot) src = v[s];
  y.re = __shfl_sync(0xffffffffu, src.re, (i + 1) & 31);
  y.im = __shfl_sync(0xffffffffu, src.im, (i + 1) & 31);
}

template <typename R, int SLOTS, int PASS>
__device__ __forceinline__ void band_group_dispatch(const cx<R>* st, int c, int nrow, int ld, int lane,
                                                    cx<R> (&v)[SLOTS], const cx<R>& bcur, cx<R>& y, cx<R>* dst) {
  const int sg = c % SLOTS;
  if (SLOTS == 1 || sg == 0) band_group32<R, SLOTS, PASS, 0>(st, c, nrow, ld, lane, v, bcur, y, dst);
  else if (SLOTS >= 2 && sg == 1) band_group32<R, SLOTS, PASS, (SLOTS >= 2 ? 1 : 0)>(st, c, nrow, ld, lane, v, bcur, y, dst);
  else if (SLOTS >= 4 && sg == 2) band_group32<R, SLOTS, PASS, (SLOTS >= 4 ? 2 : 0)>(st, c, nrow, ld, lane, v, bcur, y, dst);
  else if (SLOTS >= 4 && sg == 3) band_group32<R, SLOTS, PASS, (SLOTS >= 4 ? 3 : 0)>(st, c, nrow, ld, lane, v, bcur, y, dst);
}

template <typename R, int SLOTS>
__global__ void __launch_bounds__(32) k_band_solve_p2(const cx<R>* __restrict__ F, const cx<R>* __restrict__ G,
                                                      BandLayout L, const cx<R>* __restrict__ b,
                                                      cx<R>* __restrict__ x, const CocgScal* __restrict__ scal,
                                                      int64_t vstride, int* err) {
  constexpr int C = 32, bw = 32 * SLOTS;
  extern __shared__ __align__(128) unsigned char smem[];
  const int q = blockIdx.x;
  if (scal != nullptr && !scal[q].active) return;
  const int lane = threadIdx.x;
  const int ld = L.ld, nrow = (int)L.nrow;
  const size_t stage_elems = (size_t)C * ld;
  cx<R>* stage0 = reinterpret_cast<cx<R>*>(smem);
  cx<R>* stage1 = stage0 + stage_elems;
  uint64_t* bar = reinterpret_cast<uint64_t*>(stage1 + stage_elems);
  if (lane == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_fence_init();
  }
  __syncwarp();
  unsigned phase[2] = {0u, 0u};
  const int nchunks = (nrow + C - 1) / C;
  cx<R>* dst = x + (int64_t)q * vstride;
  const cx<R> zero = mk<R>(0, 0);
  for (int pass = 0; pass < 2; ++pass) {
    const cx<R>* Mq = (pass == 0 ? F : G) + (int64_t)q * L.mstride;
    const cx<R>* src = pass == 0 ? b + (int64_t)q * vstride : dst;
    auto chunk = [&](int c, int& klo, int& cnt) {
      const int k0 = c * C;
      cnt = min(C, nrow - k0);
      klo = pass == 0 ? k0 : nrow - k0 - cnt;
    };
    auto issue = [&](int c) {
      int klo, cnt;
      chunk(c, klo, cnt);
      cx<R>* st = (c & 1) ? stage1 : stage0;
      const unsigned bytes = (unsigned)((size_t)cnt * ld * sizeof(cx<R>));
      mbar_expect_tx(&bar[c & 1], bytes);
      bulk_g2s(st, Mq + (int64_t)klo * ld, bytes, &bar[c & 1]);
    };
    auto at = [&](int rp) -> cx<R> {
      if (rp >= nrow) return zero;
      return src[pass == 0 ? rp : nrow - 1 - rp];
    };
    if (lane == 0) {
      issue(0);
      if (nchunks > 1) issue(1);
    }
    cx<R> v[SLOTS];
#pragma unroll
    for (int s = 0; s < SLOTS; ++s) v[s] = at(lane + 32 * s);
    cx<R> bcur = at(lane + bw), bnext = at(C + lane + bw);
    cx<R> y;
    y.re = __shfl_sync(0xffffffffu, v[0].re, 0);
    y.im = __shfl_sync(0xffffffffu, v[0].im, 0);
    bool ok = true;
    for (int c = 0; c < nchunks; ++c) {
      ok = mbar_wait_bounded(&bar[c & 1], phase[c & 1]);
      if (!__all_sync(0xffffffffu, ok)) {
        ok = false;
        break;
      }
      phase[c & 1] ^= 1u;
      const cx<R> bnn = at((c + 2) * C + lane + bw);  // entering rows of chunk c + 2
      int klo, cnt;
      chunk(c, klo, cnt);
      const cx<R>* st = (c & 1) ? stage1 : stage0;
      if (cnt == C) {
        if (pass == 0) band_group_dispatch<R, SLOTS, 0>(st, c, nrow, ld, lane, v, bcur, y, dst);
        else band_group_dispatch<R, SLOTS, 1>(st, c, nrow, ld, lane, v, bcur, y, dst);
      } else {
        const int sg = c % SLOTS;
        for (int i = 0; i < cnt; ++i) {
          const cx<R>* row = st + (size_t)(pass == 0 ? i : cnt - 1 - i) * ld;
          if (pass == 0) band_step_rt<R, SLOTS, 0>(row, i, sg, c, nrow, lane, v, bcur, y, dst);
          else band_step_rt<R, SLOTS, 1>(row, i, sg, c, nrow, lane, v, bcur, y, dst);
        }
      }
      bcur = bnext;
      bnext = bnn;
      __syncwarp();
      if (lane == 0 && c + 2 < nchunks) issue(c + 2);
    }
    if (!ok) {
      if (lane == 0) {
        atomicExch(err, 2);
        for (int c2 = 0; c2 < 2; ++c2) mbar_wait_bounded(&bar[c2], phase[c2]);
      }
      return;
    }
    __syncwarp();
  }
}

// FP64 variant of the fixed-slot solve: GB300 issues FP64 at a small
// fraction of the FP32 rate per SM sub-partition, so one warp per mode is
// bound by the FP64 pipe of its sub-partition.  Here each of SLOTS warps owns
// one register slot (lanes hold rows r with (r mod bw) / 32 = warp), so the
// per-row complex FMAs of a mode spread over SLOTS sub-partitions; the
// finished row is passed through shared memory with one block barrier per row.
// (ybuf is written by other threads between the barriers, so it must not be a
// restrict pointer: that would let the compiler reuse an earlier load of it.)
template <typename R, int SLOTS, int PASS, int SG>
__device__ __forceinline__ void band_group32_mw(const cx<R>* __restrict__ st, int c, int nrow, int ld, int lane,
                                                int warp, cx<R>& v, const cx<R>& bcur, cx<R>& y,
                                                cx<R>* ybuf, cx<R>* __restrict__ dst) {
  constexpr int bw = 32 * SLOTS;
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    const cx<R>* row = st + (size_t)(PASS == 0 ? i : 31 - i) * ld;
    if (warp == SG && lane == i) {
      const int kp = 32 * c + i;
      const int k = PASS == 0 ? kp : nrow - 1 - kp;
      dst[k] = PASS == 0 ? y * row[0] : y;
    }
    if (warp == SG) {
      const int t = lane - i + (lane <= i ? bw : 0);
      const cx<R> a = row[t];
      const cx<R> base = lane == i ? bcur : v;
      v = mk<R>(fma(-a.re, y.re, fma(a.im, y.im, base.re)), fma(-a.re, y.im, fma(-a.im, y.re, base.im)));
    } else {
      const int d = (warp - SG + SLOTS) % SLOTS;
      const cx<R> a = row[lane - i + 32 * d];
      v = mk<R>(fma(-a.re, y.re, fma(a.im, y.im, v.re)), fma(-a.re, y.im, fma(-a.im, y.re, v.im)));
    }
    const int nslot = (i < 31) ? SG : (SG + 1) % SLOTS;
    if (warp == nslot && lane == ((i + 1) & 31)) ybuf[i & 1] = v;
    __syncthreads();
    y = ybuf[i & 1];
  }
}

template <typename R, int SLOTS>
__global__ void __launch_bounds__(32 * SLOTS) k_band_solve_mw(const cx<R>* __restrict__ F, const cx<R>* __restrict__ G,
                                                              BandLayout L, const cx<R>* __restrict__ b,
                                                              cx<R>* __restrict__ x, const CocgScal* __restrict__ scal,
                                                              int64_t vstride, int* err) {
  constexpr int C = 32, bw = 32 * SLOTS;
  extern __shared__ __align__(128) unsigned char smem[];
  const int q = blockIdx.x;
  if (scal != nullptr && !scal[q].active) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ld = L.ld, nrow = (int)L.nrow;
  const size_t stage_elems = (size_t)C * ld;
  cx<R>* stage0 = reinterpret_cast<cx<R>*>(smem);
  cx<R>* stage1 = stage0 + stage_elems;
  cx<R>* ybuf = stage1 + stage_elems;  // 2 entries
  uint64_t* bar = reinterpret_cast<uint64_t*>(ybuf + 2);
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_fence_init();
  }
  __syncthreads();
  unsigned phase[2] = {0u, 0u};
  const int nchunks = (nrow + C - 1) / C;
  cx<R>* dst = x + (int64_t)q * vstride;
  const cx<R> zero = mk<R>(0, 0);
  for (int pass = 0; pass < 2; ++pass) {
    const cx<R>* Mq = (pass == 0 ? F : G) + (int64_t)q * L.mstride;
    const cx<R>* src = pass == 0 ? b + (int64_t)q * vstride : dst;
    auto chunk = [&](int c, int& klo, int& cnt) {
      const int k0 = c * C;
      cnt = min(C, nrow - k0);
      klo = pass == 0 ? k0 : nrow - k0 - cnt;
    };
    auto issue = [&](int c) {
      int klo, cnt;
      chunk(c, klo, cnt);
      cx<R>* st = (c & 1) ? stage1 : stage0;
      const unsigned bytes = (unsigned)((size_t)cnt * ld * sizeof(cx<R>));
      mbar_expect_tx(&bar[c & 1], bytes);
      bulk_g2s(st, Mq + (int64_t)klo * ld, bytes, &bar[c & 1]);
    };
    auto at = [&](int rp) -> cx<R> {
      if (rp >= nrow) return zero;
      return src[pass == 0 ? rp : nrow - 1 - rp];
    };
    if (threadIdx.x == 0) {
      issue(0);
      if (nchunks > 1) issue(1);
    }
    cx<R> v = at(lane + 32 * warp);
    cx<R> bcur = at(lane + bw), bnext = at(C + lane + bw);
    if (threadIdx.x == 0) ybuf[1] = v;  // row 0 (lane 0 of warp 0)
    __syncthreads();
    cx<R> y = ybuf[1];
    bool ok = true;
    for (int c = 0; c < nchunks; ++c) {
      ok = mbar_wait_bounded(&bar[c & 1], phase[c & 1]);
      if (!__syncthreads_and(ok)) {
        ok = false;
        break;
      }
      phase[c & 1] ^= 1u;
      const cx<R> bnn = at((c + 2) * C + lane + bw);
      int klo, cnt;
      chunk(c, klo, cnt);
      const cx<R>* st = (c & 1) ? stage1 : stage0;
      const int sg = c % SLOTS;
      if (cnt == C) {
#define ST_MW_GROUP(P, S)                                                                            \
  if (sg == S) band_group32_mw<R, SLOTS, P, (S < SLOTS ? S : 0)>(st, c, nrow, ld, lane, warp, v, bcur, y, \
                                                                  ybuf, dst);
        if (pass == 0) {
          ST_MW_GROUP(0, 0) ST_MW_GROUP(0, 1) ST_MW_GROUP(0, 2) ST_MW_GROUP(0, 3)
        } else {
          ST_MW_GROUP(1, 0) ST_MW_GROUP(1, 1) ST_MW_GROUP(1, 2) ST_MW_GROUP(1, 3)
        }
#undef ST_MW_GROUP
      } else {
        for (int i = 0; i < cnt; ++i) {
          const cx<R>* row = st + (size_t)(pass == 0 ? i : cnt - 1 - i) * ld;
          if (warp == sg && lane == i) {
            const int kp = 32 * c + i;
            const int k = pass == 0 ? kp : nrow - 1 - kp;
            dst[k] = pass == 0 ? y * row[0] : y;
          }
          int t;
          cx<R> base = v;
          if (warp == sg) {
            t = lane - i + (lane <= i ? bw : 0);
            if (lane == i) base = bcur;
          } else {
            t = lane - i + 32 * ((warp - sg + SLOTS) % SLOTS);
          }
          const cx<R> a = row[t];
          v = mk<R>(fma(-a.re, y.re, fma(a.im, y.im, base.re)), fma(-a.re, y.im, fma(-a.im, y.re, base.im)));
          const int nslot = (i < 31) ? sg : (sg + 1) % SLOTS;
          if (warp == nslot && lane == ((i + 1) & 31)) ybuf[i & 1] = v;
          __syncthreads();
          y = ybuf[i & 1];
        }
      }
      bcur = bnext;
      bnext = bnn;
      __syncthreads();
      if (threadIdx.x == 0 && c + 2 < nchunks) issue(c + 2);
    }
    if (!ok) {
      if (threadIdx.x == 0) {
        atomicExch(err, 2);
        for (int c2 = 0; c2 < 2; ++c2) mbar_wait_bounded(&bar[c2], phase[c2]);
      }
      return;
    }
    __syncthreads();
  }
}

// Wide bands (3D grids: bw = n^2 + n + 1 up to 1024): the fixed-slot solve
// with one warp per 32-row slot of a window padded to W = 32 * NW >= bw rows
// (NW = ceil(bw / 32) warps; window offsets beyond bw have zero coupling), the
// band offsets computed at run time instead of unrolled.  Rows are staged in
// chunks of C rows (C divides 32) by bulk copies; the finished row of each
// step is passed through shared memory with one block barrier per row.
template <typename R>
__global__ void __launch_bounds__(1024) k_band_solve_mwg(const cx<R>* __restrict__ F, const cx<R>* __restrict__ G,
                                                         BandLayout L, int C, const cx<R>* __restrict__ b,
                                                         cx<R>* __restrict__ x, const CocgScal* __restrict__ scal,
                                                         int64_t vstride, int* err) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int q = blockIdx.x;
  if (scal != nullptr && !scal[q].active) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, NW = blockDim.x >> 5, W = 32 * NW;
  const int bw = L.bw, ld = L.ld, nrow = (int)L.nrow;
  const size_t stage_elems = (size_t)C * ld;
  cx<R>* stage0 = reinterpret_cast<cx<R>*>(smem);
  cx<R>* stage1 = stage0 + stage_elems;
  cx<R>* ybuf = stage1 + stage_elems;  // 2 entries, written by other threads between barriers
  uint64_t* bar = reinterpret_cast<uint64_t*>(ybuf + 2);
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_fence_init();
  }
  __syncthreads();
  unsigned phase[2] = {0u, 0u};
  const int nchunks = (nrow + C - 1) / C;
  cx<R>* dst = x + (int64_t)q * vstride;
  const cx<R> zero = mk<R>(0, 0);
  for (int pass = 0; pass < 2; ++pass) {
    const cx<R>* Mq = (pass == 0 ? F : G) + (int64_t)q * L.mstride;
    const cx<R>* src = pass == 0 ? b + (int64_t)q * vstride : dst;
    auto chunk = [&](int c, int& klo, int& cnt) {
      const int k0 = c * C;
      cnt = min(C, nrow - k0);
      klo = pass == 0 ? k0 : nrow - k0 - cnt;
    };
    auto issue = [&](int c) {
      int klo, cnt;
      chunk(c, klo, cnt);
      cx<R>* st = (c & 1) ? stage1 : stage0;
      const unsigned bytes = (unsigned)((size_t)cnt * ld * sizeof(cx<R>));
      mbar_expect_tx(&bar[c & 1], bytes);
      bulk_g2s(st, Mq + (int64_t)klo * ld, bytes, &bar[c & 1]);
    };
    auto at = [&](int rp) -> cx<R> {
      if (rp >= nrow) return zero;
      return src[pass == 0 ? rp : nrow - 1 - rp];
    };
    if (threadIdx.x == 0) {
      issue(0);
      if (nchunks > 1) issue(1);
    }
    cx<R> v = at(lane + 32 * warp);
    cx<R> bcur = at(lane + W), bnext = at(32 + lane + W);  // rows entering during groups 0 and 1
    if (threadIdx.x == 0) ybuf[1] = v;
    __syncthreads();
    cx<R> y = ybuf[1];
    bool ok = true;
    for (int c = 0; c < nchunks; ++c) {
      ok = mbar_wait_bounded(&bar[c & 1], phase[c & 1]);
      if (!__syncthreads_and(ok)) {
        ok = false;
        break;
      }
      phase[c & 1] ^= 1u;
      int klo, cnt;
      chunk(c, klo, cnt);
      const cx<R>* st = (c & 1) ? stage1 : stage0;
      for (int r = 0; r < cnt; ++r) {
        const int kp = c * C + r, i = kp & 31, g = kp >> 5;
        if (i == 0 && g > 0) {
          bcur = bnext;
          bnext = at(32 * (g + 1) + lane + W);
        }
        const int sg = g % NW;
        const cx<R>* row = st + (size_t)(pass == 0 ? r : cnt - 1 - r) * ld;
        if (warp == sg && lane == i) {
          const int k = pass == 0 ? kp : nrow - 1 - kp;
          dst[k] = pass == 0 ? y * row[0] : y;
        }
        int t;
        cx<R> base = v;
        if (warp == sg) {
          if (lane == i) {
            t = W;  // the row entering the window
            base = bcur;
          } else {
            t = lane - i + (lane < i ? W : 0);
          }
        } else {
          const int dd = warp - sg;
          t = lane - i + 32 * (dd < 0 ? dd + NW : dd);
        }
        const cx<R> a = t <= bw ? row[t] : zero;
        v = mk<R>(fma(-a.re, y.re, fma(a.im, y.im, base.re)), fma(-a.re, y.im, fma(-a.im, y.re, base.im)));
        const int nslot = i < 31 ? sg : (sg + 1 == NW ? 0 : sg + 1);
        if (warp == nslot && lane == ((i + 1) & 31)) ybuf[kp & 1] = v;
        __syncthreads();
        y = ybuf[kp & 1];
      }
      __syncthreads();
      if (threadIdx.x == 0 && c + 2 < nchunks) issue(c + 2);
    }
    if (!ok) {
      if (threadIdx.x == 0) {
        atomicExch(err, 2);
        for (int c2 = 0; c2 < 2; ++c2) mbar_wait_bounded(&bar[c2], phase[c2]);
      }
      return;
    }
    __syncthreads();
  }
}

std::mutex g_attr_mu;  // launches come from several host threads (one per component)

template <typename R, int SLOTS> void set_smem_attr(size_t bytes) {
  static size_t done = 0;
  std::lock_guard<std::mutex> lock(g_attr_mu);
  if (bytes > done) {
    cudaFuncSetAttribute(k_band_solve_w<R, SLOTS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    done = bytes;
  }
}

template <typename R, int SLOTS> void set_smem_attr_mw(size_t bytes) {
  static size_t done = 0;
  std::lock_guard<std::mutex> lock(g_attr_mu);
  if (bytes > done) {
    cudaFuncSetAttribute(k_band_solve_mw<R, SLOTS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    done = bytes;
  }
}

template <typename R> void set_smem_attr_mwg(size_t bytes) {
  static size_t done = 0;
  std::lock_guard<std::mutex> lock(g_attr_mu);
  if (bytes > done) {
    cudaFuncSetAttribute(k_band_solve_mwg<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    done = bytes;
  }
}

template <typename R, int SLOTS> void set_smem_attr_p2(size_t bytes) {
  static size_t done = 0;
  std::lock_guard<std::mutex> lock(g_attr_mu);
  if (bytes > done) {
    cudaFuncSetAttribute(k_band_solve_p2<R, SLOTS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    done = bytes;
  }
}

constexpr size_t kMaxWindowBytes = 200 * 1024;

template <typename R, int NC> void set_smem_attr_ldlt_dsm(size_t bytes) {
  static size_t done = 0;
  std::lock_guard<std::mutex> lock(g_attr_mu);
  if (bytes > done) {
    cudaFuncSetAttribute(k_band_ldlt_dsm<R, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    done = bytes;
  }
}

// Shared memory of k_band_ldlt_dsm with NC CTAs: its window slots and the pivot copy.
inline size_t dsm_bytes(int bw, int NC, size_t elem) {
  const size_t P = (size_t)bw + 1, nls = (P + NC - 1) / NC;
  return (nls + 1) * P * elem;
}

template <typename R> void set_smem_attr_ldlt(size_t bytes) {
  static size_t done = 0;
  std::lock_guard<std::mutex> lock(g_attr_mu);
  if (bytes > done) {
    cudaFuncSetAttribute(k_band_ldlt_win<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    done = bytes;
  }
}

}  // namespace

BandLayout band_layout(int64_t nrow, int bw) {
  BandLayout L{};
  L.nrow = nrow;
  L.bw = bw;
  L.ld = (bw + 1 + 1) & ~1;
  L.mstride = ((nrow * L.ld + 2 + 31) / 32) * 32;
  return L;
}

template <typename R>
void launch_band_form(const double* Kb, const double* Mb, const cx<double>* lam, cx<R>* F, const BandLayout& L,
                      int nmodes, cudaStream_t s) {
  k_band_form<R><<<dim3(blocks_for(L.nrow * L.ld), nmodes), kBlock, 0, s>>>(Kb, Mb, lam, F, L);
  note_launches(1);
}

template <typename R>
void launch_band_factor(cx<R>* F, cx<R>* G, const BandLayout& L, int nmodes, int* err, cudaStream_t s) {
  const size_t P = (size_t)L.bw + 1, win_bytes = P * P * sizeof(cx<R>);
  if (win_bytes <= kMaxWindowBytes) {
    // window in shared memory: RI row lanes (bw rounded up to a warp multiple) x NP column phases
    const int RI = (L.bw + 31) / 32 * 32, NP = RI >= 256 ? 1 : 256 / RI;
    set_smem_attr_ldlt<R>(win_bytes);
    k_band_ldlt_win<R><<<nmodes, RI * NP, win_bytes, s>>>(F, L, RI, NP, err);
  } else if (L.bw <= 256 && dsm_bytes(L.bw, 4, sizeof(cx<R>)) <= kMaxWindowBytes) {
    // the window over a cluster of 4 CTAs (FP64, half bandwidth 128)
    const int RI = (L.bw + 31) / 32 * 32, NP = 256 / RI;
    const size_t bytes = dsm_bytes(L.bw, 4, sizeof(cx<R>));
    set_smem_attr_ldlt_dsm<R, 4>(bytes);
    k_band_ldlt_dsm<R, 4><<<nmodes * 4, RI * NP, bytes, s>>>(F, L, RI, NP, err);
  } else if (L.bw <= 256 && dsm_bytes(L.bw, 8, sizeof(cx<R>)) <= kMaxWindowBytes) {
    // over 8 CTAs (FP64, half bandwidth 241: the 15^3 grid)
    const int RI = (L.bw + 31) / 32 * 32, NP = 256 / RI;
    const size_t bytes = dsm_bytes(L.bw, 8, sizeof(cx<R>));
    set_smem_attr_ldlt_dsm<R, 8>(bytes);
    k_band_ldlt_dsm<R, 8><<<nmodes * 8, RI * NP, bytes, s>>>(F, L, RI, NP, err);
  } else if (L.bw <= 1024) {
    // global memory, four CTAs per mode (the 31^3 grids: half bandwidth 993)
    const int RI = L.bw <= 256 ? (L.bw + 31) / 32 * 32 : 256, NP = 256 / RI;
    k_band_ldlt_cl<R><<<nmodes * kLdltCluster, RI * NP, (L.bw + 1) * sizeof(cx<R>), s>>>(F, L, RI, NP, err);
  } else {
    k_band_ldlt<R><<<nmodes, 256, (L.bw + 1) * sizeof(cx<R>), s>>>(F, L, err);
  }
  k_band_rows<R><<<dim3(blocks_for(L.nrow * L.ld), nmodes), kBlock, 0, s>>>(F, G, L);
  note_launches(2);
}

int band_chunk_rows(const BandLayout& L, size_t elem) {
  int C = (int)(32768 / (L.ld * elem));
  C = C < 2 ? 2 : (C > 32 ? 32 : C);  // at most one incoming row per lane and chunk
  return C & ~1;
}

template <typename R>
bool launch_band_solve(const cx<R>* F, const cx<R>* G, const BandLayout& L, const cx<R>* b, cx<R>* x,
                       const CocgScal* scal, int nmodes, int64_t vstride, int* err, cudaStream_t s) {
  // power-of-two bandwidths (the 2D grids): fixed-slot kernel with 32-row chunks
  const size_t smem32 = 2 * (size_t)32 * L.ld * sizeof(cx<R>) + 2 * sizeof(uint64_t);
  if (sizeof(R) == 8 && smem32 + 2 * sizeof(cx<R>) <= 160 * 1024 && (L.bw == 64 || L.bw == 128)) {
    // FP64: spread each mode over bw / 32 warps (one FP64 pipe per warp)
    const size_t sm = smem32 + 2 * sizeof(cx<R>);
    if (L.bw == 64) {
      set_smem_attr_mw<R, 2>(sm);
      k_band_solve_mw<R, 2><<<nmodes, 64, sm, s>>>(F, G, L, b, x, scal, vstride, err);
    } else {
      set_smem_attr_mw<R, 4>(sm);
      k_band_solve_mw<R, 4><<<nmodes, 128, sm, s>>>(F, G, L, b, x, scal, vstride, err);
    }
    note_launches(1);
    return true;
  }
  if (smem32 <= 160 * 1024 && (L.bw == 32 || L.bw == 64 || L.bw == 128)) {
    if (L.bw == 32) {
      set_smem_attr_p2<R, 1>(smem32);
      k_band_solve_p2<R, 1><<<nmodes, 32, smem32, s>>>(F, G, L, b, x, scal, vstride, err);
    } else if (L.bw == 64) {
      set_smem_attr_p2<R, 2>(smem32);
      k_band_solve_p2<R, 2><<<nmodes, 32, smem32, s>>>(F, G, L, b, x, scal, vstride, err);
    } else {
      set_smem_attr_p2<R, 4>(smem32);
      k_band_solve_p2<R, 4><<<nmodes, 32, smem32, s>>>(F, G, L, b, x, scal, vstride, err);
    }
    note_launches(1);
    return true;
  }
  const int C = band_chunk_rows(L, sizeof(cx<R>));
  const size_t smem = (2 * (size_t)C * L.ld + 64) * sizeof(cx<R>) + 2 * sizeof(uint64_t);
  if (L.bw <= 32) {
    set_smem_attr<R, 1>(smem);
    k_band_solve_w<R, 1><<<nmodes, 32, smem, s>>>(F, G, L, C, b, x, scal, vstride, err);
  } else if (L.bw <= 64) {
    set_smem_attr<R, 2>(smem);
    k_band_solve_w<R, 2><<<nmodes, 32, smem, s>>>(F, G, L, C, b, x, scal, vstride, err);
  } else if (L.bw <= 128) {
    set_smem_attr<R, 4>(smem);
    k_band_solve_w<R, 4><<<nmodes, 32, smem, s>>>(F, G, L, C, b, x, scal, vstride, err);
  } else if (L.bw <= 256) {
    set_smem_attr<R, 8>(smem);
    k_band_solve_w<R, 8><<<nmodes, 32, smem, s>>>(F, G, L, C, b, x, scal, vstride, err);
  } else if (L.bw <= 1024) {
    // wide 3D bands: one warp per 32-row slot of the padded window
    const int nw = (L.bw + 31) / 32;
    int cw = 32;
    while (cw > 1 && 2 * (size_t)cw * L.ld * sizeof(cx<R>) > 160 * 1024) cw >>= 1;
    const size_t smw = 2 * (size_t)cw * L.ld * sizeof(cx<R>) + 2 * sizeof(cx<R>) + 2 * sizeof(uint64_t);
    set_smem_attr_mwg<R>(smw);
    k_band_solve_mwg<R><<<nmodes, 32 * nw, smw, s>>>(F, G, L, cw, b, x, scal, vstride, err);
  } else {
    return false;
  }
  note_launches(1);
  return true;
}

#define ST_BAND_INST(R)                                                                                              \
  template void launch_band_form<R>(const double*, const double*, const cx<double>*, cx<R>*, const BandLayout&, int, \
                                    cudaStream_t);                                                                   \
  template void launch_band_factor<R>(cx<R>*, cx<R>*, const BandLayout&, int, int*, cudaStream_t);                  \
  template bool launch_band_solve<R>(const cx<R>*, const cx<R>*, const BandLayout&, const cx<R>*, cx<R>*,           \
                                     const CocgScal*, int, int64_t, int*, cudaStream_t);
ST_BAND_INST(double)
ST_BAND_INST(float)
#undef ST_BAND_INST

}  // namespace st
