// Blocked solve of the banded complex-symmetric systems (K + lam_q M) x = b
// for half bandwidths bw <= 128 (see band.h for the recurrences).
//
// With blocks of s = 32 rt >= bw rows, the unit lower factor L couples a block
// only to the one before it, through L_{i,i-1}, which is upper triangular
// (row r of block i reaches back at most bw <= s columns).  Forward:
//   w   = b_i - L_{i,i-1} y_{i-1}      (phase 0, upper-triangular tiles)
//   y_i = X_i w,  X_i = L_ii^{-1}       (phase 1, lower-triangular tiles)
// and z_i = D_i^{-1} y_i is written out.  Backward, blocks in reverse order:
//   w   = z_i - L_{i+1,i}^T x_{i+1}     (phase 0, lower-triangular tiles)
//   x_i = X_i^T w                       (phase 1, upper-triangular tiles)
// Per block both phases together apply s^2 complex multiply-adds, the same
// count as row-by-row substitution, but the chain of dependent steps is nb
// blocks long instead of nrow rows.
//
// Tile stream (per mode): pass (forward, backward) -> block step -> phase ->
// tile t, each tile 32 x 32 stored column-major (entry (row l, column k) at
// k * 32 + l, so a warp with one lane per row reads 32 consecutive entries
// for each k).  The tiles of a phase are its full off-diagonal tiles, then its
// diagonal tiles; steps with no neighbouring block carry zero tiles.
#include <algorithm>
#include <mutex>

#include <cooperative_groups.h>

#include "band.h"
#include "kernels.h"
#include "ptx.cuh"

namespace st {

namespace cg = cooperative_groups;

namespace {

constexpr int kT = 32;              // tile edge
constexpr int kTE = kT * kT;        // tile elements
// tiles in flight per CTA: 8 (FP32) or 4 (FP64) slots of 8 KB / 16 KB, so that
// two or three CTAs fit on one SM and every mode's cluster is resident at once
template <typename R> __host__ __device__ constexpr int ring_slots() { return sizeof(R) == 8 ? 4 : 8; }

__host__ __device__ constexpr int blk_nfull(int rt) { return rt * (rt - 1) / 2; }
__host__ __device__ constexpr int blk_ntiles(int rt) { return rt * (rt + 1) / 2; }
__host__ __device__ constexpr int blk_ntasks(int rt) { return blk_nfull(rt) + (rt + 1) / 2; }

// Tile t of a phase -> (row tile R, column tile C).  Upper: R <= C, lower:
// R >= C; off-diagonal tiles first (R ascending, then C), then diagonal R.
__host__ __device__ inline void blk_tile_rc(bool upper, int rt, int t, int& R, int& C) {
  const int nf = blk_nfull(rt);
  R = C = t - nf;
  if (t >= nf) return;
  int k = 0;
  for (int r = 0; r < rt; ++r)
    for (int c = 0; c < rt; ++c)
      if (upper ? (r < c) : (r > c)) {
        if (k == t) {
          R = r;
          C = c;
          return;
        }
        ++k;
      }
}

__host__ __device__ inline int blk_tile_index(bool upper, int rt, int R, int C) {
  if (R == C) return blk_nfull(rt) + R;
  int k = 0;
  for (int r = 0; r < rt; ++r)
    for (int c = 0; c < rt; ++c)
      if (upper ? (r < c) : (r > c)) {
        if (r == R && c == C) return k;
        ++k;
      }
  return -1;
}

// Stream position of tile t of phase ph at block step j of pass p.
__host__ __device__ inline int64_t blk_pos(int nb, int tp, int p, int j, int ph, int t) {
  return ((int64_t)p * 2 * nb + 2 * (int64_t)j + ph) * tp + t;
}

// ------------------------------------------------------------ preparation
// Phase-0 tiles (the coupling blocks of L), one thread per tile entry.
template <typename R>
__global__ void k_blk_pack_coupling(const cx<R>* __restrict__ F, BandLayout L, BlkLayout B, cx<R>* __restrict__ S) {
  const int tp = blk_ntiles(B.rt), p = blockIdx.y, q = blockIdx.z;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)B.nb * tp * kTE) return;
  const int j = (int)(e / ((int64_t)tp * kTE));
  const int t = (int)((e / kTE) % tp);
  const int k = (int)((e % kTE) / kT), l = (int)(e % kT);
  const bool upper = p == 0;
  int tr, tc;
  blk_tile_rc(upper, B.rt, t, tr, tc);
  int64_t row, col;
  bool exists;
  if (p == 0) {  // L_{i,i-1}: rows of block i, columns of block i-1
    const int i = j;
    exists = i >= 1;
    row = (int64_t)i * B.s + tr * kT + l;
    col = (int64_t)(i - 1) * B.s + tc * kT + k;
  } else {  // L_{i+1,i}^T: entry (a, b') = L(row of block i+1, column of block i)
    const int i = B.nb - 1 - j;
    exists = i + 1 < B.nb;
    row = (int64_t)(i + 1) * B.s + tc * kT + k;
    col = (int64_t)i * B.s + tr * kT + l;
  }
  cx<R> v = mk<R>(0, 0);
  const int64_t d = row - col;
  if (exists && row < L.nrow && d >= 1 && d <= L.bw) v = F[(int64_t)q * L.mstride + col * L.ld + d];
  S[(int64_t)q * B.tstride + blk_pos(B.nb, tp, p, j, 0, t) * kTE + k * kT + l] = v;
}

// Phase-1 tiles: X_i = L_ii^{-1} by columns (thread c owns column c and forms
// X(a, c) = -sum_{b=c}^{a-1} L(a, b) X(b, c) in FP64), then writes it into the
// lower tiles of the forward pass and, transposed, the upper tiles of the
// backward pass.  Rows past the end of the grid are identity rows.
template <typename R>
__global__ void __launch_bounds__(128) k_blk_inverse(const cx<R>* __restrict__ F, BandLayout L, BlkLayout B,
                                                      cx<R>* __restrict__ S) {
  const int i = blockIdx.x, q = blockIdx.y, c = threadIdx.x;
  const int s = B.s, rt = B.rt, tp = blk_ntiles(rt);
  if (c >= s) return;
  const int64_t r0 = (int64_t)i * s;
  const cx<R>* Fq = F + (int64_t)q * L.mstride;
  cx<double> col[128];
  for (int a = 0; a < s; ++a) col[a] = mk<double>(a == c ? 1.0 : 0.0, 0.0);
  for (int a = c + 1; a < s; ++a) {
    if (r0 + a >= L.nrow) break;  // identity rows beyond the grid
    double re = 0.0, im = 0.0;
    const int b0 = max(c, a - L.bw);
    for (int b = b0; b < a; ++b) {
      const cx<R> lv = Fq[(r0 + b) * L.ld + (a - b)];
      const cx<double> xv = col[b];
      re = fma(-(double)lv.re, xv.re, fma((double)lv.im, xv.im, re));
      im = fma(-(double)lv.re, xv.im, fma(-(double)lv.im, xv.re, im));
    }
    col[a] = mk<double>(re, im);
  }
  cx<R>* Sq = S + (int64_t)q * B.tstride;
  // forward, lower tiles (R >= C): T(k, l) = X(R*32 + l, C*32 + k), this thread = column C*32 + k
  {
    const int tc = c / kT, k = c % kT;
    for (int tr = tc; tr < rt; ++tr) {
      const int t = blk_tile_index(false, rt, tr, tc);
      cx<R>* T = Sq + blk_pos(B.nb, tp, 0, i, 1, t) * kTE + k * kT;
      for (int l = 0; l < kT; ++l) {
        const cx<double> v = col[tr * kT + l];
        T[l] = mk<R>((R)v.re, (R)v.im);
      }
    }
  }
  // backward, upper tiles (R <= C) of X^T: T(k, l) = X(C*32 + k, R*32 + l), this thread = column R*32 + l
  {
    const int tr = c / kT, l = c % kT;
    const int j = B.nb - 1 - i;
    for (int tc = tr; tc < rt; ++tc) {
      const int t = blk_tile_index(true, rt, tr, tc);
      cx<R>* T = Sq + blk_pos(B.nb, tp, 1, j, 1, t) * kTE + l;
      for (int k = 0; k < kT; ++k) {
        const cx<double> v = col[tc * kT + k];
        T[k * kT] = mk<R>((R)v.re, (R)v.im);
      }
    }
  }
}

// ------------------------------------------------------------------ solve
// Partial products of one task, split over the CTA's kW warps by column
// ranges.  A full tile: warp w takes columns k in [8w, 8w + 8) of every row.
template <typename R>
__device__ __forceinline__ cx<R> blk_full_part(const cx<R>* __restrict__ T, const cx<R>* v, int lane, int w) {
  R r0 = R(0), i0 = R(0), r1 = R(0), i1 = R(0);
#pragma unroll
  for (int k = 8 * w; k < 8 * w + 8; k += 2) {
    const cx<R> a = T[k * kT + lane], x = v[k];
    const cx<R> a1 = T[(k + 1) * kT + lane], x1 = v[k + 1];
    r0 = fma(a.re, x.re, fma(-a.im, x.im, r0));
    i0 = fma(a.re, x.im, fma(a.im, x.re, i0));
    r1 = fma(a1.re, x1.re, fma(-a1.im, x1.im, r1));
    i1 = fma(a1.re, x1.im, fma(a1.im, x1.re, i1));
  }
  return mk<R>(r0 + r1, i0 + i1);
}

// Two diagonal tiles A, B of one triangle type: lane l takes row l of A, then
// row 31 - l of B, 33 entries in all for every lane (upper tiles hold columns
// k >= row, lower tiles k <= row); warp w takes entries j in [9w, 9w + 9) of
// that sequence.  Without B (odd tile count) the lanes only take their row of A.
template <typename R, bool UPPER>
__device__ __forceinline__ void blk_diag_part(const cx<R>* __restrict__ A, const cx<R>* vA, const cx<R>* __restrict__ B,
                                              const cx<R>* vB, bool hasB, int lane, int w, cx<R>& outA,
                                              cx<R>& outB) {
  const int nA = UPPER ? kT - lane : lane + 1;  // entries of row l of A
  const int kA0 = UPPER ? lane : 0;
  const int rowB = kT - 1 - lane;
  const int kB0 = UPPER ? rowB : 0;
  const int j0 = 9 * w, j1 = min(kT + 1, j0 + 9);
  R ar = R(0), ai = R(0), sr = R(0), si = R(0);
  for (int j = j0; j < j1; ++j) {
    const bool inA = j < nA;
    if (j == nA) {  // row of A done: keep its sum, continue with row of B
      sr = ar;
      si = ai;
      ar = R(0);
      ai = R(0);
    }
    if (!inA && !hasB) continue;
    const int k = inA ? kA0 + j : kB0 + (j - nA);
    const cx<R> a = inA ? A[k * kT + lane] : B[k * kT + rowB];
    const cx<R> x = inA ? vA[k] : vB[k];
    ar = fma(a.re, x.re, fma(-a.im, x.im, ar));
    ai = fma(a.re, x.im, fma(a.im, x.re, ai));
  }
  if (nA >= j1) {  // the whole range lay in the row of A
    outA = mk<R>(ar, ai);
    outB = mk<R>(0, 0);
  } else {
    outA = mk<R>(sr, si);
    outB = mk<R>(ar, ai);
  }
}

// Shared-memory-to-shared-memory bulk copy to a CTA of the cluster,
// completing on that CTA's mbarrier (addresses of the peer from mapa).
__device__ __forceinline__ unsigned cluster_addr(const void* p, int rank) {
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_addr(p)), "r"(rank));
  return r;
}
__device__ __forceinline__ void bulk_s2peer(unsigned dst, const void* src, unsigned bytes, unsigned bar) {
  asm volatile("cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "r"(smem_addr(src)), "r"(bytes), "r"(bar)
               : "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// One cluster of blk_ntasks(RT) CTAs per mode; CTA r owns task r of every
// phase (full tile r, or a pair of diagonal tiles) and streams only that
// task's tiles through its own ring of NT shared-memory slots (one bulk copy
// per tile, completing on the slot's mbarrier; slots are refilled once the
// phase has consumed them).  Per phase the CTA's kW warps form the task's
// partial row sums, and one bulk copy per peer carries them into every CTA
// of the cluster, completing on the receiver's phase mbarrier (armed by the
// receiver for the phase's full set of partials).  Every CTA then forms all
// rows of the phase result.  Partials are double-buffered by phase parity: a
// CTA reuses a buffer two phases later, after every peer has sent it the
// next phase's partials, which a peer only does once it has read the buffer.
// Rank 0 writes the results to memory.  After a wait that ran out, a CTA
// stops copying and waiting but keeps the loop (and its cluster barriers) in
// step with its peers, which then run out once and do the same.
constexpr int kW = 4;  // warps per CTA (one per SM sub-partition)
template <typename R, int RT>
__global__ void __cluster_dims__(blk_ntasks(RT), 1, 1) __launch_bounds__(32 * kW)
    k_band_solve_blk(const cx<R>* __restrict__ F, BandLayout L, BlkLayout B, const cx<R>* __restrict__ S,
                     const cx<R>* __restrict__ b, cx<R>* x, const CocgScal* __restrict__ scal, int64_t vstride,
                     int* err) {
  constexpr int SB = kT * RT, TP = blk_ntiles(RT), NF = blk_nfull(RT), CL = blk_ntasks(RT);
  constexpr int NT = ring_slots<R>(), LNT = NT == 8 ? 3 : 2;
  extern __shared__ __align__(128) unsigned char smem[];
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int q = blockIdx.x / CL;
  if (scal != nullptr && !scal[q].active) return;  // the whole cluster returns
  cx<R>* ring = reinterpret_cast<cx<R>*>(smem);
  cx<R>* wpart = ring + (size_t)NT * kTE;  // kW x 64
  cx<R>* spart = wpart + kW * 2 * kT;      // 2 x 64: this CTA's task partial
  cx<R>* cpart = spart + 2 * 2 * kT;       // 2 x TP x 32: every tile's partial
  cx<R>* vsrc = cpart + 2 * TP * kT;       // y_{i-1} (forward) / x_{i+1} (backward)
  cx<R>* vw = vsrc + SB;                   // w
  uint64_t* bar = reinterpret_cast<uint64_t*>(vw + SB);  // NT tile slots
  uint64_t* rbar = bar + NT;                             // 2 partial buffers
  __shared__ int rowtile[2][TP];                         // [upper][t] -> row tile R
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid < 2 * TP) {
    int tr, tc;
    blk_tile_rc(tid < TP, RT, tid % TP, tr, tc);
    rowtile[tid < TP ? 1 : 0][tid % TP] = tr;
  }
  if (tid == 0) {
    for (int k = 0; k < NT; ++k) mbar_init(&bar[k], 1);
    mbar_init(&rbar[0], 1);
    mbar_init(&rbar[1], 1);
    mbar_fence_init();
  }
  if (tid < SB) vsrc[tid] = mk<R>(0, 0);
  // this CTA's task: tiles t0 (and t1 = t0 + 1) of every phase
  const bool full = rank < NF;
  const int pidx = rank - NF;
  const int t0 = full ? rank : NF + 2 * pidx;
  const bool has1 = !full && 2 * pidx + 1 < RT;
  const int t1 = t0 + 1;
  const int ntl = has1 ? 2 : 1;
  const int C0 = full ? 0 : 2 * pidx;  // source tile of a diagonal pair
  int tcU = C0, tcL = C0;              // source tile of a full tile in upper / lower phases
  if (full) {
    int tr;
    blk_tile_rc(true, RT, t0, tr, tcU);
    blk_tile_rc(false, RT, t0, tr, tcL);
  }
  __syncthreads();
  cluster.sync();  // every CTA's barriers are initialised before the first copy between CTAs
  const int nb = B.nb, nrow = (int)L.nrow, ld = L.ld;
  const int H = 4 * nb * ntl;  // tiles this CTA consumes
  const cx<R>* Sq = S + (int64_t)q * B.tstride;
  const cx<R>* Fq = F + (int64_t)q * L.mstride;
  const cx<R>* bq = b + (int64_t)q * vstride;
  cx<R>* xq = x + (int64_t)q * vstride;
  constexpr unsigned kTileBytes = kTE * sizeof(cx<R>);
  constexpr unsigned kPhaseBytes = TP * kT * sizeof(cx<R>);
  const unsigned sendBytes = (unsigned)(ntl * kT * sizeof(cx<R>));
  int issued = 0;
  bool failed = false;
  auto issue_upto = [&](int lim) {
    if (lim > H) lim = H;
    for (; issued < lim; ++issued) {
      const int slot = issued & (NT - 1);
      const int Pi = ntl == 2 ? issued >> 1 : issued;
      const int t = (issued & (ntl - 1)) == 0 ? t0 : t1;
      mbar_expect_tx(&bar[slot], kTileBytes);
      bulk_g2s(ring + (size_t)slot * kTE, Sq + ((int64_t)Pi * TP + t) * kTE, kTileBytes, &bar[slot]);
    }
  };
  if (tid == 0) issue_upto(NT);
  int P = 0;  // phase counter
  const cx<R> zero = mk<R>(0, 0);
  for (int pass = 0; pass < 2; ++pass) {
    auto rhs_of = [&](int i) -> cx<R> {
      const int row = i * SB + tid;
      if (tid >= SB || row >= nrow) return zero;
      return pass == 0 ? bq[row] : xq[row];  // z from the forward pass (cluster barrier in between)
    };
    auto dinv_of = [&](int i) -> cx<R> {
      const int row = i * SB + tid;
      if (pass != 0 || tid >= SB || row >= nrow) return zero;
      return Fq[(int64_t)row * ld];
    };
    int i = pass == 0 ? 0 : nb - 1;
    cx<R> rhs = rhs_of(i), dinv = dinv_of(i);
    for (int j = 0; j < nb; ++j) {
      const int inext = pass == 0 ? i + 1 : i - 1;
      const bool more = j + 1 < nb;
      const cx<R> rhs_n = more ? rhs_of(inext) : zero;
      const cx<R> dinv_n = more ? dinv_of(inext) : zero;
      for (int ph = 0; ph < 2; ++ph, ++P) {
        const bool upper = (pass == 0) == (ph == 0);
        const cx<R>* src = ph == 0 ? vsrc : vw;
        const int buf = (int)(P & 1);
        if (tid == 0 && !failed) mbar_expect_tx(&rbar[buf], kPhaseBytes);  // this phase's partials
        // this CTA's task
        const int h0 = P * ntl;
        const int s0 = h0 & (NT - 1), s1 = (h0 + 1) & (NT - 1);
        bool ok = true;
        if (!failed) {
          if (!mbar_wait_bounded(&bar[s0], (unsigned)((h0 >> LNT) & 1))) ok = false;
          if (has1 && !mbar_wait_bounded(&bar[s1], (unsigned)(((h0 + 1) >> LNT) & 1))) ok = false;
        }
        const cx<R>* TA = ring + (size_t)s0 * kTE;
        if (full) {
          wpart[warp * 2 * kT + lane] = blk_full_part<R>(TA, src + (upper ? tcU : tcL) * kT, lane, warp);
        } else if constexpr (sizeof(R) == 8) {
          // FP64 pipe bound: the pair costs 33 entries a lane instead of 64
          const cx<R>* TB = has1 ? ring + (size_t)s1 * kTE : TA;
          const cx<R>* vA = src + C0 * kT;
          const cx<R>* vB = has1 ? src + (C0 + 1) * kT : vA;
          cx<R> oA, oB;
          if (upper) blk_diag_part<R, true>(TA, vA, TB, vB, has1, lane, warp, oA, oB);
          else blk_diag_part<R, false>(TA, vA, TB, vB, has1, lane, warp, oA, oB);
          wpart[warp * 2 * kT + lane] = oA;
          wpart[warp * 2 * kT + kT + (kT - 1 - lane)] = oB;
        } else {
          // FP32: the diagonal tiles as full tiles (their other triangle is stored as zeros)
          wpart[warp * 2 * kT + lane] = blk_full_part<R>(TA, src + C0 * kT, lane, warp);
          if (has1)
            wpart[warp * 2 * kT + kT + lane] =
                blk_full_part<R>(ring + (size_t)s1 * kTE, src + (C0 + 1) * kT, lane, warp);
        }
        if (!__syncthreads_and(ok) && !failed) {
          failed = true;
          if (tid == 0) atomicExch(err, 2);
        }
        if (tid == 0 && !failed) issue_upto((P + 1) * ntl + NT);  // the task's slots of this phase are free again
        if (tid < ntl * kT) {
          R ar = R(0), ai = R(0);
#pragma unroll
          for (int w = 0; w < kW; ++w) {
            const cx<R> v = wpart[w * 2 * kT + tid];
            ar += v.re;
            ai += v.im;
          }
          spart[buf * 2 * kT + tid] = mk<R>(ar, ai);
          fence_proxy_async_smem();  // visible to the bulk copies below
        }
        __syncthreads();
        if (tid < CL && !failed) {
          cx<R>* dst = cpart + ((size_t)buf * TP + t0) * kT;
          bulk_s2peer(cluster_addr(dst, tid), spart + buf * 2 * kT, sendBytes, cluster_addr(&rbar[buf], tid));
        }
        bool got = true;
        if (!failed) got = mbar_wait_bounded(&rbar[buf], (unsigned)((P >> 1) & 1));
        if (tid < SB) {
          const int Rr = tid / kT, l = tid % kT;
          R ar = R(0), ai = R(0);
#pragma unroll
          for (int t = 0; t < TP; ++t)
            if (rowtile[upper][t] == Rr) {
              const cx<R> v = cpart[((size_t)buf * TP + t) * kT + l];
              ar += v.re;
              ai += v.im;
            }
          if (ph == 0) {
            vw[tid] = mk<R>(rhs.re - ar, rhs.im - ai);
          } else {
            const int row = i * SB + tid;
            const bool last = pass == 0 && j + 1 == nb;  // the backward pass starts from zero
            vsrc[tid] = last ? zero : mk<R>(ar, ai);
            if (rank == 0 && row < nrow) xq[row] = pass == 0 ? mk<R>(ar, ai) * dinv : mk<R>(ar, ai);
          }
        }
        if (!__syncthreads_and(got) && !failed) {
          failed = true;
          if (tid == 0) atomicExch(err, 2);
        }
      }
      rhs = rhs_n;
      dinv = dinv_n;
      i = inext;
    }
    // z (written by rank 0) is read by every CTA in the backward pass
    if (pass == 0) cluster.sync();
  }
  if (failed && tid == 0) {
    // let this CTA's tile copies in flight land before its shared memory is released
    for (int h = issued - NT > 0 ? issued - NT : 0; h < issued; ++h)
      mbar_wait_bounded(&bar[h & (NT - 1)], (unsigned)((h >> LNT) & 1));
  }
  cluster.sync();  // no CTA leaves while another may still copy into its shared memory
}

std::mutex g_blk_attr_mu;

template <typename R, int RT> void set_blk_smem(size_t bytes) {
  static size_t done = 0;
  std::lock_guard<std::mutex> lock(g_blk_attr_mu);
  if (bytes > done) {
    cudaFuncSetAttribute(k_band_solve_blk<R, RT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    done = bytes;
  }
}

inline unsigned nblocks(int64_t n, int per) { return (unsigned)((n + per - 1) / per); }

}  // namespace

BlkLayout blk_layout(const BandLayout& L) {
  BlkLayout B{};
  if (L.bw < 1 || L.bw > 128 || L.nrow < 1) return B;
  B.rt = (L.bw + kT - 1) / kT;
  B.s = kT * B.rt;
  B.nb = (int)((L.nrow + B.s - 1) / B.s);
  B.tstride = 4 * (int64_t)B.nb * blk_ntiles(B.rt) * kTE;
  return B;
}

template <typename R>
void launch_band_blk_prepare(const cx<R>* F, const BandLayout& L, const BlkLayout& B, cx<R>* S, int nmodes,
                             cudaStream_t s) {
  const int64_t n = (int64_t)B.nb * blk_ntiles(B.rt) * kTE;
  k_blk_pack_coupling<R><<<dim3(nblocks(n, 256), 2, nmodes), 256, 0, s>>>(F, L, B, S);
  k_blk_inverse<R><<<dim3(B.nb, nmodes), 128, 0, s>>>(F, L, B, S);
  note_launches(2);
}

template <typename R, int RT>
void blk_launch(const cx<R>* F, const BandLayout& L, const BlkLayout& B, const cx<R>* S, const cx<R>* b, cx<R>* x,
                const CocgScal* scal, int nmodes, int64_t vstride, int* err, cudaStream_t s) {
  constexpr int TP = blk_ntiles(RT), CL = blk_ntasks(RT);
  const int NT = ring_slots<R>();
  const size_t smem = (size_t)NT * kTE * sizeof(cx<R>) +
                      (size_t)(kW * 2 * kT + 2 * 2 * kT + 2 * TP * kT + 2 * kT * RT) * sizeof(cx<R>) +
                      (size_t)(NT + 2) * sizeof(uint64_t);
  set_blk_smem<R, RT>(smem);
  k_band_solve_blk<R, RT><<<nmodes * CL, 32 * kW, smem, s>>>(F, L, B, S, b, x, scal, vstride, err);
}

template <typename R>
void launch_band_solve_blk(const cx<R>* F, const BandLayout& L, const BlkLayout& B, const cx<R>* S, const cx<R>* b,
                           cx<R>* x, const CocgScal* scal, int nmodes, int64_t vstride, int* err, cudaStream_t s) {
  switch (B.rt) {
    case 1: blk_launch<R, 1>(F, L, B, S, b, x, scal, nmodes, vstride, err, s); break;
    case 2: blk_launch<R, 2>(F, L, B, S, b, x, scal, nmodes, vstride, err, s); break;
    case 3: blk_launch<R, 3>(F, L, B, S, b, x, scal, nmodes, vstride, err, s); break;
    default: blk_launch<R, 4>(F, L, B, S, b, x, scal, nmodes, vstride, err, s); break;
  }
  note_launches(1);
}

#define ST_BLK_INST(R)                                                                                            \
  template void launch_band_blk_prepare<R>(const cx<R>*, const BandLayout&, const BlkLayout&, cx<R>*, int,        \
                                           cudaStream_t);                                                         \
  template void launch_band_solve_blk<R>(const cx<R>*, const BandLayout&, const BlkLayout&, const cx<R>*,         \
                                         const cx<R>*, cx<R>*, const CocgScal*, int, int64_t, int*, cudaStream_t);
ST_BLK_INST(double)
ST_BLK_INST(float)
#undef ST_BLK_INST

}  // namespace st
