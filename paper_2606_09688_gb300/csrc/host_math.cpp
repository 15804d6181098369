// Host-side FP64 setup math.  See host_math.h for the definitions.
#include "host_math.h"

#include "bspline.h"

#include <algorithm>
#include <cmath>
#include <limits>
#include <cstring>

namespace st {

void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  // Roots of the Legendre polynomial P_n by Newton's method from the
  // asymptotic guesses cos(pi (i + 3/4) / (n + 1/2)); P_n and P_n' from the
  // three-term recurrence (k+1) P_{k+1} = (2k+1) z P_k - k P_{k-1}.
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  const double pi = std::acos(-1.0);
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = std::cos(pi * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 1; k < n; ++k) {
        double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = -z;
    x[n - 1 - i] = z;
    w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

int bspline_span(int N, double T, double t) {
  int k = (int)std::floor(t / (T / N));
  return std::min(std::max(k, 0), N - 1);
}

void bspline_local(int N, double T, int k, double t, double val[3], double d1[3], double d2[3]) {
  bs_local(N, T, k, t, val, d1, d2);
}

void build_time_level(int jt, double T, TimeLevel& tl) {
  tl.jt = jt;
  tl.N = 1 << jt;
  tl.nt = tl.N + 1;
  tl.T = T;
  const int N = tl.N, nt = tl.nt;
  const double h = T / N;
  std::vector<double> gx, gw;
  gauss_legendre(8, gx, gw);
  const int nq = 8 * N;
  tl.A.assign((size_t)nt * nt, 0.0);
  tl.B.assign((size_t)nt * nt, 0.0);
  tl.qt.assign(nq, 0.0);
  tl.qw.assign(nq, 0.0);
  tl.Q.assign((size_t)nt * nq, 0.0);
  tl.g1.assign(nt, 0.0);
  tl.d0.assign(nt, 0.0);
  for (int k = 0; k < N; ++k) {
    for (int q = 0; q < 8; ++q) {
      const double t = k * h + 0.5 * (gx[q] + 1.0) * h;
      const double wq = 0.5 * h * gw[q];
      const double we = wq * std::exp(-t / T);
      const int iq = k * 8 + q;
      tl.qt[iq] = t;
      tl.qw[iq] = wq;
      double v[3], d1[3], d2[3];
      bspline_local(N, T, k, t, v, d1, d2);
      for (int a = 0; a < 3; ++a) {
        const int i = k + a - 1;  // psi index (B_0 removed)
        if (i < 0) continue;
        tl.Q[(size_t)i * nq + iq] = we * d1[a];
        tl.g1[i] += we * d1[a];
        for (int b = 0; b < 3; ++b) {
          const int j = k + b - 1;
          if (j < 0) continue;
          tl.A[(size_t)i * nt + j] += we * d1[a] * d2[b];
          tl.B[(size_t)i * nt + j] += we * d1[a] * v[b];
        }
      }
    }
  }
  double v[3], d1[3], d2[3];
  bspline_local(N, T, 0, 0.0, v, d1, d2);
  for (int a = 1; a < 3; ++a) tl.d0[a - 1] = d1[a];
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) tl.A[(size_t)i * nt + j] += tl.d0[i] * tl.d0[j];
}

namespace {
// Knot i of the open uniform vector of degree p on (0,T) with N intervals.
double knot_p(int N, double T, int p, int i) {
  if (i <= p) return 0.0;
  if (i >= N + p) return T;
  return (double)(i - p) * (T / N);
}
// Derivative of the degree-q functions of the span from the degree-(q-1)
// quantities `lower` of the same span (B'_{i,q} = q/(t_{i+q}-t_i) B_{i,q-1}
// - q/(t_{i+q+1}-t_{i+1}) B_{i+1,q-1}); entry r is function s - q + r.
double dq(int N, double T, int p, int s, int q, int r, const double* lower) {
  const int i = s - q + r;
  double out = 0.0;
  if (r >= 1) {
    const double d = knot_p(N, T, p, i + q) - knot_p(N, T, p, i);
    if (d > 0.0) out += q / d * lower[r - 1];
  }
  if (r <= q - 1) {
    const double d = knot_p(N, T, p, i + q + 1) - knot_p(N, T, p, i + 1);
    if (d > 0.0) out -= q / d * lower[r];
  }
  return out;
}
}  // namespace

void bspline_local_p(int N, double T, int p, int k, double t, double* val, double* d1, double* d2) {
  const int s = k + p;  // knot span: t_s <= t < t_{s+1}
  // Bq[q][r] = B_{s-q+r, q}(t), the q + 1 functions of degree q non-zero on the span
  double Bq[5][5] = {};
  Bq[0][0] = 1.0;
  for (int q = 1; q <= p; ++q)
    for (int r = 0; r <= q; ++r) {
      const int i = s - q + r;
      double v = 0.0;
      if (r >= 1) {
        const double d = knot_p(N, T, p, i + q) - knot_p(N, T, p, i);
        if (d > 0.0) v += (t - knot_p(N, T, p, i)) / d * Bq[q - 1][r - 1];
      }
      if (r <= q - 1) {
        const double d = knot_p(N, T, p, i + q + 1) - knot_p(N, T, p, i + 1);
        if (d > 0.0) v += (knot_p(N, T, p, i + q + 1) - t) / d * Bq[q - 1][r];
      }
      Bq[q][r] = v;
    }
  double dlow[5] = {};
  for (int r = 0; r <= p - 1; ++r) dlow[r] = dq(N, T, p, s, p - 1, r, Bq[p - 2]);  // B'_{., p-1}
  for (int a = 0; a <= p; ++a) {
    val[a] = Bq[p][a];
    d1[a] = dq(N, T, p, s, p, a, Bq[p - 1]);
    d2[a] = dq(N, T, p, s, p, a, dlow);
  }
}

void build_time_level_p(int jt, double T, int p, TimeLevel& tl) {
  tl.jt = jt;
  tl.N = 1 << jt;
  tl.nt = tl.N + p - 1;
  tl.T = T;
  const int N = tl.N, nt = tl.nt;
  const double h = T / N;
  std::vector<double> gx, gw;
  gauss_legendre(8, gx, gw);
  const int nq = 8 * N;
  tl.A.assign((size_t)nt * nt, 0.0);
  tl.B.assign((size_t)nt * nt, 0.0);
  tl.qt.assign(nq, 0.0);
  tl.qw.assign(nq, 0.0);
  tl.Q.assign((size_t)nt * nq, 0.0);
  tl.g1.assign(nt, 0.0);
  tl.d0.assign(nt, 0.0);
  double v[5], d1[5], d2[5];
  for (int k = 0; k < N; ++k) {
    for (int q = 0; q < 8; ++q) {
      const double t = k * h + 0.5 * (gx[q] + 1.0) * h;
      const double wq = 0.5 * h * gw[q];
      const double we = wq * std::exp(-t / T);
      const int iq = k * 8 + q;
      tl.qt[iq] = t;
      tl.qw[iq] = wq;
      bspline_local_p(N, T, p, k, t, v, d1, d2);
      for (int a = 0; a <= p; ++a) {
        const int i = k + a - 1;  // psi index (B_0 removed)
        if (i < 0) continue;
        tl.Q[(size_t)i * nq + iq] = we * d1[a];
        tl.g1[i] += we * d1[a];
        for (int b = 0; b <= p; ++b) {
          const int j = k + b - 1;
          if (j < 0) continue;
          tl.A[(size_t)i * nt + j] += we * d1[a] * d2[b];
          tl.B[(size_t)i * nt + j] += we * d1[a] * v[b];
        }
      }
    }
  }
  // the penalty psi_j'(0) psi_i'(0) of A
  bspline_local_p(N, T, p, 0, 0.0, v, d1, d2);
  for (int a = 1; a <= p; ++a) tl.d0[a - 1] = d1[a];
  for (int i = 0; i < p; ++i)
    for (int j = 0; j < p; ++j) tl.A[(size_t)i * nt + j] += tl.d0[i] * tl.d0[j];
}

bool lu_solve_real(int n, std::vector<double> A, std::vector<double>& Bm, int nrhs) {
  std::vector<int> piv(n);
  for (int k = 0; k < n; ++k) {
    int p = k;
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(A[(size_t)i * n + k]) > std::fabs(A[(size_t)p * n + k])) p = i;
    if (A[(size_t)p * n + k] == 0.0) return false;
    if (p != k) {
      for (int j = 0; j < n; ++j) std::swap(A[(size_t)k * n + j], A[(size_t)p * n + j]);
      for (int j = 0; j < nrhs; ++j) std::swap(Bm[(size_t)k * nrhs + j], Bm[(size_t)p * nrhs + j]);
    }
    for (int i = k + 1; i < n; ++i) {
      const double l = A[(size_t)i * n + k] / A[(size_t)k * n + k];
      if (l == 0.0) continue;
      for (int j = k + 1; j < n; ++j) A[(size_t)i * n + j] -= l * A[(size_t)k * n + j];
      for (int j = 0; j < nrhs; ++j) Bm[(size_t)i * nrhs + j] -= l * Bm[(size_t)k * nrhs + j];
    }
  }
  for (int k = n - 1; k >= 0; --k)
    for (int j = 0; j < nrhs; ++j) {
      double s = Bm[(size_t)k * nrhs + j];
      for (int i = k + 1; i < n; ++i) s -= A[(size_t)k * n + i] * Bm[(size_t)i * nrhs + j];
      Bm[(size_t)k * nrhs + j] = s / A[(size_t)k * n + k];
    }
  return true;
}

bool lu_inverse_cplx(int n, std::vector<cplx> A, std::vector<cplx>& Ainv) {
  Ainv.assign((size_t)n * n, cplx(0.0));
  for (int i = 0; i < n; ++i) Ainv[(size_t)i * n + i] = 1.0;
  for (int k = 0; k < n; ++k) {
    int p = k;
    for (int i = k + 1; i < n; ++i)
      if (std::abs(A[(size_t)i * n + k]) > std::abs(A[(size_t)p * n + k])) p = i;
    if (std::abs(A[(size_t)p * n + k]) == 0.0) return false;
    if (p != k)
      for (int j = 0; j < n; ++j) {
        std::swap(A[(size_t)k * n + j], A[(size_t)p * n + j]);
        std::swap(Ainv[(size_t)k * n + j], Ainv[(size_t)p * n + j]);
      }
    for (int i = k + 1; i < n; ++i) {
      const cplx l = A[(size_t)i * n + k] / A[(size_t)k * n + k];
      if (l == cplx(0.0)) continue;
      for (int j = k + 1; j < n; ++j) A[(size_t)i * n + j] -= l * A[(size_t)k * n + j];
      for (int j = 0; j < n; ++j) Ainv[(size_t)i * n + j] -= l * Ainv[(size_t)k * n + j];
    }
  }
  for (int k = n - 1; k >= 0; --k)
    for (int j = 0; j < n; ++j) {
      cplx s = Ainv[(size_t)k * n + j];
      for (int i = k + 1; i < n; ++i) s -= A[(size_t)k * n + i] * Ainv[(size_t)i * n + j];
      Ainv[(size_t)k * n + j] = s / A[(size_t)k * n + k];
    }
  return true;
}

// Givens rotation [c s; -conj(s) c] with real c that maps (a, b) to (r, 0).
static void givens(cplx a, cplx b, double& c, cplx& s) {
  const double aa = std::abs(a), bb = std::abs(b);
  if (bb == 0.0) {
    c = 1.0;
    s = 0.0;
    return;
  }
  if (aa == 0.0) {
    c = 0.0;
    s = std::conj(b) / bb;
    return;
  }
  const double nrm = std::hypot(aa, bb);
  c = aa / nrm;
  s = (a / aa) * std::conj(b) / nrm;
}

bool complex_schur(int n, std::vector<cplx>& H, std::vector<cplx>& Z) {
  // Explicitly shifted QR iteration on an upper Hessenberg matrix, with
  // Wilkinson shifts, deflation on negligible subdiagonal entries and
  // exceptional shifts after 10 and 20 stagnant steps.
  auto h = [&](int i, int j) -> cplx& { return H[(size_t)i * n + j]; };
  const double eps = 2.220446049250313e-16;
  int hi = n - 1, iter = 0, total = 0;
  std::vector<double> cs(n);
  std::vector<cplx> sn(n);
  while (hi > 0) {
    int l = hi;
    for (; l > 0; --l) {
      const double scale = std::abs(h(l - 1, l - 1)) + std::abs(h(l, l));
      if (std::abs(h(l, l - 1)) <= eps * (scale > 0 ? scale : 1.0)) {
        h(l, l - 1) = 0.0;
        break;
      }
    }
    if (l == hi) {
      --hi;
      iter = 0;
      continue;
    }
    if (++total > 60 * n) return false;
    ++iter;
    cplx mu;
    if (iter % 10 == 0) {
      mu = h(hi, hi) + 0.75 * std::abs(h(hi, hi - 1));
    } else {
      const cplx a = h(hi - 1, hi - 1), b = h(hi - 1, hi), c = h(hi, hi - 1), d = h(hi, hi);
      const cplx half = 0.5 * (a - d);
      const cplx disc = std::sqrt(half * half + b * c);
      const cplx m1 = 0.5 * (a + d) + disc, m2 = 0.5 * (a + d) - disc;
      mu = (std::abs(m1 - d) < std::abs(m2 - d)) ? m1 : m2;
    }
    for (int k = l; k <= hi; ++k) h(k, k) -= mu;
    for (int k = l; k < hi; ++k) {
      double c;
      cplx s;
      givens(h(k, k), h(k + 1, k), c, s);
      cs[k] = c;
      sn[k] = s;
      for (int j = k; j < n; ++j) {
        const cplx x = h(k, j), y = h(k + 1, j);
        h(k, j) = c * x + s * y;
        h(k + 1, j) = -std::conj(s) * x + c * y;
      }
    }
    for (int k = l; k < hi; ++k) {
      const double c = cs[k];
      const cplx s = sn[k];
      const int rmax = std::min(k + 2, hi);
      for (int i = 0; i <= rmax; ++i) {
        const cplx x = h(i, k), y = h(i, k + 1);
        h(i, k) = c * x + std::conj(s) * y;
        h(i, k + 1) = -s * x + c * y;
      }
      for (int i = 0; i < n; ++i) {
        const cplx x = Z[(size_t)i * n + k], y = Z[(size_t)i * n + k + 1];
        Z[(size_t)i * n + k] = c * x + std::conj(s) * y;
        Z[(size_t)i * n + k + 1] = -s * x + c * y;
      }
    }
    for (int k = l; k <= hi; ++k) h(k, k) += mu;
  }
  return true;
}

bool time_eig(const TimeLevel& tl, TimeEig& out) {
  const int n = tl.nt;
  // C = B^{-1} A
  std::vector<double> C = tl.A;
  if (!lu_solve_real(n, tl.B, C, n)) return false;
  // Householder reduction to upper Hessenberg form, Q accumulated.
  std::vector<double> Hm = C, Qm((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) Qm[(size_t)i * n + i] = 1.0;
  std::vector<double> v(n);
  for (int k = 0; k + 2 < n; ++k) {
    double alpha = 0.0;
    for (int i = k + 1; i < n; ++i) alpha += Hm[(size_t)i * n + k] * Hm[(size_t)i * n + k];
    alpha = std::sqrt(alpha);
    if (alpha == 0.0) continue;
    if (Hm[(size_t)(k + 1) * n + k] > 0) alpha = -alpha;
    std::fill(v.begin(), v.end(), 0.0);
    for (int i = k + 1; i < n; ++i) v[i] = Hm[(size_t)i * n + k];
    v[k + 1] -= alpha;
    double vn = 0.0;
    for (int i = k + 1; i < n; ++i) vn += v[i] * v[i];
    if (vn == 0.0) continue;
    // H <- (I - 2vv^T/vn) H (I - 2vv^T/vn);  Q <- Q (I - 2vv^T/vn)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int i = k + 1; i < n; ++i) s += v[i] * Hm[(size_t)i * n + j];
      s *= 2.0 / vn;
      for (int i = k + 1; i < n; ++i) Hm[(size_t)i * n + j] -= s * v[i];
    }
    for (int i = 0; i < n; ++i) {
      double s = 0.0;
      for (int j = k + 1; j < n; ++j) s += Hm[(size_t)i * n + j] * v[j];
      s *= 2.0 / vn;
      for (int j = k + 1; j < n; ++j) Hm[(size_t)i * n + j] -= s * v[j];
      double s2 = 0.0;
      for (int j = k + 1; j < n; ++j) s2 += Qm[(size_t)i * n + j] * v[j];
      s2 *= 2.0 / vn;
      for (int j = k + 1; j < n; ++j) Qm[(size_t)i * n + j] -= s2 * v[j];
    }
    for (int i = k + 2; i < n; ++i) Hm[(size_t)i * n + k] = 0.0;
  }
  std::vector<cplx> Hc(Hm.begin(), Hm.end()), Zc(Qm.begin(), Qm.end());
  if (!complex_schur(n, Hc, Zc)) return false;
  // Eigenvectors of the triangular factor by back substitution, then Z y.
  double tnorm = 0.0;
  for (auto& x : Hc) tnorm = std::max(tnorm, std::abs(x));
  std::vector<cplx> lam(n), Vall((size_t)n * n);
  std::vector<cplx> y(n);
  for (int k = 0; k < n; ++k) {
    lam[k] = Hc[(size_t)k * n + k];
    std::fill(y.begin(), y.end(), cplx(0.0));
    y[k] = 1.0;
    for (int j = k - 1; j >= 0; --j) {
      cplx s = 0.0;
      for (int l = j + 1; l <= k; ++l) s += Hc[(size_t)j * n + l] * y[l];
      cplx den = Hc[(size_t)j * n + j] - lam[k];
      if (std::abs(den) < 1e-14 * tnorm) den = 1e-14 * tnorm;
      y[j] = -s / den;
    }
    double nrm = 0.0;
    for (int i = 0; i < n; ++i) {
      cplx s = 0.0;
      for (int l = 0; l <= k; ++l) s += Zc[(size_t)i * n + l] * y[l];
      Vall[(size_t)i * n + k] = s;
      nrm += std::norm(s);
    }
    nrm = std::sqrt(nrm);
    for (int i = 0; i < n; ++i) Vall[(size_t)i * n + k] /= nrm;
  }
  // Classify: real eigenvalues and one member (Im > 0) of each conjugate pair.
  std::vector<int> keep_real, keep_pos;
  int n_neg = 0;
  for (int k = 0; k < n; ++k) {
    const double thr = 1e-9 * std::max(1.0, std::abs(lam[k]));
    if (std::fabs(lam[k].imag()) <= thr) keep_real.push_back(k);
    else if (lam[k].imag() > 0) keep_pos.push_back(k);
    else ++n_neg;
  }
  if ((int)keep_pos.size() != n_neg) return false;
  std::vector<int> order = keep_real;
  order.insert(order.end(), keep_pos.begin(), keep_pos.end());
  std::sort(order.begin(), order.end(), [&](int a, int b) { return lam[a].real() < lam[b].real(); });
  // Full eigenvector matrix: kept columns, each complex one followed by its conjugate.
  std::vector<cplx> Vf((size_t)n * n);
  std::vector<int> col_of(order.size());
  int c = 0;
  out.nt = n;
  out.nsel = (int)order.size();
  out.lam.clear();
  out.weight.clear();
  for (size_t q = 0; q < order.size(); ++q) {
    const int k = order[q];
    const bool is_real = std::fabs(lam[k].imag()) <= 1e-9 * std::max(1.0, std::abs(lam[k]));
    std::vector<cplx> col(n);
    for (int i = 0; i < n; ++i) col[i] = Vall[(size_t)i * n + k];
    if (is_real) {
      int imax = 0;
      for (int i = 1; i < n; ++i) if (std::abs(col[i]) > std::abs(col[imax])) imax = i;
      const cplx ph = std::abs(col[imax]) > 0 ? col[imax] / std::abs(col[imax]) : cplx(1.0);
      double nrm = 0.0;
      for (int i = 0; i < n; ++i) {
        col[i] = cplx((col[i] / ph).real(), 0.0);
        nrm += std::norm(col[i]);
      }
      nrm = std::sqrt(nrm);
      for (int i = 0; i < n; ++i) col[i] /= nrm;
      out.lam.push_back(cplx(lam[k].real(), 0.0));
      out.weight.push_back(1.0);
    } else {
      out.lam.push_back(lam[k]);
      out.weight.push_back(2.0);
    }
    col_of[q] = c;
    for (int i = 0; i < n; ++i) Vf[(size_t)i * n + c] = col[i];
    ++c;
    if (!is_real) {
      for (int i = 0; i < n; ++i) Vf[(size_t)i * n + c] = std::conj(col[i]);
      ++c;
    }
  }
  if (c != n) return false;
  std::vector<cplx> Vinv;
  if (!lu_inverse_cplx(n, Vf, Vinv)) return false;
  std::vector<double> Binv((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) Binv[(size_t)i * n + i] = 1.0;
  if (!lu_solve_real(n, tl.B, Binv, n)) return false;
  out.V.assign((size_t)n * out.nsel, cplx(0.0));
  out.W.assign((size_t)out.nsel * n, cplx(0.0));
  for (int q = 0; q < out.nsel; ++q) {
    const int cq = col_of[q];
    for (int i = 0; i < n; ++i) out.V[(size_t)i * out.nsel + q] = Vf[(size_t)i * n + cq];
    for (int j = 0; j < n; ++j) {
      cplx s = 0.0;
      for (int l = 0; l < n; ++l) s += Vinv[(size_t)cq * n + l] * Binv[(size_t)l * n + j];
      out.W[(size_t)q * n + j] = s;
    }
  }
  // Diagnostics: 1-norm condition estimate and eigen-residual of the full V.
  double n1 = 0.0, n1i = 0.0;
  for (int j = 0; j < n; ++j) {
    double s = 0.0, si = 0.0;
    for (int i = 0; i < n; ++i) {
      s += std::abs(Vf[(size_t)i * n + j]);
      si += std::abs(Vinv[(size_t)i * n + j]);
    }
    n1 = std::max(n1, s);
    n1i = std::max(n1i, si);
  }
  out.cond_est = n1 * n1i;
  double rr = 0.0, cn = 0.0, vn = 0.0;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      cn += C[(size_t)i * n + j] * C[(size_t)i * n + j];
      vn += std::norm(Vf[(size_t)i * n + j]);
    }
  std::vector<cplx> lamf(n);
  {
    int cc = 0;
    for (int q = 0; q < out.nsel; ++q) {
      lamf[cc++] = out.lam[q];
      if (out.weight[q] > 1.5) lamf[cc++] = std::conj(out.lam[q]);
    }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      cplx s = 0.0;
      for (int l = 0; l < n; ++l) s += C[(size_t)i * n + l] * Vf[(size_t)l * n + j];
      s -= Vf[(size_t)i * n + j] * lamf[j];
      rr += std::norm(s);
    }
  out.resid = std::sqrt(rr) / (std::sqrt(cn) * std::sqrt(vn));
  return true;
}

// Implicit QL iteration with Wilkinson-type shifts on a symmetric tridiagonal
// matrix (diagonal d, off-diagonal e[i] coupling i and i+1; the method of
// Bowdler, Martin, Reinsch and Wilkinson, 1968), applying every plane rotation
// to the rows i, i+1 of ZT (row j of ZT ends as the eigenvector of d[j]).
static bool tridiag_ql(int n, std::vector<double>& d, std::vector<double>& e, std::vector<double>& ZT) {
  const double eps = std::numeric_limits<double>::epsilon();
  e.resize(n, 0.0);
  e[n - 1] = 0.0;
  for (int l = 0; l < n; ++l) {
    for (int iter = 0;; ++iter) {
      int m = l;
      for (; m < n - 1; ++m)
        if (std::fabs(e[m]) <= eps * (std::fabs(d[m]) + std::fabs(d[m + 1]))) break;
      if (m == l) break;
      if (iter >= 60) return false;
      // shift from the eigenvalue of the leading 2 x 2 block nearer d[l]
      double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
      double r = std::hypot(g, 1.0);
      g = d[m] - d[l] + e[l] / (g + std::copysign(r, g));
      double sn = 1.0, cs = 1.0, p = 0.0;
      bool split = false;
      for (int i = m - 1; i >= l; --i) {
        const double f = sn * e[i], bb = cs * e[i];
        r = std::hypot(f, g);
        e[i + 1] = r;
        if (r == 0.0) {  // e[i+1] underflowed: the matrix splits there
          d[i + 1] -= p;
          e[m] = 0.0;
          split = true;
          break;
        }
        sn = f / r;
        cs = g / r;
        g = d[i + 1] - p;
        r = (d[i] - g) * sn + 2.0 * cs * bb;
        p = sn * r;
        d[i + 1] = g + p;
        g = cs * r - bb;
        double* zi = &ZT[(size_t)i * n];
        double* zj = zi + n;
        for (int k = 0; k < n; ++k) {
          const double a = zi[k], c = zj[k];
          zj[k] = sn * a + cs * c;
          zi[k] = cs * a - sn * c;
        }
      }
      if (split) continue;
      d[l] -= p;
      e[l] = g;
      e[m] = 0.0;
    }
  }
  return true;
}

bool sym_gen_eig(int n, const std::vector<double>& K, const std::vector<double>& M,
                 std::vector<double>& mu, std::vector<double>& Phi) {
  // Cholesky M = L L^T and C = L^{-1} K L^{-T}; Householder reduction
  // C = Q T Q^T to tridiagonal T; implicit QL on T with the rotations
  // accumulated into Q; Phi = L^{-T} Q so that Phi^T M Phi = I and
  // Phi^T K Phi = diag(mu).  Row-major throughout, inner loops over rows.
  std::vector<double> L((size_t)n * n, 0.0);
  for (int j = 0; j < n; ++j) {
    double s = M[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) s -= L[(size_t)j * n + k] * L[(size_t)j * n + k];
    if (s <= 0) return false;
    const double dj = std::sqrt(s);
    L[(size_t)j * n + j] = dj;
    for (int i = j + 1; i < n; ++i) {
      double t = M[(size_t)i * n + j];
      const double* li = &L[(size_t)i * n];
      const double* lj = &L[(size_t)j * n];
      for (int k = 0; k < j; ++k) t -= li[k] * lj[k];
      L[(size_t)i * n + j] = t / dj;
    }
  }
  // Y <- L^{-1} Y, row by row (forward substitution on all columns at once)
  auto fwd = [&](std::vector<double>& Y) {
    for (int i = 0; i < n; ++i) {
      double* yi = &Y[(size_t)i * n];
      for (int k = 0; k < i; ++k) {
        const double lik = L[(size_t)i * n + k];
        if (lik == 0.0) continue;
        const double* yk = &Y[(size_t)k * n];
        for (int c = 0; c < n; ++c) yi[c] -= lik * yk[c];
      }
      const double inv = 1.0 / L[(size_t)i * n + i];
      for (int c = 0; c < n; ++c) yi[c] *= inv;
    }
  };
  std::vector<double> X = K;
  fwd(X);
  std::vector<double> C((size_t)n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) C[(size_t)i * n + j] = X[(size_t)j * n + i];
  fwd(C);  // C = L^{-1} (L^{-1} K)^T = (L^{-1} K L^{-T})^T
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < i; ++j) {
      const double v = 0.5 * (C[(size_t)i * n + j] + C[(size_t)j * n + i]);
      C[(size_t)i * n + j] = C[(size_t)j * n + i] = v;
    }
  // Householder tridiagonalisation: step k maps column k below the
  // subdiagonal to zero with H_k = I - 2 v v^T acting on indices k+1..n-1.
  std::vector<double> d(n, 0.0), e(n, 0.0), V((size_t)n * n, 0.0), pv(n), wv(n);
  for (int k = 0; k + 2 < n; ++k) {
    const int m0 = k + 1, m = n - m0;
    double* vk = &V[(size_t)k * n];  // v stored at indices k+1..n-1
    double xn = 0.0;
    for (int i = m0; i < n; ++i) xn += C[(size_t)k * n + i] * C[(size_t)k * n + i];
    xn = std::sqrt(xn);
    const double x0 = C[(size_t)k * n + m0];
    d[k] = C[(size_t)k * n + k];
    if (xn == 0.0) {
      e[k] = 0.0;
      continue;
    }
    const double alpha = x0 > 0 ? -xn : xn;
    for (int i = m0; i < n; ++i) vk[i] = C[(size_t)k * n + i];
    vk[m0] -= alpha;
    double vn = 0.0;
    for (int i = m0; i < n; ++i) vn += vk[i] * vk[i];
    vn = std::sqrt(vn);
    for (int i = m0; i < n; ++i) vk[i] /= vn;
    // B <- H B H = B - v w^T - w v^T with p = B v, w = 2 (p - (v.p) v)
    double beta = 0.0;
    for (int i = m0; i < n; ++i) {
      const double* ci = &C[(size_t)i * n];
      double acc = 0.0;
      for (int j = m0; j < n; ++j) acc += ci[j] * vk[j];
      pv[i] = acc;
      beta += vk[i] * acc;
    }
    for (int i = m0; i < n; ++i) wv[i] = 2.0 * (pv[i] - beta * vk[i]);
    for (int i = m0; i < n; ++i) {
      double* ci = &C[(size_t)i * n];
      const double vi = vk[i], wi = wv[i];
      for (int j = m0; j < n; ++j) ci[j] -= vi * wv[j] + wi * vk[j];
    }
    e[k] = alpha;
    (void)m;
  }
  if (n >= 2) {
    d[n - 2] = C[(size_t)(n - 2) * n + (n - 2)];
    e[n - 2] = C[(size_t)(n - 2) * n + (n - 1)];
  }
  d[n - 1] = C[(size_t)(n - 1) * n + (n - 1)];
  // Q = H_0 H_1 ... H_{n-3}, accumulated from the right end
  std::vector<double> Q((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) Q[(size_t)i * n + i] = 1.0;
  for (int k = n - 3; k >= 0; --k) {
    const int m0 = k + 1;
    const double* vk = &V[(size_t)k * n];
    std::fill(pv.begin(), pv.end(), 0.0);
    for (int i = m0; i < n; ++i) {
      const double vi = vk[i];
      if (vi == 0.0) continue;
      const double* qi = &Q[(size_t)i * n];
      for (int j = m0; j < n; ++j) pv[j] += vi * qi[j];
    }
    for (int i = m0; i < n; ++i) {
      const double vi = 2.0 * vk[i];
      if (vi == 0.0) continue;
      double* qi = &Q[(size_t)i * n];
      for (int j = m0; j < n; ++j) qi[j] -= vi * pv[j];
    }
  }
  // eigenvectors of C: Z = Q S; with ZT = Q^T the QL rotations act on rows
  std::vector<double> ZT((size_t)n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) ZT[(size_t)j * n + i] = Q[(size_t)i * n + j];
  if (!tridiag_ql(n, d, e, ZT)) return false;
  mu = d;
  // Phi = L^{-T} Z (back substitution, rows from the bottom), Z = ZT^T
  Phi.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Phi[(size_t)i * n + j] = ZT[(size_t)j * n + i];
  for (int i = n - 1; i >= 0; --i) {
    double* pi = &Phi[(size_t)i * n];
    for (int k = i + 1; k < n; ++k) {
      const double lki = L[(size_t)k * n + i];
      if (lki == 0.0) continue;
      const double* pk = &Phi[(size_t)k * n];
      for (int c = 0; c < n; ++c) pi[c] -= lki * pk[c];
    }
    const double inv = 1.0 / L[(size_t)i * n + i];
    for (int c = 0; c < n; ++c) pi[c] *= inv;
  }
  return true;
}

bool band_lu(int n, int kl, int ku, std::vector<double>& ab, std::vector<int>& piv) {
  const int kv = kl + ku, ld = 2 * kl + ku + 1;
  auto a = [&](int i, int j) -> double& { return ab[(size_t)(kv + i - j) + (size_t)j * ld]; };
  piv.assign(n, 0);
  int ju = 0;
  for (int j = 0; j < n; ++j) {
    const int km = std::min(kl, n - 1 - j);
    int p = j;
    for (int i = j + 1; i <= j + km; ++i)
      if (std::fabs(a(i, j)) > std::fabs(a(p, j))) p = i;
    piv[j] = p;
    if (a(p, j) == 0.0) return false;
    ju = std::max(ju, std::min(j + ku + (p - j), n - 1));
    if (p != j)
      for (int c = j; c <= ju; ++c) std::swap(a(p, c), a(j, c));
    if (km > 0) {
      const double inv = 1.0 / a(j, j);
      for (int i = j + 1; i <= j + km; ++i) a(i, j) *= inv;
      for (int c = j + 1; c <= ju; ++c) {
        const double ajc = a(j, c);
        if (ajc == 0.0) continue;
        for (int i = j + 1; i <= j + km; ++i) a(i, c) -= a(i, j) * ajc;
      }
    }
  }
  return true;
}

}  // namespace st
