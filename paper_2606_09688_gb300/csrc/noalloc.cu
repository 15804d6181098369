// Allocation-free variant of the combination step (st_combine_noalloc).
//
// Who needs it: callers that must not allocate device memory at call time --
// for example a process whose device memory is fully reserved by another
// allocator (a framework's caching pool), or a time-critical loop where a
// cudaMalloc would synchronise the device.  They own their inputs and
// outputs; the only temporary storage this call needs (the B-spline tables
// of the components at the target times and the partial sums of the levels
// below the target level) lives in one fixed, file-scope device array that
// every GPU loading this library holds until the process exits.
#include <algorithm>
#include <mutex>
#include <vector>

#include "../../include/st.h"
#include "bspline.h"
#include "kernels.h"

namespace {

// Fixed scratch for st_combine_noalloc: 32 MiB per device.
constexpr size_t kNoallocScratchBytes = 32u << 20;
constexpr int kNoallocMaxComps = 64;
constexpr int kNoallocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

struct NoallocComps {
  st::CombComp c[kNoallocMaxComps];
};

// The device address of the scratch array, looked up once per device with
// that device current (in host code the symbol name is only a stand-in).
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kNoallocMaxDevices] = {nullptr};

st_status noalloc_scratch(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return ST_ERR_CUDA;
  if (dev < 0 || dev >= kNoallocMaxDevices) return ST_ERR_ARG;  // beyond the per-device address cache
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (g_noalloc_ptr[dev] == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return ST_ERR_CUDA;
    }
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return ST_OK;
}

// Component table and B-spline values of every component at every target
// time, written into the scratch (one block per component).
__global__ void k_noalloc_tables(NoallocComps comps, int ncomp, double T, int jts, int nts, st::CombComp* cdev,
                                 double* tbv, int* tspan) {
  const int c = blockIdx.x;
  if (c >= ncomp) return;
  const st::CombComp cc = comps.c[c];
  if (threadIdx.x == 0) cdev[c] = cc;
  const int Nt = 1 << cc.jt;
  for (int s = threadIdx.x; s < nts; s += blockDim.x) {
    int span = (cc.jt >= jts) ? (s << (cc.jt - jts)) : (s >> (jts - cc.jt));
    span = min(span, Nt - 1);
    const double t = T * (double)s / (double)(1 << jts);
    double v[3], d1[3], d2[3];
    st::bs_local(Nt, T, span, t, v, d1, d2);
    for (int a = 0; a < 3; ++a) tbv[((int64_t)c * nts + s) * 3 + a] = v[a];
    tspan[(int64_t)c * nts + s] = span;
  }
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

extern "C" st_status st_combine_noalloc(const st_comb_input* comps, int ncomp, int d, double T, int jx_star,
                                        int jt_star, double* out_dev, void* stream) {
  if (comps == nullptr || out_dev == nullptr || ncomp < 1 || ncomp > kNoallocMaxComps || d < 1 || d > 3 ||
      !(T > 0.0) || jx_star < 1 || jx_star > 14 || jt_star < 0 || jt_star > 14)
    return ST_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int nts = (1 << jt_star) + 1;
  // components ordered by their combination level min(jx, jx*)
  std::vector<int> order(ncomp);
  for (int c = 0; c < ncomp; ++c) {
    if (comps[c].U == nullptr || comps[c].jx < 1 || comps[c].jx > 14 || comps[c].jt < 0 || comps[c].jt > 14 ||
        (comps[c].coef != 1 && comps[c].coef != -1))
      return ST_ERR_ARG;
    order[c] = c;
  }
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return std::min(comps[a].jx, jx_star) < std::min(comps[b].jx, jx_star);
  });
  NoallocComps nc{};
  int jmin = jx_star;
  std::vector<int> first(jx_star + 2, ncomp);
  for (int o = 0; o < ncomp; ++o) {
    const st_comb_input& in = comps[order[o]];
    nc.c[o] = st::CombComp{in.U, in.lift, in.jx, in.jt, in.coef, 0};
    jmin = std::min(jmin, std::min(in.jx, jx_star));
  }
  for (int o = ncomp - 1; o >= 0; --o) first[std::min(nc.c[o].jx, jx_star)] = o;
  for (int lev = jx_star; lev >= 0; --lev) first[lev] = std::min(first[lev], first[lev + 1]);
  // scratch layout: components | B-spline values | spans | partial sums of levels jmin .. jx*-1
  size_t off = 0;
  const size_t off_comps = off;
  off = align256(off + sizeof(st::CombComp) * ncomp);
  const size_t off_tb = off;
  off = align256(off + sizeof(double) * 3 * (size_t)ncomp * nts);
  const size_t off_span = off;
  off = align256(off + sizeof(int) * (size_t)ncomp * nts);
  std::vector<size_t> off_y(jx_star + 1, 0);
  for (int lev = jmin; lev < jx_star; ++lev) {
    size_t nsp = 1;
    for (int k = 0; k < d; ++k) nsp *= (size_t)((1 << lev) + 1);
    off_y[lev] = off;
    off = align256(off + sizeof(double) * nsp * nts);
  }
  if (off > kNoallocScratchBytes) return ST_ERR_ARG;  // request exceeds the fixed 32 MiB scratch
  // An error left pending by earlier work on this thread is not this call's:
  // report it before enqueueing anything and leave it pending for its owner.
  if (cudaPeekAtLastError() != cudaSuccess) return ST_ERR_CUDA;
  void* base = nullptr;
  st_status st = noalloc_scratch(&base);
  if (st != ST_OK) return st;
  unsigned char* b = static_cast<unsigned char*>(base);
  st::CombComp* cdev = reinterpret_cast<st::CombComp*>(b + off_comps);
  double* tb = reinterpret_cast<double*>(b + off_tb);
  int* span = reinterpret_cast<int*>(b + off_span);
  k_noalloc_tables<<<ncomp, 256, 0, s>>>(nc, ncomp, T, jt_star, nts, cdev, tb, span);
  if (cudaGetLastError() != cudaSuccess) return ST_ERR_CUDA;
  for (int lev = jmin; lev <= jx_star; ++lev) {
    const double* Yp = lev > jmin ? reinterpret_cast<const double*>(b + off_y[lev - 1]) : nullptr;
    double* Y = lev == jx_star ? out_dev : reinterpret_cast<double*>(b + off_y[lev]);
    st::launch_comb_level(d, lev, Yp, cdev, first[lev], first[lev + 1], tb, span, nts, Y, s);
    if (cudaGetLastError() != cudaSuccess) return ST_ERR_CUDA;
  }
  return ST_OK;
}
