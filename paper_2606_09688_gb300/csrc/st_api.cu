// C ABI of the space-time sparse-grid wave solver: setup, component solves,
// combination.  Declarations and contracts: include/st.h.
//
// Component solve (Eq. (9) in the form of Eq. (30)):
//   (A (x) M + B (x) K) vec(U) = vec(F),   U: n_t x N_x, time-major.
// Time eigenbasis method: with B^{-1} A = V Lam V^{-1} and W = V^{-1} B^{-1},
//   G = W F,  (lam_q M + K) x_q = g_q for every mode q,  U = V X,
// conjugate modes folded (U = sum_real V_q x_q + 2 Re sum_pairs V_q x_q).
// Each spatial problem is complex symmetric; it is solved by COCG with a
// geometric multigrid V-cycle whose coarsest grid resolves the mode's wave
// number and is solved by a banded LDL^T, or by the banded LDL^T alone on
// small grids.
// Space eigenbasis method (fine time levels): K Phi = M Phi diag(mu),
// Phi^T M Phi = I, so Y = F Phi, (A + mu_a B) c_a = y_a (banded LU),
// U = C Phi^T.
// Both are wrapped in FP64 iterative refinement on R = F - (A (x) M + B (x) K) U.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <tuple>
#include <string>
#include <vector>

#include "../../include/st.h"
#include "../../include/st_host.h"
#include "band.h"
#include "host_math.h"
#include "kernels.h"
#include <nvtx3/nvToolsExt.h>

using namespace st;

namespace {

// NVTX range of one phase of an entry point (visible to profilers that
// record NVTX, e.g. ncu --nvtx; a no-op without one).
struct Phase {
  explicit Phase(const char* name) { nvtxRangePushA(name); }
  ~Phase() { nvtxRangePop(); }
  Phase(const Phase&) = delete;
  Phase& operator=(const Phase&) = delete;
};

constexpr int kMaxDirectRows = 32768;  // largest grid solved by the banded direct method (3D: 31^3)
constexpr int64_t kCoarseFloor = 1024;     // multigrid coarsening stops at the largest grid of at most this size
constexpr int64_t kMaxDenseCoarse = 4096;  // coarsest multigrid grids up to this size use an explicit inverse
constexpr int kMaxBandWidth = 1024;    // widest band the warp solve supports
constexpr int kMaxCoarseBand = 256;    // widest band of a multigrid coarsest grid
constexpr int64_t kMaxCoarseRows = 16384;  // largest multigrid coarsest grid
constexpr int kModeSMaxNx = 1024;      // dense spatial eigenbasis limit
constexpr int kModeTMaxNt = 129;       // time eigenbasis used up to this many time unknowns
constexpr double kKappaFP32 = 2.0e5;   // cond(V) above which inner solves stay in FP64
constexpr double kThetaMG = 1.25;      // coarsest-grid resolution: k h_c <= theta
constexpr double kShiftMG = 0.5;       // imaginary shift (x |Re lam|) of modes the coarsest grid cannot resolve
constexpr double kOmega2D = 0.6, kOmega3D = 0.55, kOmega1D = 0.6;
constexpr int kIterPerGraph = 4;  // COCG iterations between host convergence checks

struct DevMem {
  std::vector<void*> ptrs;
  size_t bytes = 0;
  ~DevMem() {
    for (void* p : ptrs) cudaFree(p);
  }
};

struct Status {
  st_status code = ST_OK;
  std::string msg;
};

// Stencil coefficient tables of a level (element matrices of Section 3.2:
// K1 = 1/h [1 -1; -1 1], M1 = h/6 [2 1; 1 2] per direction).
StencilCoef make_coef(int d, const double* h) {
  StencilCoef sc;
  std::memset(&sc, 0, sizeof(sc));
  const int ns = ipow3(d);
  for (int s = 0; s < ns; ++s) {
    int dl[3] = {0, 0, 0};
    int ss = s, zeros = 0;
    for (int k = 0; k < d; ++k) {
      dl[k] = ss % 3 - 1;
      ss /= 3;
      if (dl[k] == 0) ++zeros;
    }
    auto K1 = [&](int k) { return dl[k] == 0 ? 1.0 / h[k] : -1.0 / h[k]; };
    auto M1 = [&](int k) { return dl[k] == 0 ? h[k] / 3.0 : h[k] / 6.0; };
    double ke = 0.0;
    for (int dir = 0; dir < d; ++dir) {
      double t = 1.0;
      for (int k = 0; k < d; ++k) t *= (k == dir) ? K1(k) : M1(k);
      ke += t;
    }
    double m = (double)(1 << zeros);
    for (int k = 0; k < d; ++k) m *= M1(k);
    sc.ke[s] = ke;
    sc.mtot[s] = m;
  }
  return sc;
}

Geo make_geo(int d, int j) {
  Geo g;
  g.d = d;
  g.N = 1 << j;
  g.n = g.N - 1;
  g.nnodes = 1;
  g.ncells = 1;
  for (int k = 0; k < d; ++k) {
    g.nnodes *= g.n;
    g.ncells *= g.N;
  }
  g.dn = make_fastdiv((unsigned)g.n);
  return g;
}

int64_t band_width(const Geo& g) {
  if (g.d == 1) return 1;
  if (g.d == 2) return (int64_t)g.n + 1;
  return (int64_t)g.n * g.n + g.n + 1;
}

// One spatial multigrid level (c^2 of the component level, or cell averages of it).
struct MGLevel {
  int j = 0;
  Geo geo{};
  StencilCoef sc{};
  StencilCoefT<float> scf{};
  std::vector<double> c2h;
  double* c2d = nullptr;
  float* c2f = nullptr;
};

struct SpaceLevel {
  int jx = 0;
  Geo geo{};
  double h[3] = {0, 0, 0};
  StencilCoef sc{};
  std::vector<double> c2h;  // cellwise c^2 at the cell centres
  double* c2d = nullptr;
  float* c2f = nullptr;
  double* lift = nullptr;   // u0 on all nodes (nullptr if u0 == 0)
  double* loads = nullptr;  // (nterm + 2) x nx: M g_r ..., M v0, K u0
  double c2min = 0.0;
  int64_t nall = 0;
};

struct TimeData {
  TimeLevel tl;
  TimeEig eig;
  bool have_eig = false;
  double* Aband = nullptr;  // nt x 5
  double* Bband = nullptr;
  double* ATband = nullptr;  // transposes (adjoint systems)
  double* BTband = nullptr;
  cx<double>* W = nullptr;  // nsel x nt
  cx<double>* V = nullptr;  // nt x nsel
  cx<double>* VT = nullptr;  // nsel x nt: forward transform of the adjoint systems
  cx<double>* WT = nullptr;  // nt x nsel: their back transform
  double* wq = nullptr;
  cx<double>* lam64 = nullptr;
  cx<float>* lam32 = nullptr;
  double* rhs_coef = nullptr;  // (nterm + 2) x nt
};

template <typename R> struct Work {
  // level-0 vectors (nsel x nx): rhs G, iterate X, residual, search P, A P, z, smoother scratch
  cx<R>* G = nullptr;
  cx<R>* X = nullptr;
  cx<R>* Rr = nullptr;
  cx<R>* P = nullptr;
  cx<R>* Wv = nullptr;
  cx<R>* Z = nullptr;
  cx<R>* T0 = nullptr;
  cx<R>* R0 = nullptr;
  std::vector<cx<R>*> bl, rl, xa, xb;  // per MG level l >= 1
  cx<R>* band = nullptr;               // F factors, nsel x mstride
  cx<R>* bandG = nullptr;              // G (rows of L), nsel x mstride
  cx<R>* cinv = nullptr;               // coarsest-level inverses, nsel x n x n (small coarse grids)
  cx<R>* blk = nullptr;                // tile streams of the blocked solve, nsel x tstride (bw <= 128)
  bool ready = false;
};

struct Component {
  int jx = 0, jt = 0, coef = 0;
  int method = 0;  // 0 = time eigenbasis, 1 = space eigenbasis
  int64_t nx = 0;
  int nt = 0;
  SpaceLevel* sl = nullptr;
  TimeData* td = nullptr;
  double* F = nullptr;
  double* U = nullptr;
  double* Rv = nullptr;
  double* KU = nullptr;
  double* MU = nullptr;
  double* Fg_all = nullptr;  // general source, time-projected on all nodes (nt x nall), or nullptr
  ds* Uds[2] = {nullptr, nullptr};  // coef (U + u0) as pairs for the combination (nt x nx), two buffers
  ds* Lds = nullptr;                 // coef u0 on all nodes as pairs, or nullptr (written once)
  bool f_ready = false;
  bool solved = false;
  // time eigenbasis
  int nsel = 0;
  bool inner64 = false;
  bool direct = false;
  int jc = 0;
  std::vector<MGLevel> mg;  // mg[0] = component level
  int64_t nrowc = 0;
  int bw = 0;
  BandLayout bl{};
  BlkLayout bk{};  // blocked-solve layout of bl (rt = 0: too wide)
  std::vector<double> Kband, Mband;
  double* Kb = nullptr;
  double* Mb = nullptr;
  Work<double> w64;
  Work<float> w32;
  CocgScal* scal = nullptr;
  double* part = nullptr;
  std::vector<CocgScal> scal_h;
  // space eigenbasis
  double* Phi = nullptr;
  double* PhiT = nullptr;
  double* ab = nullptr;
  int* piv = nullptr;
  // eigenvalues of the multigrid preconditioner per mode (the true ones, or
  // shifted for modes the coarsest grid cannot resolve)
  cx<double>* lamP64 = nullptr;
  cx<float>* lamP32 = nullptr;
  int nshifted = 0;
  double* abT = nullptr;  // LU of (A + mu B)^T per spatial mode (adjoint systems)
  int* pivT = nullptr;
  int kl = 2, ku = 2;
  // adjoint state (receiver misfit gradient): right-hand side and solution, n_t x n_x
  double* Gadj = nullptr;
  double* Lam = nullptr;
  bool adj_solved = false;
  double Snorm = 0.0;  // upper bound of ||A (x) M + B (x) K||_2
  st_solve_info info{};
  int nactive = 0;  // modes still iterating at the last host check (for byte accounting)
  // Execution context: every component runs on its own stream with its own
  // reduction scratch, so that independent components overlap on the GPU.
  cudaStream_t cs = nullptr;
  cudaEvent_t done = nullptr;
  double* cpart = nullptr;
  double* cscalar = nullptr;
  double* cscalar_h = nullptr;  // pinned
  int* cerr = nullptr;
  int64_t d2h = 0;
  std::string err;
  // CUDA graphs of the COCG start (init + first V-cycle) and of kIterPerGraph
  // iterations, captured at setup on the component stream.
  cudaGraphExec_t g_init = nullptr, g_iter = nullptr;
  int64_t g_init_nodes = 0, g_iter_nodes = 0;
  double fnorm = -1.0;             // ||F|| of the forward right-hand side (constant after setup)
  // inner tolerance of the current refinement sweep (device scalar read by
  // the COCG convergence test) and its rule (next_inner_tol)
  double* itol = nullptr;
  InnerTol itol_rule{nullptr, 0.0, 1.0, 0};
  // The whole forward solve as one graph (st_options.device_loop > 0): the
  // refinement sweeps in a WHILE node, the COCG loop of a sweep in a nested
  // one; the host reads its record once the call's work is done.
  cudaGraphExec_t g_solve = nullptr;
  int64_t gs_pro_nodes = 0, gs_sweep_nodes = 0, gs_inner_nodes = 0;  // kernels: prologue, sweep, inner body
  RefineRec* rec = nullptr;    // device
  RefineRec* rec_h = nullptr;  // pinned copy
  double* fn2 = nullptr;       // ||F||^2 (device)
  bool rec_pending = false;    // a graph solve was enqueued; its record is not read yet
};

// Algorithmic flops per node of the complex Q1 stencil (K and M parts with
// 3^d neighbours, then the complex shift) and per node-mode for the real one.
inline double stencil_flops(int d) { return 8.0 * ipow3(d) + 8.0; }

}  // namespace

struct st_handle {
  st_problem prob{};
  st_options opt{};
  cudaStream_t stream = nullptr;
  DevMem mem;
  std::map<int, std::unique_ptr<SpaceLevel>> space;
  std::map<int, std::unique_ptr<TimeData>> time;
  std::vector<std::unique_ptr<Component>> comps;
  int nterm_rows = 0;  // n_terms + 2
  double* part = nullptr;
  double* scalar = nullptr;
  double* scalar_h = nullptr;  // pinned
  int64_t launches0 = 0;
  std::string err;
  int* dev_err = nullptr;
  int* solve_err = nullptr;  // set by bounded waits inside the band solve
  cudaEvent_t entry_ev = nullptr;
  cudaStream_t join = nullptr;  // waits for the components of a call whose solves run as graphs
  // Back-to-back st_solve_combine calls overlap (st_solve_combine): api_seq
  // counts the calls that may enqueue work on the handle's stream, sc_seq is
  // the count at the last st_solve_combine, sc_parity the pair buffer its
  // successor uses, sc_done_ev[p] the end of the levels of the last call that
  // used buffer p.
  // nodal parametrisation of c^2 and of the first source term's g (copies)
  std::vector<double> c2_nodal, g_nodal;
  int64_t api_seq = 0;
  int64_t sc_seq = -1;
  int sc_parity = 0;
  cudaEvent_t sc_done_ev[2] = {nullptr, nullptr};
  bool sc_done_rec[2] = {false, false};
  struct CombTables {
    CombComp* comps = nullptr;  // components ordered by combination level
    double* tb = nullptr;
    float* tbw = nullptr;       // the same weights as floats (exact when ds_ok)
    CombCompDS* dcomps[2] = {nullptr, nullptr};  // the components' pair arrays (two buffers), table order
    bool ds_ok = false;         // every weight exact in FP32: double-single levels
    std::vector<int> jt;        // time level of each table entry
    int* span = nullptr;
    int jmin = 0;
    std::vector<int> first;     // first[lev] = first component of level lev
    std::vector<int> order;     // component index of each table entry
    std::vector<double*> Y;     // partial sums of the levels below the target
  };
  std::map<std::tuple<int, int, uint64_t>, CombTables> comb;  // per target level pair and component set

  // Receiver tables of the misfit gradient (one receiver set cached).
  struct RecTables {
    int jt = -1, nrec = 0, ncorner = 0, nts = 0;
    std::vector<double> x;        // receiver coordinates (nrec x d)
    CombComp* comps = nullptr;    // components in component order
    RecCorner* rc = nullptr;      // ncomp x nrec x 2^d
    double* tb = nullptr;         // ncomp x nts x 3 B-spline values at the target times
    int* span = nullptr;          // ncomp x nts
    double* vals = nullptr;       // nts x nrec
    double* wm = nullptr;         // weighted misfit, nts x nrec
    double* J = nullptr;          // 1
    double* ehat = nullptr;       // max nt x nrec
    double* gv = nullptr;         // max nx
  } rec;

  // Optional per-kernel-class timing: CUDA events recorded on the handle's
  // stream around every launch, with the algorithmic bytes and flops of it.
  struct ProfRec {
    int cls;
    int64_t size;  // unknowns of the grid the launch works on
    cudaEvent_t a, b;
    double bytes, flops;
  };
  bool prof_on = false;
  std::mutex prof_mu;
  std::vector<ProfRec> prof;
  std::vector<cudaEvent_t> ev_pool;
  cudaEvent_t get_event() {
    if (!ev_pool.empty()) {
      cudaEvent_t e = ev_pool.back();
      ev_pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }

  ~st_handle() {
    if (scalar_h) cudaFreeHost(scalar_h);
    for (auto& c : comps) {
      if (c->g_init) cudaGraphExecDestroy(c->g_init);
      if (c->g_iter) cudaGraphExecDestroy(c->g_iter);
      if (c->g_solve) cudaGraphExecDestroy(c->g_solve);
      if (c->cscalar_h) cudaFreeHost(c->cscalar_h);
      if (c->rec_h) cudaFreeHost(c->rec_h);
      if (c->cs) cudaStreamDestroy(c->cs);
      if (c->done) cudaEventDestroy(c->done);
    }
    if (entry_ev) cudaEventDestroy(entry_ev);
    if (join) cudaStreamDestroy(join);
    for (auto e : sc_done_ev)
      if (e) cudaEventDestroy(e);
    for (auto& r : prof) {
      cudaEventDestroy(r.a);
      cudaEventDestroy(r.b);
    }
    for (auto e : ev_pool) cudaEventDestroy(e);
  }

  template <typename T> T* alloc(size_t n) {
    std::lock_guard<std::mutex> lock(alloc_mu);
    void* p = nullptr;
    if (n == 0) n = 1;
    if (opt.mem_cap_bytes > 0 && mem.bytes + n * sizeof(T) > (size_t)opt.mem_cap_bytes) return nullptr;
    if (cudaMalloc(&p, n * sizeof(T)) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    mem.ptrs.push_back(p);
    mem.bytes += n * sizeof(T);
    return static_cast<T*>(p);
  }
  template <typename T> T* upload(const std::vector<T>& v) {
    T* p = alloc<T>(v.size());
    if (p && !v.empty()) {
      cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, stream);
      h2d_bytes += (int64_t)(v.size() * sizeof(T));
    }
    return p;
  }
  int64_t h2d_bytes = 0, d2h_bytes = 0;
  std::mutex alloc_mu;
};

namespace {

thread_local std::string g_create_error;

st_status fail(st_handle* h, st_status code, const std::string& msg) {
  if (h) h->err = msg;
  else g_create_error = msg;
  return code;
}

#define ST_CUDA(h, call)                                                                    \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess) return fail(h, ST_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define ST_NEED(h, ptr)                                                          \
  do {                                                                           \
    if ((ptr) == nullptr) return fail(h, ST_ERR_OOM, "device allocation failed"); \
  } while (0)

enum KClass {
  KC_STENCIL = 0, KC_JACOBI, KC_MG_RESID, KC_RESTRICT, KC_PROLONG, KC_BAND_SOLVE, KC_REDUCE, KC_UPDATE,
  KC_TRANSFORM, KC_RESIDUAL64, KC_NORM, KC_RHS, KC_SPACE_EIG, KC_COMBINE, KC_SETUP, KC_DENSE_COARSE, KC_COUNT
};
const char* const kClassName[KC_COUNT] = {"stencil_apply", "jacobi_smooth", "mg_residual", "mg_restrict",
                                          "mg_prolong", "band_solve", "cocg_reduce", "cocg_update",
                                          "time_transform", "st_residual_fp64", "norm_fp64", "rhs_assemble",
                                          "space_eigenbasis", "combine_level", "setup", "coarse_inverse"};

struct ProfScope {
  st_handle* h;
  cudaStream_t s;
  int cls;
  int64_t size;
  double bytes, flops;
  cudaEvent_t a = nullptr;
  ProfScope(st_handle* h_, cudaStream_t s_, int cls_, int64_t size_, double bytes_, double flops_)
      : h(h_), s(s_), cls(cls_), size(size_), bytes(bytes_), flops(flops_) {
    if (h->prof_on) {
      std::lock_guard<std::mutex> lock(h->prof_mu);
      a = h->get_event();
      cudaEventRecord(a, s);
    }
  }
  ~ProfScope() {
    if (a) {
      std::lock_guard<std::mutex> lock(h->prof_mu);
      cudaEvent_t b = h->get_event();
      cudaEventRecord(b, s);
      h->prof.push_back({cls, size, a, b, bytes, flops});
    }
  }
};
#define PROF(h, s, cls, size, bytes, flops, call) \
  do {                                           \
    ProfScope ps_(h, s, cls, size, bytes, flops); \
    call;                                        \
  } while (0)

st_status check_launch(st_handle* h, const char* where) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(h, ST_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
  return ST_OK;
}

// Evaluate a space callback at points (n x d).
st_status eval_space(st_handle* h, const st_field& f, const std::vector<double>& pts, int d, std::vector<double>& out) {
  const int64_t n = (int64_t)pts.size() / d;
  out.assign(n, 0.0);
  if (f.fn == nullptr) return ST_OK;
  if (f.fn(n, pts.data(), out.data(), f.user) != 0) return fail(h, ST_ERR_CALLBACK, "space callback failed");
  return ST_OK;
}

// Values of a nodal parameter field (level param_level, multilinear) at points.
void eval_nodal(const st_problem& p, const std::vector<double>& vals, const std::vector<double>& pts,
                std::vector<double>& out) {
  ParamGrid pg{};
  pg.d = p.d;
  pg.Np = 1 << p.param_level;
  for (int k = 0; k < p.d; ++k) {
    pg.lo[k] = p.lo[k];
    pg.h[k] = (p.hi[k] - p.lo[k]) / pg.Np;
  }
  const int64_t n = (int64_t)pts.size() / p.d;
  out.assign(n, 0.0);
  for (int64_t i = 0; i < n; ++i) {
    double x[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < p.d; ++k) x[k] = pts[(size_t)i * p.d + k];
    out[i] = p.d == 1 ? param_eval<1>(pg, vals.data(), x)
                      : (p.d == 2 ? param_eval<2>(pg, vals.data(), x) : param_eval<3>(pg, vals.data(), x));
  }
}

std::vector<double> node_points(const st_problem& p, int j) {
  const int N = 1 << j, d = p.d;
  int64_t nn = 1;
  for (int k = 0; k < d; ++k) nn *= (N + 1);
  std::vector<double> pts((size_t)nn * d);
  for (int64_t a = 0; a < nn; ++a) {
    int64_t r = a;
    for (int k = 0; k < d; ++k) {
      const int ik = (int)(r % (N + 1));
      r /= (N + 1);
      pts[(size_t)a * d + k] = p.lo[k] + (p.hi[k] - p.lo[k]) * ik / N;
    }
  }
  return pts;
}

std::vector<double> cell_centres(const st_problem& p, int j) {
  const int N = 1 << j, d = p.d;
  int64_t nc = 1;
  for (int k = 0; k < d; ++k) nc *= N;
  std::vector<double> pts((size_t)nc * d);
  for (int64_t a = 0; a < nc; ++a) {
    int64_t r = a;
    for (int k = 0; k < d; ++k) {
      const int ik = (int)(r % N);
      r /= N;
      pts[(size_t)a * d + k] = p.lo[k] + (p.hi[k] - p.lo[k]) * (ik + 0.5) / N;
    }
  }
  return pts;
}

// Real band of K(c2) and M of a level: entry (k + j, k) at [k * (bw + 1) + j].
void assemble_band(const Geo& g, const StencilCoef& sc, const std::vector<double>& c2, std::vector<double>& Kb,
                   std::vector<double>& Mb, int bw) {
  const int64_t W = bw + 1;
  Kb.assign((size_t)(g.nnodes * W), 0.0);
  Mb.assign((size_t)(g.nnodes * W), 0.0);
  const int d = g.d, n = g.n, N = g.N;
  const int ns = ipow3(d);
  for (int64_t a = 0; a < g.nnodes; ++a) {
    int i[3] = {0, 0, 0};
    int64_t r = a;
    for (int k = 0; k < d; ++k) {
      i[k] = (int)(r % n);
      r /= n;
    }
    double c[8];
    for (int e = 0; e < (1 << d); ++e) {
      int64_t idx = 0, st = 1;
      for (int k = 0; k < d; ++k) {
        idx += (int64_t)(i[k] + ((e >> k) & 1)) * st;
        st *= N;
      }
      c[e] = c2[(size_t)idx];
    }
    for (int s = 0; s < ns; ++s) {
      int ss = s;
      int64_t off = 0, st = 1;
      bool ok = true;
      int dl[3] = {0, 0, 0};
      for (int k = 0; k < d; ++k) {
        dl[k] = ss % 3 - 1;
        ss /= 3;
        const int jk = i[k] + dl[k];
        ok = ok && jk >= 0 && jk < n;
        off += (int64_t)dl[k] * st;
        st *= n;
      }
      if (!ok || off < 0) continue;
      double S = 0.0;
      for (int e = 0; e < (1 << d); ++e) {
        bool in = true;
        for (int k = 0; k < d; ++k) {
          const int ek = (e >> k) & 1;
          in = in && (dl[k] == 0 || (dl[k] == 1 && ek == 1) || (dl[k] == -1 && ek == 0));
        }
        if (in) S += c[e];
      }
      Kb[(size_t)(a * W + off)] = S * sc.ke[s];
      Mb[(size_t)(a * W + off)] = sc.mtot[s];
    }
  }
}

std::vector<double> average_c2(int d, int Nf, const std::vector<double>& cf) {
  const int Nc = Nf / 2;
  int64_t ncc = 1;
  for (int k = 0; k < d; ++k) ncc *= Nc;
  std::vector<double> cc((size_t)ncc, 0.0);
  for (int64_t a = 0; a < ncc; ++a) {
    int ic[3] = {0, 0, 0};
    int64_t r = a;
    for (int k = 0; k < d; ++k) {
      ic[k] = (int)(r % Nc);
      r /= Nc;
    }
    double s = 0.0;
    for (int e = 0; e < (1 << d); ++e) {
      int64_t idx = 0, st = 1;
      for (int k = 0; k < d; ++k) {
        idx += (int64_t)(2 * ic[k] + ((e >> k) & 1)) * st;
        st *= Nf;
      }
      s += cf[(size_t)idx];
    }
    cc[(size_t)a] = s / (1 << d);
  }
  return cc;
}

// ------------------------------------------------------------------ setup parts
st_status setup_space_level(st_handle* h, int jx, SpaceLevel& sl) {
  const st_problem& p = h->prob;
  sl.jx = jx;
  sl.geo = make_geo(p.d, jx);
  for (int k = 0; k < p.d; ++k) sl.h[k] = (p.hi[k] - p.lo[k]) / (1 << jx);
  sl.sc = make_coef(p.d, sl.h);
  st_status s = ST_OK;
  if (!h->c2_nodal.empty()) eval_nodal(p, h->c2_nodal, cell_centres(p, jx), sl.c2h);
  else s = eval_space(h, p.c2, cell_centres(p, jx), p.d, sl.c2h);
  if (s != ST_OK) return s;
  sl.c2min = 1e300;
  for (double v : sl.c2h) {
    if (!(v > 0.0) || !std::isfinite(v)) return fail(h, ST_ERR_ARG, "c^2 must be positive and finite at every cell centre");
    sl.c2min = std::min(sl.c2min, v);
  }
  sl.c2d = h->upload(sl.c2h);
  ST_NEED(h, sl.c2d);
  std::vector<float> cf(sl.c2h.begin(), sl.c2h.end());
  sl.c2f = h->upload(cf);
  ST_NEED(h, sl.c2f);
  const std::vector<double> pts = node_points(p, jx);
  sl.nall = (int64_t)pts.size() / p.d;
  const int nrows = h->nterm_rows;
  sl.loads = h->alloc<double>((size_t)nrows * sl.geo.nnodes);
  ST_NEED(h, sl.loads);
  double* tmp = h->alloc<double>((size_t)sl.nall);
  ST_NEED(h, tmp);
  std::vector<double> vals;
  auto load_row = [&](const st_field& f, int row, double aK, double aM, bool keep_lift,
                      const std::vector<double>* nodal = nullptr) -> st_status {
    if (nodal != nullptr && !nodal->empty()) {
      eval_nodal(p, *nodal, pts, vals);
    } else {
      st_status s2 = eval_space(h, f, pts, p.d, vals);
      if (s2 != ST_OK) return s2;
    }
    ST_CUDA(h, cudaMemcpyAsync(tmp, vals.data(), vals.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    h->h2d_bytes += (int64_t)(vals.size() * sizeof(double));
    launch_load(sl.geo, sl.sc, sl.c2d, tmp, sl.loads + (size_t)row * sl.geo.nnodes, aK, aM, 0, h->stream);
    if (keep_lift && f.fn != nullptr) {
      sl.lift = h->alloc<double>((size_t)sl.nall);
      ST_NEED(h, sl.lift);
      ST_CUDA(h, cudaMemcpyAsync(sl.lift, tmp, vals.size() * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    }
    ST_CUDA(h, cudaStreamSynchronize(h->stream));
    return check_launch(h, "load");
  };
  for (int r = 0; r < p.n_terms; ++r) {
    st_field g{p.terms[r].g, p.terms[r].g_user};
    if ((s = load_row(g, r, 0.0, 1.0, false, r == 0 ? &h->g_nodal : nullptr)) != ST_OK) return s;
  }
  if ((s = load_row(p.v0, p.n_terms, 0.0, 1.0, false)) != ST_OK) return s;
  if ((s = load_row(p.u0, p.n_terms + 1, 1.0, 0.0, true)) != ST_OK) return s;
  return ST_OK;
}

st_status setup_time_level(st_handle* h, int jt, TimeData& td) {
  const st_problem& p = h->prob;
  build_time_level(jt, p.T, td.tl);
  const int nt = td.tl.nt;
  std::vector<double> Ab((size_t)nt * 5, 0.0), Bb((size_t)nt * 5, 0.0);
  for (int i = 0; i < nt; ++i)
    for (int t = -2; t <= 2; ++t) {
      const int j = i + t;
      if (j < 0 || j >= nt) continue;
      Ab[(size_t)i * 5 + t + 2] = td.tl.A[(size_t)i * nt + j];
      Bb[(size_t)i * 5 + t + 2] = td.tl.B[(size_t)i * nt + j];
    }
  td.Aband = h->upload(Ab);
  td.Bband = h->upload(Bb);
  ST_NEED(h, td.Aband);
  ST_NEED(h, td.Bband);
  // transposed bands: row i holds A(j, i) for j = i - 2 .. i + 2
  std::vector<double> ATb((size_t)nt * 5, 0.0), BTb((size_t)nt * 5, 0.0);
  for (int i = 0; i < nt; ++i)
    for (int t = -2; t <= 2; ++t) {
      const int j = i + t;
      if (j < 0 || j >= nt) continue;
      ATb[(size_t)i * 5 + t + 2] = td.tl.A[(size_t)j * nt + i];
      BTb[(size_t)i * 5 + t + 2] = td.tl.B[(size_t)j * nt + i];
    }
  td.ATband = h->upload(ATb);
  td.BTband = h->upload(BTb);
  ST_NEED(h, td.ATband);
  ST_NEED(h, td.BTband);
  // RHS time coefficient rows: (s_r, psi_i')_e, psi_i'(0), -(1, psi_i')_e.
  const int nrows = h->nterm_rows;
  std::vector<double> coef((size_t)nrows * nt, 0.0);
  const int nq = (int)td.tl.qt.size();
  std::vector<double> sv(nq);
  for (int r = 0; r < p.n_terms; ++r) {
    if (p.terms[r].s == nullptr) return fail(h, ST_ERR_ARG, "source term without time factor");
    if (p.terms[r].s(nq, td.tl.qt.data(), sv.data(), p.terms[r].s_user) != 0)
      return fail(h, ST_ERR_CALLBACK, "time callback failed");
    for (int i = 0; i < nt; ++i) {
      double acc = 0.0;
      for (int q = 0; q < nq; ++q) acc += td.tl.Q[(size_t)i * nq + q] * sv[q];
      coef[(size_t)r * nt + i] = acc;
    }
  }
  for (int i = 0; i < nt; ++i) {
    coef[(size_t)p.n_terms * nt + i] = td.tl.d0[i];
    coef[(size_t)(p.n_terms + 1) * nt + i] = -td.tl.g1[i];
  }
  td.rhs_coef = h->upload(coef);
  ST_NEED(h, td.rhs_coef);
  return ST_OK;
}

// Coarsest multigrid level of a time-eigenbasis component: the coarsest grid
// must resolve the largest wave number k = sqrt(-Re lam / min c^2) of its
// modes (k h_c <= theta); grids with at most max_direct unknowns (default
// kMaxDirectRows) are solved directly.
int choose_coarse(const st_problem& p, const Component& c, int64_t max_direct) {
  double kmax = 0.0;
  for (int q = 0; q < c.td->eig.nsel; ++q)
    kmax = std::max(kmax, std::sqrt(std::max(0.0, -c.td->eig.lam[q].real()) / c.sl->c2min));
  double L = 0.0;
  for (int k = 0; k < p.d; ++k) L = std::max(L, p.hi[k] - p.lo[k]);
  // no coarser than the largest grid of at most kCoarseFloor nodes (its
  // explicit inverse is cheap): below it, extra levels only add launches to
  // every V-cycle
  int jc = 2;
  while (jc + 1 < c.jx && make_geo(p.d, jc + 1).nnodes <= kCoarseFloor) ++jc;
  while (jc < c.jx && kmax * L / (1 << jc) > kThetaMG) ++jc;
  auto fits = [&](int j) {
    const Geo g = make_geo(p.d, j);
    return g.nnodes <= max_direct && band_width(g) <= kMaxBandWidth;
  };
  if (fits(c.jx)) return c.jx;  // the banded direct solve beats a V-cycle with a large coarse grid
  // a coarsest multigrid grid is solved once per V-cycle: keep it within the
  // fast banded solves (band <= kMaxCoarseBand); modes it cannot resolve get
  // the shifted V-cycle
  auto fits_coarse = [&](int j) {
    const Geo g = make_geo(p.d, j);
    return fits(j) && g.nnodes <= kMaxCoarseRows && band_width(g) <= kMaxCoarseBand;
  };
  int jmax = 1;  // largest level the coarse banded solve handles
  while (jmax + 1 <= c.jx && fits_coarse(jmax + 1)) ++jmax;
  if (jc >= c.jx) return jmax;
  return std::min(jc, jmax);
}

// ||S||_2 <= ||A||_2 ||M||_2 + ||B||_2 ||K||_2 with ||X||_2 <= sqrt(||X||_1 ||X||_inf),
// ||M||_2 <= max row sum = prod h_k and ||K||_2 <= max_a sum_b |K_ab|.
double system_norm_bound(const Component& c) {
  const TimeLevel& tl = c.td->tl;
  const int nt = tl.nt;
  auto n2 = [&](const std::vector<double>& X) {
    double n1 = 0.0, ni = 0.0;
    for (int i = 0; i < nt; ++i) {
      double r = 0.0, cs = 0.0;
      for (int j = 0; j < nt; ++j) {
        r += std::fabs(X[(size_t)i * nt + j]);
        cs += std::fabs(X[(size_t)j * nt + i]);
      }
      ni = std::max(ni, r);
      n1 = std::max(n1, cs);
    }
    return std::sqrt(n1 * ni);
  };
  const Geo& g = c.sl->geo;
  double mnorm = 1.0;
  for (int k = 0; k < g.d; ++k) mnorm *= c.sl->h[k];
  double c2max = 0.0;
  for (double v : c.sl->c2h) c2max = std::max(c2max, v);
  double knorm = 0.0;
  const int ns = ipow3(g.d);
  for (int s = 0; s < ns; ++s) {
    int ss = s, zeros = 0;
    for (int k = 0; k < g.d; ++k) {
      if (ss % 3 == 1) ++zeros;
      ss /= 3;
    }
    knorm += (double)(1 << zeros) * c2max * std::fabs(c.sl->sc.ke[s]);
  }
  return n2(tl.A) * mnorm + n2(tl.B) * knorm;
}

st_status setup_component(st_handle* h, Component& c) {
  const st_problem& p = h->prob;
  c.nx = c.sl->geo.nnodes;
  c.nt = c.td->tl.nt;
  c.Snorm = system_norm_bound(c);
  const size_t n = (size_t)c.nx * c.nt;
  c.F = h->alloc<double>(n);
  c.U = h->alloc<double>(n);
  c.Rv = h->alloc<double>(n);
  c.KU = h->alloc<double>(n);
  c.MU = h->alloc<double>(n);
  ST_NEED(h, c.F);
  ST_NEED(h, c.U);
  ST_NEED(h, c.Rv);
  ST_NEED(h, c.KU);
  ST_NEED(h, c.MU);
  if (p.f_general != nullptr) {
    // time-projected general source on all nodes: sum_q Q[i][q] f(x, t_q)
    const std::vector<double> pts = node_points(p, c.jx);
    const int64_t nall = (int64_t)pts.size() / p.d;
    const int nq = (int)c.td->tl.qt.size();
    std::vector<double> acc((size_t)c.nt * nall, 0.0), fv(nall);
    for (int q = 0; q < nq; ++q) {
      if (p.f_general(nall, pts.data(), c.td->tl.qt[q], fv.data(), p.f_user) != 0)
        return fail(h, ST_ERR_CALLBACK, "source callback failed");
      for (int i = 0; i < c.nt; ++i) {
        const double w = c.td->tl.Q[(size_t)i * nq + q];
        if (w == 0.0) continue;
        for (int64_t a = 0; a < nall; ++a) acc[(size_t)i * nall + a] += w * fv[a];
      }
    }
    c.Fg_all = h->upload(acc);
    ST_NEED(h, c.Fg_all);
  }
  if (c.method == 1) {
    // space eigenbasis: dense K, M of the level, Phi, banded LU of A + mu B per spatial mode
    const Geo& g = c.sl->geo;
    const int bw = (int)band_width(g);
    std::vector<double> Kb, Mb;
    assemble_band(g, c.sl->sc, c.sl->c2h, Kb, Mb, bw);
    const int nx = (int)c.nx;
    std::vector<double> K((size_t)nx * nx, 0.0), M((size_t)nx * nx, 0.0);
    for (int a = 0; a < nx; ++a)
      for (int j = 0; j <= bw && a + j < nx; ++j) {
        K[(size_t)(a + j) * nx + a] = K[(size_t)a * nx + a + j] = Kb[(size_t)a * (bw + 1) + j];
        M[(size_t)(a + j) * nx + a] = M[(size_t)a * nx + a + j] = Mb[(size_t)a * (bw + 1) + j];
      }
    std::vector<double> mu, Phi;
    if (!sym_gen_eig(nx, K, M, mu, Phi)) return fail(h, ST_ERR_NUMERIC, "spatial eigen-decomposition failed");
    std::vector<double> PhiT((size_t)nx * nx);
    for (int i = 0; i < nx; ++i)
      for (int j = 0; j < nx; ++j) PhiT[(size_t)j * nx + i] = Phi[(size_t)i * nx + j];
    c.Phi = h->upload(Phi);
    c.PhiT = h->upload(PhiT);
    ST_NEED(h, c.Phi);
    ST_NEED(h, c.PhiT);
    const int nt = c.nt, kl = 2, ku = 2, ld = 2 * kl + ku + 1;
    if (time_band_smem(nt) > kTimeBandMaxSmem)
      return fail(h, ST_ERR_ARG, "time level too fine for the space-eigenbasis band solve");
    // LU of A + mu_a B (forward) and of its transpose (adjoint) per spatial mode
    for (int tr = 0; tr < 2; ++tr) {
      std::vector<double> abAll((size_t)ld * nt * nx, 0.0);
      std::vector<int> pivAll((size_t)nt * nx, 0);
      std::vector<double> ab((size_t)ld * nt);
      std::vector<int> piv;
      for (int a = 0; a < nx; ++a) {
        std::fill(ab.begin(), ab.end(), 0.0);
        for (int j = 0; j < nt; ++j)
          for (int i = std::max(0, j - ku); i <= std::min(nt - 1, j + kl); ++i) {
            const size_t e = tr == 0 ? (size_t)i * nt + j : (size_t)j * nt + i;
            ab[(size_t)(kl + ku + i - j) + (size_t)j * ld] = c.td->tl.A[e] + mu[a] * c.td->tl.B[e];
          }
        if (!band_lu(nt, kl, ku, ab, piv)) return fail(h, ST_ERR_NUMERIC, "time band LU failed");
        // mode-major for the solve kernel, the diagonal of U as its reciprocal
        for (int j = 0; j < nt; ++j) ab[(size_t)(kl + ku) + (size_t)j * ld] = 1.0 / ab[(size_t)(kl + ku) + (size_t)j * ld];
        std::copy(ab.begin(), ab.end(), abAll.begin() + (size_t)a * ld * nt);
        std::copy(piv.begin(), piv.end(), pivAll.begin() + (size_t)a * nt);
      }
      double* abd = h->upload(abAll);
      int* pivd = h->upload(pivAll);
      ST_NEED(h, abd);
      ST_NEED(h, pivd);
      (tr == 0 ? c.ab : c.abT) = abd;
      (tr == 0 ? c.piv : c.pivT) = pivd;
    }
    c.kl = kl;
    c.ku = ku;
    ST_CUDA(h, cudaStreamSynchronize(h->stream));
    return ST_OK;
  }
  // time eigenbasis
  c.nsel = c.td->eig.nsel;
  c.inner64 = (h->opt.precision == ST_FP64) || (c.td->eig.cond_est > kKappaFP32);
  c.jc = choose_coarse(p, c, h->opt.max_direct_rows > 0 ? (int64_t)h->opt.max_direct_rows : kMaxDirectRows);
  c.direct = (c.jc == c.jx);
  // multigrid hierarchy jx -> jc (level 0 uses the sampled c^2)
  c.mg.clear();
  {
    MGLevel l0;
    l0.j = c.jx;
    l0.geo = c.sl->geo;
    l0.sc = c.sl->sc;
    l0.scf = to_float(l0.sc);
    l0.c2h = c.sl->c2h;
    l0.c2d = c.sl->c2d;
    l0.c2f = c.sl->c2f;
    c.mg.push_back(l0);
  }
  for (int j = c.jx - 1; j >= c.jc; --j) {
    MGLevel l;
    l.j = j;
    l.geo = make_geo(p.d, j);
    double hh[3];
    for (int k = 0; k < p.d; ++k) hh[k] = (p.hi[k] - p.lo[k]) / (1 << j);
    l.sc = make_coef(p.d, hh);
    l.scf = to_float(l.sc);
    l.c2h = average_c2(p.d, 1 << (j + 1), c.mg.back().c2h);
    l.c2d = h->upload(l.c2h);
    std::vector<float> cf(l.c2h.begin(), l.c2h.end());
    l.c2f = h->upload(cf);
    ST_NEED(h, l.c2d);
    ST_NEED(h, l.c2f);
    c.mg.push_back(std::move(l));
  }
  // Preconditioner eigenvalues.  A mode whose wave number k_q = sqrt(-Re lam_q / min c^2)
  // is not resolved by the coarsest grid (k_q h_c > theta: the V-cycle of K + lam_q M
  // then stalls) gets the V-cycle of the shifted operator K + (lam_q + i beta |Re lam_q|) M,
  // which multigrid handles; COCG keeps the true operator, and the shifted
  // preconditioner is still complex symmetric.
  {
    double Lbox = 0.0;
    for (int k = 0; k < p.d; ++k) Lbox = std::max(Lbox, p.hi[k] - p.lo[k]);
    const double hc = Lbox / (1 << c.jc);
    std::vector<cx<double>> lp(c.nsel);
    std::vector<cx<float>> lpf(c.nsel);
    c.nshifted = 0;
    for (int q = 0; q < c.nsel; ++q) {
      const std::complex<double> l = c.td->eig.lam[q];
      double im = l.imag();
      const double kq = std::sqrt(std::max(0.0, -l.real()) / c.sl->c2min);
      if (!c.direct && kq * hc > kThetaMG) {
        im += (im >= 0.0 ? 1.0 : -1.0) * kShiftMG * std::fabs(l.real());
        ++c.nshifted;
      }
      lp[q] = mk(l.real(), im);
      lpf[q] = mk((float)l.real(), (float)im);
    }
    if (c.nshifted > 0) {
      c.lamP64 = h->upload(lp);
      c.lamP32 = h->upload(lpf);
      ST_NEED(h, c.lamP64);
      ST_NEED(h, c.lamP32);
    } else {
      c.lamP64 = c.td->lam64;
      c.lamP32 = c.td->lam32;
    }
  }
  const MGLevel& lc = c.mg.back();
  c.bw = (int)band_width(lc.geo);
  c.nrowc = lc.geo.nnodes;
  c.bl = band_layout(c.nrowc, c.bw);
  c.bl.wait = (long long)h->opt.wait_cycles;
  c.bl.stall = h->opt.inject_stall;
  assemble_band(lc.geo, lc.sc, lc.c2h, c.Kband, c.Mband, c.bw);
  c.Kb = h->upload(c.Kband);
  c.Mb = h->upload(c.Mband);
  ST_NEED(h, c.Kb);
  ST_NEED(h, c.Mb);
  c.scal = h->alloc<CocgScal>(c.nsel);
  c.part = h->alloc<double>((size_t)c.nsel * 304 * 2);
  ST_NEED(h, c.scal);
  ST_NEED(h, c.part);
  c.scal_h.resize(c.nsel);
  return ST_OK;
}

template <typename R> Work<R>& work_of(Component& c);
template <> Work<double>& work_of<double>(Component& c) { return c.w64; }
template <> Work<float>& work_of<float>(Component& c) { return c.w32; }
template <typename R> const StencilCoefT<R>& coef_of(const MGLevel& l);
template <> const StencilCoefT<double>& coef_of<double>(const MGLevel& l) { return l.sc; }
template <> const StencilCoefT<float>& coef_of<float>(const MGLevel& l) { return l.scf; }
template <typename R> const R* c2_of(const MGLevel& l);
template <> const double* c2_of<double>(const MGLevel& l) { return l.c2d; }
template <> const float* c2_of<float>(const MGLevel& l) { return l.c2f; }

st_status cfail(Component& c, st_status code, const std::string& msg) {
  if (c.err.empty()) c.err = msg;
  return code;
}

#define ST_CUDAC(c, call)                                                                                 \
  do {                                                                                                    \
    cudaError_t e_ = (call);                                                                              \
    if (e_ != cudaSuccess) return cfail(c, ST_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

st_status ccheck(Component& c, const char* where) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cfail(c, ST_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
  return ST_OK;
}

// Workspace and coarsest-level factorisations of a time-eigenbasis component.
// The factorisations run on the component's own stream (after the uploads on
// the handle's stream), so that those of different components overlap with
// each other and with the host work of the components set up after it; the
// zero-pivot flag they leave in c.cerr is read at the end of st_setup.
double omega_of(int d);

template <typename R> st_status prepare_work(st_handle* h, Component& c) {
  Work<R>& w = work_of<R>(c);
  if (w.ready) return ST_OK;
  const size_t n0 = (size_t)c.nsel * c.nx;
  w.G = h->alloc<cx<R>>(n0);
  w.X = h->alloc<cx<R>>(n0);
  ST_NEED(h, w.G);
  ST_NEED(h, w.X);
  if (!c.direct) {
    w.Rr = h->alloc<cx<R>>(n0);
    w.P = h->alloc<cx<R>>(n0);
    w.Wv = h->alloc<cx<R>>(n0);
    w.Z = h->alloc<cx<R>>(n0);
    w.T0 = h->alloc<cx<R>>(n0);
    w.R0 = h->alloc<cx<R>>(n0);
    ST_NEED(h, w.Rr);
    ST_NEED(h, w.P);
    ST_NEED(h, w.Wv);
    ST_NEED(h, w.Z);
    ST_NEED(h, w.T0);
    ST_NEED(h, w.R0);
    const int L = (int)c.mg.size();
    w.bl.assign(L, nullptr);
    w.rl.assign(L, nullptr);
    w.xa.assign(L, nullptr);
    w.xb.assign(L, nullptr);
    for (int l = 1; l < L; ++l) {
      const size_t nl = (size_t)c.nsel * c.mg[l].geo.nnodes;
      w.bl[l] = h->alloc<cx<R>>(nl);
      w.rl[l] = h->alloc<cx<R>>(nl);
      w.xa[l] = h->alloc<cx<R>>(nl);
      w.xb[l] = h->alloc<cx<R>>(nl);
      ST_NEED(h, w.bl[l]);
      ST_NEED(h, w.rl[l]);
      ST_NEED(h, w.xa[l]);
      ST_NEED(h, w.xb[l]);
    }
  }
  // coarsest-level factorisations, one per mode
  w.band = h->alloc<cx<R>>((size_t)c.nsel * c.bl.mstride);
  w.bandG = h->alloc<cx<R>>((size_t)c.nsel * c.bl.mstride);
  ST_NEED(h, w.band);
  ST_NEED(h, w.bandG);
  ST_CUDA(h, cudaEventRecord(h->entry_ev, h->stream));
  ST_CUDA(h, cudaStreamWaitEvent(c.cs, h->entry_ev, 0));
  launch_band_form<R>(c.Kb, c.Mb, c.lamP64, w.band, c.bl, c.nsel, c.cs);
  launch_band_factor<R>(w.band, w.bandG, c.bl, c.nsel, c.cerr, c.cs);
  if constexpr (sizeof(R) == 8) {
    // FP64 sweeps are bound by the FP64 pipe: the damped inverse diagonal of
    // every smoothed level and mode is formed once (the complex reciprocal is
    // about a fifth of a sweep's FP64 operations); FP32 sweeps, bound by
    // memory, keep forming it on the fly
    for (int l = 0; !c.direct && l + 1 < (int)c.mg.size(); ++l) {
      MGLevel& lv = c.mg[l];
      cx<R>* dv = h->alloc<cx<R>>((size_t)c.nsel * lv.geo.nnodes);
      ST_NEED(h, dv);
      launch_jacobi_dinv<R>(lv.geo, lv.sc, lv.c2d, c.lamP64, omega_of(lv.geo.d), c.nsel, lv.geo.nnodes, dv, c.cs);
      lv.sc.dinv = dv;
    }
  }
  c.bk = blk_layout(c.bl);
  if (c.bk.rt > 0 && (c.direct || c.bl.nrow > kMaxDenseCoarse)) {
    // banded solves in every step: blocked solve with precomputed block inverses
    w.blk = h->alloc<cx<R>>((size_t)c.nsel * c.bk.tstride);
    ST_NEED(h, w.blk);
    launch_band_blk_prepare<R>(w.band, c.bl, c.bk, w.blk, c.nsel, c.cs);
  }
  if (!c.direct && c.bl.nrow <= kMaxDenseCoarse) {
    // multigrid coarsest level: explicit inverses, column j = the banded
    // solve of e_j (all columns of one mode in one launch, factor shared)
    const int64_t nc = c.bl.nrow;
    cx<R>* ident = h->alloc<cx<R>>((size_t)(nc * nc));
    w.cinv = h->alloc<cx<R>>((size_t)(c.nsel * nc * nc));
    ST_NEED(h, ident);
    ST_NEED(h, w.cinv);
    launch_identity<R>(ident, nc, c.cs);
    BandLayout shared = c.bl;
    shared.mstride = 0;
    for (int q = 0; q < c.nsel; ++q)
      launch_band_solve<R>(w.band + (int64_t)q * c.bl.mstride, w.bandG + (int64_t)q * c.bl.mstride, shared, ident,
                           w.cinv + (int64_t)q * nc * nc, nullptr, (int)nc, nc, c.cerr, c.cs);
  }
  st_status s = check_launch(h, "band factorisation");
  if (s != ST_OK) return s;
  w.ready = true;
  return ST_OK;
}

template <typename R> const cx<R>* lam_of(const TimeData& td);
template <> const cx<double>* lam_of<double>(const TimeData& td) { return td.lam64; }
template <> const cx<float>* lam_of<float>(const TimeData& td) { return td.lam32; }
template <typename R> const cx<R>* plam_of(const Component& c);
template <> const cx<double>* plam_of<double>(const Component& c) { return c.lamP64; }
template <> const cx<float>* plam_of<float>(const Component& c) { return c.lamP32; }

// Banded solve of every active mode of the component's direct grid: the
// blocked solve when its tile streams exist, the row-by-row kernels otherwise.
template <typename R>
bool band_solve(Component& c, const cx<R>* b, cx<R>* x, const CocgScal* scal, int64_t vstride, cudaStream_t s) {
  Work<R>& w = work_of<R>(c);
  if (w.blk != nullptr) {
    launch_band_solve_blk<R>(w.band, c.bl, c.bk, w.blk, b, x, scal, c.nsel, vstride, c.cerr, s);
    return true;
  }
  return launch_band_solve<R>(w.band, w.bandG, c.bl, b, x, scal, c.nsel, vstride, c.cerr, s);
}

double omega_of(int d) { return d == 1 ? kOmega1D : (d == 2 ? kOmega2D : kOmega3D); }

// x = B_mg b on level l: damped-Jacobi sweeps before and after the coarse
// correction (one each way for FP64 inner solves, two for FP32); the pre- and
// post-smoothers are the same symmetric sweep, so B_mg stays complex symmetric.
// Returns the buffer holding the result.
template <typename R>
cx<R>* vcycle(st_handle* h, Component& c, int l, const cx<R>* b, cx<R>* xa, cx<R>* xb, cx<R>* rtmp) {
  Work<R>& w = work_of<R>(c);
  const MGLevel& lv = c.mg[l];
  const cx<R>* lam = plam_of<R>(c);
  const int64_t n = lv.geo.nnodes;
  cudaStream_t s = c.cs;
  const int L = (int)c.mg.size() - 1;
  const double m = (double)c.nactive, cs = sizeof(cx<R>), rs = sizeof(R);
  const double fl = stencil_flops(lv.geo.d);
  if (l == L) {
    if (w.cinv != nullptr) {
      PROF(h, s, KC_DENSE_COARSE, (int64_t)(n), m * (double)n * (n + 2.0) * cs, m * (double)n * n * 8.0,
           launch_dense_coarse<R>(w.cinv, n, b, xb, c.scal, c.nsel, n, s));
    } else {
      PROF(h, s, KC_BAND_SOLVE, (int64_t)(n), m * (double)n * (2.0 * c.bl.ld * cs + 3 * cs),
           m * (double)n * c.bw * 16.0, band_solve<R>(c, b, xb, c.scal, n, s));
    }
    return xb;
  }
  const double om = omega_of(lv.geo.d);
  const R* c2 = c2_of<R>(lv);
  const double cb = (double)lv.geo.ncells * rs;
  const MGLevel& lc = c.mg[l + 1];
  const double nc = (double)lc.geo.nnodes;
  if constexpr (sizeof(R) == 8) {
    // FP64 inner solves are bound by the FP64 pipe: one sweep before and one
    // after the coarse correction (V(1,1)) costs fewer FP64 operations per
    // solve than V(2,2) despite one or two more Krylov iterations.  The sweeps
    // read the damped inverse diagonal (StencilCoefT::dinv): 16 more bytes and
    // one complex product per node and mode instead of the division
    PROF(h, s, KC_JACOBI, (int64_t)(n), m * n * 3 * cs, m * n * 6.0,
         launch_stencil<R>(OP_JACOBI_ZERO, lv.geo, coef_of<R>(lv), c2, nullptr, b, xb, lam, c.scal, c.nsel, n, om, s));
    PROF(h, s, KC_MG_RESID, (int64_t)(n), m * n * 3 * cs + cb, m * n * (fl + 2.0),
         launch_stencil<R>(OP_RESID, lv.geo, coef_of<R>(lv), c2, xb, b, rtmp, lam, c.scal, c.nsel, n, om, s));
    PROF(h, s, KC_RESTRICT, (int64_t)(n), m * (n + nc) * cs, m * nc * 4.0 * ipow3(lv.geo.d),
         launch_restrict<R>(lv.geo, lc.geo, rtmp, w.bl[l + 1], c.scal, c.nsel, n, lc.geo.nnodes, s));
    cx<R>* xc = vcycle<R>(h, c, l + 1, w.bl[l + 1], w.xa[l + 1], w.xb[l + 1], w.rl[l + 1]);
    PROF(h, s, KC_PROLONG, (int64_t)(n), m * (2.0 * n + nc) * cs, m * n * 4.0 * (1 << lv.geo.d),
         launch_prolong_add<R>(lv.geo, lc.geo, xc, xb, c.scal, c.nsel, n, lc.geo.nnodes, s));
    PROF(h, s, KC_JACOBI, (int64_t)(n), m * n * 4 * cs + cb, m * n * (fl + 8.0),
         launch_stencil<R>(OP_JACOBI, lv.geo, coef_of<R>(lv), c2, xb, b, xa, lam, c.scal, c.nsel, n, om, s));
    return xa;
  }
  // FP32 inner solves are bound by latency and launches: V(2,2), fewer iterations
  PROF(h, s, KC_JACOBI, (int64_t)(n), m * n * 2 * cs + cb, m * n * 30.0,
       launch_stencil<R>(OP_JACOBI_ZERO, lv.geo, coef_of<R>(lv), c2, nullptr, b, xa, lam, c.scal, c.nsel, n, om, s));
  PROF(h, s, KC_JACOBI, (int64_t)(n), m * n * 3 * cs + cb, m * n * (fl + 30.0),
       launch_stencil<R>(OP_JACOBI, lv.geo, coef_of<R>(lv), c2, xa, b, xb, lam, c.scal, c.nsel, n, om, s));
  PROF(h, s, KC_MG_RESID, (int64_t)(n), m * n * 3 * cs + cb, m * n * (fl + 2.0),
       launch_stencil<R>(OP_RESID, lv.geo, coef_of<R>(lv), c2, xb, b, rtmp, lam, c.scal, c.nsel, n, om, s));
  PROF(h, s, KC_RESTRICT, (int64_t)(n), m * (n + nc) * cs, m * nc * 4.0 * ipow3(lv.geo.d),
       launch_restrict<R>(lv.geo, lc.geo, rtmp, w.bl[l + 1], c.scal, c.nsel, n, lc.geo.nnodes, s));
  cx<R>* xc = vcycle<R>(h, c, l + 1, w.bl[l + 1], w.xa[l + 1], w.xb[l + 1], w.rl[l + 1]);
  PROF(h, s, KC_PROLONG, (int64_t)(n), m * (2.0 * n + nc) * cs, m * n * 4.0 * (1 << lv.geo.d),
       launch_prolong_add<R>(lv.geo, lc.geo, xc, xb, c.scal, c.nsel, n, lc.geo.nnodes, s));
  PROF(h, s, KC_JACOBI, (int64_t)(n), m * n * 3 * cs + cb, m * n * (fl + 30.0),
       launch_stencil<R>(OP_JACOBI, lv.geo, coef_of<R>(lv), c2, xb, b, xa, lam, c.scal, c.nsel, n, om, s));
  PROF(h, s, KC_JACOBI, (int64_t)(n), m * n * 3 * cs + cb, m * n * (fl + 30.0),
       launch_stencil<R>(OP_JACOBI, lv.geo, coef_of<R>(lv), c2, xa, b, xb, lam, c.scal, c.nsel, n, om, s));
  return xb;
}

double inner_tol(const st_handle* h, size_t rsize) {
  if (h->opt.inner_tol > 0.0) return h->opt.inner_tol;
  // FP32: each sweep gains about four digits whatever the inner tolerance
  // (the FP32 representation of the correction limits it), so a loose
  // inner solve costs fewer iterations for the same number of sweeps.
  // FP64: the first sweep's backward error is about 3e-4 times the inner
  // tolerance on the multigrid components (3e-16 at 1e-12, 30 times below
  // the default target 1e-14), so 1e-11 still meets the target in one sweep;
  // where it does not, the next sweep solves only as far as needed
  // (next_inner_tol)
  return rsize == 8 ? 1e-11 : 1e-4;
}

// COCG start: x = 0, r = g, z = B r, rho = r . z, p = z.
template <typename R> void cocg_start(st_handle* h, Component& c) {
  Work<R>& w = work_of<R>(c);
  cudaStream_t s = c.cs;
  const int64_t n = c.nx;
  const double cs = sizeof(cx<R>);
  const double tol = inner_tol(h, sizeof(R));
  const int max_iter = h->opt.max_iter > 0 ? h->opt.max_iter : 1000;
  PROF(h, s, KC_REDUCE, (int64_t)(n), c.nsel * (double)n * 3 * cs, c.nsel * (double)n * 4.0,
       launch_cocg_init<R>(w.G, w.X, w.Rr, c.scal, c.part, c.nsel, n, n, s));
  cx<R>* z = vcycle<R>(h, c, 0, w.Rr, w.T0, w.Z, w.R0);
  PROF(h, s, KC_REDUCE, (int64_t)(n), c.nactive * (double)n * 2 * cs, c.nactive * (double)n * 8.0,
       launch_dot<R>(2, w.Rr, z, c.scal, c.part, c.nsel, n, n, tol, max_iter, s));
  PROF(h, s, KC_UPDATE, (int64_t)(n), c.nactive * (double)n * 2 * cs, 0.0, launch_update_p<R>(w.P, z, c.scal, c.nsel, n, n, 1, s));
}

// One COCG iteration: w = A p, alpha, x += alpha p, r -= alpha w (modes that
// converge are switched off on the device), z = B r, beta, p = z + beta p.
template <typename R> void cocg_iteration(st_handle* h, Component& c) {
  Work<R>& w = work_of<R>(c);
  cudaStream_t s = c.cs;
  const int64_t n = c.nx;
  const double cs = sizeof(cx<R>), rs = sizeof(R);
  const double tol = inner_tol(h, sizeof(R));
  const int max_iter = h->opt.max_iter > 0 ? h->opt.max_iter : 1000;
  const MGLevel& l0 = c.mg[0];
  const R* c2 = c2_of<R>(l0);
  const cx<R>* lam = lam_of<R>(*c.td);
  const double fl = stencil_flops(l0.geo.d), cb = (double)l0.geo.ncells * rs;
  const double m = c.nactive;
  PROF(h, s, KC_STENCIL, (int64_t)(n), m * n * 2 * cs + cb, m * n * fl,
       launch_stencil<R>(OP_APPLY, l0.geo, coef_of<R>(l0), c2, w.P, nullptr, w.Wv, lam, c.scal, c.nsel, n, 0.0, s));
  PROF(h, s, KC_REDUCE, (int64_t)(n), m * n * 2 * cs, m * n * 8.0,
       launch_dot<R>(0, w.P, w.Wv, c.scal, c.part, c.nsel, n, n, tol, max_iter, s));
  PROF(h, s, KC_UPDATE, (int64_t)(n), m * n * 6 * cs, m * n * 12.0,
       launch_update_xr<R>(w.X, w.Rr, w.P, w.Wv, c.scal, c.part, c.nsel, n, n, tol, max_iter, s, c.itol));
  cx<R>* z = vcycle<R>(h, c, 0, w.Rr, w.T0, w.Z, w.R0);
  PROF(h, s, KC_REDUCE, (int64_t)(n), m * n * 2 * cs, m * n * 8.0,
       launch_dot<R>(1, w.Rr, z, c.scal, c.part, c.nsel, n, n, tol, max_iter, s));
  PROF(h, s, KC_UPDATE, (int64_t)(n), m * n * 3 * cs, m * n * 8.0, launch_update_p<R>(w.P, z, c.scal, c.nsel, n, n, 0, s));
}

// Launch shapes of the stencil operations of every multigrid level of a
// component, timed on its own work buffers (zeroed first) before the COCG
// iterations are captured; levels below kTuneMinNodes keep the built-in rule.
// The shapes are kept process-wide, so later handles with the same grids and
// mode counts reuse them.
constexpr int64_t kTuneMinNodes = 4096;
template <typename R> st_status tune_component(st_handle* h, Component& c) {
  Work<R>& w = work_of<R>(c);
  const cx<R>* lam = plam_of<R>(c);
  const int L = (int)c.mg.size() - 1;
  for (int l = 0; l < L; ++l) {
    const MGLevel& lv = c.mg[l];
    const int64_t n = lv.geo.nnodes;
    if (n < kTuneMinNodes) continue;
    cx<R>* x = l == 0 ? w.X : w.xa[l];
    cx<R>* b = l == 0 ? w.G : w.bl[l];
    cx<R>* y = l == 0 ? w.Wv : w.xb[l];
    const size_t bytes = (size_t)c.nsel * n * sizeof(cx<R>);
    ST_CUDAC(c, cudaMemsetAsync(x, 0, bytes, c.cs));
    ST_CUDAC(c, cudaMemsetAsync(b, 0, bytes, c.cs));
    const double om = omega_of(lv.geo.d);
    const R* c2 = c2_of<R>(lv);
    const int ops[4] = {OP_JACOBI_ZERO, OP_JACOBI, OP_RESID, OP_APPLY};
    for (int op : ops) {
      if (op == OP_APPLY && l != 0) continue;
      if (tune_stencil<R>(op, lv.geo, coef_of<R>(lv), c2, x, b, y, lam, c.nsel, n, om, c.cs) < 0.f)
        return cfail(c, ST_ERR_CUDA, "stencil autotuning failed");
    }
  }
  return ccheck(c, "autotune");
}

// Capture the COCG start and kIterPerGraph iterations as CUDA graphs on the
// component stream (every pointer and size is fixed after setup; modes that
// converge are skipped on the device through their active flags).
template <typename R> st_status capture_graphs(st_handle* h, Component& c) {
  c.nactive = c.nsel;
  for (int which = 0; which < 2; ++which) {
    cudaGraph_t g = nullptr;
    const int64_t l0 = kernel_launch_count();
    ST_CUDA(h, cudaStreamBeginCapture(c.cs, cudaStreamCaptureModeThreadLocal));
    if (which == 0) cocg_start<R>(h, c);
    else
      for (int k = 0; k < kIterPerGraph; ++k) cocg_iteration<R>(h, c);
    ST_CUDA(h, cudaStreamEndCapture(c.cs, &g));
    cudaGraphExec_t ge = nullptr;
    const cudaError_t e = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(h, ST_ERR_CUDA, std::string("graph instantiation: ") + cudaGetErrorString(e));
    const int64_t nodes = kernel_launch_count() - l0;
    if (which == 0) {
      c.g_init = ge;
      c.g_init_nodes = nodes;
    } else {
      c.g_iter = ge;
      c.g_iter_nodes = nodes;
    }
  }
  return check_launch(h, "graph capture");
}

// Solve (lam_q M + K) x_q = g_q for every mode; w.G holds g, the result lands in w.X.
template <typename R> st_status inner_solve(st_handle* h, Component& c, int& iters_out) {
  Work<R>& w = work_of<R>(c);
  cudaStream_t s = c.cs;
  const int64_t n = c.nx;
  const double cs = sizeof(cx<R>);
  iters_out = 0;
  c.nactive = c.nsel;
  if (c.direct) {
    const double m = c.nsel;
    PROF(h, s, KC_BAND_SOLVE, (int64_t)(n), m * (double)n * (2.0 * c.bl.ld * cs + 3 * cs), m * (double)n * c.bw * 16.0,
         band_solve<R>(c, w.G, w.X, nullptr, n, s));
    return ccheck(c, "direct band solve");
  }
  const int max_iter = h->opt.max_iter > 0 ? h->opt.max_iter : 1000;
  const bool graphs = !h->prof_on && c.g_init != nullptr && c.g_iter != nullptr;
  if (graphs) {
    ST_CUDAC(c, cudaGraphLaunch(c.g_init, s));
    note_launches((int)c.g_init_nodes);
  } else {
    cocg_start<R>(h, c);
  }
  for (int it = 0; it < max_iter; it += kIterPerGraph) {
    if (graphs) {
      ST_CUDAC(c, cudaGraphLaunch(c.g_iter, s));
      note_launches((int)c.g_iter_nodes);
    } else {
      for (int k = 0; k < kIterPerGraph; ++k) cocg_iteration<R>(h, c);
    }
    ST_CUDAC(c, cudaMemcpyAsync(c.scal_h.data(), c.scal, c.nsel * sizeof(CocgScal), cudaMemcpyDeviceToHost, s));
    c.d2h += (int64_t)(c.nsel * sizeof(CocgScal));
    ST_CUDAC(c, cudaStreamSynchronize(s));
    st_status st = ccheck(c, "cocg");
    if (st != ST_OK) return st;
    int na = 0;
    for (const auto& q : c.scal_h) na += q.active ? 1 : 0;
    c.nactive = na;
    if (na == 0) break;
  }
  int worst = 0;
  for (const auto& q : c.scal_h) {
    iters_out = std::max(iters_out, q.iters);
    if (q.status != 0) worst = q.status;
  }
  if (worst == 4) return cfail(c, ST_ERR_NOT_CONVERGED, "COCG reached its iteration limit");
  if (worst != 0) return cfail(c, ST_ERR_NUMERIC, "COCG breakdown or non-finite value");
  return ST_OK;
}

st_status assemble_rhs(st_handle* h, Component& c) {
  if (c.f_ready) return ST_OK;
  PROF(h, c.cs, KC_RHS, (int64_t)(c.nx), (double)(h->nterm_rows + c.nt) * c.nx * 8.0, 2.0 * h->nterm_rows * c.nt * (double)c.nx,
       launch_rhs_assemble(c.td->rhs_coef, c.sl->loads, c.F, h->nterm_rows, c.nt, c.nx, c.cs));
  if (c.Fg_all != nullptr)
    for (int i = 0; i < c.nt; ++i)
      launch_load(c.sl->geo, c.sl->sc, c.sl->c2d, c.Fg_all + (size_t)i * c.sl->nall, c.F + (size_t)i * c.nx, 0.0,
                  1.0, 1, c.cs);
  c.f_ready = true;
  return ccheck(c, "rhs");
}

// ||a|| and ||b|| (2-norms) with one synchronisation.
st_status read_norm2(st_handle* h, Component& c, const double* a, const double* b, int64_t n, double& na, double& nb) {
  PROF(h, c.cs, KC_NORM, (int64_t)(n), (double)n * 8.0, 2.0 * n, launch_norm2(a, n, c.cpart, c.cscalar, c.cs));
  PROF(h, c.cs, KC_NORM, (int64_t)(n), (double)n * 8.0, 2.0 * n, launch_norm2(b, n, c.cpart, c.cscalar + 1, c.cs));
  int serr = 0;
  ST_CUDAC(c, cudaMemcpyAsync(&serr, c.cerr, sizeof(int), cudaMemcpyDeviceToHost, c.cs));
  ST_CUDAC(c, cudaMemcpyAsync(c.cscalar_h, c.cscalar, 2 * sizeof(double), cudaMemcpyDeviceToHost, c.cs));
  c.d2h += (int64_t)(2 * sizeof(double) + sizeof(int));
  ST_CUDAC(c, cudaStreamSynchronize(c.cs));
  na = std::sqrt(c.cscalar_h[0]);
  nb = std::sqrt(c.cscalar_h[1]);
  if (serr) return cfail(c, ST_ERR_TIMEOUT, "a bounded copy wait in the banded solve timed out");
  return ccheck(c, "norm");
}

st_status read_norm(st_handle* h, Component& c, const double* v, int64_t n, double& out) {
  PROF(h, c.cs, KC_NORM, (int64_t)(n), (double)n * 8.0, 2.0 * n, launch_norm2(v, n, c.cpart, c.cscalar, c.cs));
  int serr = 0;
  ST_CUDAC(c, cudaMemcpyAsync(&serr, c.cerr, sizeof(int), cudaMemcpyDeviceToHost, c.cs));
  ST_CUDAC(c, cudaMemcpyAsync(c.cscalar_h, c.cscalar, sizeof(double), cudaMemcpyDeviceToHost, c.cs));
  c.d2h += (int64_t)(sizeof(double) + sizeof(int));
  ST_CUDAC(c, cudaStreamSynchronize(c.cs));
  out = std::sqrt(*c.cscalar_h);
  if (serr) return cfail(c, ST_ERR_TIMEOUT, "a bounded copy wait in the banded solve timed out");
  return ccheck(c, "norm");
}

// The operators of one component solve: the forward system S U = F, or the
// adjoint system S^T L = G (transposed time factors; same spatial modes).
struct SolveIO {
  const double* rhs;
  double* sol;
  const cx<double>* Wf;  // forward transform (nsel x nt)
  const cx<double>* Vb;  // back transform (nt x nsel)
  const double* Ab;      // time bands of the residual
  const double* Bb;
  const double* lu_ab;   // space eigenbasis: band LU per spatial mode
  const int* lu_piv;
};

SolveIO forward_io(Component& c) {
  return SolveIO{c.F, c.U, c.td->W, c.td->V, c.td->Aband, c.td->Bband, c.ab, c.piv};
}
SolveIO adjoint_io(Component& c) {
  return SolveIO{c.Gadj, c.Lam, c.td->VT, c.td->WT, c.td->ATband, c.td->BTband, c.abT, c.pivT};
}

template <typename R>
st_status sweep_time_eig(st_handle* h, Component& c, const SolveIO& io, const double* Rin, int& iters) {
  Work<R>& w = work_of<R>(c);
  const double cs = sizeof(cx<R>), nx = (double)c.nx;
  PROF(h, c.cs, KC_TRANSFORM, (int64_t)(c.nx), c.nt * nx * 8.0 + c.nsel * nx * cs, 4.0 * c.nsel * c.nt * nx,
       launch_fwd_transform<R>(io.Wf, Rin, w.G, c.nsel, c.nt, c.nx, c.cs));
  st_status s = inner_solve<R>(h, c, iters);
  if (s != ST_OK) return s;
  PROF(h, c.cs, KC_TRANSFORM, (int64_t)(c.nx), 2.0 * c.nt * nx * 8.0 + c.nsel * nx * cs, 4.0 * c.nsel * c.nt * nx,
       launch_back_transform<R>(io.Vb, c.td->wq, w.X, io.sol, c.nsel, c.nt, c.nx, c.cs));
  return ccheck(c, "time transforms");
}

st_status sweep_space_eig(st_handle* h, Component& c, const SolveIO& io, const double* Rin) {
  const double nx = (double)c.nx, nt = c.nt;
  PROF(h, c.cs, KC_SPACE_EIG, (int64_t)(c.nx), (2.0 * nt * nx + nx * nx) * 8.0, 2.0 * nt * nx * nx,
       launch_gemm_right(Rin, c.Phi, c.KU, c.nt, c.nx, 0, 0, c.cs));
  bool ok = true;
  PROF(h, c.cs, KC_SPACE_EIG, (int64_t)(c.nx), (2.0 * nt * nx + 7.0 * nt * nx) * 8.0, 12.0 * nt * nx,
       ok = launch_time_band_solve(io.lu_ab, io.lu_piv, c.KU, c.nt, c.nx, c.kl, c.ku, c.cs));
  if (!ok) return cfail(c, ST_ERR_ARG, "time band solve: unsupported size");
  PROF(h, c.cs, KC_SPACE_EIG, (int64_t)(c.nx), (3.0 * nt * nx + nx * nx) * 8.0, 2.0 * nt * nx * nx,
       launch_gemm_right(c.KU, c.PhiT, io.sol, c.nt, c.nx, 1, 1, c.cs));
  return ccheck(c, "space eigenbasis sweep");
}

st_status enqueue_graph_solve(st_handle* h, Component& c);
bool graph_solves(const st_handle* h);

st_status solve_one(st_handle* h, Component& c, const SolveIO& io, bool adjoint) {
  if (!adjoint && graph_solves(h) && c.g_solve != nullptr) return enqueue_graph_solve(h, c);
  st_status s = ST_OK;
  if (!adjoint && (s = assemble_rhs(h, c)) != ST_OK) return s;
  const size_t n = (size_t)c.nx * c.nt;
  ST_CUDAC(c, cudaMemsetAsync(io.sol, 0, n * sizeof(double), c.cs));
  double fn = 0.0;
  if (!adjoint && c.fnorm >= 0.0) {
    fn = c.fnorm;  // F is fixed after setup
  } else {
    if ((s = read_norm(h, c, io.rhs, (int64_t)n, fn)) != ST_OK) return s;
    if (!adjoint) c.fnorm = fn;
  }
  // Refinement stops on the normwise backward error eta = ||R|| / (||S|| ||U|| + ||F||)
  // (the relative residual of an exact solution can be far above rounding
  // when S is ill-conditioned), or when a sweep no longer halves eta.
  const double tol = h->opt.tol > 0 ? h->opt.tol : 1e-14;
  const int max_sweeps = h->opt.max_sweeps > 0 ? h->opt.max_sweeps : 8;
  c.info = st_solve_info{};
  c.info.status = ST_OK;
  bool& done = adjoint ? c.adj_solved : c.solved;
  if (fn == 0.0) {
    done = true;
    return ST_OK;
  }
  double rel = 1.0, eta = 1.0, eta_prev = 1e300;
  const double* Rin = io.rhs;
  for (int sw = 0; sw < max_sweeps; ++sw) {
    int iters = 0;
    if (c.itol != nullptr) {
      const InnerTol& r = c.itol_rule;
      launch_set_scalar(c.itol, (sw > 0 && r.adaptive) ? next_inner_tol(r.base, tol, eta, r.amp) : r.base, c.cs);
    }
    if (c.method == 1) {
      s = sweep_space_eig(h, c, io, Rin);
    } else if (c.inner64) {
      s = sweep_time_eig<double>(h, c, io, Rin, iters);
    } else {
      s = sweep_time_eig<float>(h, c, io, Rin, iters);
    }
    if (s != ST_OK) {
      c.info.status = s;
      return s;
    }
    c.info.sweeps = sw + 1;
    PROF(h, c.cs, KC_RESIDUAL64, (int64_t)(c.nx), 7.0 * (double)n * 8.0 + (double)c.sl->geo.ncells * 8.0,
         (double)n * (4.0 * ipow3(c.sl->geo.d) + 20.0),
         launch_residual(c.sl->geo, c.sl->sc, c.sl->c2d, io.sol, io.rhs, io.Ab, io.Bb, c.KU, c.MU, c.Rv, c.nt,
                         c.cs));
    double rn = 0.0, un = 0.0;
    if ((s = read_norm2(h, c, c.Rv, io.sol, (int64_t)n, rn, un)) != ST_OK) return s;
    c.info.max_inner_iters = std::max(c.info.max_inner_iters, iters);
    rel = rn / fn;
    eta = rn / (c.Snorm * un + fn);
    if (!std::isfinite(rel)) {
      c.info.status = ST_ERR_NUMERIC;
      return cfail(c, ST_ERR_NUMERIC, "non-finite residual");
    }
    if (eta <= tol || eta > 0.5 * eta_prev) break;
    eta_prev = eta;
    Rin = c.Rv;
  }
  c.info.rel_residual = rel;
  c.info.backward_error = eta;
  done = true;
  if (eta > 1e3 * tol && eta > 1e-12) {
    c.info.status = ST_ERR_NOT_CONVERGED;
    return cfail(c, ST_ERR_NOT_CONVERGED, "refinement did not reach the backward-error target");
  }
  return ST_OK;
}

// ------------------------------------------------- solves as one graph
// Adds a WHILE node with condition handle hnd after the work captured so far
// on stream s and returns its (empty) body graph.
cudaError_t capture_add_while(cudaStream_t s, cudaGraphConditionalHandle hnd, cudaGraph_t* body) {
  cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(s, &cst, nullptr, &g, &deps, nullptr, &nd);
  if (e != cudaSuccess) return e;
  if (cst != cudaStreamCaptureStatusActive || g == nullptr) return cudaErrorIllegalState;
  const std::vector<cudaGraphNode_t> dv(deps, deps + nd);
  cudaGraphNodeParams cp{};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = hnd;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node = nullptr;
  e = cudaGraphAddNode(&node, g, dv.empty() ? nullptr : dv.data(), nullptr, dv.size(), &cp);
  if (e != cudaSuccess) return e;
  *body = cp.conditional.phGraph_out[0];
  return cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
}

// Every kernel node of g at stream priority prio (kernels in conditional
// bodies are launched by the device, not through the component's stream).
cudaError_t set_kernel_priority(cudaGraph_t g, int prio) {
  size_t n = 0;
  cudaError_t e = cudaGraphGetNodes(g, nullptr, &n);
  if (e != cudaSuccess || n == 0) return e;
  std::vector<cudaGraphNode_t> nodes(n);
  if ((e = cudaGraphGetNodes(g, nodes.data(), &n)) != cudaSuccess) return e;
  for (cudaGraphNode_t nd : nodes) {
    cudaGraphNodeType t;
    if ((e = cudaGraphNodeGetType(nd, &t)) != cudaSuccess) return e;
    if (t != cudaGraphNodeTypeKernel) continue;
    cudaKernelNodeAttrValue v{};
    v.priority = prio;
    if ((e = cudaGraphKernelNodeSetAttribute(nd, cudaLaunchAttributePriority, &v)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// The forward solve of a component as one CUDA graph, captured on its stream:
//   U = 0, R = F, ||F||^2, condition (k_refine_init);
//   WHILE (condition) {                       -- one refinement sweep
//     time eigenbasis: G = W R; COCG start; WHILE (any mode active)
//       { device_loop COCG iterations; condition }; U += Re(V X)
//     (direct components: the banded solve; space eigenbasis: its sweep)
//     R = F - S U; ||R||^2, ||U||^2; stopping test (k_refine_decide) }
// The same kernels as the host-driven loop, in the same order; the host reads
// the record (sweeps, backward error, status) once per call.
template <typename R> st_status capture_solve_graph(st_handle* h, Component& c) {
  const SolveIO io = forward_io(c);
  const int64_t n = c.nx * (int64_t)c.nt;
  const double tol = h->opt.tol > 0 ? h->opt.tol : 1e-14;
  const int max_sweeps = h->opt.max_sweeps > 0 ? h->opt.max_sweeps : 8;
  const bool iterative = c.method == 0 && !c.direct;
  if (c.method == 1 && time_band_smem(c.nt) > kTimeBandMaxSmem)
    return fail(h, ST_ERR_ARG, "device solve: time band solve of this size not supported");
  c.rec = h->alloc<RefineRec>(1);
  c.fn2 = h->alloc<double>(1);
  ST_NEED(h, c.rec);
  ST_NEED(h, c.fn2);
  ST_CUDA(h, cudaMallocHost(&c.rec_h, sizeof(RefineRec)));
  int prio_lo = 0, prio_hi = 0;
  ST_CUDA(h, cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi));
  cudaGraph_t g = nullptr, sweep = nullptr, inner = nullptr;
  ST_CUDA(h, cudaGraphCreate(&g, 0));
  std::string where;
  cudaError_t e = cudaSuccess;
  auto ok = [&](cudaError_t r, const char* what) {
    if (r != cudaSuccess && e == cudaSuccess) {
      e = r;
      where = what;
    }
    return e == cudaSuccess;
  };
  const cudaStreamCaptureMode mode = cudaStreamCaptureModeThreadLocal;
  cudaGraphConditionalHandle hs{}, hi{};
  // prologue
  int64_t l0 = kernel_launch_count();
  if (ok(cudaGraphConditionalHandleCreate(&hs, g, 0, cudaGraphCondAssignDefault), "sweep condition") &&
      ok(cudaStreamBeginCaptureToGraph(c.cs, g, nullptr, nullptr, 0, mode), "prologue capture")) {
    cudaMemsetAsync(io.sol, 0, (size_t)n * sizeof(double), c.cs);
    cudaMemcpyAsync(c.Rv, io.rhs, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, c.cs);
    launch_norm2(io.rhs, n, c.cpart, c.fn2, c.cs);
    launch_refine_init(c.rec, c.fn2, hs, c.itol_rule, c.cs);
    ok(capture_add_while(c.cs, hs, &sweep), "sweep node");
    cudaGraph_t out = nullptr;
    ok(cudaStreamEndCapture(c.cs, &out), "prologue capture end");
  }
  c.gs_pro_nodes = kernel_launch_count() - l0;
  // one sweep
  l0 = kernel_launch_count();
  if (e == cudaSuccess && ok(cudaStreamBeginCaptureToGraph(c.cs, sweep, nullptr, nullptr, 0, mode), "sweep capture")) {
    if (c.method == 1) {
      launch_gemm_right(c.Rv, c.Phi, c.KU, c.nt, c.nx, 0, 0, c.cs);
      launch_time_band_solve(io.lu_ab, io.lu_piv, c.KU, c.nt, c.nx, c.kl, c.ku, c.cs);
      launch_gemm_right(c.KU, c.PhiT, io.sol, c.nt, c.nx, 1, 1, c.cs);
    } else {
      Work<R>& w = work_of<R>(c);
      launch_fwd_transform<R>(io.Wf, c.Rv, w.G, c.nsel, c.nt, c.nx, c.cs);
      if (c.direct) {
        band_solve<R>(c, w.G, w.X, nullptr, c.nx, c.cs);
      } else {
        c.nactive = c.nsel;
        cocg_start<R>(h, c);
        if (ok(cudaGraphConditionalHandleCreate(&hi, sweep, 0, cudaGraphCondAssignDefault), "inner condition")) {
          launch_cocg_continue(c.scal, c.nsel, hi, nullptr, c.cs);
          ok(capture_add_while(c.cs, hi, &inner), "inner node");
        }
      }
      launch_back_transform<R>(io.Vb, c.td->wq, w.X, io.sol, c.nsel, c.nt, c.nx, c.cs);
    }
    launch_residual(c.sl->geo, c.sl->sc, c.sl->c2d, io.sol, io.rhs, io.Ab, io.Bb, c.KU, c.MU, c.Rv, c.nt, c.cs);
    launch_norm2(c.Rv, n, c.cpart, c.cscalar, c.cs);
    launch_norm2(io.sol, n, c.cpart, c.cscalar + 1, c.cs);
    launch_refine_decide(c.rec, c.cscalar, c.fn2, c.Snorm, tol, max_sweeps, iterative ? c.scal : nullptr, c.nsel,
                         c.cerr, hs, c.itol_rule, c.cs);
    cudaGraph_t out = nullptr;
    ok(cudaStreamEndCapture(c.cs, &out), "sweep capture end");
  }
  c.gs_sweep_nodes = kernel_launch_count() - l0;
  // the COCG loop body
  l0 = kernel_launch_count();
  if (e == cudaSuccess && iterative &&
      ok(cudaStreamBeginCaptureToGraph(c.cs, inner, nullptr, nullptr, 0, mode), "inner capture")) {
    for (int k = 0; k < h->opt.device_loop; ++k) cocg_iteration<R>(h, c);
    launch_cocg_continue(c.scal, c.nsel, hi, &c.rec->inner_bodies, c.cs);
    cudaGraph_t out = nullptr;
    ok(cudaStreamEndCapture(c.cs, &out), "inner capture end");
  }
  c.gs_inner_nodes = iterative ? kernel_launch_count() - l0 : 0;
  if (e == cudaSuccess) ok(cudaGetLastError(), "captured launches");
  if (e == cudaSuccess) ok(set_kernel_priority(g, prio_hi), "priority");
  if (e == cudaSuccess) ok(set_kernel_priority(sweep, prio_hi), "priority");
  if (e == cudaSuccess && inner != nullptr) ok(set_kernel_priority(inner, prio_hi), "priority");
  cudaGraphExec_t ge = nullptr;
  if (e == cudaSuccess) ok(cudaGraphInstantiate(&ge, g, 0), "instantiation");
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(h, ST_ERR_CUDA, "solve graph (" + where + "): " + cudaGetErrorString(e));
  }
  c.g_solve = ge;
  return ST_OK;
}

// Enqueues a component's forward solve as its graph, then the copy of its record.
st_status enqueue_graph_solve(st_handle* h, Component& c) {
  st_status s = assemble_rhs(h, c);
  if (s != ST_OK) return s;
  c.info = st_solve_info{};
  c.info.status = ST_OK;
  ST_CUDAC(c, cudaGraphLaunch(c.g_solve, c.cs));
  ST_CUDAC(c, cudaMemcpyAsync(c.rec_h, c.rec, sizeof(RefineRec), cudaMemcpyDeviceToHost, c.cs));
  c.d2h += (int64_t)sizeof(RefineRec);
  note_launches((int)c.gs_pro_nodes);
  c.rec_pending = true;
  return ccheck(c, "solve graph");
}

// Status of a graph solve, once the host has synchronised with an event that
// follows the record's copy: the same outcomes as the host-driven loop.
st_status finish_graph_solve(st_handle* h, Component& c) {
  if (!c.rec_pending) return ST_OK;
  c.rec_pending = false;
  const RefineRec r = *c.rec_h;
  note_launches((int)(r.sweeps * c.gs_sweep_nodes + r.inner_bodies * c.gs_inner_nodes));
  c.info.sweeps = r.sweeps;
  c.info.max_inner_iters = r.max_iters;
  c.info.rel_residual = r.rel;
  c.info.backward_error = r.eta;
  const double tol = h->opt.tol > 0 ? h->opt.tol : 1e-14;
  st_status st = ST_OK;
  if (r.status == RR_TIMEOUT) st = cfail(c, ST_ERR_TIMEOUT, "a bounded copy wait in the banded solve timed out");
  else if (r.status == RR_ITER_LIMIT) st = cfail(c, ST_ERR_NOT_CONVERGED, "COCG reached its iteration limit");
  else if (r.status != RR_OK) st = cfail(c, ST_ERR_NUMERIC, "COCG breakdown or non-finite value");
  c.solved = r.status == RR_OK;
  if (st == ST_OK && r.sweeps > 0 && r.eta > 1e3 * tol && r.eta > 1e-12)
    st = cfail(c, ST_ERR_NOT_CONVERGED, "refinement did not reach the backward-error target");
  c.info.status = st;
  return st;
}

bool graph_solves(const st_handle* h) { return h->opt.device_loop > 0 && !h->prof_on; }

// Execution context of a component: stream, completion event, reduction
// scratch, and its workspace prepared for the handle's precision.
st_status setup_context(st_handle* h, Component& c) {
  // the solves run at the highest stream priority: when a step's solves
  // overlap the previous step's combination levels (st_solve_combine), their
  // CTAs are placed first as the level kernels' CTAs drain
  int prio_lo = 0, prio_hi = 0;
  ST_CUDA(h, cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi));
  ST_CUDA(h, cudaStreamCreateWithPriority(&c.cs, cudaStreamNonBlocking, prio_hi));
  ST_CUDA(h, cudaEventCreateWithFlags(&c.done, cudaEventDisableTiming));
  c.cpart = h->alloc<double>(304);
  c.cscalar = h->alloc<double>(2);
  c.cerr = h->alloc<int>(1);
  ST_NEED(h, c.cpart);
  ST_NEED(h, c.cscalar);
  ST_NEED(h, c.cerr);
  ST_CUDA(h, cudaMemsetAsync(c.cerr, 0, sizeof(int), h->stream));
  ST_CUDA(h, cudaMallocHost(&c.cscalar_h, 2 * sizeof(double)));
  if (c.method == 0) {
    st_status s = c.inner64 ? prepare_work<double>(h, c) : prepare_work<float>(h, c);
    if (s != ST_OK) return s;
    if (!c.direct) {
      // the inner tolerance of the sweeps: FP64 inner solves tighten only as
      // far as the next sweep needs (next_inner_tol); FP32 ones, limited by
      // the FP32 representation of the correction, keep their tolerance
      c.itol = h->alloc<double>(1);
      ST_NEED(h, c.itol);
      const double base = inner_tol(h, c.inner64 ? 8 : 4);
      c.itol_rule = InnerTol{c.itol, base, std::max(10.0, 10.0 * c.td->eig.cond_est),
                             (c.inner64 && h->opt.inner_tol <= 0.0) ? 1 : 0};
      launch_set_scalar(c.itol, base, c.cs);
      if (h->opt.autotune >= 0) {
        s = c.inner64 ? tune_component<double>(h, c) : tune_component<float>(h, c);
        if (s != ST_OK) return s;
      }
      s = c.inner64 ? capture_graphs<double>(h, c) : capture_graphs<float>(h, c);
      if (s != ST_OK) return s;
    }
  }
  if (h->opt.device_loop > 0)
    return (c.method == 0 && !c.inner64) ? capture_solve_graph<float>(h, c) : capture_solve_graph<double>(h, c);
  return ST_OK;
}

// Waits (one host synchronisation) until every listed component's stream has
// passed its completion event, then reads the records of their graph solves.
st_status join_graph_solves(st_handle* h, const std::vector<Component*>& cs, std::vector<st_status>& st) {
  if (h->join == nullptr) ST_CUDA(h, cudaStreamCreateWithFlags(&h->join, cudaStreamNonBlocking));
  for (Component* c : cs) {
    ST_CUDA(h, cudaEventRecord(c->done, c->cs));
    ST_CUDA(h, cudaStreamWaitEvent(h->join, c->done, 0));
  }
  ST_CUDA(h, cudaStreamSynchronize(h->join));
  for (size_t i = 0; i < cs.size(); ++i) {
    const st_status r = finish_graph_solve(h, *cs[i]);
    if (st[i] == ST_OK) st[i] = r;
  }
  return ST_OK;
}

// Receiver tables: per component, the cell of each receiver at the
// component's level (corner indices and multilinear weights) and the
// component's B-spline values at the target times.  Rebuilt only when the
// receivers or the target time level change.
st_status build_receivers(st_handle* h, int jt_star, const double* x, int nrec) {
  const st_problem& p = h->prob;
  const int d = p.d, nc = 1 << d, ncomp = (int)h->comps.size(), nts = (1 << jt_star) + 1;
  st_handle::RecTables& R = h->rec;
  std::vector<double> xv(x, x + (size_t)nrec * d);
  if (R.jt == jt_star && R.nrec == nrec && R.x == xv) return ST_OK;
  for (int r = 0; r < nrec; ++r)
    for (int k = 0; k < d; ++k) {
      const double v = xv[(size_t)r * d + k];
      if (!(v >= p.lo[k] && v <= p.hi[k])) return fail(h, ST_ERR_ARG, "receiver outside the domain");
    }
  std::vector<CombComp> cc(ncomp);
  std::vector<RecCorner> rc((size_t)ncomp * nrec * nc);
  std::vector<double> tb((size_t)ncomp * nts * 3);
  std::vector<int> sp((size_t)ncomp * nts);
  int64_t max_nx = 1;
  int max_nt = 1;
  for (int c = 0; c < ncomp; ++c) {
    const Component& k = *h->comps[c];
    cc[c] = CombComp{k.U, k.sl->lift, k.jx, k.jt, k.coef, 0};
    max_nx = std::max(max_nx, k.nx);
    max_nt = std::max(max_nt, k.nt);
    const int N = 1 << k.jx, n = N - 1;
    for (int r = 0; r < nrec; ++r) {
      int cell[3] = {0, 0, 0};
      double f[3] = {0, 0, 0};
      for (int q = 0; q < d; ++q) {
        const double t = (xv[(size_t)r * d + q] - p.lo[q]) / ((p.hi[q] - p.lo[q]) / N);
        cell[q] = std::min(std::max((int)std::floor(t), 0), N - 1);
        f[q] = t - cell[q];
      }
      for (int e = 0; e < nc; ++e) {
        double w = 1.0;
        int64_t all = 0, in = 0, sa = 1, si = 1;
        bool interior = true;
        for (int q = 0; q < d; ++q) {
          const int b = (e >> q) & 1, P = cell[q] + b;
          w *= b ? f[q] : 1.0 - f[q];
          all += (int64_t)P * sa;
          sa *= (N + 1);
          interior = interior && P >= 1 && P <= n;
          in += (int64_t)(P - 1) * si;
          si *= n;
        }
        rc[((size_t)c * nrec + r) * nc + e] = RecCorner{interior ? (int)in : -1, (int)all, w};
      }
    }
    const int Nt = 1 << k.jt;
    for (int s = 0; s < nts; ++s) {
      int span = (k.jt >= jt_star) ? (s << (k.jt - jt_star)) : (s >> (jt_star - k.jt));
      span = std::min(span, Nt - 1);
      double v[3], d1[3], d2[3];
      bspline_local(Nt, p.T, span, p.T * (double)s / (double)(1 << jt_star), v, d1, d2);
      for (int a = 0; a < 3; ++a) tb[((size_t)c * nts + s) * 3 + a] = v[a];
      sp[(size_t)c * nts + s] = span;
    }
  }
  R.comps = h->upload(cc);
  R.rc = h->upload(rc);
  R.tb = h->upload(tb);
  R.span = h->upload(sp);
  R.vals = h->alloc<double>((size_t)nts * nrec);
  R.wm = h->alloc<double>((size_t)nts * nrec);
  R.J = h->alloc<double>(1);
  R.ehat = h->alloc<double>((size_t)max_nt * nrec);
  R.gv = h->alloc<double>((size_t)max_nx);
  if (!R.comps || !R.rc || !R.tb || !R.span || !R.vals || !R.wm || !R.J || !R.ehat || !R.gv)
    return fail(h, ST_ERR_OOM, "device allocation failed");
  R.jt = jt_star;
  R.nrec = nrec;
  R.ncorner = nc;
  R.nts = nts;
  R.x = xv;
  return ST_OK;
}

// Q1 element stiffness with unit coefficient on a cell of widths h (local
// corner c: bit k set at the upper end in direction k): the sum over
// directions of the 1D stiffness in that direction times the 1D masses in the others.
ElemK element_stiffness(int d, const double* h) {
  ElemK ke{};
  const int nc = 1 << d;
  for (int a = 0; a < nc; ++a)
    for (int b = 0; b < nc; ++b) {
      double sum = 0.0;
      for (int k = 0; k < d; ++k) {
        double term = 1.0;
        for (int l = 0; l < d; ++l) {
          const int ba = (a >> l) & 1, bb = (b >> l) & 1;
          term *= (l == k) ? (ba == bb ? 1.0 : -1.0) / h[l] : h[l] / 6.0 * (ba == bb ? 2.0 : 1.0);
        }
        sum += term;
      }
      ke.k[a * nc + b] = sum;
    }
  return ke;
}

// Q1 element mass on a cell of widths h: the tensor product of the 1D masses h/6 [[2,1],[1,2]].
ElemK element_mass(int d, const double* h) {
  ElemK me{};
  const int nc = 1 << d;
  for (int a = 0; a < nc; ++a)
    for (int b = 0; b < nc; ++b) {
      double m = 1.0;
      for (int l = 0; l < d; ++l) m *= h[l] / 6.0 * ((((a >> l) & 1) == ((b >> l) & 1)) ? 2.0 : 1.0);
      me.k[a * nc + b] = m;
    }
  return me;
}

// Combination tables for a target level pair and a component set (bit mask):
// components sorted by their combination level min(jx, jx*), B-spline values
// of every component at every target time, partial-sum buffers per level.
// Built once per (target, set) and cached on the handle.
st_status comb_tables(st_handle* h, int jx_star, int jt_star, uint64_t mask, const st_handle::CombTables** out) {
  const st_problem& p = h->prob;
  const int nts = (1 << jt_star) + 1;
  auto key = std::make_tuple(jx_star, jt_star, mask);
  auto it = h->comb.find(key);
  if (it != h->comb.end()) {
    *out = &it->second;
    return ST_OK;
  }
  std::vector<int> order;
  for (int c = 0; c < (int)h->comps.size(); ++c)
    if (mask & (1ull << c)) order.push_back(c);
  const int nc = (int)order.size();
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return std::min(h->comps[a]->jx, jx_star) < std::min(h->comps[b]->jx, jx_star);
  });
  std::vector<CombComp> cc(nc);
  std::vector<double> tb((size_t)nc * nts * 3);
  std::vector<int> tsp((size_t)nc * nts);
  st_handle::CombTables t;
  t.order = order;
  t.jmin = jx_star;
  for (int o = 0; o < nc; ++o) {
    const Component& k = *h->comps[order[o]];
    cc[o] = CombComp{k.U, k.sl->lift, k.jx, k.jt, k.coef, 0};
    const int lev = std::min(k.jx, jx_star);
    t.jmin = std::min(t.jmin, lev);
    const int Nt = 1 << k.jt;
    for (int s = 0; s < nts; ++s) {
      int span = (k.jt >= jt_star) ? (s << (k.jt - jt_star)) : (s >> (jt_star - k.jt));
      span = std::min(span, Nt - 1);
      const double tt = p.T * (double)s / (double)(1 << jt_star);
      double v[3], d1[3], d2[3];
      bspline_local(Nt, p.T, span, tt, v, d1, d2);
      for (int a = 0; a < 3; ++a) tb[((size_t)o * nts + s) * 3 + a] = v[a];
      tsp[(size_t)o * nts + s] = span;
    }
  }
  t.first.assign(jx_star + 2, nc);
  for (int o = nc - 1; o >= 0; --o) {
    const int lev = std::min(cc[o].jx, jx_star);
    t.first[lev] = o;
  }
  for (int lev = jx_star; lev >= 0; --lev) t.first[lev] = std::min(t.first[lev], t.first[lev + 1]);
  // The B-spline weights at the target times are dyadic rationals (target
  // times and knots are both multiples of T / 2^max(jt, jt*)); with at most
  // 24 significant bits they are exact floats, and the levels run in
  // double-single arithmetic.  Otherwise (time levels more than 11 apart)
  // every level runs in FP64.
  std::vector<float> tbw(tb.size());
  t.ds_ok = true;
  for (size_t i = 0; i < tb.size(); ++i) {
    tbw[i] = (float)tb[i];
    if (std::fabs((double)tbw[i] - tb[i]) > 4e-16) t.ds_ok = false;
  }
  t.jt.resize(nc);
  for (int o = 0; o < nc; ++o) t.jt[o] = cc[o].jt;
  // pair arrays of every component (kept on the component, filled per step)
  std::vector<CombCompDS> dc[2];
  dc[0].resize(nc);
  dc[1].resize(nc);
  if (t.ds_ok)
    for (int o = 0; o < nc; ++o) {
      Component& k = *h->comps[order[o]];
      if (k.Uds[0] == nullptr) {
        k.Uds[0] = h->alloc<ds>((size_t)k.nt * k.nx);
        k.Uds[1] = h->alloc<ds>((size_t)k.nt * k.nx);
        if (k.sl->lift != nullptr) k.Lds = h->alloc<ds>((size_t)k.sl->nall);
        if (k.Uds[0] == nullptr || k.Uds[1] == nullptr || (k.sl->lift != nullptr && k.Lds == nullptr))
          return fail(h, ST_ERR_OOM, "device allocation failed");
        if (k.Lds != nullptr)
          launch_comb_prep_ds(p.d, nullptr, k.sl->lift, k.coef, k.jx, k.nt, nullptr, k.Lds, h->stream);
      }
      for (int b = 0; b < 2; ++b) dc[b][o] = CombCompDS{k.Uds[b], k.Lds, k.jx, k.jt};
    }
  t.comps = h->alloc<CombComp>(nc);
  t.tb = h->alloc<double>(tb.size());
  t.tbw = h->alloc<float>(tbw.size());
  t.dcomps[0] = h->alloc<CombCompDS>(nc);
  t.dcomps[1] = h->alloc<CombCompDS>(nc);
  t.span = h->alloc<int>(tsp.size());
  if (!t.comps || !t.tb || !t.tbw || !t.dcomps[0] || !t.dcomps[1] || !t.span)
    return fail(h, ST_ERR_OOM, "device allocation failed");
  t.Y.assign(jx_star + 1, nullptr);
  for (int lev = t.jmin; lev < jx_star; ++lev) {
    int64_t nsp = 1;
    for (int k = 0; k < p.d; ++k) nsp *= ((1 << lev) + 1);
    t.Y[lev] = h->alloc<double>((size_t)nsp * nts);
    if (!t.Y[lev]) return fail(h, ST_ERR_OOM, "device allocation failed");
  }
  ST_CUDA(h, cudaMemcpyAsync(t.comps, cc.data(), nc * sizeof(CombComp), cudaMemcpyHostToDevice, h->stream));
  ST_CUDA(h, cudaMemcpyAsync(t.tb, tb.data(), tb.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  ST_CUDA(h, cudaMemcpyAsync(t.tbw, tbw.data(), tbw.size() * sizeof(float), cudaMemcpyHostToDevice, h->stream));
  for (int b = 0; b < 2; ++b)
    ST_CUDA(h, cudaMemcpyAsync(t.dcomps[b], dc[b].data(), nc * sizeof(CombCompDS), cudaMemcpyHostToDevice, h->stream));
  ST_CUDA(h, cudaMemcpyAsync(t.span, tsp.data(), tsp.size() * sizeof(int), cudaMemcpyHostToDevice, h->stream));
  ST_CUDA(h, cudaStreamSynchronize(h->stream));
  *out = &(h->comb[key] = t);
  return ST_OK;
}

// One level of the hierarchical combination on the handle's stream.
// buf: the pair buffer the level reads; prepped: the components' pairs were
// already written into it on their own streams (st_solve_combine), otherwise
// they are converted here on the handle's stream.
void enqueue_comb_level(st_handle* h, const st_handle::CombTables& t, int lev, int jx_star, int jt_star,
                        double* out_dev, int buf = 0, bool prepped = false) {
  const st_problem& p = h->prob;
  const int nts = (1 << jt_star) + 1;
  const int c0 = t.first[lev], c1 = t.first[lev + 1];
  const double* Yp = lev > t.jmin ? t.Y[lev - 1] : nullptr;
  double* Y = lev == jx_star ? out_dev : t.Y[lev];
  int64_t nsp = 1;
  for (int k = 0; k < p.d; ++k) nsp *= ((1 << lev) + 1);
  const double outb = (double)nsp * nts * 8.0, inb = Yp ? outb / (1 << p.d) : 0.0;
  // algorithmic flops per target value: the prolongation's add and three
  // multiply-adds per component
  const double flops = (double)nsp * nts * ((Yp ? 1.0 : 0.0) + 6.0 * (c1 - c0));
  if (t.ds_ok) {
    // this level's components as pairs (sign applied, u0 folded in), then the level
    if (!prepped)
      for (int o = c0; o < c1; ++o) {
        const Component& k = *h->comps[t.order[o]];
        launch_comb_prep_ds(p.d, k.U, k.sl->lift, k.coef, k.jx, k.nt, k.Uds[buf], nullptr, h->stream);
      }
    const int L = comb_ds_chunk(p.d, lev, jt_star, t.jt.data() + c0, c1 - c0);
    PROF(h, h->stream, KC_COMBINE, (int64_t)(nsp), outb + inb, flops,
         launch_comb_level_ds(p.d, lev, Yp, t.dcomps[buf], c0, c1, t.tbw, t.span, nts, L, Y, lev == jx_star,
                              h->stream));
  } else {
    PROF(h, h->stream, KC_COMBINE, (int64_t)(nsp), outb + inb, flops,
         launch_comb_level(p.d, lev, Yp, t.comps, c0, c1, t.tb, t.span, nts, Y, h->stream));
  }
}

// Forward (S U = F) or adjoint (S^T L = G) solves of components k0..k1-1.
// Component streams start after the work already queued on the handle's
// stream; independent components run concurrently, one host thread and one
// stream each (one after the other with profiling on, so that event times are
// not shared between overlapping kernels); the handle's stream then waits for
// all of them.
st_status run_solves(st_handle* h, int k0, int k1, bool adjoint, st_solve_info* info) {
  ST_CUDA(h, cudaEventRecord(h->entry_ev, h->stream));
  std::vector<st_status> st(k1 - k0, ST_OK);
  for (int i = k0; i < k1; ++i) {
    Component& c = *h->comps[i];
    c.err.clear();
    ST_CUDA(h, cudaStreamWaitEvent(c.cs, h->entry_ev, 0));
  }
  auto run = [&](int i) {
    Component& c = *h->comps[i];
    st[i - k0] = solve_one(h, c, adjoint ? adjoint_io(c) : forward_io(c), adjoint);
  };
  // graph solves: every component enqueued from this thread, one wait for all
  const bool graphs = !adjoint && graph_solves(h);
  if (k1 - k0 > 1 && !h->prof_on && !graphs) {
    std::vector<std::thread> pool;
    pool.reserve(k1 - k0);
    for (int i = k0; i < k1; ++i) pool.emplace_back(run, i);
    for (auto& t : pool) t.join();
  } else {
    for (int i = k0; i < k1; ++i) run(i);
  }
  if (graphs) {
    std::vector<Component*> cs;
    for (int i = k0; i < k1; ++i) cs.push_back(h->comps[i].get());
    st_status js = join_graph_solves(h, cs, st);
    if (js != ST_OK) return js;
  }
  st_status worst = ST_OK;
  st_solve_info agg{};
  for (int i = k0; i < k1; ++i) {
    Component& c = *h->comps[i];
    ST_CUDA(h, cudaEventRecord(c.done, c.cs));
    ST_CUDA(h, cudaStreamWaitEvent(h->stream, c.done, 0));
    const st_solve_info& ci = c.info;
    agg.sweeps = std::max(agg.sweeps, ci.sweeps);
    agg.max_inner_iters = std::max(agg.max_inner_iters, ci.max_inner_iters);
    agg.rel_residual = std::max(agg.rel_residual, ci.rel_residual);
    agg.backward_error = std::max(agg.backward_error, ci.backward_error);
    if (st[i - k0] != ST_OK && worst == ST_OK) {
      worst = st[i - k0];
      h->err = "component " + std::to_string(i) + ": " + c.err;
    }
  }
  agg.status = worst;
  if (info) {
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return fail(h, ST_ERR_CUDA, "stream synchronisation failed");
    *info = agg;
  }
  return worst;
}

// Host-side phase times of st_setup, printed to stderr when the environment
// variable ST_SETUP_TRACE is set (diagnostics only).
struct SetupTrace {
  bool on = std::getenv("ST_SETUP_TRACE") != nullptr;
  std::chrono::steady_clock::time_point t = std::chrono::steady_clock::now();
  std::map<std::string, double> acc;
  void mark(const char* phase) {
    if (!on) return;
    const auto now = std::chrono::steady_clock::now();
    acc[phase] += std::chrono::duration<double, std::milli>(now - t).count();
    t = now;
  }
  ~SetupTrace() {
    if (!on) return;
    for (const auto& kv : acc) std::fprintf(stderr, "st_setup %-28s %9.2f ms\n", kv.first.c_str(), kv.second);
  }
};

// Timeline of one st_solve_combine call on stderr (ms after entry: the end of
// every component's solve, the start and end of every combination level)
// when the environment variable ST_STEP_TRACE is set (diagnostics only).
struct StepTrace {
  bool on = std::getenv("ST_STEP_TRACE") != nullptr;
  cudaEvent_t t0 = nullptr;
  std::vector<cudaEvent_t> ev;
  std::vector<std::string> what;
  cudaEvent_t make(const std::string& name) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    ev.push_back(e);
    what.push_back(name);
    return e;
  }
  void report(cudaStream_t s) {
    if (!on || t0 == nullptr) return;
    cudaStreamSynchronize(s);
    for (size_t i = 0; i < ev.size(); ++i) {
      float ms = -1.0f;
      if (ev[i] != nullptr && cudaEventElapsedTime(&ms, t0, ev[i]) != cudaSuccess) ms = -1.0f;
      std::fprintf(stderr, "st_step %-34s %9.3f ms\n", what[i].c_str(), ms);
    }
  }
  ~StepTrace() {
    for (cudaEvent_t e : ev)
      if (e != nullptr) cudaEventDestroy(e);
    if (t0 != nullptr) cudaEventDestroy(t0);
  }
};

}  // namespace

// ====================================================================== ABI
extern "C" {

st_status st_setup(const st_problem* problem, const st_options* options, st_handle** out) {
  Phase phase_("st_setup");
  if (out == nullptr || problem == nullptr) return fail(nullptr, ST_ERR_ARG, "null argument");
  *out = nullptr;
  SetupTrace trace;
  const st_problem& p = *problem;
  if (p.d < 1 || p.d > 3) return fail(nullptr, ST_ERR_ARG, "d must be 1, 2 or 3");
  if (!(p.T > 0.0) || !std::isfinite(p.T)) return fail(nullptr, ST_ERR_ARG, "T must be positive");
  for (int k = 0; k < p.d; ++k)
    if (!(p.hi[k] > p.lo[k])) return fail(nullptr, ST_ERR_ARG, "empty box");
  if (p.J < 0 || p.mx < 1 || p.mt < 0) return fail(nullptr, ST_ERR_ARG, "levels: need J >= 0, mx >= 1, mt >= 0");
  if (p.c2.fn == nullptr && p.c2_nodal == nullptr) return fail(nullptr, ST_ERR_ARG, "c^2 callback or nodal values required");
  if ((p.c2_nodal != nullptr || p.g_nodal != nullptr) && (p.param_level < 0 || p.param_level > 12))
    return fail(nullptr, ST_ERR_ARG, "param_level must be 0..12");
  if (p.g_nodal != nullptr && p.n_terms < 1) return fail(nullptr, ST_ERR_ARG, "g_nodal needs a source term");
  if (p.n_terms < 0 || (p.n_terms > 0 && p.terms == nullptr)) return fail(nullptr, ST_ERR_ARG, "bad source terms");
  const int jx_max = p.mx + p.J, jt_max = p.mt + p.J;
  const int cap = p.d == 1 ? 20 : (p.d == 2 ? 13 : 9);
  if (jx_max > cap || jt_max > 14) return fail(nullptr, ST_ERR_ARG, "level too large for this build");
  auto h = std::make_unique<st_handle>();
  h->prob = p;
  if (options) h->opt = *options;
  if (p.c2_nodal != nullptr || p.g_nodal != nullptr) {
    int64_t np = 1;
    for (int k = 0; k < p.d; ++k) np *= (1 << p.param_level) + 1;
    if (p.c2_nodal != nullptr) h->c2_nodal.assign(p.c2_nodal, p.c2_nodal + np);
    if (p.g_nodal != nullptr) h->g_nodal.assign(p.g_nodal, p.g_nodal + np);
  }
  h->prob.c2_nodal = nullptr;  // the copies above are used from here on
  h->prob.g_nodal = nullptr;
  if (h->opt.precision != ST_FP64 && h->opt.precision != ST_FP32_IR)
    return fail(nullptr, ST_ERR_ARG, "unknown precision");
  if (!(h->opt.inner_tol >= 0.0 && h->opt.inner_tol < 1.0) || !(h->opt.tol >= 0.0 && h->opt.tol < 1.0))
    return fail(nullptr, ST_ERR_ARG, "tolerances must lie in [0, 1)");
  if (h->opt.max_direct_rows < 0) return fail(nullptr, ST_ERR_ARG, "max_direct_rows must be >= 0");
  if (h->opt.autotune < -1 || h->opt.autotune > 1) return fail(nullptr, ST_ERR_ARG, "autotune must be -1, 0 or 1");
  if (h->opt.mem_cap_bytes < 0 || h->opt.wait_cycles < 0 || h->opt.inject_stall < 0 || h->opt.inject_stall > 1)
    return fail(nullptr, ST_ERR_ARG, "mem_cap_bytes and wait_cycles must be >= 0, inject_stall 0 or 1");
  if (h->opt.device_loop != 0 && h->opt.device_loop != 4 && h->opt.device_loop != 8 && h->opt.device_loop != 16)
    return fail(nullptr, ST_ERR_ARG, "device_loop must be 0, 4, 8 or 16");
  h->stream = static_cast<cudaStream_t>(h->opt.stream);
  h->nterm_rows = p.n_terms + 2;
  h->launches0 = kernel_launch_count();
  st_handle* hp = h.get();
  trace.mark("validation");
  hp->part = hp->alloc<double>(304);
  hp->scalar = hp->alloc<double>(1);
  hp->dev_err = hp->alloc<int>(1);
  hp->solve_err = hp->alloc<int>(1);
  if (!hp->part || !hp->scalar || !hp->dev_err || !hp->solve_err) {
    g_create_error = "device allocation failed";
    return ST_ERR_OOM;
  }
  if (cudaMemsetAsync(hp->solve_err, 0, sizeof(int), hp->stream) != cudaSuccess) {
    g_create_error = "cudaMemset failed";
    return ST_ERR_CUDA;
  }
  if (cudaEventCreateWithFlags(&hp->entry_ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&hp->sc_done_ev[0], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&hp->sc_done_ev[1], cudaEventDisableTiming) != cudaSuccess) {
    g_create_error = "event creation failed";
    return ST_ERR_CUDA;
  }
  if (cudaMallocHost(&hp->scalar_h, sizeof(double)) != cudaSuccess) {
    g_create_error = "pinned allocation failed";
    return ST_ERR_CUDA;
  }
  // Components of Eq. (19)
  std::vector<std::tuple<int, int, int>> cl;
  {
    std::vector<int> lst(3 * (2 * p.J + 1));
    st_host_components(p.J, p.mx, p.mt, lst.data());
    for (int k = 0; k < 2 * p.J + 1; ++k) cl.emplace_back(lst[3 * k], lst[3 * k + 1], lst[3 * k + 2]);
  }
  for (auto& t : cl) {
    const int jx = std::get<0>(t), jt = std::get<1>(t);
    if (!hp->space.count(jx)) {
      auto sl = std::make_unique<SpaceLevel>();
      st_status s = setup_space_level(hp, jx, *sl);
      if (s != ST_OK) {
        g_create_error = hp->err;
        return s;
      }
      hp->space[jx] = std::move(sl);
      trace.mark("space levels");
    }
    const int nt = (1 << jt) + 1;
    const int64_t nx = make_geo(p.d, jx).nnodes;
    const bool space_eig = nt > kModeTMaxNt && nx <= kModeSMaxNx;
    if (!hp->time.count(jt)) {
      auto td = std::make_unique<TimeData>();
      st_status s = setup_time_level(hp, jt, *td);
      if (s != ST_OK) {
        g_create_error = hp->err;
        return s;
      }
      hp->time[jt] = std::move(td);
      trace.mark("time levels");
    }
    TimeData& td = *hp->time[jt];
    if (!space_eig && !td.have_eig) {
      if (!time_eig(td.tl, td.eig)) {
        g_create_error = "eigen-decomposition of the time matrices failed";
        return ST_ERR_NUMERIC;
      }
      td.have_eig = true;
      // upload
      const int ns = td.eig.nsel, ntt = td.tl.nt;
      std::vector<cx<double>> Wc((size_t)ns * ntt), Vc((size_t)ntt * ns), lc(ns);
      std::vector<cx<float>> lf(ns);
      for (size_t e = 0; e < Wc.size(); ++e) Wc[e] = mk(td.eig.W[e].real(), td.eig.W[e].imag());
      for (size_t e = 0; e < Vc.size(); ++e) Vc[e] = mk(td.eig.V[e].real(), td.eig.V[e].imag());
      for (int q = 0; q < ns; ++q) {
        lc[q] = mk(td.eig.lam[q].real(), td.eig.lam[q].imag());
        lf[q] = mk((float)td.eig.lam[q].real(), (float)td.eig.lam[q].imag());
      }
      td.W = hp->upload(Wc);
      td.V = hp->upload(Vc);
      // (B^-1 A)^T-side pencil of the adjoint: A^T = V^-T Lam V^T B^T, so its
      // modes are reached by V^T and left by W^T = B^-T V^-T
      std::vector<cx<double>> VTc((size_t)ns * ntt), WTc((size_t)ntt * ns);
      for (int q = 0; q < ns; ++q)
        for (int j = 0; j < ntt; ++j) {
          VTc[(size_t)q * ntt + j] = Vc[(size_t)j * ns + q];
          WTc[(size_t)j * ns + q] = Wc[(size_t)q * ntt + j];
        }
      td.VT = hp->upload(VTc);
      td.WT = hp->upload(WTc);
      if (!td.VT || !td.WT) {
        g_create_error = "device allocation failed";
        return ST_ERR_OOM;
      }
      td.lam64 = hp->upload(lc);
      td.lam32 = hp->upload(lf);
      td.wq = hp->upload(td.eig.weight);
      if (!td.W || !td.V || !td.lam64 || !td.lam32 || !td.wq) {
        g_create_error = "device allocation failed";
        return ST_ERR_OOM;
      }
      trace.mark("time eigenbasis");
    }
    auto c = std::make_unique<Component>();
    c->jx = jx;
    c->jt = jt;
    c->coef = std::get<2>(t);
    c->method = space_eig ? 1 : 0;
    c->sl = hp->space[jx].get();
    c->td = &td;
    st_status s = setup_component(hp, *c);
    trace.mark("component data");
    if (s == ST_OK) s = setup_context(hp, *c);
    trace.mark("component context");
    if (s != ST_OK) {
      g_create_error = hp->err;
      hp->comps.push_back(std::move(c));  // released with the handle
      return s;
    }
    hp->comps.push_back(std::move(c));
  }
  if (cudaStreamSynchronize(hp->stream) != cudaSuccess) {
    g_create_error = "stream synchronisation failed during setup";
    return ST_ERR_CUDA;
  }
  trace.mark("handle stream sync");
  // the factorisations enqueued on the component streams: wait, then read
  // their zero-pivot flags and clear them for the solves
  for (auto& c : hp->comps) {
    if (c->cs == nullptr || c->cerr == nullptr) continue;
    int herr = 0;
    if (cudaMemcpyAsync(&herr, c->cerr, sizeof(int), cudaMemcpyDeviceToHost, c->cs) != cudaSuccess ||
        cudaStreamSynchronize(c->cs) != cudaSuccess) {
      g_create_error = "stream synchronisation failed during setup";
      return ST_ERR_CUDA;
    }
    if (herr != 0) {
      g_create_error = "zero pivot in a banded LDL^T factorisation";
      return ST_ERR_NUMERIC;
    }
  }
  trace.mark("component stream sync");
  *out = h.release();
  return ST_OK;
}

st_status st_num_components(const st_handle* h, int* n) {
  if (!h || !n) return ST_ERR_ARG;
  *n = (int)h->comps.size();
  return ST_OK;
}

st_status st_component(const st_handle* h, int k, st_component_info* info) {
  if (!h || !info || k < 0 || k >= (int)h->comps.size()) return ST_ERR_ARG;
  const Component& c = *h->comps[k];
  info->jx = c.jx;
  info->jt = c.jt;
  info->coef = c.coef;
  info->n_space = c.nx;
  info->n_time = c.nt;
  info->method = c.method;
  info->n_modes = c.method == 1 ? (int)c.nx : c.nsel;
  return ST_OK;
}

st_status st_solve_component(st_handle* h, int k, st_solve_info* info) {
  Phase phase_("st_solve_component");
  if (!h) return ST_ERR_ARG;
  ++h->api_seq;
  if (k < -1 || k >= (int)h->comps.size()) return fail(h, ST_ERR_ARG, "component index out of range");
  const int k0 = k < 0 ? 0 : k, k1 = k < 0 ? (int)h->comps.size() : k + 1;
  return run_solves(h, k0, k1, false, info);
}

st_status st_solve_batch(st_handle* const* hs, int n, int max_threads, st_solve_info* info) {
  Phase phase_("st_solve_batch");
  if (!hs || n < 1 || max_threads < 0) return ST_ERR_ARG;
  for (int i = 0; i < n; ++i) {
    if (!hs[i]) return ST_ERR_ARG;
    for (int j = 0; j < i; ++j)
      if (hs[j] == hs[i]) return fail(hs[i], ST_ERR_ARG, "a handle is listed twice");
  }
  // every (handle, component) pair, largest first, over a bounded pool of host threads
  struct Task {
    st_handle* h;
    int k;
    int64_t cost;
  };
  std::vector<Task> tasks;
  for (int i = 0; i < n; ++i) {
    st_handle* h = hs[i];
    ST_CUDA(h, cudaEventRecord(h->entry_ev, h->stream));
    ++h->api_seq;
    for (int k = 0; k < (int)h->comps.size(); ++k) {
      Component& c = *h->comps[k];
      c.err.clear();
      ST_CUDA(h, cudaStreamWaitEvent(c.cs, h->entry_ev, 0));
      tasks.push_back(Task{h, k, c.nx * c.nt});
    }
  }
  std::stable_sort(tasks.begin(), tasks.end(), [](const Task& a, const Task& b) { return a.cost > b.cost; });
  std::vector<st_status> st(tasks.size(), ST_OK);
  bool graphs = true;
  for (int i = 0; i < n; ++i) graphs = graphs && graph_solves(hs[i]);
  if (graphs) {
    // every component's solve is one graph: all enqueued from this thread,
    // largest first, then one host synchronisation for the whole batch
    std::vector<Component*> cs;
    for (size_t t = 0; t < tasks.size(); ++t) {
      Component& c = *tasks[t].h->comps[tasks[t].k];
      st[t] = solve_one(tasks[t].h, c, forward_io(c), false);
      cs.push_back(&c);
    }
    st_status js = join_graph_solves(hs[0], cs, st);
    if (js != ST_OK) return js;
  } else {
    std::atomic<size_t> next{0};
    auto worker = [&]() {
      for (size_t t = next.fetch_add(1); t < tasks.size(); t = next.fetch_add(1)) {
        Component& c = *tasks[t].h->comps[tasks[t].k];
        st[t] = solve_one(tasks[t].h, c, forward_io(c), false);
      }
    };
    const int nth = (int)std::min<size_t>(tasks.size(), max_threads > 0 ? (size_t)max_threads : (size_t)32);
    std::vector<std::thread> pool;
    for (int i = 0; i < nth; ++i) pool.emplace_back(worker);
    for (auto& th : pool) th.join();
  }
  st_status worst = ST_OK;
  st_solve_info agg{};
  for (size_t t = 0; t < tasks.size(); ++t) {
    st_handle* h = tasks[t].h;
    Component& c = *h->comps[tasks[t].k];
    ST_CUDA(h, cudaEventRecord(c.done, c.cs));
    ST_CUDA(h, cudaStreamWaitEvent(h->stream, c.done, 0));
    agg.sweeps = std::max(agg.sweeps, c.info.sweeps);
    agg.max_inner_iters = std::max(agg.max_inner_iters, c.info.max_inner_iters);
    agg.rel_residual = std::max(agg.rel_residual, c.info.rel_residual);
    agg.backward_error = std::max(agg.backward_error, c.info.backward_error);
    if (st[t] != ST_OK && worst == ST_OK) {
      worst = st[t];
      h->err = "component " + std::to_string(tasks[t].k) + ": " + c.err;
    }
  }
  agg.status = worst;
  if (info) {
    for (int i = 0; i < n; ++i)
      if (cudaStreamSynchronize(hs[i]->stream) != cudaSuccess)
        return fail(hs[i], ST_ERR_CUDA, "stream synchronisation failed");
    *info = agg;
  }
  return worst;
}

st_status st_combine(st_handle* h, int jx_star, int jt_star, double* out_dev) {
  if (!h || !out_dev) return ST_ERR_ARG;
  std::vector<int> all(h->comps.size());
  for (size_t k = 0; k < all.size(); ++k) all[k] = (int)k;
  return st_combine_subset(h, jx_star, jt_star, all.data(), (int)all.size(), out_dev);
}

st_status st_combine_subset(st_handle* h, int jx_star, int jt_star, const int* comps, int ncomp, double* out_dev) {
  Phase phase_("st_combine");
  if (!h || !out_dev || !comps || ncomp < 1) return ST_ERR_ARG;
  ++h->api_seq;
  if (jx_star < 1 || jt_star < 0 || jx_star > 14 || jt_star > 14) return fail(h, ST_ERR_ARG, "bad target level");
  if (h->comps.size() > 64) return fail(h, ST_ERR_ARG, "more than 64 components");
  uint64_t mask = 0;
  for (int i = 0; i < ncomp; ++i) {
    const int k = comps[i];
    if (k < 0 || k >= (int)h->comps.size()) return fail(h, ST_ERR_ARG, "component index out of range");
    if (mask & (1ull << k)) return fail(h, ST_ERR_ARG, "component listed twice");
    mask |= 1ull << k;
    if (!h->comps[k]->solved) return fail(h, ST_ERR_STATE, "combine before every listed component is solved");
  }
  const st_handle::CombTables* t = nullptr;
  st_status s = comb_tables(h, jx_star, jt_star, mask, &t);
  if (s != ST_OK) return s;
  for (int lev = t->jmin; lev <= jx_star; ++lev) enqueue_comb_level(h, *t, lev, jx_star, jt_star, out_dev);
  return check_launch(h, "combine");
}

st_status st_solve_combine(st_handle* h, int jx_star, int jt_star, double* out_dev, st_solve_info* info) {
  Phase phase_("st_solve_combine");
  if (!h || !out_dev) return ST_ERR_ARG;
  ++h->api_seq;
  if (jx_star < 1 || jt_star < 0 || jx_star > 14 || jt_star > 14) return fail(h, ST_ERR_ARG, "bad target level");
  if (h->comps.size() > 64) return fail(h, ST_ERR_ARG, "more than 64 components");
  const int nc = (int)h->comps.size();
  const uint64_t mask = nc == 64 ? ~0ull : ((1ull << nc) - 1);
  const st_handle::CombTables* t = nullptr;
  // a call that directly follows another st_solve_combine on this handle (no
  // other call in between that enqueues work on its stream) may start its
  // solves while the previous call's combination levels still run
  const bool chained = h->sc_seq >= 0 && h->api_seq == h->sc_seq + 1;
  st_status s = comb_tables(h, jx_star, jt_star, mask, &t);
  if (s != ST_OK) return s;
  h->sc_seq = -1;  // set again once this call has enqueued everything
  const bool overlap = t->ds_ok;
  const int buf = h->sc_parity;
  // every component on its own stream and host thread; each records its
  // completion event and reports; the combination levels are enqueued on the
  // handle's stream level by level, each as soon as the components it adds
  // have finished (a level also follows the previous one on that stream).
  // The levels read pair copies of the components (buffer `buf`), written on
  // the component's stream right after its solve: so the next call's solves
  // may overwrite the components while these levels run, and only the call
  // after that, which reuses buffer `buf`, waits for them.
  if (overlap && chained) {
    for (auto& c : h->comps) {
      c->err.clear();
      if (h->sc_done_rec[buf]) ST_CUDA(h, cudaStreamWaitEvent(c->cs, h->sc_done_ev[buf], 0));
    }
  } else {
    ST_CUDA(h, cudaEventRecord(h->entry_ev, h->stream));
    for (auto& c : h->comps) {
      c->err.clear();
      ST_CUDA(h, cudaStreamWaitEvent(c->cs, h->entry_ev, 0));
    }
  }
  StepTrace trace;
  std::vector<cudaEvent_t> comp_ev(nc, nullptr);
  if (trace.on && cudaEventCreate(&trace.t0) == cudaSuccess) {
    cudaEventRecord(trace.t0, h->stream);
    for (int i = 0; i < nc; ++i)
      comp_ev[i] = trace.make("component (" + std::to_string(h->comps[i]->jx) + "," +
                              std::to_string(h->comps[i]->jt) + ") solved");
  }
  std::vector<st_status> st(nc, ST_OK);
  std::vector<char> done(nc, 0);
  std::mutex mu;
  std::condition_variable cv;
  auto run = [&](int i) {
    Component& c = *h->comps[i];
    st_status r = solve_one(h, c, forward_io(c), false);
    if (r == ST_OK && overlap) {
      launch_comb_prep_ds(h->prob.d, c.U, c.sl->lift, c.coef, c.jx, c.nt, c.Uds[buf], nullptr, c.cs);
      r = ccheck(c, "combination pairs");
    }
    if (r == ST_OK && cudaEventRecord(c.done, c.cs) != cudaSuccess) r = cfail(c, ST_ERR_CUDA, "event record failed");
    if (comp_ev[i] != nullptr) cudaEventRecord(comp_ev[i], c.cs);
    {
      std::lock_guard<std::mutex> lock(mu);
      st[i] = r;
      done[i] = 1;
    }
    cv.notify_all();
  };
  // graph solves are enqueued inline (they return at once); host-driven
  // solves run on a thread each, except when profiling
  const bool graphs = graph_solves(h);
  std::vector<std::thread> pool;
  if (graphs) {
    // largest first: the finest components are the step's critical path
    std::vector<int> byc(nc);
    for (int i = 0; i < nc; ++i) byc[i] = i;
    std::stable_sort(byc.begin(), byc.end(), [&](int a, int b) {
      return h->comps[a]->nx * h->comps[a]->nt > h->comps[b]->nx * h->comps[b]->nt;
    });
    for (int i : byc) run(i);
  } else if (!h->prof_on) {
    pool.reserve(nc);
    for (int i = 0; i < nc; ++i) pool.emplace_back(run, i);
  }
  bool failed = false;
  for (int lev = t->jmin; lev <= jx_star; ++lev) {
    const int c0 = t->first[lev], c1 = t->first[lev + 1];
    for (int o = c0; o < c1 && !failed; ++o) {
      const int k = t->order[o];
      if (graphs) {
        // enqueued above
      } else if (h->prof_on) {
        run(k);
      } else {
        std::unique_lock<std::mutex> lock(mu);
        cv.wait(lock, [&] { return done[k] != 0; });
      }
      if (st[k] != ST_OK) failed = true;
      else if (cudaStreamWaitEvent(h->stream, h->comps[k]->done, 0) != cudaSuccess) failed = true;
    }
    if (failed) break;
    cudaEvent_t lb = trace.t0 ? trace.make("level " + std::to_string(lev) + " combination start") : nullptr;
    if (lb != nullptr) cudaEventRecord(lb, h->stream);
    enqueue_comb_level(h, *t, lev, jx_star, jt_star, out_dev, buf, overlap);
    cudaEvent_t le = trace.t0 ? trace.make("level " + std::to_string(lev) + " combination end") : nullptr;
    if (le != nullptr) cudaEventRecord(le, h->stream);
  }
  for (auto& th : pool) th.join();
  if (graphs) {
    // one host synchronisation: the solves' records (the levels may still run)
    std::vector<Component*> cs;
    std::vector<st_status> gst;
    std::vector<int> idx;
    for (int i = 0; i < nc; ++i)
      if (done[i] && h->comps[i]->rec_pending) {
        cs.push_back(h->comps[i].get());
        gst.push_back(st[i]);
        idx.push_back(i);
      }
    st_status js = join_graph_solves(h, cs, gst);
    if (js != ST_OK) return js;
    for (size_t j = 0; j < idx.size(); ++j) st[idx[j]] = gst[j];
  }
  st_status worst = ST_OK;
  st_solve_info agg{};
  for (int i = 0; i < nc; ++i) {
    Component& c = *h->comps[i];
    if (!done[i]) continue;  // not started (profiling run stopped at an earlier failure)
    if (st[i] == ST_OK) {
      ST_CUDA(h, cudaEventRecord(c.done, c.cs));
      ST_CUDA(h, cudaStreamWaitEvent(h->stream, c.done, 0));
    }
    agg.sweeps = std::max(agg.sweeps, c.info.sweeps);
    agg.max_inner_iters = std::max(agg.max_inner_iters, c.info.max_inner_iters);
    agg.rel_residual = std::max(agg.rel_residual, c.info.rel_residual);
    agg.backward_error = std::max(agg.backward_error, c.info.backward_error);
    if (st[i] != ST_OK && worst == ST_OK) {
      worst = st[i];
      h->err = "component " + std::to_string(i) + ": " + c.err;
    }
  }
  agg.status = worst;
  if (worst == ST_OK && failed) worst = fail(h, ST_ERR_CUDA, "stream wait failed");
  if (worst == ST_OK && overlap) {
    ST_CUDA(h, cudaEventRecord(h->sc_done_ev[buf], h->stream));
    h->sc_done_rec[buf] = true;
    h->sc_parity ^= 1;
    h->sc_seq = h->api_seq;
  }
  trace.report(h->stream);
  if (info) {
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return fail(h, ST_ERR_CUDA, "stream synchronisation failed");
    *info = agg;
  }
  if (worst != ST_OK) return worst;
  return check_launch(h, "solve and combine");
}

st_status st_receiver_values(st_handle* h, int jt_star, const double* x_rec, int n_rec, double* out_dev) {
  Phase phase_("st_receiver_values");
  if (!h || !x_rec || !out_dev || n_rec < 1) return ST_ERR_ARG;
  ++h->api_seq;
  if (jt_star < 0 || jt_star > 14) return fail(h, ST_ERR_ARG, "bad target time level");
  for (auto& c : h->comps)
    if (!c->solved) return fail(h, ST_ERR_STATE, "receiver values before every component is solved");
  st_status s = build_receivers(h, jt_star, x_rec, n_rec);
  if (s != ST_OK) return s;
  const st_handle::RecTables& R = h->rec;
  launch_receiver_eval(R.comps, (int)h->comps.size(), R.rc, n_rec, R.ncorner, R.tb, R.span, R.nts, out_dev, h->stream);
  return check_launch(h, "receiver values");
}

st_status st_misfit_gradient(st_handle* h, int jt_star, const double* x_rec, int n_rec, const double* d_obs_dev,
                             int jp, double* J_out, double* dc2_dev, double* dg_dev, st_solve_info* info) {
  Phase phase_("st_misfit_gradient");
  if (!h || !x_rec || !d_obs_dev || n_rec < 1 || !J_out || !dc2_dev || !dg_dev) return ST_ERR_ARG;
  ++h->api_seq;
  const st_problem& p = h->prob;
  if (jt_star < 0 || jt_star > 14 || jp < 0 || jp > 12) return fail(h, ST_ERR_ARG, "bad level");
  if (p.u0.fn != nullptr) return fail(h, ST_ERR_ARG, "the c^2 gradient is implemented for u0 = 0 only");
  if (h->c2_nodal.empty() || (p.n_terms > 0 && h->g_nodal.empty()))
    return fail(h, ST_ERR_STATE, "the gradient is taken with respect to nodal c^2 and g: set c2_nodal (and g_nodal)");
  if (jp != p.param_level) return fail(h, ST_ERR_ARG, "jp differs from the problem's param_level");
  for (auto& c : h->comps)
    if (!c->solved) return fail(h, ST_ERR_STATE, "gradient before every component is solved");
  st_status s = build_receivers(h, jt_star, x_rec, n_rec);
  if (s != ST_OK) return s;
  const st_handle::RecTables& R = h->rec;
  const int ncomp = (int)h->comps.size();
  launch_receiver_eval(R.comps, ncomp, R.rc, n_rec, R.ncorner, R.tb, R.span, R.nts, R.vals, h->stream);
  launch_misfit(R.vals, d_obs_dev, R.nts, n_rec, p.T, R.wm, R.J, h->stream);
  // adjoint right-hand sides G_k = coef_k E_k^T (w * e)
  for (int c = 0; c < ncomp; ++c) {
    Component& k = *h->comps[c];
    const size_t n = (size_t)k.nt * k.nx;
    if (k.Gadj == nullptr) {
      k.Gadj = h->alloc<double>(n);
      k.Lam = h->alloc<double>(n);
      if (!k.Gadj || !k.Lam) return fail(h, ST_ERR_OOM, "device allocation failed");
    }
    ST_CUDA(h, cudaMemsetAsync(k.Gadj, 0, n * sizeof(double), h->stream));
    launch_adjoint_rhs(R.wm, R.nts, n_rec, R.tb + (size_t)c * R.nts * 3, R.span + (size_t)c * R.nts, k.nt,
                       R.rc + (size_t)c * n_rec * R.ncorner, R.ncorner, (double)k.coef, k.nx, R.ehat, k.Gadj,
                       h->stream);
  }
  if ((s = check_launch(h, "adjoint right-hand sides")) != ST_OK) return s;
  // adjoint solves S_k^T L_k = G_k, all components concurrently
  s = run_solves(h, 0, ncomp, true, info);
  if (s != ST_OK) return s;
  // gradient reductions onto the parameter grid
  ParamGrid pg{};
  pg.d = p.d;
  pg.Np = 1 << jp;
  for (int k = 0; k < 3; ++k) {
    pg.lo[k] = k < p.d ? p.lo[k] : 0.0;
    pg.h[k] = k < p.d ? (p.hi[k] - p.lo[k]) / pg.Np : 1.0;
  }
  int64_t np = 1;
  for (int k = 0; k < p.d; ++k) np *= (pg.Np + 1);
  ST_CUDA(h, cudaMemsetAsync(dc2_dev, 0, np * sizeof(double), h->stream));
  ST_CUDA(h, cudaMemsetAsync(dg_dev, 0, np * sizeof(double), h->stream));
  for (int c = 0; c < ncomp; ++c) {
    Component& k = *h->comps[c];
    const ElemK ke = element_stiffness(p.d, k.sl->h);
    launch_grad_c2(k.sl->geo, pg.lo, k.nt, k.td->Bband, k.U, k.Lam, ke, pg, dc2_dev, h->stream);
    if (p.n_terms >= 1)
      launch_grad_g(k.sl->geo, pg.lo, k.sl->sc, k.nt, k.td->rhs_coef, k.Lam, R.gv, pg, dg_dev, h->stream);
  }
  ST_CUDA(h, cudaMemcpyAsync(h->scalar_h, R.J, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  ST_CUDA(h, cudaStreamSynchronize(h->stream));
  *J_out = *h->scalar_h;
  return check_launch(h, "gradient");
}

st_status st_set_tuned_shape(const int* entry) {
  if (!entry) return ST_ERR_ARG;
  return set_stencil_shape(entry[0], entry[1], entry[2], entry[3], entry[4], entry[5], entry[6]) ? ST_OK
                                                                                                  : ST_ERR_ARG;
}

st_status st_tuned_shapes(int* out, int max_entries, int* n_out) {
  if (!n_out || max_entries < 0) return ST_ERR_ARG;
  *n_out = tuned_stencil_shapes(out, max_entries);
  return ST_OK;
}

st_status st_energy(st_handle* h, const double* times, int ntimes, int jx_eval, double* energy_out) {
  Phase phase_("st_energy");
  if (!h || !times || !energy_out || ntimes < 1) return ST_ERR_ARG;
  ++h->api_seq;
  const st_problem& p = h->prob;
  const int nc = (int)h->comps.size();
  int jmax = 0;
  for (auto& c : h->comps) {
    if (!c->solved) return fail(h, ST_ERR_STATE, "energy before every component is solved");
    jmax = std::max(jmax, c->jx);
  }
  if (jx_eval == 0) jx_eval = jmax;
  if (jx_eval != jmax) return fail(h, ST_ERR_ARG, "jx_eval must be 0 or the finest spatial level of the components");
  for (int i = 0; i < ntimes; ++i)
    if (!(times[i] >= 0.0 && times[i] <= p.T)) return fail(h, ST_ERR_ARG, "times must lie in [0, T]");
  const SpaceLevel& sl = *h->space[jx_eval];
  const int d = p.d, N = 1 << jx_eval;
  int64_t nall = 1, ncell = 1;
  for (int k = 0; k < d; ++k) {
    nall *= N + 1;
    ncell *= N;
  }
  // components in level order; the combination levels evaluate u^CF and d_t u^CF
  // on all nodes of level jx_eval at a batch of times
  std::vector<int> order(nc);
  for (int c = 0; c < nc; ++c) order[c] = c;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return h->comps[a]->jx < h->comps[b]->jx; });
  const int jmin = h->comps[order[0]]->jx;
  std::vector<int> first(jx_eval + 2, nc);
  for (int o = nc - 1; o >= 0; --o) first[h->comps[order[o]]->jx] = o;
  for (int lev = jx_eval; lev >= 0; --lev) first[lev] = std::min(first[lev], first[lev + 1]);
  std::vector<CombComp> cv(nc), cd(nc);
  for (int o = 0; o < nc; ++o) {
    const Component& k = *h->comps[order[o]];
    cv[o] = CombComp{k.U, k.sl->lift, k.jx, k.jt, k.coef, 0};
    cd[o] = CombComp{k.U, nullptr, k.jx, k.jt, k.coef, 0};
  }
  const int64_t budget = (int64_t)256 << 20;  // device bytes for the level arrays of one batch
  const int B = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)ntimes, 256, budget / (nall * 8 * 4)}));
  const unsigned nblk = (unsigned)((ncell + 255) / 256);
  cudaStream_t st = h->stream;
  // call-local device memory, stream-ordered
  std::vector<void*> bufs;
  auto dalloc = [&](size_t bytes) -> void* {
    void* q = nullptr;
    if (cudaMallocAsync(&q, bytes, st) != cudaSuccess) return nullptr;
    bufs.push_back(q);
    return q;
  };
  auto release = [&]() {
    for (void* q : bufs) cudaFreeAsync(q, st);
    bufs.clear();
  };
  CombComp* dcv = (CombComp*)dalloc(sizeof(CombComp) * nc);
  CombComp* dcd = (CombComp*)dalloc(sizeof(CombComp) * nc);
  double* tbv = (double*)dalloc(sizeof(double) * 3 * nc * B);
  double* tbd = (double*)dalloc(sizeof(double) * 3 * nc * B);
  int* tsp = (int*)dalloc(sizeof(int) * nc * B);
  double* part = (double*)dalloc(sizeof(double) * (size_t)nblk * B);
  double* eout = (double*)dalloc(sizeof(double) * ntimes);
  std::vector<double*> Yv(jx_eval + 1, nullptr), Yd(jx_eval + 1, nullptr);
  bool ok = dcv && dcd && tbv && tbd && tsp && part && eout;
  for (int lev = jmin; lev <= jx_eval && ok; ++lev) {
    int64_t nsp = 1;
    for (int k = 0; k < d; ++k) nsp *= (1 << lev) + 1;
    Yv[lev] = (double*)dalloc(sizeof(double) * nsp * B);
    Yd[lev] = (double*)dalloc(sizeof(double) * nsp * B);
    ok = Yv[lev] && Yd[lev];
  }
  if (!ok) {
    cudaGetLastError();
    release();
    return fail(h, ST_ERR_OOM, "device allocation failed");
  }
  ST_CUDA(h, cudaMemcpyAsync(dcv, cv.data(), sizeof(CombComp) * nc, cudaMemcpyHostToDevice, st));
  ST_CUDA(h, cudaMemcpyAsync(dcd, cd.data(), sizeof(CombComp) * nc, cudaMemcpyHostToDevice, st));
  const ElemK me = element_mass(d, sl.h), ke = element_stiffness(d, sl.h);
  std::vector<double> hv((size_t)3 * nc * B), hd((size_t)3 * nc * B);
  std::vector<int> hs((size_t)nc * B);
  for (int t0 = 0; t0 < ntimes; t0 += B) {
    const int nb = std::min(B, ntimes - t0);
    for (int o = 0; o < nc; ++o) {
      const Component& k = *h->comps[order[o]];
      const int Nt = 1 << k.jt;
      for (int b = 0; b < nb; ++b) {
        const double t = times[t0 + b];
        const int span = std::min(Nt - 1, std::max(0, (int)std::floor(t * Nt / p.T)));
        double v[3], d1[3], d2[3];
        bspline_local(Nt, p.T, span, t, v, d1, d2);
        for (int a = 0; a < 3; ++a) {
          hv[((size_t)o * nb + b) * 3 + a] = v[a];
          hd[((size_t)o * nb + b) * 3 + a] = d1[a];
        }
        hs[(size_t)o * nb + b] = span;
      }
    }
    ST_CUDA(h, cudaMemcpyAsync(tbv, hv.data(), sizeof(double) * 3 * nc * nb, cudaMemcpyHostToDevice, st));
    ST_CUDA(h, cudaMemcpyAsync(tbd, hd.data(), sizeof(double) * 3 * nc * nb, cudaMemcpyHostToDevice, st));
    ST_CUDA(h, cudaMemcpyAsync(tsp, hs.data(), sizeof(int) * nc * nb, cudaMemcpyHostToDevice, st));
    for (int lev = jmin; lev <= jx_eval; ++lev) {
      const double* pv = lev > jmin ? Yv[lev - 1] : nullptr;
      const double* pd = lev > jmin ? Yd[lev - 1] : nullptr;
      launch_comb_level(d, lev, pv, dcv, first[lev], first[lev + 1], tbv, tsp, nb, Yv[lev], st);
      launch_comb_level(d, lev, pd, dcd, first[lev], first[lev + 1], tbd, tsp, nb, Yd[lev], st);
    }
    launch_energy_cells(d, N, sl.c2d, Yv[jx_eval], Yd[jx_eval], nall, nb, me, ke, part, eout + t0, st);
    // the host tables are overwritten by the next batch: wait for this batch's copies
    ST_CUDA(h, cudaStreamSynchronize(st));
  }
  ST_CUDA(h, cudaMemcpyAsync(energy_out, eout, sizeof(double) * ntimes, cudaMemcpyDeviceToHost, st));
  release();
  ST_CUDA(h, cudaStreamSynchronize(st));
  h->d2h_bytes += (int64_t)(sizeof(double) * ntimes);
  return check_launch(h, "energy");
}

st_status st_component_coeffs(st_handle* h, int k, double* host_out) {
  if (!h || !host_out || k < 0 || k >= (int)h->comps.size()) return ST_ERR_ARG;
  ++h->api_seq;
  Component& c = *h->comps[k];
  if (!c.solved) return fail(h, ST_ERR_STATE, "component not solved");
  ST_CUDA(h, cudaMemcpyAsync(host_out, c.U, (size_t)c.nx * c.nt * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  ST_CUDA(h, cudaStreamSynchronize(h->stream));
  return ST_OK;
}

st_status st_total_dofs(const st_handle* h, int64_t* dofs) {
  if (!h || !dofs) return ST_ERR_ARG;
  int64_t s = 0;
  for (auto& c : h->comps) s += c->nx * c->nt;
  *dofs = s;
  return ST_OK;
}

st_status st_transfer_bytes(const st_handle* h, int64_t* h2d, int64_t* d2h) {
  if (!h) return ST_ERR_ARG;
  if (h2d) *h2d = h->h2d_bytes;
  if (d2h) {
    int64_t s = h->d2h_bytes;
    for (auto& c : h->comps) s += c->d2h;
    *d2h = s;
  }
  return ST_OK;
}

st_status st_kernel_launches(const st_handle* h, int64_t* count) {
  if (!h || !count) return ST_ERR_ARG;
  *count = kernel_launch_count() - h->launches0;
  return ST_OK;
}

st_status st_profile(st_handle* h, int enable) {
  if (!h) return ST_ERR_ARG;
  ++h->api_seq;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return fail(h, ST_ERR_CUDA, "stream synchronisation failed");
  for (auto& r : h->prof) {
    h->ev_pool.push_back(r.a);
    h->ev_pool.push_back(r.b);
  }
  h->prof.clear();
  h->prof_on = enable != 0;
  return ST_OK;
}

st_status st_profile_read(st_handle* h, st_kernel_stat* out, int max_out, int* n_out) {
  if (!h || !n_out) return ST_ERR_ARG;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return fail(h, ST_ERR_CUDA, "stream synchronisation failed");
  for (auto& c : h->comps)
    if (cudaStreamSynchronize(c->cs) != cudaSuccess) return fail(h, ST_ERR_CUDA, "stream synchronisation failed");
  // one entry per (kernel class, grid size): the class name with "@<unknowns>"
  std::map<std::pair<int, int64_t>, st_kernel_stat> agg;
  for (auto& r : h->prof) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) return fail(h, ST_ERR_CUDA, "event timing failed");
    st_kernel_stat& s = agg[std::make_pair(r.cls, r.size)];
    s.launches += 1;
    s.ms += ms;
    s.bytes += r.bytes;
    s.flops += r.flops;
  }
  int n = 0;
  for (auto& kv : agg) {
    if (out && n < max_out) {
      out[n] = kv.second;
      std::snprintf(out[n].name, sizeof(out[n].name), "%s@%lld", kClassName[kv.first.first],
                    (long long)kv.first.second);
    }
    ++n;
  }
  *n_out = n;
  return ST_OK;
}

st_status st_destroy(st_handle* h) {
  if (!h) return ST_OK;
  if (h->stream) cudaStreamSynchronize(h->stream);
  else cudaDeviceSynchronize();
  delete h;
  return ST_OK;
}

const char* st_last_error(const st_handle* h) {
  if (!h) return g_create_error.c_str();
  return h->err.c_str();
}

}  // extern "C"
