// Host runtime behind the C ABI of include/mgrit_sl.h: level hierarchy, workspace, and the MGRIT
// V-cycle orchestration (Sec. 2.2, 3.4) over the kernels of setup_kernels.cu / relax_kernels.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/mgrit_sl.h"
#include "kernels.h"

using namespace mgrit;

namespace {

thread_local std::string g_last_error;

mgrit_status fail(mgrit_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

#define MG_CUDA(call)                                                                              \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess) return fail(MGRIT_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define MG_TRY(call)                       \
  do {                                     \
    mgrit_status s_ = (call);              \
    if (s_ != MGRIT_OK) return s_;         \
  } while (0)

struct Level {
  int nt = 0;  // steps on this level
  int m = 0;   // coarsening factor from the level above (0 on level 0)
  double* s64 = nullptr;
  double* sigma = nullptr;
  uint16_t* shift = nullptr;
  double* w64 = nullptr;
  float* eps32 = nullptr;
  float* eps_lo = nullptr;  // level 0 of 1D FP32-bulk handles: the FP32 pairs of its FP64 passes
  void* solver = nullptr;   // stored factorisation (FP64 coarse levels)
  float* sig32 = nullptr;   // sigma as FP32 rows (FP32 coarse levels, factorised on the fly)
  float* pcr32 = nullptr;   // FP32 coarse levels, p <= 3: block-PCR coefficients of every step
  unsigned pcr_floats = 0;
  float* band32 = nullptr;  // FP32 coarse levels: the banded separator inverse of every step (probed in setup)
  float* band_ind = nullptr;  // [32] its decay indicators (k_sep_band): 8 colours at 1..4, 16 colours at 17..24
  int band_w = 0;           // half-bandwidth in use (0: block PCR / on the fly), chosen in setup_finish
  float band_decay[4] = {};  // the probed indicator at partition distances 1..4 (host copy)
  size_t solver_stride = 0;
  int P = 0;
  int is_double = 1;  // arithmetic of this level's cycle
  void* E = nullptr;  // coarse levels: unknown, full level array [(nt+1)][npts]
  void* G = nullptr;  // coarse levels: right-hand side, full level array
  // adjoint (built on first use): floor ranges, factorisation of M^T, d s / d a (level 0)
  int2* frange = nullptr;
  void* solverT = nullptr;
  double* ds = nullptr;  // 2D: x block then y block
  int* bstart = nullptr;  // 2D: arrival points grouped by stencil base node (transposed step)
  int* bperm = nullptr;
};

// Device workspace comes from a stream-ordered memory pool per device owned by the library: blocks a
// destroyed handle returns stay cached for the next setup (no cudaMalloc / cudaFree device
// synchronisation per solve).  An allocation that fails trims the pool and is retried once.
cudaMemPool_t workspace_pool() {
  static std::mutex mu;
  static cudaMemPool_t pools[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(mu);
  if (!pools[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    if (cudaMemPoolCreate(&p, &props) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
    pools[dev] = p;
  }
  return pools[dev];
}

// Small pinned host blocks (norm read-back) reused across handles.
std::mutex& pinned_mu() {
  static std::mutex* mu = new std::mutex;
  return *mu;
}
std::vector<double*>& pinned_free() {
  static std::vector<double*>* v = new std::vector<double*>;
  return *v;
}
// Stream-ordered scratch from the library's pool (kept between calls), else the device's default pool.
cudaError_t scratch_alloc(void** p, size_t bytes, cudaStream_t st) {
  cudaMemPool_t pool = workspace_pool();
  if (pool && cudaMallocFromPoolAsync(p, bytes, pool, st) == cudaSuccess) return cudaSuccess;
  cudaGetLastError();
  return cudaMallocAsync(p, bytes, st);
}

double* pinned_take() {
  {
    std::lock_guard<std::mutex> lk(pinned_mu());
    if (!pinned_free().empty()) {
      double* p = pinned_free().back();
      pinned_free().pop_back();
      return p;
    }
  }
  double* p = nullptr;
  if (cudaMallocHost((void**)&p, 8 * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}
void pinned_give(double* p) {
  std::lock_guard<std::mutex> lk(pinned_mu());
  pinned_free().push_back(p);
}

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

}  // namespace

struct mgrit_handle {
  mgrit_grid grid;
  mgrit_wavespeed wave;
  int order = 1;
  mgrit_options opt;
  cudaStream_t stream = nullptr;
  int device = 0;  // CUDA device current at setup (the handle's workspace lives there)
  bool gmres1d = false;  // solve_mode 1 on a 1D handle: coarse levels solve their correction by GMRES
  int npts = 0;
  std::vector<Level> levels;
  std::vector<void*> allocs;
  std::vector<char> pooled;  // allocs[i] came from the workspace pool
  int64_t bytes = 0;
  // level-0 C-point state and scratch
  double* X = nullptr;
  double* Y = nullptr;
  double* r64 = nullptr;   // FP32-bulk: FP64 residual at the C-points
  float* EC = nullptr;     // FP32-bulk: C-relaxed error (= r) in FP32
  double* norm_partial = nullptr;
  double* norm_dev = nullptr;
  double* norm_host = nullptr;  // pinned
  int* flag_dev = nullptr;
  int* err_dev = nullptr;  // set by kernels whose bounded wait gave up
  int trans_mode = 0;      // 1 while the reversed, transposed (adjoint) problem is being solved
  Scratch2d s2d{};         // 2D work buffers (allocated in mgrit_setup)
  bool adjoint_ready = false;
  double setup_ms = 0.0;
  double setup_t0 = 0.0;
  // launch accounting and optional per-phase event timing
  int64_t setup_launches = 0, call_launches = 0;
  int setup_phase_launches[MGRIT_NUM_PHASES] = {};
  double setup_phase_ms[MGRIT_NUM_PHASES] = {};
  int phase_launches[MGRIT_NUM_PHASES] = {};
  double phase_ms[MGRIT_NUM_PHASES] = {};
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, int>> ev_used;  // (phase, index of the start event)
  size_t ev_next = 0;

  ~mgrit_handle() {
    for (size_t i = 0; i < allocs.size(); ++i) {
      if (pooled[i]) cudaFreeAsync(allocs[i], stream);
      else cudaFree(allocs[i]);
    }
    if (norm_host) pinned_give(norm_host);
    for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
  }

  void reset_call_counters() {
    call_launches = 0;
    for (int i = 0; i < MGRIT_NUM_PHASES; ++i) {
      phase_launches[i] = 0;
      phase_ms[i] = 0.0;
    }
    ev_used.clear();
    ev_next = 0;
  }

  // Record a phase boundary; returns the event index or -1 (profiling off / pool exhausted).
  int phase_begin() {
    if (!opt.profile || ev_next + 2 > ev_pool.size()) return -1;
    const int i = (int)ev_next;
    ev_next += 2;
    cudaEventRecord(ev_pool[i], stream);
    return i;
  }
  void phase_end(int phase, int ev, int launches) {
    call_launches += launches;
    phase_launches[phase] += launches;
    if (ev >= 0) {
      cudaEventRecord(ev_pool[ev + 1], stream);
      ev_used.push_back({phase, ev});
    }
  }
  // After a stream synchronisation: accumulate the recorded phase times.
  void collect_phase_times() {
    for (auto& pr : ev_used) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, ev_pool[pr.second], ev_pool[pr.second + 1]) == cudaSuccess)
        phase_ms[pr.first] += ms;
    }
    ev_used.clear();
    ev_next = 0;
  }

  template <typename T>
  mgrit_status alloc(T** p, size_t count) {
    *p = nullptr;
    if (count == 0) return MGRIT_OK;
    void* q = nullptr;
    const size_t nb = count * sizeof(T);
    cudaMemPool_t pool = workspace_pool();
    cudaError_t e = cudaErrorMemoryAllocation;
    if (pool) {
      e = cudaMallocFromPoolAsync(&q, nb, pool, stream);
      if (e != cudaSuccess) {  // give cached blocks back to the device and retry once
        cudaGetLastError();
        cudaStreamSynchronize(stream);
        cudaMemPoolTrimTo(pool, 0);
        e = cudaMallocFromPoolAsync(&q, nb, pool, stream);
      }
    } else {
      e = cudaMalloc(&q, nb);
    }
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(MGRIT_ENOMEM, "device allocation of " + std::to_string(nb) + " bytes failed");
    }
    allocs.push_back(q);
    pooled.push_back(pool ? 1 : 0);
    bytes += (int64_t)(count * sizeof(T));
    *p = (T*)q;
    return MGRIT_OK;
  }

  int J1() const { return levels[0].nt / levels[1].m; }

  LevelTables tables(int l, int is_double) const {
    const Level& L = levels[l];
    LevelTables T{};
    T.nx = grid.nx;
    T.npts = npts;
    T.p = order;
    T.shift = L.shift;
    T.w64 = L.w64;
    T.eps32 = L.eps32;
    T.eps_lo = L.eps_lo;
    T.df = 0;
    T.table_stride = npts;
    T.nt = L.nt;
    // 2D: sigma for the GMRES correction solves, FP32 copy on FP32 levels
    T.solver = (l > 0 && opt.coarse_op == 0)
                   ? ((grid.dim == 2 || gmres1d) ? (!is_double && L.sig32 ? (const void*)L.sig32 : (const void*)L.sigma)
                                                 : L.solver)
                   : nullptr;
    T.solver_stride = L.solver_stride;
    T.s64 = L.s64;
    T.err = err_dev;
    T.otf = 0;
    T.gather_stage = 0;
    T.pcr = nullptr;
    T.pcr_floats = 0;
    T.band = 0;
    T.cf_src = nullptr;
    T.cf_stride = 0;
    T.cf_floats = 0;
    T.trans = 0;
    T.reverse = 0;
    T.frange = L.frange;
    T.bstart = L.bstart;
    T.bperm = L.bperm;
    T.cluster = opt.cluster_coarse;
    T.test_wait = opt.test_wait_cycles;
    if (trans_mode) {
      T.trans = 1;
      T.reverse = 1;
      if (T.solver && grid.dim == 1) T.solver = L.solverT;  // 2D: GMRES with M^T on the same sigma
      return T;
    }
    if (l == 0 && is_double && L.eps_lo) {  // the FP64 passes of level 0 in FP32 pairs (tables from global)
      T.df = 1;
      T.gather_stage = 0;
      return T;
    }
    if (grid.dim == 1 && !is_double) {
      T.gather_stage = 1;  // TMA bulk copies of each step's eps32 / shift rows into shared memory
      if (l > 0 && opt.coarse_op == 0) {  // coarse: factorised on the fly from sigma (also staged)
        T.otf = 1;
        T.solver = L.sig32;
        T.solver_stride = (size_t)grid.nx;
        T.pcr = L.pcr32;  // p <= 3: the block-PCR coefficients precomputed in setup
        T.pcr_floats = L.pcr_floats;
        if (L.band_w > 0) {  // the banded separator inverse, rows -W .. W of the stored record
          const unsigned row = band_row_size(grid.nx, order);
          T.band = L.band_w;
          T.cf_src = L.band32 + (size_t)(kBandMaxHalfWidth - L.band_w) * row;
          T.cf_stride = band_record_size(grid.nx, order);
          T.cf_floats = (unsigned)(2 * L.band_w + 1) * row;
        } else if (L.pcr32) {
          T.cf_src = L.pcr32;
          T.cf_stride = L.pcr_floats;
          T.cf_floats = L.pcr_floats;
        }
      }
    }
    return T;
  }
};

namespace {

mgrit_status check_grid(const mgrit_grid* g, const mgrit_wavespeed* w, int order, int m) {
  if (!g || !w) return fail(MGRIT_EINVAL, "grid and wave must not be NULL");
  if (g->dim != 1 && g->dim != 2) return fail(MGRIT_EINVAL, "dim must be 1 or 2");
  if (g->nx < 16 || (g->nx & (g->nx - 1)) != 0) return fail(MGRIT_EINVAL, "nx must be a power of two >= 16");
  if (g->nt < 2) return fail(MGRIT_EINVAL, "nt must be >= 2");
  if (!(g->xmax > g->xmin)) return fail(MGRIT_EINVAL, "xmax must exceed xmin");
  if (!(g->cfl > 0.0) || !std::isfinite(g->cfl)) return fail(MGRIT_EINVAL, "cfl must be positive and finite");
  if (order != 1 && order != 3 && order != 5) return fail(MGRIT_EINVAL, "order must be 1, 3 or 5");
  if (m < 2) return fail(MGRIT_EINVAL, "m must be >= 2");
  const bool k1 = w->kind >= 0 && w->kind <= 3, k2 = w->kind >= 10 && w->kind <= 12;
  if ((g->dim == 1 && !k1) || (g->dim == 2 && !k2)) return fail(MGRIT_EINVAL, "wave kind does not match dim");
  if (!std::isfinite(w->a) || !std::isfinite(w->k) || !std::isfinite(w->a2))
    return fail(MGRIT_EINVAL, "wave parameters must be finite");
  if (g->dim == 1 && g->nx > 4096) return fail(MGRIT_EUNSUPPORTED, "1D slices are kept on chip: nx <= 4096");
  if (g->dim == 2 && g->nx > 2048) return fail(MGRIT_EUNSUPPORTED, "2D grids: nx <= 2048");
  return MGRIT_OK;
}

// The coarsening factors (level 1, 2, ...), as in the oracle's rule.
std::vector<int> factors(int nt, int m, int m_first, int levels, int max_coarsest) {
  std::vector<int> out;
  int n = nt;
  while (true) {
    if (levels > 0 && (int)out.size() + 1 >= levels) break;
    const int f = (out.empty() && m_first > 0) ? m_first : m;
    if (levels == 0 && n <= max_coarsest) break;
    if (n % f != 0 || n / f < 1) break;
    out.push_back(f);
    n /= f;
  }
  return out;
}

mgrit_status relax(mgrit_handle* h, int l, int is_double, const RelaxArgs& a, int phase) {
  LevelTables T = h->tables(l, is_double);
  const int ev = h->phase_begin();
  if (h->grid.dim == 2 || (h->gmres1d && l > 0)) MG_CUDA(launch_relax_2d(T, a, h->s2d, is_double, h->stream));
  else MG_CUDA(launch_relax_1d(T, a, is_double, h->stream));
  h->phase_end(phase, ev, 1);
  return MGRIT_OK;
}

RelaxArgs args0() {
  RelaxArgs a;
  std::memset(&a, 0, sizeof(a));
  return a;
}

// Coarse cycle on level l >= 1: E_l from right-hand side G_l (both full level arrays).
mgrit_status coarse_cycle(mgrit_handle* h, int l) {
  Level& L = h->levels[l];
  const int np = h->npts;
  const int dbl = L.is_double;
  if (l == (int)h->levels.size() - 1) {  // coarsest: sequential stepping (Sec. 2.2)
    if (h->grid.dim == 1 && dbl && h->opt.cluster_coarse && h->opt.coarse_op == 0 && !h->trans_mode && !h->gmres1d) {
      // FP64: one interval of nt steps through the relaxation pass (FC: F-points stored, the last step
      // is the C-point), which splits the slice over a thread-block cluster
      RelaxArgs a = args0();
      a.m = L.nt;
      a.J = 1;
      a.nsteps = L.nt;
      a.mode = MODE_FC;
      a.start_wb = L.E;
      a.g = L.G;
      a.fstore = L.E;
      a.cout = L.E;
      a.c_stride = (long long)L.nt * np;
      return relax(h, l, dbl, a, MGRIT_PHASE_COARSEST);
    }
    LevelTables T = h->tables(l, dbl);
    const int ev = h->phase_begin();
    if (h->grid.dim == 2 || h->gmres1d)
      MG_CUDA(launch_sequential_2d(T, L.nt, L.G, nullptr, L.E, 1, h->s2d, dbl, h->stream));
    else MG_CUDA(launch_sequential_1d(T, L.nt, L.G, nullptr, L.E, 1, dbl, h->stream));
    h->phase_end(MGRIT_PHASE_COARSEST, ev, 1);
    return MGRIT_OK;
  }
  Level& Lc = h->levels[l + 1];
  const int m = Lc.m, J = L.nt / m;
  const bool fcf = h->opt.relax == 0;
  RelaxArgs a;
  if (fcf) {
    // F- then C-relaxation from a zero initial guess
    a = args0();
    a.m = m;
    a.J = J;
    a.nsteps = m;
    a.mode = MODE_FC;
    a.g = L.G;
    a.cout = L.E;
    a.c_stride = (long long)m * np;
    MG_TRY(relax(h, l, dbl, a, MGRIT_PHASE_COARSE));
  }
  // F-relaxation and the C-point residual -> right-hand side of level l+1 (F-relaxation only: from the
  // zero initial guess, whose C-points stay zero)
  a = args0();
  a.m = m;
  a.J = J;
  a.nsteps = m;
  a.mode = MODE_RES;
  a.start = fcf ? L.E : nullptr;
  a.start_stride = (long long)m * np;
  a.g = L.G;
  a.g_at_c = 1;
  a.cin = fcf ? L.E : nullptr;
  a.c_stride = (long long)m * np;
  a.rout = Lc.G;
  a.r_stride = np;
  MG_TRY(relax(h, l, dbl, a, MGRIT_PHASE_COARSE));
  MG_TRY(coarse_cycle(h, l + 1));
  // correction by injection and post F-relaxation
  a = args0();
  a.m = m;
  a.J = J;
  a.nsteps = m - 1;
  a.mode = MODE_POST;
  a.start = fcf ? L.E : nullptr;
  a.start_stride = (long long)m * np;
  a.corr = Lc.E;
  a.corr_stride = np;
  a.start_wb = L.E;
  a.wb_stride = (long long)m * np;
  a.extra_cta = 1;
  a.g = L.G;
  a.fstore = L.E;
  MG_TRY(relax(h, l, dbl, a, MGRIT_PHASE_COARSE));
  return MGRIT_OK;
}

// Enqueues the residual norm's reduction and its read-back (norm and error flag) into pinned memory.
mgrit_status enqueue_norm(mgrit_handle* h, int J) {
  const int ev = h->phase_begin();
  launch_sum(h->norm_partial, J, h->norm_dev, h->stream);
  h->phase_end(MGRIT_PHASE_MISC, ev, 1);
  MG_CUDA(cudaMemcpyAsync(h->norm_host, h->norm_dev, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  MG_CUDA(cudaMemcpyAsync(h->norm_host + 1, h->err_dev, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  return MGRIT_OK;
}

// Waits for the stream and returns the norm read back by enqueue_norm.
mgrit_status finish_norm(mgrit_handle* h, double* out) {
  MG_CUDA(cudaStreamSynchronize(h->stream));
  int err = 0;
  std::memcpy(&err, h->norm_host + 1, sizeof(int));
  if (err) return fail(MGRIT_ETIMEOUT, "a bounded device wait gave up (TMA staging did not complete)");
  *out = std::sqrt(h->norm_host[0]);
  return MGRIT_OK;
}

// One captured cycle: the executable graph, the phase events it records and the launches it issues.
struct CycleGraph {
  cudaGraphExec_t exec = nullptr;
  std::vector<std::pair<int, int>> ev;
  int launches[MGRIT_NUM_PHASES] = {};
  int64_t total = 0;
  ~CycleGraph() {
    if (exec) cudaGraphExecDestroy(exec);
  }
};

// Runs `body` (which enqueues one cycle on the handle's stream) as a CUDA graph: captured on first use,
// replayed afterwards.  If the capture fails the body runs directly (same kernels) and *graph_ok is
// cleared so later cycles do too.
template <class F>
mgrit_status run_cycle(mgrit_handle* h, CycleGraph& G, bool* graph_ok, F&& body) {
  if (!*graph_ok) return body();
  if (!G.exec) {
    const size_t ev0 = h->ev_used.size();
    int pl0[MGRIT_NUM_PHASES];
    std::memcpy(pl0, h->phase_launches, sizeof(pl0));
    const int64_t cl0 = h->call_launches;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      *graph_ok = false;
      return body();
    }
    const mgrit_status st = body();
    const cudaError_t e = cudaStreamEndCapture(h->stream, &g);
    cudaError_t ei = cudaErrorUnknown;
    if (st == MGRIT_OK && e == cudaSuccess && g) ei = cudaGraphInstantiate(&G.exec, g, 0);
    if (g) cudaGraphDestroy(g);
    // the capture executed nothing: undo its bookkeeping, keep it for the replays
    G.ev.assign(h->ev_used.begin() + ev0, h->ev_used.end());
    h->ev_used.resize(ev0);
    for (int i = 0; i < MGRIT_NUM_PHASES; ++i) {
      G.launches[i] = h->phase_launches[i] - pl0[i];
      h->phase_launches[i] = pl0[i];
    }
    G.total = h->call_launches - cl0;
    h->call_launches = cl0;
    if (st != MGRIT_OK) return st;
    if (e != cudaSuccess || ei != cudaSuccess) {
      cudaGetLastError();
      if (G.exec) cudaGraphExecDestroy(G.exec);
      G.exec = nullptr;
      G.ev.clear();
      *graph_ok = false;
      return body();
    }
  }
  MG_CUDA(cudaGraphLaunch(G.exec, h->stream));
  for (int i = 0; i < MGRIT_NUM_PHASES; ++i) h->phase_launches[i] += G.launches[i];
  h->call_launches += G.total;
  return MGRIT_OK;
}

// After the stream synchronised: add the replayed graph's phase times.
void collect_graph_times(mgrit_handle* h, const CycleGraph& G) {
  for (auto& pr : G.ev) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->ev_pool[pr.second], h->ev_pool[pr.second + 1]) == cudaSuccess)
      h->phase_ms[pr.first] += ms;
  }
}

}  // namespace

extern "C" {

mgrit_status mgrit_default_options(mgrit_options* opt) {
  if (!opt) return fail(MGRIT_EINVAL, "opt is NULL");
  std::memset(opt, 0, sizeof(*opt));
  opt->precision = 0;
  opt->coarse_op = 0;
  opt->norm_mode = 1;
  opt->max_iter = 200;
  opt->rtol = 1e-10;
  opt->max_coarsest = 1;
  opt->m_first = 0;
  opt->coarse_fp64 = 0;
  opt->use_graph = 1;
  opt->profile = 0;
  opt->gmres_maxit = 10;
  opt->gmres_rtol = 1e-2;
  opt->relax = 0;
  opt->cluster_coarse = 1;
  opt->diverge_ratio = 1e3;
  opt->fine_only = 0;
  opt->solve_mode = 0;
  opt->coarse_band = 1;
  opt->test_wait_cycles = 0;
  return MGRIT_OK;
}

// Completes a setup enqueued by setup_impl: waits for the handle's stream, checks for execution errors
// and singular correction matrices (the handle is destroyed and *out cleared on failure), records times.
static mgrit_status setup_finish(mgrit_handle** out) {
  mgrit_handle* h = *out;
  const cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    delete h;
    *out = nullptr;
    return fail(MGRIT_ECUDA, std::string("setup: ") + cudaGetErrorString(e));
  }
  int flag = 0;
  std::memcpy(&flag, h->norm_host + 3, sizeof(int));
  if (flag) {
    delete h;
    *out = nullptr;
    return fail(MGRIT_ESINGULAR, "a correction matrix has a (near) zero pivot");
  }
  // half-bandwidth of each FP32 coarse level's separator inverse: the smallest W beyond which every probed
  // entry is below kBandTolerance of the diagonal blocks, if its record fits the shared memory of the
  // relaxation kernel; else the block PCR (p <= 3) or the on-the-fly factorisation (p = 5).  The 8-colour
  // probe of the setup decides W <= 3 (entries probed to distance 4); levels it rejects, where a band of
  // half-width kBandMaxHalfWidth would still fit, are probed again with 16 colours (W <= 6, entries to 8),
  // all such levels at once before one synchronisation.
  auto fits = [&](size_t l, int w) {
    Level& L = h->levels[l];
    L.band_w = w;
    int buf;
    size_t smem, region;
    relax_smem_need(h->tables((int)l, 0), 0, &buf, &smem, &region);
    L.band_w = 0;
    return smem <= 227 * 1024;
  };
  auto choose = [](const float* ind, int wmax, int tmax) {
    for (int w = 1; w <= wmax; ++w) {
      bool under = true;
      for (int t = w + 1; t <= tmax; ++t) under = under && ind[t] < kBandTolerance;  // NaN fails
      if (under) return w;
    }
    return 0;
  };
  std::vector<int> widths(h->levels.size(), 0);
  std::vector<char> reprobe(h->levels.size(), 0);
  bool any16 = false;
  for (size_t l = 1; l < h->levels.size(); ++l) {
    Level& L = h->levels[l];
    if (!L.band_ind) continue;
    float ind[5] = {};
    if (cudaMemcpy(ind, L.band_ind, sizeof(ind), cudaMemcpyDeviceToHost) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    for (int t = 0; t < 4; ++t) L.band_decay[t] = ind[t + 1];
    int W = choose(ind, 3, 4);
    if (W > 0 && !fits(l, W)) W = 0;
    widths[l] = W;
    if (W == 0 && fits(l, kBandMaxHalfWidth) &&
        launch_sep_band(L.sig32, L.nt, h->grid.nx, h->order, 16, L.band32, L.band_ind + 16, h->stream) ==
            cudaSuccess) {
      reprobe[l] = 1;
      any16 = true;
    }
  }
  if (any16 && cudaStreamSynchronize(h->stream) != cudaSuccess) {
    cudaGetLastError();
    std::fill(reprobe.begin(), reprobe.end(), 0);
  }
  for (size_t l = 1; l < h->levels.size(); ++l) {
    Level& L = h->levels[l];
    if (!L.band_ind) continue;
    int W = widths[l];
    float ind16[9] = {};
    if (reprobe[l] && cudaMemcpy(ind16, L.band_ind + 16, sizeof(ind16), cudaMemcpyDeviceToHost) == cudaSuccess)
      W = choose(ind16, kBandMaxHalfWidth, 8);
    cudaGetLastError();
    L.band_w = W;
    if (W == 0 && L.pcr_floats && !L.pcr32) {  // band rejected: the block-PCR record after all
      mgrit_status st = h->alloc(&L.pcr32, (size_t)L.nt * L.pcr_floats);
      if (st == MGRIT_OK && launch_pcr_coef(L.sig32, L.nt, h->grid.nx, h->order, L.pcr32, h->stream) != cudaSuccess)
        st = fail(MGRIT_ECUDA, "setup: block-PCR coefficients");
      if (st == MGRIT_OK && cudaStreamSynchronize(h->stream) != cudaSuccess)
        st = fail(MGRIT_ECUDA, std::string("setup: ") + cudaGetErrorString(cudaGetLastError()));
      if (st != MGRIT_OK) {
        delete h;
        *out = nullptr;
        return st;
      }
    }
  }
  h->collect_phase_times();
  h->setup_launches = h->call_launches;
  for (int i = 0; i < MGRIT_NUM_PHASES; ++i) {
    h->setup_phase_launches[i] = h->phase_launches[i];
    h->setup_phase_ms[i] = h->phase_ms[i];
  }
  h->reset_call_counters();
  h->setup_ms = now_ms() - h->setup_t0;
  return MGRIT_OK;
}

// The work of mgrit_setup enqueued on the handle's stream; defer = true returns before the stream is
// synchronised (setup_finish completes it), so several problems' setups can overlap.
static mgrit_status setup_impl(const mgrit_grid* grid, const mgrit_wavespeed* wave, int order, int m, int levels,
                               const mgrit_options* opt_in, void* stream, mgrit_handle** out, bool defer) {
  if (!out) return fail(MGRIT_EINVAL, "out is NULL");
  *out = nullptr;
  MG_TRY(check_grid(grid, wave, order, m));
  mgrit_options opt;
  if (opt_in) opt = *opt_in;
  else mgrit_default_options(&opt);
  if (opt.precision != 0 && opt.precision != 1) return fail(MGRIT_EINVAL, "precision must be 0 or 1");
  if (opt.coarse_op != 0 && opt.coarse_op != 1) return fail(MGRIT_EINVAL, "coarse_op must be 0 or 1");
  if (opt.norm_mode != 1) return fail(MGRIT_EUNSUPPORTED, "only norm_mode 1 is implemented on the GPU");
  if (opt.max_iter < 1 || opt.max_iter > 100000) return fail(MGRIT_EINVAL, "max_iter out of range");
  if (!(opt.rtol > 0.0 && opt.rtol < 1.0)) return fail(MGRIT_EINVAL, "rtol must be in (0, 1)");
  if (opt.max_coarsest < 1) return fail(MGRIT_EINVAL, "max_coarsest must be >= 1");
  if (opt.m_first < 0 || opt.m_first == 1) return fail(MGRIT_EINVAL, "m_first must be 0 or >= 2");
  if (opt.coarse_fp64 != 0 && opt.coarse_fp64 != 1) return fail(MGRIT_EINVAL, "coarse_fp64 must be 0 or 1");
  if (opt.coarse_fp64 && opt.precision != 1) return fail(MGRIT_EINVAL, "coarse_fp64 applies to precision 1 only");
  if (opt.gmres_maxit < 1 || opt.gmres_maxit > 10) return fail(MGRIT_EINVAL, "gmres_maxit must be in 1..10");
  if (!(opt.gmres_rtol >= 0.0 && opt.gmres_rtol < 1.0)) return fail(MGRIT_EINVAL, "gmres_rtol must be in [0, 1)");
  if (opt.relax != 0 && opt.relax != 1) return fail(MGRIT_EINVAL, "relax must be 0 (FCF) or 1 (F)");
  if (opt.cluster_coarse < 0 || opt.cluster_coarse > 16 || (opt.cluster_coarse & (opt.cluster_coarse - 1)) != 0)
    return fail(MGRIT_EINVAL, "cluster_coarse must be 0, 1, 2, 4, 8 or 16");
  if (!(opt.diverge_ratio >= 0.0)) return fail(MGRIT_EINVAL, "diverge_ratio must be >= 0");
  if (opt.test_wait_cycles < 0) return fail(MGRIT_EINVAL, "test_wait_cycles must be >= 0");
  if (opt.fine_only != 0 && opt.fine_only != 1) return fail(MGRIT_EINVAL, "fine_only must be 0 or 1");
  if (opt.solve_mode < 0 || opt.solve_mode > 2) return fail(MGRIT_EINVAL, "solve_mode must be 0, 1 or 2");
  if (opt.solve_mode == 2 && grid->dim == 2 && opt.precision == 1 && !opt.coarse_fp64)
    return fail(MGRIT_EUNSUPPORTED, "exact 2D correction solves (solve_mode 2) need FP64 coarse levels");
  if (opt.coarse_band != 0 && opt.coarse_band != 1) return fail(MGRIT_EINVAL, "coarse_band must be 0 or 1");
  if (opt.solve_mode == 1 && grid->dim == 1 && opt.precision == 1 && !opt.coarse_fp64)
    return fail(MGRIT_EUNSUPPORTED, "1D GMRES correction solves (solve_mode 1) need FP64 coarse levels");
  if (opt.fine_only && grid->dim != 1) return fail(MGRIT_EUNSUPPORTED, "fine_only handles are 1D");
  if (levels < 0 || levels == 1) return fail(MGRIT_EINVAL, "levels must be 0 or >= 2");
  std::vector<int> fac = factors(grid->nt, m, opt.m_first, levels, opt.max_coarsest);
  if (fac.empty()) return fail(MGRIT_EINVAL, "nt does not allow a coarse level with this m");
  if (levels > 0 && (int)fac.size() + 1 != levels)
    return fail(MGRIT_EINVAL, "nt is not divisible by the coarsening factors for the requested levels");

  const double t0 = now_ms();
  mgrit_handle* h = new mgrit_handle();
  h->grid = *grid;
  h->wave = *wave;
  h->order = order;
  h->opt = opt;
  h->stream = (cudaStream_t)stream;
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return fail(MGRIT_ECUDA, "cudaGetDevice failed");
  }
  h->npts = grid->dim == 2 ? grid->nx * grid->nx : grid->nx;
  h->gmres1d = grid->dim == 1 && opt.solve_mode == 1 && opt.coarse_op == 0;
  const int nx = grid->nx, np = h->npts, dim = grid->dim;
  const double hgrid = (grid->xmax - grid->xmin) / nx;
  const double dt = grid->cfl * hgrid;
  const int fp32 = opt.precision == 1;
  const int cf64 = fp32 && opt.coarse_fp64;  // FP32 bulk on level 0 only, FP64 coarse cycle

  auto cleanup_fail = [&](mgrit_status s) {
    delete h;
    return s;
  };
  // levels (fine_only: the fine level alone)
  const bool fine_only = opt.fine_only != 0;
  h->levels.resize(fine_only ? 1 : fac.size() + 1);
  h->levels[0].nt = grid->nt;
  for (size_t l = 1; l < h->levels.size(); ++l) {
    h->levels[l].m = fac[l - 1];
    h->levels[l].nt = h->levels[l - 1].nt / fac[l - 1];
  }
  mgrit_status st = MGRIT_OK;
  const int p = order;
  for (size_t l = 0; l < h->levels.size(); ++l) {
    Level& L = h->levels[l];
    const size_t rows = (size_t)L.nt * np * dim;  // 2D: x block then y block
    L.is_double = (fp32 && !(cf64 && l > 0)) ? 0 : 1;
    if ((st = h->alloc(&L.s64, rows)) != MGRIT_OK) return cleanup_fail(st);
    if ((st = h->alloc(&L.shift, rows)) != MGRIT_OK) return cleanup_fail(st);
    // FP64 levels read precomputed weights (2D: per axis); level 0 of a 1D FP32-bulk handle runs its FP64
    // passes in FP32 pairs from eps32 and eps_lo instead (fine_only handles too: their FP64 single steps)
    const bool pairs = l == 0 && fp32 && dim == 1;
    const bool need64 = L.is_double || (l == 0 && !pairs);
    const bool need32 = !L.is_double;
    if (need64 && (st = h->alloc(&L.w64, rows * (p + 1))) != MGRIT_OK) return cleanup_fail(st);
    if (need32 && (st = h->alloc(&L.eps32, rows)) != MGRIT_OK) return cleanup_fail(st);
    if (pairs && (st = h->alloc(&L.eps_lo, rows)) != MGRIT_OK) return cleanup_fail(st);
    if (l > 0) {
      if ((st = h->alloc(&L.sigma, rows)) != MGRIT_OK) return cleanup_fail(st);
      const size_t full = (size_t)(L.nt + 1) * np;
      const size_t esz = L.is_double ? sizeof(double) : sizeof(float);
      if ((st = h->alloc((char**)&L.E, full * esz)) != MGRIT_OK) return cleanup_fail(st);
      if ((st = h->alloc((char**)&L.G, full * esz)) != MGRIT_OK) return cleanup_fail(st);
      if (opt.coarse_op == 0 && dim == 2 && !L.is_double &&
          (st = h->alloc(&L.sig32, rows)) != MGRIT_OK)  // FP32 sigma of the FP32 GMRES solves
        return cleanup_fail(st);
      if (opt.coarse_op == 0 && dim == 1 && !h->gmres1d) {
        L.P = nx / 8;
        if (L.is_double) {
          L.solver_stride = solver_reals(nx, p);
          const size_t tot = L.solver_stride * L.nt * sizeof(double);
          if ((st = h->alloc((char**)&L.solver, tot)) != MGRIT_OK) return cleanup_fail(st);
        } else {
          if ((st = h->alloc(&L.sig32, (size_t)L.nt * nx)) != MGRIT_OK) return cleanup_fail(st);
          const bool probe = opt.coarse_band && nx / 8 >= 16 && nx / 8 <= 512;  // 8-row partitions, a thread each
          if (p <= 3) {  // with a probed band, the PCR record is built only if the band is rejected (setup_finish)
            L.pcr_floats = pcr_record_size(nx, p);
            if (!probe && (st = h->alloc(&L.pcr32, (size_t)L.nt * L.pcr_floats)) != MGRIT_OK) return cleanup_fail(st);
          }
          if (probe) {
            if ((st = h->alloc(&L.band32, (size_t)L.nt * band_record_size(nx, p))) != MGRIT_OK) return cleanup_fail(st);
            if ((st = h->alloc(&L.band_ind, 32)) != MGRIT_OK) return cleanup_fail(st);  // [0, 5) and [16, 25)
          }
        }
      }
    }
  }
  const int J1 = fine_only ? 1 : h->J1();
  if (dim == 2 || h->gmres1d) {  // work buffers of the passes over slices in global memory (2D, 1D GMRES)
    size_t jmax = (size_t)J1, jc = 1;
    for (size_t l = 1; l + 1 < h->levels.size(); ++l)
      jc = std::max(jc, (size_t)(h->levels[l].nt / h->levels[l + 1].m));
    jmax = dim == 2 ? std::max(jmax, jc) : jc;  // 1D: only the coarse passes use these slices
    const size_t rsz = (fp32 && !cf64) ? sizeof(float) : sizeof(double);  // coarse GMRES basis
    h->s2d.kmax = opt.gmres_maxit;
    h->s2d.rtol = opt.gmres_rtol;
    h->s2d.restarts = 1;
    if (opt.solve_mode == 2) {  // exact 2D correction solves: restarted GMRES(10) to 1e-14
      h->s2d.kmax = 10;
      h->s2d.rtol = 1e-14;
      h->s2d.restarts = 100;
    }
    if ((st = h->alloc((char**)&h->s2d.cur, jmax * np * sizeof(double))) != MGRIT_OK) return cleanup_fail(st);
    if ((st = h->alloc((char**)&h->s2d.nxt, jmax * np * sizeof(double))) != MGRIT_OK) return cleanup_fail(st);
    if (opt.coarse_op == 0 &&
        (st = h->alloc((char**)&h->s2d.basis, jc * (h->s2d.kmax + (h->s2d.restarts > 1 ? 2 : 1)) * np * rsz)) !=
            MGRIT_OK)
      return cleanup_fail(st);
    if ((st = h->alloc(&h->s2d.partial, jmax * 64)) != MGRIT_OK) return cleanup_fail(st);
  }
  if ((st = h->alloc(&h->X, (size_t)(J1 + 1) * np)) != MGRIT_OK) return cleanup_fail(st);
  if ((st = h->alloc(&h->Y, (size_t)(J1 + 1) * np)) != MGRIT_OK) return cleanup_fail(st);
  if (fp32) {
    if ((st = h->alloc(&h->r64, (size_t)(J1 + 1) * np)) != MGRIT_OK) return cleanup_fail(st);
    if ((st = h->alloc(&h->EC, (size_t)(J1 + 1) * np)) != MGRIT_OK) return cleanup_fail(st);
  }
  if ((st = h->alloc(&h->norm_partial, (size_t)J1 + 1)) != MGRIT_OK) return cleanup_fail(st);
  if ((st = h->alloc(&h->norm_dev, 2)) != MGRIT_OK) return cleanup_fail(st);
  if ((st = h->alloc(&h->flag_dev, 1)) != MGRIT_OK) return cleanup_fail(st);
  if ((st = h->alloc(&h->err_dev, 1)) != MGRIT_OK) return cleanup_fail(st);
  if (!(h->norm_host = pinned_take())) return cleanup_fail(fail(MGRIT_ENOMEM, "pinned host allocation failed"));

  cudaStream_t s = h->stream;
  WaveParams wp{wave->kind, wave->a, wave->k, wave->a2};
  auto launch_fail = [&](const char* what) {  // launch errors; execution errors surface in setup_finish
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cleanup_fail(fail(MGRIT_ECUDA, std::string(what) + ": " + cudaGetErrorString(e)));
    return MGRIT_OK;
  };
  if (opt.profile) {
    h->ev_pool.resize(defer ? 64 : 4096);  // a batched problem times only its setup phases
    for (auto& e : h->ev_pool)
      if (cudaEventCreate(&e) != cudaSuccess) return cleanup_fail(fail(MGRIT_ECUDA, "cudaEventCreate failed"));
  }
  h->reset_call_counters();
  cudaMemsetAsync(h->flag_dev, 0, sizeof(int), s);
  cudaMemsetAsync(h->err_dev, 0, sizeof(int), s);
  // fine departure points and tables
  {
    const int ev = h->phase_begin();
    if (dim == 2) {
      Level& L0 = h->levels[0];
      launch_departure_2d(wp, p, nx, grid->nt, grid->xmin, hgrid, dt, L0.s64, L0.s64 + (size_t)L0.nt * np, s);
    } else {
      launch_departure_1d(wp, p, nx, grid->nt, grid->xmin, hgrid, dt, h->levels[0].s64, opt.precision == 1, s);
    }
    h->phase_end(MGRIT_PHASE_DEPARTURE, ev, 1);
  }
  for (size_t l = 0; l < h->levels.size(); ++l) {
    Level& L = h->levels[l];
    const size_t blk = (size_t)L.nt * np;  // one component block
    if (l > 0) {
      Level& Lp = h->levels[l - 1];
      const size_t pblk = (size_t)Lp.nt * np;
      const int ev = h->phase_begin();
      if (dim == 2)
        launch_backtrack_2d(Lp.s64, Lp.s64 + pblk, l > 1 ? Lp.sigma : nullptr, l > 1 ? Lp.sigma + pblk : nullptr, L.m,
                            L.nt, nx, p, L.s64, L.s64 + blk, L.sigma, L.sigma + blk, s);
      else
        launch_backtrack_1d(Lp.s64, l > 1 ? Lp.sigma : nullptr, Lp.eps_lo ? Lp.eps32 : nullptr, Lp.eps_lo,
                            opt.precision == 1, L.m, L.nt, nx, p, L.s64, L.sigma, s);
      h->phase_end(MGRIT_PHASE_BACKTRACK, ev, 1);
    }
    {
      const int ev = h->phase_begin();
      for (int c = 0; c < dim; ++c)
        launch_build_tables(L.s64 + c * blk, L.nt, nx, np, p, L.shift + c * blk,
                            L.w64 ? L.w64 + (size_t)c * blk * (p + 1) : nullptr, L.eps32 ? L.eps32 + c * blk : nullptr,
                            L.eps_lo ? L.eps_lo + c * blk : nullptr, s);
      h->phase_end(MGRIT_PHASE_TABLES, ev, dim);
    }
    if (l > 0 && L.solver) {
      const int ev = h->phase_begin();
      const int nl = launch_factor_1d(L.sigma, L.nt, nx, p, (double*)L.solver, h->flag_dev, s);
      h->phase_end(MGRIT_PHASE_FACTOR, ev, nl);
    }
    if (l > 0 && L.sig32) {
      const int ev = h->phase_begin();
      launch_axpy_convert(1, L.sigma, L.sig32, nullptr, (long long)L.nt * np * dim, s);
      if (L.pcr32) launch_pcr_coef(L.sig32, L.nt, nx, p, L.pcr32, s);
      if (L.band32) {
        cudaMemsetAsync(L.band_ind, 0, 32 * sizeof(float), s);
        launch_sep_band(L.sig32, L.nt, nx, p, 8, L.band32, L.band_ind, s);
      }
      h->phase_end(MGRIT_PHASE_FACTOR, ev, (L.pcr32 ? 2 : 1) + (L.band32 ? 1 : 0));
    }
    if ((st = launch_fail("setup")) != MGRIT_OK) return st;
  }
  // zero rows that are read but never written: E_l[0], G_l[0], r64[0], EC[0]
  for (size_t l = 1; l < h->levels.size(); ++l) {
    Level& L = h->levels[l];
    const size_t esz = L.is_double ? sizeof(double) : sizeof(float);
    cudaMemsetAsync(L.E, 0, (size_t)(L.nt + 1) * np * esz, s);
    cudaMemsetAsync(L.G, 0, (size_t)(L.nt + 1) * np * esz, s);
  }
  if (fp32) {
    cudaMemsetAsync(h->r64, 0, (size_t)(J1 + 1) * np * sizeof(double), s);
    cudaMemsetAsync(h->EC, 0, (size_t)(J1 + 1) * np * sizeof(float), s);
  }
  // the pivot flag travels with the stream; setup_finish reads it after the synchronisation
  cudaMemcpyAsync(h->norm_host + 3, h->flag_dev, sizeof(int), cudaMemcpyDeviceToHost, s);
  if ((st = launch_fail("setup")) != MGRIT_OK) return st;
  h->setup_t0 = t0;
  *out = h;
  if (defer) return MGRIT_OK;
  return setup_finish(out);
}

mgrit_status mgrit_setup(const mgrit_grid* grid, const mgrit_wavespeed* wave, int order, int m, int levels,
                         const mgrit_options* opt_in, void* stream, mgrit_handle** out) {
  return setup_impl(grid, wave, order, m, levels, opt_in, stream, out, false);
}

}  // extern "C"

namespace {

// The MGRIT iteration.  u0 / u_init may be host or device pointers (kinds given); u_out is on the device.
// d_final_ref != NULL: the final-slice stopping rule (mgrit_solve_to_reference) with tolerance final_tol.
mgrit_status solve_impl(mgrit_handle* h, const double* d_u0, cudaMemcpyKind u0_kind, const double* d_u_init,
                        cudaMemcpyKind init_kind, double* d_u_out, mgrit_stats* stats,
                        const double* d_final_ref = nullptr, double final_tol = 0.0) {
  if (h->levels.size() < 2) return fail(MGRIT_EUNSUPPORTED, "a fine_only handle has no MGRIT hierarchy");
  const double t0 = now_ms();
  cudaStream_t s = h->stream;
  const int np = h->npts;
  const int m1 = h->levels[1].m, J = h->J1();
  const int fp32 = h->opt.precision == 1;
  h->reset_call_counters();
  MG_CUDA(cudaMemsetAsync(h->err_dev, 0, sizeof(int), s));  // a timeout of an earlier call is not this one's
  // initial iterate at the C-points
  MG_CUDA(cudaMemcpyAsync(h->X, d_u0, np * sizeof(double), u0_kind, s));
  MG_CUDA(cudaMemcpyAsync(h->Y, h->X, np * sizeof(double), cudaMemcpyDeviceToDevice, s));
  if (d_u_init) {
    MG_CUDA(cudaMemcpy2DAsync(h->X + np, np * sizeof(double), d_u_init + (size_t)m1 * np,
                              (size_t)m1 * np * sizeof(double), np * sizeof(double), J, init_kind, s));
  } else {
    MG_CUDA(cudaMemsetAsync(h->X + np, 0, (size_t)J * np * sizeof(double), s));
  }
  Level& L1 = h->levels[1];
  std::vector<double> hist;
  double r0 = 0.0, rk = 0.0;
  int iters = 0;
  bool converged = false;
  mgrit_status status = MGRIT_OK;
  // one cycle's device work (FP64: reads X, writes Y; the caller swaps the pointers afterwards)
  const bool fcf = h->opt.relax == 0;
  auto cycle_body = [&](int k) -> mgrit_status {
    if (!fp32 && !fcf) {
      // F-relaxation only: one pass from the corrected C-points X + E_1 (written to Y for the next
      // cycle), F-relaxation and the C-point residual against the corrected C-points
      RelaxArgs a = args0();
      a.m = m1;
      a.J = J;
      a.nsteps = m1;
      a.mode = MODE_RES;
      a.start = h->X;
      a.start_stride = np;
      a.corr = k > 0 ? L1.E : nullptr;
      a.corr_stride = np;
      a.start_wb = h->Y;
      a.wb_stride = np;
      a.extra_cta = 1;
      a.cin = h->X;
      a.cin_corr = k > 0 ? L1.E : nullptr;
      a.c_stride = np;
      a.rout = L1.G;
      a.r_stride = np;
      a.norm_partial = h->norm_partial;
      MG_TRY(relax(h, 0, 1, a, MGRIT_PHASE_FINE64_RES));
      MG_TRY(coarse_cycle(h, 1));
    } else if (!fp32) {
      // FCF relaxation on level 0; the correction of the previous cycle is fused into the first pass
      RelaxArgs a = args0();
      a.m = m1;
      a.J = J;
      a.nsteps = m1;
      a.mode = MODE_FC;
      a.start = h->X;
      a.start_stride = np;
      a.corr = k > 0 ? L1.E : nullptr;
      a.corr_stride = np;
      a.cout = h->Y;
      a.c_stride = np;
      MG_TRY(relax(h, 0, 1, a, MGRIT_PHASE_FINE64_FC));
      a = args0();
      a.m = m1;
      a.J = J;
      a.nsteps = m1;
      a.mode = MODE_RES;
      a.start = h->Y;
      a.start_stride = np;
      a.cin = h->Y;
      a.c_stride = np;
      a.rout = L1.G;
      a.r_stride = np;
      a.norm_partial = h->norm_partial;
      MG_TRY(relax(h, 0, 1, a, MGRIT_PHASE_FINE64_RES));
      MG_TRY(coarse_cycle(h, 1));
    } else {
      // FP64 residual of the current iterate (F-relaxation + C-point residual)
      RelaxArgs a = args0();
      a.m = m1;
      a.J = J;
      a.nsteps = m1;
      a.mode = MODE_RES;
      a.start = h->X;
      a.start_stride = np;
      a.cin = h->X;
      a.c_stride = np;
      a.rout = h->r64;
      a.r_stride = np;
      if (!fcf) {
        // F-relaxation only: on the error equation from a zero guess the F-points stay zero and the
        // C-point residual is r itself, the right-hand side of level 1; then u_C += E_1
        if (L1.is_double) a.rout = L1.G;  // FP64 coarse cycle: r is its right-hand side as it is
        else a.rout32 = (float*)L1.G;
        a.norm_partial = h->norm_partial;
        MG_TRY(relax(h, 0, 1, a, MGRIT_PHASE_FINE64_RES));
        MG_TRY(coarse_cycle(h, 1));
        const int ev = h->phase_begin();
        launch_axpy_convert(L1.is_double ? 4 : 2, L1.E, h->X, nullptr, (long long)(J + 1) * np, s);
        h->phase_end(MGRIT_PHASE_MISC, ev, 1);
        return enqueue_norm(h, J);
      }
      a.rout32 = h->EC;  // C-relaxation of the error equation from a zero guess gives e_C = r (FP32)
      // FP32-pair residual pass (1D): r64 receives the C-relaxed value S^m u_C(j) = u_C(j+1) + r(j+1)
      const bool cval = h->levels[0].eps_lo != nullptr;
      a.rout_value = cval ? 1 : 0;
      MG_TRY(relax(h, 0, 1, a, MGRIT_PHASE_FINE64_RES));
      // F-relaxation + residual of the error equation in FP32
      a = args0();
      a.m = m1;
      a.J = J;
      a.nsteps = m1;
      a.mode = MODE_RES;
      a.start = h->EC;
      a.start_stride = np;
      a.rout = L1.G;
      a.rout_f64 = L1.is_double;
      a.r_stride = np;
      a.norm_partial = h->norm_partial;
      MG_TRY(relax(h, 0, 0, a, MGRIT_PHASE_FINE32_RES));
      MG_TRY(coarse_cycle(h, 1));
      // u_C += r + E_1 (with the C-relaxed values: u_C(j) = r64(j) + E_1(j), j >= 1; u_C(0) stays u0)
      {
        const int ev = h->phase_begin();
        if (cval)
          launch_axpy_convert(L1.is_double ? 9 : 8, h->r64 + np, h->X + np,
                              L1.is_double ? (const void*)((const double*)L1.E + np) : (const void*)((const float*)L1.E + np),
                              (long long)J * np, s);
        else
          launch_axpy_convert(L1.is_double ? 7 : 5, h->r64, h->X, L1.E, (long long)(J + 1) * np, s);
        h->phase_end(MGRIT_PHASE_MISC, ev, 1);
      }
    }
    return enqueue_norm(h, J);
  };
  // with a final-slice reference: the squared distance of u(T) after this cycle's correction (FP64:
  // the relaxed C-points in Y plus E_1, applied by the next pass; FP32 bulk: X, already corrected)
  auto cycle = [&](int k) -> mgrit_status {
    MG_TRY(cycle_body(k));
    if (d_final_ref) {
      const size_t last = (size_t)J * np;
      const int ev = h->phase_begin();
      launch_dist2(fp32 ? h->X + last : h->Y + last, fp32 ? nullptr : (const double*)L1.E + last, d_final_ref, np,
                   h->norm_dev + 1, s);
      h->phase_end(MGRIT_PHASE_MISC, ev, 1);
      MG_CUDA(cudaMemcpyAsync(h->norm_host + 2, h->norm_dev + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
    }
    return MGRIT_OK;
  };
  const double wgt = std::pow((h->grid.xmax - h->grid.xmin) / h->grid.nx, (double)h->grid.dim);
  double ek = 0.0;
  // CUDA graphs (use_graph): FP32-bulk cycles are identical; FP64 cycles k >= 1 alternate X / Y
  CycleGraph graphs[2];
  bool graph_ok = h->opt.use_graph != 0;
  for (int k = 0; k < h->opt.max_iter; ++k) {
    const bool graphed = graph_ok && (fp32 || k >= 1);
    CycleGraph& G = graphs[fp32 ? 0 : (k & 1)];
    if (graphed) MG_TRY(run_cycle(h, G, &graph_ok, [&] { return cycle(k); }));
    else MG_TRY(cycle(k));
    MG_TRY(finish_norm(h, &rk));
    if (graphed && graph_ok) collect_graph_times(h, G);
    if (!fp32) std::swap(h->X, h->Y);
    hist.push_back(rk);
    iters = k + 1;
    if (k == 0) r0 = rk;
    if (!std::isfinite(rk) || (h->opt.diverge_ratio > 0.0 && rk > h->opt.diverge_ratio * r0)) {
      status = fail(MGRIT_EDIVERGED, "residual norm diverged");
      break;
    }
    if (d_final_ref) {
      ek = std::sqrt(wgt * h->norm_host[2]);
      if (ek <= final_tol) {
        converged = true;
        break;
      }
    } else if (k >= 1 && rk < h->opt.rtol * r0) {
      converged = true;
      break;
    }
  }
  // post F-relaxation from the (corrected) C-points into the full output
  {
    RelaxArgs a = args0();
    a.m = m1;
    a.J = J;
    a.nsteps = m1 - 1;
    a.mode = MODE_POST;
    a.start = h->X;
    a.start_stride = np;
    a.corr = fp32 ? nullptr : L1.E;
    a.corr_stride = np;
    a.start_wb = d_u_out;
    a.wb_stride = (long long)m1 * np;
    a.extra_cta = 1;
    a.fstore = d_u_out;
    MG_TRY(relax(h, 0, 1, a, MGRIT_PHASE_FINE64_POST));
  }
  MG_CUDA(cudaStreamSynchronize(s));
  h->collect_phase_times();
  if (status == MGRIT_OK && !converged) status = fail(MGRIT_ENOTCONVERGED, "max_iter reached");
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    stats->iterations = iters;
    stats->converged = converged ? 1 : 0;
    stats->levels = (int)h->levels.size();
    stats->r0 = r0;
    stats->r_final = rk;
    stats->final_error = ek;
    const int nh = (int)hist.size() < 256 ? (int)hist.size() : 256;
    stats->history_len = nh;
    for (int i = 0; i < nh; ++i) stats->residual_history[i] = hist[i];
    stats->setup_ms = h->setup_ms;
    stats->solve_ms = now_ms() - t0;
    stats->device_bytes = h->bytes;
    stats->kernel_launches = h->setup_launches + h->call_launches;
    for (int i = 0; i < MGRIT_NUM_PHASES; ++i) {
      stats->phase_ms[i] = h->setup_phase_ms[i] + h->phase_ms[i];
      stats->phase_launches[i] = h->setup_phase_launches[i] + h->phase_launches[i];
    }
  }
  return status;
}

}  // namespace

extern "C" {

mgrit_status mgrit_solve(mgrit_handle* h, const double* d_u0, const double* d_u_init, double* d_u_out,
                         mgrit_stats* stats) {
  if (!h || !d_u0 || !d_u_out) return fail(MGRIT_EINVAL, "handle, u0 and u_out must not be NULL");
  return solve_impl(h, d_u0, cudaMemcpyDeviceToDevice, d_u_init, cudaMemcpyDeviceToDevice, d_u_out, stats);
}

mgrit_status mgrit_solve_to_reference(mgrit_handle* h, const double* d_u0, const double* d_u_init, double* d_u_out,
                                      const double* d_u_final_ref, double tol, mgrit_stats* stats) {
  if (!h || !d_u0 || !d_u_out || !d_u_final_ref)
    return fail(MGRIT_EINVAL, "handle, u0, u_out and u_final_ref must not be NULL");
  if (!(tol >= 0.0)) return fail(MGRIT_EINVAL, "tol must be >= 0");
  return solve_impl(h, d_u0, cudaMemcpyDeviceToDevice, d_u_init, cudaMemcpyDeviceToDevice, d_u_out, stats,
                    d_u_final_ref, tol);
}

mgrit_status mgrit_solve_host(mgrit_handle* h, const double* h_u0, const double* h_u_init, double* h_u_out,
                              mgrit_stats* stats) {
  if (!h || !h_u0 || !h_u_out) return fail(MGRIT_EINVAL, "handle, u0 and u_out must not be NULL");
  const size_t np = h->npts, nt = h->grid.nt;
  double* d_out = nullptr;
  cudaStream_t s = h->stream;
  MG_CUDA(scratch_alloc((void**)&d_out, (nt + 1) * np * sizeof(double), s));
  // the initial iterate is read only at the C-points, straight from host memory
  mgrit_status st = solve_impl(h, h_u0, cudaMemcpyHostToDevice, h_u_init, cudaMemcpyHostToDevice, d_out, stats);
  cudaMemcpyAsync(h_u_out, d_out, (nt + 1) * np * sizeof(double), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(d_out, s);
  MG_CUDA(cudaStreamSynchronize(s));
  return st;
}

mgrit_status sl_step_sequential(mgrit_handle* h, const double* d_u0, double* d_u_out, int store_all) {
  if (!h || !d_u0 || !d_u_out) return fail(MGRIT_EINVAL, "handle, u0 and u_out must not be NULL");
  const double t0 = now_ms();
  const int np = h->npts, nt = h->grid.nt;
  cudaStream_t s = h->stream;
  LevelTables T = h->tables(0, h->opt.precision == 0 ? 1 : 0);  // the tables of the stepping precision
  T.solver = nullptr;
  h->reset_call_counters();
  const int ev = h->phase_begin();
  // 1D: one thread-block cluster over the slice; the single-CTA kernel where no cluster can be formed
  auto seq1d = [&](const void* u0, void* out, int dbl) -> cudaError_t {
    cudaError_t e = h->grid.nx >= 256 ? launch_sequential_cluster_1d(T, nt, u0, out, store_all, dbl, s)
                                      : cudaErrorNotSupported;
    if (e == cudaErrorNotSupported) {
      cudaGetLastError();
      e = launch_sequential_1d(T, nt, nullptr, u0, out, store_all, dbl, s);
    }
    return e;
  };
  if (h->opt.precision == 0) {
    if (h->grid.dim == 2) MG_CUDA(launch_sequential_2d(T, nt, nullptr, d_u0, d_u_out, store_all, h->s2d, 1, s));
    else MG_CUDA(seq1d(d_u0, d_u_out, 1));
  } else {
    const size_t rows = store_all ? (size_t)(nt + 1) : 1;
    float *u0f = nullptr, *outf = nullptr;
    MG_CUDA(scratch_alloc((void**)&u0f, np * sizeof(float), s));
    MG_CUDA(scratch_alloc((void**)&outf, rows * np * sizeof(float), s));
    launch_axpy_convert(1, d_u0, u0f, nullptr, np, s);
    if (h->grid.dim == 2) MG_CUDA(launch_sequential_2d(T, nt, nullptr, u0f, outf, store_all, h->s2d, 0, s));
    else MG_CUDA(seq1d(u0f, outf, 0));
    launch_axpy_convert(3, outf, d_u_out, nullptr, (long long)rows * np, s);
    cudaFreeAsync(u0f, s);
    cudaFreeAsync(outf, s);
  }
  h->phase_end(MGRIT_PHASE_SEQUENTIAL, ev, h->opt.precision == 0 ? 1 : 3);
  MG_CUDA(cudaGetLastError());
  (void)t0;
  return MGRIT_OK;
}

}  // extern "C"

namespace {

// Builds the data the adjoint needs on first use: per-step floor ranges of every level, the
// factorisation of M^T of every coarse step, and d s / d a on level 0.
mgrit_status ensure_adjoint(mgrit_handle* h) {
  if (h->adjoint_ready) return MGRIT_OK;
  cudaStream_t s = h->stream;
  const int nx = h->grid.nx, np = h->npts, p = h->order;
  const double hg = (h->grid.xmax - h->grid.xmin) / nx;
  WaveParams wp{h->wave.kind, h->wave.a, h->wave.k, h->wave.a2};
  if (h->grid.dim == 2) {
    for (size_t l = 0; l < h->levels.size(); ++l) {
      Level& L = h->levels[l];
      MG_TRY(h->alloc(&L.bstart, (size_t)L.nt * (np + 1)));
      MG_TRY(h->alloc(&L.bperm, (size_t)L.nt * np));
      MG_CUDA(launch_bucket_build(L.shift, L.nt, nx, L.bstart, L.bperm, s));
    }
    Level& L0 = h->levels[0];
    MG_TRY(h->alloc(&L0.ds, (size_t)2 * L0.nt * np));
    launch_departure_da_2d(wp, p, nx, L0.nt, h->grid.xmin, hg, h->grid.cfl * hg, L0.ds, L0.ds + (size_t)L0.nt * np,
                           s);
    MG_CUDA(cudaGetLastError());
    MG_CUDA(cudaStreamSynchronize(s));
    h->adjoint_ready = true;
    return MGRIT_OK;
  }
  for (size_t l = 0; l < h->levels.size(); ++l) {
    Level& L = h->levels[l];
    MG_TRY(h->alloc(&L.frange, (size_t)L.nt));
    launch_floor_range(L.s64, L.nt, nx, L.frange, s);
    if (l > 0 && L.solver) {
      MG_TRY(h->alloc((char**)&L.solverT, L.solver_stride * L.nt * sizeof(double)));
      launch_factor_1d(L.sigma, L.nt, nx, p, (double*)L.solverT, h->flag_dev, s, 1);
    }
  }
  Level& L0 = h->levels[0];
  MG_TRY(h->alloc(&L0.ds, (size_t)L0.nt * np));
  launch_departure_da_1d(wp, p, nx, L0.nt, h->grid.xmin, hg, h->grid.cfl * hg, L0.ds, s);
  int flag = 0;
  MG_CUDA(cudaMemcpyAsync(&flag, h->flag_dev, sizeof(int), cudaMemcpyDeviceToHost, s));
  MG_CUDA(cudaStreamSynchronize(s));
  if (flag) return fail(MGRIT_ESINGULAR, "a transposed correction matrix has a (near) zero pivot");
  h->adjoint_ready = true;
  return MGRIT_OK;
}

}  // namespace

extern "C" {

mgrit_status mgrit_adjoint_solve(mgrit_handle* h, const double* d_u_target, const double* d_C_checkpoints,
                                 double* d_dJ_du0, double* d_dJ_dparams, mgrit_stats* stats) {
  if (!h || !d_u_target || !d_C_checkpoints || !d_dJ_du0 || !d_dJ_dparams)
    return fail(MGRIT_EINVAL, "NULL argument");
  if (h->opt.precision != 0) return fail(MGRIT_EUNSUPPORTED, "the adjoint solve needs an FP64 handle (precision 0)");
  if (h->levels.size() < 2) return fail(MGRIT_EUNSUPPORTED, "a fine_only handle has no MGRIT hierarchy");
  if (h->gmres1d) return fail(MGRIT_EUNSUPPORTED, "the 1D adjoint uses exact correction solves (solve_mode 0)");
  MG_TRY(ensure_adjoint(h));
  cudaStream_t s = h->stream;
  const int np = h->npts, nt = h->grid.nt, m1 = h->levels[1].m, J = h->J1();
  double *mu0 = nullptr, *mu = nullptr;
  MG_CUDA(scratch_alloc((void**)&mu0, (size_t)np * sizeof(double), s));
  MG_CUDA(scratch_alloc((void**)&mu, (size_t)(nt + 1) * np * sizeof(double), s));
  // mu_0 = lambda_nt = u_nt - u_target; u_nt is the last checkpoint (nt is a C-point)
  launch_axpy_convert(6, d_C_checkpoints + (size_t)J * np, mu0, d_u_target, np, s);
  // the reversed problem mu_{k+1} = Phi_{nt-1-k}^T mu_k by MGRIT from a zero initial iterate
  h->trans_mode = 1;
  mgrit_status st = solve_impl(h, mu0, cudaMemcpyDeviceToDevice, nullptr, cudaMemcpyDeviceToDevice, mu, stats);
  h->trans_mode = 0;
  if (st == MGRIT_OK) {
    // dJ/du0 = lambda_0 = mu_nt
    cudaMemcpyAsync(d_dJ_du0, mu + (size_t)nt * np, (size_t)np * sizeof(double), cudaMemcpyDeviceToDevice, s);
    // dJ/da = sum_n lambda_{n+1}^T (dPhi_n/da) u_n, u_n recomputed from the checkpoints
    LevelTables T0 = h->tables(0, 1);
    T0.solver = nullptr;
    const Level& L0 = h->levels[0];
    cudaError_t e = h->grid.dim == 2
                        ? launch_gradient_a_2d(T0, L0.ds, d_C_checkpoints, mu, nt, m1, J, h->s2d, h->norm_partial, s)
                        : launch_gradient_a_1d(T0, L0.s64, L0.ds, d_C_checkpoints, mu, nt, m1, h->norm_partial, s);
    if (e != cudaSuccess) st = fail(MGRIT_ECUDA, std::string("gradient kernel: ") + cudaGetErrorString(e));
    launch_sum(h->norm_partial, J, h->norm_dev, s);
    cudaMemcpyAsync(d_dJ_dparams, h->norm_dev, sizeof(double), cudaMemcpyDeviceToDevice, s);
  }
  cudaFreeAsync(mu0, s);
  cudaFreeAsync(mu, s);
  MG_CUDA(cudaStreamSynchronize(s));
  return st;
}

mgrit_status mgrit_level_info(const mgrit_handle* h, int level, int* nt_level, int* m_level) {
  if (!h) return fail(MGRIT_EINVAL, "handle is NULL");
  if (level < 0 || level >= (int)h->levels.size()) {
    if (nt_level) *nt_level = (int)h->levels.size();
    return fail(MGRIT_EINVAL, "level out of range");
  }
  if (nt_level) *nt_level = h->levels[level].nt;
  if (m_level) *m_level = h->levels[level].m;
  return MGRIT_OK;
}

mgrit_status mgrit_level_band(const mgrit_handle* h, int level, int* half_width, float* decay) {
  if (!h || !half_width) return fail(MGRIT_EINVAL, "NULL argument");
  if (level < 0 || level >= (int)h->levels.size()) return fail(MGRIT_EINVAL, "level out of range");
  *half_width = h->levels[level].band_w;
  if (decay)
    for (int t = 0; t < 4; ++t) decay[t] = h->levels[level].band_decay[t];
  return MGRIT_OK;
}

mgrit_status mgrit_copy_offsets(const mgrit_handle* h, int level, double* d_out) {
  if (!h || !d_out) return fail(MGRIT_EINVAL, "NULL argument");
  if (level < 0 || level >= (int)h->levels.size()) return fail(MGRIT_EINVAL, "level out of range");
  const Level& L = h->levels[level];
  MG_CUDA(cudaMemcpyAsync(d_out, L.s64, (size_t)L.nt * h->npts * h->grid.dim * sizeof(double),
                          cudaMemcpyDeviceToDevice, h->stream));
  MG_CUDA(cudaStreamSynchronize(h->stream));
  return MGRIT_OK;
}

mgrit_status mgrit_copy_sigma(const mgrit_handle* h, int level, double* d_out) {
  if (!h || !d_out) return fail(MGRIT_EINVAL, "NULL argument");
  if (level < 1 || level >= (int)h->levels.size()) return fail(MGRIT_EINVAL, "level out of range (>= 1)");
  const Level& L = h->levels[level];
  MG_CUDA(cudaMemcpyAsync(d_out, L.sigma, (size_t)L.nt * h->npts * h->grid.dim * sizeof(double),
                          cudaMemcpyDeviceToDevice, h->stream));
  MG_CUDA(cudaStreamSynchronize(h->stream));
  return MGRIT_OK;
}

mgrit_status mgrit_apply_step(mgrit_handle* h, int level, int n0, int count, const double* d_in, double* d_out) {
  if (!h || !d_in || !d_out) return fail(MGRIT_EINVAL, "NULL argument");
  if (level < 0 || level >= (int)h->levels.size()) return fail(MGRIT_EINVAL, "level out of range");
  const Level& L = h->levels[level];
  if (count < 0 || n0 < 0 || n0 + count > L.nt) return fail(MGRIT_EINVAL, "step range out of range");
  const int np = h->npts;
  cudaStream_t s = h->stream;
  const int dbl = L.is_double;
  LevelTables T = h->tables(level, dbl);
  if (dbl) {
    if (h->grid.dim == 2 || (h->gmres1d && level > 0))
      MG_CUDA(launch_apply_steps_2d(T, n0, count, d_in, d_out, h->s2d, 1, s));
    else MG_CUDA(launch_apply_steps_1d(T, n0, count, d_in, d_out, 1, s));
  } else {
    float *fi = nullptr, *fo = nullptr;
    MG_CUDA(scratch_alloc((void**)&fi, (size_t)count * np * sizeof(float), s));
    MG_CUDA(scratch_alloc((void**)&fo, (size_t)count * np * sizeof(float), s));
    launch_axpy_convert(1, d_in, fi, nullptr, (long long)count * np, s);
    if (h->grid.dim == 2) MG_CUDA(launch_apply_steps_2d(T, n0, count, fi, fo, h->s2d, 0, s));
    else MG_CUDA(launch_apply_steps_1d(T, n0, count, fi, fo, 0, s));
    launch_axpy_convert(3, fo, d_out, nullptr, (long long)count * np, s);
    cudaFreeAsync(fi, s);
    cudaFreeAsync(fo, s);
  }
  MG_CUDA(cudaStreamSynchronize(s));
  return MGRIT_OK;
}

}  // extern "C"

namespace {

// Staging memory of mgrit_apply_step_noalloc: two buffers of kNoAllocMaxElems FP32 values (8 MiB in
// total) in file-scope device memory.  Every GPU that loads this library holds it until the process
// exits.  In host code `g_noalloc_stage` only names a host-side stand-in, so its device address on the
// current device is looked up with cudaGetSymbolAddress on every call (cheap, and never stale).
constexpr long long kNoAllocMaxElems = 1LL << 20;
static __device__ __align__(256) float g_noalloc_stage[2 * kNoAllocMaxElems];

mgrit_status noalloc_stage_address(float** out) {
  void* p = nullptr;
  MG_CUDA(cudaGetSymbolAddress(&p, g_noalloc_stage));
  *out = static_cast<float*>(p);
  return MGRIT_OK;
}

}  // namespace

extern "C" {

mgrit_status mgrit_apply_step_noalloc(mgrit_handle* h, int level, int n0, int count, const double* d_in,
                                      double* d_out) {
  if (!h || !d_in || !d_out) return fail(MGRIT_EINVAL, "NULL argument");
  if (level < 0 || level >= (int)h->levels.size()) return fail(MGRIT_EINVAL, "level out of range");
  const Level& L = h->levels[level];
  if (count < 0 || n0 < 0 || n0 + count > L.nt) return fail(MGRIT_EINVAL, "step range out of range");
  const int np = h->npts;
  const long long elems = (long long)count * np;
  if (elems > kNoAllocMaxElems)
    return fail(MGRIT_EINVAL, "count * slice size exceeds the no-allocation staging capacity of " +
                                  std::to_string(kNoAllocMaxElems) + " values");
  int dev = -1;
  MG_CUDA(cudaGetDevice(&dev));
  if (dev != h->device)
    return fail(MGRIT_EINVAL, "the current device (" + std::to_string(dev) + ") is not the handle's device (" +
                                  std::to_string(h->device) + ")");
  cudaStream_t s = h->stream;
  const int dbl = L.is_double;
  LevelTables T = h->tables(level, dbl);
  if (dbl) {
    if (h->grid.dim == 2 || (h->gmres1d && level > 0))
      MG_CUDA(launch_apply_steps_2d(T, n0, count, d_in, d_out, h->s2d, 1, s));
    else MG_CUDA(launch_apply_steps_1d(T, n0, count, d_in, d_out, 1, s));
  } else {
    float* stage = nullptr;
    MG_TRY(noalloc_stage_address(&stage));
    float* fi = stage;
    float* fo = stage + kNoAllocMaxElems;
    launch_axpy_convert(1, d_in, fi, nullptr, elems, s);
    if (h->grid.dim == 2) MG_CUDA(launch_apply_steps_2d(T, n0, count, fi, fo, h->s2d, 0, s));
    else MG_CUDA(launch_apply_steps_1d(T, n0, count, fi, fo, 0, s));
    launch_axpy_convert(3, fo, d_out, nullptr, elems, s);
  }
  MG_CUDA(cudaGetLastError());
  MG_CUDA(cudaStreamSynchronize(s));
  return MGRIT_OK;
}

void mgrit_destroy(mgrit_handle* h) { delete h; }

}  // extern "C"

// ---- batched problems ------------------------------------------------------------------------------

struct mgrit_batch {
  cudaStream_t stream = nullptr;
  std::vector<mgrit_handle*> hs;
  mgrit_options opt;
  struct Phase {
    int kind;  // 0 relax, 1 sequential
    int is_double, coarse;
    int tile_off, ntiles;
    int buf;
    size_t smem;
    size_t region;  // coarse shared region (on-the-fly solve) after the slice buffers
    int order;      // tile order chosen by the tuner (0: as built, 1: longest first)
    int threads;    // CTA size of an FP32 relaxation phase (its tiles' slices hold at most 8 * threads points)
  };
  std::vector<Phase> down, up;
  std::vector<Phase> final_post;  // the post F-relaxation into the outputs, one launch per CTA size
  std::vector<int> final_args;     // per problem: its RelaxArgs of the final post F-relaxation
  std::vector<BatchTile> tiles;
  std::vector<LevelTables> tabs;
  std::vector<RelaxArgs> args;
  std::vector<SeqArgs> seqs;
  LevelTables* d_tabs = nullptr;
  RelaxArgs* d_args = nullptr;
  SeqArgs* d_seq = nullptr;
  BatchTile* d_tiles = nullptr;
  int* d_active = nullptr;
  Segment* d_seg = nullptr;
  double* d_norms = nullptr;
  double* h_norms = nullptr;
  int* h_active = nullptr;    // pinned: uploaded before every cycle
  Segment* h_seg = nullptr;   // pinned: 3 * nprob segments
  long long maxn_all = 0;     // largest C-point array of any problem (launch size of the batched axpy)
  cudaGraphExec_t graph = nullptr;  // one cycle, captured on the first solve (use_graph)
  int final_args_off = 0;
  int64_t setup_launches = 0;       // the problems' setup kernels and the tuner's timed runs
  int* d_err = nullptr;             // bounded-wait flag of every batched launch (LevelTables.err)
  std::vector<cudaEvent_t> ev;      // profile = 1: a start / end pair per launch of one cycle

  ~mgrit_batch() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    if (graph) cudaGraphExecDestroy(graph);
    if (h_active) cudaFreeHost(h_active);
    if (h_seg) cudaFreeHost(h_seg);
    for (mgrit_handle* h : hs) delete h;
    cudaFree(d_tabs);
    cudaFree(d_args);
    cudaFree(d_seq);
    cudaFree(d_tiles);
    cudaFree(d_active);
    cudaFree(d_seg);
    cudaFree(d_norms);
    cudaFree(d_err);
    if (h_norms) cudaFreeHost(h_norms);
  }
};

namespace {

// Tile order and CTA size of each relaxation phase, chosen by measurement.  The tiles of one phase carry
// different work (nx * steps varies 16-fold across a batch); the GPU starts CTAs in launch order, so the
// order decides the tail.  Order candidates: as built (problem by problem) and longest first; CTA sizes
// (FP32 phases): the size of the phase's slice class (cta_threads) and up to two doublings.  Each
// candidate is timed on the phase itself (CUDA events, best of two runs after one warm-up; the cycle
// state is rebuilt by every solve, so these runs leave nothing behind); the fastest is kept.  Choices
// are cached per batch signature (problem shapes and options), so only the first setup of a batch pays.
std::mutex& tune_mu() {
  static std::mutex* m = new std::mutex;
  return *m;
}
std::map<std::string, std::vector<char>>& tune_cache() {
  static auto* c = new std::map<std::string, std::vector<char>>;
  return *c;
}

mgrit_status tune_tile_order(mgrit_batch* b, const mgrit_grid* grids, const mgrit_wavespeed* waves,
                             const int* orders, const int* ms) {
  const int nprob = (int)b->hs.size();
  std::string key;
  for (int q = 0; q < nprob; ++q) {
    char buf[160];
    std::snprintf(buf, sizeof(buf), "%d,%d,%d,%d,%d,%.17g,%.17g,%.17g,%.17g;", grids[q].nx, grids[q].nt, orders[q],
                  ms[q], waves[q].kind, waves[q].a, waves[q].k, waves[q].a2, grids[q].cfl);
    key += buf;
  }
  key += std::to_string(b->opt.max_coarsest) + "," + std::to_string(b->opt.m_first);
  std::vector<mgrit_batch::Phase*> phases;
  for (auto& ph : b->down)
    if (ph.kind == 0 && ph.ntiles > 1) phases.push_back(&ph);
  for (auto& ph : b->up)
    if (ph.kind == 0 && ph.ntiles > 1) phases.push_back(&ph);
  auto longest_first = [&](const mgrit_batch::Phase& ph) {
    std::vector<BatchTile> t(b->tiles.begin() + ph.tile_off, b->tiles.begin() + ph.tile_off + ph.ntiles);
    std::stable_sort(t.begin(), t.end(), [&](const BatchTile& x, const BatchTile& y) {
      const long long wx = (long long)b->tabs[x.table].nx * b->args[x.args].nsteps;
      const long long wy = (long long)b->tabs[y.table].nx * b->args[y.args].nsteps;
      return wx > wy;
    });
    return t;
  };
  std::vector<char> choice;
  {
    std::lock_guard<std::mutex> lk(tune_mu());
    auto it = tune_cache().find(key);
    if (it != tune_cache().end() && it->second.size() == phases.size()) choice = it->second;
  }
  cudaStream_t s = b->stream;
  if (choice.empty()) {
    for (int q = 0; q < nprob; ++q) b->h_active[q] = 1;
    MG_CUDA(cudaMemcpyAsync(b->d_active, b->h_active, nprob * sizeof(int), cudaMemcpyHostToDevice, s));
    cudaEvent_t e0, e1;
    MG_CUDA(cudaEventCreate(&e0));
    MG_CUDA(cudaEventCreate(&e1));
    for (mgrit_batch::Phase* ph : phases) {
      const std::vector<BatchTile> built(b->tiles.begin() + ph->tile_off, b->tiles.begin() + ph->tile_off + ph->ntiles);
      const std::vector<BatchTile> sorted = longest_first(*ph);
      // candidates: tile order x CTA size (FP32 phases: the class size and up to two doublings, <= 512)
      const int max_shift = ph->is_double == 1 ? 0 : (ph->threads <= 128 ? 2 : (ph->threads <= 256 ? 1 : 0));
      float best_t = 1e30f;
      int best_code = 0;
      for (int c = 0; c < 2; ++c) {
        const std::vector<BatchTile>& t = c == 0 ? built : sorted;
        MG_CUDA(cudaMemcpyAsync(b->d_tiles + ph->tile_off, t.data(), t.size() * sizeof(BatchTile),
                                cudaMemcpyHostToDevice, s));
        for (int sh = 0; sh <= max_shift; ++sh) {
          float bt = 1e30f;
          for (int rep = 0; rep < 3; ++rep) {
            ++b->setup_launches;
            MG_CUDA(cudaEventRecord(e0, s));
            MG_CUDA(launch_relax_batched(b->d_tabs, b->d_args, b->d_tiles + ph->tile_off, ph->ntiles, b->d_active,
                                         ph->is_double, ph->coarse, ph->buf, ph->smem, ph->threads << sh, s));
            MG_CUDA(cudaEventRecord(e1, s));
            MG_CUDA(cudaEventSynchronize(e1));
            float ms_ = 0.f;
            MG_CUDA(cudaEventElapsedTime(&ms_, e0, e1));
            if (rep > 0) bt = std::min(bt, ms_);
          }
          if (bt < best_t) {
            best_t = bt;
            best_code = c | (sh << 1);
          }
        }
      }
      choice.push_back((char)best_code);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    std::lock_guard<std::mutex> lk(tune_mu());
    tune_cache()[key] = choice;
  }
  for (size_t i = 0; i < phases.size(); ++i) {
    mgrit_batch::Phase* ph = phases[i];
    const int order = choice[i] & 1, sh = choice[i] >> 1;
    if (order) {
      const std::vector<BatchTile> t = longest_first(*ph);
      std::copy(t.begin(), t.end(), b->tiles.begin() + ph->tile_off);
    }
    ph->order = order;
    ph->threads <<= sh;
  }
  MG_CUDA(cudaMemcpyAsync(b->d_tiles, b->tiles.data(), b->tiles.size() * sizeof(BatchTile), cudaMemcpyHostToDevice, s));
  MG_CUDA(cudaStreamSynchronize(s));
  return MGRIT_OK;
}

size_t batched_smem(int buf, int is_double, size_t region) {
  size_t b = 2 * (size_t)buf * (is_double ? 8 : 4) + 64 * sizeof(double);
  if (region) b = ((b + 127) & ~(size_t)127) + region;
  return b;
}

// Appends a phase of relax tiles; per problem q: J tiles (plus one if extra) using tabs[tab_of(q)] and
// args[args_of(q)].
// CTA size for the FP32 tiles of a problem: one thread per 8 slice points, between 32 and 512.  Problems
// with short slices then keep several intervals resident on an SM instead of one 512-thread CTA each.
int cta_threads(int nx) {
  const int t = nx / 8;
  return t < 32 ? 32 : (t > 512 ? 512 : t);
}

// coarse: 0 fine-level tiles; 1 coarse tiles solved by block PCR or on the fly; 2 coarse tiles with the
// banded separator inverse (each kind is its own kernel instantiation, so a phase takes one of them).
template <class F>
mgrit_batch::Phase add_relax_phase(mgrit_batch* b, int is_double, int coarse, F per_problem, int threads = 0) {
  mgrit_batch::Phase ph{0, is_double, coarse, (int)b->tiles.size(), 0, 0, 0, 0, 0, threads ? threads : 512};
  for (int q = 0; q < (int)b->hs.size(); ++q) {
    if (threads && cta_threads(b->hs[q]->grid.nx) != threads) continue;
    LevelTables T;
    RelaxArgs a;
    int ntile = 0;
    if (!per_problem(q, T, a, ntile)) continue;
    if (coarse && (T.band > 0 ? 2 : 1) != coarse) continue;
    T.err = b->d_err;
    const int ti = (int)b->tabs.size(), ai = (int)b->args.size();
    b->tabs.push_back(T);
    b->args.push_back(a);
    int buf;
    size_t smem, region;
    relax_smem_need(T, is_double, &buf, &smem, &region);
    ph.buf = std::max(ph.buf, buf);
    ph.region = std::max(ph.region, region);
    for (int j = 0; j < ntile; ++j) b->tiles.push_back(BatchTile{ti, ai, j, q});
  }
  ph.ntiles = (int)b->tiles.size() - ph.tile_off;
  // a common buffer length for every tile, then the largest coarse region after it
  ph.smem = batched_smem(ph.buf, is_double, ph.region);
  return ph;
}

// The phases of one relaxation pass: FP64 passes in one launch of 512-thread CTAs, FP32 and FP32-pair
// (is_double = 2) passes in one launch per CTA size (cta_threads), each over the problems of that size.
template <class F>
void add_relax_phases(mgrit_batch* b, int is_double, int coarse, F per_problem, std::vector<mgrit_batch::Phase>& list) {
  if (is_double == 1) {
    list.push_back(add_relax_phase(b, is_double, coarse, per_problem));
    return;
  }
  // coarse passes: the band tiles and the others in separate launches (their kernels differ)
  const int kinds[2] = {coarse ? 2 : 0, 1};
  const int nkinds = coarse ? 2 : 1;
  for (int t : {512, 256, 128, 64, 32})
    for (int i = 0; i < nkinds; ++i) {
      mgrit_batch::Phase ph = add_relax_phase(b, is_double, kinds[i], per_problem, t);
      if (ph.ntiles) list.push_back(ph);
    }
}

}  // namespace

extern "C" {

mgrit_status mgrit_setup_batched(int nprob, const mgrit_grid* grids, const mgrit_wavespeed* waves, const int* orders,
                                 const int* ms, const mgrit_options* opt_in, void* stream, mgrit_batch** out) {
  if (!out || !grids || !waves || !orders || !ms || nprob < 1) return fail(MGRIT_EINVAL, "bad batched arguments");
  *out = nullptr;
  mgrit_options opt;
  if (opt_in) opt = *opt_in;
  else mgrit_default_options(&opt);
  if (opt.precision != 1 && !(opt.fine_only && opt.precision == 0))
    return fail(MGRIT_EUNSUPPORTED, "batched solves run the FP32-bulk mode (precision 1)");
  if (opt.relax != 0) return fail(MGRIT_EUNSUPPORTED, "batched solves run FCF relaxation (relax 0)");
  if (opt.coarse_fp64 != 0) return fail(MGRIT_EUNSUPPORTED, "batched solves run FP32 coarse levels (coarse_fp64 0)");
  if (opt.coarse_op != 0) return fail(MGRIT_EUNSUPPORTED, "batched solves use the corrected coarse operator");
  if (opt.solve_mode != 0) return fail(MGRIT_EUNSUPPORTED, "batched solves use exact correction solves (solve_mode 0)");
  for (int q = 0; q < nprob; ++q)
    if (grids[q].dim != 1) return fail(MGRIT_EUNSUPPORTED, "batched solves are 1D");
  const double t0 = now_ms();
  mgrit_batch* b = new mgrit_batch();
  b->stream = (cudaStream_t)stream;
  b->opt = opt;
  // the problems' setups are enqueued on a few streams of their own so that they overlap, then completed
  // one by one; afterwards every handle works on the batch's stream
  {
    std::vector<cudaStream_t> ss((size_t)std::min(nprob, 8), nullptr);
    for (cudaStream_t& x : ss)
      if (cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        x = (cudaStream_t)stream;
      }
    if (stream) cudaStreamSynchronize((cudaStream_t)stream);  // work the caller queued before the setups
    mgrit_status st = MGRIT_OK;
    std::string err;
    for (int q = 0; q < nprob && st == MGRIT_OK; ++q) {
      mgrit_handle* h = nullptr;
      st = setup_impl(&grids[q], &waves[q], orders[q], ms[q], 0, &opt, (void*)ss[q % ss.size()], &h, true);
      if (st == MGRIT_OK) b->hs.push_back(h);
      else err = "problem " + std::to_string(q) + ": " + g_last_error;
    }
    for (size_t q = 0; q < b->hs.size(); ++q) {
      const mgrit_status fs = setup_finish(&b->hs[q]);
      if (fs != MGRIT_OK && st == MGRIT_OK) {
        st = fs;
        err = "problem " + std::to_string(q) + ": " + g_last_error;
      }
    }
    for (mgrit_handle* h : b->hs)
      if (h) h->stream = (cudaStream_t)stream;
    for (cudaStream_t x : ss)
      if (x && x != (cudaStream_t)stream) cudaStreamDestroy(x);
    if (st != MGRIT_OK) {
      std::vector<mgrit_handle*> keep;
      for (mgrit_handle* h : b->hs)
        if (h) keep.push_back(h);
      b->hs = keep;
      delete b;
      return fail(st, err);
    }
  }
  if (cudaMalloc((void**)&b->d_err, sizeof(int)) != cudaSuccess || cudaMemset(b->d_err, 0, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return fail(MGRIT_ENOMEM, "batched workspace allocation failed");
  }
  if (opt.fine_only) {  // sequential stepping only: no cycle phases
    *out = b;
    return MGRIT_OK;
  }
  // phases of one cycle (the level-0 FP64 passes in FP32 pairs: is_double = 2)
  add_relax_phases(b, 2, 0, [&](int q, LevelTables& T, RelaxArgs& a, int& nt) {
    mgrit_handle* h = b->hs[q];
    const int np = h->npts, m1 = h->levels[1].m, J = h->J1();
    T = h->tables(0, 1);
    a = args0();
    a.m = m1; a.J = J; a.nsteps = m1; a.mode = MODE_RES;
    a.start = h->X; a.start_stride = np; a.cin = h->X; a.c_stride = np; a.rout = h->r64; a.r_stride = np;
    a.rout32 = h->EC;  // e_C = r in FP32
    a.rout_value = 1;  // r64 receives the C-relaxed value S^m u_C(j) = u_C(j+1) + r(j+1)
    nt = J;
    return true;
  }, b->down);
  add_relax_phases(b, 0, 0, [&](int q, LevelTables& T, RelaxArgs& a, int& nt) {
    mgrit_handle* h = b->hs[q];
    const int np = h->npts, m1 = h->levels[1].m, J = h->J1();
    T = h->tables(0, 0);
    a = args0();
    a.m = m1; a.J = J; a.nsteps = m1; a.mode = MODE_RES;
    a.start = h->EC; a.start_stride = np; a.rout = h->levels[1].G; a.r_stride = np; a.norm_partial = h->norm_partial;
    nt = J;
    return true;
  }, b->down);
  int maxL = 0;
  for (mgrit_handle* h : b->hs) maxL = std::max(maxL, (int)h->levels.size());
  for (int d = 1; d < maxL; ++d) {
    for (int pass = 0; pass < 2; ++pass)
      add_relax_phases(b, 0, 1, [&](int q, LevelTables& T, RelaxArgs& a, int& nt) {
        mgrit_handle* h = b->hs[q];
        if ((int)h->levels.size() - 1 <= d) return false;
        Level& L = h->levels[d];
        Level& Lc = h->levels[d + 1];
        const int np = h->npts, m = Lc.m, J = L.nt / m;
        T = h->tables(d, 0);
        a = args0();
        a.m = m; a.J = J; a.nsteps = m; a.g = L.G;
        if (pass == 0) {
          a.mode = MODE_FC; a.cout = L.E; a.c_stride = (long long)m * np;
        } else {
          a.mode = MODE_RES; a.start = L.E; a.start_stride = (long long)m * np; a.g_at_c = 1; a.cin = L.E;
          a.c_stride = (long long)m * np; a.rout = Lc.G; a.r_stride = np;
        }
        nt = J;
        return true;
      }, b->down);
    // coarsest levels reached at this depth: sequential solves (band and other solves in separate phases)
    for (int cs : {2, 1}) {
      mgrit_batch::Phase ph{1, 0, cs, (int)b->tiles.size(), 0, 0, 0, 0, 0, 512};
      for (int q = 0; q < nprob; ++q) {
        mgrit_handle* h = b->hs[q];
        if ((int)h->levels.size() - 1 != d) continue;
        Level& L = h->levels[d];
        LevelTables T = h->tables(d, 0);
        if ((T.band > 0 ? 2 : 1) != cs) continue;
        T.err = b->d_err;
        SeqArgs sa{L.nt, L.G, nullptr, L.E, 1};
        const int ti = (int)b->tabs.size(), ai = (int)b->seqs.size();
        b->tabs.push_back(T);
        b->seqs.push_back(sa);
        int buf;
        size_t smem, region;
        relax_smem_need(T, 0, &buf, &smem, &region);
        ph.buf = std::max(ph.buf, buf);
        ph.region = std::max(ph.region, region);
        b->tiles.push_back(BatchTile{ti, ai, 0, q});
      }
      ph.ntiles = (int)b->tiles.size() - ph.tile_off;
      ph.smem = batched_smem(ph.buf, 0, ph.region);
      if (ph.ntiles) b->down.push_back(ph);
    }
  }
  for (int d = maxL - 2; d >= 1; --d)
    add_relax_phases(b, 0, 1, [&](int q, LevelTables& T, RelaxArgs& a, int& nt) {
      mgrit_handle* h = b->hs[q];
      if ((int)h->levels.size() - 1 <= d) return false;
      Level& L = h->levels[d];
      Level& Lc = h->levels[d + 1];
      const int np = h->npts, m = Lc.m, J = L.nt / m;
      T = h->tables(d, 0);
      a = args0();
      a.m = m; a.J = J; a.nsteps = m - 1; a.mode = MODE_POST; a.start = L.E; a.start_stride = (long long)m * np;
      a.corr = Lc.E; a.corr_stride = np; a.start_wb = L.E; a.wb_stride = (long long)m * np; a.extra_cta = 1;
      a.g = L.G; a.fstore = L.E;
      nt = J + 1;
      return true;
    }, b->up);
  b->final_args_off = (int)b->args.size();
  add_relax_phases(b, 2, 0, [&](int q, LevelTables& T, RelaxArgs& a, int& nt) {
    mgrit_handle* h = b->hs[q];
    const int np = h->npts, m1 = h->levels[1].m, J = h->J1();
    T = h->tables(0, 1);
    a = args0();
    a.m = m1; a.J = J; a.nsteps = m1 - 1; a.mode = MODE_POST; a.start = h->X; a.start_stride = np;
    a.wb_stride = (long long)m1 * np; a.extra_cta = 1;  // start_wb / fstore set per call
    nt = J + 1;
    return true;
  }, b->final_post);
  b->final_args.assign(b->hs.size(), -1);
  for (const auto& ph : b->final_post)
    for (int t = 0; t < ph.ntiles; ++t) b->final_args[b->tiles[ph.tile_off + t].problem] = b->tiles[ph.tile_off + t].args;
  auto up = [&](void** d, const void* h, size_t bytes) -> bool {
    if (bytes == 0) return true;
    if (cudaMalloc(d, bytes) != cudaSuccess) return false;
    return cudaMemcpyAsync(*d, h, bytes, cudaMemcpyHostToDevice, b->stream) == cudaSuccess;
  };
  bool ok = up((void**)&b->d_tabs, b->tabs.data(), b->tabs.size() * sizeof(LevelTables)) &&
            up((void**)&b->d_args, b->args.data(), b->args.size() * sizeof(RelaxArgs)) &&
            up((void**)&b->d_seq, b->seqs.data(), b->seqs.size() * sizeof(SeqArgs)) &&
            up((void**)&b->d_tiles, b->tiles.data(), b->tiles.size() * sizeof(BatchTile));
  ok = ok && cudaMalloc((void**)&b->d_active, nprob * sizeof(int)) == cudaSuccess &&
       cudaMalloc((void**)&b->d_seg, 3 * (size_t)nprob * sizeof(Segment)) == cudaSuccess &&
       cudaMalloc((void**)&b->d_norms, nprob * sizeof(double)) == cudaSuccess &&
       cudaMallocHost((void**)&b->h_norms, nprob * sizeof(double)) == cudaSuccess;
  ok = ok && cudaMallocHost((void**)&b->h_active, nprob * sizeof(int)) == cudaSuccess &&
       cudaMallocHost((void**)&b->h_seg, 3 * (size_t)nprob * sizeof(Segment)) == cudaSuccess;
  if (!ok || cudaStreamSynchronize(b->stream) != cudaSuccess) {
    delete b;
    return fail(MGRIT_ENOMEM, "batched workspace allocation failed");
  }
  for (mgrit_handle* h : b->hs) {
    b->maxn_all = std::max(b->maxn_all, (long long)(h->J1() + 1) * h->npts);
    b->setup_launches += h->setup_launches;
  }
  if (opt.profile) {  // two events per launch of one cycle (phases, batched update, sum) and the final pass
    b->ev.resize(2 * (b->down.size() + b->up.size() + b->final_post.size() + 2));
    for (auto& e : b->ev)
      if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return fail(MGRIT_ECUDA, "cudaEventCreate failed");
      }
  }
  {
    const mgrit_status st = tune_tile_order(b, grids, waves, orders, ms);
    if (st != MGRIT_OK) {
      delete b;
      return st;
    }
  }
  (void)t0;
  *out = b;
  return MGRIT_OK;
}

}  // extern "C"

namespace {

// Timing category (MGRIT_PHASE_*) of a batched phase.
int batch_phase_index(const mgrit_batch::Phase& ph) {
  if (ph.kind == 1) return MGRIT_PHASE_COARSEST;
  if (ph.coarse) return MGRIT_PHASE_COARSE;
  return ph.is_double ? MGRIT_PHASE_FINE64_RES : MGRIT_PHASE_FINE32_RES;
}

// The batched MGRIT iteration.  u0[q] / init[q] are device (kind DeviceToDevice) or host
// (HostToDevice) pointers; init_compact: init[q] holds only the C-point rows j = 1 .. J (row 0 first,
// ignored), else the full (nt + 1) x N iterate.  d_out[q] are device arrays.
mgrit_status batched_solve_impl(mgrit_batch* b, const double* const* u0, const double* const* init,
                                cudaMemcpyKind kind, bool init_compact, double* const* d_out, mgrit_stats* stats) {
  if (b->opt.fine_only) return fail(MGRIT_EUNSUPPORTED, "a fine_only batch has no MGRIT hierarchy");
  const double t0 = now_ms();
  cudaStream_t s = b->stream;
  const int nprob = (int)b->hs.size();
  for (int q = 0; q < nprob; ++q) {
    mgrit_handle* h = b->hs[q];
    const int np = h->npts, m1 = h->levels[1].m, J = h->J1();
    MG_CUDA(cudaMemcpyAsync(h->X, u0[q], np * sizeof(double), kind, s));
    if (init && init[q] && init_compact)
      MG_CUDA(cudaMemcpyAsync(h->X + np, init[q] + np, (size_t)J * np * sizeof(double), kind, s));
    else if (init && init[q])
      MG_CUDA(cudaMemcpy2DAsync(h->X + np, np * sizeof(double), init[q] + (size_t)m1 * np,
                                (size_t)m1 * np * sizeof(double), np * sizeof(double), J, kind, s));
    else
      MG_CUDA(cudaMemsetAsync(h->X + np, 0, (size_t)J * np * sizeof(double), s));
    // per-call output pointers of the final post F-relaxation
    RelaxArgs& a = b->args[b->final_args[q]];
    a.start_wb = d_out[q];
    a.fstore = d_out[q];
  }
  MG_CUDA(cudaMemcpyAsync(b->d_args + b->final_args_off, b->args.data() + b->final_args_off,
                          nprob * sizeof(RelaxArgs), cudaMemcpyHostToDevice, s));
  MG_CUDA(cudaMemsetAsync(b->d_err, 0, sizeof(int), s));  // a timeout of an earlier call is not this one's
  std::vector<int> active(nprob, 1), iters(nprob, 0), conv(nprob, 0);
  std::vector<double> r0(nprob, 0.0), rk(nprob, 0.0);
  std::vector<std::vector<double>> hist(nprob);
  const bool prof = !b->ev.empty();
  double phase_ms[MGRIT_NUM_PHASES] = {};
  int phase_n[MGRIT_NUM_PHASES] = {};
  std::vector<int> ev_phase;  // phase of each recorded event pair of the current cycle
  int64_t launches = 0;
  auto ev_begin = [&]() -> int {
    if (!prof || 2 * ev_phase.size() + 2 > b->ev.size()) return -1;
    const int i = (int)ev_phase.size();
    cudaEventRecord(b->ev[2 * i], s);
    return i;
  };
  auto ev_end = [&](int i, int phase) {
    ++launches;
    ++phase_n[phase];
    if (i < 0) return;
    cudaEventRecord(b->ev[2 * i + 1], s);
    ev_phase.push_back(phase);
  };
  auto ev_collect = [&]() {
    for (size_t i = 0; i < ev_phase.size(); ++i) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, b->ev[2 * i], b->ev[2 * i + 1]) == cudaSuccess) phase_ms[ev_phase[i]] += ms;
    }
    ev_phase.clear();
  };
  auto run = [&](const mgrit_batch::Phase& ph, int phase) -> mgrit_status {
    if (ph.ntiles == 0) return MGRIT_OK;
    const int e = ev_begin();
    cudaError_t err = ph.kind == 0
                          ? launch_relax_batched(b->d_tabs, b->d_args, b->d_tiles + ph.tile_off, ph.ntiles, b->d_active,
                                                 ph.is_double, ph.coarse, ph.buf, ph.smem, ph.threads, s)
                          : launch_sequential_batched(b->d_tabs, b->d_seq, b->d_tiles + ph.tile_off, ph.ntiles,
                                                      b->d_active, ph.is_double, ph.coarse, ph.buf, ph.smem, s);
    ev_end(e, phase);
    if (err != cudaSuccess) return fail(MGRIT_ECUDA, std::string("batched phase: ") + cudaGetErrorString(err));
    return MGRIT_OK;
  };
  // one cycle of every active problem; the active mask and the segment table are read from device memory
  // (uploaded before each cycle), so the cycle is the same launch sequence every time
  auto cycle = [&]() -> mgrit_status {
    for (auto& ph : b->down) MG_TRY(run(ph, batch_phase_index(ph)));  // down[0]: FP64 residual, e_C = r
    for (auto& ph : b->up) MG_TRY(run(ph, MGRIT_PHASE_COARSE));
    int e = ev_begin();
    launch_axpy_batched(8, b->d_seg + nprob, nprob, b->maxn_all, s);  // u_C = S^m u_C + E_1 (= u_C + r + E_1)
    ev_end(e, MGRIT_PHASE_MISC);
    e = ev_begin();
    launch_sum_batched(b->d_seg + 2 * nprob, nprob, s);
    ev_end(e, MGRIT_PHASE_MISC);
    MG_CUDA(cudaMemcpyAsync(b->h_norms, b->d_norms, nprob * sizeof(double), cudaMemcpyDeviceToHost, s));
    return MGRIT_OK;
  };
  // CUDA graph of one cycle (not while profiling: the events then surround each launch)
  bool graph_ok = b->opt.use_graph != 0 && !prof;
  int n_active = nprob;
  int64_t cycle_launches = 0;
  for (int k = 0; k < b->opt.max_iter && n_active > 0; ++k) {
    for (int q = 0; q < nprob; ++q) {
      mgrit_handle* h = b->hs[q];
      const long long n = active[q] ? (long long)h->J1() * h->npts : 0;  // C-points 1 .. J
      b->h_active[q] = active[q];
      b->h_seg[q] = Segment{nullptr, nullptr, nullptr, 0};
      b->h_seg[nprob + q] = Segment{h->r64 + h->npts, h->X + h->npts, (const float*)h->levels[1].E + h->npts, n};
      b->h_seg[2 * nprob + q] = Segment{h->norm_partial, b->d_norms + q, nullptr, active[q] ? (long long)h->J1() : 0};
    }
    MG_CUDA(cudaMemcpyAsync(b->d_active, b->h_active, nprob * sizeof(int), cudaMemcpyHostToDevice, s));
    MG_CUDA(cudaMemcpyAsync(b->d_seg, b->h_seg, 3 * (size_t)nprob * sizeof(Segment), cudaMemcpyHostToDevice, s));
    if (graph_ok && !b->graph) {  // capture the cycle once
      cudaGraph_t g = nullptr;
      const int64_t l0 = launches;
      int n0[MGRIT_NUM_PHASES];
      std::memcpy(n0, phase_n, sizeof(n0));
      if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        const mgrit_status st = cycle();
        const cudaError_t e = cudaStreamEndCapture(s, &g);
        if (st != MGRIT_OK) {
          if (g) cudaGraphDestroy(g);
          return st;
        }
        if (e != cudaSuccess || !g || cudaGraphInstantiate(&b->graph, g, 0) != cudaSuccess) b->graph = nullptr;
        if (g) cudaGraphDestroy(g);
      }
      cudaGetLastError();
      cycle_launches = launches - l0;  // the capture executed nothing
      launches = l0;
      std::memcpy(phase_n, n0, sizeof(n0));
      if (!b->graph) graph_ok = false;
    }
    if (graph_ok) {
      MG_CUDA(cudaGraphLaunch(b->graph, s));
      if (!cycle_launches) {  // captured by an earlier solve: count the launches of one cycle
        for (auto& ph : b->down) cycle_launches += ph.ntiles ? 1 : 0;
        for (auto& ph : b->up) cycle_launches += ph.ntiles ? 1 : 0;
        cycle_launches += 2;
      }
      launches += cycle_launches;
    } else {
      MG_TRY(cycle());
    }
    MG_CUDA(cudaStreamSynchronize(s));
    ev_collect();
    for (int q = 0; q < nprob; ++q) {
      if (!active[q]) continue;
      const double r = std::sqrt(b->h_norms[q]);
      hist[q].push_back(r);
      iters[q] = k + 1;
      rk[q] = r;
      if (k == 0) r0[q] = r;
      if (!std::isfinite(r) || (b->opt.diverge_ratio > 0.0 && r > b->opt.diverge_ratio * r0[q])) {
        active[q] = 0;
        --n_active;
      } else if (k >= 1 && r < b->opt.rtol * r0[q]) {
        conv[q] = 1;
        active[q] = 0;
        --n_active;
      }
    }
  }
  // every problem: post F-relaxation into its output
  for (int q = 0; q < nprob; ++q) b->h_active[q] = 1;
  MG_CUDA(cudaMemcpyAsync(b->d_active, b->h_active, nprob * sizeof(int), cudaMemcpyHostToDevice, s));
  for (auto& ph : b->final_post) MG_TRY(run(ph, MGRIT_PHASE_FINE64_POST));
  MG_CUDA(cudaStreamSynchronize(s));
  ev_collect();
  int timed_out = 0;
  MG_CUDA(cudaMemcpy(&timed_out, b->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  bool all_conv = true;
  for (int q = 0; q < nprob; ++q) {
    all_conv = all_conv && conv[q];
    if (stats) {
      mgrit_stats& st = stats[q];
      mgrit_handle* h = b->hs[q];
      std::memset(&st, 0, sizeof(st));
      st.iterations = iters[q];
      st.converged = conv[q];
      st.levels = (int)h->levels.size();
      st.r0 = r0[q];
      st.r_final = rk[q];
      st.history_len = std::min<int>(256, (int)hist[q].size());
      for (int i = 0; i < st.history_len; ++i) st.residual_history[i] = hist[q][i];
      st.setup_ms = h->setup_ms;
      st.solve_ms = now_ms() - t0;
      st.device_bytes = h->bytes;
      // setup phases: this problem's kernels; cycle phases: the batch's launches, which serve every problem
      st.kernel_launches = q == 0 ? b->setup_launches + launches : 0;
      for (int i = 0; i < MGRIT_NUM_PHASES; ++i) {
        const bool setup_phase = i <= MGRIT_PHASE_FACTOR;
        st.phase_ms[i] = setup_phase ? h->setup_phase_ms[i] : phase_ms[i];
        st.phase_launches[i] = setup_phase ? h->setup_phase_launches[i] : phase_n[i];
      }
    }
  }
  if (timed_out) return fail(MGRIT_ETIMEOUT, "a bounded device wait gave up (TMA staging did not complete)");
  return all_conv ? MGRIT_OK : fail(MGRIT_ENOTCONVERGED, "some problems did not converge");
}

}  // namespace

extern "C" {

mgrit_status mgrit_solve_batched(mgrit_batch* b, const double* const* d_u0, const double* const* d_u_init,
                                 double* const* d_u_out, mgrit_stats* stats) {
  if (!b || !d_u0 || !d_u_out) return fail(MGRIT_EINVAL, "NULL argument");
  for (size_t q = 0; q < b->hs.size(); ++q)
    if (!d_u0[q] || !d_u_out[q]) return fail(MGRIT_EINVAL, "NULL problem buffer");
  return batched_solve_impl(b, d_u0, d_u_init, cudaMemcpyDeviceToDevice, false, d_u_out, stats);
}

mgrit_status mgrit_solve_batched_host(mgrit_batch* b, const double* const* h_u0, const double* const* h_u_init_c,
                                      double* const* h_u_out, mgrit_stats* stats) {
  if (!b || !h_u0 || !h_u_out) return fail(MGRIT_EINVAL, "NULL argument");
  const int nprob = (int)b->hs.size();
  size_t total = 0;
  for (int q = 0; q < nprob; ++q) {
    if (!h_u0[q] || !h_u_out[q]) return fail(MGRIT_EINVAL, "NULL problem buffer");
    total += (size_t)(b->hs[q]->grid.nt + 1) * b->hs[q]->npts;
  }
  cudaStream_t s = b->stream;
  double* d = nullptr;
  MG_CUDA(scratch_alloc((void**)&d, total * sizeof(double), s));
  std::vector<double*> outs(nprob);
  size_t off = 0;
  for (int q = 0; q < nprob; ++q) {
    outs[q] = d + off;
    off += (size_t)(b->hs[q]->grid.nt + 1) * b->hs[q]->npts;
  }
  mgrit_status st = batched_solve_impl(b, h_u0, h_u_init_c, cudaMemcpyHostToDevice, true, outs.data(), stats);
  for (int q = 0; q < nprob; ++q)
    cudaMemcpyAsync(h_u_out[q], outs[q], (size_t)(b->hs[q]->grid.nt + 1) * b->hs[q]->npts * sizeof(double),
                    cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(d, s);
  MG_CUDA(cudaStreamSynchronize(s));
  return st;
}

mgrit_status sl_step_sequential_batched(mgrit_batch* b, const double* const* d_u0, double* const* d_u_out) {
  if (!b || !d_u0 || !d_u_out) return fail(MGRIT_EINVAL, "NULL argument");
  const int nprob = (int)b->hs.size();
  for (int q = 0; q < nprob; ++q)
    if (!d_u0[q] || !d_u_out[q]) return fail(MGRIT_EINVAL, "NULL problem buffer");
  cudaStream_t s = b->stream;
  const int dbl = b->opt.precision == 0;  // FP64 (fine_only batches of precision 0) or FP32 stepping
  size_t total = 0;
  for (mgrit_handle* h : b->hs) total += h->npts;
  float* f = nullptr;  // FP32 stepping: the start slices, then the final slices
  if (!dbl) MG_CUDA(scratch_alloc((void**)&f, 2 * total * sizeof(float), s));
  std::vector<LevelTables> tabs(nprob);
  std::vector<SeqArgs> args(nprob);
  std::vector<BatchTile> tiles(nprob);
  std::vector<Segment> seg(2 * nprob);
  int buf = 0;
  size_t region = 0;
  size_t off = 0;
  long long maxn = 0;
  for (int q = 0; q < nprob; ++q) {
    mgrit_handle* h = b->hs[q];
    tabs[q] = h->tables(0, dbl);
    tabs[q].solver = nullptr;
    tabs[q].err = b->d_err;
    if (dbl) args[q] = SeqArgs{h->grid.nt, nullptr, d_u0[q], d_u_out[q], 0};
    else args[q] = SeqArgs{h->grid.nt, nullptr, f + off, f + total + off, 0};
    tiles[q] = BatchTile{q, q, 0, q};
    seg[q] = Segment{d_u0[q], f ? f + off : nullptr, nullptr, h->npts};
    seg[nprob + q] = Segment{f ? f + total + off : nullptr, d_u_out[q], nullptr, h->npts};
    off += h->npts;
    maxn = std::max(maxn, (long long)h->npts);
    int bq;
    size_t smq, rq;
    relax_smem_need(tabs[q], dbl, &bq, &smq, &rq);
    buf = std::max(buf, bq);
    region = std::max(region, rq);
  }
  // one device block for the per-problem launch records (stream-ordered, freed below)
  const size_t tb = nprob * sizeof(LevelTables), ab = nprob * sizeof(SeqArgs), ib = nprob * sizeof(BatchTile),
               sb = 2 * nprob * sizeof(Segment);
  char* rec = nullptr;
  MG_CUDA(scratch_alloc((void**)&rec, tb + ab + ib + sb, s));
  std::vector<char> hrec(tb + ab + ib + sb);
  std::memcpy(hrec.data(), tabs.data(), tb);
  std::memcpy(hrec.data() + tb, args.data(), ab);
  std::memcpy(hrec.data() + tb + ab, tiles.data(), ib);
  std::memcpy(hrec.data() + tb + ab + ib, seg.data(), sb);
  MG_CUDA(cudaMemsetAsync(b->d_err, 0, sizeof(int), s));
  MG_CUDA(cudaMemcpyAsync(rec, hrec.data(), hrec.size(), cudaMemcpyHostToDevice, s));
  const Segment* d_seg = (const Segment*)(rec + tb + ab + ib);
  if (!dbl) launch_axpy_batched(1, d_seg, nprob, maxn, s);  // FP64 -> FP32 start slices
  MG_CUDA(launch_sequential_batched((const LevelTables*)rec, (const SeqArgs*)(rec + tb), (const BatchTile*)(rec + tb + ab),
                                    nprob, nullptr, dbl, 0, buf, batched_smem(buf, dbl, region), s));
  if (!dbl) launch_axpy_batched(3, d_seg + nprob, nprob, maxn, s);  // FP32 -> FP64 final slices
  MG_CUDA(cudaGetLastError());
  // the host record must outlive the copy
  MG_CUDA(cudaStreamSynchronize(s));
  cudaFreeAsync(rec, s);
  if (f) cudaFreeAsync(f, s);
  MG_CUDA(cudaStreamSynchronize(s));
  int timed_out = 0;
  MG_CUDA(cudaMemcpy(&timed_out, b->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (timed_out) return fail(MGRIT_ETIMEOUT, "a bounded device wait gave up (TMA staging did not complete)");
  return MGRIT_OK;
}

void mgrit_destroy_batched(mgrit_batch* b) { delete b; }

const char* mgrit_status_string(mgrit_status s) {
  switch (s) {
    case MGRIT_OK: return "ok";
    case MGRIT_EINVAL: return "invalid argument";
    case MGRIT_ENOMEM: return "out of device memory";
    case MGRIT_ECUDA: return "CUDA error";
    case MGRIT_ENOTCONVERGED: return "not converged";
    case MGRIT_EDIVERGED: return "diverged";
    case MGRIT_ETIMEOUT: return "device wait timed out";
    case MGRIT_EUNSUPPORTED: return "unsupported";
    case MGRIT_ESINGULAR: return "singular correction matrix";
  }
  return "unknown status";
}

const char* mgrit_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
