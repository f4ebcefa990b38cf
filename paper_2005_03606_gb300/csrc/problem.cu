// Problem lifecycle, V-cycle and outer-loop orchestration, delayed assembly
// and the C ABI entry points for single problems (declared in include/mg.h).
//
// Level l = 0 is the finest grid (N cells per axis), level L-1 the coarsest
// (3 cells per axis).  The finest operator is split into chunks of whole cell
// layers along the last axis; each chunk holds the stencils of one accuracy s
// and is replaced as a unit when a better one has been assembled (the
// marker p1 of Section "Stencil assembly variants" per chunk; the in-flight
// marker p2 is the chunk's pending job).  Coarse levels hold element matrices
// produced by the Galerkin kernel.
#include "mg_internal.cuh"
#include "mg.h"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

namespace mg {

static thread_local std::string t_err;

void set_error(const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  t_err = buf;
}

bool cuda_ok(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return true;
  set_error("%s: %s", what, cudaGetErrorString(e));
  return false;
}

const char* last_error() { return t_err.c_str(); }

static std::atomic<long long> g_launches{0};
static thread_local long long t_launches = 0;
void count_launches(long long n) {
  g_launches.fetch_add(n, std::memory_order_relaxed);
  t_launches += n;
}
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }
long long thread_launch_count() { return t_launches; }

}  // namespace mg

using namespace mg;

#define MG_CHECK(call)                              \
  do {                                              \
    cudaError_t e_ = (call);                        \
    if (e_ != cudaSuccess) {                        \
      set_error("%s: %s", #call, cudaGetErrorString(e_)); \
      return MG_ERR_CUDA;                           \
    }                                               \
  } while (0)

namespace {

struct ChunkStore {
  int s = 0;
  void* a64 = nullptr;            // FP64 full storage [NP][chunk_cells]
  uint8_t* cls = nullptr;         // compressed: padded classes
  uint32_t* seg_base = nullptr;   // compressed: [3][nseg]
  uint8_t* pool[3] = {nullptr, nullptr, nullptr};
  uint32_t totals[3] = {0, 0, 0};
  size_t bytes = 0;
  double* x64 = nullptr;          // exact mode: FP64 surplus [interface list][NP] (nullptr at s = 1)
};

struct Level {
  int N = 0;
  long long ncell = 0, nvert = 0;
  LevelOp op{};
  FullChunk* d_full = nullptr;
  CmpChunk* d_cmp = nullptr;
  void* full_store = nullptr;     // coarse levels: single chunk
  void* stencil = nullptr;        // assembled vertex stencils (levels with full storage)
  void* b = nullptr;              // V-cycle right-hand side (TV)
  void* x0 = nullptr;             // V-cycle iterates (TV)
  void* x1 = nullptr;
  float* eps_c = nullptr;         // coarse compression: eps at the cell centres (FP32)
  uint8_t* cls = nullptr;         // coarse compression: storage class per cell
  bool u1_ready = false;          // x1 holds omega D^-1 b (written with b by the restriction)
};

struct Job {
  int s = 0, chunk = 0;
  cudaEvent_t ev = nullptr;
  ChunkStore store;
  int status = MG_OK;
  std::string msg;   // the worker thread's error message when status != MG_OK
};

}  // namespace

struct mg_problem {
  mg_problem_desc desc{};
  EpsDev eps{};
  int dim = 0, N = 0, L = 0;
  int device = 0;                 // CUDA device current at creation
  bool mixed = false, delayed = false;
  cudaStream_t st = nullptr, side = nullptr;
  bool own_stream = false;
  size_t tv = 8;                  // V-cycle vector element size
  std::vector<Level> lev;
  // finest-level chunking
  int nchunk = 1, layers = 1, nseg_x = 1;
  long long chunk_cells = 0, chunk_rows = 0, chunk_nseg = 0;
  std::vector<ChunkStore> cur;
  std::vector<FullChunk> h_full;
  std::vector<CmpChunk> h_cmp;
  void* eps_c = nullptr;          // float (mixed) or double per cell
  // outer FP64 vectors
  double *u = nullptr, *f = nullptr, *r = nullptr, *p = nullptr, *q = nullptr;
  double* partials = nullptr;
  long long npartials = 0;
  DevScalars* sc = nullptr;
  DevScalars* h_sc = nullptr;     // pinned
  // mg_solve's iteration pipeline: pinned scalar slots and events of the
  // iteration being tested and of one enqueued ahead of the test
  DevScalars* h_slot[2] = {nullptr, nullptr};
  cudaEvent_t slot_ev[2] = {nullptr, nullptr};
  bool speculate = true;          // mixed flexible CG: enqueue the next iteration before testing this one
  double rin_hist[2] = {-1.0, -1.0};  // inner residuals of the last two iterations since the last restart
  double* Lc = nullptr;           // coarse Cholesky factor, then the coarse inverse
  uint8_t* scratch = nullptr;     // assembly records of one chunk (mixed)
  // interface cells per chunk (fields with piecewise-constant eps): only these
  // are integrated at s > 1, every other cell keeps its geometric stencil
  // exact FP64 operator of the mixed paths on piecewise-constant fields
  bool exact = false;
  double* eps64 = nullptr;        // FP64 cell-centre eps
  int* xpos = nullptr;            // per cell: position in its chunk's interface list, -1 if none
  int* touched64 = nullptr;       // 3D split residual: vertices next to an interface cell
  int* ntouched64 = nullptr;
  int* ilist = nullptr;           // [nchunk][chunk_cells] local cell indices
  std::vector<int> ilist_n;       // count per chunk (host)
  std::vector<mg_trace_entry> trace_log;   // per outer iteration of the last solve
  bool resid_fresh = false;       // rr is the true FP64 residual of the current u and operator
  bool u_zero = true;             // u is still the zero initial guess
  // adaptive accuracy (desc.adapt_C > 0)
  bool adapt = false;
  uint8_t* final_flags = nullptr; // [nchunk][chunk_cells]: 1 once the cell stopped refining
  uint8_t* s_cell = nullptr;      // [nchunk][chunk_cells]: accuracy of the cell's latest matrix
  int* awork = nullptr;           // work list of one chunk
  int* anwork = nullptr;          // its length (device)
  std::vector<ChunkStore> wlast;  // latest store integrated per chunk (published or not)
  uint32_t* d_totals = nullptr;   // per stream: [0..2] main, [4..6] side
  uint32_t* h_totals = nullptr;   // pinned, same layout
  // mixed 3D finest level: vertices touched by cells with a surplus record
  int* touched = nullptr;
  int* ntouched = nullptr;
  uint8_t* tflags = nullptr;
  uint32_t* tcounts = nullptr;
  float* tcoef = nullptr;
  float* eps_pad = nullptr;
  // fused residual + restriction on that level: touched-vertex bit mask,
  // z-restricted residual planes
  uint32_t* tmask = nullptr;
  float* zr = nullptr;
  // mixed paths: FP32 inner solve (iterative refinement)
  float *p32 = nullptr, *q32 = nullptr, *e32 = nullptr;
  // w32 = omega D^-1 of the finest level (rebuilt after every change of its
  // operator, w_dirty): the restart's residual scaling and every flexible-CG
  // update also write u1 = w32 r_in into lev[0].x1, the next V-cycle's first
  // smoothing step from the zero iterate (u1_ready until a V-cycle uses it)
  float* w32 = nullptr;
  bool w_dirty = true;
  bool w_ok = false;
  bool u1_ready = false;
  // V-cycle enqueue: when set, the finest level's last post-smoothing sweep
  // also forms z . vdot_q (its partials, vdot_nb of them, left in partials)
  const float* vdot_q = nullptr;
  bool vdot_done = false;
  int vdot_nb = 0;
  int inner_its = 0;
  int last_inner_its = 0;
  bool have_correction = false;
  bool e_pending = false;         // e32 still lacks the last step alpha p (FP32 flexible CG)
  bool trace = false;             // MG_TRACE: outer-loop trace on stderr
  double eta_min = 1e-2;          // smallest relative reduction asked of one FP32 inner solve
  double eta2 = 1e-10;            // inner tolerance (squared, relative to the unit-scaled residual)
  std::vector<void*> allocs;      // long-lived device allocations
  // outer-loop state
  bool first = true, need_restart = true;
  bool keep_dir = false;          // next restart is a reliable update (see outer_restart)
  double ff = 0.0, rr = 0.0, rr_first = 0.0;
  int cycles = 0, publishes = 0;
  cudaGraphExec_t g_iter[2] = {nullptr, nullptr};
  long long g_kernels[2] = {0, 0};   // kernels per graph replay
  bool use_graphs = true;
  // delayed assembly
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Job> todo, ready;
  std::vector<Job> held;          // finished jobs not yet published (see publish_ready)
  int held_since = -1;            // cycle at which the oldest held job was taken
  int in_flight = 0;
  bool stop = false;
  int inject_fail = 0;
};

namespace {

int ipow3(int L) {
  int r = 1;
  while (L-- > 0) r *= 3;
  return r;
}

}  // namespace

cudaError_t mg::mg_malloc_async(void** p, size_t bytes, cudaStream_t st) {
  static std::mutex mu;
  static cudaMemPool_t pools[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaMallocAsync(p, bytes, st);
  cudaMemPool_t pool;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (!pools[dev]) {
      cudaMemPoolProps props = {};
      props.allocType = cudaMemAllocationTypePinned;
      props.location.type = cudaMemLocationTypeDevice;
      props.location.id = dev;
      cudaMemPool_t np;
      e = cudaMemPoolCreate(&np, &props);
      if (e != cudaSuccess) return cudaMallocAsync(p, bytes, st);
      unsigned long long keep = ~0ull;
      cudaMemPoolSetAttribute(np, cudaMemPoolAttrReleaseThreshold, &keep);
      pools[dev] = np;
    }
    pool = pools[dev];
  }
  return cudaMallocFromPoolAsync(p, bytes, pool, st);
}

namespace {

template <typename T>
cudaError_t dalloc(mg_problem* P, T** ptr, size_t bytes, bool track = true) {
  void* p = nullptr;
  cudaError_t e = mg_malloc_async(&p, bytes ? bytes : 16, P->st);
  if (e != cudaSuccess) return e;
  *ptr = (T*)p;
  if (track) P->allocs.push_back(p);
  return cudaSuccess;
}

mg_status oom_or_cuda(cudaError_t e, const char* what) {
  set_error("%s: %s", what, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? MG_ERR_OOM : MG_ERR_CUDA;
}

void fill_eps(const mg_eps_desc& d, int dim, EpsDev* e) {
  memset(e, 0, sizeof(*e));
  e->kind = d.kind;
  e->dim = dim;
  e->n_modes = d.n_modes;
  e->n_boxes = d.n_boxes;
  e->v_out = d.v_out;
  e->v_in = d.v_in;
  for (int a = 0; a < 3; ++a) e->center[a] = d.center[a];
  e->r2lim = d.radius * d.radius;
  e->amp = d.n_modes > 0 ? d.sigma * std::sqrt(2.0 / d.n_modes) : 0.0;
  e->theta = d.theta;
  e->jump_x = d.jump_x;
  e->jump_factor = d.jump_factor;
  for (int m = 0; m < MG_MAX_MODES; ++m) {
    for (int a = 0; a < 3; ++a) e->k[m][a] = d.k[m][a];
    e->phi_over_pi[m] = d.phase[m] / 3.14159265358979323846;
  }
  for (int b = 0; b < MG_MAX_BOXES; ++b)
    for (int a = 0; a < 3; ++a) {
      e->box_lo[b][a] = d.box_lo[b][a];
      e->box_hi[b][a] = d.box_hi[b][a];
    }
  e->amp_f = (float)e->amp;
  e->v_out_f = (float)e->v_out;
  e->v_in_f = (float)e->v_in;
  e->jump_factor_f = (float)e->jump_factor;
  for (int m = 0; m < MG_MAX_MODES; ++m) e->phi_over_pi_f[m] = (float)e->phi_over_pi[m];
}

// Checks of an eps descriptor shared by problem creation and the
// allocation-free assembly: kind, mode and box counts within the device
// tables, wavenumbers, positive values.
mg_status validate_eps(const mg_eps_desc& e) {
  if (e.kind < 0 || e.kind > 4) {
    set_error("unknown eps kind %d", e.kind);
    return MG_ERR_INVALID;
  }
  if (e.kind == MG_EPS_FOURIER && (e.n_modes < 1 || e.n_modes > MG_MAX_MODES)) {
    set_error("n_modes out of range");
    return MG_ERR_INVALID;
  }
  if (e.kind == MG_EPS_FOURIER)
    for (int m = 0; m < e.n_modes; ++m)
      for (int a = 0; a < 3; ++a)
        if (std::abs(e.k[m][a]) > 64) {
          set_error("wavenumber component above 64");
          return MG_ERR_INVALID;
        }
  if (e.kind == MG_EPS_BOXES && (e.n_boxes < 1 || e.n_boxes > MG_MAX_BOXES)) {
    set_error("n_boxes out of range");
    return MG_ERR_INVALID;
  }
  if (!(e.jump_factor > 0.0) || !(e.v_out > 0.0)) {
    set_error("eps must be positive");
    return MG_ERR_INVALID;
  }
  if ((e.kind == MG_EPS_DISC || e.kind == MG_EPS_BOXES) && !(e.v_in > 0.0)) {
    set_error("eps must be positive");
    return MG_ERR_INVALID;
  }
  return MG_OK;
}

mg_status validate(const mg_problem_desc* d) {
  if (!d) {
    set_error("null descriptor");
    return MG_ERR_INVALID;
  }
  if (d->dim != 2 && d->dim != 3) {
    set_error("dim must be 2 or 3 (got %d)", d->dim);
    return MG_ERR_INVALID;
  }
  int n = d->n_cells;
  if (n < 9) {
    set_error("n_cells must be 3^L with L >= 2 (got %d)", n);
    return MG_ERR_INVALID;
  }
  while (n % 3 == 0 && n > 1) n /= 3;
  if (n != 1) {
    set_error("n_cells must be a power of 3 (got %d)", d->n_cells);
    return MG_ERR_INVALID;
  }
  if (d->dim == 3 && d->n_cells > 729) {
    set_error("3D n_cells above 729 not supported");
    return MG_ERR_INVALID;
  }
  if (d->dim == 2 && d->n_cells > 19683) {
    set_error("2D n_cells above 19683 not supported");
    return MG_ERR_INVALID;
  }
  if (!(d->adapt_C >= 0.0) || !std::isfinite(d->adapt_C)) {
    set_error("adapt_C must be a finite value >= 0");
    return MG_ERR_INVALID;
  }
  if (d->adapt_keep != 0 && d->adapt_keep != 1) {
    set_error("adapt_keep must be 0 or 1");
    return MG_ERR_INVALID;
  }
  if (validate_eps(d->eps) != MG_OK) return MG_ERR_INVALID;
  if (d->n_s < 1 || d->n_s > 8) {
    set_error("n_s must be 1..8");
    return MG_ERR_INVALID;
  }
  for (int i = 0; i < d->n_s; ++i) {
    if (d->s_schedule[i] < 1 || d->s_schedule[i] > 64 || (i && d->s_schedule[i] <= d->s_schedule[i - 1])) {
      set_error("s_schedule must increase within 1..64");
      return MG_ERR_INVALID;
    }
  }
  if (!(d->coarse_tau >= 0.0) || !std::isfinite(d->coarse_tau) ||
      (d->coarse_tau > 0.0 && d->path != MG_PATH_MIXED_DELAYED && d->path != MG_PATH_MIXED_PLAIN)) {
    set_error("coarse_tau must be finite, >= 0, and 0 on the FP64 paths");
    return MG_ERR_INVALID;
  }
  if (d->cycle < MG_CYCLE_V || d->cycle > MG_CYCLE_ADAFAC_JAC) {
    set_error("unknown cycle %d", d->cycle);
    return MG_ERR_INVALID;
  }
  if (d->path < 0 || d->path > 3) {
    set_error("unknown path %d", d->path);
    return MG_ERR_INVALID;
  }
  return MG_OK;
}

LevelOp& fine_op(mg_problem* P) { return P->lev[0].op; }

// ------------------------------------------------------------ assembly of one chunk
// Adaptive accuracy (Section "Adaptive stencil integration"): a level s of a
// chunk is judged against the chunk's previous level once that one is at
// least the first level of the schedule; the first judged level is the one
// right after it.
bool adaptive_judged(const mg_problem* P, int s, int chunk) {
  return P->adapt && s > 1 && P->wlast[chunk].s >= P->desc.s_schedule[0];
}
int adaptive_first(const mg_problem* P, int chunk) { return P->wlast[chunk].s == P->desc.s_schedule[0]; }

mg_status assemble_chunk(mg_problem* P, int s, int chunk, cudaStream_t st, ChunkStore* out, int tot_slot) {
  const int D = P->dim;
  const int NP = D == 3 ? 28 : 6;
  const long long cell0 = (long long)chunk * P->chunk_cells;
  ChunkStore cs;
  cs.s = s;
  if (!P->mixed) {
    cudaError_t e = mg_malloc_async(&cs.a64, sizeof(double) * NP * P->chunk_cells, st);
    if (e != cudaSuccess) return oom_or_cuda(e, "chunk storage");
    cs.bytes = sizeof(double) * NP * P->chunk_cells;
    if (s == 1 || P->ilist) {
      MG_CHECK(launch_geometric_full(D, P->N, fine_op(P).hfac, (const double*)P->eps_c, cell0, P->chunk_cells,
                                     (double*)cs.a64, st));
    }
    const bool judge = adaptive_judged(P, s, chunk);
    long long nwork = -1;   // adaptive: cells still refining in this chunk
    if (judge) {
      const size_t off = (size_t)chunk * P->chunk_cells;
      MG_CHECK(launch_adaptive_prepare(D, P->N, P->nseg_x, P->chunk_cells, 1, P->final_flags + off, CmpChunk{},
                                       (const double*)P->wlast[chunk].a64, nullptr, nullptr, (double*)cs.a64,
                                       P->ilist ? P->ilist + off : nullptr,
                                       P->ilist ? P->ilist_n[chunk] : P->chunk_cells, P->awork, P->anwork,
                                       P->s_cell + off, s, adaptive_first(P, chunk) && !P->desc.adapt_keep, st));
      int h = 0;
      MG_CHECK(cudaMemcpyAsync(&h, P->anwork, sizeof(int), cudaMemcpyDeviceToHost, st));
      MG_CHECK(cudaStreamSynchronize(st));
      nwork = h;
    } else if (P->adapt && s > 1) {
      MG_CHECK(cudaMemsetAsync(P->s_cell + (size_t)chunk * P->chunk_cells, s, P->chunk_cells, st));
    }
    if (s > 1 && (judge ? nwork > 0 : (!P->ilist || P->ilist_n[chunk] > 0))) {
      AsmLaunch a{};
      a.dim = D;
      a.N = P->N;
      a.s = s;
      a.kind = P->eps.kind;
      a.prec64 = 1;
      a.cell0 = cell0;
      a.ncell = P->chunk_cells;
      a.eps_host = &P->eps;
      a.hfac = fine_op(P).hfac;
      a.eps_c = P->eps_c;
      a.out_full = cs.a64;
      a.nseg_x = P->nseg_x;
      a.tau = 0;
      if (judge) {
        const size_t off = (size_t)chunk * P->chunk_cells;
        a.list = P->awork;
        a.nlist = nwork;
        a.prev_full = (const double*)P->wlast[chunk].a64;
        a.final_flags = P->final_flags + off;
        a.s_cell = P->s_cell + off;
        a.adapt_C = P->desc.adapt_C;
        a.adapt_keep = P->desc.adapt_keep;
      } else if (P->ilist) {
        a.list = P->ilist + (size_t)chunk * P->chunk_cells;
        a.nlist = P->ilist_n[chunk];
      }
      MG_CHECK(launch_assemble(a, st));
    }
    if (P->adapt) P->wlast[chunk] = cs;
    *out = cs;
    return MG_OK;
  }
  const size_t cls_bytes = (size_t)P->chunk_nseg * kSegCells;
  cudaError_t e = mg_malloc_async(&cs.cls, cls_bytes, st);
  if (e == cudaSuccess) e = mg_malloc_async(&cs.seg_base, sizeof(uint32_t) * 3 * P->chunk_nseg, st);
  if (e != cudaSuccess) return oom_or_cuda(e, "chunk classes");
  MG_CHECK(cudaMemsetAsync(cs.cls, 0, cls_bytes, st));
  cs.bytes = cls_bytes + sizeof(uint32_t) * 3 * P->chunk_nseg;
  if (s == 1) {
    MG_CHECK(cudaMemsetAsync(cs.seg_base, 0, sizeof(uint32_t) * 3 * P->chunk_nseg, st));
    *out = cs;
    return MG_OK;
  }
  AsmLaunch a{};
  a.dim = D;
  a.N = P->N;
  a.s = s;
  a.kind = P->eps.kind;
  a.prec64 = 0;
  a.cell0 = cell0;
  a.ncell = P->chunk_cells;
  a.eps_host = &P->eps;
  a.hfac = fine_op(P).hfac;
  a.eps_c = P->eps_c;
  a.out_rec = P->scratch;
  a.out_cls = cs.cls;
  a.nseg_x = P->nseg_x;
  a.tau = P->desc.compress_tau;
  const bool judge = adaptive_judged(P, s, chunk);
  if (P->adapt && !judge) MG_CHECK(cudaMemsetAsync(P->s_cell + (size_t)chunk * P->chunk_cells, s, P->chunk_cells, st));
  if (judge) {
    // final cells keep their previous record; the others not final are integrated
    const ChunkStore& pv = P->wlast[chunk];
    CmpChunk prev{};
    prev.cls = pv.cls;
    prev.seg_base = pv.seg_base;
    for (int k = 0; k < 3; ++k) prev.pool[k] = pv.pool[k];
    prev.nseg = P->chunk_nseg;
    const size_t off = (size_t)chunk * P->chunk_cells;
    MG_CHECK(launch_adaptive_prepare(D, P->N, P->nseg_x, P->chunk_cells, 0, P->final_flags + off, prev, nullptr,
                                     P->scratch, cs.cls, nullptr, P->ilist ? P->ilist + off : nullptr,
                                     P->ilist ? P->ilist_n[chunk] : P->chunk_cells, P->awork, P->anwork,
                                     P->s_cell + off, s, adaptive_first(P, chunk) && !P->desc.adapt_keep, st));
    int h = 0;
    MG_CHECK(cudaMemcpyAsync(&h, P->anwork, sizeof(int), cudaMemcpyDeviceToHost, st));
    MG_CHECK(cudaStreamSynchronize(st));
    a.list = P->awork;
    a.nlist = h;
    a.prev_cmp = prev;
    a.final_flags = P->final_flags + off;
    a.s_cell = P->s_cell + off;
    a.adapt_C = P->desc.adapt_C;
    a.adapt_keep = P->desc.adapt_keep;
  } else if (P->ilist) {   // only the interface cells can carry a surplus (the class bytes start at 0)
    a.list = P->ilist + (size_t)chunk * P->chunk_cells;
    a.nlist = P->ilist_n[chunk];
  }
  if (P->exact && P->ilist_n[chunk] > 0) {
    // FP64 integration of the interface cells; the exact surplus goes to the
    // store's list-ordered FP64 array (adaptive: final cells keep the
    // previous level's entries)
    const size_t xb = sizeof(double) * NP * (size_t)P->ilist_n[chunk];
    if ((e = mg_malloc_async(&cs.x64, xb, st)) != cudaSuccess) return oom_or_cuda(e, "exact surplus");
    cs.bytes += xb;
    const double* px = judge ? P->wlast[chunk].x64 : nullptr;
    if (px) MG_CHECK(cudaMemcpyAsync(cs.x64, px, xb, cudaMemcpyDeviceToDevice, st));
    else if (judge) MG_CHECK(cudaMemsetAsync(cs.x64, 0, xb, st));
    a.eps64 = P->eps64;
    a.out_x64 = cs.x64;
    a.xpos = P->xpos;
    a.prev_x64 = px;
  }
  if ((!P->ilist && !judge) || a.nlist > 0) MG_CHECK(launch_assemble(a, st));
  uint32_t* dt = P->d_totals + tot_slot;
  uint32_t* ht = P->h_totals + tot_slot;
  MG_CHECK(launch_pack_count(D, P->N, P->chunk_rows, P->nseg_x, cs.cls, cs.seg_base, dt, st));
  MG_CHECK(cudaMemcpyAsync(ht, dt, sizeof(uint32_t) * 3, cudaMemcpyDeviceToHost, st));
  MG_CHECK(cudaStreamSynchronize(st));
  const int rb[3] = {D == 3 ? 32 : 16, D == 3 ? 64 : 16, D == 3 ? 112 : 32};
  for (int k = 0; k < 3; ++k) {
    cs.totals[k] = ht[k];
    if (ht[k]) {
      e = mg_malloc_async(&cs.pool[k], (size_t)ht[k] * rb[k], st);
      if (e != cudaSuccess) return oom_or_cuda(e, "payload pool");
      cs.bytes += (size_t)ht[k] * rb[k];
    }
  }
  MG_CHECK(launch_pack_copy(D, P->N, P->chunk_rows, P->nseg_x, cs.cls, cs.seg_base, P->scratch, cs.pool[0],
                            cs.pool[1], cs.pool[2], st));
  if (P->adapt) P->wlast[chunk] = cs;
  *out = cs;
  return MG_OK;
}

void free_store(ChunkStore& cs, cudaStream_t st) {
  if (cs.a64) cudaFreeAsync(cs.a64, st);
  if (cs.cls) cudaFreeAsync(cs.cls, st);
  if (cs.seg_base) cudaFreeAsync(cs.seg_base, st);
  for (int k = 0; k < 3; ++k)
    if (cs.pool[k]) cudaFreeAsync(cs.pool[k], st);
  if (cs.x64) cudaFreeAsync(cs.x64, st);
  cs = ChunkStore();
}

// install a store as the published operator of a chunk (host mirror only)
void install(mg_problem* P, int chunk, const ChunkStore& cs) {
  free_store(P->cur[chunk], P->st);   // stream-ordered: kernels already queued keep the old store
  P->cur[chunk] = cs;
  if (P->mixed) {
    CmpChunk c{};
    c.cls = cs.cls;
    c.seg_base = cs.seg_base;
    for (int k = 0; k < 3; ++k) c.pool[k] = cs.pool[k];
    c.nseg = P->chunk_nseg;
    c.x64 = cs.x64;
    P->h_cmp[chunk] = c;
  } else {
    P->h_full[chunk].a = cs.a64;
  }
}

mg_status upload_tables(mg_problem* P) {
  Level& l0 = P->lev[0];
  if (P->mixed)
    MG_CHECK(cudaMemcpyAsync(l0.d_cmp, P->h_cmp.data(), sizeof(CmpChunk) * P->nchunk, cudaMemcpyHostToDevice, P->st));
  else
    MG_CHECK(cudaMemcpyAsync(l0.d_full, P->h_full.data(), sizeof(FullChunk) * P->nchunk, cudaMemcpyHostToDevice,
                             P->st));
  // pageable source: the copy is staged before return, the host mirror may change afterwards
  if (P->touched) {
    MG_CHECK(launch_build_touched(l0.op, P->tflags, P->tcounts, P->touched, P->ntouched, P->st));
  }
  if (l0.stencil) MG_CHECK(launch_build_stencil(l0.op, l0.stencil, P->st));
  P->w_dirty = true;
  return MG_OK;
}

// w32 = omega D^-1 of the finest level's FP32 operator: the zero-iterate
// smoothing step applied to a vector of ones (the same kernels, so u1 = w32 b
// is that step for any b up to one rounding)
mg_status build_w(mg_problem* P) {
  P->w_dirty = false;
  P->w_ok = false;
  if (!P->w32) return MG_OK;
  Level& l0 = P->lev[0];
  float* ones = nullptr;
  cudaError_t e = mg_malloc_async(&ones, sizeof(float) * l0.nvert, P->st);
  if (e != cudaSuccess) return oom_or_cuda(e, "scratch");
  MG_CHECK(launch_fill(l0.nvert, 1.f, ones, P->st));
  // boundary entries stay zero (some sweeps write interior vertices only), so
  // u1 = w32 r is zero there
  MG_CHECK(cudaMemsetAsync(P->w32, 0, sizeof(float) * l0.nvert, P->st));
  e = launch_sweep(l0.op, SW_JACOBI0, 0, ones, ones, P->w32, P->desc.omega, nullptr, nullptr, P->st);
  cudaFreeAsync(ones, P->st);
  if (e == cudaErrorNotSupported) return MG_OK;   // no zero-iterate sweep on this level: no shortcut
  MG_CHECK(e);
  P->w_ok = true;
  return MG_OK;
}

mg_status rebuild_coarse(mg_problem* P) {
  for (int l = 0; l + 1 < P->L; ++l) {
    Level& lc = P->lev[l + 1];
    MG_CHECK(launch_galerkin(P->lev[l].op, P->mixed ? 0 : 1, lc.full_store, P->st));
    if (lc.cls)   // stored as a lossy surplus: every later use sees the decoded operator
      MG_CHECK(launch_compress_coarse(P->dim, lc.ncell, (float*)lc.full_store, lc.eps_c, lc.op.hfac,
                                      P->desc.coarse_tau, lc.cls, nullptr, P->st));
    if (lc.stencil) MG_CHECK(launch_build_stencil(lc.op, lc.stencil, P->st));
  }
  MG_CHECK(launch_coarse_factor(P->lev[P->L - 1].op, P->Lc, P->st));
  return MG_OK;
}

// ------------------------------------------------------------ V-cycle
void* vcycle_enqueue(mg_problem* P, int l, mg_status* stt) {
  Level& lv = P->lev[l];
  const int vec64 = P->mixed ? 0 : 1;
  cudaStream_t st = P->st;
  cudaError_t e;
  if (l == P->L - 1) {
    e = launch_coarse_solve(P->dim, P->Lc, vec64, lv.b, lv.x0, st);
    if (e != cudaSuccess) *stt = oom_or_cuda(e, "coarse solve");
    return lv.x0;
  }
  const size_t vb = P->tv * lv.nvert;
  const double om = P->desc.omega;
  auto uses_tail = [&](int lev) {
    return lev == P->L - 2 && !vec64 && vcycle_tail_supported(P->lev[lev].op) && !getenv("MG_NO_VTAIL");
  };
  if (uses_tail(l)) {
    // this level and the coarsest in one block
    e = launch_vcycle_tail(lv.op, P->Lc, (const float*)lv.b, (float*)lv.x0, (float)om, P->desc.nu_pre,
                           P->desc.nu_post, st);
    if (e != cudaSuccess) *stt = oom_or_cuda(e, "V-cycle tail");
    return lv.x0;
  }
  void* cur = lv.x0;
  void* oth = lv.x1;
  // the V-cycle starts from a zero iterate: the first pre-smoothing step is
  // omega D^-1 b where the sweep supports it (no zeroing, no read of x); on
  // the finest level of the mixed flexible-CG iteration the kernel that wrote
  // b also wrote that step into x1
  int k0 = 0;
  const bool have_u1 = l == 0 ? P->u1_ready && !vec64 : lv.u1_ready;
  if (l == 0) P->u1_ready = false;
  lv.u1_ready = false;
  if (have_u1 && P->desc.nu_pre > 0) {
    std::swap(cur, oth);
    k0 = 1;
  } else if (P->desc.nu_pre > 0) {
    e = launch_sweep(lv.op, SW_JACOBI0, vec64, cur, lv.b, oth, om, nullptr, nullptr, st);
    if (e == cudaSuccess) {
      std::swap(cur, oth);
      k0 = 1;
    } else if (e != cudaErrorNotSupported) {
      *stt = oom_or_cuda(e, "pre-smooth");
    }
  }
  if (k0 == 0 && (e = cudaMemsetAsync(cur, 0, vb, st)) != cudaSuccess) *stt = oom_or_cuda(e, "zero");
  for (int k = k0; k < P->desc.nu_pre; ++k) {
    if ((e = launch_sweep(lv.op, SW_JACOBI, vec64, cur, lv.b, oth, om, nullptr, nullptr, st)) != cudaSuccess)
      *stt = oom_or_cuda(e, "pre-smooth");
    std::swap(cur, oth);
  }
  Level& lc = P->lev[l + 1];
  // b_c = R (b - A u): fused where the level supports it (oth then holds the
  // touched vertices' residuals only), else a residual sweep and a restriction.
  // A coarse level that starts with the zero-iterate step of its stencil sweep
  // receives that step, omega b_c / diag, from the restriction as well.
  const bool pass_u1 = l + 1 < P->L - 1 && !uses_tail(l + 1) && lc.stencil && P->desc.nu_pre > 0 &&
                       !getenv("MG_NO_U1");
  const void* cdiag = pass_u1 ? lc.stencil : nullptr;
  void* cu1 = pass_u1 ? lc.x1 : nullptr;
  e = l == 0 ? launch_resid_restrict(lv.op, vec64, cur, lv.b, oth, P->zr, lc.b, st, cdiag, om, cu1)
             : cudaErrorNotSupported;
  if (e == cudaErrorNotSupported) {
    if ((e = launch_sweep(lv.op, SW_RESID, vec64, cur, lv.b, oth, om, nullptr, nullptr, st)) != cudaSuccess)
      *stt = oom_or_cuda(e, "residual");
    if ((e = launch_restrict(P->dim, lc.N, vec64, oth, lc.b, st, cdiag, om, cu1)) != cudaSuccess)
      *stt = oom_or_cuda(e, "restrict");
  } else if (e != cudaSuccess) {
    *stt = oom_or_cuda(e, "residual and restriction");
  }
  lc.u1_ready = pass_u1 && e == cudaSuccess;
  void* ec = vcycle_enqueue(P, l + 1, stt);
  if ((e = launch_prolong_add(P->dim, lc.N, vec64, ec, cur, st)) != cudaSuccess) *stt = oom_or_cuda(e, "prolong");
  for (int k = 0; k < P->desc.nu_post; ++k) {
    e = cudaErrorNotSupported;
    if (l == 0 && k == P->desc.nu_post - 1 && P->vdot_q && !vec64) {   // with the Krylov dot product
      e = launch_jacobi_dot(lv.op, (const float*)cur, (const float*)lv.b, (float*)oth, (float)om, P->vdot_q,
                            P->partials, &P->vdot_nb, st);
      P->vdot_done = e == cudaSuccess;
    }
    if (e == cudaErrorNotSupported) e = launch_sweep(lv.op, SW_JACOBI, vec64, cur, lv.b, oth, om, nullptr, nullptr, st);
    if (e != cudaSuccess) *stt = oom_or_cuda(e, "post-smooth");
    std::swap(cur, oth);
  }
  return cur;
}

// Additive cycles (Section "adaFAC-x", Eq. "adaFAC-x", in correction form)
// for A e = lev[0].b from e = 0; returns the correction (lev[0].x0).  The fine
// residual is restricted to every level; the coarsest is solved exactly and
// every other level takes one damped Jacobi step from zero on its residual,
// c_l = omega D_l^-1 r_l.  adaFAC-PI subtracts from c_l the prolongation of
// one damped Jacobi step s on the next coarser level of the auxiliary
// right-hand side I r_l (injection); adaFAC-Jac takes s from R (r_l - A_l c_l)
// (the transpose of the Jacobi-smoothed prolongation applied to r_l) and
// removes it through the level's own smoother, c_l = S_l (r_l - A_l P s)
// (the AFACx form: P~ = S_l A_l P).  The corrections are summed from the
// coarsest level up.  Levels are processed
// coarse to fine, so a level's b and x1 are free for the auxiliary step of
// the level above it.
void* additive_enqueue(mg_problem* P, mg_status* stt) {
  const int vec64 = P->mixed ? 0 : 1;
  const int L = P->L;
  const int cyc = P->desc.cycle;
  cudaStream_t st = P->st;
  const double om = P->desc.omega;
  cudaError_t e;
  for (int l = 0; l + 1 < L; ++l)
    if ((e = launch_restrict(P->dim, P->lev[l + 1].N, vec64, P->lev[l].b, P->lev[l + 1].b, st)) != cudaSuccess)
      *stt = oom_or_cuda(e, "restrict");
  Level& lcst = P->lev[L - 1];
  if ((e = launch_coarse_solve(P->dim, P->Lc, vec64, lcst.b, lcst.x0, st)) != cudaSuccess)
    *stt = oom_or_cuda(e, "coarse solve");
  // y = w D^-1 b on a level (one Jacobi step from zero).  Where the level's
  // sweep has no zero-iterate form (the finest level of the plane-streaming
  // sweep), a Jacobi step reads a zeroed scratch vector instead; coarser
  // levels sweep stencils, which always have it.
  auto jacobi0 = [&](Level& lv, void* b, void* y, double w, void* zero_scratch) {
    cudaError_t r = launch_sweep(lv.op, SW_JACOBI0, vec64, y, b, y, w, nullptr, nullptr, st);
    if (r == cudaErrorNotSupported && zero_scratch) {
      r = cudaMemsetAsync(zero_scratch, 0, P->tv * lv.nvert, st);
      if (r == cudaSuccess) r = launch_sweep(lv.op, SW_JACOBI, vec64, zero_scratch, b, y, w, nullptr, nullptr, st);
    }
    if (r != cudaSuccess) *stt = oom_or_cuda(r, "additive smoothing");
  };
  for (int l = L - 2; l >= 0; --l) {
    Level& lv = P->lev[l];
    Level& lc = P->lev[l + 1];
    jacobi0(lv, lv.b, lv.x0, om, lv.x1);
    if (cyc == MG_CYCLE_ADAFAC_PI) {
      // c_l = S_l r_l - P S_(l-1) I r_l
      e = launch_inject(P->dim, lc.N, vec64, lv.b, lc.b, st);
      if (e != cudaSuccess) *stt = oom_or_cuda(e, "auxiliary residual");
      jacobi0(lc, lc.b, lc.x1, -om, nullptr);   // minus the auxiliary step ...
      if ((e = launch_prolong_add(P->dim, lc.N, vec64, lc.x1, lv.x0, st)) != cudaSuccess)   // ... prolongated
        *stt = oom_or_cuda(e, "auxiliary prolongation");
    } else if (cyc == MG_CYCLE_ADAFAC_JAC) {
      // s = S_(l-1) R (r_l - A_l S_l r_l), then c_l = S_l (r_l - A_l P s):
      // one Jacobi step from y = P s, minus y
      e = launch_sweep(lv.op, SW_RESID, vec64, lv.x0, lv.b, lv.x1, om, nullptr, nullptr, st);
      if (e == cudaSuccess) e = launch_restrict(P->dim, lc.N, vec64, lv.x1, lc.b, st);
      if (e != cudaSuccess) *stt = oom_or_cuda(e, "auxiliary residual");
      jacobi0(lc, lc.b, lc.x1, om, nullptr);
      e = cudaMemsetAsync(lv.x0, 0, P->tv * lv.nvert, st);
      if (e == cudaSuccess) e = launch_prolong_add(P->dim, lc.N, vec64, lc.x1, lv.x0, st);
      if (e == cudaSuccess) e = launch_sweep(lv.op, SW_JACOBI, vec64, lv.x0, lv.b, lv.x1, om, nullptr, nullptr, st);
      if (e == cudaSuccess) e = launch_sub_from(lv.nvert, vec64, lv.x0, lv.x1, st);   // x0 = x1 - x0
      if (e != cudaSuccess) *stt = oom_or_cuda(e, "auxiliary correction");
    }
    if ((e = launch_prolong_add(P->dim, lc.N, vec64, lc.x0, lv.x0, st)) != cudaSuccess)
      *stt = oom_or_cuda(e, "prolong");
  }
  return P->lev[0].x0;
}

void* cycle_enqueue(mg_problem* P, mg_status* stt) {
  return P->desc.cycle == MG_CYCLE_V ? vcycle_enqueue(P, 0, stt) : additive_enqueue(P, stt);
}

// ------------------------------------------------------------ outer loop
// r = f - A u (FP64) and rr = r.r.  FP64 paths: the V-cycle reads r and the
// Krylov direction is reset.  Mixed paths (iterative refinement): the FP32
// inner solve starts on the unit-scaled residual r_in = r / ||r|| with e = 0.
mg_status outer_restart(mg_problem* P) {
  cudaStream_t st = P->st;
  Level& l0 = P->lev[0];
  int nb = 0;
  if (P->u_zero) {   // r = f - A 0 = f, and r.r = f.f (computed at creation)
    MG_CHECK(cudaMemcpyAsync(P->r, P->f, sizeof(double) * l0.nvert, cudaMemcpyDeviceToDevice, st));
    MG_CHECK(cudaMemcpyAsync(&P->sc->rr, &P->sc->ff, sizeof(double), cudaMemcpyDeviceToDevice, st));
  } else {
    MG_CHECK(launch_sweep(l0.op, SW_RESID, 1, P->u, P->f, P->r, 0.0, nullptr, nullptr, st));
    MG_CHECK(launch_dot(P->r, P->r, l0.nvert, P->partials, &nb, st));
    MG_CHECK(launch_reduce_finish(P->partials, nb, 1, &P->sc->rr, st));
  }
  if (P->mixed) {
    if (P->w_dirty) {
      mg_status sw = build_w(P);
      if (sw != MG_OK) return sw;
    }
    const bool u1 = P->w_ok && P->desc.cycle == MG_CYCLE_V;
    MG_CHECK(launch_scale_residual(l0.nvert, P->r, (float*)l0.b, P->sc, st, u1 ? P->w32 : nullptr,
                                   u1 ? (float*)l0.x1 : nullptr));
    P->u1_ready = u1;
    MG_CHECK(cudaMemsetAsync(P->e32, 0, sizeof(float) * l0.nvert, st));
    if (P->e_pending) {   // a discarded correction: its deferred step goes with it
      MG_CHECK(cudaMemsetAsync(&P->sc->alpha, 0, sizeof(double), st));
      P->e_pending = false;
    }
    P->last_inner_its = P->inner_its;
    P->inner_its = 0;
    P->rin_hist[0] = P->rin_hist[1] = -1.0;
    P->have_correction = false;
  }
  // A restart after a reliable update (same operator, the FP32 correction
  // folded into u) keeps the flexible-CG search direction p and q = A p: only
  // the residual is replaced by the true one, so the Krylov process goes on
  // instead of starting over.  After a publication the operator changed and
  // the iteration starts afresh.
  P->first = !(P->mixed && P->keep_dir);
  P->keep_dir = false;
  P->need_restart = false;
  P->resid_fresh = true;
  return MG_OK;
}

// u += s e (mixed paths): the FP32 correction of the inner solve in FP64
mg_status apply_inner_correction(mg_problem* P, bool reliable = false) {
  if (!P->mixed || !P->have_correction) return MG_OK;
  if (P->e_pending) {
    // the deferred step; alpha then reads zero, so that a next iteration that
    // keeps the search direction adds nothing to the fresh correction
    MG_CHECK(launch_fcg32_flush(P->lev[0].nvert, P->e32, P->p32, P->sc, P->st));
    MG_CHECK(cudaMemsetAsync(&P->sc->alpha, 0, sizeof(double), P->st));
    P->e_pending = false;
  }
  MG_CHECK(launch_apply_correction(P->lev[0].nvert, P->u, P->e32, P->sc, P->st));
  P->have_correction = false;
  P->resid_fresh = false;
  P->u_zero = false;
  P->need_restart = true;
  P->keep_dir = reliable && P->desc.outer == MG_OUTER_FCG;
  return MG_OK;
}

// one iteration, enqueue only
mg_status outer_iteration_enqueue(mg_problem* P, int first) {
  cudaStream_t st = P->st;
  Level& l0 = P->lev[0];
  const long long n = l0.nvert;
  const int z64 = P->mixed ? 0 : 1;
  mg_status stt = MG_OK;
  // the flexible-CG dot z . q of the mixed path, fused into the V-cycle's
  // last sweep where the finest level supports it
  P->vdot_q = (P->mixed && !first && P->desc.outer == MG_OUTER_FCG) ? P->q32 : nullptr;
  P->vdot_done = false;
  void* z = cycle_enqueue(P, &stt);
  P->vdot_q = nullptr;
  if (stt != MG_OK) return stt;
  int nb = 0;
  if (P->mixed) {
    const float* zf = (const float*)z;
    float* rin = (float*)l0.b;
    if (P->desc.outer == MG_OUTER_RICHARDSON) {   // e = V(r_in), applied after this iteration
      MG_CHECK(cudaMemcpyAsync(P->e32, zf, sizeof(float) * n, cudaMemcpyDeviceToDevice, st));
      return MG_OK;
    }
    // FP32 flexible CG on A e = r_in, preconditioned by the FP32 V-cycle
    if (!first) {
      if (P->vdot_done) nb = P->vdot_nb;
      else MG_CHECK(launch_dot_f32f32(zf, P->q32, n, P->partials, &nb, st));
      MG_CHECK(launch_reduce_finish(P->partials, nb, 1, &P->sc->zq, st, P->sc, SC_SET_BETA));
    }
    MG_CHECK(launch_fcg32_direction(n, first, zf, P->p32, P->e32, P->sc, st));
    MG_CHECK(launch_sweep(l0.op, SW_MATVEC, 0, P->p32, rin, P->q32, 0.0, P->partials, &nb, st));
    MG_CHECK(launch_reduce_finish(P->partials, nb, 2, &P->sc->pq, st, P->sc, SC_SET_ALPHA));
    const bool u1 = P->w_ok && P->desc.cycle == MG_CYCLE_V;
    MG_CHECK(launch_fcg32_update(n, rin, P->q32, P->sc, P->partials, &nb, st, u1 ? P->w32 : nullptr,
                                 u1 ? (float*)l0.x1 : nullptr));
    P->u1_ready = u1;
    MG_CHECK(launch_reduce_finish(P->partials, nb, 1, &P->sc->rr_in, st));
    return MG_OK;
  }
  if (P->desc.outer == MG_OUTER_RICHARDSON) {
    MG_CHECK(launch_richardson_update(n, P->u, z64, z, st));
    MG_CHECK(launch_sweep(l0.op, SW_RESID, 1, P->u, P->f, P->r, 0.0, nullptr, nullptr, st));
    MG_CHECK(launch_dot(P->r, P->r, n, P->partials, &nb, st));
    MG_CHECK(launch_reduce_finish(P->partials, nb, 1, &P->sc->rr, st));
    if (P->mixed) MG_CHECK(launch_convert(n, 0, P->r, l0.b, st));
    return MG_OK;
  }
  if (!first) {
    if (z64) MG_CHECK(launch_dot((const double*)z, P->q, n, P->partials, &nb, st));
    else MG_CHECK(launch_dot_f32((const float*)z, P->q, n, P->partials, &nb, st));
    MG_CHECK(launch_reduce_finish(P->partials, nb, 1, &P->sc->zq, st, P->sc, SC_SET_BETA));
  }
  MG_CHECK(launch_fcg_direction(n, first, z64, z, P->p, P->sc, st));
  MG_CHECK(launch_sweep(l0.op, SW_MATVEC, 1, P->p, P->r, P->q, 0.0, P->partials, &nb, st));
  MG_CHECK(launch_reduce_finish(P->partials, nb, 2, &P->sc->pq, st, P->sc, SC_SET_ALPHA));
  MG_CHECK(launch_fcg_update(n, P->u, P->r, P->p, P->q, P->sc, P->mixed ? 1 : 0, P->mixed ? l0.b : nullptr,
                             P->partials, &nb, st));
  MG_CHECK(launch_reduce_finish(P->partials, nb, 1, &P->sc->rr, st));
  return MG_OK;
}

mg_status outer_iteration(mg_problem* P) {
  const int first = P->first ? 1 : 0;
  if (!P->mixed) {   // the FP64 iteration updates u and a recurrence residual
    P->resid_fresh = false;
    P->u_zero = false;
  }
  if (P->use_graphs) {
    if (!P->g_iter[first]) {
      cudaGraph_t g;
      MG_CHECK(cudaStreamBeginCapture(P->st, cudaStreamCaptureModeThreadLocal));
      const long long before = thread_launch_count();
      mg_status s = outer_iteration_enqueue(P, first);
      cudaError_t e = cudaStreamEndCapture(P->st, &g);
      P->g_kernels[first] = thread_launch_count() - before;
      count_launches(-P->g_kernels[first]);  // captured, not launched
      if (s != MG_OK) return s;
      if (e != cudaSuccess) return oom_or_cuda(e, "end capture");
      e = cudaGraphInstantiate(&P->g_iter[first], g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return oom_or_cuda(e, "graph instantiate");
    }
    MG_CHECK(cudaGraphLaunch(P->g_iter[first], P->st));
    count_launches(P->g_kernels[first]);
  } else {
    mg_status s = outer_iteration_enqueue(P, first);
    if (s != MG_OK) return s;
  }
  P->first = false;
  P->cycles++;
  return MG_OK;
}

mg_status read_scalars(mg_problem* P) {
  MG_CHECK(cudaMemcpyAsync(P->h_sc, P->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, P->st));
  MG_CHECK(cudaStreamSynchronize(P->st));
  P->rr = P->h_sc->rr;
  return MG_OK;
}

// Inner tolerance of the mixed path after an outer residual: reduce the
// unit-scaled residual to 0.3 rtol ||f|| / ||r|| (enough to finish), but at
// least to 1e-5 (about what FP32 arithmetic resolves) and at most to 0.1.
constexpr int kMaxInner = 400;

void set_inner_tolerance(mg_problem* P) {
  const double rel = std::sqrt(P->rr / (P->ff > 0 ? P->ff : 1.0));
  double eta = 0.3 * P->desc.rtol / std::max(rel, 1e-300);
  eta = std::min(std::max(eta, P->eta_min), 0.1);
  P->eta2 = eta * eta;
}

// After one inner iteration of the mixed path: apply the correction and ask
// for a new outer residual once the inner residual met its tolerance.
mg_status mixed_after_iteration(mg_problem* P, double rin, bool* diverged) {
  P->inner_its++;
  P->have_correction = true;
  if (P->desc.outer == MG_OUTER_FCG) P->e_pending = true;
  P->rin_hist[1] = P->rin_hist[0];
  P->rin_hist[0] = rin;
  *diverged = !std::isfinite(rin) || rin > 1e8;
  if (*diverged) return MG_OK;
  if (P->desc.outer == MG_OUTER_RICHARDSON || rin <= P->eta2 || P->inner_its >= kMaxInner)
    return apply_inner_correction(P, true);
  return MG_OK;
}

// ------------------------------------------------------------ delayed assembly
void worker_main(mg_problem* P) {
  cudaSetDevice(P->device);
  for (;;) {
    Job job;
    bool inject = false;
    {
      std::unique_lock<std::mutex> lk(P->mu);
      P->cv.wait(lk, [&] { return P->stop || !P->todo.empty(); });
      if (P->stop) return;
      job = P->todo.front();
      P->todo.pop_front();
      inject = P->inject_fail != 0 && job.s == P->inject_fail;
    }
    if (inject) {
      job.status = MG_ERR_INJECTED;
    } else {
      job.status = assemble_chunk(P, job.s, job.chunk, P->side, &job.store, 4);
      if (job.status == MG_OK && cudaEventRecord(job.ev, P->side) != cudaSuccess) {
        job.status = MG_ERR_CUDA;
        set_error("event record failed");
      }
      if (job.status != MG_OK) job.msg = last_error();
    }
    {
      std::lock_guard<std::mutex> lk(P->mu);
      P->ready.push_back(job);
    }
    P->cv.notify_all();
  }
}

void start_worker(mg_problem* P) {
  if (!P->worker.joinable()) P->worker = std::thread(worker_main, P);
}

mg_status enqueue_async(mg_problem* P, int s) {
  std::lock_guard<std::mutex> lk(P->mu);
  for (int c = 0; c < P->nchunk; ++c) {
    Job j;
    j.s = s;
    j.chunk = c;
    if (cudaEventCreateWithFlags(&j.ev, cudaEventDisableTiming) != cudaSuccess) {
      set_error("event create failed");
      return MG_ERR_CUDA;
    }
    P->todo.push_back(j);
    P->in_flight++;
  }
  P->cv.notify_all();
  return MG_OK;
}

// Publishes every completed job (at a cycle boundary).  wait = 1 blocks for
// at least one job when any is in flight.  Returns the number published.
constexpr int kHoldCycles = 16;

mg_status publish_ready(mg_problem* P, bool wait, int* npub) {
  *npub = 0;
  std::vector<Job> done;
  {
    std::unique_lock<std::mutex> lk(P->mu);
    if (wait && P->in_flight > 0 && P->ready.empty())
      P->cv.wait(lk, [&] { return !P->ready.empty() || P->stop; });
    for (auto it = P->ready.begin(); it != P->ready.end();) {
      bool complete = it->status != MG_OK;
      if (!complete) {
        cudaError_t q = wait && done.empty() ? cudaEventSynchronize(it->ev) : cudaEventQuery(it->ev);
        complete = q == cudaSuccess;
        if (q != cudaSuccess && q != cudaErrorNotReady) {
          it->status = MG_ERR_CUDA;
          complete = true;
        }
      }
      if (complete) {
        done.push_back(*it);
        it = P->ready.erase(it);
        P->in_flight--;
      } else {
        ++it;
      }
    }
  }
  mg_status bad = MG_OK;
  for (Job& j : done) {
    if (j.ev) cudaEventDestroy(j.ev);
    if (j.status != MG_OK) {
      bad = (mg_status)j.status;
      if (j.status == MG_ERR_INJECTED) set_error("injected assembly failure");
      else set_error("assembly job (s = %d, chunk %d) failed: %s", j.s, j.chunk, j.msg.c_str());
      free_store(j.store, P->st);
      continue;
    }
    if (P->held.empty()) P->held_since = P->cycles;
    P->held.push_back(j);
  }
  if (P->held.empty()) return bad;
  // Every publication costs a Galerkin rebuild, a new FP64 residual and a
  // restart of the Krylov iteration, so finished chunks are held back until
  // the schedule is done, the solver waits, or kHoldCycles cycles have passed
  // since the first one finished.  (Publishing each accuracy level as soon as
  // it is complete restarted the iteration once per level when the levels
  // finish a cycle apart, and made the cycle count depend on that timing.)
  bool now = wait || P->cycles - P->held_since >= kHoldCycles;
  if (!now) {
    std::lock_guard<std::mutex> lk(P->mu);
    now = P->todo.empty() && P->in_flight == 0;
  }
  if (!now) return bad;
  for (Job& j : P->held) {
    if (j.store.s > P->cur[j.chunk].s) {
      install(P, j.chunk, j.store);
      (*npub)++;
    } else {
      free_store(j.store, P->st);
    }
  }
  P->held.clear();
  if (*npub) {
    mg_status s = upload_tables(P);
    if (s != MG_OK) return s;
    s = rebuild_coarse(P);
    if (s != MG_OK) return s;
    P->publishes += *npub;
    P->need_restart = true;
    P->resid_fresh = false;
    P->keep_dir = false;
  }
  return bad;
}

void stop_worker(mg_problem* P) {
  {
    std::lock_guard<std::mutex> lk(P->mu);
    P->stop = true;
  }
  P->cv.notify_all();
  if (P->worker.joinable()) P->worker.join();
  cudaStreamSynchronize(P->side);
  for (Job& j : P->ready) {
    if (j.ev) cudaEventDestroy(j.ev);
    free_store(j.store, P->side);
  }
  for (Job& j : P->todo)
    if (j.ev) cudaEventDestroy(j.ev);
  for (Job& j : P->held) free_store(j.store, P->side);
  P->ready.clear();
  P->todo.clear();
  P->held.clear();
  P->in_flight = 0;
}

int final_s(const mg_problem* P) { return P->desc.s_schedule[P->desc.n_s - 1]; }

bool all_final(const mg_problem* P) {
  for (const ChunkStore& c : P->cur)
    if (c.s < final_s(P)) return false;
  return true;
}

int min_s(const mg_problem* P) {
  int m = 1 << 30;
  for (const ChunkStore& c : P->cur) m = std::min(m, c.s);
  return m;
}

}  // namespace

namespace mg {
// whether a problem replays its outer iteration as a captured CUDA graph
// (the serving loop's mg_server_desc.use_graphs)
void problem_use_graphs(mg_problem* P, bool on) {
  if (P) P->use_graphs = on;
}
// field descriptor of the C ABI to the device layout (used by other translation units)
void eps_desc_to_dev(const mg_eps_desc& d, int dim, EpsDev* e) { fill_eps(d, dim, e); }
// the descriptor checks of problem creation (MG_OK or MG_ERR_INVALID with the message set)
mg_status eps_desc_check(const mg_eps_desc& d) { return validate_eps(d); }
}  // namespace mg

// ====================================================================== C ABI
extern "C" {

const char* mg_last_error(void) { return mg::last_error(); }
const char* mg_version(void) { return "mg-gb300 1.0"; }

mg_status mg_create_problem(const mg_problem_desc* desc, void* cuda_stream, mg_problem** out) {
  if (!out) {
    set_error("null output pointer");
    return MG_ERR_INVALID;
  }
  *out = nullptr;
  mg_status v = validate(desc);
  if (v != MG_OK) return v;
  mg_problem* P = new mg_problem();
  P->desc = *desc;
  mg_problem_desc& d = P->desc;
  if (d.compress_tau <= 0) d.compress_tau = 1e-6;
  if (d.omega <= 0) d.omega = 0.6;
  if (d.nu_pre <= 0 && d.nu_post <= 0) d.nu_pre = d.nu_post = 2;
  if (d.rtol <= 0) d.rtol = 1e-8;
  if (d.max_cycles <= 0) d.max_cycles = 500;
  P->dim = d.dim;
  P->N = d.n_cells;
  P->mixed = d.path == MG_PATH_MIXED_DELAYED || d.path == MG_PATH_MIXED_PLAIN;
  P->delayed = d.path == MG_PATH_FP64_DELAYED || d.path == MG_PATH_MIXED_DELAYED;
  P->tv = P->mixed ? 4 : 8;
  fill_eps(d.eps, d.dim, &P->eps);
  if (cudaGetDevice(&P->device) != cudaSuccess) P->device = 0;
  if (const char* ng = getenv("MG_NO_GRAPHS")) P->use_graphs = ng[0] == '0';
  if (getenv("MG_NO_SPECULATE")) P->speculate = false;
  P->trace = getenv("MG_TRACE") != nullptr;
  auto fail = [&](mg_status s) {
    mg_destroy_problem(P);
    return s;
  };
  if (cuda_stream) {
    P->st = (cudaStream_t)cuda_stream;
  } else {
    if (!cuda_ok(cudaStreamCreateWithFlags(&P->st, cudaStreamNonBlocking), "stream")) return fail(MG_ERR_CUDA);
    P->own_stream = true;
  }
  // The side stream runs at the greatest priority: its assembly proceeds at
  // full speed and the solver's kernels fill the device around it.  (The
  // paper's background tasks use cores the solver leaves idle; on one GPU
  // both saturate the device, and cycles on stale stencils are the less
  // valuable work: giving the solver precedence made the delayed solves
  // slower, with more cycles before the final publication.)
  {
    int lo = 0, hi = 0;
    if (!cuda_ok(cudaDeviceGetStreamPriorityRange(&lo, &hi), "priority range") ||
        !cuda_ok(cudaStreamCreateWithPriority(&P->side, cudaStreamNonBlocking, hi), "side stream"))
      return fail(MG_ERR_CUDA);
  }
  // levels
  int L = 0;
  for (int n = P->N; n >= 3; n /= 3) ++L;
  P->L = L;
  P->lev.resize(L);
  const int D = P->dim;
  const int NP = D == 3 ? 28 : 6;
  for (int l = 0; l < L; ++l) {
    Level& lv = P->lev[l];
    lv.N = P->N / ipow3(l);
    lv.ncell = (long long)lv.N * lv.N * (D == 3 ? lv.N : 1);
    lv.nvert = (long long)(lv.N + 1) * (lv.N + 1) * (D == 3 ? (lv.N + 1) : 1);
    double h = 1.0 / lv.N;
    LevelOp& op = lv.op;
    op.N = lv.N;
    op.dim = D;
    op.hfac = D == 3 ? h : 1.0;
    op.gk64 = op.hfac * (-1.0 / 12.0);
    op.gk32 = (float)op.gk64;
    op.nseg_x = (lv.N + kSegCells - 1) / kSegCells;
    cudaError_t e;
    if (l > 0) {
      op.layers = lv.N;
      op.nchunk = 1;
      op.chunk_cells = lv.ncell;
      op.compressed = 0;
      op.elem64 = P->mixed ? 0 : 1;
      if ((e = dalloc(P, &lv.full_store, (size_t)NP * lv.ncell * (P->mixed ? 4 : 8))) != cudaSuccess)
        return fail(oom_or_cuda(e, "coarse storage"));
      if ((e = dalloc(P, &lv.d_full, sizeof(FullChunk))) != cudaSuccess) return fail(oom_or_cuda(e, "table"));
      FullChunk fc{lv.full_store};
      if (!cuda_ok(cudaMemcpyAsync(lv.d_full, &fc, sizeof(fc), cudaMemcpyHostToDevice, P->st), "table upload"))
        return fail(MG_ERR_CUDA);
      op.full = lv.d_full;
      if (P->mixed && d.coarse_tau > 0.0) {
        if ((e = dalloc(P, &lv.eps_c, sizeof(float) * lv.ncell)) != cudaSuccess ||
            (e = dalloc(P, &lv.cls, lv.ncell)) != cudaSuccess)
          return fail(oom_or_cuda(e, "coarse compression"));
        if (!cuda_ok(launch_eps_centre(D, lv.N, &P->eps, 0, lv.eps_c, P->st), "coarse eps"))
          return fail(MG_ERR_CUDA);
      }
    }
    // assembled vertex stencils for the levels swept with full storage (not the
    // coarsest, which is solved directly, nor the compressed finest level)
    // (mixed 3D fields without flat cells, e.g. lognormal: every cell carries a
    // surplus, so the finest level is also swept from assembled FP32 stencils)
    const bool dense0 = l == 0 && P->mixed && D == 3 && L > 1 && P->eps.kind != EPS_BOXES &&
                        P->eps.kind != EPS_DISC && P->eps.kind != EPS_CONST && !getenv("MG_NO_DENSE_STENCIL");
    if (l < L - 1 && (l > 0 || !P->mixed || dense0)) {
      const size_t sb = (size_t)(D == 3 ? 14 : 5) * lv.nvert * (P->mixed ? 4 : 8);   // symmetric storage
      if ((e = dalloc(P, &lv.stencil, sb)) != cudaSuccess) return fail(oom_or_cuda(e, "stencils"));
      cudaMemsetAsync(lv.stencil, 0, sb, P->st);
      op.stencil = lv.stencil;
    }
    const size_t vb = P->tv * lv.nvert;
    if ((e = dalloc(P, &lv.b, vb)) != cudaSuccess || (e = dalloc(P, &lv.x0, vb)) != cudaSuccess ||
        (e = dalloc(P, &lv.x1, vb)) != cudaSuccess)
      return fail(oom_or_cuda(e, "level vectors"));
    cudaMemsetAsync(lv.b, 0, vb, P->st);
    cudaMemsetAsync(lv.x0, 0, vb, P->st);
    cudaMemsetAsync(lv.x1, 0, vb, P->st);
  }
  // finest level chunking: slabs of whole cell layers along the last axis
  Level& l0 = P->lev[0];
  int nch = d.chunks > 0 ? d.chunks : (P->N >= 27 ? 9 : 1);
  if (nch > P->N) nch = P->N;
  P->layers = (P->N + nch - 1) / nch;
  P->nchunk = (P->N + P->layers - 1) / P->layers;
  if (P->N % P->layers != 0) {  // keep equal chunk sizes: fall back to one chunk
    P->layers = P->N;
    P->nchunk = 1;
  }
  P->nseg_x = l0.op.nseg_x;
  P->chunk_cells = l0.ncell / P->nchunk;
  P->chunk_rows = P->chunk_cells / P->N;
  P->chunk_nseg = P->chunk_rows * P->nseg_x;
  l0.op.layers = P->layers;
  l0.op.nchunk = P->nchunk;
  l0.op.chunk_cells = P->chunk_cells;
  l0.op.compressed = P->mixed ? 1 : 0;
  l0.op.elem64 = P->mixed ? 0 : 1;
  P->cur.resize(P->nchunk);
  P->h_full.resize(P->nchunk);
  P->h_cmp.resize(P->nchunk);
  cudaError_t e;
  if (P->mixed) {
    if ((e = dalloc(P, &l0.d_cmp, sizeof(CmpChunk) * P->nchunk)) != cudaSuccess) return fail(oom_or_cuda(e, "table"));
    l0.op.cmp = l0.d_cmp;
    if ((e = dalloc(P, &P->scratch, (size_t)P->chunk_cells * (D == 3 ? 112 : 32))) != cudaSuccess)
      return fail(oom_or_cuda(e, "scratch"));
  } else {
    if ((e = dalloc(P, &l0.d_full, sizeof(FullChunk) * P->nchunk)) != cudaSuccess) return fail(oom_or_cuda(e, "table"));
    l0.op.full = l0.d_full;
  }
  if ((e = dalloc(P, &P->eps_c, (size_t)l0.ncell * (P->mixed ? 4 : 8))) != cudaSuccess)
    return fail(oom_or_cuda(e, "eps_c"));
  if (P->mixed) l0.op.eps_c = (const float*)P->eps_c;
  if (P->mixed && D == 3 && P->N >= 27 && (P->N + 1) % 4 == 0 && !getenv("MG_NO_SPLIT_SWEEP")) {
    // split sweep (geometric bulk pass + fix-up of vertices next to surplus cells)
    const long long ng = (l0.nvert + 31) / 32;
    if ((e = dalloc(P, &P->touched, sizeof(int) * l0.nvert)) != cudaSuccess ||
        (e = dalloc(P, &P->ntouched, sizeof(int))) != cudaSuccess ||
        (e = dalloc(P, &P->tflags, (size_t)l0.nvert)) != cudaSuccess ||
        (e = dalloc(P, &P->tcounts, sizeof(uint32_t) * (ng + (ng + 2047) / 2048 + 1))) != cudaSuccess)
      return fail(oom_or_cuda(e, "touched list"));
    // stencil table for up to a quarter of the vertices (more touched vertices
    // are recomputed from their cell records in the fix-up pass)
    const long long ni = (long long)(P->N - 1) * (P->N - 1) * (P->N - 1);
    long long cap = l0.nvert / 4 > 65536 ? l0.nvert / 4 : 65536;
    cap = cap < ni ? cap : ni;
    if (l0.stencil) cap = 0;   // swept from full stencils: the table is not used
    if (const char* ev = getenv("MG_STENCIL_CAP")) {   // smaller table (tests of the record path)
      const long long c2 = atoll(ev);
      if (c2 >= 1 && c2 < cap) cap = c2;
    }
    if (cap > 0 && (e = dalloc(P, &P->tcoef, sizeof(float) * 27 * (size_t)cap)) != cudaSuccess)
      return fail(oom_or_cuda(e, "stencil table"));
    cudaMemsetAsync(P->ntouched, 0, sizeof(int), P->st);
    l0.op.touched = P->touched;
    l0.op.ntouched = P->ntouched;
    l0.op.tcoef = P->tcoef;
    l0.op.tcap = (int)cap;
    // eps_c with padded rows for the bulk pass
    if ((e = dalloc(P, &P->eps_pad, sizeof(float) * (size_t)P->N * P->N * (P->N + 1))) != cudaSuccess)
      return fail(oom_or_cuda(e, "padded eps"));
    l0.op.eps_pad = P->eps_pad;
    if (!l0.stencil) {
      // touched-vertex bits (the sweeps fused with a restriction or a dot product)
      if ((e = dalloc(P, &P->tmask, sizeof(uint32_t) * tmask_words(P->N))) != cudaSuccess)
        return fail(oom_or_cuda(e, "touched mask"));
      l0.op.tmask = P->tmask;
      const size_t nzr = (size_t)(P->N / 3 + 1) * (P->N + 1) * (P->N + 1);
      // the fused residual + restriction (MG_FUSED_RESTRICT=1; measured slower
      // than the residual sweep and the tiled restriction on this part: the
      // bulk pass is latency-bound and gains nothing from the write it saves)
      if (getenv("MG_FUSED_RESTRICT") && (e = dalloc(P, &P->zr, sizeof(float) * nzr)) != cudaSuccess)
        return fail(oom_or_cuda(e, "fused restriction buffer"));
    }
  }
  // outer vectors
  const size_t v8 = sizeof(double) * l0.nvert;
  if ((e = dalloc(P, &P->u, v8)) != cudaSuccess || (e = dalloc(P, &P->f, v8)) != cudaSuccess ||
      (e = dalloc(P, &P->r, v8)) != cudaSuccess || (e = dalloc(P, &P->p, v8)) != cudaSuccess ||
      (e = dalloc(P, &P->q, v8)) != cudaSuccess)
    return fail(oom_or_cuda(e, "outer vectors"));
  cudaMemsetAsync(P->u, 0, v8, P->st);
  cudaMemsetAsync(P->r, 0, v8, P->st);
  cudaMemsetAsync(P->p, 0, v8, P->st);
  cudaMemsetAsync(P->q, 0, v8, P->st);
  if (!P->mixed) {
    // FP64 V-cycle reads its right-hand side straight from r
    P->allocs.erase(std::find(P->allocs.begin(), P->allocs.end(), l0.b));
    cudaFreeAsync(l0.b, P->st);
    l0.b = P->r;
  } else {
    const size_t v4 = sizeof(float) * l0.nvert;
    if ((e = dalloc(P, &P->p32, v4)) != cudaSuccess || (e = dalloc(P, &P->q32, v4)) != cudaSuccess ||
        (e = dalloc(P, &P->e32, v4)) != cudaSuccess)
      return fail(oom_or_cuda(e, "inner vectors"));
    if (!getenv("MG_NO_U1") && (e = dalloc(P, &P->w32, v4)) != cudaSuccess)
      return fail(oom_or_cuda(e, "inverse diagonal"));
    cudaMemsetAsync(P->p32, 0, v4, P->st);
    cudaMemsetAsync(P->q32, 0, v4, P->st);
    cudaMemsetAsync(P->e32, 0, v4, P->st);
  }
  {
    const long long ni = P->N - 1;
    long long sweep_blocks = ((ni + 31) / 32) * ((ni + 7) / 8) * (D == 3 ? ni : 1);
    P->npartials = 2 * std::max<long long>(sweep_blocks, 152 * 8) + 64;
  }
  if ((e = dalloc(P, &P->partials, sizeof(double) * P->npartials)) != cudaSuccess ||
      (e = dalloc(P, &P->sc, sizeof(DevScalars))) != cudaSuccess ||
      (e = dalloc(P, &P->Lc, sizeof(double) * 128)) != cudaSuccess ||
      (e = dalloc(P, &P->d_totals, sizeof(uint32_t) * 8)) != cudaSuccess)
    return fail(oom_or_cuda(e, "scalars"));
  cudaMemsetAsync(P->sc, 0, sizeof(DevScalars), P->st);
  if (!cuda_ok(cudaMallocHost(&P->h_sc, sizeof(DevScalars)), "pinned") ||
      !cuda_ok(cudaMallocHost(&P->h_slot[0], sizeof(DevScalars)), "pinned") ||
      !cuda_ok(cudaMallocHost(&P->h_slot[1], sizeof(DevScalars)), "pinned") ||
      !cuda_ok(cudaEventCreateWithFlags(&P->slot_ev[0], cudaEventDisableTiming), "event") ||
      !cuda_ok(cudaEventCreateWithFlags(&P->slot_ev[1], cudaEventDisableTiming), "event") ||
      !cuda_ok(cudaMallocHost(&P->h_totals, sizeof(uint32_t) * 8), "pinned"))
    return fail(MG_ERR_CUDA);
  // load vector f_v = f_const h^d, initial guess
  double hd = 1.0;
  for (int a = 0; a < D; ++a) hd /= P->N;
  if (!cuda_ok(launch_load_vector(D, P->N, d.f_const * hd, P->f, P->st), "load vector")) return fail(MG_ERR_CUDA);
  if (d.u0) {
    P->u_zero = false;
    if (!cuda_ok(cudaMemcpyAsync(P->u, d.u0, v8, cudaMemcpyHostToDevice, P->st), "u0 upload") ||
        !cuda_ok(cudaStreamSynchronize(P->st), "u0 sync"))
      return fail(MG_ERR_CUDA);
    // boundary values are forced to zero by the operator (Dirichlet rows are never written)
  }
  P->desc.u0 = nullptr;
  {
    // ||f||^2 (or later ||r_0||^2 when f = 0)
    int nb = 0;
    if (!cuda_ok(launch_dot(P->f, P->f, l0.nvert, P->partials, &nb, P->st), "dot") ||
        !cuda_ok(launch_reduce_finish(P->partials, nb, 1, &P->sc->ff, P->st), "reduce"))
      return fail(MG_ERR_CUDA);
  }
  // cell-centre eps and the geometric (s = 1) operator
  if (!cuda_ok(launch_eps_centre(D, P->N, &P->eps, P->mixed ? 0 : 1, P->eps_c, P->st), "eps centre"))
    return fail(MG_ERR_CUDA);
  if (P->eps_pad && !cuda_ok(launch_pad_eps(P->N, (const float*)P->eps_c, P->eps_pad, P->st), "padded eps"))
    return fail(MG_ERR_CUDA);
  // interface cells of piecewise-constant fields (the only cells with a surplus)
  if (!getenv("MG_NO_INTERFACE_LIST") &&
      (P->eps.kind == EPS_BOXES || P->eps.kind == EPS_DISC || P->eps.kind == EPS_CONST)) {
    int* counts = nullptr;
    if ((e = dalloc(P, &P->ilist, sizeof(int) * (size_t)P->chunk_cells * P->nchunk)) != cudaSuccess ||
        (e = mg_malloc_async(&counts, sizeof(int) * P->nchunk, P->st)) != cudaSuccess)
      return fail(oom_or_cuda(e, "interface cells"));
    P->ilist_n.assign(P->nchunk, 0);
    if (!cuda_ok(cudaMemsetAsync(counts, 0, sizeof(int) * P->nchunk, P->st), "memset") ||
        !cuda_ok(launch_interface_cells(D, P->N, &P->eps, P->chunk_cells, P->ilist, counts, P->st), "interface") ||
        !cuda_ok(cudaMemcpyAsync(P->ilist_n.data(), counts, sizeof(int) * P->nchunk, cudaMemcpyDeviceToHost, P->st),
                 "counts") ||
        !cuda_ok(cudaStreamSynchronize(P->st), "interface sync"))
      return fail(MG_ERR_CUDA);
    cudaFreeAsync(counts, P->st);
  }
  // Mixed paths on piecewise-constant fields: the FP64 outer residual and
  // matvec apply the exact FP64 operator (FP64 cell-centre eps everywhere,
  // FP64 surplus of the interface cells, which are integrated in FP64), so
  // that the solution meets the residual target under the operator the FP64
  // paths assemble; the FP32 V-cycle keeps reading the lossy records.
  if (P->mixed && P->ilist && !getenv("MG_LOSSY_RESIDUAL")) {
    P->exact = true;
    if ((e = dalloc(P, &P->eps64, sizeof(double) * (size_t)l0.ncell)) != cudaSuccess ||
        (e = dalloc(P, &P->xpos, sizeof(int) * (size_t)l0.ncell)) != cudaSuccess)
      return fail(oom_or_cuda(e, "exact operator"));
    if (!cuda_ok(launch_eps_centre(D, P->N, &P->eps, 1, P->eps64, P->st), "eps centre") ||
        !cuda_ok(launch_xpos(P->chunk_cells, P->nchunk, P->ilist, P->ilist_n.data(), P->xpos, P->st), "positions"))
      return fail(MG_ERR_CUDA);
    l0.op.eps64 = P->eps64;
    l0.op.xpos = P->xpos;
    if (P->touched) {
      if ((e = dalloc(P, &P->touched64, sizeof(int) * (size_t)l0.nvert)) != cudaSuccess ||
          (e = dalloc(P, &P->ntouched64, sizeof(int))) != cudaSuccess)
        return fail(oom_or_cuda(e, "exact touched list"));
      if (!cuda_ok(launch_build_touched(l0.op, P->tflags, P->tcounts, P->touched64, P->ntouched64, P->st, 1),
                   "exact touched list"))
        return fail(MG_ERR_CUDA);
      l0.op.touched64 = P->touched64;
      l0.op.ntouched64 = P->ntouched64;
    }
  }
  // FP64 bulk pass of the split finest level in vertex form (weights built
  // once from the cell-centre eps; MG_CELL_FORM64=1 keeps the cell form)
  if (P->touched && !getenv("MG_CELL_FORM64")) {
    const size_t nv = (size_t)l0.nvert;
    double* w[4] = {nullptr, nullptr, nullptr, nullptr};
    double* es = nullptr;
    for (int m = 0; m < 4; ++m)
      if ((e = dalloc(P, &w[m], sizeof(double) * nv)) != cudaSuccess) return fail(oom_or_cuda(e, "FP64 weights"));
    if ((e = dalloc(P, &es, sizeof(double) * (size_t)P->N * P->N * (P->N + 1))) != cudaSuccess)
      return fail(oom_or_cuda(e, "FP64 weights"));
    if (!cuda_ok(launch_geo_weights64(l0.op, w, es, P->st), "FP64 weights")) return fail(MG_ERR_CUDA);
    for (int m = 0; m < 4; ++m) l0.op.w64[m] = w[m];
    l0.op.es64 = es;
  }
  if (d.adapt_C > 0.0 && d.n_s >= 2) {
    P->adapt = true;
    P->wlast.resize(P->nchunk);
    const size_t nc = (size_t)P->chunk_cells * P->nchunk;
    if ((e = dalloc(P, &P->final_flags, nc)) != cudaSuccess || (e = dalloc(P, &P->s_cell, nc)) != cudaSuccess ||
        (e = dalloc(P, &P->awork, sizeof(int) * (size_t)P->chunk_cells)) != cudaSuccess ||
        (e = dalloc(P, &P->anwork, sizeof(int))) != cudaSuccess)
      return fail(oom_or_cuda(e, "adaptive accuracy"));
    // cells with eps constant over them have the exact matrix at every s:
    // they are final from the start (all other cells are judged)
    e = P->ilist ? launch_adaptive_init(P->chunk_cells, P->nchunk, P->ilist, P->ilist_n.data(), P->final_flags, P->st)
                 : cudaMemsetAsync(P->final_flags, 0, nc, P->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(P->s_cell, 1, nc, P->st);   // the centre sample
    if (!cuda_ok(e, "adaptive init")) return fail(MG_ERR_CUDA);
  }
  for (int c = 0; c < P->nchunk; ++c) {
    ChunkStore cs;
    mg_status s = assemble_chunk(P, 1, c, P->st, &cs, 0);
    if (s != MG_OK) return fail(s);
    install(P, c, cs);
  }
  if (P->adapt) P->wlast = P->cur;
  mg_status s = upload_tables(P);
  if (s == MG_OK) s = rebuild_coarse(P);
  if (s != MG_OK) return fail(s);
  if (!cuda_ok(read_scalars(P) == MG_OK ? cudaSuccess : cudaErrorUnknown, "create sync")) return fail(MG_ERR_CUDA);
  P->ff = P->h_sc->ff;
  P->need_restart = true;
  *out = P;
  return MG_OK;
}

mg_status mg_destroy_problem(mg_problem* P) {
  if (!P) return MG_OK;
  stop_worker(P);
  if (P->st) cudaStreamSynchronize(P->st);
  for (int g = 0; g < 2; ++g)
    if (P->g_iter[g]) cudaGraphExecDestroy(P->g_iter[g]);
  cudaStream_t st = P->st;
  if (st) {
    for (ChunkStore& c : P->cur) free_store(c, st);
    for (void* a : P->allocs) cudaFreeAsync(a, st);
    cudaStreamSynchronize(st);
  }
  if (P->h_sc) cudaFreeHost(P->h_sc);
  for (int i = 0; i < 2; ++i) {
    if (P->h_slot[i]) cudaFreeHost(P->h_slot[i]);
    if (P->slot_ev[i]) cudaEventDestroy(P->slot_ev[i]);
  }
  if (P->h_totals) cudaFreeHost(P->h_totals);
  if (P->side) cudaStreamDestroy(P->side);
  if (P->own_stream && P->st) cudaStreamDestroy(P->st);
  delete P;
  return MG_OK;
}

mg_status mg_assemble_level(mg_problem* P, int s, int async) {
  if (!P || s < 1 || s > 64) {
    set_error("bad problem or accuracy");
    return MG_ERR_INVALID;
  }
  if (async) {
    start_worker(P);
    return enqueue_async(P, s);
  }
  // synchronous: wait for in-flight jobs first (the scratch buffer is shared)
  for (;;) {
    int npub = 0;
    {
      std::lock_guard<std::mutex> lk(P->mu);
      if (P->in_flight == 0 && P->held.empty()) break;
    }
    mg_status st = publish_ready(P, true, &npub);
    if (st != MG_OK) return st;
  }
  for (int c = 0; c < P->nchunk; ++c) {
    ChunkStore cs;
    mg_status st = assemble_chunk(P, s, c, P->st, &cs, 0);
    if (st != MG_OK) return st;
    install(P, c, cs);
  }
  mg_status st = upload_tables(P);
  if (st == MG_OK) st = rebuild_coarse(P);
  P->need_restart = true;
  P->resid_fresh = false;
  return st;
}

mg_status mg_vcycle(mg_problem* P, int n, double* rel_residual) {
  if (!P || n < 0) {
    set_error("bad arguments");
    return MG_ERR_INVALID;
  }
  for (int it = 0; it < n; ++it) {
    int npub = 0;
    mg_status s = publish_ready(P, false, &npub);
    if (s != MG_OK) return s;
    if (npub) {
      s = apply_inner_correction(P);
      if (s != MG_OK) return s;
    }
    if (P->need_restart) {
      s = outer_restart(P);
      if (s == MG_OK && P->mixed) {
        s = read_scalars(P);
        set_inner_tolerance(P);
      }
      if (s != MG_OK) return s;
    }
    s = outer_iteration(P);
    if (s != MG_OK) return s;
    if (P->mixed) {
      s = read_scalars(P);
      bool diverged = false;
      if (s == MG_OK) s = mixed_after_iteration(P, P->h_sc->rr_in, &diverged);
      if (s != MG_OK) return s;
    }
  }
  mg_status sc_ = apply_inner_correction(P);
  if (sc_ != MG_OK) return sc_;
  // true residual of the current iterate
  Level& l0 = P->lev[0];
  int nb = 0;
  MG_CHECK(launch_sweep(l0.op, SW_RESID, 1, P->u, P->f, P->p, 0.0, nullptr, nullptr, P->st));
  MG_CHECK(launch_dot(P->p, P->p, l0.nvert, P->partials, &nb, P->st));
  MG_CHECK(launch_reduce_finish(P->partials, nb, 1, &P->sc->r0, P->st));
  mg_status s = read_scalars(P);
  if (s != MG_OK) return s;
  P->need_restart = true;  // p was used as scratch
  const double ref = P->ff > 0 ? P->ff : 1.0;
  if (rel_residual) *rel_residual = std::sqrt(P->h_sc->r0 / ref);
  return MG_OK;
}

mg_status mg_solve(mg_problem* P, mg_solve_info* info) {
  if (!P) {
    set_error("null problem");
    return MG_ERR_INVALID;
  }
  auto t0 = std::chrono::steady_clock::now();
  double asm_ms = 0.0;
  const mg_problem_desc& d = P->desc;
  P->cycles = 0;
  P->publishes = 0;
  if (!P->delayed) {
    auto ta = std::chrono::steady_clock::now();
    if (P->adapt) {   // the adaptive rule needs every level of the schedule, in order
      for (int i = 0; i < d.n_s; ++i)
        if (d.s_schedule[i] > min_s(P)) {
          mg_status s = mg_assemble_level(P, d.s_schedule[i], 0);
          if (s != MG_OK) return s;
        }
    } else if (min_s(P) < final_s(P)) {
      mg_status s = mg_assemble_level(P, final_s(P), 0);
      if (s != MG_OK) return s;
    }
    MG_CHECK(cudaStreamSynchronize(P->st));
    asm_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - ta).count();
  } else {
    start_worker(P);
    for (int i = 0; i < d.n_s; ++i)
      if (d.s_schedule[i] > min_s(P)) {
        mg_status s = enqueue_async(P, d.s_schedule[i]);
        if (s != MG_OK) return s;
      }
  }
  const double ref = P->ff > 0 ? P->ff : 1.0;
  const double tol2 = d.rtol * d.rtol;
  mg_status result = MG_ERR_NOT_CONVERGED;
  bool have_first = false;
  bool restarted = false;
  P->trace_log.clear();
  double seg_rr = 0.0;
  int seg_cycles = 0;
  double op_rr = 0.0;   // mixed paths: true residual at the first restart on the current operator
  int op_cycles = 0;
  bool pipe_next = false;   // an iteration enqueued ahead awaits its test (scalars in h_slot[pipe_slot])
  int pipe_slot = 0;
  int ahead_count = 0;
  // trace entry of an iteration enqueued ahead whose step a correction folded
  // in before its test (its scalars are read once it has completed)
  auto trace_folded = [&](int slot) -> mg_status {
    MG_CHECK(cudaEventSynchronize(P->slot_ev[slot]));
    mg_trace_entry t{};
    t.cycle = P->cycles;
    {
      std::lock_guard<std::mutex> lk(P->mu);
      t.pending_jobs = P->in_flight + (int)P->held.size();
    }
    t.publishes = P->publishes;
    const double ffn = P->ff > 0 ? P->ff : 1.0;
    t.rel_residual_est = std::sqrt(P->rr / ffn) * std::sqrt(std::max(P->h_slot[slot]->rr_in, 0.0));
    t.time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    P->trace_log.push_back(t);
    return MG_OK;
  };
  while (P->cycles < d.max_cycles || pipe_next) {
    int npub = 0;
    mg_status s = publish_ready(P, false, &npub);
    if (s != MG_OK) {
      result = s;
      break;
    }
    if (npub) op_rr = 0.0;
    if (npub) {   // the correction computed so far belongs to the old operator: apply it
      s = apply_inner_correction(P);
      if (s != MG_OK) return s;
      if (P->need_restart && pipe_next) {   // the iteration enqueued ahead is folded in
        if ((s = trace_folded(pipe_slot)) != MG_OK) return s;
        pipe_next = false;
      }
    }
    if (P->need_restart) {
      s = outer_restart(P);
      if (s != MG_OK) return s;
      s = read_scalars(P);
      if (s != MG_OK) return s;
      if (!have_first) {
        P->rr_first = P->rr;
        have_first = true;
      }
      if (P->ff <= 0) P->ff = P->rr > 0 ? P->rr : 1.0;
      if (P->mixed) set_inner_tolerance(P);
      if (P->trace)   // MG_TRACE=1: one line per outer restart on stderr
        fprintf(stderr, "mg: restart at cycle %d  rel %.3e  inner its %d  eta %.1e  final %d  ahead %d\n", P->cycles,
                std::sqrt(P->rr / (P->ff > 0 ? P->ff : 1.0)), P->last_inner_its, std::sqrt(P->eta2),
                all_final(P) ? 1 : 0, ahead_count);
      // divergence is judged against the residual of the current operator
      // at the last restart (a publication changes the operator)
      seg_rr = P->rr;
      seg_cycles = 0;
      restarted = true;
      // the mixed paths restart at every correction; their divergence is judged
      // against the first true residual on the current operator
      if (P->mixed) {
        if (op_rr == 0.0) {
          op_rr = P->rr;
          op_cycles = 0;
        } else if (!std::isfinite(P->rr) || (op_cycles > 5 && P->rr > 1e4 * std::max(op_rr, 1e-300))) {
          result = MG_ERR_DIVERGED;
          set_error("residual diverged: ||r||^2 = %.3e after %d cycles (%.3e on this operator at first)", P->rr,
                    P->cycles, op_rr);
          break;
        }
      }
    }
    const double refn = P->ff > 0 ? P->ff : ref;
    if (P->rr <= tol2 * refn) {
      bool pending;
      {
        std::lock_guard<std::mutex> lk(P->mu);
        pending = P->in_flight > 0 || !P->held.empty();
      }
      if (all_final(P) && !pending) {
        result = MG_OK;
        break;
      }
      if (pending) {  // converged on stale stencils: wait for the next publication
        s = publish_ready(P, true, &npub);
        if (s != MG_OK) {
          result = s;
          break;
        }
        if (npub) op_rr = 0.0;   // a new operator: its first residual is the new reference
        continue;
      }
      // not final and nothing pending: the schedule was cut short
      result = MG_OK;
      break;
    }
    // Iteration pipeline.  Every iteration copies its scalars into a pinned
    // slot and records an event; the host tests it after that event only.
    // Mixed flexible CG: when the last two inner residuals predict that the
    // iteration under test stays at least ten times above the inner
    // tolerance, the next one is enqueued before the test, so the GPU works
    // on it during the host's round trip.  A wrong guess adds one more
    // flexible-CG step to the correction (folded in when it is applied).
    auto enqueue_iter = [&](int slot) -> mg_status {
      mg_status r = outer_iteration(P);
      if (r != MG_OK) return r;
      MG_CHECK(cudaMemcpyAsync(P->h_slot[slot], P->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, P->st));
      MG_CHECK(cudaEventRecord(P->slot_ev[slot], P->st));
      return MG_OK;
    };
    int cur = pipe_slot;
    if (!pipe_next) {
      cur = 0;
      if ((s = enqueue_iter(cur)) != MG_OK) return s;
    }
    bool ahead = false;
    if (P->mixed && P->speculate && d.outer == MG_OUTER_FCG && P->cycles + 1 < d.max_cycles &&
        P->inner_its + 2 < kMaxInner && P->rin_hist[0] > 0.0 && P->rin_hist[1] > 0.0) {
      const double pred = P->rin_hist[0] * (P->rin_hist[0] / P->rin_hist[1]);
      if (std::isfinite(pred) && pred > 10.0 * P->eta2) {
        if ((s = enqueue_iter(cur ^ 1)) != MG_OK) return s;
        ahead = true;
      }
    }
    MG_CHECK(cudaEventSynchronize(P->slot_ev[cur]));
    const DevScalars& hs = *P->h_slot[cur];
    P->rr = hs.rr;
    *P->h_sc = hs;
    ++seg_cycles;
    ++op_cycles;
    {
      mg_trace_entry t{};
      t.cycle = ahead ? P->cycles - 1 : P->cycles;
      {
        std::lock_guard<std::mutex> lk(P->mu);
        t.pending_jobs = P->in_flight + (int)P->held.size();
      }
      t.publishes = P->publishes;
      t.restarted = restarted ? 1 : 0;
      const double ffn = P->ff > 0 ? P->ff : 1.0;
      t.rel_residual_est = P->mixed ? std::sqrt(P->rr / ffn) * std::sqrt(std::max(hs.rr_in, 0.0))
                                    : std::sqrt(P->rr / ffn);
      t.time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
      P->trace_log.push_back(t);
      restarted = false;
    }
    bool stop = false;
    if (P->mixed) {
      bool diverged = false;
      s = mixed_after_iteration(P, hs.rr_in, &diverged);
      if (s != MG_OK) return s;
      if (diverged) {
        result = MG_ERR_DIVERGED;
        set_error("inner residual diverged after %d cycles", P->cycles);
        stop = true;
      }
    }
    // the iteration enqueued ahead is tested next, unless a correction applied
    // now already folded it in
    if (ahead) ++ahead_count;
    if (ahead && !stop && P->need_restart && (s = trace_folded(cur ^ 1)) != MG_OK) return s;
    pipe_next = ahead && !stop && !P->need_restart;
    pipe_slot = cur ^ 1;
    if (stop) break;
    if (P->mixed) continue;
    if (!std::isfinite(P->rr) || (seg_cycles > 5 && P->rr > 1e4 * std::max(seg_rr, 1e-300))) {
      result = MG_ERR_DIVERGED;
      set_error("residual diverged: ||r||^2 = %.3e after %d cycles (%.3e at the last restart)", P->rr,
                P->cycles, seg_rr);
      break;
    }
  }
  // verify with the true residual (already at hand when the last restart
  // computed it for the current u and operator)
  double rel = 0.0;
  if (P->resid_fresh && !P->have_correction) {
    rel = std::sqrt(P->rr / (P->ff > 0 ? P->ff : 1.0));
    P->need_restart = true;
  } else {
    mg_status s = apply_inner_correction(P);
    if (s != MG_OK) return s;
    Level& l0 = P->lev[0];
    int nb = 0;
    MG_CHECK(launch_sweep(l0.op, SW_RESID, 1, P->u, P->f, P->p, 0.0, nullptr, nullptr, P->st));
    MG_CHECK(launch_dot(P->p, P->p, l0.nvert, P->partials, &nb, P->st));
    MG_CHECK(launch_reduce_finish(P->partials, nb, 1, &P->sc->r0, P->st));
    s = read_scalars(P);
    if (s != MG_OK) return s;
    rel = std::sqrt(P->h_sc->r0 / (P->ff > 0 ? P->ff : 1.0));
    P->need_restart = true;
  }
  if (result == MG_OK && rel > 2.0 * d.rtol) result = MG_ERR_NOT_CONVERGED;
  if (result == MG_ERR_NOT_CONVERGED) set_error("not converged: rel residual %.3e after %d cycles", rel, P->cycles);
  if (info) {
    memset(info, 0, sizeof(*info));
    info->status = result;
    info->cycles = P->cycles;
    info->publishes = P->publishes;
    info->final_s = min_s(P);
    info->rel_residual = rel;
    info->time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    info->assembly_ms = asm_ms;
    long long n0 = 0;
    int64_t bytes = 0;
    for (const ChunkStore& c : P->cur) {
      for (int k = 0; k < 3; ++k) info->cells_by_class[k + 1] += c.totals[k];
      n0 += P->chunk_cells - (c.totals[0] + c.totals[1] + c.totals[2]);
      bytes += (int64_t)c.bytes;
    }
    info->cells_by_class[0] = P->mixed ? n0 : 0;
    bytes += (int64_t)P->lev[0].ncell * (P->mixed ? 4 : 0);
    info->payload_bytes = bytes;
  }
  return result;
}

mg_status mg_inject_assembly_failure(mg_problem* P, int s) {
  if (!P || s < 0) {
    set_error("bad arguments");
    return MG_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lk(P->mu);
  P->inject_fail = s;
  return MG_OK;
}

mg_status mg_get_solution(const mg_problem* P, double* host_dst, size_t n) {
  if (!P || !host_dst || n != (size_t)P->lev[0].nvert) {
    set_error("bad arguments (n must be (N+1)^d)");
    return MG_ERR_INVALID;
  }
  MG_CHECK(cudaMemcpyAsync(host_dst, P->u, sizeof(double) * n, cudaMemcpyDeviceToHost, P->st));
  MG_CHECK(cudaStreamSynchronize(P->st));
  return MG_OK;
}

mg_status mg_get_element_matrices(const mg_problem* Pc, int level, double* host_dst, size_t n) {
  mg_problem* P = const_cast<mg_problem*>(Pc);
  if (!P || !host_dst || level < 0 || level >= P->L) {
    set_error("bad arguments");
    return MG_ERR_INVALID;
  }
  const Level& lv = P->lev[level];
  const int nv = 1 << P->dim;
  if (n != (size_t)lv.ncell * nv * nv) {
    set_error("n must be cells * 4^d");
    return MG_ERR_INVALID;
  }
  double* tmp = nullptr;
  cudaError_t e = mg_malloc_async(&tmp, sizeof(double) * n, P->st);
  if (e != cudaSuccess) return oom_or_cuda(e, "decode buffer");
  MG_CHECK(launch_decode_matrices(lv.op, nullptr, 0, tmp, P->st));
  MG_CHECK(cudaMemcpyAsync(host_dst, tmp, sizeof(double) * n, cudaMemcpyDeviceToHost, P->st));
  cudaFreeAsync(tmp, P->st);
  MG_CHECK(cudaStreamSynchronize(P->st));
  return MG_OK;
}

mg_status mg_get_cell_matrices(const mg_problem* Pc, int level, const int64_t* cells, size_t ncells,
                               double* host_dst) {
  mg_problem* P = const_cast<mg_problem*>(Pc);
  if (!P || !cells || !host_dst || level < 0 || level >= P->L) {
    set_error("bad arguments");
    return MG_ERR_INVALID;
  }
  const Level& lv = P->lev[level];
  for (size_t i = 0; i < ncells; ++i)
    if (cells[i] < 0 || cells[i] >= lv.ncell) {
      set_error("cell index %lld out of range", (long long)cells[i]);
      return MG_ERR_INVALID;
    }
  if (ncells == 0) return MG_OK;
  const int nv = 1 << P->dim;
  long long* dc = nullptr;
  double* tmp = nullptr;
  cudaError_t e = mg_malloc_async(&dc, sizeof(long long) * ncells, P->st);
  if (e == cudaSuccess) e = mg_malloc_async(&tmp, sizeof(double) * ncells * nv * nv, P->st);
  if (e != cudaSuccess) return oom_or_cuda(e, "gather buffers");
  MG_CHECK(cudaMemcpyAsync(dc, cells, sizeof(long long) * ncells, cudaMemcpyHostToDevice, P->st));
  MG_CHECK(launch_decode_matrices(lv.op, dc, (long long)ncells, tmp, P->st));
  MG_CHECK(cudaMemcpyAsync(host_dst, tmp, sizeof(double) * ncells * nv * nv, cudaMemcpyDeviceToHost, P->st));
  cudaFreeAsync(dc, P->st);
  cudaFreeAsync(tmp, P->st);
  MG_CHECK(cudaStreamSynchronize(P->st));
  return MG_OK;
}

mg_status mg_get_trace(const mg_problem* P, mg_trace_entry* out, size_t cap, size_t* n) {
  if (!P || !n || (cap && !out)) {
    set_error("bad arguments");
    return MG_ERR_INVALID;
  }
  *n = P->trace_log.size();
  for (size_t i = 0; i < cap && i < P->trace_log.size(); ++i) out[i] = P->trace_log[i];
  return MG_OK;
}

mg_status mg_get_cell_accuracy(const mg_problem* Pc, int32_t* s_out, size_t n) {
  mg_problem* P = const_cast<mg_problem*>(Pc);
  if (!P || !s_out || n != (size_t)P->lev[0].ncell) {
    set_error("bad arguments (n must be cells)");
    return MG_ERR_INVALID;
  }
  MG_CHECK(cudaStreamSynchronize(P->st));
  if (P->side) MG_CHECK(cudaStreamSynchronize(P->side));
  if (P->adapt) {
    std::vector<uint8_t> t(n);
    MG_CHECK(cudaMemcpy(t.data(), P->s_cell, n, cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < n; ++i) s_out[i] = t[i];
  } else {
    for (int c = 0; c < P->nchunk; ++c)
      for (long long i = 0; i < P->chunk_cells; ++i) s_out[(size_t)c * P->chunk_cells + i] = P->cur[c].s;
  }
  return MG_OK;
}

mg_status mg_paper_format(const mg_problem* Pc, double delta, uint8_t* p3_host, double* decoded_host, size_t n,
                          mg_paper_format_stats* stats) {
  mg_problem* P = const_cast<mg_problem*>(Pc);
  if (!P || n != (size_t)P->lev[0].ncell || !(delta >= 0.0) || !std::isfinite(delta)) {
    set_error("bad arguments (n must be cells, delta finite and >= 0)");
    return MG_ERR_INVALID;
  }
  const Level& l0 = P->lev[0];
  const int nv = 1 << P->dim;
  const size_t ne = (size_t)nv * nv;
  double* A = nullptr;
  double* At = nullptr;
  uint8_t* p3 = nullptr;
  unsigned long long* cnt = nullptr;   // hist[9], then the max-error bits
  cudaError_t e = mg_malloc_async(&A, sizeof(double) * n * ne, P->st);
  if (e == cudaSuccess && decoded_host) e = mg_malloc_async(&At, sizeof(double) * n * ne, P->st);
  if (e == cudaSuccess) e = mg_malloc_async(&p3, n, P->st);
  if (e == cudaSuccess) e = mg_malloc_async(&cnt, sizeof(unsigned long long) * 10, P->st);
  if (e != cudaSuccess) return oom_or_cuda(e, "paper format buffers");
  unsigned long long h[10];
  MG_CHECK(cudaMemsetAsync(cnt, 0, sizeof(h), P->st));
  MG_CHECK(launch_decode_matrices(l0.op, nullptr, 0, A, P->st));
  MG_CHECK(launch_paper_format(P->dim, (long long)n, A, P->eps_c, P->mixed ? 0 : 1, l0.op.hfac, delta, p3, At, cnt,
                               cnt + 9, P->st));
  MG_CHECK(cudaMemcpyAsync(h, cnt, sizeof(h), cudaMemcpyDeviceToHost, P->st));
  if (p3_host) MG_CHECK(cudaMemcpyAsync(p3_host, p3, n, cudaMemcpyDeviceToHost, P->st));
  if (decoded_host) MG_CHECK(cudaMemcpyAsync(decoded_host, At, sizeof(double) * n * ne, cudaMemcpyDeviceToHost, P->st));
  cudaFreeAsync(A, P->st);
  if (At) cudaFreeAsync(At, P->st);
  cudaFreeAsync(p3, P->st);
  cudaFreeAsync(cnt, P->st);
  MG_CHECK(cudaStreamSynchronize(P->st));
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    double paper = 0.0;
    for (int k = 0; k < 9; ++k) {
      stats->cells_by_p3[k] = (int64_t)h[k];
      paper += (double)h[k] * (1.0 + (double)ne * k);
    }
    stats->bytes_full = (double)n * ne * 8.0;
    stats->bytes_paper = paper;
    stats->compression = paper > 0 ? stats->bytes_full / paper : 0.0;
    double em;
    memcpy(&em, &h[9], sizeof(em));
    stats->max_abs_error = em;
  }
  return MG_OK;
}

namespace {
struct StateHeader {
  char magic[8];
  int32_t dim, n_cells, mixed, nchunk;
  int64_t chunk_cells, chunk_nseg, nvert;
  int32_t adapt, np;
  int32_t exact, pad0;
};
constexpr char kStateMagic[8] = {'M', 'G', 'S', 'T', 'A', 'T', 'E', '2'};

struct ChunkHeader {
  int32_t s;
  uint32_t totals[3];
};

// record bytes of classes 1..3 in the class pools
int pool_rec_bytes(int dim, int k) {
  static const int r3[3] = {32, 64, 112}, r2[3] = {16, 16, 32};
  return dim == 3 ? r3[k] : r2[k];
}

// exact mode: the FP64 surplus of a chunk's interface cells (none at s = 1)
size_t exact_state_bytes(const mg_problem* P, int chunk, int s) {
  const int NP = P->dim == 3 ? 28 : 6;
  return P->exact && s > 1 ? sizeof(double) * NP * (size_t)P->ilist_n[chunk] : 0;
}

size_t chunk_state_bytes(const mg_problem* P, const uint32_t totals[3]) {
  const int NP = P->dim == 3 ? 28 : 6;
  if (!P->mixed) return sizeof(double) * NP * (size_t)P->chunk_cells;
  size_t b = (size_t)P->chunk_nseg * kSegCells + sizeof(uint32_t) * 3 * (size_t)P->chunk_nseg;
  for (int k = 0; k < 3; ++k) b += (size_t)totals[k] * pool_rec_bytes(P->dim, k);
  return b;
}

bool jobs_pending(mg_problem* P) {
  std::lock_guard<std::mutex> lk(P->mu);
  return P->in_flight > 0 || !P->held.empty();
}
}  // namespace

mg_status mg_export_state(mg_problem* P, void* buf, size_t cap, size_t* size) {
  if (!P || !size) {
    set_error("bad arguments");
    return MG_ERR_INVALID;
  }
  if (jobs_pending(P)) {
    set_error("delayed assembly jobs are in flight");
    return MG_ERR_PENDING;
  }
  mg_status s = apply_inner_correction(P);
  if (s != MG_OK) return s;
  const Level& l0 = P->lev[0];
  size_t total = sizeof(StateHeader) + sizeof(double) * (size_t)l0.nvert;
  for (int c = 0; c < P->nchunk; ++c)
    total += sizeof(ChunkHeader) + chunk_state_bytes(P, P->cur[c].totals) + exact_state_bytes(P, c, P->cur[c].s);
  if (P->adapt) total += 2 * (size_t)P->chunk_cells * P->nchunk;
  *size = total;
  if (!buf) return MG_OK;
  if (cap < total) {
    set_error("buffer of %zu bytes, the state needs %zu", cap, total);
    return MG_ERR_INVALID;
  }
  MG_CHECK(cudaStreamSynchronize(P->st));
  uint8_t* w = static_cast<uint8_t*>(buf);
  StateHeader h{};
  memcpy(h.magic, kStateMagic, 8);
  h.dim = P->dim;
  h.n_cells = P->N;
  h.mixed = P->mixed ? 1 : 0;
  h.nchunk = P->nchunk;
  h.chunk_cells = P->chunk_cells;
  h.chunk_nseg = P->chunk_nseg;
  h.nvert = l0.nvert;
  h.adapt = P->adapt ? 1 : 0;
  h.np = P->dim == 3 ? 28 : 6;
  h.exact = P->exact ? 1 : 0;
  memcpy(w, &h, sizeof(h));
  w += sizeof(h);
  MG_CHECK(cudaMemcpy(w, P->u, sizeof(double) * (size_t)l0.nvert, cudaMemcpyDeviceToHost));
  w += sizeof(double) * (size_t)l0.nvert;
  for (int ci = 0; ci < P->nchunk; ++ci) {
    const ChunkStore& c = P->cur[ci];
    ChunkHeader ch{};
    ch.s = c.s;
    for (int k = 0; k < 3; ++k) ch.totals[k] = c.totals[k];
    memcpy(w, &ch, sizeof(ch));
    w += sizeof(ch);
    if (!P->mixed) {
      const size_t b = chunk_state_bytes(P, c.totals);
      MG_CHECK(cudaMemcpy(w, c.a64, b, cudaMemcpyDeviceToHost));
      w += b;
      continue;
    }
    const size_t cb = (size_t)P->chunk_nseg * kSegCells, sb = sizeof(uint32_t) * 3 * (size_t)P->chunk_nseg;
    MG_CHECK(cudaMemcpy(w, c.cls, cb, cudaMemcpyDeviceToHost));
    w += cb;
    MG_CHECK(cudaMemcpy(w, c.seg_base, sb, cudaMemcpyDeviceToHost));
    w += sb;
    for (int k = 0; k < 3; ++k) {
      const size_t pb = (size_t)c.totals[k] * pool_rec_bytes(P->dim, k);
      if (pb) MG_CHECK(cudaMemcpy(w, c.pool[k], pb, cudaMemcpyDeviceToHost));
      w += pb;
    }
    const size_t xb = exact_state_bytes(P, ci, c.s);
    if (xb) MG_CHECK(cudaMemcpy(w, c.x64, xb, cudaMemcpyDeviceToHost));
    w += xb;
  }
  if (P->adapt) {
    const size_t nc = (size_t)P->chunk_cells * P->nchunk;
    MG_CHECK(cudaMemcpy(w, P->final_flags, nc, cudaMemcpyDeviceToHost));
    w += nc;
    MG_CHECK(cudaMemcpy(w, P->s_cell, nc, cudaMemcpyDeviceToHost));
  }
  return MG_OK;
}

mg_status mg_import_state(mg_problem* P, const void* buf, size_t size) {
  if (!P || !buf || size < sizeof(StateHeader)) {
    set_error("bad arguments");
    return MG_ERR_INVALID;
  }
  if (jobs_pending(P)) {
    set_error("delayed assembly jobs are in flight");
    return MG_ERR_PENDING;
  }
  const uint8_t* r = static_cast<const uint8_t*>(buf);
  const uint8_t* end = r + size;
  StateHeader h;
  memcpy(&h, r, sizeof(h));
  r += sizeof(h);
  const Level& l0 = P->lev[0];
  if (memcmp(h.magic, kStateMagic, 8) != 0 || h.dim != P->dim || h.n_cells != P->N ||
      h.mixed != (P->mixed ? 1 : 0) || h.nchunk != P->nchunk || h.chunk_cells != P->chunk_cells ||
      h.chunk_nseg != P->chunk_nseg || h.nvert != l0.nvert || h.adapt != (P->adapt ? 1 : 0) ||
      h.exact != (P->exact ? 1 : 0)) {
    set_error("not a state of a problem with this descriptor");
    return MG_ERR_INVALID;
  }
  // validate the whole layout before changing anything
  const uint8_t* q = r + sizeof(double) * (size_t)l0.nvert;
  std::vector<ChunkHeader> chs(P->nchunk);
  for (int c = 0; c < P->nchunk; ++c) {
    if (q + sizeof(ChunkHeader) > end) {
      set_error("truncated state");
      return MG_ERR_INVALID;
    }
    memcpy(&chs[c], q, sizeof(ChunkHeader));
    if (chs[c].s < 1 || chs[c].s > 64 ||
        (uint64_t)chs[c].totals[0] + chs[c].totals[1] + chs[c].totals[2] > (uint64_t)P->chunk_cells) {
      set_error("corrupt chunk header");
      return MG_ERR_INVALID;
    }
    q += sizeof(ChunkHeader) + chunk_state_bytes(P, chs[c].totals) + exact_state_bytes(P, c, chs[c].s);
  }
  if (P->adapt) q += 2 * (size_t)P->chunk_cells * P->nchunk;
  if (q != end) {
    set_error("state size %zu does not match its contents", size);
    return MG_ERR_INVALID;
  }
  cudaStream_t st = P->st;
  MG_CHECK(cudaMemcpyAsync(P->u, r, sizeof(double) * (size_t)l0.nvert, cudaMemcpyHostToDevice, st));
  r += sizeof(double) * (size_t)l0.nvert;
  for (int c = 0; c < P->nchunk; ++c) {
    r += sizeof(ChunkHeader);
    ChunkStore cs;
    cs.s = chs[c].s;
    for (int k = 0; k < 3; ++k) cs.totals[k] = chs[c].totals[k];
    cudaError_t e;
    if (!P->mixed) {
      const size_t b = chunk_state_bytes(P, cs.totals);
      if ((e = mg_malloc_async(&cs.a64, b, st)) != cudaSuccess) return oom_or_cuda(e, "chunk storage");
      MG_CHECK(cudaMemcpyAsync(cs.a64, r, b, cudaMemcpyHostToDevice, st));
      cs.bytes = b;
      r += b;
    } else {
      const size_t cb = (size_t)P->chunk_nseg * kSegCells, sb = sizeof(uint32_t) * 3 * (size_t)P->chunk_nseg;
      e = mg_malloc_async(&cs.cls, cb, st);
      if (e == cudaSuccess) e = mg_malloc_async(&cs.seg_base, sb, st);
      if (e != cudaSuccess) return oom_or_cuda(e, "chunk classes");
      MG_CHECK(cudaMemcpyAsync(cs.cls, r, cb, cudaMemcpyHostToDevice, st));
      r += cb;
      MG_CHECK(cudaMemcpyAsync(cs.seg_base, r, sb, cudaMemcpyHostToDevice, st));
      r += sb;
      cs.bytes = cb + sb;
      for (int k = 0; k < 3; ++k) {
        const size_t pb = (size_t)cs.totals[k] * pool_rec_bytes(P->dim, k);
        if (pb) {
          if ((e = mg_malloc_async(&cs.pool[k], pb, st)) != cudaSuccess) return oom_or_cuda(e, "payload pool");
          MG_CHECK(cudaMemcpyAsync(cs.pool[k], r, pb, cudaMemcpyHostToDevice, st));
        }
        cs.bytes += pb;
        r += pb;
      }
      const size_t xb = exact_state_bytes(P, c, cs.s);
      if (xb) {
        if ((e = mg_malloc_async(&cs.x64, xb, st)) != cudaSuccess) return oom_or_cuda(e, "exact surplus");
        MG_CHECK(cudaMemcpyAsync(cs.x64, r, xb, cudaMemcpyHostToDevice, st));
        cs.bytes += xb;
        r += xb;
      }
    }
    // the copies read pageable host memory: they are staged before the call returns
    install(P, c, cs);
  }
  if (P->adapt) {
    const size_t nc = (size_t)P->chunk_cells * P->nchunk;
    MG_CHECK(cudaMemcpyAsync(P->final_flags, r, nc, cudaMemcpyHostToDevice, st));
    r += nc;
    MG_CHECK(cudaMemcpyAsync(P->s_cell, r, nc, cudaMemcpyHostToDevice, st));
    P->wlast = P->cur;
  }
  mg_status s = upload_tables(P);
  if (s == MG_OK) s = rebuild_coarse(P);
  if (s != MG_OK) return s;
  MG_CHECK(cudaStreamSynchronize(st));
  P->have_correction = false;
  P->need_restart = true;
  P->keep_dir = false;
  P->resid_fresh = false;
  P->u_zero = false;
  return MG_OK;
}

mg_status mg_get_coarse_classes(const mg_problem* P, int level, uint8_t* cls, size_t n) {
  if (!P || !cls || level < 1 || level >= P->L || n != (size_t)P->lev[level].ncell || !P->lev[level].cls) {
    set_error("bad arguments (level >= 1, n cells of the level, coarse compression on)");
    return MG_ERR_INVALID;
  }
  MG_CHECK(cudaStreamSynchronize(P->st));
  MG_CHECK(cudaMemcpy(cls, P->lev[level].cls, n, cudaMemcpyDeviceToHost));
  return MG_OK;
}

mg_status mg_get_cell_data(const mg_problem* Pc, uint8_t* cls, double* eps_c, size_t n) {
  mg_problem* P = const_cast<mg_problem*>(Pc);
  if (!P || n != (size_t)P->lev[0].ncell) {
    set_error("bad arguments (n must be cells)");
    return MG_ERR_INVALID;
  }
  MG_CHECK(cudaStreamSynchronize(P->st));
  if (cls) {
    std::vector<uint8_t> pad((size_t)P->chunk_nseg * kSegCells);
    for (int c = 0; c < P->nchunk; ++c) {
      if (!P->mixed) {
        memset(cls + (size_t)c * P->chunk_cells, 0, P->chunk_cells);
        continue;
      }
      MG_CHECK(cudaMemcpy(pad.data(), P->cur[c].cls, pad.size(), cudaMemcpyDeviceToHost));
      for (long long row = 0; row < P->chunk_rows; ++row)
        for (int x = 0; x < P->N; ++x)
          cls[(size_t)c * P->chunk_cells + row * P->N + x] =
              pad[(size_t)(row * P->nseg_x + x / kSegCells) * kSegCells + (x % kSegCells)];
    }
  }
  if (eps_c) {
    if (P->mixed) {
      std::vector<float> t(n);
      MG_CHECK(cudaMemcpy(t.data(), P->eps_c, sizeof(float) * n, cudaMemcpyDeviceToHost));
      for (size_t i = 0; i < n; ++i) eps_c[i] = t[i];
    } else {
      MG_CHECK(cudaMemcpy(eps_c, P->eps_c, sizeof(double) * n, cudaMemcpyDeviceToHost));
    }
  }
  return MG_OK;
}

mg_status mg_apply_level(mg_problem* P, int level, int op, int inner, const double* x, const double* b, double* y) {
  if (!P || level < 0 || level >= P->L || op < 0 || op > 2 || !x || !y || (op != 0 && !b)) {
    set_error("bad arguments");
    return MG_ERR_INVALID;
  }
  Level& lv = P->lev[level];
  const int vec64 = (inner && P->mixed) ? 0 : 1;
  const size_t n = lv.nvert;
  const size_t eb = vec64 ? 8 : 4;
  void *dx = nullptr, *db = nullptr, *dy = nullptr;
  double* tmp = nullptr;
  cudaError_t e = mg_malloc_async(&dx, eb * n, P->st);
  if (e == cudaSuccess) e = mg_malloc_async(&db, eb * n, P->st);
  if (e == cudaSuccess) e = mg_malloc_async(&dy, eb * n, P->st);
  if (e == cudaSuccess) e = mg_malloc_async(&tmp, 8 * n, P->st);
  if (e != cudaSuccess) return oom_or_cuda(e, "buffers");
  std::vector<double> zeros;
  const double* bsrc = b;
  if (!b) {
    zeros.assign(n, 0.0);
    bsrc = zeros.data();
  }
  MG_CHECK(cudaMemsetAsync(dy, 0, eb * n, P->st));
  if (vec64) {
    MG_CHECK(cudaMemcpyAsync(dx, x, 8 * n, cudaMemcpyHostToDevice, P->st));
    MG_CHECK(cudaMemcpyAsync(db, bsrc, 8 * n, cudaMemcpyHostToDevice, P->st));
  } else {
    MG_CHECK(cudaMemcpyAsync(tmp, x, 8 * n, cudaMemcpyHostToDevice, P->st));
    MG_CHECK(launch_convert(n, 0, tmp, dx, P->st));
    MG_CHECK(cudaStreamSynchronize(P->st));
    MG_CHECK(cudaMemcpyAsync(tmp, bsrc, 8 * n, cudaMemcpyHostToDevice, P->st));
    MG_CHECK(launch_convert(n, 0, tmp, db, P->st));
  }
  const int mode = op == 0 ? SW_MATVEC : (op == 1 ? SW_JACOBI : SW_RESID);
  int nb = 0;
  MG_CHECK(launch_sweep(lv.op, mode, vec64, dx, db, dy, P->desc.omega, P->partials, &nb, P->st));
  if (vec64) {
    MG_CHECK(cudaMemcpyAsync(y, dy, 8 * n, cudaMemcpyDeviceToHost, P->st));
  } else {
    MG_CHECK(launch_convert(n, 1, dy, tmp, P->st));
    MG_CHECK(cudaMemcpyAsync(y, tmp, 8 * n, cudaMemcpyDeviceToHost, P->st));
  }
  MG_CHECK(cudaStreamSynchronize(P->st));
  cudaFreeAsync(dx, P->st);
  cudaFreeAsync(db, P->st);
  cudaFreeAsync(dy, P->st);
  cudaFreeAsync(tmp, P->st);
  MG_CHECK(cudaStreamSynchronize(P->st));
  return MG_OK;
}

mg_status mg_apply_transfer(mg_problem* P, int level, int op, int inner, const double* x, const double* b,
                            const double* c, double* out) {
  if (!P || level < 0 || level + 1 >= P->L || op < 0 || op > 1 || !x || !b || !out || (op == 1 && !c)) {
    set_error("bad arguments");
    return MG_ERR_INVALID;
  }
  Level& lv = P->lev[level];
  Level& lc = P->lev[level + 1];
  const int vec64 = (inner && P->mixed) ? 0 : 1;
  const size_t n = lv.nvert, nc = lc.nvert;
  const size_t eb = vec64 ? 8 : 4;
  void *dx = nullptr, *db = nullptr, *dy = nullptr, *dc = nullptr;
  double* tmp = nullptr;
  cudaError_t e = mg_malloc_async(&dx, eb * n, P->st);
  if (e == cudaSuccess) e = mg_malloc_async(&db, eb * n, P->st);
  if (e == cudaSuccess) e = mg_malloc_async(&dy, eb * n, P->st);
  if (e == cudaSuccess) e = mg_malloc_async(&dc, eb * nc, P->st);
  if (e == cudaSuccess) e = mg_malloc_async(&tmp, 8 * n, P->st);
  if (e != cudaSuccess) return oom_or_cuda(e, "buffers");
  // host FP64 -> device vector of the level's arithmetic
  auto upload = [&](const double* h, void* d, size_t m) -> cudaError_t {
    if (vec64) return cudaMemcpyAsync(d, h, 8 * m, cudaMemcpyHostToDevice, P->st);
    cudaError_t r = cudaMemcpyAsync(tmp, h, 8 * m, cudaMemcpyHostToDevice, P->st);
    if (r == cudaSuccess) r = launch_convert(m, 0, tmp, d, P->st);
    if (r == cudaSuccess) r = cudaStreamSynchronize(P->st);   // tmp is reused
    return r;
  };
  auto download = [&](const void* d, double* h, size_t m) -> cudaError_t {
    if (vec64) return cudaMemcpyAsync(h, d, 8 * m, cudaMemcpyDeviceToHost, P->st);
    cudaError_t r = launch_convert(m, 1, d, tmp, P->st);
    if (r == cudaSuccess) r = cudaMemcpyAsync(h, tmp, 8 * m, cudaMemcpyDeviceToHost, P->st);
    return r;
  };
  MG_CHECK(upload(x, dx, n));
  MG_CHECK(upload(b, db, n));
  MG_CHECK(cudaMemsetAsync(dc, 0, eb * nc, P->st));
  MG_CHECK(cudaMemsetAsync(dy, 0, eb * n, P->st));
  if (op == 0) {
    e = level == 0 ? launch_resid_restrict(lv.op, vec64, dx, db, dy, P->zr, dc, P->st) : cudaErrorNotSupported;
    if (e == cudaErrorNotSupported) {
      MG_CHECK(launch_sweep(lv.op, SW_RESID, vec64, dx, db, dy, P->desc.omega, nullptr, nullptr, P->st));
      e = launch_restrict(P->dim, lc.N, vec64, dy, dc, P->st);
    }
    MG_CHECK(e);
    MG_CHECK(download(dc, out, nc));
  } else {
    MG_CHECK(upload(c, dc, nc));
    MG_CHECK(launch_prolong_add(P->dim, lc.N, vec64, dc, dx, P->st));
    MG_CHECK(launch_sweep(lv.op, SW_JACOBI, vec64, dx, db, dy, P->desc.omega, nullptr, nullptr, P->st));
    MG_CHECK(download(dy, out, n));
  }
  MG_CHECK(cudaStreamSynchronize(P->st));
  cudaFreeAsync(dx, P->st);
  cudaFreeAsync(db, P->st);
  cudaFreeAsync(dy, P->st);
  cudaFreeAsync(dc, P->st);
  cudaFreeAsync(tmp, P->st);
  MG_CHECK(cudaStreamSynchronize(P->st));
  return MG_OK;
}

mg_status mg_profile_kernel(mg_problem* P, int which, int reps, double* ms_per_launch) {
  if (!P || reps < 1 || which < 0 || which > 11 || !ms_per_launch || (which >= 5 && which <= 9 && P->L < 2) ||
      (which == 9 && P->L < 3) || (which >= 10 && !P->mixed)) {
    set_error("bad arguments");
    return MG_ERR_INVALID;
  }
  Level& l0 = P->lev[0];
  const int vec64 = P->mixed ? 0 : 1;
  // which = 4: the integration kernel alone on chunk 0 at the final accuracy
  // (its interface cells, or every cell), into scratch outputs
  AsmLaunch a{};
  void* asm_out = nullptr;
  uint8_t* asm_cls = nullptr;
  if (which == 4) {
    if (jobs_pending(P)) {
      set_error("delayed assembly jobs are in flight");
      return MG_ERR_PENDING;
    }
    const int NP = P->dim == 3 ? 28 : 6;
    a.dim = P->dim;
    a.N = P->N;
    a.s = final_s(P);
    a.kind = P->eps.kind;
    a.prec64 = P->mixed ? 0 : 1;
    a.cell0 = 0;
    a.ncell = P->chunk_cells;
    a.eps_host = &P->eps;
    a.hfac = fine_op(P).hfac;
    a.eps_c = P->eps_c;
    a.nseg_x = P->nseg_x;
    a.tau = P->desc.compress_tau;
    if (P->ilist) {
      a.list = P->ilist;
      a.nlist = P->ilist_n[0];
    }
    cudaError_t e = P->mixed ? mg_malloc_async(&asm_cls, (size_t)P->chunk_nseg * kSegCells, P->st)
                             : mg_malloc_async(&asm_out, sizeof(double) * NP * (size_t)P->chunk_cells, P->st);
    if (e == cudaSuccess && P->exact && P->ilist_n[0] > 0)
      e = mg_malloc_async(&a.out_x64, sizeof(double) * NP * (size_t)P->ilist_n[0], P->st);
    if (e != cudaSuccess) return oom_or_cuda(e, "profile buffers");
    if (P->mixed) {
      a.out_rec = P->scratch;
      a.out_cls = asm_cls;
      if (P->exact) {
        a.eps64 = P->eps64;
        a.xpos = P->xpos;
      }
    } else {
      a.out_full = asm_out;
    }
  }
  cudaEvent_t e0, e1;
  MG_CHECK(cudaEventCreate(&e0));
  MG_CHECK(cudaEventCreate(&e1));
  auto launch = [&](int i) -> cudaError_t {
    void* x = (i & 1) ? l0.x1 : l0.x0;
    void* y = (i & 1) ? l0.x0 : l0.x1;
    switch (which) {
      case 0: return launch_sweep(l0.op, SW_JACOBI, vec64, x, l0.b, y, P->desc.omega, nullptr, nullptr, P->st);
      case 1: return launch_sweep(l0.op, SW_MATVEC, 1, P->p, P->r, P->q, 0.0, P->partials, nullptr, P->st);
      case 2: return launch_sweep(l0.op, SW_RESID, 1, P->u, P->f, P->q, 0.0, nullptr, nullptr, P->st);
      case 3: return launch_galerkin(l0.op, P->mixed ? 0 : 1, P->lev[1].full_store, P->st);
      case 5: {   // b_c = R (b - A u) as in the V-cycle
        cudaError_t r = launch_resid_restrict(l0.op, vec64, l0.x0, l0.b, l0.x1, P->zr, P->lev[1].b, P->st);
        if (r != cudaErrorNotSupported) return r;
        r = launch_sweep(l0.op, SW_RESID, vec64, l0.x0, l0.b, l0.x1, P->desc.omega, nullptr, nullptr, P->st);
        return r == cudaSuccess ? launch_restrict(P->dim, P->lev[1].N, vec64, l0.x1, P->lev[1].b, P->st) : r;
      }
      case 6: return launch_restrict(P->dim, P->lev[1].N, vec64, l0.x1, P->lev[1].b, P->st);
      case 7:
      case 8:
      case 9: {   // one V-cycle from the finest level, or from the next coarser ones
        mg_status stt = MG_OK;
        P->u1_ready = false;   // the whole cycle, its first smoothing step included
        vcycle_enqueue(P, which - 7, &stt);
        return stt == MG_OK ? cudaSuccess : cudaErrorUnknown;
      }
      default: return launch_assemble(a, P->st);
    }
  };
  if (which >= 10) {
    // one inner iteration of the mixed path as the solve runs it (continuing
    // the Krylov process of the last solve), back to back (10) or each
    // followed by the host's read of the scalars, as the solve does (11)
    mg_status s = apply_inner_correction(P);
    if (s == MG_OK && P->need_restart) s = outer_restart(P);
    if (s != MG_OK) return s;
    P->first = false;
    auto iter = [&]() -> mg_status {
      mg_status r = outer_iteration(P);
      if (r == MG_OK && which == 11) r = read_scalars(P);
      return r;
    };
    for (int i = 0; i < 3; ++i)
      if ((s = iter()) != MG_OK) return s;
    MG_CHECK(cudaEventRecord(e0, P->st));
    for (int i = 0; i < reps; ++i)
      if ((s = iter()) != MG_OK) return s;
    MG_CHECK(cudaEventRecord(e1, P->st));
    MG_CHECK(cudaEventSynchronize(e1));
    float ms = 0.f;
    MG_CHECK(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms_per_launch = ms / reps;
    P->have_correction = false;   // the extra iterations' correction is dropped
    P->e_pending = false;
    P->need_restart = true;
    return MG_OK;
  }
  for (int i = 0; i < 3; ++i) MG_CHECK(launch(i));
  MG_CHECK(cudaEventRecord(e0, P->st));
  for (int i = 0; i < reps; ++i) MG_CHECK(launch(i));
  MG_CHECK(cudaEventRecord(e1, P->st));
  MG_CHECK(cudaEventSynchronize(e1));
  float ms = 0.f;
  MG_CHECK(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (asm_out) cudaFreeAsync(asm_out, P->st);
  if (asm_cls) cudaFreeAsync(asm_cls, P->st);
  if (a.out_x64) cudaFreeAsync(a.out_x64, P->st);
  *ms_per_launch = ms / reps;
  P->need_restart = true;
  return MG_OK;
}

uint64_t mg_launch_count(void) { return (uint64_t)launch_count(); }

mg_status mg_vcycle_apply(mg_problem* P, const double* b, double* e_out) {
  if (!P || !b || !e_out) {
    set_error("bad arguments");
    return MG_ERR_INVALID;
  }
  Level& l0 = P->lev[0];
  const size_t n = l0.nvert;
  double* tmp = nullptr;
  cudaError_t e = mg_malloc_async(&tmp, 8 * n, P->st);
  if (e != cudaSuccess) return oom_or_cuda(e, "buffer");
  // the V-cycle reads lev[0].b (aliases r on FP64 paths): stage b there
  P->u1_ready = false;
  if (P->mixed) {
    MG_CHECK(cudaMemcpyAsync(tmp, b, 8 * n, cudaMemcpyHostToDevice, P->st));
    MG_CHECK(launch_convert(n, 0, tmp, l0.b, P->st));
  } else {
    MG_CHECK(cudaMemcpyAsync(l0.b, b, 8 * n, cudaMemcpyHostToDevice, P->st));
  }
  mg_status stt = MG_OK;
  void* z = cycle_enqueue(P, &stt);
  if (stt != MG_OK) return stt;
  if (P->mixed) {
    MG_CHECK(launch_convert(n, 1, z, tmp, P->st));
    MG_CHECK(cudaMemcpyAsync(e_out, tmp, 8 * n, cudaMemcpyDeviceToHost, P->st));
  } else {
    MG_CHECK(cudaMemcpyAsync(e_out, z, 8 * n, cudaMemcpyDeviceToHost, P->st));
  }
  cudaFreeAsync(tmp, P->st);
  MG_CHECK(cudaStreamSynchronize(P->st));
  P->need_restart = true;
  return MG_OK;
}

}  // extern "C"
