// Internal definitions shared by the CUDA translation units of libmg.so.
//
// Element matrices (Eq. "weak-form-of-assembly", one 2^d x 2^d matrix per
// cell) are symmetric with zero row sums, so only the NP = 2^d (2^d - 1) / 2
// off-diagonal entries a < b are stored; the diagonal is minus the row sum.
// Pair p(a, b), a < b, is numbered lexicographically.
#pragma once
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <stdint.h>

namespace mg {

constexpr int kMaxLevels = 12;
constexpr int kMaxModes = 32;
constexpr int kMaxBoxes = 64;
constexpr int kSegCells = 32;  // cells per storage segment along x

template <int D>
struct Dim {
  static constexpr int NV = 1 << D;                 // vertices per cell
  static constexpr int NP = NV * (NV - 1) / 2;      // stored off-diagonal pairs
  static constexpr int F = NV - 1;                  // entries per row besides the diagonal
  // record bytes of storage classes 1 (FP8 + scale), 2 (FP16 + scale), 3 (FP32)
  static constexpr int REC1 = D == 3 ? 32 : 16;
  static constexpr int REC2 = D == 3 ? 64 : 16;
  static constexpr int REC3 = D == 3 ? 112 : 32;
  static constexpr int REC_MAX = REC3;
};

__host__ __device__ constexpr inline int pair_index(int nv, int a, int b) {
  // a < b
  return a * (2 * nv - a - 1) / 2 + (b - a - 1);
}
__host__ __device__ constexpr inline int pair_of(int nv, int a, int b) {
  return a < b ? pair_index(nv, a, b) : pair_index(nv, b, a);
}
__host__ __device__ constexpr inline int popc_small(int x) {
  return (x & 1) + ((x >> 1) & 1) + ((x >> 2) & 1);
}

// eps = 1 element matrix on the unit reference cell (constant-eps precompute
// of Section "Numerical computation of stencils"): off-diagonal value by the
// Hamming distance of the two local vertices; physical matrix = h^(d-2) times it.
template <int D>
__host__ __device__ constexpr inline double kref_off(int ham) {
  return D == 2 ? (ham == 1 ? -1.0 / 6.0 : -1.0 / 3.0) : (ham == 1 ? 0.0 : -1.0 / 12.0);
}
template <int D>
__host__ __device__ constexpr inline double kref_diag() {
  return D == 2 ? 2.0 / 3.0 : 1.0 / 3.0;
}

// ------------------------------------------------------------ material field
enum EpsKind { EPS_CONST = 0, EPS_DISC = 1, EPS_FOURIER = 2, EPS_BOXES = 3, EPS_THETA = 4 };

struct EpsDev {
  int kind, dim, n_modes, n_boxes;
  double v_out, v_in;
  double center[3];
  double r2lim;        // radius * radius (IEEE product)
  double amp;          // sigma * sqrt(2 / M)
  double theta;
  double jump_x, jump_factor;
  int k[kMaxModes][3];
  double phi_over_pi[kMaxModes];   // phase / pi
  double box_lo[kMaxBoxes][3];
  double box_hi[kMaxBoxes][3];
  // FP32 copies for the FP32 arithmetic path
  float amp_f, v_out_f, v_in_f, jump_factor_f;
  float phi_over_pi_f[kMaxModes];
};

// Sample positions x(m) = (2m + 1) / (2 N s), m = i s + j the global sub-box
// index along an axis, are monotone in m, so the FP64 decisions lo <= x(m),
// x(m) < hi and x(m) >= jump_x reduce to integer thresholds computed once on
// the host with the same FP64 expression: lo <= x(m) < hi  <=>  mlo <= m < mhi.
struct SampleThresholds {
  int mlo[kMaxBoxes][3], mhi[kMaxBoxes][3];
  int mjump;   // x(m) >= jump_x  <=>  m >= mjump (INT_MAX when there is no jump)
};

// ------------------------------------------------------------ operator storage
// Compressed finest level (mixed paths), one chunk = a slab of whole cell
// layers along the last axis.  cls holds one byte per cell, padded to
// kSegCells per x-row segment: cls[(row * nseg_x + sx) * 32 + lane].  Records
// of class k (1..3) are stored in pool[k-1] ordered by segment then x;
// seg_base[(k-1) * nseg + seg] is the number of class-k cells before segment seg.
struct CmpChunk {
  const uint8_t* cls;
  const uint32_t* seg_base;
  const uint8_t* pool[3];
  long long nseg;
  // exact FP64 surplus of the chunk's interface cells [list position][NP]
  // (piecewise-constant fields on the mixed paths; nullptr: all zero, s = 1)
  const double* x64;
};

// Full storage: SoA off-diagonals a[p * chunk_cells + local_cell].
struct FullChunk {
  const void* a;
};

struct LevelOp {
  int N;                  // cells per axis
  int dim;
  int layers;             // cell layers (last axis) per chunk
  int nchunk;
  long long chunk_cells;  // cells per chunk (layers * N^(d-1))
  int nseg_x;             // segments per x-row
  int compressed;         // 1: CmpChunk + eps_c; 0: FullChunk
  int elem64;             // full storage element type: 1 double, 0 float
  const float* eps_c;     // compressed: cell-centre eps (FP32) of all cells
  const CmpChunk* cmp;    // device array [nchunk]
  const FullChunk* full;  // device array [nchunk]
  double hfac;            // h^(d-2)
  float gk32;             // 3D: h * (-1/12), the nonzero off-diagonal of K_ref h^(d-2)
  double gk64;
  // compressed 3D finest level: vertices with an adjacent cell of class > 0
  const int* touched;     // vertex indices (nullptr: no split sweep)
  const int* ntouched;    // device count
  // 27-point stencils of the first tcap touched vertices, SoA [27][tcap]:
  // entry 13 is the diagonal, the others the off-diagonal couplings (the
  // operator is applied in difference form, sum_k c_k (u_k - u_v))
  float* tcoef;
  int tcap;
  // bit v of tmask: vertex v is in the touched list (nullptr: no fused
  // residual + restriction)
  uint32_t* tmask;
  // split sweep: eps_c with rows padded to N+1 floats (zero pad), for float4 loads
  const float* eps_pad;
  // levels with full storage (and finest levels whose cells all carry a
  // surplus): assembled 3^d-point vertex stencils, symmetric storage SoA
  // [(3^d+1)/2][(N+1)^d]: entry 0 the diagonal, entry m > 0 the coupling to
  // the neighbour at block offset C + m (C the centre of the 3^d block); the
  // coupling to C - m is the neighbour's entry m.  Rebuilt with the cell matrices.
  const void* stencil;
  // Exact FP64 operator of the mixed paths on piecewise-constant fields (the
  // FP64 outer residual and matvec read it; the FP32 sweeps read the lossy
  // records): FP64 cell-centre eps of every cell, the position of each cell
  // in its chunk's interface list (-1: no surplus) and the vertices next to
  // an interface cell.  eps64 == nullptr: the FP64 applications use the
  // stored (lossy) operator.
  const double* eps64;
  const int* xpos;
  const int* touched64;
  const int* ntouched64;
  // FP64 bulk pass in vertex form (split finest level; nullptr: the cell
  // form), built once from the cell-centre eps (eps64, else eps_c), h = 1/N:
  // w64[0][v] = 5 h/12 G_v (G_v: eps summed over the 8 cells at v),
  // w64[1..3][v] = h/12 W of the edges (v, v+x), (v, v+y), (v, v+z) (eps summed
  // over the 4 cells at the edge), es64 = h/12 eps_c with rows padded to N+1
  // cells (zero pad)
  const double* w64[4];
  const double* es64;
};

// ------------------------------------------------------------ programmatic dependent launch
// A kernel launched with programmatic stream serialization may start while
// its predecessor in the stream still runs.  griddepcontrol.wait blocks the
// calling thread until the predecessor grid completed and its memory is
// visible (a no-op in a kernel launched without the attribute);
// griddepcontrol.launch_dependents lets the next such kernel be scheduled
// once every block of this grid executed it (or exited), so a grid never
// waits on a dependent that took the slots its own unscheduled blocks need.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
// kernels launched by launch_chain begin with this.  The wait comes first: a
// dependent may then be scheduled only once this grid's predecessors have
// completed, so a dependent that reads before its own wait (the fix-up pass,
// which reads only inputs of the sweep before waiting) never sees data of a
// kernel still running two steps back.
__device__ __forceinline__ void pdl_begin() {
  pdl_wait();
  pdl_trigger();
}

// whether the coarse-level and transfer kernels are launched as programmatic
// dependents of their predecessors (MG_NO_PDL=1 turns it off)
bool pdl_enabled();

// launches kern (which calls pdl_begin() before reading what a predecessor
// writes) with programmatic stream serialization when enabled
template <typename... KArgs, typename... Args>
inline cudaError_t launch_chain(void (*kern)(KArgs...), dim3 g, dim3 b, size_t smem, cudaStream_t st,
                                Args... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = g;
  cfg.blockDim = b;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// ------------------------------------------------------------ helpers
__device__ __forceinline__ long long cell_index(int D, int N, int i, int j, int k) {
  return D == 2 ? (long long)j * N + i : ((long long)k * N + j) * N + i;
}

// rank of `lane` among the cells of class k in a 32-byte class segment
__device__ __forceinline__ unsigned rank_in_segment(const uint8_t* seg, int lane, int k) {
  const uint4* q = reinterpret_cast<const uint4*>(seg);
  uint4 w0 = __ldg(q), w1 = __ldg(q + 1);
  unsigned words[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
  unsigned kk = 0x01010101u * (unsigned)k;
  unsigned cnt = 0;
#pragma unroll
  for (int w = 0; w < 8; ++w) {
    unsigned eq = __vcmpeq4(words[w], kk);          // 0xff per equal byte
    int lo = w * 4;
    unsigned keep;
    if (lane >= lo + 4) keep = 0xffffffffu;
    else if (lane <= lo) keep = 0u;
    else keep = 0xffffffffu >> (8 * (4 - (lane - lo)));
    cnt += __popc(eq & keep);
  }
  return cnt >> 3;
}

// Decoded surplus entry p of a record of class cls (1..3).
template <int D>
__device__ __forceinline__ float decode_entry(const uint8_t* rec, int cls, int p) {
  if (cls == 1) {
    float scale = *reinterpret_cast<const float*>(rec);
    __nv_fp8_e4m3 v;
    v.__x = rec[4 + p];
    return float(v) * scale;
  } else if (cls == 2) {
    float scale = *reinterpret_cast<const float*>(rec);
    __half v = *reinterpret_cast<const __half*>(rec + 4 + 2 * p);
    return __half2float(v) * scale;
  } else {
    return *reinterpret_cast<const float*>(rec + 4 * p);
  }
}

// Pointer to the record of a cell with class cls > 0 in a compressed chunk.
template <int D>
__device__ __forceinline__ const uint8_t* cell_record(const CmpChunk& ck, int N, int nseg_x,
                                                      long long local_cell, int cls) {
  long long row = local_cell / N;
  int x = (int)(local_cell - row * N);
  long long seg = row * nseg_x + (x >> 5);
  const uint8_t* sg = ck.cls + seg * kSegCells;
  unsigned r = rank_in_segment(sg, x & 31, cls);
  unsigned base = ck.seg_base[(cls - 1) * ck.nseg + seg];
  int recb = cls == 1 ? Dim<D>::REC1 : (cls == 2 ? Dim<D>::REC2 : Dim<D>::REC3);
  return ck.pool[cls - 1] + (size_t)(base + r) * recb;
}

__device__ __forceinline__ uint8_t cell_class(const CmpChunk& ck, int N, int nseg_x, long long local_cell) {
  long long row = local_cell / N;
  int x = (int)(local_cell - row * N);
  return ck.cls[(row * nseg_x + (x >> 5)) * kSegCells + (x & 31)];
}

// ------------------------------------------------------------ host API (internal)
struct DevScalars {     // per-problem scalars written by reductions
  double rr, pq, pr, zq, alpha, beta, ff, r0;
  double rr_in;   // mixed path: inner (FP32) residual norm^2 of the unit-scaled residual equation
  double s;       // mixed path: scale of the current outer residual (its 2-norm)
};

void set_error(const char* fmt, ...);
bool cuda_ok(cudaError_t e, const char* what);

// Counts kernels of this library enqueued on a stream (launch wrappers call
// it once per kernel); graph replays add their captured kernel count.
void count_launches(long long n);
long long launch_count();
inline cudaError_t launched() {
  count_launches(1);
  return cudaGetLastError();
}

// assemble.cu
struct AsmLaunch {
  int dim, N, s, kind;
  int prec64;            // 1: FP64 arithmetic, FP64 full store; 0: FP32, compressed records
  long long cell0, ncell;   // chunk cell range (whole layers)
  const EpsDev* eps_host;   // field (copied into kernel parameters)
  double hfac;
  const void* eps_c;     // cell-centre eps of all cells (double for prec64, float otherwise)
  void* out_full;        // prec64: SoA double [NP][ncell]
  uint8_t* out_rec;      // !prec64: scratch records [ncell][REC_MAX]
  uint8_t* out_cls;      // !prec64: padded class bytes of the chunk
  int nseg_x;
  double tau;
  // optional list of the chunk's cells to integrate (local indices, nlist of
  // them); the others are left alone (nullptr: every cell of the chunk)
  const int* list;
  long long nlist;
  // adaptive accuracy (Section "Adaptive stencil integration"): the chunk's
  // previously stored matrices, its per-cell final flags (set here when the
  // relative max-norm change falls below adapt_C) and the accuracy of each
  // stored matrix; final_flags == nullptr: not adaptive
  CmpChunk prev_cmp;
  const double* prev_full;
  uint8_t* final_flags;
  uint8_t* s_cell;
  double adapt_C;
  int adapt_keep;        // 1: a cell that passes the test keeps its previous matrix
  // exact surplus of the mixed paths (eps64 != nullptr): FP64 arithmetic with
  // eps64 as the reference, the lossy records against the FP32 eps_c, and
  // the FP64 surplus written to out_x64 at the cell's list position xpos;
  // prev_x64: the previous level's exact surplus for the adaptive test
  const double* eps64;
  double* out_x64;
  const int* xpos;
  const double* prev_x64;
};
// adaptive accuracy, before the integration of one chunk at a new level: the
// cells already final keep their previous matrix (copied into the new store:
// records + class bytes, or the FP64 entries), and the work list receives the
// candidate cells (the interface list, or every cell) that are not final.
// first = 1 on the first judged level: the cells final before any judgement
// (constant eps over the cell) take accuracy s there.
cudaError_t launch_adaptive_prepare(int dim, int N, int nseg_x, long long chunk_cells, int prec64,
                                    const uint8_t* final_flags, const CmpChunk& prev_cmp, const double* prev_full,
                                    uint8_t* out_rec, uint8_t* out_cls, double* out_full, const int* cand,
                                    long long ncand, int* work, int* nwork, uint8_t* s_cell, int s, int first,
                                    cudaStream_t st);
// marks every cell final except the listed candidate cells of each chunk
cudaError_t launch_adaptive_init(long long chunk_cells, int nchunk, const int* lists, const int* counts_host,
                                 uint8_t* final_flags, cudaStream_t st);
cudaError_t launch_eps_centre(int dim, int N, const EpsDev* eps, int prec64, void* eps_c, cudaStream_t st);
// stream-ordered allocation from the library's memory pool on the current
// device: freed blocks stay in the pool for the next problems (no release
// back to the driver), so creating and destroying problems does not pay for
// driver allocations each time
cudaError_t mg_malloc_async(void** p, size_t bytes, cudaStream_t st);
template <typename T>
inline cudaError_t mg_malloc_async(T** p, size_t bytes, cudaStream_t st) {
  return mg_malloc_async(reinterpret_cast<void**>(p), bytes, st);
}
// interface cells: cells that a discontinuity of eps (box face, disc boundary,
// planar jump) crosses; every other cell sees one eps value at all its sample
// points, so its element matrix is the geometric one at every accuracy s.
// Appends the local index of each such cell to lists[chunk * chunk_cells + ...]
// and counts them in counts[chunk].  Returns cudaErrorNotSupported for fields
// without a flat-cell notion (every cell must be integrated).
cudaError_t launch_interface_cells(int dim, int N, const EpsDev* eps, long long chunk_cells, int* lists,
                                   int* counts, cudaStream_t st);
cudaError_t launch_assemble(const AsmLaunch& a, cudaStream_t st);
cudaError_t launch_geometric_full(int dim, int N, double hfac, const double* eps_c, long long cell0,
                                  long long ncell, double* out, cudaStream_t st);
cudaError_t launch_pack_count(int dim, int N, long long nrows, int nseg_x, const uint8_t* cls,
                              uint32_t* seg_base, uint32_t* totals, cudaStream_t st);
cudaError_t launch_pack_copy(int dim, int N, long long nrows, int nseg_x, const uint8_t* cls,
                             const uint32_t* seg_base, const uint8_t* rec, uint8_t* p1, uint8_t* p2,
                             uint8_t* p3, cudaStream_t st);

// sweep.cu
// SW_JACOBI0: damped Jacobi from a zero iterate, y = omega D^-1 b (x is not
// read); launch_sweep returns cudaErrorNotSupported (launching nothing) on the
// paths without it, where the caller zeroes x and runs SW_JACOBI
// SW_RESID_RZ, SW_JACOBI_DOT: internal to launch_resid_restrict and
// launch_jacobi_dot
enum SweepMode { SW_JACOBI = 0, SW_RESID = 1, SW_MATVEC = 2, SW_JACOBI0 = 3, SW_RESID_RZ = 4, SW_JACOBI_DOT = 5 };
cudaError_t launch_sweep(const LevelOp& op, int mode, int vec64, const void* x, const void* b,
                         void* y, double omega, double* partials, int* nblocks, cudaStream_t st);
// b_c = R r_f; with diag (the coarse level's stencil diagonals), also
// u1 = omega b_c / diag, the coarse V-cycle's first smoothing step from zero
cudaError_t launch_restrict(int dim, int Nc, int vec64, const void* rf, void* bc, cudaStream_t st,
                            const void* diag = nullptr, double omega = 0.0, void* u1 = nullptr);
// Fused residual + restriction (Section "Stencil assembly variants": the
// residual sweep and R = P^T in one pass) on a split compressed finest level
// (3D, FP32): the bulk pass restricts its residuals along z into zr (the
// fine x-y grid at every coarse plane, (Nc + 1) (N + 1)^2 floats) leaving out
// the touched vertices, the fix-up pass writes their residuals into rt (a fine
// vector, other entries untouched), a third pass adds them to zr and an x-y
// pass forms bc.  cudaErrorNotSupported (nothing launched) on levels without
// that split or without zr.
cudaError_t launch_resid_restrict(const LevelOp& op, int vec64, const void* x, const void* b, void* rt, void* zr,
                                  void* bc, cudaStream_t st, const void* diag = nullptr, double omega = 0.0,
                                  void* u1 = nullptr);
// Damped Jacobi sweep y = x + omega D^-1 (b - A x) fused with the dot product
// y . dq (the flexible-CG coefficient of the preconditioned residual y) on a
// split compressed finest level (3D, FP32): partials receives one FP64 partial
// per block, *nblocks of them.  cudaErrorNotSupported (nothing launched)
// elsewhere.
cudaError_t launch_jacobi_dot(const LevelOp& op, const float* x, const float* b, float* y, float omega,
                              const float* dq, double* partials, int* nblocks, cudaStream_t st);
// words of the touched-vertex bit mask of a split level
size_t tmask_words(int N);
cudaError_t launch_prolong_add(int dim, int Nc, int vec64, const void* ec, void* ef, cudaStream_t st);
cudaError_t launch_inject(int dim, int Nc, int vec64, const void* rf, void* bc, cudaStream_t st);
cudaError_t launch_zero(void* p, size_t bytes, cudaStream_t st);
cudaError_t launch_build_stencil(const LevelOp& op, void* out, cudaStream_t st);
// the two coarsest levels of an FP32 V-cycle in one block (level N = 9 with
// full storage and stencils, then the coarsest level solved with the inverse
// at Lc + n^2); cudaErrorNotSupported (nothing launched) otherwise
bool vcycle_tail_supported(const LevelOp& op);
cudaError_t launch_vcycle_tail(const LevelOp& op, const double* Lc, const float* b, float* x, float omega,
                               int nu_pre, int nu_post, cudaStream_t st);
cudaError_t launch_pad_eps(int N, const float* eps_c, float* eps_pad, cudaStream_t st);
// from_xpos = 0: vertices next to a cell with a surplus record (and their
// stencil table); 1: vertices next to an interface cell (op.xpos >= 0)
// the vertex-form FP64 bulk weights of LevelOp::w64 / es64 (w: four arrays
// of (N+1)^3, es: N * N * (N+1)) from eps64 if non-null, else from eps_c
cudaError_t launch_geo_weights64(const LevelOp& op, double* const w[4], double* es, cudaStream_t st);
cudaError_t launch_build_touched(const LevelOp& op, uint8_t* flags, uint32_t* counts, int* list, int* ntouched,
                                 cudaStream_t st, int from_xpos = 0);
// xpos[chunk * chunk_cells + list[chunk][i]] = i for every interface cell, -1 elsewhere
// a = b - a over n entries (FP64 when vec64, else FP32)
cudaError_t launch_sub_from(long long n, int vec64, void* a, const void* b, cudaStream_t st);
cudaError_t launch_xpos(long long chunk_cells, int nchunk, const int* lists, const int* counts_host, int* xpos,
                        cudaStream_t st);

// vector ops for the outer loop (FP64 vectors; n = vertices)
cudaError_t launch_dot(const double* a, const double* b, long long n, double* partials, int* nblocks,
                       cudaStream_t st);
cudaError_t launch_dot_f32(const float* a, const double* b, long long n, double* partials, int* nblocks,
                           cudaStream_t st);
enum ScalarOp { SC_SET_BETA = 0, SC_SET_ALPHA = 1 };
// out[c] = sum over the nblocks partials of component c (ncomp interleaved
// components); with sc, then the scalar update op on sc (one launch)
cudaError_t launch_reduce_finish(const double* partials, int nblocks, int ncomp, double* out,
                                 cudaStream_t st, DevScalars* sc = nullptr, int op = -1);
cudaError_t launch_scalar_op(DevScalars* sc, int op, cudaStream_t st);
cudaError_t launch_fcg_direction(long long n, int first, int z64, const void* z, double* p,
                                 const DevScalars* sc, cudaStream_t st);
cudaError_t launch_fcg_update(long long n, double* u, double* r, const double* p, const double* q,
                              const DevScalars* sc, int r32_out, void* rin, double* partials,
                              int* nblocks, cudaStream_t st);
cudaError_t launch_richardson_update(long long n, double* u, int z64, const void* z, cudaStream_t st);
// FP32 inner solve of the mixed path
// p = z + beta p (first = 1: p = z); first = 0 also applies the deferred
// correction step e += alpha p of the previous iteration (alpha in sc)
cudaError_t launch_fcg32_direction(long long n, int first, const float* z, float* p, float* e, const DevScalars* sc,
                                   cudaStream_t st);
// r -= alpha q and partials of r.r (the matching e += alpha p is deferred);
// with w = omega D^-1 of the finest level, also u1 = w r (the next V-cycle's
// first smoothing step from the zero iterate)
cudaError_t launch_fcg32_update(long long n, float* r, const float* q, const DevScalars* sc, double* partials,
                                int* nblocks, cudaStream_t st, const float* w = nullptr, float* u1 = nullptr);
// p[0 .. n) = v
cudaError_t launch_fill(long long n, float v, float* p, cudaStream_t st);
// e += alpha p: applies the last deferred correction step
cudaError_t launch_fcg32_flush(long long n, float* e, const float* p, const DevScalars* sc, cudaStream_t st);
// r_in = r / ||r|| in FP32 (||r||^2 from sc->rr); with w, also u1 = w r_in
cudaError_t launch_scale_residual(long long n, const double* r, float* rin, DevScalars* sc, cudaStream_t st,
                                  const float* w = nullptr, float* u1 = nullptr);
cudaError_t launch_apply_correction(long long n, double* u, const float* e, const DevScalars* sc, cudaStream_t st);
cudaError_t launch_dot_f32f32(const float* a, const float* b, long long n, double* partials, int* nblocks,
                              cudaStream_t st);
cudaError_t launch_convert(long long n, int to64, const void* src, void* dst, cudaStream_t st);
cudaError_t launch_load_vector(int dim, int N, double val, double* f, cudaStream_t st);

// galerkin.cu
cudaError_t launch_galerkin(const LevelOp& fine, int out64, void* coarse_full, cudaStream_t st);
cudaError_t launch_galerkin_range(const LevelOp& fine, int out64, void* coarse_full, int last0, int last1,
                                  cudaStream_t st);
cudaError_t launch_coarse_factor(const LevelOp& coarsest, double* L, cudaStream_t st);
cudaError_t launch_coarse_solve(int dim, const double* L, int vec64, const void* b, void* e,
                                cudaStream_t st);
cudaError_t launch_decode_matrices(const LevelOp& op, const long long* cells, long long ncells, double* out,
                                   cudaStream_t st);

// galerkin.cu: lossy surplus storage of a coarse level's FP32 Galerkin store, in place
cudaError_t launch_compress_coarse(int dim, long long ncell, float* a, const float* eps_c, double hfac, double tau,
                                   uint8_t* cls_out, unsigned long long* counts, cudaStream_t st);

// paper_format.cu: the paper's truncated storage of a level's surplus
cudaError_t launch_paper_format(int dim, long long ncell, const double* A, const void* eps_c, int eps64,
                                double hfac, double delta, uint8_t* p3_out, double* At, unsigned long long* hist,
                                unsigned long long* maxerr_bits, cudaStream_t st);

}  // namespace mg
