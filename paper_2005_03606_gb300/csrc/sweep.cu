// Matrix-free operator application on one level: residual, damped Jacobi
// sweep and FP64 matvec (Section "Numerical computation of stencils in a task
// language": the element matrices of the 2^d cells around a vertex feed its
// residual, then the point smoother S = omega diag^-1(A) of Section
// "adaFAC-x" acts on it), the 3:1 d-linear transfers P and R = P^T, and the
// vector kernels of the outer FP64 loop.
//
// Element matrices have zero row sums, so the row of vertex v (local index a
// in cell c) contributes sum_{b != a} A_ab (u_b - u_a) and the diagonal is
// -sum_{b != a} A_ab.  On the compressed finest level A = eps_c K_ref h^(d-2)
// + decode(surplus), the geometric part from constants and the cell-centre
// eps, the surplus only for cells of storage class > 0.
#include "mg_internal.cuh"

#include <mutex>
#include <type_traits>

namespace mg {

namespace {

constexpr int kBX = 32, kBY = 8;

// Record of a cell of storage class cls > 0: the rank of the cell among the
// class-cls cells of its 32-cell segment (from the segment's class bytes)
// plus the segment's base offset.  seg = segment index within the chunk.
template <int D>
__device__ __forceinline__ const uint8_t* record_at(const CmpChunk& ck, int seg, int lane, int cls) {
  const unsigned r = rank_in_segment(ck.cls + (size_t)seg * kSegCells, lane, cls);
  const unsigned base = __ldg(ck.seg_base + (size_t)(cls - 1) * ck.nseg + seg);
  const int recb = cls == 1 ? Dim<D>::REC1 : (cls == 2 ? Dim<D>::REC2 : Dim<D>::REC3);
  return ck.pool[cls - 1] + (size_t)(base + r) * recb;
}

// (A u)_v and diag_v at interior vertex (i, j, k) from the 3^d neighbourhood u
// (vertex-per-thread form, used for 2D and for small 3D levels).  All index
// arithmetic is 32-bit and done per cell layer (the layer along the last axis
// fixes the chunk).
template <int D, typename TA, bool CMP, typename TS>
__device__ __forceinline__ void vertex_apply(const LevelOp& op, int i, int j, int k, const TA* u,
                                             TA* Au, TA* dg) {
  constexpr int NV = Dim<D>::NV;
  const int N = op.N;
  TA acc = 0, dgs = 0;
#pragma unroll
  for (int ol = 0; ol < 2; ++ol) {
    const int cl = (D == 3 ? k : j) - 1 + ol;
    int ch = cl / op.layers;
    ch = ch < op.nchunk ? ch : op.nchunk - 1;
    const int ll = cl - ch * op.layers;  // layer within the chunk
#pragma unroll
    for (int om = 0; om < (D == 3 ? 2 : 1); ++om) {
      const int cy = D == 3 ? j - 1 + om : cl;
      const int row = D == 3 ? ll * N + cy : ll;              // x-row within the chunk
      const int cbase = D == 3 ? (cl * N + cy) * N : cl * N;  // global cell index of x = 0
      const int segrow = row * op.nseg_x;
#pragma unroll
      for (int ox = 0; ox < 2; ++ox) {
        const int cx = i - 1 + ox;
        const int oy = D == 3 ? om : ol, oz = D == 3 ? ol : 0;
        const int a = (1 - ox) | ((1 - oy) << 1) | (D == 3 ? (1 - oz) << 2 : 0);
        const TA u_a = u[D == 3 ? 13 : 4];
        if (CMP && sizeof(TA) == 8 && op.eps64) {
          // exact FP64 operator: FP64 eps_c K_ref h^(d-2) + the exact surplus of interface cells
          const TA ge = (TA)__ldg(op.eps64 + cbase + cx) * (TA)op.hfac;
#pragma unroll
          for (int b = 0; b < NV; ++b) {
            if (b == a) continue;
            const double kv = kref_off<D>(popc_small(a ^ b));
            if (kv == 0.0) continue;
            const int ub = (ox + (b & 1)) + 3 * (oy + ((b >> 1) & 1)) + (D == 3 ? 9 * (oz + ((b >> 2) & 1)) : 0);
            acc += ge * (TA)kv * (u[ub] - u_a);
          }
          dgs += ge * (TA)kref_diag<D>();
          const int ps = __ldg(op.xpos + cbase + cx);
          const double* xs = op.cmp[ch].x64;
          if (ps >= 0 && xs) {
            const double* xr = xs + (size_t)ps * Dim<D>::NP;
#pragma unroll
            for (int b = 0; b < NV; ++b) {
              if (b == a) continue;
              const TA dv = (TA)__ldg(xr + pair_of(NV, a, b));
              const int ub = (ox + (b & 1)) + 3 * (oy + ((b >> 1) & 1)) + (D == 3 ? 9 * (oz + ((b >> 2) & 1)) : 0);
              acc += dv * (u[ub] - u_a);
              dgs -= dv;
            }
          }
        } else if (CMP) {
          const TA ge = (TA)__ldg(op.eps_c + cbase + cx) * (TA)(sizeof(TA) == 4 ? (double)(float)op.hfac : op.hfac);
#pragma unroll
          for (int b = 0; b < NV; ++b) {
            if (b == a) continue;
            const double kv = kref_off<D>(popc_small(a ^ b));
            if (kv == 0.0) continue;
            const int ub = (ox + (b & 1)) + 3 * (oy + ((b >> 1) & 1)) + (D == 3 ? 9 * (oz + ((b >> 2) & 1)) : 0);
            acc += ge * (TA)kv * (u[ub] - u_a);
          }
          dgs += ge * (TA)kref_diag<D>();
          const CmpChunk& ck = op.cmp[ch];
          const int seg = segrow + (cx >> 5);
          const int cls = __ldg(ck.cls + (size_t)seg * kSegCells + (cx & 31));
          if (cls) {
            const uint8_t* rec = record_at<D>(ck, seg, cx & 31, cls);
#pragma unroll
            for (int b = 0; b < NV; ++b) {
              if (b == a) continue;
              const TA dv = (TA)decode_entry<D>(rec, cls, pair_of(NV, a, b));
              const int ub = (ox + (b & 1)) + 3 * (oy + ((b >> 1) & 1)) + (D == 3 ? 9 * (oz + ((b >> 2) & 1)) : 0);
              acc += dv * (u[ub] - u_a);
              dgs -= dv;
            }
          }
        } else {
          const TS* A = reinterpret_cast<const TS*>(op.full[ch].a);
          const size_t cc = (size_t)op.chunk_cells;
          const int lc = row * N + cx;
          TA t = 0, rs = 0;
#pragma unroll
          for (int b = 0; b < NV; ++b) {
            if (b == a) continue;
            const TA av = (TA)__ldg(A + (size_t)pair_of(NV, a, b) * cc + lc);
            const int ub = (ox + (b & 1)) + 3 * (oy + ((b >> 1) & 1)) + (D == 3 ? 9 * (oz + ((b >> 2) & 1)) : 0);
            t += av * u[ub];
            rs += av;
          }
          acc += t - rs * u_a;
          dgs -= rs;
        }
      }
    }
  }
  *Au = acc;
  *dg = dgs;
}

// The 27-point stencil of interior vertex (i, j, k) of a compressed 3D level
// in FP32: c[ub] for the 26 neighbours ub = dx + 3 dy + 9 dz (the sum over the
// cells that hold both vertices of eps_c K_ref h plus the decoded surplus) and
// the diagonal in c[13].  Same terms as vertex_apply, gathered by neighbour.
__device__ __forceinline__ void vertex_coeffs3(const LevelOp& op, int i, int j, int k, float (&c)[27]) {
  constexpr int NV = 8;
  const int N = op.N;
#pragma unroll
  for (int q = 0; q < 27; ++q) c[q] = 0.f;
  float dgs = 0.f;
  const float hf = (float)op.hfac;
#pragma unroll
  for (int oz = 0; oz < 2; ++oz) {
    const int cl = k - 1 + oz;
    if (cl < 0 || cl >= N) continue;   // cells outside the grid (boundary vertices)
    int ch = cl / op.layers;
    ch = ch < op.nchunk ? ch : op.nchunk - 1;
    const int ll = cl - ch * op.layers;
#pragma unroll
    for (int oy = 0; oy < 2; ++oy) {
      const int cy = j - 1 + oy;
      if (cy < 0 || cy >= N) continue;
      const int row = ll * N + cy;
      const int cbase = (cl * N + cy) * N;
      const int segrow = row * op.nseg_x;
#pragma unroll
      for (int ox = 0; ox < 2; ++ox) {
        const int cx = i - 1 + ox;
        if (cx < 0 || cx >= N) continue;
        const int a = (1 - ox) | ((1 - oy) << 1) | ((1 - oz) << 2);
        const float ge = __ldg(op.eps_c + cbase + cx) * hf;
#pragma unroll
        for (int b = 0; b < NV; ++b) {
          if (b == a) continue;
          const double kv = kref_off<3>(popc_small(a ^ b));
          if (kv == 0.0) continue;
          const int ub = (ox + (b & 1)) + 3 * (oy + ((b >> 1) & 1)) + 9 * (oz + ((b >> 2) & 1));
          c[ub] += ge * (float)kv;
        }
        dgs += ge * (float)kref_diag<3>();
        const CmpChunk& ck = op.cmp[ch];
        const int seg = segrow + (cx >> 5);
        const int cls = __ldg(ck.cls + (size_t)seg * kSegCells + (cx & 31));
        if (cls) {
          const uint8_t* rec = record_at<3>(ck, seg, cx & 31, cls);
#pragma unroll
          for (int b = 0; b < NV; ++b) {
            if (b == a) continue;
            const float dv = decode_entry<3>(rec, cls, pair_of(NV, a, b));
            const int ub = (ox + (b & 1)) + 3 * (oy + ((b >> 1) & 1)) + 9 * (oz + ((b >> 2) & 1));
            c[ub] += dv;
            dgs -= dv;
          }
        }
      }
    }
  }
  c[13] = dgs;
}

template <typename T>
__device__ __forceinline__ T block_sum(T v, T* sh) {
  for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int nw = (blockDim.x * blockDim.y) >> 5;
  __syncthreads();
  if ((tid & 31) == 0) sh[tid >> 5] = v;
  __syncthreads();
  T r = 0;
  if (tid == 0)
    for (int w = 0; w < nw; ++w) r += sh[w];
  return r;
}

// One sweep over the interior vertices of one level, one vertex per thread.
//  SW_JACOBI: y = x + omega (b - A x) / diag
//  SW_RESID : y = b - A x
//  SW_MATVEC: y = A x; partials += (x.y, x.b) per block
template <int D, typename TV, typename TA, typename TS, int MODE, bool CMP>
__global__ void __launch_bounds__(kBX * kBY) sweep_kernel(const LevelOp op, const TV* __restrict__ x,
                                                          const TV* __restrict__ b, TV* __restrict__ y,
                                                          TA omega, double* __restrict__ partials) {
  __shared__ double sh[2][kBX * kBY / 32];
  const int N = op.N, n1 = N + 1;
  const int i = 1 + blockIdx.x * kBX + threadIdx.x;
  const int j = 1 + blockIdx.y * kBY + threadIdx.y;
  const int k = D == 3 ? 1 + blockIdx.z : 0;
  const bool valid = i < N && j < N;
  double d1 = 0.0, d2 = 0.0;
  if (valid) {
    TA u[D == 3 ? 27 : 9];
    const int v = D == 2 ? j * n1 + i : (k * n1 + j) * n1 + i;
    const int plane = n1 * n1;
#pragma unroll
    for (int dz = 0; dz < (D == 3 ? 3 : 1); ++dz)
#pragma unroll
      for (int dy = 0; dy < 3; ++dy) {
        const TV* xr = x + (v + (dy - 1) * n1 + (D == 3 ? (dz - 1) * plane : 0));
#pragma unroll
        for (int dx = 0; dx < 3; ++dx) u[dx + 3 * dy + 9 * dz] = MODE == SW_JACOBI0 ? (TA)0 : (TA)__ldg(xr + (dx - 1));
      }
    TA Au, dg;
    vertex_apply<D, TA, CMP, TS>(op, i, j, k, u, &Au, &dg);
    const TA uv = u[D == 3 ? 13 : 4];
    if (MODE == SW_JACOBI0) {
      y[v] = (TV)(omega * (TA)b[v] / dg);
    } else if (MODE == SW_JACOBI) {
      y[v] = (TV)(uv + omega * ((TA)b[v] - Au) / dg);
    } else if (MODE == SW_RESID) {
      y[v] = (TV)((TA)b[v] - Au);
    } else {
      y[v] = (TV)Au;
      d1 = (double)uv * (double)Au;
      d2 = (double)uv * (double)b[v];
    }
  }
  if (MODE == SW_MATVEC) {
    const double s1 = block_sum(d1, sh[0]);
    const double s2 = block_sum(d2, sh[1]);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      const long long blk = blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
      partials[2 * blk] = s1;
      partials[2 * blk + 1] = s2;
    }
  }
}

// ---------------------------------------------------------------- assembled vertex stencils
// Levels stored as full cell matrices (Galerkin coarse levels; the finest
// level of the FP64 paths) also keep the assembled 3^d-point stencil of every
// vertex, gathered once per rebuild of the cell matrices.  A sweep then costs
// 3^d coefficient loads and multiply-adds per vertex instead of decoding the
// 2^d cells around it.
template <int D, typename TS>
__global__ void build_stencil_kernel(const LevelOp op, TS* __restrict__ out) {
  constexpr int NV = Dim<D>::NV, NS = D == 3 ? 27 : 9, C = D == 3 ? 13 : 4;
  const int N = op.N, n1 = N + 1;
  const long long nv = D == 3 ? (long long)n1 * n1 * n1 : (long long)n1 * n1;
  // every vertex, boundary ones included: the backward couplings of an
  // interior vertex to the boundary are read from the boundary vertex's entries
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nv;
       v += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(v % n1);
    const int j = (int)((v / n1) % n1);
    const int k = D == 3 ? (int)(v / ((long long)n1 * n1)) : 0;
    TS c[NS];
#pragma unroll
    for (int q = 0; q < NS; ++q) c[q] = 0;
    TS dg = 0;
#pragma unroll
    for (int ol = 0; ol < 2; ++ol) {
      const int cl = (D == 3 ? k : j) - 1 + ol;
      if (cl < 0 || cl >= N) continue;   // cells outside the grid
      int ch = cl / op.layers;
      ch = ch < op.nchunk ? ch : op.nchunk - 1;
      const int ll = cl - ch * op.layers;
      const TS* A = reinterpret_cast<const TS*>(op.full[ch].a);
      const size_t cc = (size_t)op.chunk_cells;
#pragma unroll
      for (int om = 0; om < (D == 3 ? 2 : 1); ++om) {
        const int cy = D == 3 ? j - 1 + om : cl;
        if (cy < 0 || cy >= N) continue;
        const int row = D == 3 ? ll * N + cy : ll;
#pragma unroll
        for (int ox = 0; ox < 2; ++ox) {
          const int cx = i - 1 + ox;
          if (cx < 0 || cx >= N) continue;
          const int oy = D == 3 ? om : ol, oz = D == 3 ? ol : 0;
          const int a = (1 - ox) | ((1 - oy) << 1) | (D == 3 ? (1 - oz) << 2 : 0);
          const int lc = row * N + cx;
#pragma unroll
          for (int bb = 0; bb < NV; ++bb) {
            if (bb == a) continue;
            const TS av = __ldg(A + (size_t)pair_of(NV, a, bb) * cc + lc);
            const int ub = (ox + (bb & 1)) + 3 * (oy + ((bb >> 1) & 1)) + (D == 3 ? 9 * (oz + ((bb >> 2) & 1)) : 0);
            c[ub] += av;
            dg -= av;
          }
        }
      }
    }
    c[C] = dg;
    // symmetric storage: the diagonal and the couplings to the forward half of
    // the neighbourhood (q > C); the others are the neighbours' own entries
#pragma unroll
    for (int q = C; q < NS; ++q) out[(size_t)(q - C) * nv + v] = c[q];
  }
}

// NT > 0: the grid size as a compile-time constant (strides fold into address
// arithmetic of constants); NT = 0: from the LevelOp
template <int D, typename TV, typename TA, typename TS, int MODE, int NT = 0>
__global__ void __launch_bounds__(kBX * kBY) stencil_sweep_kernel(const LevelOp op, const TV* __restrict__ x,
                                                                  const TV* __restrict__ b, TV* __restrict__ y,
                                                                  TA omega, double* __restrict__ partials) {
  pdl_begin();
  constexpr int C = D == 3 ? 13 : 4;   // centre of the 3^d stencil
  __shared__ double sh[2][kBX * kBY / 32];
  const int N = NT ? NT : op.N, n1 = N + 1;
  const int i = 1 + blockIdx.x * kBX + threadIdx.x;
  const int j = 1 + blockIdx.y * kBY + threadIdx.y;
  const int k = D == 3 ? 1 + blockIdx.z : 0;
  const bool valid = i < N && j < N;
  const size_t nv = D == 3 ? (size_t)n1 * n1 * n1 : (size_t)n1 * n1;
  double d1 = 0.0, d2 = 0.0;
  if (valid) {
    const int v = D == 2 ? j * n1 + i : (k * n1 + j) * n1 + i;
    const int plane = n1 * n1;
    const TS* S0 = reinterpret_cast<const TS*>(op.stencil);
    const TS* S = S0 + v;
    const TA dg = (TA)__ldg(S);
    if (MODE == SW_JACOBI0) {
      y[v] = (TV)(omega * (TA)b[v] / dg);
      return;
    }
    const TA uv = (TA)__ldg(x + v);
    // FP32: difference form sum_q c_q (u_q - u_v) (exact for constants); FP64:
    // plain sum_q c_q u_q, half the FP64 operations, rounding far below need
    constexpr bool kDiff = sizeof(TA) == 4;
    TA acc = kDiff ? (TA)0 : dg * uv;
#pragma unroll
    for (int dz = 0; dz < (D == 3 ? 3 : 1); ++dz)
#pragma unroll
      for (int dy = 0; dy < 3; ++dy)
#pragma unroll
        for (int dx = 0; dx < 3; ++dx) {
          const int q = dx + 3 * dy + 9 * dz;
          if (q == C) continue;
          const int nb = v + (dx - 1) + (dy - 1) * n1 + (D == 3 ? (dz - 1) * plane : 0);
          const TA uq = (TA)__ldg(x + nb);
          // forward couplings are stored at v, backward ones at the neighbour (symmetry)
          const TA cq = q > C ? (TA)__ldg(S + (size_t)(q - C) * nv) : (TA)__ldg(S0 + (size_t)(C - q) * nv + nb);
          acc += cq * (kDiff ? uq - uv : uq);
        }
    const TA Au = acc;
    if (MODE == SW_JACOBI) {
      y[v] = (TV)(uv + omega * ((TA)b[v] - Au) / dg);
    } else if (MODE == SW_RESID) {
      y[v] = (TV)((TA)b[v] - Au);
    } else {
      y[v] = (TV)Au;
      d1 = (double)uv * (double)Au;
      d2 = (double)uv * (double)b[v];
    }
  }
  if (MODE == SW_MATVEC) {
    const double s1 = block_sum(d1, sh[0]);
    const double s2 = block_sum(d2, sh[1]);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      const long long blk = blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
      partials[2 * blk] = s1;
      partials[2 * blk + 1] = s2;
    }
  }
}

// ---------------------------------------------------------------- 3D streaming tile sweep
// A CTA owns a 32 x 8 column of vertices and walks kZC vertex planes along z,
// one vertex per thread and plane.  u planes (34 x 10 with halo), b planes,
// cell layers (33 x 9 cell-centre eps) and the layers' storage-class bytes
// stream into shared-memory rings through asynchronous copies (cp.async)
// issued kPF planes ahead, so a CTA keeps about kPF planes of traffic in
// flight; one barrier per plane.  Cells with a surplus record (class > 0)
// are resolved per vertex: the rank inside the cell's 32-cell segment comes
// from the class bytes already in shared memory, the record from global
// memory (L1/L2 serve the 8 vertices of the cell).
__device__ __forceinline__ void cp_async4(void* s, const void* g) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(s);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async8(void* s, const void* g) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(s);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async16(void* s, const void* g) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(s);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <typename T>
__device__ __forceinline__ void cp_async_elem(T* s, const T* g) {
  if (sizeof(T) == 4) cp_async4(s, g);
  else cp_async8(s, g);
}

constexpr int kTX = 32, kTY = 8, kZC = 32;
constexpr int kUW = kTX + 2, kUH = kTY + 2;   // u tile with halo
constexpr int kCW = kTX + 1, kCH = kTY + 1;   // cell tile
constexpr int kCells = kCW * kCH;
constexpr int kPF = 4;                        // planes fetched ahead
// Ring depths.  At step k (vertex plane k) the copies for plane k+kPF, b plane
// k+kPF and cell layer k+kPF-1 are issued, and planes k-1..k+1, b plane k,
// layers k-1..k are read.  A slot filled at step k must not be read at step
// k-1 (no barrier between the two): rings of kPF+3 planes / kPF+2 layers
// (and kPF+2 b planes) guarantee that.
constexpr int kPS = kPF + 3, kLS = kPF + 2, kBS = kPF + 2;

// rank of byte `lane` among the bytes equal to k in a 16-byte-aligned row of 32 bytes (shared memory)
__device__ __forceinline__ int rank_in_row(const uint8_t* row, int lane, int k) {
  const unsigned kk = 0x01010101u * (unsigned)k;
  const unsigned* w = reinterpret_cast<const unsigned*>(row);
  int cnt = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int lo = 4 * q;
    if (lo >= lane) break;
    unsigned eq = __vcmpeq4(w[q], kk);
    const int nb = lane - lo;   // bytes of this word before `lane`
    if (nb < 4) eq &= 0xffffffffu >> (8 * (4 - nb));
    cnt += __popc(eq);
  }
  return cnt >> 3;
}

template <typename TA>
__device__ __forceinline__ TA jacobi_div(TA num, TA den) {
  return num / den;
}
template <>
__device__ __forceinline__ float jacobi_div<float>(float num, float den) {
  return __fdividef(num, den);   // smoother arithmetic of the FP32 V-cycle
}

__device__ __forceinline__ int ring_next(int s, int n) { return s + 1 == n ? 0 : s + 1; }
__device__ __forceinline__ int ring_add(int s, int d, int n) { return s + d >= n ? s + d - n : s + d; }

template <typename TV, typename TA, typename TS, int MODE, bool CMP>
__global__ void __launch_bounds__(kTX * kTY, 3) sweep3_stream(const LevelOp op, const TV* __restrict__ x,
                                                              const TV* __restrict__ b, TV* __restrict__ y,
                                                              TA omega, double* __restrict__ partials) {
  constexpr int NV = 8;
  constexpr int NT = kTX * kTY;
  __shared__ TV su[kPS][kUH * kUW];
  __shared__ TV sb[kBS][NT];
  __shared__ float sge[CMP ? kLS : 1][kCells];
  __shared__ __align__(16) uint8_t scls[CMP ? kLS : 1][kCH][48];
  __shared__ int s_ch[CMP ? kLS : 1];
  __shared__ double sh[2][NT / 32];
  const int N = op.N, n1 = N + 1;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kTX + tx;
  const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY;
  const int i = x0 + tx + 1, j = y0 + ty + 1;
  const bool col_ok = i < N && j < N;
  const int k0 = 1 + blockIdx.z * kZC;
  const int k1 = min(N - 1, k0 + kZC - 1);
  const size_t plane = (size_t)n1 * n1;
  double d1 = 0.0, d2 = 0.0;

  // per-thread copy descriptors (the tile geometry is the same for every plane)
  const int u_g0 = [&] {
    const int dy = tid / kUW, dx = tid - dy * kUW;
    return (x0 + dx <= N && y0 + dy <= N) ? (y0 + dy) * n1 + x0 + dx : -1;
  }();
  const int t1 = tid + NT;   // second u element of this thread (84 of them exist)
  const int u_g1 = [&] {
    if (t1 >= kUH * kUW) return -2;
    const int dy = t1 / kUW, dx = t1 - dy * kUW;
    return (x0 + dx <= N && y0 + dy <= N) ? (y0 + dy) * n1 + x0 + dx : -1;
  }();
  const int b_g = col_ok ? j * n1 + i : -1;
  const int c_g0 = [&] {
    const int dy = tid / kCW, dx = tid - dy * kCW;
    return (x0 + dx < N && y0 + dy < N) ? (y0 + dy) * N + x0 + dx : -1;
  }();
  const int c_g1 = [&] {
    if (t1 >= kCells) return -2;
    const int dy = t1 / kCW, dx = t1 - dy * kCW;
    return (x0 + dx < N && y0 + dy < N) ? (y0 + dy) * N + x0 + dx : -1;
  }();
  // class bytes: thread tid < 27 copies 16 bytes of row tid/3 (segment x0/32
  // of the row, then the first 16 bytes of the next segment)
  int cl_off = -1;
  if (CMP && tid < kCH * 3) {
    const int dy = tid / 3, part = tid - dy * 3;
    const int cy = y0 + dy, sx = (x0 >> 5) + (part == 2 ? 1 : 0);
    if (cy < N && sx < op.nseg_x) cl_off = (cy * op.nseg_x + sx) * kSegCells + (part == 1 ? 16 : 0);
  }

  auto fetch_plane = [&](int p, int s) {
    TV* dst = su[s];
    const TV* src = x + (size_t)p * plane;
    if (u_g0 >= 0) cp_async_elem<TV>(dst + tid, src + u_g0);
    else dst[tid] = TV(0);
    if (u_g1 >= 0) cp_async_elem<TV>(dst + t1, src + u_g1);
    else if (u_g1 == -1) dst[t1] = TV(0);
  };
  auto fetch_b = [&](int p, int s) {
    if (b_g >= 0) cp_async_elem<TV>(&sb[s][tid], b + (size_t)p * plane + b_g);
  };
  // cell layer l (eps_c and class bytes) into slot s
  auto fetch_layer = [&](int l, int s) {
    if (!CMP) return;
    const float* src = op.eps_c + (size_t)l * N * N;
    if (c_g0 >= 0) cp_async4(&sge[s][tid], src + c_g0);
    else sge[s][tid] = 0.f;
    if (c_g1 >= 0) cp_async4(&sge[s][t1], src + c_g1);
    else if (c_g1 == -1) sge[s][t1] = 0.f;
    if (tid < kCH * 3) {
      int ch = l / op.layers;
      ch = ch < op.nchunk ? ch : op.nchunk - 1;
      uint8_t* dst = &scls[s][tid / 3][16 * (tid % 3)];
      if (cl_off >= 0)
        cp_async16(dst, op.cmp[ch].cls + (size_t)(l - ch * op.layers) * N * op.nseg_x * kSegCells + cl_off);
      else
        *reinterpret_cast<uint4*>(dst) = make_uint4(0u, 0u, 0u, 0u);
      if (tid == 0) s_ch[s] = ch;
    }
  };

  const TA gscale = (TA)(sizeof(TA) == 4 ? (double)op.gk32 : op.gk64);
  // prologue: planes k0-1 .. k0+kPF-1, b planes and layers k0-1 .. k0+kPF-2
  int sp = 0, sbq = 0, sl = 0;   // next slot to fill in each ring
  if (k0 <= k1) {
    for (int p = k0 - 1; p <= k0 + kPF - 1; ++p) {
      if (p <= N) fetch_plane(p, sp);
      if (p >= k0 && p <= k1) fetch_b(p, sbq);
      if (p - 1 >= k0 - 1 && p - 1 <= N - 1) fetch_layer(p - 1, sl);
      cp_async_commit();
      sp = ring_next(sp, kPS);
      if (p >= k0) sbq = ring_next(sbq, kBS);
      if (p - 1 >= k0 - 1) sl = ring_next(sl, kLS);
    }
  }
  // slots read at step k: planes k-1, k, k+1 start at ring slot 0; layers k-1, k at 0; b plane k at 0
  int rp = 0, rl = 0, rb = 0;
  for (int k = k0; k <= k1; ++k) {
    // issue step k + kPF: plane k+kPF, b plane k+kPF, layer k+kPF-1
    {
      const int p = k + kPF;
      if (p <= N) fetch_plane(p, sp);
      if (p <= k1) fetch_b(p, sbq);
      if (p - 1 <= N - 1) fetch_layer(p - 1, sl);
      cp_async_commit();
      sp = ring_next(sp, kPS);
      sbq = ring_next(sbq, kBS);
      sl = ring_next(sl, kLS);
    }
    cp_async_wait<kPF - 1>();   // groups up to plane k+1 / layer k / b plane k have landed
    __syncthreads();
    if (col_ok) {
      const TV* um = su[rp];
      const TV* uc = su[ring_add(rp, 1, kPS)];
      const TV* up = su[ring_add(rp, 2, kPS)];
      const int base = ty * kUW + tx;
      auto U = [&](int pz, int idx) -> TA {
        const int off = base + (idx / 3) * kUW + (idx % 3);
        return (TA)(pz == 0 ? um[off] : (pz == 1 ? uc[off] : up[off]));
      };
      const TA u_a = U(1, 4);
      TA acc = 0, dgs = 0;
      const int lm = rl, lc = ring_next(rl, kLS);
      if (CMP) {
        // geometric part: every nonzero off-diagonal of the 3D K_ref is -1/12, so
        // cell c adds (-eps_c h / 12) (sum of its 4 face/body-diagonal
        // neighbours of v - 4 u_v)
        TA ag = 0, gs = 0;
#pragma unroll
        for (int o = 0; o < NV; ++o) {
          const int ox = o & 1, oy = (o >> 1) & 1, oz = o >> 2;
          const int a = (1 - ox) | ((1 - oy) << 1) | ((1 - oz) << 2);
          const TA gv = (TA)sge[oz ? lc : lm][(ty + oy) * kCW + tx + ox];
          TA s4 = 0;
#pragma unroll
          for (int bb = 0; bb < NV; ++bb)
            if (bb != a && popc_small(a ^ bb) >= 2)
              s4 += U(oz + ((bb >> 2) & 1), (ox + (bb & 1)) + 3 * (oy + ((bb >> 1) & 1)));
          ag += gv * (s4 - (TA)4 * u_a);
          gs += gv;
        }
        acc = ag * gscale;
        dgs = (TA)-4 * gscale * gs;
        // surplus of cells with a record
        unsigned any = 0;
#pragma unroll
        for (int o = 0; o < NV; ++o) {
          const int ox = o & 1, oy = (o >> 1) & 1, oz = o >> 2;
          any |= scls[oz ? lc : lm][ty + oy][tx + ox];
        }
        if (any) {
#pragma unroll 1
          for (int o = 0; o < NV; ++o) {
            const int ox = o & 1, oy = (o >> 1) & 1, oz = o >> 2;
            const int ls = oz ? lc : lm;
            const int cls = scls[ls][ty + oy][tx + ox];
            if (!cls) continue;
            const int a = (1 - ox) | ((1 - oy) << 1) | ((1 - oz) << 2);
            const int l = k - 1 + oz;
            const int ch = s_ch[ls];
            const CmpChunk& ck = op.cmp[ch];
            const int cx = i - 1 + ox, cy = j - 1 + oy;
            const int seg = ((l - ch * op.layers) * N + cy) * op.nseg_x + (cx >> 5);
            const int dx = tx + ox;
            const int r = dx < kTX ? rank_in_row(&scls[ls][ty + oy][0], dx, cls) : 0;
            const unsigned base_r = __ldg(ck.seg_base + (size_t)(cls - 1) * ck.nseg + seg);
            const int recb = cls == 1 ? Dim<3>::REC1 : (cls == 2 ? Dim<3>::REC2 : Dim<3>::REC3);
            const uint8_t* rec = ck.pool[cls - 1] + (size_t)(base_r + r) * recb;
#pragma unroll
            for (int bb = 0; bb < NV; ++bb) {
              if (bb == a) continue;
              const TA dv = (TA)decode_entry<3>(rec, cls, pair_of(NV, a, bb));
              const int pz = oz + ((bb >> 2) & 1);
              const int idx = (ox + (bb & 1)) + 3 * (oy + ((bb >> 1) & 1));
              acc += dv * (U(pz, idx) - u_a);
              dgs -= dv;
            }
          }
        }
      } else {
#pragma unroll
        for (int o = 0; o < NV; ++o) {
          const int ox = o & 1, oy = (o >> 1) & 1, oz = o >> 2;
          const int a = (1 - ox) | ((1 - oy) << 1) | ((1 - oz) << 2);
          const int l = k - 1 + oz;
          int ch = l / op.layers;
          ch = ch < op.nchunk ? ch : op.nchunk - 1;
          const TS* A = reinterpret_cast<const TS*>(op.full[ch].a);
          const int lcell = ((l - ch * op.layers) * N + (j - 1 + oy)) * N + (i - 1 + ox);
          const size_t ccs = (size_t)op.chunk_cells;
          // row a: sum_b A_ab u_b - (sum_b A_ab) u_a, the row sum is minus the diagonal
          TA t = 0, rs = 0;
#pragma unroll
          for (int bb = 0; bb < NV; ++bb) {
            if (bb == a) continue;
            const TA av = (TA)__ldg(A + (size_t)pair_of(NV, a, bb) * ccs + lcell);
            t += av * U(oz + ((bb >> 2) & 1), (ox + (bb & 1)) + 3 * (oy + ((bb >> 1) & 1)));
            rs += av;
          }
          acc += t - rs * u_a;
          dgs -= rs;
        }
      }
      const size_t v = (size_t)k * plane + (size_t)j * n1 + i;
      const TA bv = (TA)sb[rb][tid];
      if (MODE == SW_JACOBI) {
        y[v] = (TV)(u_a + omega * jacobi_div<TA>(bv - acc, dgs));
      } else if (MODE == SW_RESID) {
        y[v] = (TV)(bv - acc);
      } else {
        y[v] = (TV)acc;
        d1 += (double)u_a * (double)acc;
        d2 += (double)u_a * (double)bv;
      }
    }
    rp = ring_next(rp, kPS);
    rl = ring_next(rl, kLS);
    rb = ring_next(rb, kBS);
  }
  if (MODE == SW_MATVEC) {
    const double s1 = block_sum(d1, sh[0]);
    const double s2 = block_sum(d2, sh[1]);
    if (tid == 0) {
      const long long blk = blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
      partials[2 * blk] = s1;
      partials[2 * blk + 1] = s2;
    }
  }
}

// ---------------------------------------------------------------- 3D FP32 geometric bulk sweep
// The finest compressed level in FP32 splits each sweep in two kernels:
//  (1) a class-blind bulk pass that applies only the geometric part
//      eps_c K_ref h to every interior vertex, and
//  (2) a fix-up pass over the list of vertices touched by a cell with a
//      surplus record, which recomputes those vertices with every term.
//
// Bulk pass arithmetic.  The trilinear reference matrix satisfies
// 12 K_ref = 5 I + E - J (E: adjacency along cell edges, J: all ones), so
//   (A u)_v = h/12 [ 5 u_v G_v + sum_{6 axis neighbours w} W_vw u_w - sum_c eps_c T_c ]
// with G_v the sum of eps over the 8 cells at v, W_vw the sum of eps over the
// 4 cells that share the edge vw, and T_c the sum of u over the 8 vertices of
// cell c.  Cell sums are built separably (pairs along x, then y, then z) and
// shared by the 4 vertices of a thread and by consecutive planes of its z
// march, so a vertex costs about a third of the per-cell form's arithmetic.
//
// Layout: a thread owns 4 consecutive vertices in x (rows of (N+1) floats with
// (N+1) % 4 == 0 keep float4 loads aligned) of row j and marches in z,
// loading the next plane's three u rows, eps rows and b one plane ahead and
// prefetching the rows kGeoPF planes further into L2.  Blocks (persistent
// grid, no wave tail) take equal shares of the z runs of all columns.
constexpr int kGeoBX = 32, kGeoBY = 8;
#ifndef MG_GEO_PF
#define MG_GEO_PF 2
#endif
constexpr int kGeoPF = MG_GEO_PF;   // planes of L2 prefetch ahead of the z march

// Balanced static partition of a bulk pass: the (x-tile, y-tile) columns of
// interior planes 1 .. N-1 are laid end to end (plane fastest) and block b
// takes the b-th of gridDim.x equal contiguous shares -- one z run, or the
// end of one column and the start of the next.  Every block then does the
// same number of plane steps (a tile grid of fixed z runs left whole runs
// for a fraction of the blocks: up to 1.3x the average at 243^3).
struct GeoRun {
  int tx, ty, k0, k1;
};

__device__ __forceinline__ bool next_geo_run(long long& w, long long w1, int nk, int ntx, GeoRun& r) {
  if (w >= w1) return false;
  const long long col = w / nk;
  const long long wend = min(w1, (col + 1) * (long long)nk);
  r.tx = (int)(col % ntx);
  r.ty = (int)(col / ntx);
  r.k0 = 1 + (int)(w - col * nk);
  r.k1 = r.k0 + (int)(wend - w) - 1;
  w = wend;
  return true;
}

// nk: work items per column (interior planes, or coarse planes for the fused
// residual + restriction)
__device__ __forceinline__ void geo_share(int ntx, int nty, int nk, long long& w0, long long& w1) {
  const long long total = (long long)ntx * nty * nk;
  const long long per = (total + gridDim.x - 1) / gridDim.x;
  w0 = min(total, (long long)blockIdx.x * per);
  w1 = min(total, w0 + per);
}

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialization may start while its predecessor in the stream still runs;
// griddepcontrol.wait blocks the calling thread until the predecessor grid
// has completed and its memory operations are visible.
#ifndef MG_FIX_PDL
#define MG_FIX_PDL 1
#endif

// L2 prefetch of one address (no register, no scoreboard wait)
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

struct Rows6 {   // x[q-1], x[q..q+3], x[q+4] of three rows j-1, j, j+1
  float v[3][6];
};

__device__ __forceinline__ void load_rows6(const float* __restrict__ x, size_t rowbase, int n1, int q,
                                           bool has_left, bool has_right, Rows6& r) {
#pragma unroll
  for (int dy = 0; dy < 3; ++dy) {
    const float* p = x + rowbase + (size_t)(dy - 1) * n1 + q;
    const float4 c = __ldg(reinterpret_cast<const float4*>(p));
    r.v[dy][0] = has_left ? __ldg(p - 1) : 0.f;
    r.v[dy][1] = c.x;
    r.v[dy][2] = c.y;
    r.v[dy][3] = c.z;
    r.v[dy][4] = c.w;
    r.v[dy][5] = has_right ? __ldg(p + 4) : 0.f;
  }
}

// eps of the 5 cells x = q-1 .. q+3 of cell rows j-1 (r = 0) and j (r = 1) of
// layer l, from the copy of eps_c whose rows are padded to N+1 floats (one
// float4 per row plus the left neighbour; cell x = N reads the zero pad, and
// cells outside the grid only reach boundary vertices)
__device__ __forceinline__ void load_eps10(const float* __restrict__ eps_pad, int N, int l, int j, int q,
                                           bool has_left, bool /*has_right*/, float (&g)[2][5]) {
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const float* e = eps_pad + ((size_t)l * N + (j - 1 + r)) * (N + 1) + q;
    const float4 c = __ldg(reinterpret_cast<const float4*>(e));
    g[r][0] = has_left ? __ldg(e - 1) : 0.f;
    g[r][1] = c.x;
    g[r][2] = c.y;
    g[r][3] = c.z;
    g[r][4] = c.w;
  }
}

// Py[r][c] = sum of u over the 4 vertices (x, x+1) x (row r, row r+1) of plane rows
__device__ __forceinline__ void pair_sums(const Rows6& u, float (&py)[2][5]) {
  float px[3][5];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 5; ++c) px[r][c] = u.v[r][c] + u.v[r][c + 1];
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int c = 0; c < 5; ++c) py[r][c] = px[r][c] + px[r + 1][c];
}

// NT > 0: the grid size as a compile-time constant (the strides of every
// neighbour access fold into address immediates); NT = 0: from the LevelOp
template <int NT>
struct GeoCtx {
  const float* x;
  const float* b;
  float* y;
  const float* eps;
  float* zr;              // fused residual + restriction: z-restricted residual planes
  const float* dq;        // Jacobi sweep with a dot product: the other operand
  const uint32_t* tmask;  // touched-vertex bits (their residuals are added later)
  int N, n1, q, j;
  int k1;                 // last plane of the current z run
  int K0;                 // fused residual + restriction: first coarse plane of the run
  size_t plane, row0;
  bool hl, hr;
  bool first_row, last_row;   // edge rows of the block also prefetch the halo rows
  float h12, h3, omega;
  __device__ __forceinline__ int gN() const { return NT ? NT : N; }
  __device__ __forceinline__ int gn1() const { return NT ? NT + 1 : n1; }
  __device__ __forceinline__ size_t gplane() const { return NT ? (size_t)(NT + 1) * (NT + 1) : plane; }
};

// the lines plane k + 1 + kGeoPF (u) and k + kGeoPF (b, eps) of a thread's rows
template <int NT>
__device__ __forceinline__ void geo_prefetch(const GeoCtx<NT>& c, int k) {
  if (kGeoPF == 0 || k + kGeoPF > c.k1) return;
  const int kp = k + kGeoPF;
  const float* u = c.x + (size_t)(kp + 1) * c.gplane() + c.row0 + c.q;
  prefetch_l2(u);
  prefetch_l2(c.b + (size_t)kp * c.gplane() + c.row0 + c.q);
  const float* e = c.eps + ((size_t)kp * c.gN() + c.j) * (c.gN() + 1) + c.q;   // eps row j of layer kp
  prefetch_l2(e);
  if (c.first_row) {
    prefetch_l2(u - c.gn1());
    prefetch_l2(e - (c.gN() + 1));
  }
  if (c.last_row) prefetch_l2(u + c.gn1());
}

// One plane k of the bulk pass.  In: u rows of plane k (uc), their pair sums
// (pyc), eps of cell layer k-1 (gm) and its eps-weighted cell sums (yTm).
// Out: the same quantities one plane up (un, pyn, gc, yTc), loaded or formed
// here, so that a two-step unrolled loop swaps roles instead of copying.
template <int MODE, int NT>
__device__ __forceinline__ void geo_step(const GeoCtx<NT>& c, int k, const Rows6& uc, Rows6& un,
                                         const float (&pyc)[2][5], float (&pyn)[2][5], const float (&gm)[2][5],
                                         float (&gc)[2][5], const float (&yTm)[5], float (&yTc)[5], float& d1,
                                         float& d2, float (&za)[4], float (&zb)[4]) {
  const size_t v0 = (size_t)k * c.gplane() + c.row0 + c.q;
  unsigned tw = 0;
  if (MODE == SW_RESID_RZ || MODE == SW_JACOBI_DOT) tw = __ldg(c.tmask + (v0 >> 5));
  float4 q4 = make_float4(0.f, 0.f, 0.f, 0.f);
  if (MODE == SW_JACOBI_DOT) q4 = __ldg(reinterpret_cast<const float4*>(c.dq + v0));
  load_rows6(c.x, (size_t)(k + 1) * c.gplane() + c.row0, c.gn1(), c.q, c.hl, c.hr, un);
  load_eps10(c.eps, c.gN(), k, c.j, c.q, c.hl, c.hr, gc);   // c.eps: padded rows
  geo_prefetch(c, k);
  const float4 b4 = __ldg(reinterpret_cast<const float4*>(c.b + (size_t)k * c.gplane() + c.row0 + c.q));
  // plane k-1, row j (read two planes ago: an L1/L2 hit)
  const float4 m4 = __ldg(reinterpret_cast<const float4*>(c.x + (size_t)(k - 1) * c.gplane() + c.row0 + c.q));
  // layer k: cell sums T = Py(k) + Py(k+1), weighted by eps and summed over the two cell rows
  pair_sums(un, pyn);
#pragma unroll
  for (int i = 0; i < 5; ++i)
    yTc[i] = gc[0][i] * (pyc[0][i] + pyn[0][i]) + gc[1][i] * (pyc[1][i] + pyn[1][i]);
  // eps sums: per cell row over layers k-1, k (ez), per column (ey), per layer over rows (el)
  float ez[2][5], ey[5], elm[5], elc[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    ez[0][i] = gm[0][i] + gc[0][i];
    ez[1][i] = gm[1][i] + gc[1][i];
    ey[i] = ez[0][i] + ez[1][i];
    elm[i] = gm[0][i] + gm[1][i];
    elc[i] = gc[0][i] + gc[1][i];
  }
  const float bb4[4] = {b4.x, b4.y, b4.z, b4.w};
  const float um1[4] = {m4.x, m4.y, m4.z, m4.w};
  float yT[5];   // eps-weighted cell sums of both layers, per cell column
#pragma unroll
  for (int i = 0; i < 5; ++i) yT[i] = yTm[i] + yTc[i];
  float out[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const float uv = uc.v[1][e + 1];
    const float G = ey[e] + ey[e + 1];
    const float ST = yT[e] + yT[e + 1];
    float w = 5.f * uv * G - ST;
    w = fmaf(ey[e], uc.v[1][e], w);                         // x - 1
    w = fmaf(ey[e + 1], uc.v[1][e + 2], w);                 // x + 1
    w = fmaf(ez[0][e] + ez[0][e + 1], uc.v[0][e + 1], w);   // y - 1
    w = fmaf(ez[1][e] + ez[1][e + 1], uc.v[2][e + 1], w);   // y + 1
    w = fmaf(elm[e] + elm[e + 1], um1[e], w);               // z - 1
    w = fmaf(elc[e] + elc[e + 1], un.v[1][e + 1], w);       // z + 1
    const int i = c.q + e;
    const bool valid = i >= 1 && i <= c.gN() - 1;
    float r;
    // Jacobi: u + omega (b - h/12 w) / (h/3 G), with omega / (h/3) folded into c.omega
    if (MODE == SW_JACOBI || MODE == SW_JACOBI_DOT) r = fmaf(c.omega, __fdividef(fmaf(-c.h12, w, bb4[e]), G), uv);
    else if (MODE == SW_RESID || MODE == SW_RESID_RZ) r = fmaf(-c.h12, w, bb4[e]);
    else {
      const float acc = c.h12 * w;
      r = acc;
      if (valid) {
        d1 += uv * acc;
        d2 += uv * bb4[e];
      }
    }
    out[e] = valid ? r : 0.f;   // boundary vertices stay zero
  }
  if (MODE == SW_JACOBI_DOT) {   // touched vertices: their term comes from the fix-up pass
    const unsigned tb = (tw >> (unsigned)(v0 & 31)) & 0xFu;
    d1 += ((tb & 1u) ? 0.f : out[0] * q4.x) + ((tb & 2u) ? 0.f : out[1] * q4.y) +
          ((tb & 4u) ? 0.f : out[2] * q4.z) + ((tb & 8u) ? 0.f : out[3] * q4.w);
  }
  if (MODE == SW_RESID_RZ) {
    // z restriction: plane k = 3 cz + m adds (1 - m/3) r to coarse plane cz and
    // (m/3) r to cz + 1; cz is complete after m = 2.  Touched vertices add
    // nothing here (zr_fix_kernel adds their fix-up residuals).
    const unsigned tb = (tw >> (unsigned)(v0 & 31)) & 0xFu;
#pragma unroll
    for (int e = 0; e < 4; ++e)
      if ((tb >> e) & 1u) out[e] = 0.f;
    const float wa = 1.f / 3.f, wb = 2.f / 3.f;
    const int cz = k / 3, m = k - 3 * cz;
    if (m == 0) {
#pragma unroll
      for (int e = 0; e < 4; ++e) za[e] += out[e];
    } else if (m == 1) {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        za[e] = fmaf(wb, out[e], za[e]);
        zb[e] = fmaf(wa, out[e], zb[e]);
      }
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        za[e] = fmaf(wa, out[e], za[e]);
        zb[e] = fmaf(wb, out[e], zb[e]);
      }
      if (cz >= c.K0)
        *reinterpret_cast<float4*>(c.zr + (size_t)cz * c.gplane() + c.row0 + c.q) = make_float4(za[0], za[1], za[2], za[3]);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        za[e] = zb[e];
        zb[e] = 0.f;
      }
    }
    return;
  }
  *reinterpret_cast<float4*>(c.y + v0) = make_float4(out[0], out[1], out[2], out[3]);
}

template <int MODE, int NT>
__global__ void __launch_bounds__(kGeoBX * kGeoBY, 2) sweep3_geo4(const LevelOp op, const float* __restrict__ x,
                                                                  const float* __restrict__ b,
                                                                  float* __restrict__ y, float omega,
                                                                  double* __restrict__ partials, int ntx, int nty,
                                                                  float* __restrict__ zr) {
  pdl_begin();
  __shared__ double sh[2][8];
  GeoCtx<NT> c;
  c.x = x;
  c.b = b;
  c.y = y;
  c.eps = op.eps_pad;
  c.zr = zr;
  c.dq = zr;   // SW_JACOBI_DOT: the dot operand comes in the last argument
  c.tmask = op.tmask;
  c.K0 = 0;
  c.N = NT ? NT : op.N;
  c.n1 = c.N + 1;
  c.plane = (size_t)c.n1 * c.n1;
  c.h12 = -op.gk32;   // h / 12
  c.h3 = 4.f * c.h12;   // h / 3
  c.omega = omega / c.h3;   // the Jacobi step divides by h/3 G
  // per-thread partial dot products in FP32 (a few hundred terms; they only
  // set the Krylov step lengths), summed over the block in FP64
  float d1 = 0.f, d2 = 0.f;
  long long w, w1;
  // work items: (column, interior plane), or (column, interior coarse plane)
  // for the fused residual + restriction, whose run over coarse planes
  // K0 .. K1 marches the fine planes 3 K0 - 2 .. 3 K1 + 2
  const int nk = MODE == SW_RESID_RZ ? c.gN() / 3 - 1 : c.gN() - 1;
  geo_share(ntx, nty, nk, w, w1);
  GeoRun run;
  float za[4] = {0.f, 0.f, 0.f, 0.f}, zb[4] = {0.f, 0.f, 0.f, 0.f};
  while (next_geo_run(w, w1, nk, ntx, run)) {
    c.q = 4 * (run.tx * kGeoBX + threadIdx.x);   // vertices q .. q+3
    c.j = 1 + run.ty * kGeoBY + threadIdx.y;
    int k0 = run.k0, k1 = run.k1;
    if (MODE == SW_RESID_RZ) {
      c.K0 = k0;
      k0 = 3 * k0 - 2;
      k1 = 3 * k1 + 2;
#pragma unroll
      for (int e = 0; e < 4; ++e) za[e] = zb[e] = 0.f;
    }
    if (c.q >= c.gn1() || c.j >= c.gN()) continue;
    c.k1 = k1;
    c.hl = c.q > 0;
    c.hr = c.q + 4 <= c.gN();
    c.first_row = threadIdx.y == 0;
    c.last_row = threadIdx.y == kGeoBY - 1 || c.j == c.gN() - 1;
    c.row0 = (size_t)c.j * c.gn1();
    // prologue: rows and pair sums of plane k0, eps and weighted cell sums of layer k0-1
    Rows6 ua, ub;
    float pa[2][5], pb[2][5], ga[2][5], gb[2][5], ta[5], tb[5];
    load_rows6(x, (size_t)(k0 - 1) * c.gplane() + c.row0, c.gn1(), c.q, c.hl, c.hr, ub);
    load_rows6(x, (size_t)k0 * c.gplane() + c.row0, c.gn1(), c.q, c.hl, c.hr, ua);
    load_eps10(op.eps_pad, c.gN(), k0 - 1, c.j, c.q, c.hl, c.hr, ga);
    pair_sums(ub, pb);
    pair_sums(ua, pa);
#pragma unroll
    for (int i = 0; i < 5; ++i) ta[i] = ga[0][i] * (pb[0][i] + pa[0][i]) + ga[1][i] * (pb[1][i] + pa[1][i]);
    for (int k = k0; k <= k1; k += 2) {
      geo_step<MODE, NT>(c, k, ua, ub, pa, pb, ga, gb, ta, tb, d1, d2, za, zb);
      if (k + 1 > k1) break;
      geo_step<MODE, NT>(c, k + 1, ub, ua, pb, pa, gb, ga, tb, ta, d1, d2, za, zb);
    }
  }
  if (MODE == SW_MATVEC) {
    const double s1 = block_sum((double)d1, sh[0]);
    const double s2 = block_sum((double)d2, sh[1]);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      partials[2 * blockIdx.x] = s1;
      partials[2 * blockIdx.x + 1] = s2;
    }
  } else if (MODE == SW_JACOBI_DOT) {
    const double s1 = block_sum((double)d1, sh[0]);
    if (threadIdx.x == 0 && threadIdx.y == 0) partials[blockIdx.x] = s1;
  }
}

// Fix-up pass: vertices in op.touched (count *op.ntouched) recomputed with the
// full operator (geometric part and decoded surplus): from the precomputed
// 27-point stencil for the first op.tcap of them, else from the cell records.
// For SW_MATVEC the difference to the value the bulk pass wrote is added to
// the dot products; for SW_JACOBI_DOT (dot operand dq, touched vertices left
// out of the bulk pass's sum) the touched vertices' terms.
template <int MODE>
__global__ void __launch_bounds__(256) sweep3_fixup(const LevelOp op, const float* __restrict__ x,
                                                    const float* __restrict__ b, float* __restrict__ y,
                                                    float omega, double* __restrict__ partials,
                                                    const float* __restrict__ dq) {
  // the next kernel may be scheduled now: it waits for this grid, which ends
  // after the bulk pass (this grid was scheduled once the bulk pass's own wait
  // had returned, so x and b are complete)
  pdl_trigger();
  __shared__ double sh[2][8];
  const int N = op.N, n1 = N + 1;
  const int nt = *op.ntouched;
  const int cap = op.tcap;
  float d1 = 0.f;
  // Launched as a programmatic dependent of the bulk pass: everything up to
  // the first access of y (written by the bulk pass) overlaps its tail.
  bool waited = false;
  auto wait_bulk = [&]() {
    if (!waited) pdl_wait();
    waited = true;
  };
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += gridDim.x * blockDim.x) {
    const int v = op.touched[t];
    if constexpr (MODE == SW_JACOBI0) {   // zero iterate: only the diagonal is needed
      float dg;
      if (t < cap) {
        dg = __ldg(op.tcoef + t + (size_t)13 * cap);
      } else {
        float u0[27];
#pragma unroll
        for (int q = 0; q < 27; ++q) u0[q] = 0.f;
        float Au0;
        const int i = v % n1, j = (v / n1) % n1, k = v / (n1 * n1);
        vertex_apply<3, float, true, float>(op, i, j, k, u0, &Au0, &dg);
      }
      const float r = omega * __ldg(b + v) / dg;
      wait_bulk();
      y[v] = r;
    } else {
      float u[27];
#pragma unroll
      for (int dz = 0; dz < 3; ++dz)
#pragma unroll
        for (int dy = 0; dy < 3; ++dy)
#pragma unroll
          for (int dx = 0; dx < 3; ++dx)
            u[dx + 3 * dy + 9 * dz] = __ldg(x + (size_t)v + (dx - 1) + (dy - 1) * n1 + (size_t)(dz - 1) * n1 * n1);
      float Au, dg;
      const float uv = u[13];
      // right-hand side (the bulk pass's value for the matvec) fetched up front
      if (MODE == SW_MATVEC) wait_bulk();
      const float bv = MODE == SW_MATVEC ? y[v] : __ldg(b + v);
      if (t < cap) {
        // all 27 coefficient loads issued before the first use (independent of u)
        const float* cf = op.tcoef + t;
        float c[27];
#pragma unroll
        for (int q = 0; q < 27; ++q) c[q] = __ldg(cf + (size_t)q * cap);
        float acc = 0.f;
#pragma unroll
        for (int q = 0; q < 27; ++q)
          if (q != 13) acc = fmaf(c[q], u[q] - uv, acc);
        Au = acc;
        dg = c[13];
      } else {
        const int i = v % n1, j = (v / n1) % n1, k = v / (n1 * n1);
        vertex_apply<3, float, true, float>(op, i, j, k, u, &Au, &dg);
      }
      if (MODE == SW_JACOBI) {
        const float r = uv + omega * (bv - Au) / dg;
        wait_bulk();
        y[v] = r;
      } else if (MODE == SW_JACOBI_DOT) {
        const float r = uv + omega * (bv - Au) / dg;
        d1 += r * __ldg(dq + v);   // the bulk pass left the touched vertices out
        wait_bulk();
        y[v] = r;
      } else if (MODE == SW_RESID) {
        const float r = bv - Au;
        wait_bulk();
        y[v] = r;
      } else {
        y[v] = Au;
        d1 += uv * (Au - bv);   // bv: the bulk pass's value at v
      }
    }
  }
  wait_bulk();   // the grid never completes before the bulk pass
  if (MODE == SW_MATVEC) {
    const double s1 = block_sum((double)d1, sh[0]);
    if (threadIdx.x == 0) {
      partials[2 * blockIdx.x] = s1;
      partials[2 * blockIdx.x + 1] = 0.0;
    }
  } else if (MODE == SW_JACOBI_DOT) {
    const double s1 = block_sum((double)d1, sh[0]);
    if (threadIdx.x == 0) partials[blockIdx.x] = s1;
  }
}

// stencils of the first min(*ntouched, tcap) touched vertices
__global__ void touched_stencil_kernel(const LevelOp op) {
  const int n1 = op.N + 1;
  const int nt = min(*op.ntouched, op.tcap);
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += gridDim.x * blockDim.x) {
    const int v = op.touched[t];
    const int i = v % n1, j = (v / n1) % n1, k = v / (n1 * n1);
    float c[27];
    vertex_coeffs3(op, i, j, k, c);
#pragma unroll
    for (int q = 0; q < 27; ++q) op.tcoef[(size_t)q * op.tcap + t] = c[q];
  }
}

#ifndef MG_J0_BLOCKS_PER_SM
#define MG_J0_BLOCKS_PER_SM 5
#endif
#ifndef MG_FIX_BLOCKS_PER_SM
#define MG_FIX_BLOCKS_PER_SM 3
#endif
// fix-up grids: the FP32 pass holds three 256-thread blocks per SM at its
// register count (the FP64 one two; its surplus blocks wait for a slot)
constexpr int kFixBlocks = 152 * MG_FIX_BLOCKS_PER_SM;

// ---------------------------------------------------------------- 3D FP64 split residual / matvec
// The outer FP64 iteration of the mixed paths needs r = f - A u and A p on the
// compressed finest level in FP64, where the FP64 pipe (1/64 of FP32 on this
// part) is the bound.  The same split as the FP32 sweep: a class-blind bulk
// pass applies the geometric part in the factored form (fewest FP64 operations
// per vertex, about 40), then a fix-up pass adds the decoded surplus of the
// cells with records at the touched vertices (exact FP32 entries, FP64 sums).
// Bulk: 2 vertices per thread (double2 rows), z march as in the FP32 pass.
template <typename T>
struct Vec2T;
template <>
struct Vec2T<float> {
  using type = float2;
};
template <>
struct Vec2T<double> {
  using type = double2;
};

template <typename T>
struct Rows4 {   // x[q-1], x[q], x[q+1], x[q+2] of three rows j-1, j, j+1
  T v[3][4];
};

template <typename T>
__device__ __forceinline__ void load_rows4(const T* __restrict__ p, int n1, bool has_left, bool has_right,
                                           Rows4<T>& r) {
  using V2 = typename Vec2T<T>::type;
#pragma unroll
  for (int dy = 0; dy < 3; ++dy) {
    const T* q = p + (dy - 1) * n1;
    const V2 c = __ldg(reinterpret_cast<const V2*>(q));
    r.v[dy][0] = has_left ? __ldg(q - 1) : (T)0;
    r.v[dy][1] = c.x;
    r.v[dy][2] = c.y;
    r.v[dy][3] = has_right ? __ldg(q + 2) : (T)0;
  }
}

// eps of cells x = q-1, q, q+1 of cell rows j-1 (r = 0) and j (r = 1) of layer l
template <typename T>
__device__ __forceinline__ void load_eps6(const float* __restrict__ eps, int N, int l, int j, int q,
                                          bool has_left, bool has_right, T (&g)[2][3]) {
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const float* e = eps + ((size_t)l * N + (j - 1 + r)) * N + q;
    g[r][0] = has_left ? (T)__ldg(e - 1) : (T)0;
    g[r][1] = (T)__ldg(e);
    g[r][2] = has_right ? (T)__ldg(e + 1) : (T)0;
  }
}

template <typename T>
__device__ __forceinline__ void pair_sums4(const Rows4<T>& u, T (&py)[2][3]) {
  T px[3][3];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) px[r][c] = u.v[r][c] + u.v[r][c + 1];
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) py[r][c] = px[r][c] + px[r + 1][c];
}

// the same from the FP64 cell-centre eps (exact operator of the FP64 residual)
template <typename T>
__device__ __forceinline__ void load_eps6(const double* __restrict__ eps, int N, int l, int j, int q,
                                          bool has_left, bool has_right, T (&g)[2][3]) {
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const double* e = eps + ((size_t)l * N + (j - 1 + r)) * N + q;
    g[r][0] = has_left ? (T)__ldg(e - 1) : (T)0;
    g[r][1] = (T)__ldg(e);
    g[r][2] = has_right ? (T)__ldg(e + 1) : (T)0;
  }
}

template <typename T>
struct Geo2Ctx {
  const T* x;
  const T* b;
  T* y;
  const float* eps;
  const double* eps64;   // non-null: FP64 cell-centre eps (FP64 instance, exact operator)
  int N, n1, q, j;
  size_t plane, row0;
  bool hl, hr, hr2;
  T h12, h3, omega;
};

template <typename T, int MODE>
__device__ __forceinline__ void geo2_step(const Geo2Ctx<T>& c, int k, const Rows4<T>& uc, Rows4<T>& un,
                                          const T (&pyc)[2][3], T (&pyn)[2][3], const T (&gm)[2][3], T (&gc)[2][3],
                                          const T (&yTm)[3], T (&yTc)[3], double& d1, double& d2) {
  using V2 = typename Vec2T<T>::type;
  load_rows4<T>(c.x + (size_t)(k + 1) * c.plane + c.row0 + c.q, c.n1, c.hl, c.hr, un);
  if (sizeof(T) == 8 && c.eps64) load_eps6<T>(c.eps64, c.N, k, c.j, c.q, c.hl, c.hr2, gc);
  else load_eps6<T>(c.eps, c.N, k, c.j, c.q, c.hl, c.hr2, gc);
  const V2 b2 = __ldg(reinterpret_cast<const V2*>(c.b + (size_t)k * c.plane + c.row0 + c.q));
  const V2 m2 = __ldg(reinterpret_cast<const V2*>(c.x + (size_t)(k - 1) * c.plane + c.row0 + c.q));
  pair_sums4<T>(un, pyn);
  T yZ[3], ez[2][3], ey[3], elm[3], elc[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    yTc[i] = gc[0][i] * (pyc[0][i] + pyn[0][i]) + gc[1][i] * (pyc[1][i] + pyn[1][i]);
    yZ[i] = yTm[i] + yTc[i];
    ez[0][i] = gm[0][i] + gc[0][i];
    ez[1][i] = gm[1][i] + gc[1][i];
    ey[i] = ez[0][i] + ez[1][i];
    elm[i] = gm[0][i] + gm[1][i];
    elc[i] = gc[0][i] + gc[1][i];
  }
  const T bb[2] = {b2.x, b2.y};
  const T um1[2] = {m2.x, m2.y};
  T out[2];
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const T uv = uc.v[1][e + 1];
    const T G = ey[e] + ey[e + 1];
    T w = fma((T)5 * uv, G, -(yZ[e] + yZ[e + 1]));
    w = fma(ey[e], uc.v[1][e], w);                         // x - 1
    w = fma(ey[e + 1], uc.v[1][e + 2], w);                 // x + 1
    w = fma(ez[0][e] + ez[0][e + 1], uc.v[0][e + 1], w);   // y - 1
    w = fma(ez[1][e] + ez[1][e + 1], uc.v[2][e + 1], w);   // y + 1
    w = fma(elm[e] + elm[e + 1], um1[e], w);               // z - 1
    w = fma(elc[e] + elc[e + 1], un.v[1][e + 1], w);       // z + 1
    const T acc = c.h12 * w;
    const int i = c.q + e;
    const bool valid = i >= 1 && i <= c.N - 1;
    T r;
    if (MODE == SW_JACOBI) {
      if (sizeof(T) == 4) r = uv + c.omega * __fdividef((float)(bb[e] - acc), (float)(c.h3 * G));
      else r = uv + c.omega * (bb[e] - acc) / (c.h3 * G);
    } else if (MODE == SW_RESID) {
      r = bb[e] - acc;
    } else {
      r = acc;
      if (valid) {
        d1 += (double)uv * (double)acc;
        d2 += (double)uv * (double)bb[e];
      }
    }
    out[e] = valid ? r : (T)0;
  }
  V2 o;
  o.x = out[0];
  o.y = out[1];
  *reinterpret_cast<V2*>(c.y + (size_t)k * c.plane + c.row0 + c.q) = o;
}

// The factored bulk pass with 2 vertices per thread (vec2 rows), used in FP64
// for the outer residual.  (An FP32 instance with 3 blocks per SM ran no faster
// than the 4-vertex FP32 pass: both are bound by loads in flight per SM.)
template <typename T, int MODE, int MINB>
__global__ void __launch_bounds__(kGeoBX * kGeoBY, MINB) sweep3_geo2(const LevelOp op, const T* __restrict__ x,
                                                                      const T* __restrict__ b, T* __restrict__ y,
                                                                      T omega, double* __restrict__ partials,
                                                                      int ntx, int nty) {
  __shared__ double sh[2][8];
  Geo2Ctx<T> c;
  c.x = x;
  c.b = b;
  c.y = y;
  c.eps = op.eps_c;
  c.eps64 = sizeof(T) == 8 ? op.eps64 : nullptr;
  c.N = op.N;
  c.n1 = op.N + 1;
  c.plane = (size_t)c.n1 * c.n1;
  c.h12 = sizeof(T) == 4 ? (T)-op.gk32 : (T)-op.gk64;   // h / 12
  c.h3 = (T)4 * c.h12;
  c.omega = omega;
  double d1 = 0.0, d2 = 0.0;
  long long w, w1;
  geo_share(ntx, nty, c.N - 1, w, w1);
  GeoRun run;
  while (next_geo_run(w, w1, c.N - 1, ntx, run)) {
    c.q = 2 * (run.tx * kGeoBX + threadIdx.x);   // vertices q, q+1
    c.j = 1 + run.ty * kGeoBY + threadIdx.y;
    const int k0 = run.k0, k1 = run.k1;
    if (c.q >= c.n1 || c.j >= c.N) continue;
    c.hl = c.q > 0;
    c.hr = c.q + 2 <= c.N;      // vertex q+2 exists
    c.hr2 = c.q + 1 <= c.N - 1; // cell q+1 exists
    c.row0 = (size_t)c.j * c.n1;
    Rows4<T> ua, ub;
    T pa[2][3], pb[2][3], ga[2][3], gb[2][3], ta[3], tb[3];
    load_rows4<T>(x + (size_t)(k0 - 1) * c.plane + c.row0 + c.q, c.n1, c.hl, c.hr, ub);
    load_rows4<T>(x + (size_t)k0 * c.plane + c.row0 + c.q, c.n1, c.hl, c.hr, ua);
    if (c.eps64) load_eps6<T>(c.eps64, c.N, k0 - 1, c.j, c.q, c.hl, c.hr2, ga);
    else load_eps6<T>(op.eps_c, c.N, k0 - 1, c.j, c.q, c.hl, c.hr2, ga);
    pair_sums4<T>(ub, pb);
    pair_sums4<T>(ua, pa);
#pragma unroll
    for (int i = 0; i < 3; ++i) ta[i] = ga[0][i] * (pb[0][i] + pa[0][i]) + ga[1][i] * (pb[1][i] + pa[1][i]);
    for (int k = k0; k <= k1; k += 2) {
      geo2_step<T, MODE>(c, k, ua, ub, pa, pb, ga, gb, ta, tb, d1, d2);
      if (k + 1 > k1) break;
      geo2_step<T, MODE>(c, k + 1, ub, ua, pb, pa, gb, ga, tb, ta, d1, d2);
    }
  }
  if (MODE == SW_MATVEC) {
    const double s1 = block_sum(d1, sh[0]);
    const double s2 = block_sum(d2, sh[1]);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      partials[2 * blockIdx.x] = s1;
      partials[2 * blockIdx.x + 1] = s2;
    }
  }
}

// surplus part sum_c Delta_c u at the touched vertices, added in FP64 (RESID:
// y -= it; MATVEC: y += it and its contribution to u . A u)
template <int MODE>
__global__ void __launch_bounds__(256) sweep3_fixup64(const LevelOp op, const double* __restrict__ x,
                                                      double* __restrict__ y, double* __restrict__ partials) {
  constexpr int NV = 8;
  __shared__ double sh[2][8];
  const int N = op.N, n1 = N + 1;
  // exact operator: every vertex next to an interface cell, the FP64 surplus;
  // otherwise the vertices next to a cell with a record, the decoded surplus
  const bool exact = op.eps64 != nullptr;
  const int* tl = exact ? op.touched64 : op.touched;
  const int nt = exact ? *op.ntouched64 : *op.ntouched;
  double d1 = 0.0;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += gridDim.x * blockDim.x) {
    const int v = tl[t];
    const int i = v % n1, j = (v / n1) % n1, k = v / (n1 * n1);
    double u[27];
#pragma unroll
    for (int dz = 0; dz < 3; ++dz)
#pragma unroll
      for (int dy = 0; dy < 3; ++dy)
#pragma unroll
        for (int dx = 0; dx < 3; ++dx)
          u[dx + 3 * dy + 9 * dz] = __ldg(x + (size_t)v + (dx - 1) + (dy - 1) * n1 + (size_t)(dz - 1) * n1 * n1);
    double acc = 0.0;
#pragma unroll
    for (int oz = 0; oz < 2; ++oz) {
      const int cl = k - 1 + oz;
      int ch = cl / op.layers;
      ch = ch < op.nchunk ? ch : op.nchunk - 1;
      const int ll = cl - ch * op.layers;
      const CmpChunk& ck = op.cmp[ch];
#pragma unroll
      for (int oy = 0; oy < 2; ++oy) {
        const int segrow = (ll * N + (j - 1 + oy)) * op.nseg_x;
#pragma unroll
        for (int ox = 0; ox < 2; ++ox) {
          const int cx = i - 1 + ox;
          const int a = (1 - ox) | ((1 - oy) << 1) | ((1 - oz) << 2);
          if (exact) {
            const int ps = __ldg(op.xpos + ((size_t)cl * N + (j - 1 + oy)) * N + cx);
            if (ps < 0 || !ck.x64) continue;
            const double* xr = ck.x64 + (size_t)ps * 28;
#pragma unroll
            for (int bb = 0; bb < NV; ++bb) {
              if (bb == a) continue;
              const double dv = __ldg(xr + pair_of(NV, a, bb));
              const int ub = (ox + (bb & 1)) + 3 * (oy + ((bb >> 1) & 1)) + 9 * (oz + ((bb >> 2) & 1));
              acc += dv * (u[ub] - u[13]);
            }
            continue;
          }
          const int seg = segrow + (cx >> 5);
          const int cls = __ldg(ck.cls + (size_t)seg * kSegCells + (cx & 31));
          if (!cls) continue;
          const uint8_t* rec = record_at<3>(ck, seg, cx & 31, cls);
#pragma unroll
          for (int bb = 0; bb < NV; ++bb) {
            if (bb == a) continue;
            const double dv = (double)decode_entry<3>(rec, cls, pair_of(NV, a, bb));
            const int ub = (ox + (bb & 1)) + 3 * (oy + ((bb >> 1) & 1)) + 9 * (oz + ((bb >> 2) & 1));
            acc += dv * (u[ub] - u[13]);
          }
        }
      }
    }
    if (MODE == SW_RESID) {
      y[v] -= acc;
    } else {
      y[v] += acc;
      d1 += u[13] * acc;
    }
  }
  if (MODE == SW_MATVEC) {
    const double s1 = block_sum(d1, sh[0]);
    if (threadIdx.x == 0) {
      partials[2 * blockIdx.x] = s1;
      partials[2 * blockIdx.x + 1] = 0.0;
    }
  }
}

// ---- FP64 bulk pass in vertex form.  With the weights built once per
// problem, (A u)_v = gs_v u_v + sum over the 6 axis neighbours w of W_vw u_w
// - sum over the 8 cells c at v of es_c T_c (gs = 5 h/12 G, W and es scaled by
// h/12, T_c the sum of u over the vertices of c): the same terms as the cell
// form above, but the eps sums per vertex and edge are loaded instead of
// formed in every application, which cuts the FP64 operations per vertex
// from about 38 to 25 (the pass is bound by the FP64 pipe).
__global__ void geo_weights64_kernel(int N, const double* __restrict__ eps64, const float* __restrict__ eps32,
                                     double h12, double* __restrict__ gs, double* __restrict__ wx,
                                     double* __restrict__ wy, double* __restrict__ wz, double* __restrict__ es) {
  const int n1 = N + 1;
  const long long nv = (long long)n1 * n1 * n1;
  auto E = [&](int cx, int cy, int cz) -> double {
    if (cx < 0 || cx >= N || cy < 0 || cy >= N || cz < 0 || cz >= N) return 0.0;
    const size_t c = ((size_t)cz * N + cy) * N + cx;
    return eps64 ? eps64[c] : (double)eps32[c];
  };
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nv;
       v += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(v % n1), j = (int)((v / n1) % n1), k = (int)(v / ((long long)n1 * n1));
    // e[c][b][a]: eps of the cell (i - 1 + a, j - 1 + b, k - 1 + c) at v (0 outside)
    double e[2][2][2];
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int a = 0; a < 2; ++a) e[c][b][a] = E(i - 1 + a, j - 1 + b, k - 1 + c);
    double g = 0.0, ex = 0.0, ey = 0.0, ez = 0.0;
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        ex += e[c][b][1];   // cells at the edge (v, v+x): x index i
        ey += e[c][1][b];
        ez += e[1][c][b];
#pragma unroll
        for (int a = 0; a < 2; ++a) g += e[c][b][a];
      }
    gs[v] = 5.0 * h12 * g;
    wx[v] = h12 * ex;
    wy[v] = h12 * ey;
    wz[v] = h12 * ez;
    // padded cell row: cell (i, j, k) for i < N, zero at i = N
    if (j < N && k < N) es[((size_t)k * N + j) * n1 + i] = h12 * e[1][1][1];   // zero at i = N
  }
}

// three consecutive doubles e[-1], e[0], e[1] of a padded row (e[-1] = 0 when !has_left)
__device__ __forceinline__ void load_es3(const double* __restrict__ e, bool has_left, double (&g)[3]) {
  const double2 c = __ldg(reinterpret_cast<const double2*>(e));
  g[0] = has_left ? __ldg(e - 1) : 0.0;
  g[1] = c.x;
  g[2] = c.y;
}

struct GeoW64Ctx {
  const double* x;
  const double* b;
  double* y;
  const double* w[4];
  const double* es;
  int N, n1, q, j;
  size_t plane, row0;
  bool hl, hr;
};

// one plane k of the vertex-form FP64 pass: 2 vertices (q, q+1) of row j
template <int MODE>
__device__ __forceinline__ void geow64_step(const GeoW64Ctx& c, int k, const Rows4<double>& uc, Rows4<double>& un,
                                            const double (&pyc)[2][3], double (&pyn)[2][3],
                                            const double (&yTm)[3], double (&yTc)[3], double (&wzm)[2],
                                            double& d1, double& d2) {
  const size_t v0 = (size_t)k * c.plane + c.row0 + c.q;
  // row j of plane k-1: the centre row of the buffer refilled below
  const double um1[2] = {un.v[1][1], un.v[1][2]};
  load_rows4<double>(c.x + v0 + c.plane, c.n1, c.hl, c.hr, un);
  double gc[2][3];
  const size_t erow = ((size_t)k * c.N + (c.j - 1)) * c.n1 + c.q;   // cell row j-1 of layer k, cell q
  load_es3(c.es + erow, c.hl, gc[0]);
  load_es3(c.es + erow + c.n1, c.hl, gc[1]);
  const double2 b2 = __ldg(reinterpret_cast<const double2*>(c.b + v0));
  const double2 gs = __ldg(reinterpret_cast<const double2*>(c.w[0] + v0));
  const double2 wx = __ldg(reinterpret_cast<const double2*>(c.w[1] + v0));
  const double wxl = c.hl ? __ldg(c.w[1] + v0 - 1) : 0.0;
  const double2 wy = __ldg(reinterpret_cast<const double2*>(c.w[2] + v0));
  const double2 wym = __ldg(reinterpret_cast<const double2*>(c.w[2] + v0 - c.n1));
  const double2 wz = __ldg(reinterpret_cast<const double2*>(c.w[3] + v0));
  pair_sums4<double>(un, pyn);
  double yZ[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    yTc[i] = gc[0][i] * (pyc[0][i] + pyn[0][i]) + gc[1][i] * (pyc[1][i] + pyn[1][i]);
    yZ[i] = yTm[i] + yTc[i];
  }
  const double bb[2] = {b2.x, b2.y}, g5[2] = {gs.x, gs.y}, wxr[2] = {wx.x, wx.y}, wxm[2] = {wxl, wx.x};
  const double wyp[2] = {wy.x, wy.y}, wyn[2] = {wym.x, wym.y}, wzp[2] = {wz.x, wz.y};
  double out[2];
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const double uv = uc.v[1][e + 1];
    double w = fma(g5[e], uv, -(yZ[e] + yZ[e + 1]));
    w = fma(wxr[e], uc.v[1][e + 2], w);   // x + 1
    w = fma(wxm[e], uc.v[1][e], w);       // x - 1
    w = fma(wyp[e], uc.v[2][e + 1], w);   // y + 1
    w = fma(wyn[e], uc.v[0][e + 1], w);   // y - 1
    w = fma(wzp[e], un.v[1][e + 1], w);   // z + 1
    w = fma(wzm[e], um1[e], w);           // z - 1
    const int i = c.q + e;
    const bool valid = i >= 1 && i <= c.N - 1;
    double r;
    if (MODE == SW_RESID) {
      r = bb[e] - w;
    } else {
      r = w;
      if (valid) {
        d1 += uv * w;
        d2 += uv * bb[e];
      }
    }
    out[e] = valid ? r : 0.0;
  }
  wzm[0] = wz.x;
  wzm[1] = wz.y;
  *reinterpret_cast<double2*>(c.y + v0) = make_double2(out[0], out[1]);
}

template <int MODE>
__global__ void __launch_bounds__(kGeoBX * kGeoBY, 2) sweep3_geow64(const LevelOp op, const double* __restrict__ x,
                                                                    const double* __restrict__ b,
                                                                    double* __restrict__ y,
                                                                    double* __restrict__ partials, int ntx, int nty) {
  __shared__ double sh[2][8];
  GeoW64Ctx c;
  c.x = x;
  c.b = b;
  c.y = y;
#pragma unroll
  for (int m = 0; m < 4; ++m) c.w[m] = op.w64[m];
  c.es = op.es64;
  c.N = op.N;
  c.n1 = op.N + 1;
  c.plane = (size_t)c.n1 * c.n1;
  double d1 = 0.0, d2 = 0.0;
  long long w, w1;
  geo_share(ntx, nty, c.N - 1, w, w1);
  GeoRun run;
  while (next_geo_run(w, w1, c.N - 1, ntx, run)) {
    c.q = 2 * (run.tx * kGeoBX + threadIdx.x);   // vertices q, q+1
    c.j = 1 + run.ty * kGeoBY + threadIdx.y;
    const int k0 = run.k0, k1 = run.k1;
    if (c.q >= c.n1 || c.j >= c.N) continue;
    c.hl = c.q > 0;
    c.hr = c.q + 2 <= c.N;
    c.row0 = (size_t)c.j * c.n1;
    Rows4<double> ua, ub;
    double pa[2][3], pb[2][3], ta[3], tb[3], ga[2][3], wzm[2];
    const size_t v0 = (size_t)k0 * c.plane + c.row0 + c.q;
    load_rows4<double>(x + v0 - c.plane, c.n1, c.hl, c.hr, ub);
    load_rows4<double>(x + v0, c.n1, c.hl, c.hr, ua);
    const size_t erow = ((size_t)(k0 - 1) * c.N + (c.j - 1)) * c.n1 + c.q;   // layer k0-1
    load_es3(c.es + erow, c.hl, ga[0]);
    load_es3(c.es + erow + c.n1, c.hl, ga[1]);
    const double2 wz0 = __ldg(reinterpret_cast<const double2*>(c.w[3] + v0 - c.plane));
    wzm[0] = wz0.x;
    wzm[1] = wz0.y;
    pair_sums4<double>(ub, pb);
    pair_sums4<double>(ua, pa);
#pragma unroll
    for (int i = 0; i < 3; ++i) ta[i] = ga[0][i] * (pb[0][i] + pa[0][i]) + ga[1][i] * (pb[1][i] + pa[1][i]);
    for (int k = k0; k <= k1; k += 2) {
      geow64_step<MODE>(c, k, ua, ub, pa, pb, ta, tb, wzm, d1, d2);
      if (k + 1 > k1) break;
      geow64_step<MODE>(c, k + 1, ub, ua, pb, pa, tb, ta, wzm, d1, d2);
    }
  }
  if (MODE == SW_MATVEC) {
    const double s1 = block_sum(d1, sh[0]);
    const double s2 = block_sum(d2, sh[1]);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      partials[2 * blockIdx.x] = s1;
      partials[2 * blockIdx.x + 1] = s2;
    }
  }
}

cudaError_t launch_geo64(const LevelOp& op, int mode, const double* x, const double* b, double* y,
                         double* partials, int* nblocks, cudaStream_t st) {
  const int np = (op.N + 1) / 2;
  const int ntx = (np + kGeoBX - 1) / kGeoBX, nty = (op.N - 1 + kGeoBY - 1) / kGeoBY;
  const long long ntiles = (long long)ntx * nty * (op.N - 1);
  static int nsm = 0;
  if (!nsm) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (nsm <= 0) nsm = 152;
  }
  const int nb = ntiles < 2 * nsm ? (int)ntiles : 2 * nsm;
  const dim3 blk(kGeoBX, kGeoBY, 1);
  double* pfix = partials ? partials + 2 * (size_t)nb : nullptr;
  const bool vform = op.w64[0] != nullptr;
  if (mode == SW_RESID) {
    if (vform) sweep3_geow64<SW_RESID><<<nb, blk, 0, st>>>(op, x, b, y, partials, ntx, nty);
    else sweep3_geo2<double, SW_RESID, 2><<<nb, blk, 0, st>>>(op, x, b, y, 0.0, partials, ntx, nty);
    count_launches(1);
    sweep3_fixup64<SW_RESID><<<kFixBlocks, 256, 0, st>>>(op, x, y, pfix);
  } else {
    if (vform) sweep3_geow64<SW_MATVEC><<<nb, blk, 0, st>>>(op, x, b, y, partials, ntx, nty);
    else sweep3_geo2<double, SW_MATVEC, 2><<<nb, blk, 0, st>>>(op, x, b, y, 0.0, partials, ntx, nty);
    count_launches(1);
    sweep3_fixup64<SW_MATVEC><<<kFixBlocks, 256, 0, st>>>(op, x, y, pfix);
  }
  if (nblocks) *nblocks = nb + kFixBlocks;
  return launched();
}

// ---- list of vertices touched by a cell with a surplus record (finest compressed level)
__global__ void touched_mark_kernel(const LevelOp op, uint8_t* __restrict__ flags, int from_xpos) {
  const int N = op.N, n1 = N + 1;
  const long long ncell = (long long)N * N * N;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
       c += (long long)gridDim.x * blockDim.x) {
    const int cx = (int)(c % N), cy = (int)((c / N) % N), cz = (int)(c / ((long long)N * N));
    int ch = cz / op.layers;
    ch = ch < op.nchunk ? ch : op.nchunk - 1;
    const int row = (cz - ch * op.layers) * N + cy;
    const int cls = from_xpos ? (op.xpos[c] >= 0 ? 1 : 0)
                              : op.cmp[ch].cls[((size_t)row * op.nseg_x + (cx >> 5)) * kSegCells + (cx & 31)];
    if (!cls) continue;
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int vx = cx + (a & 1), vy = cy + ((a >> 1) & 1), vz = cz + (a >> 2);
      if (vx > 0 && vx < N && vy > 0 && vy < N && vz > 0 && vz < N) flags[((size_t)vz * n1 + vy) * n1 + vx] = 1;
    }
  }
}

// counts of the touched vertices per 32-vertex group; mask (optional) receives
// the group's bits
__global__ void touched_count_kernel(long long nv, const uint8_t* __restrict__ flags, uint32_t* __restrict__ counts,
                                     uint32_t* __restrict__ mask) {
  const int lane = threadIdx.x & 31;
  const long long ng = (nv + 31) / 32;
  for (long long g = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; g < ng;
       g += ((long long)gridDim.x * blockDim.x) >> 5) {
    const long long v = g * 32 + lane;
    const unsigned m = __ballot_sync(0xffffffffu, v < nv && flags[v]);
    if (lane == 0) {
      counts[g] = __popc(m);
      if (mask) mask[g] = m;
    }
  }
}

// exclusive scan of counts[0..n) in place (one block), total to *total
__global__ void scan1_kernel(long long n, uint32_t* __restrict__ c, int* __restrict__ total) {
  __shared__ uint32_t part[1024];
  const long long per = (n + blockDim.x - 1) / blockDim.x;
  const long long b0 = threadIdx.x * per;
  const long long b1 = b0 + per < n ? b0 + per : n;
  uint32_t sum = 0;
  for (long long i = b0; i < b1; ++i) sum += c[i];
  part[threadIdx.x] = sum;
  __syncthreads();
  for (int off = 1; off < (int)blockDim.x; off <<= 1) {
    const uint32_t v = threadIdx.x >= (unsigned)off ? part[threadIdx.x - off] : 0u;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  uint32_t run = part[threadIdx.x] - sum;
  for (long long i = b0; i < b1; ++i) {
    const uint32_t v = c[i];
    c[i] = run;
    run += v;
  }
  if (threadIdx.x == blockDim.x - 1) *total = (int)part[threadIdx.x];
}

// tile-local exclusive scan of c (2048 entries per block of 1024 threads); tile totals to tot
__global__ void scan_tiles_kernel(long long n, uint32_t* __restrict__ c, uint32_t* __restrict__ tot) {
  __shared__ uint32_t s[2048];
  const long long base = (long long)blockIdx.x * 2048;
  for (int t = threadIdx.x; t < 2048; t += blockDim.x) s[t] = base + t < n ? c[base + t] : 0u;
  __syncthreads();
  // Hillis-Steele over pairs: thread t owns s[2t], s[2t+1]
  const int t = threadIdx.x;
  uint32_t a0 = s[2 * t], a1 = s[2 * t + 1];
  uint32_t own = a0 + a1;
  __shared__ uint32_t ps[1024];
  ps[t] = own;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    const uint32_t v = t >= off ? ps[t - off] : 0u;
    __syncthreads();
    ps[t] += v;
    __syncthreads();
  }
  const uint32_t excl = ps[t] - own;
  if (base + 2 * t < n) c[base + 2 * t] = excl;
  if (base + 2 * t + 1 < n) c[base + 2 * t + 1] = excl + a0;
  if (t == 1023) tot[blockIdx.x] = ps[t];
}

__global__ void scan_add_kernel(long long n, uint32_t* __restrict__ c, const uint32_t* __restrict__ tot) {
  const long long base = (long long)blockIdx.x * 2048;
  const uint32_t add = tot[blockIdx.x];
  for (int t = threadIdx.x; t < 2048; t += blockDim.x)
    if (base + t < n) c[base + t] += add;
}

__global__ void touched_write_kernel(long long nv, const uint8_t* __restrict__ flags,
                                     const uint32_t* __restrict__ base, int* __restrict__ list) {
  const int lane = threadIdx.x & 31;
  const long long ng = (nv + 31) / 32;
  for (long long g = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; g < ng;
       g += ((long long)gridDim.x * blockDim.x) >> 5) {
    const long long v = g * 32 + lane;
    const bool f = v < nv && flags[v];
    const unsigned m = __ballot_sync(0xffffffffu, f);
    if (f) list[base[g] + __popc(m & ((1u << lane) - 1u))] = (int)v;
  }
}

// Zero-iterate damped Jacobi on the finest compressed 3D level, geometric
// part: y = omega b / (h/3 G) with G the sum of eps over the 8 cells at the
// vertex (b and the padded eps rows are the only reads; the fix-up pass
// handles the vertices next to surplus cells).
__global__ void __launch_bounds__(kGeoBX * kGeoBY) sweep3_jacobi0(const LevelOp op, const float* __restrict__ b,
                                                                  float* __restrict__ y, float omega, int ntx,
                                                                  int nty) {
  pdl_begin();
  const int N = op.N, n1 = N + 1;
  const size_t plane = (size_t)n1 * n1;
  const float c0 = omega / (4.f * -op.gk32);   // omega / (h / 3)
  long long w, w1;
  geo_share(ntx, nty, N - 1, w, w1);
  GeoRun run;
  while (next_geo_run(w, w1, N - 1, ntx, run)) {
    const int q = 4 * (run.tx * kGeoBX + threadIdx.x);
    const int j = 1 + run.ty * kGeoBY + threadIdx.y;
    const int k0 = run.k0, k1 = run.k1;
    if (q >= n1 || j >= N) continue;
    const bool hl = q > 0;
    unsigned vmask = 0;
#pragma unroll
    for (int e = 0; e < 4; ++e)
      if (q + e >= 1 && q + e <= N - 1) vmask |= 1u << e;
    float g[2][5], elm[5];
    load_eps10(op.eps_pad, N, k0 - 1, j, q, hl, true, g);
#pragma unroll
    for (int c = 0; c < 5; ++c) elm[c] = g[0][c] + g[1][c];
    for (int k = k0; k <= k1; ++k) {
      load_eps10(op.eps_pad, N, k, j, q, hl, true, g);
      const float4 b4 = __ldg(reinterpret_cast<const float4*>(b + (size_t)k * plane + (size_t)j * n1 + q));
      if (kGeoPF > 0 && k + kGeoPF <= k1) {
        const float* e = op.eps_pad + ((size_t)(k + kGeoPF) * N + j) * n1 + q;
        prefetch_l2(b + (size_t)(k + kGeoPF) * plane + (size_t)j * n1 + q);
        prefetch_l2(e);
        if (threadIdx.y == 0) prefetch_l2(e - n1);
      }
      float ey[5];
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        const float elc = g[0][c] + g[1][c];
        ey[c] = elm[c] + elc;
        elm[c] = elc;
      }
      const float bb[4] = {b4.x, b4.y, b4.z, b4.w};
      float out[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) out[e] = (vmask >> e) & 1u ? __fdividef(c0 * bb[e], ey[e] + ey[e + 1]) : 0.f;
      *reinterpret_cast<float4*>(y + (size_t)k * plane + (size_t)j * n1 + q) = make_float4(out[0], out[1], out[2], out[3]);
    }
  }
}

// pdl = false: launched after its predecessor completes (the fix-up reads x
// and b before its first wait, so it may only overlap a predecessor that
// writes neither)
template <int MODE>
void launch_fixup(const LevelOp& op, const float* x, const float* b, float* y, float omega, double* pfix,
                  cudaStream_t st, bool pdl = true, const float* dq = nullptr) {
  if (!pdl) {
    sweep3_fixup<MODE><<<kFixBlocks, 256, 0, st>>>(op, x, b, y, omega, pfix, dq);
    return;
  }
#if MG_FIX_PDL
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(kFixBlocks);
  cfg.blockDim = dim3(256);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, sweep3_fixup<MODE>, op, x, b, y, omega, pfix, dq);
#else
  sweep3_fixup<MODE><<<kFixBlocks, 256, 0, st>>>(op, x, b, y, omega, pfix, dq);
#endif
}

cudaError_t launch_geo4(const LevelOp& op, int mode, const float* x, const float* b, float* y, float omega,
                        double* partials, int* nblocks, cudaStream_t st) {
  const int nq = (op.N + 1) / 4;
  const int ntx = (nq + kGeoBX - 1) / kGeoBX, nty = (op.N - 1 + kGeoBY - 1) / kGeoBY;
  const long long ntiles = (long long)ntx * nty * (op.N - 1);   // plane steps of 32 x 8 threads
  // persistent grid: the resident blocks of all SMs (two per SM by the launch bounds)
  static int nsm = 0;
  if (!nsm) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (nsm <= 0) nsm = 152;
  }
  const int nb_bulk = ntiles < 2 * nsm ? (int)ntiles : 2 * nsm;
  const dim3 blk(kGeoBX, kGeoBY, 1);
  double* pfix = partials ? partials + 2 * (size_t)nb_bulk : nullptr;
  if (mode == SW_JACOBI0) {
    // a streaming pass at 48 registers: five resident blocks per SM instead of the bulk pass's two
    const int nb0 = ntiles < MG_J0_BLOCKS_PER_SM * nsm ? (int)ntiles : MG_J0_BLOCKS_PER_SM * nsm;
    launch_chain(sweep3_jacobi0, nb0, blk, 0, st, op, b, y, omega, ntx, nty);
    count_launches(1);
    launch_fixup<SW_JACOBI0>(op, x, b, y, omega, pfix, st);
  } else if (mode == SW_JACOBI) {
    if (op.N == 243)
      launch_chain(sweep3_geo4<SW_JACOBI, 243>, nb_bulk, blk, 0, st, op, x, b, y, omega, partials, ntx, nty, nullptr);
    else
      launch_chain(sweep3_geo4<SW_JACOBI, 0>, nb_bulk, blk, 0, st, op, x, b, y, omega, partials, ntx, nty, nullptr);
    count_launches(1);
    launch_fixup<SW_JACOBI>(op, x, b, y, omega, pfix, st);
  } else if (mode == SW_RESID) {
    if (op.N == 243)
      launch_chain(sweep3_geo4<SW_RESID, 243>, nb_bulk, blk, 0, st, op, x, b, y, omega, partials, ntx, nty, nullptr);
    else
      launch_chain(sweep3_geo4<SW_RESID, 0>, nb_bulk, blk, 0, st, op, x, b, y, omega, partials, ntx, nty, nullptr);
    count_launches(1);
    launch_fixup<SW_RESID>(op, x, b, y, omega, pfix, st);
  } else {
    if (op.N == 243)
      launch_chain(sweep3_geo4<SW_MATVEC, 243>, nb_bulk, blk, 0, st, op, x, b, y, omega, partials, ntx, nty, nullptr);
    else
      launch_chain(sweep3_geo4<SW_MATVEC, 0>, nb_bulk, blk, 0, st, op, x, b, y, omega, partials, ntx, nty, nullptr);
    count_launches(1);
    launch_fixup<SW_MATVEC>(op, x, b, y, omega, pfix, st);
  }
  if (nblocks) *nblocks = nb_bulk + kFixBlocks;
  return launched();
}

// 3D FP32 stencil sweep, specialised for the grid sizes of the benchmark's levels
template <int NT>
void launch_stencil3f(const LevelOp& op, int mode, const float* x, const float* b, float* y, float omega,
                      double* partials, dim3 grd, dim3 blk, cudaStream_t st) {
  if (mode == SW_JACOBI0)
    launch_chain(stencil_sweep_kernel<3, float, float, float, SW_JACOBI0, NT>, grd, blk, 0, st, op, x, b, y, omega,
                 partials);
  else if (mode == SW_JACOBI)
    launch_chain(stencil_sweep_kernel<3, float, float, float, SW_JACOBI, NT>, grd, blk, 0, st, op, x, b, y, omega,
                 partials);
  else if (mode == SW_RESID)
    launch_chain(stencil_sweep_kernel<3, float, float, float, SW_RESID, NT>, grd, blk, 0, st, op, x, b, y, omega,
                 partials);
  else
    launch_chain(stencil_sweep_kernel<3, float, float, float, SW_MATVEC, NT>, grd, blk, 0, st, op, x, b, y, omega,
                 partials);
}

void launch_stencil3f_any(const LevelOp& op, int mode, const float* x, const float* b, float* y, float omega,
                          double* partials, dim3 grd, dim3 blk, cudaStream_t st) {
  if (op.N == 27) launch_stencil3f<27>(op, mode, x, b, y, omega, partials, grd, blk, st);
  else if (op.N == 81) launch_stencil3f<81>(op, mode, x, b, y, omega, partials, grd, blk, st);
  else if (op.N == 243) launch_stencil3f<243>(op, mode, x, b, y, omega, partials, grd, blk, st);
  else launch_stencil3f<0>(op, mode, x, b, y, omega, partials, grd, blk, st);
}

template <int D, typename TV, typename TA, typename TS, bool CMP>
cudaError_t sweep_dispatch(const LevelOp& op, int mode, const void* x, const void* b, void* y, double omega,
                           double* partials, int* nblocks, cudaStream_t st) {
  const int ni = op.N - 1;
  const TV* xv = (const TV*)x;
  const TV* bv = (const TV*)b;
  TV* yv = (TV*)y;
  if (D == 3 && CMP && sizeof(TV) == 4 && op.stencil) {   // dense surplus: assembled FP32 stencils
    dim3 blk(kBX, kBY, 1);
    dim3 grd((ni + kBX - 1) / kBX, (ni + kBY - 1) / kBY, ni);
    if (nblocks) *nblocks = (int)(grd.x * grd.y * grd.z);
    launch_stencil3f_any(op, mode, (const float*)x, (const float*)b, (float*)y, (float)omega, partials, grd, blk, st);
    return launched();
  }
  if (D == 3 && CMP && sizeof(TV) == 4 && op.N >= 27 && (op.N + 1) % 4 == 0 && op.touched && op.eps_pad)
    return launch_geo4(op, mode, (const float*)x, (const float*)b, (float*)y, (float)omega, partials, nblocks, st);
  if (D == 3 && CMP && sizeof(TV) == 8 && (mode == SW_RESID || mode == SW_MATVEC) && op.N >= 27 && (op.N + 1) % 4 == 0 && op.touched)
    return launch_geo64(op, mode, (const double*)x, (const double*)b, (double*)y, partials, nblocks, st);
  if (!CMP && op.stencil) {
    dim3 blk(kBX, kBY, 1);
    dim3 grd((ni + kBX - 1) / kBX, (ni + kBY - 1) / kBY, D == 3 ? ni : 1);
    if (nblocks) *nblocks = (int)(grd.x * grd.y * grd.z);
    if (D == 3 && sizeof(TV) == 4 && sizeof(TA) == 4 && sizeof(TS) == 4) {
      launch_stencil3f_any(op, mode, (const float*)x, (const float*)b, (float*)y, (float)omega, partials, grd, blk,
                           st);
      return launched();
    }
    if (mode == SW_JACOBI0)
      launch_chain(stencil_sweep_kernel<D, TV, TA, TS, SW_JACOBI0>, grd, blk, 0, st, op, xv, bv, yv, (TA)omega, partials);
    else if (mode == SW_JACOBI)
      launch_chain(stencil_sweep_kernel<D, TV, TA, TS, SW_JACOBI>, grd, blk, 0, st, op, xv, bv, yv, (TA)omega, partials);
    else if (mode == SW_RESID)
      launch_chain(stencil_sweep_kernel<D, TV, TA, TS, SW_RESID>, grd, blk, 0, st, op, xv, bv, yv, (TA)omega, partials);
    else
      launch_chain(stencil_sweep_kernel<D, TV, TA, TS, SW_MATVEC>, grd, blk, 0, st, op, xv, bv, yv, (TA)omega, partials);
    return launched();
  }
  // the plane-streaming kernel needs enough (x, y, z-run) tiles to fill the GPU;
  // smaller grids run one vertex per thread
  if (D == 3 && op.N >= 243) {
    if (mode == SW_JACOBI0) return cudaErrorNotSupported;
    dim3 blk(kTX, kTY, 1);
    dim3 grd((ni + kTX - 1) / kTX, (ni + kTY - 1) / kTY, (ni + kZC - 1) / kZC);
    if (nblocks) *nblocks = (int)(grd.x * grd.y * grd.z);
    if (mode == SW_JACOBI)
      sweep3_stream<TV, TA, TS, SW_JACOBI, CMP><<<grd, blk, 0, st>>>(op, xv, bv, yv, (TA)omega, partials);
    else if (mode == SW_RESID)
      sweep3_stream<TV, TA, TS, SW_RESID, CMP><<<grd, blk, 0, st>>>(op, xv, bv, yv, (TA)omega, partials);
    else
      sweep3_stream<TV, TA, TS, SW_MATVEC, CMP><<<grd, blk, 0, st>>>(op, xv, bv, yv, (TA)omega, partials);
    return launched();
  }
  dim3 blk(kBX, kBY, 1);
  dim3 grd((ni + kBX - 1) / kBX, (ni + kBY - 1) / kBY, D == 3 ? ni : 1);
  if (nblocks) *nblocks = (int)(grd.x * grd.y * grd.z);
  if (mode == SW_JACOBI0)
    sweep_kernel<D, TV, TA, TS, SW_JACOBI0, CMP><<<grd, blk, 0, st>>>(op, xv, bv, yv, (TA)omega, partials);
  else if (mode == SW_JACOBI)
    sweep_kernel<D, TV, TA, TS, SW_JACOBI, CMP><<<grd, blk, 0, st>>>(op, xv, bv, yv, (TA)omega, partials);
  else if (mode == SW_RESID)
    sweep_kernel<D, TV, TA, TS, SW_RESID, CMP><<<grd, blk, 0, st>>>(op, xv, bv, yv, (TA)omega, partials);
  else
    sweep_kernel<D, TV, TA, TS, SW_MATVEC, CMP><<<grd, blk, 0, st>>>(op, xv, bv, yv, (TA)omega, partials);
  return launched();
}

// ---------------------------------------------------------------- transfers
// b_c(I) = sum_{|delta| <= 2} prod_a w(delta_a) r_f(3 I + delta),
// w(d) = 1 - |d| / 3   (R = P^T).
//
// Tiled and separable: a block owns kRTX x kRTY coarse vertices (I, J).  Per
// input plane it stages the tile's fine region (x from 3 I0 - 2 to 3 I1 + 2,
// rows 3 J0 - 2 to 3 J1 + 2) in shared memory with asynchronous copies (the
// next plane's copies fly while the current plane is restricted), restricts
// it along x (one entry per fine row and coarse column), then along y (one
// coarse vertex per thread).  In 3D a block marches over the fine planes
// 3 K0 - 2 .. 3 K1 + 2 of its chunk of coarse planes K0 .. K1: fine plane
// k = 3 c + m adds w(m) = 1 - m/3 of its x-y restriction to coarse plane c
// and m/3 to plane c + 1, and plane c is complete after k = 3 c + 2.
// Neighbouring chunks share two fine planes (the second read mostly hits L2).
constexpr int kRTX = 32, kRTY = 8;
constexpr int kRFX = 3 * kRTX + 2;   // fine columns of a tile
constexpr int kRFY = 3 * kRTY + 2;   // fine rows of a tile
constexpr int kRFP = 3 * kRTX + 4;   // padded row: 16-byte aligned rows, whole 4-element groups

// S staged input planes: S - 1 planes of copies are in flight while one is
// restricted (four for FP32 in 45 KB; two for FP64)
template <typename TV, int S>
struct __align__(16) RTile {
  TV f[S][kRFY][kRFP];
  TV rx[kRFY][kRTX];   // restricted along x
};

// asynchronous copy of B (4, 8 or 16) bytes global -> shared, both sides
// B-aligned; zero fill when !valid (nothing is read)
template <int B>
__device__ __forceinline__ void cp_async_bytes(void* dst, const void* src, bool valid) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
  const unsigned n = valid ? (unsigned)B : 0u;
  if (B == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(src), "r"(n) : "memory");
  else if (B == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(sa), "l"(src), "r"(n) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(src), "r"(n) : "memory");
}

// issues (and commits as one group) the copies of the tile at (I0, J0) of the
// input plane starting at src + zbase.  A row's window starts at the fine x
// xs = (3 I0 - 2) rounded down to a multiple of 4 elements and holds kRFP
// elements (the tile's columns sit at offset (3 I0 - 2) - xs); it is copied in
// the widest pieces its global alignment allows (row starts are 16-byte
// aligned only when (N + 1) is a multiple of the elements per 16 bytes).
// Rows past the last interior row N - 1 and pieces starting past x = N are
// zero filled; the other pieces may read the boundary vertex x = N and the
// start of the next row (inside the array, since the row is at most N - 1):
// only coarse vertices outside the grid use those entries.
template <typename TV>
__device__ __forceinline__ void rtile_stage(TV (&f)[kRFY][kRFP], const TV* __restrict__ src, int N, long long zbase,
                                            int I0, int J0) {
  const int nf1 = N + 1, xs = (3 * I0 - 2) & ~3, y0 = 3 * J0 - 2;
  constexpr int E = 16 / sizeof(TV), NQ = kRFP / E;   // 16-byte pieces per row
  if (nf1 % E == 0) {
    // every row start is 16-byte aligned: the block's threads take the
    // (row, piece) pairs of the tile in turn
    const TV* g0 = src + zbase + (long long)y0 * nf1 + xs;
    const int tid = threadIdx.y * kRTX + threadIdx.x;
#pragma unroll
    for (int it = 0; it < (kRFY * NQ + kRTX * kRTY - 1) / (kRTX * kRTY); ++it) {
      const int e = tid + it * kRTX * kRTY;
      if (e >= kRFY * NQ) break;
      const int r = e / NQ, q = e - r * NQ;
      cp_async_bytes<16>(&f[r][E * q], g0 + r * nf1 + E * q, y0 + r <= N - 1 && xs + E * q <= N);
    }
    cp_async_commit();
    return;
  }
#pragma unroll
  for (int rr = 0; rr < (kRFY + kRTY - 1) / kRTY; ++rr) {
    const int r = threadIdx.y + rr * kRTY;   // warp-uniform
    if (r >= kRFY) break;
    const int y = y0 + r;
    const TV* g = src + zbase + (long long)y * nf1 + xs;
    const unsigned al = (unsigned)((uintptr_t)g & 15);
    if (al == 0) {
      constexpr int E = 16 / sizeof(TV);
      for (int q = threadIdx.x; q < kRFP / E; q += kRTX)
        cp_async_bytes<16>(&f[r][E * q], g + E * q, y <= N - 1 && xs + E * q <= N);
    } else if ((al & 7) == 0) {
      constexpr int E = 8 / sizeof(TV);
      for (int q = threadIdx.x; q < kRFP / E; q += kRTX)
        cp_async_bytes<8>(&f[r][E * q], g + E * q, y <= N - 1 && xs + E * q <= N);
    } else {
      for (int q = threadIdx.x; q < kRFP; q += kRTX)
        cp_async_bytes<4>(&f[r][q], g + q, y <= N - 1 && xs + q <= N);
    }
  }
  cp_async_commit();
}

// x-y restriction of a staged tile whose copies have landed and are visible
// to the block; one barrier between the x and the y pass.  Returns the value
// of coarse vertex (I0 + threadIdx.x, J0 + threadIdx.y).
template <typename TV>
__device__ __forceinline__ TV rtile_xy(const TV (&f)[kRFY][kRFP], TV (&rx)[kRFY][kRTX]) {
  const TV wa = (TV)(1.0 / 3.0), wb = (TV)(2.0 / 3.0);
  // x pass: a thread takes four consecutive coarse columns 4t .. 4t + 3 of one
  // row, whose windows o + 3k .. o + 3k + 4 (o = (3 I0 - 2) mod 4, 1 for
  // tiles of 32 columns) lie in the 16 staged values 12t .. 12t + 15 (read as
  // 16-byte vectors)
  const int tid = threadIdx.y * kRTX + threadIdx.x;
  if (tid < kRFY * (kRTX / 4)) {
    const int r = tid / (kRTX / 4), t = tid - r * (kRTX / 4);
    TV v[16];
    if constexpr (sizeof(TV) == 4) {
      const float4* p = reinterpret_cast<const float4*>(&f[r][12 * t]);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float4 a = p[q];
        v[4 * q] = a.x;
        v[4 * q + 1] = a.y;
        v[4 * q + 2] = a.z;
        v[4 * q + 3] = a.w;
      }
    } else {
      const double2* p = reinterpret_cast<const double2*>(&f[r][12 * t]);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const double2 a = p[q];
        v[2 * q] = a.x;
        v[2 * q + 1] = a.y;
      }
    }
    constexpr int o = (3 * 1 - 2) & 3;   // the same for every tile: 3 I0 - 2 = 1 + 3 kRTX m
    static_assert((3 * kRTX) % 4 == 0, "tile origins must share the offset o");
#pragma unroll
    for (int k = 0; k < 4; ++k)
      rx[r][4 * t + k] = wa * v[o + 3 * k] + wb * v[o + 3 * k + 1] + v[o + 3 * k + 2] + wb * v[o + 3 * k + 3] +
                         wa * v[o + 3 * k + 4];
  }
  __syncthreads();
  const TV* q = &rx[3 * threadIdx.y][threadIdx.x];
  return wa * q[0] + wb * q[kRTX] + q[2 * kRTX] + wb * q[3 * kRTX] + wa * q[4 * kRTX];
}

// TIN = false: the input is the fine vector; the fine planes 3 K0 - 2 ..
// 3 K1 + 2 are marched and weighted along z.  TIN = true: the input is the
// z-restricted residual planes of the fused residual + restriction, input
// plane K is coarse plane K.
// With diag (the coarse level's stencil diagonals), also u1 = omega b_c / diag:
// the coarse V-cycle's first smoothing step from the zero iterate.
template <typename TV, bool TIN>
__global__ void __launch_bounds__(kRTX * kRTY) restrict3_tile_kernel(int Nc, int kchunk, const TV* __restrict__ src,
                                                                     TV* __restrict__ bc, const TV* __restrict__ diag,
                                                                     TV omega, TV* __restrict__ u1) {
  pdl_begin();
  constexpr int S = sizeof(TV) == 4 ? 4 : 2;
  __shared__ RTile<TV, S> s;
  const int N = 3 * Nc, nf1 = N + 1, nc1 = Nc + 1;
  const long long plane = (long long)nf1 * nf1;
  const int I0 = 1 + blockIdx.x * kRTX, J0 = 1 + blockIdx.y * kRTY;
  const int K0 = 1 + blockIdx.z * kchunk, K1 = min(Nc - 1, K0 + kchunk - 1);
  const int I = I0 + threadIdx.x, J = J0 + threadIdx.y;
  const bool valid = I <= Nc - 1 && J <= Nc - 1;
  const TV wa = (TV)(1.0 / 3.0), wb = (TV)(2.0 / 3.0);
  const int p0 = TIN ? K0 : 3 * K0 - 2, p1 = TIN ? K1 : 3 * K1 + 2;
  TV acc0 = 0, acc1 = 0;   // coarse planes c and c + 1
  // one commit group per plane (empty past the last plane), so that waiting
  // for all but the newest S - 1 groups waits for the current plane
#pragma unroll
  for (int q = 0; q < S - 1; ++q) {
    if (p0 + q <= p1) rtile_stage<TV>(s.f[q], src, N, (long long)(p0 + q) * plane, I0, J0);
    else cp_async_commit();
  }
  for (int p = p0; p <= p1; ++p) {
    const int i = p - p0;
    // buffer (i + S - 1) % S was last read by the x pass of plane p - 1,
    // which every thread finished before that plane's second barrier
    if (p + S - 1 <= p1) rtile_stage<TV>(s.f[(i + S - 1) % S], src, N, (long long)(p + S - 1) * plane, I0, J0);
    else cp_async_commit();
    cp_async_wait<S - 1>();
    __syncthreads();
    const TV v = rtile_xy(s.f[i % S], s.rx);
    if (TIN) {
      if (valid) {
        const long long o = ((long long)p * nc1 + J) * nc1 + I;
        bc[o] = v;
        if (diag) u1[o] = omega * v / __ldg(diag + o);
      }
      continue;
    }
    const int c = p / 3, m = p - 3 * c;
    if (m == 0) {
      acc0 += v;
    } else if (m == 1) {
      acc0 += wb * v;
      acc1 += wa * v;
    } else {
      acc0 += wa * v;
      acc1 += wb * v;
      if (c >= K0 && valid) {
        const long long o = ((long long)c * nc1 + J) * nc1 + I;
        bc[o] = acc0;
        if (diag) u1[o] = omega * acc0 / __ldg(diag + o);
      }
      acc0 = acc1;
      acc1 = 0;
    }
  }
}

template <typename TV>
__global__ void __launch_bounds__(kRTX * kRTY) restrict2_tile_kernel(int Nc, const TV* __restrict__ rf,
                                                                     TV* __restrict__ bc, const TV* __restrict__ diag,
                                                                     TV omega, TV* __restrict__ u1) {
  pdl_begin();
  __shared__ RTile<TV, 1> s;
  const int N = 3 * Nc, nc1 = Nc + 1;
  const int I0 = 1 + blockIdx.x * kRTX, J0 = 1 + blockIdx.y * kRTY;
  const int I = I0 + threadIdx.x, J = J0 + threadIdx.y;
  rtile_stage<TV>(s.f[0], rf, N, 0, I0, J0);
  cp_async_wait<0>();
  __syncthreads();
  const TV v = rtile_xy(s.f[0], s.rx);
  if (I <= Nc - 1 && J <= Nc - 1) {
    const long long o = (long long)J * nc1 + I;
    bc[o] = v;
    if (diag) u1[o] = omega * v / __ldg(diag + o);
  }
}

// b_c = I r_f: interior coarse vertices take the fine value at the coinciding
// vertex (the restriction of adaFAC-PI's auxiliary equation)
template <int D, typename TV>
__global__ void inject_kernel(int Nc, const TV* __restrict__ rf, TV* __restrict__ bc) {
  const int nc1 = Nc + 1, nf1 = 3 * Nc + 1;
  long long ni = 1;
  for (int a = 0; a < D; ++a) ni *= (Nc - 1);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < ni;
       t += (long long)gridDim.x * blockDim.x) {
    const int I = 1 + (int)(t % (Nc - 1));
    const int J = 1 + (int)((t / (Nc - 1)) % (Nc - 1));
    const int K = D == 3 ? 1 + (int)(t / ((long long)(Nc - 1) * (Nc - 1))) : 0;
    const long long vc = D == 3 ? ((long long)K * nc1 + J) * nc1 + I : (long long)J * nc1 + I;
    const long long vf = D == 3 ? ((long long)(3 * K) * nf1 + 3 * J) * nf1 + 3 * I : (long long)(3 * J) * nf1 + 3 * I;
    bc[vc] = rf[vf];
  }
}

// e_f += P e_c (d-linear interpolation on the 3:1 refined grid)
template <int D, typename TV>
__global__ void prolong_kernel(int Nc, const TV* __restrict__ ec, TV* __restrict__ ef) {
  pdl_begin();
  // one thread per interior fine vertex: x from the block's x range, y from
  // blockIdx.y/threadIdx.y, z from blockIdx.z (3D)
  const int nc1 = Nc + 1, Nf = 3 * Nc, nf1 = Nf + 1;
  int f[3];
  f[0] = 1 + blockIdx.x * blockDim.x + threadIdx.x;
  f[1] = 1 + blockIdx.y * blockDim.y + threadIdx.y;
  f[2] = D == 3 ? 1 + blockIdx.z : 0;
  if (f[0] >= Nf || f[1] >= Nf) return;
  int c0[3] = {0, 0, 0};
  TV w0[3] = {1, 1, 1}, w1[3] = {0, 0, 0};
#pragma unroll
  for (int a = 0; a < D; ++a) {
    c0[a] = f[a] / 3;
    const int r = f[a] - 3 * c0[a];
    w1[a] = (TV)r * (TV)(1.0 / 3.0);
    w0[a] = (TV)1 - w1[a];
  }
  TV acc = 0;
#pragma unroll
  for (int corner = 0; corner < (1 << D); ++corner) {
    TV w = 1;
    int cv[3] = {0, 0, 0};
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const int up = (corner >> a) & 1;
      w *= up ? w1[a] : w0[a];
      cv[a] = c0[a] + up;
    }
    if (w != (TV)0) {
      const int vc = D == 3 ? (cv[2] * nc1 + cv[1]) * nc1 + cv[0] : cv[1] * nc1 + cv[0];
      acc += w * __ldg(ec + vc);
    }
  }
  const size_t vf = D == 3 ? ((size_t)f[2] * nf1 + f[1]) * nf1 + f[0] : (size_t)f[1] * nf1 + f[0];
  ef[vf] += acc;
}

// 3D FP32 prolongation with 4 consecutive fine x-vertices per thread (rows of
// (3 Nc + 1) % 4 == 0 floats): the 2 x 2 coarse (y, z) neighbours are first
// combined for the 3 coarse columns the quad spans, then interpolated along x;
// one float4 read-modify-write per thread.  Fine boundary vertices in x get
// P e_c = 0 added (the coarse boundary values are zero).
__global__ void prolong3_x4_kernel(int Nc, const float* __restrict__ ec, float* __restrict__ ef) {
  pdl_begin();
  const int nc1 = Nc + 1, Nf = 3 * Nc, nf1 = Nf + 1;
  const int q = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
  const int fy = 1 + blockIdx.y * blockDim.y + threadIdx.y;
  const int fz = 1 + blockIdx.z;
  if (q >= nf1 || fy >= Nf) return;
  const int cy = fy / 3, cz = fz / 3;
  const float wy1 = (float)(fy - 3 * cy) * (1.f / 3.f), wz1 = (float)(fz - 3 * cz) * (1.f / 3.f);
  const float wy0 = 1.f - wy1, wz0 = 1.f - wz1;
  const int cx0 = q / 3;
  float V[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int cx = min(cx0 + c, Nc);
    const float* e = ec + ((size_t)cz * nc1 + cy) * nc1 + cx;
    const float a00 = __ldg(e), a01 = __ldg(e + nc1), a10 = __ldg(e + (size_t)nc1 * nc1),
                a11 = __ldg(e + (size_t)nc1 * nc1 + nc1);
    V[c] = wz0 * (wy0 * a00 + wy1 * a01) + wz1 * (wy0 * a10 + wy1 * a11);
  }
  float4* dst = reinterpret_cast<float4*>(ef + ((size_t)fz * nf1 + fy) * nf1 + q);
  float4 o = *dst;
  float add[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int x = q + e, cx = x / 3, r = x - 3 * cx;
    const int jx = cx - cx0;
    const float w1 = (float)r * (1.f / 3.f);
    add[e] = (1.f - w1) * (jx == 0 ? V[0] : V[1]) + w1 * (jx == 0 ? V[1] : V[2]);
  }
  o.x += add[0];
  o.y += add[1];
  o.z += add[2];
  o.w += add[3];
  *dst = o;
}

// ---------------------------------------------------------------- V-cycle tail in one block
// The two coarsest levels of an FP32 V-cycle (N = 9 with its assembled
// stencils, and the 3^d-cell coarsest level solved with its precomputed
// inverse) in a single block, everything in shared memory: pre-smoothing
// from the zero iterate, residual, restriction, coarse solve, prolongation
// and post-smoothing, the same steps and arithmetic as the per-level kernels,
// without their launch latencies.  One thread per interior vertex.
constexpr int kTailN = 9;
constexpr int kTailThreads = 512;

template <int D>
struct TailDims {
  static constexpr int n1 = kTailN + 1;
  static constexpr int nv = D == 3 ? n1 * n1 * n1 : n1 * n1;
  static constexpr int NS = D == 3 ? 14 : 5;   // symmetric storage: diagonal + forward couplings
  static constexpr int ni = kTailN - 1;
  static constexpr int nint = D == 3 ? ni * ni * ni : ni * ni;
  static constexpr int nc = D == 3 ? 8 : 4;    // interior vertices of the coarsest level
};

template <int D>
constexpr int tail_smem_bytes() {
  return (TailDims<D>::NS + 4) * TailDims<D>::nv * (int)sizeof(float);
}

template <int D>
__global__ void __launch_bounds__(kTailThreads) vcycle_tail_kernel(const float* __restrict__ stencil,
                                                                   const float* __restrict__ b,
                                                                   float* __restrict__ xout,
                                                                   const double* __restrict__ Ainv, float omega,
                                                                   int nu_pre, int nu_post) {
  pdl_begin();
  using T = TailDims<D>;
  constexpr int n1 = T::n1, nv = T::nv, NS = T::NS, C = D == 3 ? 13 : 4;   // C: centre of the 3^d block
  extern __shared__ float tail_smem[];
  float* S = tail_smem;            // [NS][nv]
  float* xa = S + NS * nv;
  float* xb = xa + nv;
  float* bs = xb + nv;
  float* rs = bs + nv;
  __shared__ float bc[T::nc], ec[D == 3 ? 64 : 16];   // coarsest rhs; coarsest iterate on its 4^d grid
  const int t = threadIdx.x;
  for (int i = t; i < NS * nv; i += blockDim.x) S[i] = __ldg(stencil + i);
  for (int i = t; i < nv; i += blockDim.x) {
    bs[i] = __ldg(b + i);
    xa[i] = 0.f;
    xb[i] = 0.f;
  }
  for (int i = t; i < (D == 3 ? 64 : 16); i += blockDim.x) ec[i] = 0.f;
  __syncthreads();
  // this thread's interior vertex
  const bool act = t < T::nint;
  int vi = 1 + t % T::ni, vj = 1 + (t / T::ni) % T::ni, vk = D == 3 ? 1 + t / (T::ni * T::ni) : 0;
  const int v = act ? (D == 3 ? (vk * n1 + vj) * n1 + vi : vj * n1 + vi) : 0;
  auto apply = [&](const float* x) -> float {   // sum_q c_q (x_q - x_v)
    const float xv = x[v];
    float acc = 0.f;
#pragma unroll
    for (int dz = 0; dz < (D == 3 ? 3 : 1); ++dz)
#pragma unroll
      for (int dy = 0; dy < 3; ++dy)
#pragma unroll
        for (int dx = 0; dx < 3; ++dx) {
          const int q = dx + 3 * dy + 9 * dz;
          if (q == C) continue;
          const int nb = v + (dx - 1) + (dy - 1) * n1 + (D == 3 ? (dz - 1) * n1 * n1 : 0);
          const float cq = q > C ? S[(q - C) * nv + v] : S[(C - q) * nv + nb];
          acc += cq * (x[nb] - xv);
        }
    return acc;
  };
  float* cur = xa;
  float* oth = xb;
  // pre-smoothing: omega D^-1 b from the zero iterate, then damped Jacobi
  if (nu_pre > 0) {
    if (act) cur[v] = omega * bs[v] / S[v];
    __syncthreads();
  }
  for (int k = 1; k < nu_pre; ++k) {
    if (act) oth[v] = cur[v] + omega * (bs[v] - apply(cur)) / S[v];
    __syncthreads();
    float* tmp = cur;
    cur = oth;
    oth = tmp;
  }
  // residual, restricted to the coarsest level (R = P^T, 1D weights 1/3, 2/3, 1, 2/3, 1/3)
  if (act) rs[v] = bs[v] - apply(cur);   // (boundary entries of rs are never read)
  __syncthreads();
  if (t < T::nc) {
    const int I = 1 + (t & 1), J = 1 + ((t >> 1) & 1), K = D == 3 ? 1 + ((t >> 2) & 1) : 0;
    const float w1[5] = {1.f / 3.f, 2.f / 3.f, 1.f, 2.f / 3.f, 1.f / 3.f};
    float acc = 0.f;
    for (int dz = (D == 3 ? -2 : 0); dz <= (D == 3 ? 2 : 0); ++dz)
      for (int dy = -2; dy <= 2; ++dy)
        for (int dx = -2; dx <= 2; ++dx) {
          const int fx = 3 * I + dx, fy = 3 * J + dy, fz = 3 * K + dz;
          const bool inner = fx >= 1 && fx <= kTailN - 1 && fy >= 1 && fy <= kTailN - 1 &&
                             (D == 2 || (fz >= 1 && fz <= kTailN - 1));
          const float val = inner ? rs[D == 3 ? (fz * n1 + fy) * n1 + fx : fy * n1 + fx] : 0.f;
          acc += w1[dx + 2] * w1[dy + 2] * (D == 3 ? w1[dz + 2] : 1.f) * val;
        }
    bc[t] = acc;
  }
  __syncthreads();
  // coarsest solve with the precomputed inverse (FP64 accumulation)
  if (t < T::nc) {
    double z = 0.0;
    for (int k = 0; k < T::nc; ++k) z += Ainv[t * T::nc + k] * (double)bc[k];
    const int I = 1 + (t & 1), J = 1 + ((t >> 1) & 1), K = D == 3 ? 1 + ((t >> 2) & 1) : 0;
    ec[D == 3 ? (K * 4 + J) * 4 + I : J * 4 + I] = (float)z;
  }
  __syncthreads();
  // prolongation (d-linear, 3:1)
  if (act) {
    int f[3] = {vi, vj, vk}, c0[3] = {0, 0, 0};
    float w0[3] = {1.f, 1.f, 1.f}, w1[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int a = 0; a < D; ++a) {
      c0[a] = f[a] / 3;
      w1[a] = (float)(f[a] - 3 * c0[a]) * (1.f / 3.f);
      w0[a] = 1.f - w1[a];
    }
    float acc = 0.f;
#pragma unroll
    for (int corner = 0; corner < (1 << D); ++corner) {
      float w = 1.f;
      int cv[3] = {0, 0, 0};
#pragma unroll
      for (int a = 0; a < D; ++a) {
        const int up = (corner >> a) & 1;
        w *= up ? w1[a] : w0[a];
        cv[a] = c0[a] + up;
      }
      acc += w * ec[D == 3 ? (cv[2] * 4 + cv[1]) * 4 + cv[0] : cv[1] * 4 + cv[0]];
    }
    cur[v] += acc;
  }
  __syncthreads();
  for (int k = 0; k < nu_post; ++k) {
    if (act) oth[v] = cur[v] + omega * (bs[v] - apply(cur)) / S[v];
    __syncthreads();
    float* tmp = cur;
    cur = oth;
    oth = tmp;
  }
  for (int i = t; i < nv; i += blockDim.x) xout[i] = cur[i];
}

int vgrid(long long n) {
  long long b = (n + 255) / 256;
  if (b > 152LL * 32) b = 152LL * 32;
  if (b < 1) b = 1;
  return (int)b;
}

// ---------------------------------------------------------------- vector kernels
constexpr int kRedBlocks = 152 * 8;

__device__ __forceinline__ bool aligned16(const void* p) { return ((uintptr_t)p & 15) == 0; }

// FP32 dot product: float4 body when both operands are 16-byte aligned, scalar tail
__global__ void dot4_kernel(const float* __restrict__ a, const float* __restrict__ b, long long n,
                            double* partials) {
  pdl_begin();
  __shared__ double sh[8];
  float acc = 0.f;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long n4 = 0;
  if (aligned16(a) && aligned16(b)) {
    n4 = n / 4;
    const float4* a4 = reinterpret_cast<const float4*>(a);
    const float4* b4 = reinterpret_cast<const float4*>(b);
    for (long long t = t0; t < n4; t += stride) {
      const float4 x = __ldg(a4 + t), y = __ldg(b4 + t);
      acc += x.x * y.x + x.y * y.y + x.z * y.z + x.w * y.w;
    }
  }
  for (long long t = 4 * n4 + t0; t < n; t += stride) acc += a[t] * b[t];
  const double s = block_sum((double)acc, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

template <typename TA, typename TB>
__global__ void dot_kernel(const TA* __restrict__ a, const TB* __restrict__ b, long long n, double* partials) {
  // FP32 operands accumulate per thread in FP32 (about a hundred terms), FP64 otherwise
  typedef typename std::conditional<sizeof(TA) == 4 && sizeof(TB) == 4, float, double>::type Acc;
  __shared__ double sh[8];
  Acc acc = 0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    acc += (Acc)a[t] * (Acc)b[t];
  const double s = block_sum((double)acc, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__device__ __forceinline__ void scalar_op(DevScalars* sc, int op) {
  if (op == SC_SET_BETA) sc->beta = sc->pq != 0.0 ? -sc->zq / sc->pq : 0.0;
  else if (op == SC_SET_ALPHA) sc->alpha = sc->pq != 0.0 ? sc->pr / sc->pq : 0.0;
}

// out[c] = sum of the partials of component c; then (sc != nullptr) the
// scalar update op that reads them
__global__ void reduce_finish_kernel(const double* __restrict__ partials, int nblocks, int ncomp, double* out,
                                     DevScalars* sc, int op) {
  pdl_begin();
  __shared__ double sh[32];
  for (int c = 0; c < ncomp; ++c) {
    double acc = 0.0;
    for (int t = threadIdx.x; t < nblocks; t += blockDim.x) acc += partials[(long long)t * ncomp + c];
    const double s = block_sum(acc, sh);
    if (threadIdx.x == 0) out[c] = s;
    __syncthreads();
  }
  if (sc && threadIdx.x == 0) scalar_op(sc, op);
}

__global__ void scalar_kernel(DevScalars* sc, int op) { scalar_op(sc, op); }

template <typename TZ>
__global__ void fcg_direction_kernel(long long n, int first, const TZ* __restrict__ z, double* __restrict__ p,
                                     const DevScalars* __restrict__ sc) {
  const double beta = first ? 0.0 : sc->beta;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    p[t] = (double)z[t] + (first ? 0.0 : beta * p[t]);
}

template <typename TR>
__global__ void fcg_update_kernel(long long n, double* __restrict__ u, double* __restrict__ r,
                                  const double* __restrict__ p, const double* __restrict__ q,
                                  const DevScalars* __restrict__ sc, TR* __restrict__ rin, double* partials) {
  __shared__ double sh[8];
  const double alpha = sc->alpha;
  double acc = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    u[t] += alpha * p[t];
    const double rv = r[t] - alpha * q[t];
    r[t] = rv;
    if (rin) rin[t] = (TR)rv;
    acc += rv * rv;
  }
  const double s = block_sum(acc, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

template <typename TZ>
__global__ void richardson_kernel(long long n, double* __restrict__ u, const TZ* __restrict__ z) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    u[t] += (double)z[t];
}

template <typename TS, typename TD>
__global__ void convert_kernel(long long n, const TS* __restrict__ s, TD* __restrict__ d) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    d[t] = (TD)s[t];
}

template <int D>
__global__ void load_vector_kernel(int N, double val, double* f) {
  const int n1 = N + 1;
  long long nv = 1;
  for (int a = 0; a < D; ++a) nv *= n1;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nv; t += (long long)gridDim.x * blockDim.x) {
    long long r = t;
    bool inside = true;
    for (int a = 0; a < D; ++a) {
      const int c = (int)(r % n1);
      r /= n1;
      inside = inside && c > 0 && c < N;
    }
    f[t] = inside ? val : 0.0;
  }
}

}  // namespace

bool pdl_enabled() { return getenv("MG_NO_PDL") == nullptr; }

cudaError_t launch_geo_weights64(const LevelOp& op, double* const w[4], double* es, cudaStream_t st) {
  geo_weights64_kernel<<<152 * 8, 256, 0, st>>>(op.N, op.eps64, op.eps_c, -op.gk64, w[0], w[1], w[2], w[3], es);
  count_launches(1);
  return launched();
}

// y = x + omega D^-1 (b - A x) and partials[...] of y . dq on a split finest
// level (bulk pass: one partial per block, then one per fix-up block);
// cudaErrorNotSupported (nothing launched) elsewhere
cudaError_t launch_jacobi_dot(const LevelOp& op, const float* x, const float* b, float* y, float omega,
                              const float* dq, double* partials, int* nblocks, cudaStream_t st) {
  if (op.dim != 3 || !op.compressed || op.stencil || !op.touched || !op.tmask || !op.eps_pad || op.N < 27 ||
      (op.N + 1) % 4 != 0 || !dq || !partials)
    return cudaErrorNotSupported;
  const int nq = (op.N + 1) / 4;
  const int ntx = (nq + kGeoBX - 1) / kGeoBX, nty = (op.N - 1 + kGeoBY - 1) / kGeoBY;
  const long long ntiles = (long long)ntx * nty * (op.N - 1);
  static int nsm = 0;
  if (!nsm) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (nsm <= 0) nsm = 152;
  }
  const int nb_bulk = ntiles < 2 * nsm ? (int)ntiles : 2 * nsm;
  const dim3 blk(kGeoBX, kGeoBY, 1);
  float* dqf = const_cast<float*>(dq);   // read only (passed in the zr slot)
  if (op.N == 243)
    launch_chain(sweep3_geo4<SW_JACOBI_DOT, 243>, nb_bulk, blk, 0, st, op, x, b, y, omega, partials, ntx, nty, dqf);
  else
    launch_chain(sweep3_geo4<SW_JACOBI_DOT, 0>, nb_bulk, blk, 0, st, op, x, b, y, omega, partials, ntx, nty, dqf);
  count_launches(1);
  launch_fixup<SW_JACOBI_DOT>(op, x, b, y, omega, partials + nb_bulk, st, true, dq);
  *nblocks = nb_bulk + kFixBlocks;
  return launched();
}

bool vcycle_tail_supported(const LevelOp& op) {
  return op.N == kTailN && !op.compressed && !op.elem64 && op.stencil != nullptr;
}

cudaError_t launch_vcycle_tail(const LevelOp& op, const double* Lc, const float* b, float* x, float omega,
                               int nu_pre, int nu_post, cudaStream_t st) {
  if (!vcycle_tail_supported(op)) return cudaErrorNotSupported;
  const int n = op.dim == 3 ? 8 : 4;
  if (op.dim == 3) {
    static const cudaError_t attr = cudaFuncSetAttribute(
        vcycle_tail_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, tail_smem_bytes<3>());
    if (attr != cudaSuccess) return attr;
    launch_chain(vcycle_tail_kernel<3>, 1, kTailThreads, tail_smem_bytes<3>(), st, (const float*)op.stencil, b, x, Lc + n * n,
                                                                          omega, nu_pre, nu_post);
  } else {
    launch_chain(vcycle_tail_kernel<2>, 1, kTailThreads, tail_smem_bytes<2>(), st, (const float*)op.stencil, b, x, Lc + n * n,
                                                                          omega, nu_pre, nu_post);
  }
  return launched();
}


cudaError_t launch_sweep(const LevelOp& op, int mode, int vec64, const void* x, const void* b, void* y,
                         double omega, double* partials, int* nblocks, cudaStream_t st) {
  if (op.N < 2) return cudaErrorInvalidValue;
  // arithmetic: FP64 when the vectors are FP64, FP32 otherwise
#define MG_SW(D, TV, TA, TS, CMP) \
  return sweep_dispatch<D, TV, TA, TS, CMP>(op, mode, x, b, y, omega, partials, nblocks, st)
  if (op.dim == 2) {
    if (op.compressed) {
      if (vec64) MG_SW(2, double, double, float, true);
      MG_SW(2, float, float, float, true);
    }
    if (vec64) {
      if (op.elem64) MG_SW(2, double, double, double, false);
      MG_SW(2, double, double, float, false);
    }
    if (op.elem64) MG_SW(2, float, float, double, false);
    MG_SW(2, float, float, float, false);
  }
  if (op.compressed) {
    if (vec64) MG_SW(3, double, double, float, true);
    MG_SW(3, float, float, float, true);
  }
  if (vec64) {
    if (op.elem64) MG_SW(3, double, double, double, false);
    MG_SW(3, double, double, float, false);
  }
  if (op.elem64) MG_SW(3, float, float, double, false);
  MG_SW(3, float, float, float, false);
#undef MG_SW
}

// coarse planes per block of the 3D restriction: about four resident blocks
// per SM (their shared-memory rings)
static int restrict_chunk(int Nc) {
  const long long ntx = (Nc - 1 + kRTX - 1) / kRTX, nty = (Nc - 1 + kRTY - 1) / kRTY;
  const long long want = 152LL * 4;
  const int k = (int)(((long long)(Nc - 1) * ntx * nty + want - 1) / want);
  return k < 1 ? 1 : k;
}

size_t tmask_words(int N) {
  const long long n1 = N + 1;
  return (size_t)((n1 * n1 * n1 + 31) / 32);
}

// fused residual + restriction: adds the touched vertices' residuals (rt,
// from the fix-up pass; zero in the bulk pass) to the z-restricted planes.
// The sum over the touched vertices (i, j, 3K + dz), |dz| <= 2, of column
// (i, j) and coarse plane K is formed, in the order of dz, by the one with the
// smallest dz: one writer per entry, no atomics.
__global__ void zr_fix_kernel(const LevelOp op, const float* __restrict__ rt, float* __restrict__ zr) {
  pdl_begin();
  const int N = op.N, n1 = N + 1, Nc = N / 3;
  const long long plane = (long long)n1 * n1;
  const int nt = *op.ntouched;
  const float wz[5] = {1.f / 3.f, 2.f / 3.f, 1.f, 2.f / 3.f, 1.f / 3.f};
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += gridDim.x * blockDim.x) {
    const long long v = op.touched[t];
    const int k = (int)(v / plane);
    const long long ij = v - (long long)k * plane;
    // coarse planes K with |k - 3K| <= 2
    const int Klo = max(1, k / 3), Khi = min(Nc - 1, (k + 2) / 3);
    if (Klo > Khi) continue;
    // touched bits of column (i, j) at the planes kb = 3 Klo - 2 .. 3 Khi + 2
    // (at most eight), read together
    const int kb = 3 * Klo - 2, ke = 3 * Khi + 2;
    unsigned bits = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const long long vp = (long long)(kb + q) * plane + ij;
      if (kb + q <= ke && ((__ldg(op.tmask + (vp >> 5)) >> (vp & 31)) & 1u)) bits |= 1u << q;
    }
    for (int K = Klo; K <= Khi; ++K) {
      const int base = 3 * K - 2 - kb;   // bit of plane 3K - 2
      // the sum's owner: no touched vertex of the column below k in the window
      if ((bits >> base) & ((1u << (k - (3 * K - 2))) - 1u)) continue;
      float add = 0.f;
#pragma unroll
      for (int dz = -2; dz <= 2; ++dz) {
        const long long vp = (long long)(3 * K + dz) * plane + ij;
        if ((bits >> (base + dz + 2)) & 1u) add = fmaf(wz[dz + 2], __ldg(rt + vp), add);
      }
      zr[(long long)K * plane + ij] += add;
    }
  }
}

cudaError_t launch_resid_restrict(const LevelOp& op, int vec64, const void* x, const void* b, void* rt, void* zr,
                                  void* bc, cudaStream_t st, const void* diag, double omega, void* u1) {
  if (vec64 || op.dim != 3 || !op.compressed || op.stencil || !zr || !op.tmask || !op.touched || !op.eps_pad ||
      op.N < 27 || (op.N + 1) % 4 != 0)
    return cudaErrorNotSupported;
  const int N = op.N, Nc = N / 3;
  const float* xf = (const float*)x;
  const float* bf = (const float*)b;
  // 1. bulk pass: residuals (zero at the touched vertices) restricted along z
  const int nq = (N + 1) / 4;
  const int ntx = (nq + kGeoBX - 1) / kGeoBX, nty = (N - 1 + kGeoBY - 1) / kGeoBY;
  const long long nitems = (long long)ntx * nty * (Nc - 1);
  static int nsm = 0;
  if (!nsm) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (nsm <= 0) nsm = 152;
  }
  const int nb = nitems < 2 * nsm ? (int)nitems : 2 * nsm;
  const dim3 blk(kGeoBX, kGeoBY, 1);
  if (N == 243)
    launch_chain(sweep3_geo4<SW_RESID_RZ, 243>, nb, blk, 0, st, op, xf, bf, nullptr, 0.f, nullptr, ntx, nty, (float*)zr);
  else
    launch_chain(sweep3_geo4<SW_RESID_RZ, 0>, nb, blk, 0, st, op, xf, bf, nullptr, 0.f, nullptr, ntx, nty, (float*)zr);
  count_launches(1);
  // 2. residuals of the touched vertices (full operator) into rt: independent
  // of the bulk pass, launched as its programmatic dependent
  launch_fixup<SW_RESID>(op, xf, bf, (float*)rt, 0.f, nullptr, st);
  count_launches(1);
  // 3. their z-weighted sums into the z-restricted planes
  launch_chain(zr_fix_kernel, 152 * 16, 256, 0, st, op, (const float*)rt, (float*)zr);
  count_launches(1);
  // 4. x-y restriction of the z-restricted planes
  const int kchunk = restrict_chunk(Nc);
  const dim3 g((Nc - 1 + kRTX - 1) / kRTX, (Nc - 1 + kRTY - 1) / kRTY, (Nc - 1 + kchunk - 1) / kchunk);
  launch_chain(restrict3_tile_kernel<float, true>, g, dim3(kRTX, kRTY, 1), 0, st, Nc, kchunk, (const float*)zr,
               (float*)bc, (const float*)diag, (float)omega, (float*)u1);
  return launched();
}

cudaError_t launch_restrict(int dim, int Nc, int vec64, const void* rf, void* bc, cudaStream_t st, const void* diag,
                            double omega, void* u1) {
  if (Nc < 2) return cudaSuccess;   // no interior coarse vertex
  const int ntx = (Nc - 1 + kRTX - 1) / kRTX, nty = (Nc - 1 + kRTY - 1) / kRTY;
  const dim3 blk(kRTX, kRTY, 1);
  if (dim == 2) {
    const dim3 g(ntx, nty, 1);
    if (vec64)
      launch_chain(restrict2_tile_kernel<double>, g, blk, 0, st, Nc, (const double*)rf, (double*)bc,
                   (const double*)diag, omega, (double*)u1);
    else
      launch_chain(restrict2_tile_kernel<float>, g, blk, 0, st, Nc, (const float*)rf, (float*)bc, (const float*)diag,
                   (float)omega, (float*)u1);
    return launched();
  }
  const int kchunk = restrict_chunk(Nc);
  const dim3 g(ntx, nty, (Nc - 1 + kchunk - 1) / kchunk);
  if (vec64)
    launch_chain(restrict3_tile_kernel<double, false>, g, blk, 0, st, Nc, kchunk, (const double*)rf, (double*)bc,
                 (const double*)diag, omega, (double*)u1);
  else
    launch_chain(restrict3_tile_kernel<float, false>, g, blk, 0, st, Nc, kchunk, (const float*)rf, (float*)bc,
                 (const float*)diag, (float)omega, (float*)u1);
  return launched();
}

cudaError_t launch_inject(int dim, int Nc, int vec64, const void* rf, void* bc, cudaStream_t st) {
  long long ni = 1;
  for (int a = 0; a < dim; ++a) ni *= (Nc - 1);
  const int g = vgrid(ni);
  if (dim == 2) {
    if (vec64) inject_kernel<2, double><<<g, 256, 0, st>>>(Nc, (const double*)rf, (double*)bc);
    else inject_kernel<2, float><<<g, 256, 0, st>>>(Nc, (const float*)rf, (float*)bc);
  } else {
    if (vec64) inject_kernel<3, double><<<g, 256, 0, st>>>(Nc, (const double*)rf, (double*)bc);
    else inject_kernel<3, float><<<g, 256, 0, st>>>(Nc, (const float*)rf, (float*)bc);
  }
  return launched();
}

cudaError_t launch_prolong_add(int dim, int Nc, int vec64, const void* ec, void* ef, cudaStream_t st) {
  if (dim == 3 && !vec64 && (3 * Nc + 1) % 4 == 0 && ((uintptr_t)ef & 15) == 0) {
    const int nq = (3 * Nc + 1) / 4;
    const dim3 blk(32, 8, 1);
    const dim3 g((nq + 31) / 32, (3 * Nc - 1 + 7) / 8, 3 * Nc - 1);
    launch_chain(prolong3_x4_kernel, g, blk, 0, st, Nc, (const float*)ec, (float*)ef);
    return launched();
  }
  const int nf = 3 * Nc - 1;
  const dim3 blk(32, 8, 1);
  const dim3 g((nf + 31) / 32, (nf + 7) / 8, dim == 3 ? nf : 1);
  if (dim == 2) {
    if (vec64) launch_chain(prolong_kernel<2, double>, g, blk, 0, st, Nc, (const double*)ec, (double*)ef);
    else launch_chain(prolong_kernel<2, float>, g, blk, 0, st, Nc, (const float*)ec, (float*)ef);
  } else {
    if (vec64) launch_chain(prolong_kernel<3, double>, g, blk, 0, st, Nc, (const double*)ec, (double*)ef);
    else launch_chain(prolong_kernel<3, float>, g, blk, 0, st, Nc, (const float*)ec, (float*)ef);
  }
  return launched();
}

cudaError_t launch_zero(void* p, size_t bytes, cudaStream_t st) { return cudaMemsetAsync(p, 0, bytes, st); }

// eps_c with rows padded to N+1 floats (zero pad)
__global__ void pad_eps_kernel(int N, const float* __restrict__ src, float* __restrict__ dst) {
  const int n1 = N + 1;
  const long long total = (long long)N * N * n1;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int xx = (int)(t % n1);
    const long long r = t / n1;
    dst[t] = xx < N ? src[r * N + xx] : 0.f;
  }
}

cudaError_t launch_pad_eps(int N, const float* eps_c, float* eps_pad, cudaStream_t st) {
  pad_eps_kernel<<<152 * 8, 256, 0, st>>>(N, eps_c, eps_pad);
  return launched();
}

// full FP32 stencils of a compressed 3D level (fields where every cell carries a surplus)
__global__ void build_stencil_cmp3_kernel(const LevelOp op, float* __restrict__ out) {
  const int N = op.N, n1 = N + 1;
  const long long nv = (long long)n1 * n1 * n1;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nv;
       v += (long long)gridDim.x * blockDim.x) {   // boundary vertices too (their forward couplings)
    const int i = (int)(v % n1);
    const int j = (int)((v / n1) % n1);
    const int k = (int)(v / ((long long)n1 * n1));
    float c[27];
    vertex_coeffs3(op, i, j, k, c);
#pragma unroll
    for (int q = 13; q < 27; ++q) out[(size_t)(q - 13) * nv + v] = c[q];   // symmetric storage
  }
}

cudaError_t launch_build_stencil(const LevelOp& op, void* out, cudaStream_t st) {
  if (!out || (op.compressed && op.dim != 3)) return cudaErrorInvalidValue;
  const long long n1 = op.N + 1;
  if (op.compressed) {
    build_stencil_cmp3_kernel<<<vgrid(n1 * n1 * n1), 256, 0, st>>>(op, (float*)out);
    return launched();
  }
  const int g = vgrid(op.dim == 3 ? n1 * n1 * n1 : n1 * n1);
  if (op.dim == 2) {
    if (op.elem64) build_stencil_kernel<2, double><<<g, 256, 0, st>>>(op, (double*)out);
    else build_stencil_kernel<2, float><<<g, 256, 0, st>>>(op, (float*)out);
  } else {
    if (op.elem64) build_stencil_kernel<3, double><<<g, 256, 0, st>>>(op, (double*)out);
    else build_stencil_kernel<3, float><<<g, 256, 0, st>>>(op, (float*)out);
  }
  return launched();
}

cudaError_t launch_build_touched(const LevelOp& op, uint8_t* flags, uint32_t* counts, int* list, int* ntouched,
                                 cudaStream_t st, int from_xpos) {
  const long long nv = (long long)(op.N + 1) * (op.N + 1) * (op.N + 1);
  const long long ng = (nv + 31) / 32;
  cudaError_t e = cudaMemsetAsync(flags, 0, (size_t)nv, st);
  if (e != cudaSuccess) return e;
  touched_mark_kernel<<<152 * 16, 256, 0, st>>>(op, flags, from_xpos);
  count_launches(1);
  uint32_t* tmask = from_xpos ? nullptr : op.tmask;
  touched_count_kernel<<<152 * 16, 256, 0, st>>>(nv, flags, counts, tmask);
  count_launches(1);
  // exclusive scan of the group counts in 2048-entry tiles, then of the tile totals
  const long long ntiles = (ng + 2047) / 2048;
  uint32_t* tile_tot = counts + ng;   // the counts buffer holds ng + ntiles entries
  scan_tiles_kernel<<<(unsigned)ntiles, 1024, 0, st>>>(ng, counts, tile_tot);
  count_launches(1);
  scan1_kernel<<<1, 1024, 0, st>>>(ntiles, tile_tot, ntouched);
  count_launches(1);
  scan_add_kernel<<<(unsigned)ntiles, 1024, 0, st>>>(ng, counts, tile_tot);
  count_launches(1);
  touched_write_kernel<<<152 * 16, 256, 0, st>>>(nv, flags, counts, list);
  if (!from_xpos && op.tcoef && op.tcap > 0) {
    count_launches(1);
    touched_stencil_kernel<<<152 * 8, 256, 0, st>>>(op);
  }
  return launched();
}

template <typename T>
__global__ void sub_from_kernel(long long n, T* __restrict__ a, const T* __restrict__ b) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    a[i] = b[i] - a[i];
}

cudaError_t launch_sub_from(long long n, int vec64, void* a, const void* b, cudaStream_t st) {
  long long g = (n + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  if (g < 1) g = 1;
  if (vec64) sub_from_kernel<double><<<(int)g, 256, 0, st>>>(n, (double*)a, (const double*)b);
  else sub_from_kernel<float><<<(int)g, 256, 0, st>>>(n, (float*)a, (const float*)b);
  return launched();
}

__global__ void xpos_kernel(long long chunk_cells, const int* __restrict__ list, int n, int* __restrict__ xpos) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) xpos[list[i]] = i;
}

cudaError_t launch_xpos(long long chunk_cells, int nchunk, const int* lists, const int* counts_host, int* xpos,
                        cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(xpos, 0xff, sizeof(int) * (size_t)chunk_cells * nchunk, st);
  if (e != cudaSuccess) return e;
  for (int c = 0; c < nchunk; ++c) {
    const int n = counts_host[c];
    if (n <= 0) continue;
    count_launches(1);
    const int g = (n + 255) / 256 < 152 * 8 ? (n + 255) / 256 : 152 * 8;
    xpos_kernel<<<g, 256, 0, st>>>(chunk_cells, lists + (size_t)c * chunk_cells, n,
                                                  xpos + (size_t)c * chunk_cells);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_dot(const double* a, const double* b, long long n, double* partials, int* nblocks, cudaStream_t st) {
  *nblocks = kRedBlocks;
  dot_kernel<double, double><<<kRedBlocks, 256, 0, st>>>(a, b, n, partials);
  return launched();
}

cudaError_t launch_dot_f32f32(const float* a, const float* b, long long n, double* partials, int* nblocks,
                              cudaStream_t st) {
  *nblocks = kRedBlocks;
  launch_chain(dot4_kernel, kRedBlocks, 256, 0, st, a, b, n, partials);
  return launched();
}

cudaError_t launch_dot_f32(const float* a, const double* b, long long n, double* partials, int* nblocks,
                           cudaStream_t st) {
  *nblocks = kRedBlocks;
  dot_kernel<float, double><<<kRedBlocks, 256, 0, st>>>(a, b, n, partials);
  return launched();
}

cudaError_t launch_reduce_finish(const double* partials, int nblocks, int ncomp, double* out, cudaStream_t st,
                                 DevScalars* sc, int op) {
  launch_chain(reduce_finish_kernel, 1, 1024, 0, st, partials, nblocks, ncomp, out, sc, op);
  return launched();
}

cudaError_t launch_scalar_op(DevScalars* sc, int op, cudaStream_t st) {
  scalar_kernel<<<1, 1, 0, st>>>(sc, op);
  return launched();
}

cudaError_t launch_fcg_direction(long long n, int first, int z64, const void* z, double* p, const DevScalars* sc,
                                 cudaStream_t st) {
  if (z64) fcg_direction_kernel<double><<<vgrid(n), 256, 0, st>>>(n, first, (const double*)z, p, sc);
  else fcg_direction_kernel<float><<<vgrid(n), 256, 0, st>>>(n, first, (const float*)z, p, sc);
  return launched();
}

cudaError_t launch_fcg_update(long long n, double* u, double* r, const double* p, const double* q,
                              const DevScalars* sc, int r32_out, void* rin, double* partials, int* nblocks,
                              cudaStream_t st) {
  *nblocks = kRedBlocks;
  if (r32_out) fcg_update_kernel<float><<<kRedBlocks, 256, 0, st>>>(n, u, r, p, q, sc, (float*)rin, partials);
  else fcg_update_kernel<double><<<kRedBlocks, 256, 0, st>>>(n, u, r, p, q, sc, (double*)rin, partials);
  return launched();
}

// ---- FP32 inner flexible CG of the mixed path (vectors FP32, dot products FP64)
// p = z + beta p; first = 0 also applies the previous iteration's deferred
// correction step e += alpha p (alpha still holds that iteration's step length)
// before p is overwritten: one pass reads p for both.  first = 1: p = z.
__global__ void fcg32_direction_kernel(long long n, int first, const float* __restrict__ z, float* __restrict__ p,
                                       float* __restrict__ e, const DevScalars* __restrict__ sc) {
  pdl_begin();
  const float beta = first ? 0.f : (float)sc->beta;
  const float alpha = first ? 0.f : (float)sc->alpha;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long n4 = 0;
  if (aligned16(z) && aligned16(p) && aligned16(e)) {
    n4 = n / 4;
    const float4* z4 = reinterpret_cast<const float4*>(z);
    float4* p4 = reinterpret_cast<float4*>(p);
    float4* e4 = reinterpret_cast<float4*>(e);
    for (long long t = t0; t < n4; t += stride) {
      const float4 a = __ldg(z4 + t);
      if (first) {
        p4[t] = a;
      } else {
        const float4 o = p4[t];
        float4 ev = e4[t];
        ev.x = fmaf(alpha, o.x, ev.x);
        ev.y = fmaf(alpha, o.y, ev.y);
        ev.z = fmaf(alpha, o.z, ev.z);
        ev.w = fmaf(alpha, o.w, ev.w);
        e4[t] = ev;
        p4[t] = make_float4(fmaf(beta, o.x, a.x), fmaf(beta, o.y, a.y), fmaf(beta, o.z, a.z), fmaf(beta, o.w, a.w));
      }
    }
  }
  for (long long t = 4 * n4 + t0; t < n; t += stride) {
    if (first) {
      p[t] = z[t];
    } else {
      const float o = p[t];
      e[t] = fmaf(alpha, o, e[t]);
      p[t] = fmaf(beta, o, z[t]);
    }
  }
}

// r -= alpha q and the partials of r.r (the correction e += alpha p is deferred
// to the next direction update or fcg32_flush_kernel).  With w (= omega D^-1 of
// the finest level), also u1 = w r: the next V-cycle's first smoothing step
// from the zero iterate.
__global__ void fcg32_update_kernel(long long n, float* __restrict__ r, const float* __restrict__ q,
                                    const DevScalars* __restrict__ sc, double* partials,
                                    const float* __restrict__ w, float* __restrict__ u1) {
  pdl_begin();
  __shared__ double sh[8];
  const float alpha = (float)sc->alpha;
  float acc = 0.f;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long n4 = 0;
  const bool smooth = w != nullptr;
  if (aligned16(r) && aligned16(q) && (!smooth || (aligned16(w) && aligned16(u1)))) {
    n4 = n / 4;
    float4* r4 = reinterpret_cast<float4*>(r);
    const float4* q4 = reinterpret_cast<const float4*>(q);
    for (long long t = t0; t < n4; t += stride) {
      const float4 qv = __ldg(q4 + t);
      float4 rv = r4[t];
      rv.x = fmaf(-alpha, qv.x, rv.x);
      rv.y = fmaf(-alpha, qv.y, rv.y);
      rv.z = fmaf(-alpha, qv.z, rv.z);
      rv.w = fmaf(-alpha, qv.w, rv.w);
      r4[t] = rv;
      if (smooth) {
        const float4 wv = __ldg(reinterpret_cast<const float4*>(w) + t);
        reinterpret_cast<float4*>(u1)[t] = make_float4(wv.x * rv.x, wv.y * rv.y, wv.z * rv.z, wv.w * rv.w);
      }
      acc += rv.x * rv.x + rv.y * rv.y + rv.z * rv.z + rv.w * rv.w;
    }
  }
  for (long long t = 4 * n4 + t0; t < n; t += stride) {
    const float rv = r[t] - alpha * q[t];
    r[t] = rv;
    if (smooth) u1[t] = w[t] * rv;
    acc += rv * rv;
  }
  const double s = block_sum((double)acc, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// e += alpha p: the last deferred correction step, before e is used
__global__ void fcg32_flush_kernel(long long n, float* __restrict__ e, const float* __restrict__ p,
                                   const DevScalars* __restrict__ sc) {
  pdl_begin();
  const float alpha = (float)sc->alpha;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    e[t] = fmaf(alpha, p[t], e[t]);
}

// r_in = r / s with s = sqrt(rr) (the residual scaled to unit norm, FP32)
// with w, also u1 = w r_in (as in fcg32_update_kernel)
__global__ void scale_residual_kernel(long long n, const double* __restrict__ r, float* __restrict__ rin,
                                      DevScalars* __restrict__ sc, const float* __restrict__ w,
                                      float* __restrict__ u1) {
  pdl_begin();
  const double s = sc->rr > 0.0 ? sqrt(sc->rr) : 1.0;
  if (blockIdx.x == 0 && threadIdx.x == 0) sc->s = s;
  // the scaling in FP32 after the conversion (one FP64-pipe operation per
  // entry instead of two; the entry is rounded to FP32 either way)
  const float inv = (float)(1.0 / s);
  const long long n2 = n / 2;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t <= n2;
       t += (long long)gridDim.x * blockDim.x) {
    if (t < n2) {
      const double2 r2 = reinterpret_cast<const double2*>(r)[t];
      const float2 v = make_float2((float)r2.x * inv, (float)r2.y * inv);
      reinterpret_cast<float2*>(rin)[t] = v;
      if (w) {
        const float2 w2 = reinterpret_cast<const float2*>(w)[t];
        reinterpret_cast<float2*>(u1)[t] = make_float2(w2.x * v.x, w2.y * v.y);
      }
    } else if (2 * t < n) {   // odd n: the last entry
      const float v = (float)r[2 * t] * inv;
      rin[2 * t] = v;
      if (w) u1[2 * t] = w[2 * t] * v;
    }
  }
}

// u += s e (the scaled FP32 correction applied in FP64)
__global__ void apply_correction_kernel(long long n, double* __restrict__ u, const float* __restrict__ e,
                                        const DevScalars* __restrict__ sc) {
  pdl_begin();
  const double s = sc->s;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    u[t] += s * (double)e[t];
}

cudaError_t launch_fcg32_direction(long long n, int first, const float* z, float* p, float* e, const DevScalars* sc,
                                   cudaStream_t st) {
  launch_chain(fcg32_direction_kernel, vgrid((n + 3) / 4), 256, 0, st, n, first, z, p, e, sc);
  return launched();
}

cudaError_t launch_fcg32_update(long long n, float* r, const float* q, const DevScalars* sc, double* partials,
                                int* nblocks, cudaStream_t st, const float* w, float* u1) {
  *nblocks = kRedBlocks;
  launch_chain(fcg32_update_kernel, kRedBlocks, 256, 0, st, n, r, q, sc, partials, w, u1);
  return launched();
}

__global__ void fill_kernel(long long n, float v, float* __restrict__ p) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    p[t] = v;
}

cudaError_t launch_fill(long long n, float v, float* p, cudaStream_t st) {
  fill_kernel<<<vgrid(n), 256, 0, st>>>(n, v, p);
  return launched();
}

cudaError_t launch_fcg32_flush(long long n, float* e, const float* p, const DevScalars* sc, cudaStream_t st) {
  launch_chain(fcg32_flush_kernel, vgrid(n), 256, 0, st, n, e, p, sc);
  return launched();
}

cudaError_t launch_scale_residual(long long n, const double* r, float* rin, DevScalars* sc, cudaStream_t st,
                                  const float* w, float* u1) {
  launch_chain(scale_residual_kernel, vgrid(n / 2 + 1), 256, 0, st, n, r, rin, sc, w, u1);
  return launched();
}

cudaError_t launch_apply_correction(long long n, double* u, const float* e, const DevScalars* sc, cudaStream_t st) {
  launch_chain(apply_correction_kernel, vgrid(n), 256, 0, st, n, u, e, sc);
  return launched();
}

cudaError_t launch_richardson_update(long long n, double* u, int z64, const void* z, cudaStream_t st) {
  if (z64) richardson_kernel<double><<<vgrid(n), 256, 0, st>>>(n, u, (const double*)z);
  else richardson_kernel<float><<<vgrid(n), 256, 0, st>>>(n, u, (const float*)z);
  return launched();
}

cudaError_t launch_convert(long long n, int to64, const void* src, void* dst, cudaStream_t st) {
  if (to64) convert_kernel<float, double><<<vgrid(n), 256, 0, st>>>(n, (const float*)src, (double*)dst);
  else convert_kernel<double, float><<<vgrid(n), 256, 0, st>>>(n, (const double*)src, (float*)dst);
  return launched();
}

cudaError_t launch_load_vector(int dim, int N, double val, double* f, cudaStream_t st) {
  long long nv = 1;
  for (int a = 0; a < dim; ++a) nv *= (N + 1);
  if (dim == 2) load_vector_kernel<2><<<vgrid(nv), 256, 0, st>>>(N, val, f);
  else load_vector_kernel<3><<<vgrid(nv), 256, 0, st>>>(N, val, f);
  return launched();
}

}  // namespace mg
