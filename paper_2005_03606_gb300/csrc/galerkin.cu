// Ritz-Galerkin coarse operators A_{l-1} = R A_l P with d-linear 3:1
// transfers (Section "Rediscretisation and geometric projections between
// levels vs. Ritz-Galerkin plus algebraic operators"), computed element by
// element: for coarse cell C,
//   A_C = sum over its 3^d children f of P_f^T A_f P_f,
// P_f the d-linear interpolation from C's vertices to f's vertices.  With
// A_f = -sum_{a<b} A_ab (e_a - e_b)(e_a - e_b)^T (symmetric, zero row sums),
//   (A_C)_IJ = -sum_f sum_{a<b} A_f,ab (P_aI - P_bI)(P_aJ - P_bJ),
// which keeps zero row sums by construction.  Children stored as
// eps_c K_ref + surplus contribute eps_c * G_f (G_f = P_f^T K_ref P_f, a
// constant table) plus the surplus term, so children of storage class 0 cost
// one multiply per coarse entry.
//
// The coarsest level (3 cells per axis, 2^d interior unknowns) is solved by
// an FP64 Cholesky factorisation formed once per operator update.
#include "mg_internal.cuh"

#include <mutex>
#include <type_traits>

namespace mg {

namespace {

__constant__ double c_G2[9][6];
__constant__ double c_G3[27][28];
// the same tables rounded to FP32, for the FP32 products (no FP64 -> FP32
// conversion per coarse entry in the kernel)
__constant__ float c_G2f[9][6];
__constant__ float c_G3f[27][28];
bool g_tables_ready = false;

template <int D>
__host__ __device__ inline double pweight(int o, int bit_fine, int bit_coarse) {
  const double t = (o + bit_fine) / 3.0;
  return bit_coarse ? t : 1.0 - t;
}

template <int D>
__host__ __device__ inline void child_P(int ch, double P[Dim<D>::NV][Dim<D>::NV]) {
  constexpr int NV = Dim<D>::NV;
  int o[3] = {ch % 3, (ch / 3) % 3, ch / 9};
  for (int a = 0; a < NV; ++a)
    for (int I = 0; I < NV; ++I) {
      double w = 1.0;
      for (int m = 0; m < D; ++m) w *= pweight<D>(o[m], (a >> m) & 1, (I >> m) & 1);
      P[a][I] = w;
    }
}

template <int D>
void host_G(double* G) {  // [nchild][NP]
  constexpr int NV = Dim<D>::NV, NP = Dim<D>::NP;
  const int nch = D == 3 ? 27 : 9;
  for (int ch = 0; ch < nch; ++ch) {
    double P[NV][NV];
    child_P<D>(ch, P);
    for (int I = 0; I < NV; ++I)
      for (int J = I + 1; J < NV; ++J) {
        double acc = 0.0;
        for (int a = 0; a < NV; ++a)
          for (int b = a + 1; b < NV; ++b) {
            const double k = kref_off<D>(popc_small(a ^ b));
            acc -= k * (P[a][I] - P[b][I]) * (P[a][J] - P[b][J]);
          }
        G[ch * NP + pair_index(NV, I, J)] = acc;
      }
  }
}

std::mutex g_tables_mu;

cudaError_t ensure_tables() {
  std::lock_guard<std::mutex> lk(g_tables_mu);
  if (g_tables_ready) return cudaSuccess;
  double g2[9 * 6], g3[27 * 28];
  host_G<2>(g2);
  host_G<3>(g3);
  float g2f[9 * 6], g3f[27 * 28];
  for (int i = 0; i < 9 * 6; ++i) g2f[i] = (float)g2[i];
  for (int i = 0; i < 27 * 28; ++i) g3f[i] = (float)g3[i];
  cudaError_t e = cudaMemcpyToSymbol(c_G2, g2, sizeof(g2));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_G2f, g2f, sizeof(g2f));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_G3f, g3f, sizeof(g3f));
  if (e != cudaSuccess) return e;
  e = cudaMemcpyToSymbol(c_G3, g3, sizeof(g3));
  if (e == cudaSuccess) g_tables_ready = true;
  return e;
}

// entry p of the table G of child ch in the arithmetic type
template <int D, typename TA>
__device__ __forceinline__ TA gtab(int ch, int p) {
  if constexpr (std::is_same<TA, float>::value) return D == 3 ? c_G3f[ch][p] : c_G2f[ch][p];
  else return D == 3 ? c_G3[ch][p] : c_G2[ch][p];
}

// off-diagonals of the fine cell (i,j,k) (full storage) into A[NP]
template <int D, typename TA, typename TS>
__device__ __forceinline__ void load_full(const LevelOp& op, int ci, int cj, int ck, TA* A) {
  constexpr int NP = Dim<D>::NP;
  const int N = op.N;
  const long long c = D == 2 ? (long long)cj * N + ci : ((long long)ck * N + cj) * N + ci;
  int ch = (D == 2 ? cj : ck) / op.layers;
  if (ch >= op.nchunk) ch = op.nchunk - 1;
  const long long lc = c - (long long)ch * op.chunk_cells;
  const TS* a = reinterpret_cast<const TS*>(op.full[ch].a);
#pragma unroll
  for (int p = 0; p < NP; ++p) A[p] = (TA)a[(long long)p * op.chunk_cells + lc];
}

template <int D, typename TA, typename TS, typename TC, bool CMP>
__global__ void galerkin_kernel(const LevelOp fine, int last0, int last1, TC* __restrict__ out) {
  constexpr int NV = Dim<D>::NV, NP = Dim<D>::NP;
  const int Nc = fine.N / 3;
  const long long per_layer = D == 2 ? (long long)Nc : (long long)Nc * Nc;
  const long long ncc_total = per_layer * Nc;
  const long long c_begin = (long long)last0 * per_layer, c_end = (long long)last1 * per_layer;
  for (long long C = c_begin + blockIdx.x * (long long)blockDim.x + threadIdx.x; C < c_end;
       C += (long long)gridDim.x * blockDim.x) {
    const int I0 = (int)(C % Nc);
    const int J0 = (int)((C / Nc) % Nc);
    const int K0 = D == 3 ? (int)(C / ((long long)Nc * Nc)) : 0;
    TA acc[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) acc[p] = 0;
    const int nch = D == 3 ? 27 : 9;
    for (int ch = 0; ch < nch; ++ch) {
      const int ox = ch % 3, oy = (ch / 3) % 3, oz = ch / 9;
      const int fi = 3 * I0 + ox, fj = 3 * J0 + oy, fk = D == 3 ? 3 * K0 + oz : 0;
      TA A[NP];
      bool have_full = true;
      if (CMP) {
        const long long c = D == 2 ? (long long)fj * fine.N + fi : ((long long)fk * fine.N + fj) * fine.N + fi;
        const TA ge = (TA)fine.eps_c[c] * (TA)fine.hfac;
#pragma unroll
        for (int p = 0; p < NP; ++p) acc[p] += ge * gtab<D, TA>(ch, p);
        int chn = (D == 2 ? fj : fk) / fine.layers;
        if (chn >= fine.nchunk) chn = fine.nchunk - 1;
        const long long lc = c - (long long)chn * fine.chunk_cells;
        const CmpChunk& ck = fine.cmp[chn];
        const int cls = cell_class(ck, fine.N, fine.nseg_x, lc);
        if (cls == 0) {
          have_full = false;
        } else {
          const uint8_t* rec = cell_record<D>(ck, fine.N, fine.nseg_x, lc, cls);
#pragma unroll
          for (int p = 0; p < NP; ++p) A[p] = (TA)decode_entry<D>(rec, cls, p);
        }
      } else {
        load_full<D, TA, TS>(fine, fi, fj, fk, A);
      }
      if (!have_full) continue;
      // interpolation weights of this child: P[a][I] = prod_m w(o_m, a_m, I_m)
      TA P[NV][NV];
#pragma unroll
      for (int a = 0; a < NV; ++a)
#pragma unroll
        for (int I = 0; I < NV; ++I) {
          TA w = 1;
#pragma unroll
          for (int m = 0; m < D; ++m) {
            const int o = m == 0 ? ox : (m == 1 ? oy : oz);
            const TA t = (TA)(o + ((a >> m) & 1)) / (TA)3;
            w *= ((I >> m) & 1) ? t : (TA)1 - t;
          }
          P[a][I] = w;
        }
#pragma unroll
      for (int a = 0; a < NV; ++a)
#pragma unroll
        for (int b = a + 1; b < NV; ++b) {
          const TA v = A[pair_index(NV, a, b)];
          TA q[NV];
#pragma unroll
          for (int I = 0; I < NV; ++I) q[I] = P[a][I] - P[b][I];
#pragma unroll
          for (int I = 0; I < NV; ++I)
#pragma unroll
            for (int J = I + 1; J < NV; ++J) acc[pair_index(NV, I, J)] -= v * q[I] * q[J];
        }
    }
#pragma unroll
    for (int p = 0; p < NP; ++p) out[(long long)p * ncc_total + C] = (TC)acc[p];
  }
}

// 3D FP32 Galerkin product of a compressed fine level, one thread per coarse
// cell, in two phases.  (1) The 27 children's eps and classes are loaded
// together (one memory latency instead of 27 dependent ones), their
// geometric part eps_c G_ch is summed, and the children with a surplus are
// marked.  (2) The marked (cell, child) pairs of a warp go through a queue in
// shared memory and their pair products run 32 at a time, one per lane
// (one thread per coarse cell would run them child position by child
// position, mostly with one or two lanes active); each coarse cell then adds
// the contributions of its own children in child order.
constexpr int kGalWarps = 4;

// P[a][I] = wx[a0][I0] wy[a1][I1] wz[a2][I2]: the d-linear interpolation
// weight of coarse vertex I at vertex a of child (ox, oy, oz)
__device__ __forceinline__ void child_weights1d(int o, float (&w)[2][2]) {
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    const float t = (float)(o + a) / 3.f;
    w[a][0] = 1.f - t;
    w[a][1] = t;
  }
}

__global__ void __launch_bounds__(32 * kGalWarps) galerkin3q_kernel(const LevelOp fine, int last0, int last1,
                                                                     float* __restrict__ out) {
  constexpr int NV = 8, NP = 28;
  __shared__ unsigned short q_s[kGalWarps][64];
  __shared__ float c_s[kGalWarps][32][NP + 1];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned short* q = q_s[wid];
  float(*cs)[NP + 1] = c_s[wid];
  const int N = fine.N, Nc = N / 3;
  const long long per_layer = (long long)Nc * Nc;
  const long long ncc_total = per_layer * Nc;
  const long long c_begin = (long long)last0 * per_layer, c_end = (long long)last1 * per_layer;
  const long long wstride = (long long)gridDim.x * kGalWarps * 32;
  const float hfac = (float)fine.hfac;
  for (long long base = c_begin + ((long long)blockIdx.x * kGalWarps + wid) * 32; base < c_end; base += wstride) {
    const long long C = base + lane;
    const bool valid = C < c_end;
    const long long Cv = valid ? C : c_end - 1;
    const int I0 = (int)(Cv % Nc), J0 = (int)((Cv / Nc) % Nc), K0 = (int)(Cv / per_layer);
    float acc[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) acc[p] = 0.f;
    // (1) geometric part and the surplus children
    float ge[27];
    uint8_t cls[27];
#pragma unroll
    for (int ch = 0; ch < 27; ++ch) {
      const int fi = 3 * I0 + ch % 3, fj = 3 * J0 + (ch / 3) % 3, fk = 3 * K0 + ch / 9;
      const long long c = ((long long)fk * N + fj) * N + fi;
      int chn = fk / fine.layers;
      if (chn >= fine.nchunk) chn = fine.nchunk - 1;
      ge[ch] = __ldg(fine.eps_c + c);
      // the cell's row within its chunk, without dividing the cell index
      const long long row = (long long)(fk - chn * fine.layers) * N + fj;
      cls[ch] = fine.cmp[chn].cls[(row * fine.nseg_x + (fi >> 5)) * kSegCells + (fi & 31)];
    }
    unsigned mine = 0;
#pragma unroll
    for (int ch = 0; ch < 27; ++ch) {
      const float g = ge[ch] * hfac;
#pragma unroll
      for (int p = 0; p < NP; ++p) acc[p] = fmaf(g, c_G3f[ch][p], acc[p]);
      if (cls[ch] && valid) mine |= 1u << ch;
    }
    // (2) the surplus children, in rounds (each lane's next child) through the queue
    int qn = 0;
    bool more = __any_sync(0xffffffffu, mine != 0u);
    while (more || qn > 0) {
      if (more) {
        const unsigned m = __ballot_sync(0xffffffffu, mine != 0u);
        if (mine) {
          const int ch = __ffs(mine) - 1;
          mine &= mine - 1;
          q[qn + __popc(m & ((1u << lane) - 1u))] = (unsigned short)(lane | (ch << 5));
        }
        qn += __popc(m);
        more = __any_sync(0xffffffffu, mine != 0u);
      }
      if (qn < 32 && more) continue;
      // one batch: the first min(qn, 32) queued pairs, one per lane
      __syncwarp();
      const int nb = qn < 32 ? qn : 32;
      if (lane < nb) {
        const int e = q[lane], o = e & 31, ch = e >> 5;
        const long long Co = base + o;
        const int oI = (int)(Co % Nc), oJ = (int)((Co / Nc) % Nc), oK = (int)(Co / per_layer);
        const int ox = ch % 3, oy = (ch / 3) % 3, oz = ch / 9;
        const int fi = 3 * oI + ox, fj = 3 * oJ + oy, fk = 3 * oK + oz;
        const long long c = ((long long)fk * N + fj) * N + fi;
        int chn = fk / fine.layers;
        if (chn >= fine.nchunk) chn = fine.nchunk - 1;
        const CmpChunk& ck = fine.cmp[chn];
        const long long lc = c - (long long)chn * fine.chunk_cells;
        const int cl = cell_class(ck, N, fine.nseg_x, lc);
        const uint8_t* rec = cell_record<3>(ck, N, fine.nseg_x, lc, cl);
        float A[NP];
#pragma unroll
        for (int p = 0; p < NP; ++p) A[p] = decode_entry<3>(rec, cl, p);
        float wx[2][2], wy[2][2], wz[2][2];
        child_weights1d(ox, wx);
        child_weights1d(oy, wy);
        child_weights1d(oz, wz);
        float con[NP];
#pragma unroll
        for (int p = 0; p < NP; ++p) con[p] = 0.f;
#pragma unroll
        for (int a = 0; a < NV; ++a)
#pragma unroll
          for (int b = a + 1; b < NV; ++b) {
            const float v = A[pair_index(NV, a, b)];
            float d[NV], vd[NV];
#pragma unroll
            for (int I = 0; I < NV; ++I) {
              const float pa = wx[a & 1][I & 1] * wy[(a >> 1) & 1][(I >> 1) & 1] * wz[a >> 2][I >> 2];
              const float pb = wx[b & 1][I & 1] * wy[(b >> 1) & 1][(I >> 1) & 1] * wz[b >> 2][I >> 2];
              d[I] = pa - pb;
              vd[I] = -v * d[I];
            }
#pragma unroll
            for (int I = 0; I < NV; ++I)
#pragma unroll
              for (int J = I + 1; J < NV; ++J) con[pair_index(NV, I, J)] = fmaf(vd[I], d[J], con[pair_index(NV, I, J)]);
          }
#pragma unroll
        for (int p = 0; p < NP; ++p) cs[lane][p] = con[p];
      }
      __syncwarp();
      for (int t = 0; t < nb; ++t)
        if ((q[t] & 31) == lane) {
#pragma unroll
          for (int p = 0; p < NP; ++p) acc[p] += cs[t][p];
        }
      __syncwarp();
      // keep the pairs beyond the batch
      const int rest = qn - nb;
      const unsigned short keep = lane < rest ? q[nb + lane] : 0;
      __syncwarp();
      if (lane < rest) q[lane] = keep;
      __syncwarp();
      qn = rest;
    }
    if (valid) {
#pragma unroll
      for (int p = 0; p < NP; ++p) out[(long long)p * ncc_total + C] = acc[p];
    }
  }
}

// dense interior system of the coarsest level (N = 3) and its Cholesky factor
template <int D, typename TS>
__global__ void coarse_factor_kernel(const LevelOp op, double* L) {
  constexpr int NV = Dim<D>::NV, NP = Dim<D>::NP;
  constexpr int NC = D == 3 ? 27 : 9;   // cells of the coarsest level (3 per axis)
  // thread c < NC writes cell c's contribution to the dense interior system;
  // the contributions are then summed in cell order (as one thread would)
  __shared__ double S[NC][NV * NV];
  __shared__ double Ms[NV * NV];
  const int n = NV;  // 2^d interior vertices (1..2 per axis)
  const TS* a = reinterpret_cast<const TS*>(op.full[0].a);
  const long long ncell = op.chunk_cells;
  const int c = threadIdx.x;
  if (c < NC) {
    const int ci = c % 3, cj = (c / 3) % 3, ck = c / 9;
    int gidx[NV];
#pragma unroll
    for (int b = 0; b < NV; ++b) {
      const int vx = ci + (b & 1), vy = cj + ((b >> 1) & 1), vz = D == 3 ? ck + ((b >> 2) & 1) : 1;
      const bool in = vx >= 1 && vx <= 2 && vy >= 1 && vy <= 2 && vz >= 1 && vz <= 2;
      gidx[b] = in ? (vx - 1) + 2 * (vy - 1) + (D == 3 ? 4 * (vz - 1) : 0) : -1;
    }
    double A[NV][NV];
#pragma unroll
    for (int x = 0; x < NV; ++x) A[x][x] = 0.0;
#pragma unroll
    for (int x = 0; x < NV; ++x)
#pragma unroll
      for (int y = x + 1; y < NV; ++y) {
        const double v = (double)a[(long long)pair_index(NV, x, y) * ncell + c];
        A[x][y] = v;
        A[y][x] = v;
        A[x][x] -= v;
        A[y][y] -= v;
      }
    for (int e = 0; e < NV * NV; ++e) S[c][e] = 0.0;
#pragma unroll
    for (int x = 0; x < NV; ++x)
#pragma unroll
      for (int y = 0; y < NV; ++y)
        if (gidx[x] >= 0 && gidx[y] >= 0) S[c][gidx[x] * NV + gidx[y]] = A[x][y];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < NV * NV; e += blockDim.x) {
    double sum = 0.0;
    for (int k = 0; k < NC; ++k) sum += S[k][e];
    Ms[e] = sum;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  // factor and inverse of the 2^d x 2^d system, loops unrolled so that the
  // matrix stays in registers
  double M[NV][NV];
#pragma unroll
  for (int i = 0; i < n; ++i)
#pragma unroll
    for (int j = 0; j < n; ++j) M[i][j] = Ms[i * NV + j];
  (void)NP;
#pragma unroll
  for (int j = 0; j < n; ++j) {
    double s = M[j][j];
#pragma unroll
    for (int k = 0; k < j; ++k) s -= M[j][k] * M[j][k];
    M[j][j] = sqrt(s);
#pragma unroll
    for (int i = j + 1; i < n; ++i) {
      double t = M[i][j];
#pragma unroll
      for (int k = 0; k < j; ++k) t -= M[i][k] * M[j][k];
      M[i][j] = t / M[j][j];
    }
  }
#pragma unroll
  for (int i = 0; i < n; ++i)
#pragma unroll
    for (int j = 0; j < n; ++j) L[i * n + j] = j <= i ? M[i][j] : 0.0;
  // the inverse, column by column from the factor (L[n*n ..]: row-major, used
  // by the single-block tail of the FP32 V-cycle)
  double* Ainv = L + n * n;
#pragma unroll
  for (int c = 0; c < n; ++c) {
    double z[NV];
#pragma unroll
    for (int i = 0; i < n; ++i) {
      double t = i == c ? 1.0 : 0.0;
#pragma unroll
      for (int k = 0; k < i; ++k) t -= M[i][k] * z[k];
      z[i] = t / M[i][i];
    }
#pragma unroll
    for (int i = n - 1; i >= 0; --i) {
      double t = z[i];
#pragma unroll
      for (int k = i + 1; k < n; ++k) t -= M[k][i] * z[k];
      z[i] = t / M[i][i];
    }
#pragma unroll
    for (int i = 0; i < n; ++i) Ainv[i * n + c] = z[i];
  }
}

template <int D, typename TV>
__global__ void coarse_solve_kernel(const double* __restrict__ L, const TV* __restrict__ b, TV* __restrict__ e) {
  pdl_begin();
  constexpr int n = Dim<D>::NV;
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double z[n];
  long long vid[n];
  for (int t = 0; t < n; ++t) {
    const int vx = 1 + (t & 1), vy = 1 + ((t >> 1) & 1), vz = D == 3 ? 1 + ((t >> 2) & 1) : 0;
    vid[t] = D == 3 ? ((long long)vz * 4 + vy) * 4 + vx : (long long)vy * 4 + vx;
  }
  for (int i = 0; i < n; ++i) {
    double t = (double)b[vid[i]];
    for (int k = 0; k < i; ++k) t -= L[i * n + k] * z[k];
    z[i] = t / L[i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double t = z[i];
    for (int k = i + 1; k < n; ++k) t -= L[k * n + i] * z[k];
    z[i] = t / L[i * n + i];
  }
  for (int i = 0; i < n; ++i) e[vid[i]] = (TV)z[i];
}

template <int D, typename TS, bool CMP>
__global__ void decode_kernel(const LevelOp op, const long long* __restrict__ cells, long long nout,
                              double* __restrict__ out) {
  constexpr int NV = Dim<D>::NV, NP = Dim<D>::NP;
  const int N = op.N;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nout;
       t += (long long)gridDim.x * blockDim.x) {
    const long long c = cells ? cells[t] : t;
    const int ci = (int)(c % N), cj = (int)((c / N) % N), ck = D == 3 ? (int)(c / ((long long)N * N)) : 0;
    double A[NP];
    if (CMP) {
      const double ge = (double)op.eps_c[c] * op.hfac;
      int ch = (D == 2 ? cj : ck) / op.layers;
      if (ch >= op.nchunk) ch = op.nchunk - 1;
      const long long lc = c - (long long)ch * op.chunk_cells;
      const CmpChunk& chk = op.cmp[ch];
      const int cls = cell_class(chk, N, op.nseg_x, lc);
      const uint8_t* rec = cls ? cell_record<D>(chk, N, op.nseg_x, lc, cls) : nullptr;
      for (int a = 0; a < NV; ++a)
        for (int b = a + 1; b < NV; ++b) {
          const int p = pair_index(NV, a, b);
          double v = ge * kref_off<D>(popc_small(a ^ b));
          if (cls) v += (double)decode_entry<D>(rec, cls, p);
          A[p] = v;
        }
    } else {
      load_full<D, double, TS>(op, ci, cj, ck, A);
    }
    double* M = out + t * NV * NV;
    for (int a = 0; a < NV; ++a) M[a * NV + a] = 0.0;
    for (int a = 0; a < NV; ++a)
      for (int b = a + 1; b < NV; ++b) {
        const double v = A[pair_index(NV, a, b)];
        M[a * NV + b] = v;
        M[b * NV + a] = v;
        M[a * NV + a] -= v;
        M[b * NV + b] -= v;
      }
  }
}

int ggrid(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  if (b > 152LL * 32) b = 152LL * 32;
  if (b < 1) b = 1;
  return (int)b;
}

// Compressed coarse-level operators (Section "Precision toggling and
// information density": store only the hierarchical surplus of an operator
// over its one-sample rediscretisation, with as few bytes as the error bound
// allows).  In place, cell by cell of a coarse level's FP32 Galerkin store
// (SoA [NP][ncell]): the surplus over eps_C K_ref h^(d-2) (eps_C the field at
// the coarse cell centre, FP32) takes the storage class of the finest level's
// rule with bound tau, is encoded (FP8 e4m3 or FP16 with an FP32 scale, or
// FP32) and decoded again, so every later use of the level (its stencils, the
// next Galerkin product, the coarsest factor) sees the stored operator.
template <int D>
__global__ void compress_coarse_kernel(long long ncell, float* __restrict__ a, const float* __restrict__ eps_c,
                                       float hfac, float tau, uint8_t* __restrict__ cls_out,
                                       unsigned long long* __restrict__ counts) {
  constexpr int NV = Dim<D>::NV, NP = Dim<D>::NP;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
       c += (long long)gridDim.x * blockDim.x) {
    const float ge = eps_c[c] * hfac;
    float dl[NP], g[NP];
    float Dm = 0.f, An = 0.f, rs[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) rs[v] = 0.f;
#pragma unroll
    for (int x = 0; x < NV; ++x)
#pragma unroll
      for (int y = x + 1; y < NV; ++y) {
        const int p = pair_index(NV, x, y);
        const float av = a[(long long)p * ncell + c];
        g[p] = ge * (float)kref_off<D>(popc_small(x ^ y));
        dl[p] = av - g[p];
        Dm = fmaxf(Dm, fabsf(dl[p]));
        An = fmaxf(An, fabsf(av));
        rs[x] += av;
        rs[y] += av;
      }
#pragma unroll
    for (int v = 0; v < NV; ++v) An = fmaxf(An, fabsf(rs[v]));   // the diagonal is minus the row sum
    const float Fm = (float)Dim<D>::F;
    int cls;
    if (Fm * Dm <= tau * An) cls = 0;
    else if (Fm * Dm * (16.f / 448.f) <= tau * An) cls = 1;
    else if (Fm * Dm * (16.f / 65504.f) <= tau * An) cls = 2;
    else cls = 3;
    uint8_t rec[Dim<D>::REC_MAX];
    if (cls == 1) {
      const float sc = Dm / 448.f;
      *reinterpret_cast<float*>(rec) = sc;
#pragma unroll
      for (int p = 0; p < NP; ++p) {
        __nv_fp8_e4m3 q(dl[p] / sc);
        rec[4 + p] = q.__x;
      }
    } else if (cls == 2) {
      const float sc = Dm / 65504.f;
      *reinterpret_cast<float*>(rec) = sc;
#pragma unroll
      for (int p = 0; p < NP; ++p) *reinterpret_cast<__half*>(rec + 4 + 2 * p) = __float2half_rn(dl[p] / sc);
    } else if (cls == 3) {
#pragma unroll
      for (int p = 0; p < NP; ++p) *reinterpret_cast<float*>(rec + 4 * p) = dl[p];
    }
#pragma unroll
    for (int p = 0; p < NP; ++p) a[(long long)p * ncell + c] = g[p] + (cls ? decode_entry<D>(rec, cls, p) : 0.f);
    cls_out[c] = (uint8_t)cls;
    if (counts) atomicAdd(counts + cls, 1ull);
  }
}

}  // namespace

// Galerkin over the coarse cell layers [last0, last1) along the last axis.
cudaError_t launch_galerkin_range(const LevelOp& fine, int out64, void* coarse_full, int last0, int last1,
                                  cudaStream_t st) {
  cudaError_t e = ensure_tables();
  if (e != cudaSuccess) return e;
  const int Nc = fine.N / 3;
  const long long per_layer = fine.dim == 2 ? (long long)Nc : (long long)Nc * Nc;
  const long long n = per_layer * (last1 - last0);
  if (n <= 0) return cudaSuccess;
  const int T = 128;
  const int g = ggrid(n, T);
#define MG_GAL(D, TA, TS, TC, CMP) \
  galerkin_kernel<D, TA, TS, TC, CMP><<<g, T, 0, st>>>(fine, last0, last1, (TC*)coarse_full)
  if (fine.dim == 2) {
    if (fine.compressed) {
      if (out64) MG_GAL(2, double, float, double, true);
      else MG_GAL(2, float, float, float, true);
    } else if (fine.elem64) {
      if (out64) MG_GAL(2, double, double, double, false);
      else MG_GAL(2, double, double, float, false);
    } else {
      if (out64) MG_GAL(2, double, float, double, false);
      else MG_GAL(2, float, float, float, false);
    }
  } else {
    if (fine.compressed) {
      if (out64) {
        MG_GAL(3, double, float, double, true);
      } else if (!getenv("MG_GALERKIN_THREAD")) {   // queued surplus products (see galerkin3q_kernel)
        const long long nwarps = (n + 31) / 32;
        long long nblk = (nwarps + kGalWarps - 1) / kGalWarps;
        nblk = nblk < 152LL * 16 ? nblk : 152LL * 16;
        galerkin3q_kernel<<<(int)nblk, 32 * kGalWarps, 0, st>>>(fine, last0, last1, (float*)coarse_full);
      } else {
        MG_GAL(3, float, float, float, true);
      }
    } else if (fine.elem64) {
      if (out64) MG_GAL(3, double, double, double, false);
      else MG_GAL(3, double, double, float, false);
    } else {
      if (out64) MG_GAL(3, double, float, double, false);
      else MG_GAL(3, float, float, float, false);
    }
  }
#undef MG_GAL
  return launched();
}

cudaError_t launch_galerkin(const LevelOp& fine, int out64, void* coarse_full, cudaStream_t st) {
  return launch_galerkin_range(fine, out64, coarse_full, 0, fine.N / 3, st);
}

cudaError_t launch_compress_coarse(int dim, long long ncell, float* a, const float* eps_c, double hfac, double tau,
                                   uint8_t* cls_out, unsigned long long* counts, cudaStream_t st) {
  if (ncell <= 0) return cudaSuccess;
  const int g = ggrid(ncell, 128);
  if (dim == 3)
    compress_coarse_kernel<3><<<g, 128, 0, st>>>(ncell, a, eps_c, (float)hfac, (float)tau, cls_out, counts);
  else
    compress_coarse_kernel<2><<<g, 128, 0, st>>>(ncell, a, eps_c, (float)hfac, (float)tau, cls_out, counts);
  return launched();
}

cudaError_t launch_coarse_factor(const LevelOp& coarsest, double* L, cudaStream_t st) {
  if (coarsest.N != 3 || coarsest.compressed) return cudaErrorInvalidValue;
  if (coarsest.dim == 2) {
    if (coarsest.elem64) coarse_factor_kernel<2, double><<<1, 32, 0, st>>>(coarsest, L);
    else coarse_factor_kernel<2, float><<<1, 32, 0, st>>>(coarsest, L);
  } else {
    if (coarsest.elem64) coarse_factor_kernel<3, double><<<1, 32, 0, st>>>(coarsest, L);
    else coarse_factor_kernel<3, float><<<1, 32, 0, st>>>(coarsest, L);
  }
  return launched();
}

cudaError_t launch_coarse_solve(int dim, const double* L, int vec64, const void* b, void* e, cudaStream_t st) {
  if (dim == 2) {
    if (vec64) launch_chain(coarse_solve_kernel<2, double>, 1, 32, 0, st, L, (const double*)b, (double*)e);
    else launch_chain(coarse_solve_kernel<2, float>, 1, 32, 0, st, L, (const float*)b, (float*)e);
  } else {
    if (vec64) launch_chain(coarse_solve_kernel<3, double>, 1, 32, 0, st, L, (const double*)b, (double*)e);
    else launch_chain(coarse_solve_kernel<3, float>, 1, 32, 0, st, L, (const float*)b, (float*)e);
  }
  return launched();
}

cudaError_t launch_decode_matrices(const LevelOp& op, const long long* cells, long long ncells, double* out,
                                   cudaStream_t st) {
  const long long ncell = cells ? ncells : (long long)op.N * op.N * (op.dim == 3 ? op.N : 1);
  const int g = ggrid(ncell, 128);
  if (op.dim == 2) {
    if (op.compressed) decode_kernel<2, float, true><<<g, 128, 0, st>>>(op, cells, ncell, out);
    else if (op.elem64) decode_kernel<2, double, false><<<g, 128, 0, st>>>(op, cells, ncell, out);
    else decode_kernel<2, float, false><<<g, 128, 0, st>>>(op, cells, ncell, out);
  } else {
    if (op.compressed) decode_kernel<3, float, true><<<g, 128, 0, st>>>(op, cells, ncell, out);
    else if (op.elem64) decode_kernel<3, double, false><<<g, 128, 0, st>>>(op, cells, ncell, out);
    else decode_kernel<3, float, false><<<g, 128, 0, st>>>(op, cells, ncell, out);
  }
  return launched();
}

}  // namespace mg
