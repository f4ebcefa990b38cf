// Element-matrix integration at accuracy s (the paper's A^(geo)(n), Section
// "Numerical computation of stencils"), the hierarchical surplus against the
// geometric stencil and its lossy per-cell storage (Section "Precision
// toggling and information density"), and the packing of the stored records.
//
// Integration.  eps is constant on each of the s^d sub-boxes of a cell and
// taken at the sub-box centre x = (2(i s + j) + 1) / (2 N s).  In reference
// coordinates xi in [0,1]^d the element matrix is
//   A_pq = h^(d-2) sum_k sigma_k(p) sigma_k(q) int eps prod_{m != k} psi_{p_m} psi_{q_m}(xi_m) dxi,
// psi_0 = 1 - t, psi_1 = t, sigma = -1 / +1.  Per sub-box the integral
// factorises into 1D integrals of 1, (1-t)^2, t(1-t), t^2 over the sub-interval,
// so a cell needs, per derivative direction k, the 3^(d-1) sums
//   W_k[types of the other axes] = sum_sub eps' I_0(j_k) prod_{m != k} J_type(j_m)
// with J_00 = int (1-t)^2, J_01 = int t(1-t), J_11 = int t^2.  The kernel
// accumulates them row by row (a row = all sub-boxes with the same
// (j_y[, j_z])), first the x-sums S_0, S_1, S_2 = sum eps' {1, t1, t2}(j_x),
// then the row's 27 (3D) / 6 (2D) products.  eps' = eps - eps_c, so the result
// is directly the surplus A(s) - A(1) and A(1) = eps_c K_ref h^(d-2).
//
// Work split: one warp handles a batch of cells; the G lanes of a group share
// one cell (rows strided over the lanes) and reduce their partial sums with
// warp shuffles; 32/G cells are in flight per warp.
#include "mg_internal.cuh"

#include <algorithm>
#include <mutex>
#include <set>
#include <utility>
#include <vector>
#include <cstdio>
#include <climits>
#include <cmath>

namespace mg {

namespace {

constexpr int kAsmThreads = 256;
constexpr int kMaxS = 64;

template <typename T> __device__ __forceinline__ T t_exp(T x);
template <> __device__ __forceinline__ float t_exp<float>(float x) { return __expf(x); }
template <> __device__ __forceinline__ double t_exp<double>(double x) { return exp(x); }
template <typename T> __device__ __forceinline__ void t_sincospi(T x, T* s, T* c);
template <> __device__ __forceinline__ void t_sincospi<float>(float x, float* s, float* c) { sincospif(x, s, c); }
template <> __device__ __forceinline__ void t_sincospi<double>(double x, double* s, double* c) { sincospi(x, s, c); }
template <typename T> __device__ __forceinline__ T t_cospi(T x);
template <> __device__ __forceinline__ float t_cospi<float>(float x) { return cospif(x); }
template <> __device__ __forceinline__ double t_cospi<double>(double x) { return cospi(x); }

// sample coordinate (FP64, one IEEE division, as on the host)
__device__ __forceinline__ double sample_x(int N, int s, int i, int j) {
  return __ddiv_rn((double)(2 * (i * s + j) + 1), (double)(2 * N * s));
}

// fraction n/(N s) in [0,2) of the phase 2 pi k.x, from the exact integer
// k.(2 m + 1) mod 2 N s, m the global sub-index along each axis
__device__ __forceinline__ int phase_num(const EpsDev& F, int m, int D, const int* gm, int twoNs) {
  int acc = 0;
  for (int a = 0; a < D; ++a) {
    int t = (F.k[m][a] * (2 * gm[a] + 1)) % twoNs;
    acc += t;
  }
  acc %= twoNs;
  if (acc < 0) acc += twoNs;
  return acc;
}

// smooth part of theta field along one axis: exp(-theta x) cos(pi theta x)
template <typename T>
__device__ __forceinline__ T theta_factor(const EpsDev& F, double x) {
  return (T)(t_exp<T>((T)(-F.theta * x)) * t_cospi<T>((T)(F.theta * x)));
}

// field constants in the arithmetic precision T
template <typename T>
struct FieldT {
  T amp, v_out, v_in, jump_factor;
  __device__ __forceinline__ explicit FieldT(const EpsDev& F) {
    if (sizeof(T) == 4) {
      amp = (T)F.amp_f;
      v_out = (T)F.v_out_f;
      v_in = (T)F.v_in_f;
      jump_factor = (T)F.jump_factor_f;
    } else {
      amp = (T)F.amp;
      v_out = (T)F.v_out;
      v_in = (T)F.v_in;
      jump_factor = (T)F.jump_factor;
    }
  }
  __device__ __forceinline__ static T phi(const EpsDev& F, int m) {
    return sizeof(T) == 4 ? (T)F.phi_over_pi_f[m] : (T)F.phi_over_pi[m];
  }
};

// box membership of sample indices (m_x, m_y, m_z) through the integer thresholds
__device__ __forceinline__ bool in_box(const SampleThresholds& TH, int b, int D, const int* m) {
  bool in = true;
  for (int a = 0; a < D; ++a) in = in && TH.mlo[b][a] <= m[a] && m[a] < TH.mhi[b][a];
  return in;
}

// eps at the centre of every cell (s = 1), FP64 or FP32
template <int D, typename T>
__global__ void eps_centre_kernel(const EpsDev F, const SampleThresholds TH, int N, T* __restrict__ out) {
  long long ncell = 1;
  for (int a = 0; a < D; ++a) ncell *= N;
  const FieldT<T> FT(F);
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
       c += (long long)gridDim.x * blockDim.x) {
    int ci[3] = {0, 0, 0};
    long long t = c;
    for (int a = 0; a < D; ++a) {
      ci[a] = (int)(t % N);
      t /= N;
    }
    T e = FT.v_out;
    if (F.kind == EPS_DISC) {
      double r2 = 0.0;
      for (int a = 0; a < D; ++a) {
        double d = __dsub_rn(sample_x(N, 1, ci[a], 0), F.center[a]);
        r2 = __dadd_rn(r2, __dmul_rn(d, d));
      }
      e = r2 < F.r2lim ? FT.v_in : FT.v_out;
    } else if (F.kind == EPS_BOXES) {
      bool in = false;
      for (int b = 0; b < F.n_boxes && !in; ++b) in = in_box(TH, b, D, ci);
      e = in ? FT.v_in : FT.v_out;
    } else if (F.kind == EPS_THETA) {
      T p = (T)1;
      for (int a = 0; a < D; ++a) p *= theta_factor<T>(F, sample_x(N, 1, ci[a], 0));
      e = (T)1 + (T)(0.3 / D) * p;
    } else if (F.kind == EPS_FOURIER) {
      int gm[3] = {ci[0], ci[1], ci[2]};
      const int twoN = 2 * N;
      T g = 0;
      for (int m = 0; m < F.n_modes; ++m) {
        int n = phase_num(F, m, D, gm, twoN);
        T arg = (T)n / (T)N + FieldT<T>::phi(F, m);
        g += t_cospi<T>(arg);
      }
      e = FT.v_out * t_exp<T>(FT.amp * g);
    }
    if (ci[0] >= TH.mjump) e *= FT.jump_factor;
    out[c] = e;
  }
}

// per-sample x-axis data of a cell, in the arithmetic precision T (the
// discontinuity decisions behind `bits` and `jmul` are taken in FP64)
template <typename T>
struct XEntryT {
  unsigned long long bits;  // BOXES: mask of boxes whose x-interval holds the sample; DISC: dx^2 (FP64 bits)
  T jmul;                   // planar jump multiplier
  T th;                     // THETA: x-factor
};

template <typename T>
struct Cplx {   // (cos, sin) pair
  T c, s;
};

// MODES: compile-time bound of the Fourier mode loops (>= F.n_modes), so that
// the per-row phases stay in registers; FP32 instances and the
// piecewise-constant FP64 ones are held to two resident blocks per SM
template <int D, typename T, int KIND, int MODES>
__global__ void __launch_bounds__(kAsmThreads, (sizeof(T) == 4 || KIND == EPS_BOXES || KIND == EPS_DISC) ? 2 : 1)
    assemble_kernel(const EpsDev F, const SampleThresholds TH, const AsmLaunch A) {
  constexpr int NV = Dim<D>::NV, NP = Dim<D>::NP;
  constexpr int NW = D == 3 ? 27 : 6;
  const int N = A.N, s = A.s;
  __shared__ T s_t1[kMaxS], s_t2[kMaxS];
  __shared__ XEntryT<T> s_x[kAsmThreads / 32][64];
  // FP64 exact mode: a group's reduced moment sums, staged for its lanes
  // (at most 8 cell groups per warp in 3D, 16 in 2D)
  __shared__ T s_W[sizeof(T) == 8 ? kAsmThreads / 32 : 1][sizeof(T) == 8 ? (D == 3 ? 8 : 16) * NW : 1];
  const FieldT<T> FT(F);
  const T vin = FT.v_in, vout = FT.v_out;
  for (int j = threadIdx.x; j < s; j += blockDim.x) {
    s_t1[j] = (T)(2 * j + 1) / (T)(2 * s);
    s_t2[j] = (T)(3 * j * j + 3 * j + 1) / (T)(3 * s * s);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int R = 1;
  for (int a = 1; a < D; ++a) R *= s;
  int G = 1;
  while (G * 2 <= R && G < 32) G *= 2;
  const int CPW = 32 / G;
  const int grp = lane / G, lig = lane % G;
  // Fourier fields (dynamic shared memory, sized at the launch): the phase
  // e^{i pi (k.(2m + 1) / (N s) + phi)} of mode m at the global sample index m
  // is the cell's start phase C (at the cell's first sample) times the
  // per-axis rotations tX[jx] tY[jy] tZ[jz], tA[j] = e^{i pi 2 k_a j / (N s)}:
  // one rotation table per axis for the block, C per cell (computed by the
  // cell's lanes), so that a row costs two complex products per mode.  Modes
  // beyond n_modes are zero.  tX is [jx][MODES]: every lane of a warp reads the
  // same jx (a broadcast), at fixed offsets, two modes per 16-byte load in
  // FP32; tY and tZ are [MODES][s]: the lanes of a cell read different rows j
  // (consecutive j in consecutive banks).
  extern __shared__ __align__(16) unsigned char asm_dyn[];
  Cplx<T>* tX = reinterpret_cast<Cplx<T>*>(asm_dyn);
  Cplx<T>* tY = tX + (KIND == EPS_FOURIER ? MODES * s : 0);
  Cplx<T>* tZ = tY + (KIND == EPS_FOURIER ? MODES * s : 0);
  Cplx<T>* tC = tZ + (KIND == EPS_FOURIER && D == 3 ? MODES * s : 0);
  if (KIND == EPS_FOURIER) {
    for (int idx = threadIdx.x; idx < MODES * s; idx += blockDim.x) {
      const int j = idx / MODES, m = idx - j * MODES;
      for (int a = 0; a < D; ++a) {
        T sn = 0, cs = 0;
        if (m < F.n_modes) t_sincospi<T>((T)(2.0 * F.k[m][a] * j / ((double)N * s)), &sn, &cs);
        Cplx<T>* t = a == 0 ? tX + idx : (a == 1 ? tY : tZ) + m * s + j;
        t->c = cs;
        t->s = sn;
      }
    }
  }
  __syncthreads();
  // this group's cell start phases (groups MODES + 1 apart: the groups of a
  // warp read the same mode in different banks)
  Cplx<T>* cellC = tC + (warp * CPW + grp) * (MODES + 1);
  XEntryT<T>* xt = &s_x[warp][0];
  const int xt_stride = s;  // entries per group (CPW * s <= 64 by construction)
  const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
  const long long gwarp = (long long)blockIdx.x * (blockDim.x >> 5) + warp;
  const T* eps_c = reinterpret_cast<const T*>(A.eps_c);
  const T invs = (T)1 / (T)s;

  const long long count = A.list ? A.nlist : A.ncell;
  for (long long base = gwarp * CPW; base < count; base += nwarps * CPW) {
    const long long idx = base + grp;
    const bool valid = idx < count;
    const long long lc = !valid ? 0 : (A.list ? (long long)__ldg(A.list + idx) : idx);
    const long long c = A.cell0 + lc;
    int ci[3] = {0, 0, 0};
    {
      long long t = c;
      for (int a = 0; a < D; ++a) {
        ci[a] = (int)(t % N);
        t /= N;
      }
    }
    // reference of the surplus: the path's cell-centre eps (exact mode: FP64)
    const T eref = A.eps64 ? (T)A.eps64[c] : eps_c[c];
    // global sample indices of the cell's first sub-box along each axis
    const int m0[3] = {ci[0] * s, ci[1] * s, D == 3 ? ci[2] * s : 0};
    // x-axis table of the group's cell
    for (int jx = lig; jx < s; jx += G) {
      const int mx = m0[0] + jx;
      XEntryT<T> e;
      e.bits = 0;
      e.th = 0;
      e.jmul = mx >= TH.mjump ? FT.jump_factor : (T)1;
      if (KIND == EPS_BOXES) {
        unsigned long long m = 0;
        for (int b = 0; b < F.n_boxes; ++b)
          if (TH.mlo[b][0] <= mx && mx < TH.mhi[b][0]) m |= 1ull << b;
        e.bits = m;
      } else if (KIND == EPS_DISC) {
        double d = __dsub_rn(sample_x(N, s, ci[0], jx), F.center[0]);
        e.bits = (unsigned long long)__double_as_longlong(__dmul_rn(d, d));
      } else if (KIND == EPS_THETA) {
        e.th = theta_factor<T>(F, sample_x(N, s, ci[0], jx));
      }
      xt[grp * xt_stride + jx] = e;
    }
    if (KIND == EPS_FOURIER) {
      const int twoNs = 2 * N * s;
      for (int m = lig; m < MODES; m += G) {
        T sn = 0, cs = 0;
        if (m < F.n_modes) {
          const int n = phase_num(F, m, D, m0, twoNs);
          t_sincospi<T>((T)n / (T)(N * s) + FieldT<T>::phi(F, m), &sn, &cs);
        }
        cellC[m].c = cs;
        cellC[m].s = sn;
      }
    }
    __syncwarp();
    unsigned long long cand = 0;
    bool inside_all = false;
    if (KIND == EPS_BOXES) {
      // boxes holding some x-sample, kept only if their y (and z) range can hold
      // a sample of the cell too (a superset of the boxes that contain a
      // sample); inside_all: one box holds every sample of the cell
      unsigned long long xany = 0;
      for (int jx = 0; jx < s; ++jx) xany |= xt[grp * xt_stride + jx].bits;
      unsigned long long m = xany;
      while (m) {
        const int bx = __ffsll((long long)m) - 1;
        m &= m - 1;
        bool reach = true, all = true;
        for (int a = 0; a < D; ++a) {
          const int lo = TH.mlo[bx][a], hi = TH.mhi[bx][a];
          if (a > 0) reach = reach && lo <= m0[a] + s - 1 && m0[a] < hi;
          all = all && lo <= m0[a] && m0[a] + s - 1 < hi;
        }
        if (reach) cand |= 1ull << bx;
        inside_all = inside_all || all;
      }
    }
    // eps is the same at every sample of this cell (outside all boxes, or inside
    // one box): every sample equals the cell-centre value, the surplus is zero
    const bool flat = KIND == EPS_BOXES && TH.mjump == INT_MAX &&
                      ((cand == 0 && eref == vout) || (inside_all && eref == vin));

    T W[NW];
#pragma unroll
    for (int q = 0; q < NW; ++q) W[q] = 0;
    // Exact moments (FP64 exact mode, boxes or disc without a planar jump):
    // eps - eps_c is (v_in - v_out) times +-1 on the samples on the other side
    // of the discontinuity from the cell centre, and 0 elsewhere, so the
    // moment sums are integers: with D = 6 s^2, sum_x {1, t1, t2} over those
    // samples is {D n0, 3 s n1, 2 n2} / D (n1 = sum (2j + 1), n2 = sum
    // (3 j^2 + 3 j + 1)), and the J-type factors of the other axes are
    // integers over D too.  Accumulated in integers, scaled once.
    constexpr bool kIntPath = (KIND == EPS_BOXES || KIND == EPS_DISC) && sizeof(T) == 8;
    const bool use_int = kIntPath && A.eps64 != nullptr && TH.mjump == INT_MAX;
    T wscale = (T)1;
    const int Dd = 6 * s * s;
    const bool cin = eref == vin;   // the cell centre lies inside
    // one lane's rows, summed in AccT: a row adds at most 48 s^5 in magnitude,
    // so 32-bit sums hold a lane's rows for s <= 16; 64-bit ones beyond
    auto int_rows = [&](auto acc0) {
      using AccT = decltype(acc0);
      AccT WI[NW];
#pragma unroll
      for (int q = 0; q < NW; ++q) WI[q] = 0;
      for (int r = lig; r < R && valid && !flat; r += G) {
        const int jy = r % s, jz = (D == 3) ? r / s : 0;
        const int my = m0[1] + jy, mz = m0[2] + jz;
        unsigned long long rowbits = 0;
        double rowd = 0.0;
        if (KIND == EPS_BOXES) {
          unsigned long long cb = cand;
          while (cb) {
            int b = __ffsll((long long)cb) - 1;
            cb &= cb - 1;
            bool ok = TH.mlo[b][1] <= my && my < TH.mhi[b][1];
            if (D == 3) ok = ok && TH.mlo[b][2] <= mz && mz < TH.mhi[b][2];
            if (ok) rowbits |= 1ull << b;
          }
        } else {
          double dy = __dsub_rn(sample_x(N, s, ci[1], jy), F.center[1]);
          rowd = __dmul_rn(dy, dy);
          if (D == 3) {
            double dz = __dsub_rn(sample_x(N, s, ci[2], jz), F.center[2]);
            rowd = __dadd_rn(rowd, __dmul_rn(dz, dz));
          }
        }
        int n0 = 0, n1 = 0, n2 = 0;
        for (int jx = 0; jx < s; ++jx) {
          const XEntryT<T>& xe = xt[grp * xt_stride + jx];
          bool inside;
          if (KIND == EPS_BOXES) inside = (xe.bits & rowbits) != 0;
          else inside = __dadd_rn(__longlong_as_double((long long)xe.bits), rowd) < F.r2lim;
          if (inside != cin) {
            n0 += 1;
            n1 += 2 * jx + 1;
            n2 += 3 * jx * jx + 3 * jx + 1;
          }
        }
        const int X0 = Dd * n0, X1 = 3 * s * n1, X2 = 2 * n2;
        const int RJ[3] = {X0 - 2 * X1 + X2, X1 - X2, X2};
        const int Y1 = 3 * s * (2 * jy + 1), Y2 = 2 * (3 * jy * jy + 3 * jy + 1);
        const int Jy[3] = {Dd - 2 * Y1 + Y2, Y1 - Y2, Y2};
        if (D == 2) {
#pragma unroll
          for (int t = 0; t < 3; ++t) {
            WI[t] += (AccT)n0 * Jy[t];
            WI[3 + t] += RJ[t];
          }
        } else {
          const int Z1 = 3 * s * (2 * jz + 1), Z2 = 2 * (3 * jz * jz + 3 * jz + 1);
          const int Jz[3] = {Dd - 2 * Z1 + Z2, Z1 - Z2, Z2};
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            const int p0 = n0 * Jy[a];
#pragma unroll
            for (int b = 0; b < 3; ++b) {
              WI[a * 3 + b] += (AccT)p0 * Jz[b];
              WI[9 + a * 3 + b] += (AccT)RJ[a] * Jz[b];
              WI[18 + a * 3 + b] += (AccT)RJ[a] * Jy[b];
            }
          }
        }
      }
#pragma unroll
      for (int q = 0; q < NW; ++q) W[q] = (T)WI[q];
    };
    if (kIntPath && use_int) {
      if (s <= 16) int_rows(0);
      else int_rows(0LL);
      // the lanes' sums: integers below 2^53, exact in FP64
      for (int off = G / 2; off >= 1; off >>= 1) {
#pragma unroll
        for (int q = 0; q < NW; ++q) W[q] += __shfl_xor_sync(0xffffffffu, W[q], off);
      }
      const T dv = cin ? vout - vin : vin - vout;
      wscale = D == 3 ? dv / ((T)Dd * (T)Dd) : dv / (T)Dd;
    } else {
      for (int r = lig; r < R && valid && !flat; r += G) {
        const int jy = r % s, jz = (D == 3) ? r / s : 0;
        // per-row set-up
        unsigned long long rowbits = ~0ull;
        double rowd = 0.0;
        T rowth = (T)1;
        T P_re[KIND == EPS_FOURIER ? MODES : 1], P_im[KIND == EPS_FOURIER ? MODES : 1];
        const int my = m0[1] + jy, mz = m0[2] + jz;
        if (KIND == EPS_BOXES) {
          unsigned long long m = 0, cb = cand;
          while (cb) {
            int b = __ffsll((long long)cb) - 1;
            cb &= cb - 1;
            bool ok = TH.mlo[b][1] <= my && my < TH.mhi[b][1];
            if (D == 3) ok = ok && TH.mlo[b][2] <= mz && mz < TH.mhi[b][2];
            if (ok) m |= 1ull << b;
          }
          rowbits = m;
        } else if (KIND == EPS_DISC) {
          double dy = __dsub_rn(sample_x(N, s, ci[1], jy), F.center[1]);
          rowd = __dmul_rn(dy, dy);
        } else if (KIND == EPS_THETA) {
          rowth = theta_factor<T>(F, sample_x(N, s, ci[1], jy));
          if (D == 3) rowth = rowth * theta_factor<T>(F, sample_x(N, s, ci[2], jz));
        } else if (KIND == EPS_FOURIER) {
  #pragma unroll
          for (int m = 0; m < MODES; ++m) {   // (zero beyond n_modes)
            const Cplx<T> c = cellC[m], y = tY[m * s + jy];
            T ar = c.c * y.c - c.s * y.s, ai = c.c * y.s + c.s * y.c;
            if (D == 3) {
              const Cplx<T> z = tZ[m * s + jz];
              const T br = ar * z.c - ai * z.s;
              ai = ar * z.s + ai * z.c;
              ar = br;
            }
            P_re[m] = ar;
            P_im[m] = ai;
          }
        }
        double dz2 = 0.0;
        if (KIND == EPS_DISC && D == 3) {
          double dz = __dsub_rn(sample_x(N, s, ci[2], jz), F.center[2]);
          dz2 = __dmul_rn(dz, dz);
        }
        T S0 = 0, S1 = 0, S2 = 0;
        for (int jx = 0; jx < s; ++jx) {
          const XEntryT<T>& xe = xt[grp * xt_stride + jx];
          T e;
          if (KIND == EPS_CONST) {
            e = vout;
          } else if (KIND == EPS_BOXES) {
            e = (xe.bits & rowbits) ? vin : vout;
          } else if (KIND == EPS_DISC) {
            double r2 = __dadd_rn(__longlong_as_double((long long)xe.bits), rowd);
            if (D == 3) r2 = __dadd_rn(r2, dz2);
            e = r2 < F.r2lim ? vin : vout;
          } else if (KIND == EPS_THETA) {
            e = (T)1 + (T)(0.3 / D) * (xe.th * rowth);
          } else {
            // g = sum_m Re(P_m X_m[jx]) (modes beyond n_modes have P = 0)
            T g = 0;
            const Cplx<T>* xr = tX + jx * MODES;
            if (sizeof(T) == 4 && MODES % 2 == 0) {
              // two modes per 16-byte load, four independent partial sums
              const float4* x4 = reinterpret_cast<const float4*>(xr);
              T g0 = 0, g1 = 0, g2 = 0, g3 = 0;
  #pragma unroll
              for (int m = 0; m < MODES; m += 2) {
                const float4 x = x4[m / 2];
                g0 = fma(P_re[m], (T)x.x, g0);
                g1 = fma(P_im[m], (T)x.y, g1);
                g2 = fma(P_re[m + 1], (T)x.z, g2);
                g3 = fma(P_im[m + 1], (T)x.w, g3);
              }
              g = (g0 - g1) + (g2 - g3);
            } else {
  #pragma unroll
              for (int m = 0; m < MODES; ++m) {
                const Cplx<T> x = xr[m];
                g = fma(P_re[m], x.c, g);
                g = fma(-P_im[m], x.s, g);
              }
            }
            e = vout * t_exp<T>(FT.amp * g);
          }
          e *= xe.jmul;
          const T ep = e - eref;
          S0 += ep;
          S1 += ep * s_t1[jx];
          S2 += ep * s_t2[jx];
        }
        // J-type sums along x: (1-t)^2 = 1 - 2t + t^2, t(1-t) = t - t^2, t^2
        const T RJ[3] = {S0 - (T)2 * S1 + S2, S1 - S2, S2};
        const T t1y = s_t1[jy], t2y = s_t2[jy];
        const T jyv[3] = {(T)1 - (T)2 * t1y + t2y, t1y - t2y, t2y};
        if (D == 2) {
  #pragma unroll
          for (int t = 0; t < 3; ++t) {
            W[t] += S0 * jyv[t];      // d/dx term: other axis y
            W[3 + t] += RJ[t];        // d/dy term: other axis x
          }
        } else {
          const T t1z = s_t1[jz], t2z = s_t2[jz];
          const T jzv[3] = {(T)1 - (T)2 * t1z + t2z, t1z - t2z, t2z};
  #pragma unroll
          for (int a = 0; a < 3; ++a)
  #pragma unroll
            for (int b = 0; b < 3; ++b) {
              W[a * 3 + b] += S0 * jyv[a] * jzv[b];      // d/dx: (y, z)
              W[9 + a * 3 + b] += RJ[a] * jzv[b];        // d/dy: (x, z)
              W[18 + a * 3 + b] += RJ[a] * jyv[b];       // d/dz: (x, y)
            }
        }
      }
      // reduce over the group's lanes
      for (int off = G / 2; off >= 1; off >>= 1) {
  #pragma unroll
        for (int q = 0; q < NW; ++q) W[q] += __shfl_xor_sync(0xffffffffu, W[q], off);
      }
    }
    // FP64 exact mode without the adaptive test: the cell's epilogue is split
    // over its group's lanes (FP64 runs at a small fraction of the FP32 rate
    // here; one lane doing all of it left the FP64 pipe as the bound)
    const bool par_epi = sizeof(T) == 8 && !A.prec64 && !A.final_flags;
    if (par_epi) {
      if (valid) {
        const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (grp * G));
        T* Wg = &s_W[warp][grp * NW];
#pragma unroll
        for (int q = 0; q < NW; ++q)
          if (q % G == lig) Wg[q] = W[q];
        __syncwarp(gmask);
        T scale = (T)A.hfac * wscale;
        for (int a = 0; a < D; ++a) scale *= invs;
        const T ge = eref * (T)A.hfac;
        const T ge32 = (A.eps64 ? (T)reinterpret_cast<const float*>(A.eps_c)[c] : eref) * (T)A.hfac;
        // surplus entry (a, b), a < b, from the staged sums (as in the serial epilogue)
        auto dl_of = [&](int a, int b) -> T {
          T v = 0;
          for (int k = 0; k < D; ++k) {
            const T sg = (((a >> k) & 1) == ((b >> k) & 1)) ? (T)1 : (T)-1;
            int idx = 0;
            for (int m = 0; m < D; ++m)
              if (m != k) idx = idx * 3 + (((a >> m) & 1) + ((b >> m) & 1));
            v += sg * Wg[k * (NW / D) + idx];
          }
          return v * scale;
        };
        auto pair_ab = [&](int p, int* a, int* b) {
          int q = p, r = 0;
          while (q >= NV - 1 - r) {
            q -= NV - 1 - r;
            ++r;
          }
          *a = r;
          *b = r + 1 + q;
        };
        T Dm = 0, An = 0;
        for (int p = lig; p < NP; p += G) {
          int a, b;
          pair_ab(p, &a, &b);
          const T kv = (T)kref_off<D>(popc_small(a ^ b));
          const T v = dl_of(a, b);
          const T full = ge * kv + v;
          Dm = fmax(Dm, fabs(full - ge32 * kv));
          An = fmax(An, fabs(full));
        }
        for (int a = lig; a < NV; a += G) {   // diagonal entries: minus the row sums
          T rs = 0;
          for (int b = 0; b < NV; ++b)
            if (b != a) rs += dl_of(a < b ? a : b, a < b ? b : a);
          An = fmax(An, fabs(ge * (T)kref_diag<D>() - rs));
        }
        for (int off = G / 2; off >= 1; off >>= 1) {
          Dm = fmax(Dm, __shfl_xor_sync(gmask, Dm, off));
          An = fmax(An, __shfl_xor_sync(gmask, An, off));
        }
        const T Fm = (T)Dim<D>::F, tau = (T)A.tau;
        int cls;
        if (Fm * Dm <= tau * An) cls = 0;
        else if (Fm * Dm * ((T)16 / (T)448) <= tau * An) cls = 1;
        else if (Fm * Dm * ((T)16 / (T)65504) <= tau * An) cls = 2;
        else cls = 3;
        uint8_t* rec = A.out_rec + (size_t)lc * Dim<D>::REC_MAX;
        const float sc = cls == 1 ? (float)(Dm / (T)448) : (float)(Dm / (T)65504);
        if (lig == 0 && (cls == 1 || cls == 2)) *reinterpret_cast<float*>(rec) = sc;
        double* xo = A.out_x64 ? A.out_x64 + (size_t)A.xpos[c] * NP : nullptr;
        for (int p = lig; p < NP; p += G) {
          int a, b;
          pair_ab(p, &a, &b);
          const T kv = (T)kref_off<D>(popc_small(a ^ b));
          const T v = dl_of(a, b);
          const T d = ge * kv + v - ge32 * kv;
          if (xo) xo[p] = (double)v;
          if (cls == 1) {
            __nv_fp8_e4m3 q((float)(d / (T)sc));
            rec[4 + p] = q.__x;
          } else if (cls == 2) {
            *reinterpret_cast<__half*>(rec + 4 + 2 * p) = __float2half_rn((float)(d / (T)sc));
          } else if (cls == 3) {
            *reinterpret_cast<float*>(rec + 4 * p) = (float)d;
          }
        }
        if (lig == 0) {
          const long long row = lc / N;
          const int x = (int)(lc - row * N);
          A.out_cls[(row * A.nseg_x + (x >> 5)) * kSegCells + (x & 31)] = (uint8_t)cls;
        }
      }
    } else if (lig == 0 && valid) {
      T scale = (T)A.hfac * wscale;
      for (int a = 0; a < D; ++a) scale *= invs;
      T dl[NP];
#pragma unroll
      for (int a = 0; a < NV; ++a)
#pragma unroll
        for (int b = a + 1; b < NV; ++b) {
          T v = 0;
#pragma unroll
          for (int k = 0; k < D; ++k) {
            const T sg = (((a >> k) & 1) == ((b >> k) & 1)) ? (T)1 : (T)-1;
            int idx = 0;
#pragma unroll
            for (int m = 0; m < D; ++m)
              if (m != k) idx = idx * 3 + (((a >> m) & 1) + ((b >> m) & 1));
            v += sg * W[k * (NW / D) + idx];
          }
          dl[pair_index(NV, a, b)] = v * scale;
        }
      // adaptive accuracy, keep-old reading: a cell that passes the test keeps
      // its previously stored matrix (and accuracy)
      bool keep_prev = false;
      int pcls = 0;
      const uint8_t* prec = nullptr;
      if (A.final_flags) {
        // adaptive accuracy: relative change against the previously stored
        // matrix in the element-wise maximum norm (diagonals included)
        const T ge = eref * (T)A.hfac;
        pcls = A.prec64 ? 0 : cell_class(A.prev_cmp, N, A.nseg_x, lc);
        prec = pcls ? cell_record<D>(A.prev_cmp, N, A.nseg_x, lc, pcls) : nullptr;
        T num = 0, den = 0, rsn[NV], rso[NV];
#pragma unroll
        for (int a = 0; a < NV; ++a) rsn[a] = rso[a] = 0;
#pragma unroll
        for (int a = 0; a < NV; ++a)
#pragma unroll
          for (int b = a + 1; b < NV; ++b) {
            const int p = pair_index(NV, a, b);
            const T geo = ge * (T)kref_off<D>(popc_small(a ^ b));
            const T vn = geo + dl[p];
            T vo;
            if (A.prec64) vo = (T)A.prev_full[(long long)p * A.ncell + lc];
            else if (A.eps64) vo = geo + (A.prev_x64 ? (T)A.prev_x64[(size_t)A.xpos[c] * NP + p] : (T)0);
            else vo = geo + (pcls ? (T)decode_entry<D>(prec, pcls, p) : (T)0);
            num = fmax(num, fabs(vn - vo));
            den = fmax(den, fabs(vo));
            rsn[a] += vn;
            rsn[b] += vn;
            rso[a] += vo;
            rso[b] += vo;
          }
#pragma unroll
        for (int a = 0; a < NV; ++a) {
          num = fmax(num, fabs(rso[a] - rsn[a]));
          den = fmax(den, fabs(rso[a]));
        }
        const bool passed = num < (T)A.adapt_C * den;
        if (passed) A.final_flags[lc] = 1;
        keep_prev = passed && A.adapt_keep;
        if (!keep_prev) A.s_cell[lc] = (uint8_t)s;
      }
      if (A.prec64) {
        double* out = reinterpret_cast<double*>(A.out_full);
#pragma unroll
        for (int a = 0; a < NV; ++a)
#pragma unroll
          for (int b = a + 1; b < NV; ++b) {
            const int p = pair_index(NV, a, b);
            out[(long long)p * A.ncell + lc] =
                keep_prev ? A.prev_full[(long long)p * A.ncell + lc]
                          : (double)eref * kref_off<D>(popc_small(a ^ b)) * A.hfac + (double)dl[p];
          }
      } else if (keep_prev) {
        // the previous record and class (exact mode: the FP64 surplus array
        // already holds the previous level's entries)
        uint8_t* rec = A.out_rec + (size_t)lc * Dim<D>::REC_MAX;
        const int rb = pcls == 1 ? Dim<D>::REC1 : (pcls == 2 ? Dim<D>::REC2 : Dim<D>::REC3);
        if (pcls)
          for (int q = 0; q < rb; q += 4) *reinterpret_cast<uint32_t*>(rec + q) = *reinterpret_cast<const uint32_t*>(prec + q);
        const long long row = lc / N;
        const int x = (int)(lc - row * N);
        A.out_cls[(row * A.nseg_x + (x >> 5)) * kSegCells + (x & 31)] = (uint8_t)pcls;
      } else {
        // storage class from the surplus size (the oracle's rule; in FP32 on
        // the FP32 assembly, in FP64 in exact mode).  The records hold the
        // surplus against the FP32 cell-centre stencil: in exact mode the
        // integration ran against the FP64 one, and d = dl + (e64 - e32) K h.
        T Dm = 0, An = 0;
        T rs[NV], d32[NP];
#pragma unroll
        for (int a = 0; a < NV; ++a) rs[a] = 0;
        const T ge = eref * (T)A.hfac;
        const T ge32 = A.eps64 ? (T)reinterpret_cast<const float*>(A.eps_c)[c] * (T)A.hfac : ge;
#pragma unroll
        for (int a = 0; a < NV; ++a)
#pragma unroll
          for (int b = a + 1; b < NV; ++b) {
            const int p = pair_index(NV, a, b);
            const T kv = (T)kref_off<D>(popc_small(a ^ b));
            const T full = ge * kv + dl[p];
            const T d = full - ge32 * kv;
            d32[p] = A.eps64 ? d : dl[p];
            Dm = fmax(Dm, fabs(d32[p]));
            An = fmax(An, fabs(full));
            rs[a] += dl[p];
            rs[b] += dl[p];
          }
#pragma unroll
        for (int a = 0; a < NV; ++a) An = fmax(An, fabs(ge * (T)kref_diag<D>() - rs[a]));
        if (A.out_x64) {
          double* o = A.out_x64 + (size_t)A.xpos[c] * NP;
#pragma unroll
          for (int p = 0; p < NP; ++p) o[p] = (double)dl[p];
        }
        const T Fm = (T)Dim<D>::F, tau = (T)A.tau;
        int cls;
        if (Fm * Dm <= tau * An) cls = 0;
        else if (Fm * Dm * ((T)16 / (T)448) <= tau * An) cls = 1;
        else if (Fm * Dm * ((T)16 / (T)65504) <= tau * An) cls = 2;
        else cls = 3;
        uint8_t* rec = A.out_rec + (size_t)lc * Dim<D>::REC_MAX;
        if (cls == 1) {
          const float sc = (float)(Dm / (T)448);
          *reinterpret_cast<float*>(rec) = sc;
#pragma unroll
          for (int p = 0; p < NP; ++p) {
            __nv_fp8_e4m3 q((float)(d32[p] / (T)sc));
            rec[4 + p] = q.__x;
          }
        } else if (cls == 2) {
          const float sc = (float)(Dm / (T)65504);
          *reinterpret_cast<float*>(rec) = sc;
#pragma unroll
          for (int p = 0; p < NP; ++p)
            *reinterpret_cast<__half*>(rec + 4 + 2 * p) = __float2half_rn((float)(d32[p] / (T)sc));
        } else if (cls == 3) {
#pragma unroll
          for (int p = 0; p < NP; ++p) *reinterpret_cast<float*>(rec + 4 * p) = (float)d32[p];
        }
        const long long row = lc / N;
        const int x = (int)(lc - row * N);
        A.out_cls[(row * A.nseg_x + (x >> 5)) * kSegCells + (x & 31)] = (uint8_t)cls;
      }
    }
    __syncwarp();
  }
}

// FP64 full store of the geometric stencils eps_c K_ref h^(d-2) (s = 1)
template <int D>
__global__ void geometric_full_kernel(double hfac, const double* __restrict__ eps_c, long long cell0,
                                      long long ncell, double* __restrict__ out) {
  constexpr int NV = Dim<D>::NV;
  for (long long lc = blockIdx.x * (long long)blockDim.x + threadIdx.x; lc < ncell;
       lc += (long long)gridDim.x * blockDim.x) {
    const double e = eps_c[cell0 + lc] * hfac;
#pragma unroll
    for (int a = 0; a < NV; ++a)
#pragma unroll
      for (int b = a + 1; b < NV; ++b)
        out[(long long)pair_index(NV, a, b) * ncell + lc] = e * kref_off<D>(popc_small(a ^ b));
  }
}

// per-segment class counts (one warp per segment)
__global__ void pack_count_kernel(long long nseg, const uint8_t* __restrict__ cls,
                                  uint32_t* __restrict__ counts) {
  const int lane = threadIdx.x & 31;
  for (long long seg = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; seg < nseg;
       seg += ((long long)gridDim.x * blockDim.x) >> 5) {
    const int c = cls[seg * kSegCells + lane];
    for (int k = 1; k <= 3; ++k) {
      const unsigned m = __ballot_sync(0xffffffffu, c == k);
      if (lane == 0) counts[(k - 1) * nseg + seg] = __popc(m);
    }
  }
}

// exclusive scan of counts[k][0..nseg) in place, one block per class; totals[k]
__global__ void scan_kernel(long long nseg, uint32_t* __restrict__ counts, uint32_t* __restrict__ totals) {
  __shared__ uint32_t part[1024];
  uint32_t* c = counts + blockIdx.x * nseg;
  const long long per = (nseg + blockDim.x - 1) / blockDim.x;
  const long long b0 = threadIdx.x * per;
  const long long b1 = b0 + per < nseg ? b0 + per : nseg;
  uint32_t sum = 0;
  for (long long i = b0; i < b1; ++i) sum += c[i];
  part[threadIdx.x] = sum;
  __syncthreads();
  for (int off = 1; off < (int)blockDim.x; off <<= 1) {
    uint32_t v = threadIdx.x >= (unsigned)off ? part[threadIdx.x - off] : 0u;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  uint32_t run = part[threadIdx.x] - sum;
  for (long long i = b0; i < b1; ++i) {
    uint32_t v = c[i];
    c[i] = run;
    run += v;
  }
  if (threadIdx.x == blockDim.x - 1) totals[blockIdx.x] = part[threadIdx.x];
}

template <int D>
__global__ void pack_copy_kernel(long long nseg, const uint8_t* __restrict__ cls,
                                 const uint32_t* __restrict__ seg_base, int N, int nseg_x,
                                 const uint8_t* __restrict__ rec, uint8_t* __restrict__ p1,
                                 uint8_t* __restrict__ p2, uint8_t* __restrict__ p3) {
  const int lane = threadIdx.x & 31;
  for (long long seg = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; seg < nseg;
       seg += ((long long)gridDim.x * blockDim.x) >> 5) {
    const int c = cls[seg * kSegCells + lane];
    const long long row = seg / nseg_x;
    const int x = (int)(seg - row * nseg_x) * kSegCells + lane;
    for (int k = 1; k <= 3; ++k) {
      const unsigned m = __ballot_sync(0xffffffffu, c == k);
      if (c == k && x < N) {
        const unsigned r = __popc(m & ((1u << lane) - 1u));
        const int rb = k == 1 ? Dim<D>::REC1 : (k == 2 ? Dim<D>::REC2 : Dim<D>::REC3);
        uint8_t* dst = (k == 1 ? p1 : (k == 2 ? p2 : p3)) + (size_t)(seg_base[(k - 1) * nseg + seg] + r) * rb;
        const uint4* src = reinterpret_cast<const uint4*>(rec + (size_t)(row * N + x) * Dim<D>::REC_MAX);
        uint4* d4 = reinterpret_cast<uint4*>(dst);
        for (int q = 0; q < rb / 16; ++q) d4[q] = src[q];
      }
    }
  }
}

// x(m) = (2m + 1) / (2 N s), evaluated exactly as the FP64 sample position
double sample_x_host(int N, int s, long long m) { return (double)(2 * m + 1) / (double)(2 * (long long)N * s); }

// smallest m in [0, N s] with x(m) >= v (N s when there is none)
int first_at_or_above(double v, int N, int s) {
  const long long M = (long long)N * s;
  double t = std::floor((v * 2.0 * (double)M - 1.0) / 2.0) - 2.0;
  long long m = t < 0.0 ? 0 : (t > (double)M ? M : (long long)t);
  while (m < M && sample_x_host(N, s, m) < v) ++m;
  while (m > 0 && sample_x_host(N, s, m - 1) >= v) --m;
  return (int)m;
}

void make_thresholds(const EpsDev& F, int N, int s, SampleThresholds* TH) {
  for (int b = 0; b < kMaxBoxes; ++b)
    for (int a = 0; a < 3; ++a) {
      const bool used = F.kind == EPS_BOXES && b < F.n_boxes && a < F.dim;
      TH->mlo[b][a] = used ? first_at_or_above(F.box_lo[b][a], N, s) : 0;
      TH->mhi[b][a] = used ? first_at_or_above(F.box_hi[b][a], N, s) : 0;
    }
  TH->mjump = F.jump_factor != 1.0 ? first_at_or_above(F.jump_x, N, s) : INT_MAX;
}

int grid_for(long long work, int threads) {
  long long b = (work + threads - 1) / threads;
  if (b > 152LL * 64) b = 152LL * 64;
  if (b < 1) b = 1;
  return (int)b;
}

// raises a kernel's dynamic shared-memory limit once per device and kernel
cudaError_t opt_in_smem(const void* kern, size_t bytes) {
  static std::mutex mu;
  static std::set<std::pair<int, const void*>> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  if (done.count({dev, kern})) return cudaSuccess;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) done.insert({dev, kern});
  return e;
}

template <int D, typename T>
cudaError_t launch_assemble_t(const AsmLaunch& a, cudaStream_t st) {
  int R = 1;
  for (int d = 1; d < D; ++d) R *= a.s;
  int G = 1;
  while (G * 2 <= R && G < 32) G *= 2;
  const long long warps = ((a.list ? a.nlist : a.ncell) * G + 31) / 32;
  long long blocks = (warps + kAsmThreads / 32 - 1) / (kAsmThreads / 32);
  const long long cap = 152LL * 16;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  const EpsDev& F = *a.eps_host;
  SampleThresholds TH;
  make_thresholds(F, a.N, a.s, &TH);
  // Fourier tables: D rotation tables [n_modes][s] and the cell start phases
  // [warps][cells per warp][MODES], as complex pairs
  auto fourier_launch = [&](auto kern, int modes) -> cudaError_t {
    const size_t bytes =
        sizeof(Cplx<T>) * ((size_t)D * modes * a.s + (size_t)(kAsmThreads / 32) * (32 / G) * (modes + 1));
    // static plus dynamic shared memory may pass the 48 KB default: opt in once
    // per instance (assembly runs on several host threads), for its largest
    // footprint (s = kMaxS, eight cell groups per warp)
    cudaError_t e = opt_in_smem((const void*)kern,
                                sizeof(Cplx<T>) * ((size_t)D * modes * kMaxS + (size_t)(kAsmThreads / 32) * 8 * (modes + 1)));
    if (e != cudaSuccess) return e;
    kern<<<(int)blocks, kAsmThreads, bytes, st>>>(F, TH, a);
    return cudaSuccess;
  };
  switch (F.kind) {
    case EPS_CONST: assemble_kernel<D, T, EPS_CONST, 1><<<(int)blocks, kAsmThreads, 0, st>>>(F, TH, a); break;
    case EPS_DISC: assemble_kernel<D, T, EPS_DISC, 1><<<(int)blocks, kAsmThreads, 0, st>>>(F, TH, a); break;
    case EPS_FOURIER: {
      cudaError_t e;
      if (F.n_modes <= 8) e = fourier_launch(assemble_kernel<D, T, EPS_FOURIER, 8>, 8);
      else if (F.n_modes <= 16) e = fourier_launch(assemble_kernel<D, T, EPS_FOURIER, 16>, 16);
      else e = fourier_launch(assemble_kernel<D, T, EPS_FOURIER, kMaxModes>, kMaxModes);
      if (e != cudaSuccess) return e;
      break;
    }
    case EPS_BOXES: assemble_kernel<D, T, EPS_BOXES, 1><<<(int)blocks, kAsmThreads, 0, st>>>(F, TH, a); break;
    case EPS_THETA: assemble_kernel<D, T, EPS_THETA, 1><<<(int)blocks, kAsmThreads, 0, st>>>(F, TH, a); break;
    default: return cudaErrorInvalidValue;
  }
  return launched();
}

// Interface cells: a discontinuity crosses the open cell.  Cells touched only
// on their boundary are flat (sample points lie strictly inside); decisions
// carry a margin of 1e-9 h, so rounding can only add cells.
//  - boxes and the planar jump: the cells crossed by a face form a box of cell
//    indices (the face's cell layer times the box's overlap range in the other
//    axes), found on the host and marked here;
//  - the disc: one thread per cell.
struct CellRegion {
  int lo[3], hi[3];   // inclusive cell index ranges
};

__global__ void mark_regions_kernel(const CellRegion* __restrict__ regions, const long long* __restrict__ start,
                                    int nreg, int dim, int N, uint8_t* __restrict__ flags) {
  const long long total = start[nreg];
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    int r = 0, rh = nreg - 1;   // the region with start[r] <= t < start[r + 1]
    while (r < rh) {
      const int mid = (r + rh + 1) / 2;
      if (start[mid] <= t) r = mid;
      else rh = mid - 1;
    }
    const CellRegion& g = regions[r];
    long long u = t - start[r];
    int ci[3] = {0, 0, 0};
    for (int a = 0; a < dim; ++a) {
      const int w = g.hi[a] - g.lo[a] + 1;
      ci[a] = g.lo[a] + (int)(u % w);
      u /= w;
    }
    const long long c = dim == 3 ? ((long long)ci[2] * N + ci[1]) * N + ci[0] : (long long)ci[1] * N + ci[0];
    flags[c] = 1;
  }
}

template <int D>
__global__ void mark_disc_kernel(const EpsDev F, int N, uint8_t* __restrict__ flags) {
  long long ncell = 1;
  for (int a = 0; a < D; ++a) ncell *= N;
  const double h = 1.0 / N;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
       c += (long long)gridDim.x * blockDim.x) {
    long long t = c;
    double dmin = 0.0, dmax = 0.0;
    for (int a = 0; a < D; ++a) {
      const int ci = (int)(t % N);
      t /= N;
      const double lo = ci * h, hi = (ci + 1) * h, x = F.center[a];
      const double near = x < lo ? lo - x : (x > hi ? x - hi : 0.0);
      const double far = fmax(fabs(x - lo), fabs(x - hi));
      dmin += near * near;
      dmax += far * far;
    }
    if (dmin <= F.r2lim * (1.0 + 1e-9) && dmax >= F.r2lim * (1.0 - 1e-9)) flags[c] = 1;
  }
}

// local index of every flagged cell appended to its chunk's list
// Ordered compaction of the flagged cells into per-chunk lists (local cell
// indices, ascending): tiles of kListTile cells per chunk count their flags,
// one block per chunk scans the tile counts, and each tile writes its cells
// at its offset in cell order (so that two problems with the same field get
// the same list, and data kept in list order can move between them).
constexpr int kListTile = 1024;

__global__ void __launch_bounds__(kListTile) list_tile_count_kernel(long long chunk_cells, int ntpc,
                                                                    const uint8_t* __restrict__ flags,
                                                                    int* __restrict__ tcount) {
  const int ch = blockIdx.x / ntpc, t = blockIdx.x % ntpc;
  const long long lc = (long long)t * kListTile + threadIdx.x;
  const int f = lc < chunk_cells && flags[(long long)ch * chunk_cells + lc] ? 1 : 0;
  const int n = __syncthreads_count(f);
  if (threadIdx.x == 0) tcount[blockIdx.x] = n;
}

__global__ void __launch_bounds__(1024) list_tile_scan_kernel(int ntpc, int* __restrict__ tcount,
                                                              int* __restrict__ counts) {
  __shared__ int part[1024];
  int* c = tcount + (long long)blockIdx.x * ntpc;
  const int per = (ntpc + blockDim.x - 1) / blockDim.x;
  const int b0 = threadIdx.x * per, b1 = min(b0 + per, ntpc);
  int sum = 0;
  for (int i = b0; i < b1; ++i) sum += c[i];
  part[threadIdx.x] = sum;
  __syncthreads();
  for (int off = 1; off < (int)blockDim.x; off <<= 1) {
    const int v = threadIdx.x >= (unsigned)off ? part[threadIdx.x - off] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  int run = part[threadIdx.x] - sum;
  for (int i = b0; i < b1; ++i) {
    const int v = c[i];
    c[i] = run;
    run += v;
  }
  if (threadIdx.x == blockDim.x - 1) counts[blockIdx.x] = part[threadIdx.x];
}

__global__ void __launch_bounds__(kListTile) list_tile_write_kernel(long long chunk_cells, int ntpc,
                                                                    const uint8_t* __restrict__ flags,
                                                                    const int* __restrict__ toff,
                                                                    int* __restrict__ lists) {
  __shared__ int wsum[kListTile / 32];
  const int ch = blockIdx.x / ntpc, t = blockIdx.x % ntpc;
  const long long lc = (long long)t * kListTile + threadIdx.x;
  const bool f = lc < chunk_cells && flags[(long long)ch * chunk_cells + lc];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned m = __ballot_sync(0xffffffffu, f);
  if (lane == 0) wsum[warp] = __popc(m);
  __syncthreads();
  int before = 0;
  for (int w = 0; w < warp; ++w) before += wsum[w];
  if (f) {
    const int pos = toff[blockIdx.x] + before + __popc(m & ((1u << lane) - 1u));
    lists[(long long)ch * chunk_cells + pos] = (int)lc;
  }
}

// cells (inclusive range) whose closed interval meets [a, b] (with margin), and
// whose open interval contains x (with margin; lo > hi when none)
void overlap_range(double a, double b, int N, int* lo, int* hi) {
  const double h = 1.0 / N, tol = 1e-9 * h;
  *lo = N;
  *hi = -1;
  for (int c = 0; c < N; ++c)
    if (a <= (c + 1) * h + tol && b >= c * h - tol) {
      *lo = std::min(*lo, c);
      *hi = std::max(*hi, c);
    }
}
void face_range(double x, int N, int* lo, int* hi) {
  const double h = 1.0 / N, tol = 1e-9 * h;
  *lo = N;
  *hi = -1;
  for (int c = 0; c < N; ++c)
    if (x > c * h - tol && x < (c + 1) * h + tol) {
      *lo = std::min(*lo, c);
      *hi = std::max(*hi, c);
    }
}

// adaptive accuracy: the final cells' previous matrices into the new store
template <int D>
__global__ void carry_final_kernel(long long ncell, int N, int nseg_x, const uint8_t* __restrict__ flags,
                                   const CmpChunk prev, uint8_t* __restrict__ out_rec, uint8_t* __restrict__ out_cls,
                                   uint8_t* __restrict__ s_cell, int s, int first) {
  for (long long lc = blockIdx.x * (long long)blockDim.x + threadIdx.x; lc < ncell;
       lc += (long long)gridDim.x * blockDim.x) {
    if (!flags[lc]) continue;
    if (first) s_cell[lc] = (uint8_t)s;
    const int cls = cell_class(prev, N, nseg_x, lc);
    const long long row = lc / N;
    const int x = (int)(lc - row * N);
    out_cls[(row * nseg_x + (x >> 5)) * kSegCells + (x & 31)] = (uint8_t)cls;
    if (cls) {
      const uint8_t* src = cell_record<D>(prev, N, nseg_x, lc, cls);
      const int bytes = cls == 1 ? Dim<D>::REC1 : (cls == 2 ? Dim<D>::REC2 : Dim<D>::REC3);
      uint8_t* dst = out_rec + (size_t)lc * Dim<D>::REC_MAX;
      for (int i = 0; i < bytes; ++i) dst[i] = src[i];
    }
  }
}

__global__ void carry_final64_kernel(long long ncell, int np, const uint8_t* __restrict__ flags,
                                     const double* __restrict__ prev, double* __restrict__ out,
                                     uint8_t* __restrict__ s_cell, int s, int first) {
  for (long long lc = blockIdx.x * (long long)blockDim.x + threadIdx.x; lc < ncell;
       lc += (long long)gridDim.x * blockDim.x) {
    if (!flags[lc]) continue;
    if (first) s_cell[lc] = (uint8_t)s;
    for (int p = 0; p < np; ++p) out[(long long)p * ncell + lc] = prev[(long long)p * ncell + lc];
  }
}

// work list: the candidate cells (cand, or 0 .. ncand-1) that are not final
__global__ void adaptive_work_kernel(long long ncand, const int* __restrict__ cand, const uint8_t* __restrict__ flags,
                                     int* __restrict__ work, int* __restrict__ nwork) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < ncand;
       t += (long long)gridDim.x * blockDim.x) {
    const int lc = cand ? cand[t] : (int)t;
    if (!flags[lc]) work[atomicAdd(nwork, 1)] = lc;
  }
}

__global__ void clear_listed_kernel(long long n, const int* __restrict__ list, uint8_t* __restrict__ flags) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    flags[list[t]] = 0;
}

}  // namespace

cudaError_t launch_adaptive_prepare(int dim, int N, int nseg_x, long long chunk_cells, int prec64,
                                    const uint8_t* final_flags, const CmpChunk& prev_cmp, const double* prev_full,
                                    uint8_t* out_rec, uint8_t* out_cls, double* out_full, const int* cand,
                                    long long ncand, int* work, int* nwork, uint8_t* s_cell, int s, int first,
                                    cudaStream_t st) {
  const int g = grid_for(chunk_cells, 256);
  if (prec64) {
    carry_final64_kernel<<<g, 256, 0, st>>>(chunk_cells, dim == 3 ? 28 : 6, final_flags, prev_full, out_full, s_cell,
                                            s, first);
  } else if (dim == 3) {
    carry_final_kernel<3><<<g, 256, 0, st>>>(chunk_cells, N, nseg_x, final_flags, prev_cmp, out_rec, out_cls, s_cell,
                                             s, first);
  } else {
    carry_final_kernel<2><<<g, 256, 0, st>>>(chunk_cells, N, nseg_x, final_flags, prev_cmp, out_rec, out_cls, s_cell,
                                             s, first);
  }
  cudaError_t e = launched();
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(nwork, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  if (ncand > 0) adaptive_work_kernel<<<grid_for(ncand, 256), 256, 0, st>>>(ncand, cand, final_flags, work, nwork);
  return launched();
}

cudaError_t launch_adaptive_init(long long chunk_cells, int nchunk, const int* lists, const int* counts_host,
                                 uint8_t* final_flags, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(final_flags, 1, (size_t)chunk_cells * nchunk, st);
  for (int c = 0; c < nchunk && e == cudaSuccess; ++c) {
    if (counts_host[c] <= 0) continue;
    clear_listed_kernel<<<grid_for(counts_host[c], 256), 256, 0, st>>>(counts_host[c], lists + (size_t)c * chunk_cells,
                                                                     final_flags + (size_t)c * chunk_cells);
    e = launched();
  }
  return e;
}

cudaError_t launch_interface_cells(int dim, int N, const EpsDev* eps, long long chunk_cells, int* lists,
                                   int* counts, cudaStream_t st) {
  if (eps->kind != EPS_BOXES && eps->kind != EPS_DISC && eps->kind != EPS_CONST) return cudaErrorNotSupported;
  const long long ncell = (long long)N * N * (dim == 3 ? N : 1);
  uint8_t* flags = nullptr;
  cudaError_t e = mg_malloc_async(&flags, (size_t)ncell, st);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(flags, 0, (size_t)ncell, st);
  // face regions of the boxes and of the planar jump
  std::vector<CellRegion> regs;
  auto add_face = [&](int axis, double x, const int* olo, const int* ohi) {
    int flo, fhi;
    face_range(x, N, &flo, &fhi);
    if (flo > fhi) return;
    CellRegion g{};
    for (int a = 0; a < 3; ++a) {
      g.lo[a] = a < dim ? olo[a] : 0;
      g.hi[a] = a < dim ? ohi[a] : 0;
    }
    g.lo[axis] = flo;
    g.hi[axis] = fhi;
    for (int a = 0; a < dim; ++a)
      if (g.lo[a] > g.hi[a]) return;
    regs.push_back(g);
  };
  if (eps->kind == EPS_BOXES) {
    for (int b = 0; b < eps->n_boxes; ++b) {
      int olo[3], ohi[3];
      bool any = true;
      for (int a = 0; a < dim; ++a) {
        overlap_range(eps->box_lo[b][a], eps->box_hi[b][a], N, &olo[a], &ohi[a]);
        any = any && olo[a] <= ohi[a];
      }
      if (!any) continue;
      for (int a = 0; a < dim; ++a) {
        add_face(a, eps->box_lo[b][a], olo, ohi);
        add_face(a, eps->box_hi[b][a], olo, ohi);
      }
    }
  }
  if (eps->jump_factor != 1.0) {
    const int olo[3] = {0, 0, 0}, ohi[3] = {N - 1, N - 1, N - 1};
    add_face(0, eps->jump_x, olo, ohi);
  }
  CellRegion* d_regs = nullptr;
  long long* d_start = nullptr;
  std::vector<long long> start(regs.size() + 1, 0);
  for (size_t r = 0; r < regs.size(); ++r) {
    long long v = 1;
    for (int a = 0; a < dim; ++a) v *= regs[r].hi[a] - regs[r].lo[a] + 1;
    start[r + 1] = start[r] + v;
  }
  if (e == cudaSuccess && !regs.empty()) {
    e = mg_malloc_async(&d_regs, sizeof(CellRegion) * regs.size(), st);
    if (e == cudaSuccess) e = mg_malloc_async(&d_start, sizeof(long long) * start.size(), st);
    // pageable sources: staged before the calls return
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_regs, regs.data(), sizeof(CellRegion) * regs.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_start, start.data(), sizeof(long long) * start.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
      mark_regions_kernel<<<grid_for(start.back(), 256), 256, 0, st>>>(d_regs, d_start, (int)regs.size(), dim, N,
                                                                        flags);
      e = launched();
    }
  }
  if (e == cudaSuccess && eps->kind == EPS_DISC) {
    if (dim == 2) mark_disc_kernel<2><<<grid_for(ncell, 256), 256, 0, st>>>(*eps, N, flags);
    else mark_disc_kernel<3><<<grid_for(ncell, 256), 256, 0, st>>>(*eps, N, flags);
    e = launched();
  }
  if (e == cudaSuccess) {
    const int nchunk = (int)(ncell / chunk_cells);
    const int ntpc = (int)((chunk_cells + kListTile - 1) / kListTile);
    int* tcount = nullptr;
    e = mg_malloc_async(&tcount, sizeof(int) * (size_t)nchunk * ntpc, st);
    if (e == cudaSuccess) {
      list_tile_count_kernel<<<nchunk * ntpc, kListTile, 0, st>>>(chunk_cells, ntpc, flags, tcount);
      e = launched();
    }
    if (e == cudaSuccess) {
      list_tile_scan_kernel<<<nchunk, 1024, 0, st>>>(ntpc, tcount, counts);
      e = launched();
    }
    if (e == cudaSuccess) {
      list_tile_write_kernel<<<nchunk * ntpc, kListTile, 0, st>>>(chunk_cells, ntpc, flags, tcount, lists);
      e = launched();
    }
    if (tcount) cudaFreeAsync(tcount, st);
  }
  if (d_regs) cudaFreeAsync(d_regs, st);
  if (d_start) cudaFreeAsync(d_start, st);
  cudaFreeAsync(flags, st);
  return e;
}

cudaError_t launch_eps_centre(int dim, int N, const EpsDev* eps, int prec64, void* eps_c, cudaStream_t st) {
  SampleThresholds TH;
  make_thresholds(*eps, N, 1, &TH);
  long long ncell = (long long)N * N * (dim == 3 ? N : 1);
  int g = grid_for(ncell, 256);
  if (dim == 2) {
    if (prec64) eps_centre_kernel<2, double><<<g, 256, 0, st>>>(*eps, TH, N, (double*)eps_c);
    else eps_centre_kernel<2, float><<<g, 256, 0, st>>>(*eps, TH, N, (float*)eps_c);
  } else {
    if (prec64) eps_centre_kernel<3, double><<<g, 256, 0, st>>>(*eps, TH, N, (double*)eps_c);
    else eps_centre_kernel<3, float><<<g, 256, 0, st>>>(*eps, TH, N, (float*)eps_c);
  }
  return launched();
}

cudaError_t launch_assemble(const AsmLaunch& a, cudaStream_t st) {
  if (a.s < 1 || a.s > kMaxS) return cudaErrorInvalidValue;
  const bool f64 = a.prec64 || a.eps64;   // FP64 arithmetic: FP64 paths and the exact mode
  if (a.dim == 2) return f64 ? launch_assemble_t<2, double>(a, st) : launch_assemble_t<2, float>(a, st);
  return f64 ? launch_assemble_t<3, double>(a, st) : launch_assemble_t<3, float>(a, st);
}

cudaError_t launch_geometric_full(int dim, int N, double hfac, const double* eps_c, long long cell0,
                                  long long ncell, double* out, cudaStream_t st) {
  (void)N;
  int g = grid_for(ncell, 256);
  if (dim == 2) geometric_full_kernel<2><<<g, 256, 0, st>>>(hfac, eps_c, cell0, ncell, out);
  else geometric_full_kernel<3><<<g, 256, 0, st>>>(hfac, eps_c, cell0, ncell, out);
  return launched();
}

cudaError_t launch_pack_count(int dim, int N, long long nrows, int nseg_x, const uint8_t* cls,
                              uint32_t* seg_base, uint32_t* totals, cudaStream_t st) {
  (void)dim;
  (void)N;
  const long long nseg = nrows * nseg_x;
  pack_count_kernel<<<grid_for(nseg * 32, 256), 256, 0, st>>>(nseg, cls, seg_base);
  cudaError_t e = launched();
  if (e != cudaSuccess) return e;
  scan_kernel<<<3, 1024, 0, st>>>(nseg, seg_base, totals);
  return launched();
}

cudaError_t launch_pack_copy(int dim, int N, long long nrows, int nseg_x, const uint8_t* cls,
                             const uint32_t* seg_base, const uint8_t* rec, uint8_t* p1, uint8_t* p2,
                             uint8_t* p3, cudaStream_t st) {
  const long long nseg = nrows * nseg_x;
  const int g = grid_for(nseg * 32, 256);
  if (dim == 2) pack_copy_kernel<2><<<g, 256, 0, st>>>(nseg, cls, seg_base, N, nseg_x, rec, p1, p2, p3);
  else pack_copy_kernel<3><<<g, 256, 0, st>>>(nseg, cls, seg_base, N, nseg_x, rec, p1, p2, p3);
  return launched();
}

}  // namespace mg
