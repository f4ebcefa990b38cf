// The paper's own storage format for the hierarchical surplus (Section
// "Precision toggling and information density"), applied to a level's stored
// operator: mg_paper_format in include/mg.h.
//
// An entry held with p3 bytes (2 <= p3 < 8) keeps a sign bit, a truncated
// mantissa of m = 8 (p3 - 1) - 1 bits and a signed-char exponent without bias;
// p3 = 8 is plain FP64 and p3 = 0 stores nothing.  A cell's p3 is 0 when the
// Frobenius norm of its surplus A - eps_c K is below the absolute threshold
// delta, else the smallest p3 whose truncation error is at most delta in every
// entry.  Here the truncation works on the IEEE-754 encoding: inside the
// format's exponent range it clears the low 52 - m mantissa bits; below 2^-127
// the format has no normalised encoding and holds multiples of 2^-(127 + m);
// at or above 2^128 it saturates.  The surplus and its norm are formed with
// explicitly rounded operations (no fused multiply-add), entry by entry in
// row-major order, so that the byte choice is reproducible.
#include "mg_internal.cuh"
#include "mg.h"

namespace mg {
namespace {

__device__ __forceinline__ double pow2(int k) {   // 2^k for -1022 <= k <= 1023
  return __longlong_as_double((long long)(k + 1023) << 52);
}

__device__ double pf_trunc(double x, int p3) {
  if (p3 >= 8) return x;
  if (p3 <= 0 || x == 0.0) return 0.0;
  const int m = 8 * (p3 - 1) - 1;
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const unsigned long long sign = bits & 0x8000000000000000ull;
  const int E = (int)((bits >> 52) & 0x7FF);
  const int e = E - 1023;   // unbiased exponent of a normal double
  unsigned long long r;
  if (E != 0 && e > 127) {
    // largest encoding (2 - 2^-m) 2^127: exponent 127, the top m mantissa bits set
    const unsigned long long man = ((1ull << m) - 1) << (52 - m);
    r = ((unsigned long long)(127 + 1023) << 52) | man;
  } else if (E != 0 && e >= -127) {
    r = (bits & 0x7FFFFFFFFFFFFFFFull) & ~((1ull << (52 - m)) - 1);
  } else {
    // non-normalised range: multiples of 2^-(127 + m) (exact power-of-two scalings)
    const double a = fabs(x);
    const double q = floor(a * pow2(127 + m));
    r = (unsigned long long)__double_as_longlong(q * pow2(-(127 + m)));
  }
  return __longlong_as_double((long long)(sign | r));
}

template <int D>
__global__ void paper_format_kernel(long long ncell, const double* __restrict__ A, const void* __restrict__ eps_c,
                                    int eps64, double hfac, double delta, uint8_t* __restrict__ p3_out,
                                    double* __restrict__ At, unsigned long long* __restrict__ hist,
                                    unsigned long long* __restrict__ maxerr_bits) {
  constexpr int NV = 1 << D, NE = NV * NV;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
       c += (long long)gridDim.x * blockDim.x) {
    const double ec = eps64 ? reinterpret_cast<const double*>(eps_c)[c]
                            : (double)reinterpret_cast<const float*>(eps_c)[c];
    const double* a = A + c * NE;
    double dA[NE], g[NE];
    double f2 = 0.0;
#pragma unroll
    for (int i = 0; i < NE; ++i) {
      const int r = i / NV, q = i % NV;
      const double k = r == q ? kref_diag<D>() : kref_off<D>(popc_small(r ^ q));
      g[i] = __dmul_rn(ec, __dmul_rn(k, hfac));
      dA[i] = __dsub_rn(a[i], g[i]);
      f2 = __dadd_rn(f2, __dmul_rn(dA[i], dA[i]));
    }
    int p3 = 0;
    if (!(sqrt(f2) < delta)) {
      p3 = 8;
      for (int t = 2; t <= 7; ++t) {
        double err = 0.0;
#pragma unroll
        for (int i = 0; i < NE; ++i) err = fmax(err, fabs(__dsub_rn(dA[i], pf_trunc(dA[i], t))));
        if (err <= delta) {
          p3 = t;
          break;
        }
      }
    }
    p3_out[c] = (uint8_t)p3;
    atomicAdd(hist + p3, 1ull);
    double emax = 0.0;
#pragma unroll
    for (int i = 0; i < NE; ++i) {
      const double st = __dadd_rn(g[i], pf_trunc(dA[i], p3));
      if (At) At[c * NE + i] = st;
      emax = fmax(emax, fabs(__dsub_rn(st, a[i])));
    }
    // non-negative doubles order like their bit patterns
    atomicMax(maxerr_bits, (unsigned long long)__double_as_longlong(emax));
  }
}

}  // namespace

// The stored operator of a level as full FP64 matrices (A), its one-sample
// matrices eps_c K h^(d-2), and the format's p3 per cell; hist[9] and
// *maxerr_bits (the bits of a non-negative double) accumulate on the device.
cudaError_t launch_paper_format(int dim, long long ncell, const double* A, const void* eps_c, int eps64,
                                double hfac, double delta, uint8_t* p3_out, double* At, unsigned long long* hist,
                                unsigned long long* maxerr_bits, cudaStream_t st) {
  if (ncell <= 0) return cudaSuccess;
  long long nb = (ncell + 127) / 128;
  if (nb > 152LL * 32) nb = 152LL * 32;
  if (dim == 3)
    paper_format_kernel<3><<<(unsigned)nb, 128, 0, st>>>(ncell, A, eps_c, eps64, hfac, delta, p3_out, At, hist,
                                                         maxerr_bits);
  else
    paper_format_kernel<2><<<(unsigned)nb, 128, 0, st>>>(ncell, A, eps_c, eps64, hfac, delta, p3_out, At, hist,
                                                         maxerr_bits);
  return launched();
}

}  // namespace mg
