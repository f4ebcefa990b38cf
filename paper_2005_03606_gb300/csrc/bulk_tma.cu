// Geometric bulk pass of the finest-level FP32 sweep, staged through shared
// memory by the Tensor Memory Accelerator.
//
// Arithmetic (the same as the register-only bulk pass in sweep.cu): with
// 12 K_ref = 5 I + E - J for the trilinear reference matrix,
//   (A u)_v = h/12 [ 5 u_v G_v + sum_{axis neighbours w} W_vw u_w - sum_c eps_c T_c ],
// G_v = sum of eps over the 8 cells at v, W_vw = sum of eps over the 4 cells
// sharing edge vw, T_c = sum of u over the 8 vertices of cell c; cell sums
// are formed separably and carried along the z march.
//
// Data movement.  A CTA owns tiles of 128 (x) by 8 (y) vertices by kTZ planes
// (z).  For every plane p of a tile (p = k0-1 .. k1+1) one ring stage holds
// the u rows j0-1 .. j0+8 of plane p, the eps rows of cell layer p and the b
// rows of plane p, each one TMA box (3D tensor maps, x from q0-4 so that the
// box starts on a 16-byte boundary; out-of-range boxes read zeros).  Output
// plane k is formed once the stage of plane k+1 has landed, from stages
// k-1 .. k+1; the stage of plane k-1 is then refilled kS-2 stages ahead.  The
// producer (thread 0) runs ahead across tile boundaries, so the pipeline does
// not drain between tiles.  Every wait on a stage barrier is bounded: on a
// timeout the CTA records an error code and leaves.
#include "mg_internal.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

namespace mg {
namespace {

constexpr int kS = 5;                  // ring stages (3 in use, kS - 2 in flight)
constexpr int kTX = 128, kTY = 8;      // tile: vertices in x (32 lanes x 4) and rows in y (8 warps)
constexpr int kTZ = 8;                 // output planes per tile
constexpr int kUW = kTX + 8;           // u / eps box width: x = q0-4 .. q0+131
constexpr int kUBytes = (kTY + 2) * kUW * 4;   // u rows j0-1 .. j0+8
constexpr int kEBytes = (kTY + 1) * kUW * 4;   // eps cell rows j0-1 .. j0+7
constexpr int kBBytes = kTY * kTX * 4;         // b rows j0 .. j0+7
constexpr int kUOff = 0;
constexpr int kEOff = (kUBytes + 127) / 128 * 128;
constexpr int kBOff = kEOff + (kEBytes + 127) / 128 * 128;
constexpr int kStage = kBOff + kBBytes;
constexpr int kSmem = kS * kStage + 128;
constexpr long long kWaitLimit = 1ll << 22;   // try_wait polls per stage before giving up

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait for the phase with the given parity
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (long long i = 0; i < kWaitLimit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void tma_load3(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
          "r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

struct BulkArgs {
  float* y;
  double* partials;
  int* err;
  int N, ntx, nty, ntiles;
  float h12, omega;
};

// stage sequence of one CTA: its tiles (round robin) and, per tile, planes k0-1 .. k1+1
struct StageIt {
  int tile, t, k0, nk, q0, j0;
  __device__ void set_tile(const BulkArgs& a, int tl) {
    tile = tl;
    t = 0;
    if (tl < a.ntiles) {
      const int tx = tl % a.ntx, ty = (tl / a.ntx) % a.nty, tz = tl / (a.ntx * a.nty);
      q0 = tx * kTX;
      j0 = 1 + ty * kTY;
      k0 = 1 + tz * kTZ;
      nk = min(a.N - 1, k0 + kTZ - 1) - k0 + 1;
    }
  }
  __device__ bool valid(const BulkArgs& a) const { return tile < a.ntiles; }
  __device__ void next(const BulkArgs& a) {
    if (++t == nk + 2) set_tile(a, tile + gridDim.x);
  }
};

__device__ __forceinline__ void issue_stage(const StageIt& it, uint8_t* smem, uint64_t* full, int slot,
                                            const CUtensorMap* tmu, const CUtensorMap* tme, const CUtensorMap* tmb) {
  const int p = it.k0 - 1 + it.t;
  const bool need_e = it.t <= it.nk;               // eps layer p is read for planes p and p+1
  const bool need_b = it.t >= 1 && it.t <= it.nk;  // b of output planes only
  const uint32_t bar = smem_addr(&full[slot]);
  const uint32_t bytes = kUBytes + (need_e ? kEBytes : 0) + (need_b ? kBBytes : 0);
  mbar_expect_tx(bar, bytes);
  uint8_t* st = smem + (size_t)slot * kStage;
  tma_load3(smem_addr(st + kUOff), tmu, it.q0 - 4, it.j0 - 1, p, bar);
  if (need_e) tma_load3(smem_addr(st + kEOff), tme, it.q0 - 4, it.j0 - 1, p, bar);
  if (need_b) tma_load3(smem_addr(st + kBOff), tmb, it.q0, it.j0, p, bar);
}

// u of rows r0 .. r0+2 of a stage at the thread's columns x = q-1 .. q+4
// (halo values from the neighbouring lanes; lanes 0 and 31 read them)
__device__ __forceinline__ void rows_from_stage(const float* U, int r0, int lane, float (&v)[3][6]) {
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const float* row = U + (r0 + r) * kUW;
    const float4 c = *reinterpret_cast<const float4*>(row + 4 + 4 * lane);
    float left = __shfl_up_sync(0xffffffffu, c.w, 1);
    float right = __shfl_down_sync(0xffffffffu, c.x, 1);
    if (lane == 0) left = row[3];
    if (lane == 31) right = row[8 + 4 * 31];
    v[r][0] = left;
    v[r][1] = c.x;
    v[r][2] = c.y;
    v[r][3] = c.z;
    v[r][4] = c.w;
    v[r][5] = right;
  }
}

// eps of cells x = q-1 .. q+3 of cell rows r0, r0+1 of a stage
__device__ __forceinline__ void eps_from_stage(const float* E, int r0, int lane, float (&g)[2][5]) {
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const float* row = E + (r0 + r) * kUW;
    const float4 c = *reinterpret_cast<const float4*>(row + 4 + 4 * lane);
    float left = __shfl_up_sync(0xffffffffu, c.w, 1);
    if (lane == 0) left = row[3];
    g[r][0] = left;
    g[r][1] = c.x;
    g[r][2] = c.y;
    g[r][3] = c.z;
    g[r][4] = c.w;
  }
}

__device__ __forceinline__ void pair_sums6(const float (&u)[3][6], float (&py)[2][5]) {
  float px[3][5];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 5; ++c) px[r][c] = u[r][c] + u[r][c + 1];
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int c = 0; c < 5; ++c) py[r][c] = px[r][c] + px[r + 1][c];
}

template <int MODE>
__global__ void __launch_bounds__(256, 2) geo_bulk_tma(const __grid_constant__ CUtensorMap tmu,
                                                       const __grid_constant__ CUtensorMap tme,
                                                       const __grid_constant__ CUtensorMap tmb, const BulkArgs a) {
  extern __shared__ __align__(128) uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full[kS];
  // TMA destinations on 128-byte boundaries (the launch adds 128 bytes of slack)
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  __shared__ double sh[2][8];
  const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
  const int N = a.N, n1 = N + 1;
  const size_t plane = (size_t)n1 * n1;
  const float h12 = a.h12, h3 = 4.f * a.h12;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kS; ++s) mbar_init(smem_addr(&full[s]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  StageIt prod, cons;
  prod.set_tile(a, blockIdx.x);
  cons.set_tile(a, blockIdx.x);
  long long gp = 0;   // stages issued (thread 0)
  if (threadIdx.x == 0) {
    for (; gp < kS - 2 && prod.valid(a); ++gp, prod.next(a))
      issue_stage(prod, smem, full, (int)(gp % kS), &tmu, &tme, &tmb);
  }
  float d1 = 0.f, d2 = 0.f;
  float gm[2][5], pyc[2][5], yTm[5];
  bool failed = false;
  for (long long g = 0; cons.valid(a); ++g, cons.next(a)) {
    const int slot = (int)(g % kS);
    const bool ok = mbar_wait(smem_addr(&full[slot]), (uint32_t)((g / kS) & 1));
    const uint8_t* cur = smem + (size_t)slot * kStage;
    const float* Ucur = reinterpret_cast<const float*>(cur + kUOff);
    if (cons.t == 0) {   // plane k0-1: pair sums; eps layer k0-1
      float u0[3][6];
      rows_from_stage(Ucur, wy, lane, u0);
      pair_sums6(u0, pyc);
      eps_from_stage(reinterpret_cast<const float*>(cur + kEOff), wy, lane, gm);
    } else if (cons.t == 1) {   // plane k0: weighted cell sums of layer k0-1
      float u1[3][6], py1[2][5];
      rows_from_stage(Ucur, wy, lane, u1);
      pair_sums6(u1, py1);
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        yTm[c] = gm[0][c] * (pyc[0][c] + py1[0][c]) + gm[1][c] * (pyc[1][c] + py1[1][c]);
        pyc[0][c] = py1[0][c];
        pyc[1][c] = py1[1][c];
      }
    } else {   // output plane k = p - 1 from the stages of planes k-1, k, k+1
      const int k = cons.k0 + cons.t - 2;
      const uint8_t* prv = smem + (size_t)((g + kS - 1) % kS) * kStage;
      const uint8_t* pp = smem + (size_t)((g + kS - 2) % kS) * kStage;
      float un[3][6], uc[3][6], pyn[2][5], gc[2][5];
      rows_from_stage(Ucur, wy, lane, un);
      rows_from_stage(reinterpret_cast<const float*>(prv + kUOff), wy, lane, uc);
      eps_from_stage(reinterpret_cast<const float*>(prv + kEOff), wy, lane, gc);
      const float4 m4 = *reinterpret_cast<const float4*>(reinterpret_cast<const float*>(pp + kUOff) +
                                                         (wy + 1) * kUW + 4 + 4 * lane);
      const float4 b4 = *reinterpret_cast<const float4*>(reinterpret_cast<const float*>(prv + kBOff) + wy * kTX +
                                                         4 * lane);
      pair_sums6(un, pyn);
      float yTc[5], ez[2][5], ey[5], elm[5], elc[5];
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        yTc[c] = gc[0][c] * (pyc[0][c] + pyn[0][c]) + gc[1][c] * (pyc[1][c] + pyn[1][c]);
        ez[0][c] = gm[0][c] + gc[0][c];
        ez[1][c] = gm[1][c] + gc[1][c];
        ey[c] = ez[0][c] + ez[1][c];
        elm[c] = gm[0][c] + gm[1][c];
        elc[c] = gc[0][c] + gc[1][c];
      }
      const float bb4[4] = {b4.x, b4.y, b4.z, b4.w};
      const float um1[4] = {m4.x, m4.y, m4.z, m4.w};
      const int q = cons.q0 + 4 * lane, j = cons.j0 + wy;
      float out[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float uv = uc[1][e + 1];
        const float G = ey[e] + ey[e + 1];
        const float ST = (yTm[e] + yTm[e + 1]) + (yTc[e] + yTc[e + 1]);
        float w = 5.f * uv * G - ST;
        w = fmaf(ey[e], uc[1][e], w);                         // x - 1
        w = fmaf(ey[e + 1], uc[1][e + 2], w);                 // x + 1
        w = fmaf(ez[0][e] + ez[0][e + 1], uc[0][e + 1], w);   // y - 1
        w = fmaf(ez[1][e] + ez[1][e + 1], uc[2][e + 1], w);   // y + 1
        w = fmaf(elm[e] + elm[e + 1], um1[e], w);             // z - 1
        w = fmaf(elc[e] + elc[e + 1], un[1][e + 1], w);       // z + 1
        const float acc = h12 * w;
        const int i = q + e;
        const bool valid = i >= 1 && i <= N - 1 && j <= N - 1;
        float r;
        if (MODE == SW_JACOBI) r = uv + a.omega * __fdividef(bb4[e] - acc, h3 * G);
        else if (MODE == SW_RESID) r = bb4[e] - acc;
        else {
          r = acc;
          if (valid) {
            d1 += uv * acc;
            d2 += uv * bb4[e];
          }
        }
        out[e] = valid ? r : 0.f;   // boundary vertices stay zero
      }
      if (q < n1 && j <= N - 1)
        *reinterpret_cast<float4*>(a.y + (size_t)k * plane + (size_t)j * n1 + q) =
            make_float4(out[0], out[1], out[2], out[3]);
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        pyc[0][c] = pyn[0][c];
        pyc[1][c] = pyn[1][c];
        yTm[c] = yTc[c];
        gm[0][c] = gc[0][c];
        gm[1][c] = gc[1][c];
      }
    }
    // every thread is done with the stage of plane p-2: refill its slot kS-2 stages ahead
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    if (threadIdx.x == 0 && prod.valid(a)) {
      issue_stage(prod, smem, full, (int)(gp % kS), &tmu, &tme, &tmb);
      ++gp;
      prod.next(a);
    }
  }
  if (failed) {
    if (threadIdx.x == 0) {
      atomicExch(a.err, 1);
      // let the copies still in flight land before the CTA leaves (bounded)
      for (long long s = 0; s < kS; ++s) mbar_wait(smem_addr(&full[s]), 0u), mbar_wait(smem_addr(&full[s]), 1u);
    }
    __syncthreads();
  }
  if (MODE == SW_MATVEC) {
    double v1 = (double)d1, v2 = (double)d2;
    for (int off = 16; off >= 1; off >>= 1) {
      v1 += __shfl_xor_sync(0xffffffffu, v1, off);
      v2 += __shfl_xor_sync(0xffffffffu, v2, off);
    }
    if (lane == 0) {
      sh[0][wy] = v1;
      sh[1][wy] = v2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double s1 = 0.0, s2 = 0.0;
      for (int w = 0; w < 8; ++w) {
        s1 += sh[0][w];
        s2 += sh[1][w];
      }
      a.partials[2 * blockIdx.x] = s1;
      a.partials[2 * blockIdx.x + 1] = s2;
    }
  }
}

__global__ void pad_eps_kernel(int N, const float* __restrict__ src, float* __restrict__ dst) {
  const int n1 = N + 1;
  const long long total = (long long)N * N * n1;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(t % n1);
    const long long row = t / n1;
    dst[t] = x < N ? src[row * N + x] : 0.f;
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

bool encode3(CUtensorMap* m, const void* base, int dx, int dy, int dz, int bx, int by) {
  auto enc = encoder();
  if (!enc) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)dx, (cuuint64_t)dy, (cuuint64_t)dz};
  const cuuint64_t strides[2] = {(cuuint64_t)dx * 4, (cuuint64_t)dx * dy * 4};
  const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(base), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int MODE>
cudaError_t launch_mode(const CUtensorMap& mu, const CUtensorMap& me, const CUtensorMap& mb, const BulkArgs& a,
                        int grid, cudaStream_t st) {
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [] {
    attr = cudaFuncSetAttribute(geo_bulk_tma<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
  });
  if (attr != cudaSuccess) return attr;
  geo_bulk_tma<MODE><<<grid, 256, kSmem, st>>>(mu, me, mb, a);
  return cudaSuccess;
}

}  // namespace

bool geo_bulk_tma_usable(const LevelOp& op, const void* x, const void* b) {
  return op.eps_pad && op.err && encoder() && ((uintptr_t)x % 16) == 0 && ((uintptr_t)b % 16) == 0 &&
         (op.N + 1) % 4 == 0;
}

cudaError_t launch_geo_bulk_tma(const LevelOp& op, int mode, const float* x, const float* b, float* y, float omega,
                                double* partials, int* nblocks, cudaStream_t st) {
  const int N = op.N, n1 = N + 1;
  CUtensorMap mu, me, mb;
  if (!encode3(&mu, x, n1, n1, n1, kUW, kTY + 2) || !encode3(&mb, b, n1, n1, n1, kTX, kTY) ||
      !encode3(&me, op.eps_pad, n1, N, N, kUW, kTY + 1))
    return cudaErrorInvalidValue;
  BulkArgs a;
  a.y = y;
  a.partials = partials;
  a.err = op.err;
  a.N = N;
  a.ntx = (n1 + kTX - 1) / kTX;
  a.nty = (N - 1 + kTY - 1) / kTY;
  a.ntiles = a.ntx * a.nty * ((N - 1 + kTZ - 1) / kTZ);
  a.h12 = -op.gk32;
  a.omega = omega;
  static int nsm = 0;
  if (!nsm) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (nsm <= 0) nsm = 152;
  }
  const int grid = a.ntiles < 2 * nsm ? a.ntiles : 2 * nsm;
  if (nblocks) *nblocks = grid;
  cudaError_t e;
  if (mode == SW_JACOBI) e = launch_mode<SW_JACOBI>(mu, me, mb, a, grid, st);
  else if (mode == SW_RESID) e = launch_mode<SW_RESID>(mu, me, mb, a, grid, st);
  else e = launch_mode<SW_MATVEC>(mu, me, mb, a, grid, st);
  if (e != cudaSuccess) return e;
  return launched();
}

cudaError_t launch_pad_eps(int N, const float* eps_c, float* eps_pad, cudaStream_t st) {
  pad_eps_kernel<<<152 * 8, 256, 0, st>>>(N, eps_c, eps_pad);
  return launched();
}

}  // namespace mg
