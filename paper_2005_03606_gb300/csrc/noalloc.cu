// Allocation-free assembly of the mixed-precision element data of a slab of
// cells (mg_assemble_surplus_noalloc in include/mg.h).
//
// Some callers cannot allocate device memory while they run: processes that
// plan their whole device footprint up front (a serving process with a fixed
// memory budget, an embedding application whose own allocator owns the
// device), and code paths where an allocation would synchronise the device
// or fragment a pool at the wrong moment.  This entry point lets them compute
// the stored element data into buffers they already own.  The intermediate
// data of the assembly (the per-cell records and the padded class bytes that
// the regular path keeps in a cudaMalloc'd scratch buffer) live instead in a
// fixed file-scope device array, so the call allocates nothing.
#include "mg_internal.cuh"
#include "mg.h"

#include <mutex>

namespace mg {
void eps_desc_to_dev(const mg_eps_desc& d, int dim, EpsDev* e);
mg_status eps_desc_check(const mg_eps_desc& d);
}

using namespace mg;

namespace {

// Scratch for one call: records (up to 112 bytes per cell) followed by the
// padded class bytes.  Every GPU that loads the library holds it until exit.
constexpr size_t kNoAllocScratchBytes = 64ull << 20;
static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {nullptr};

// device address of the scratch array on the current device (set up once per device)
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}

// classes and decoded surplus entries of the slab's cells from the scratch records
template <int D>
__global__ void unpack_kernel(int N, int nseg_x, long long ncell, const uint8_t* __restrict__ rec,
                              const uint8_t* __restrict__ cls_pad, uint8_t* __restrict__ out_cls,
                              float* __restrict__ out_surplus) {
  constexpr int NP = Dim<D>::NP;
  for (long long lc = blockIdx.x * (long long)blockDim.x + threadIdx.x; lc < ncell;
       lc += (long long)gridDim.x * blockDim.x) {
    const long long row = lc / N;
    const int x = (int)(lc - row * N);
    const int cls = cls_pad[(row * nseg_x + (x >> 5)) * kSegCells + (x & 31)];
    out_cls[lc] = (uint8_t)cls;
    const uint8_t* r = rec + (size_t)lc * Dim<D>::REC_MAX;
    for (int p = 0; p < NP; ++p) out_surplus[lc * NP + p] = cls ? decode_entry<D>(r, cls, p) : 0.f;
  }
}

}  // namespace

extern "C" mg_status mg_assemble_surplus_noalloc(const mg_eps_desc* eps, int dim, int n_cells, int s, double tau,
                                                 int64_t cell0, int64_t ncell, float* eps_c_out, uint8_t* cls_out,
                                                 float* surplus_out, void* cuda_stream) {
  if (!eps || !eps_c_out || !cls_out || !surplus_out || (dim != 2 && dim != 3) || n_cells < 3 || s < 1 ||
      s > 64 || ncell <= 0 || cell0 < 0) {
    set_error("mg_assemble_surplus_noalloc: bad arguments");
    return MG_ERR_INVALID;
  }
  // the same field checks as problem creation: the device tables hold at most
  // MG_MAX_MODES modes and MG_MAX_BOXES boxes, and eps must be positive
  if (eps_desc_check(*eps) != MG_OK) return MG_ERR_INVALID;
  const long long N = n_cells;
  const long long total = dim == 3 ? N * N * N : N * N;
  if (cell0 + ncell > total || cell0 % N != 0 || ncell % N != 0) {
    set_error("mg_assemble_surplus_noalloc: the cell range must be whole x-rows inside the grid");
    return MG_ERR_INVALID;
  }
  const int rec_max = dim == 3 ? Dim<3>::REC_MAX : Dim<2>::REC_MAX;
  const int nseg_x = (int)((N + kSegCells - 1) / kSegCells);
  const long long rows = ncell / N;
  // scratch rule: ncell * REC_MAX record bytes rounded up to 256, then
  // rows * ceil(N/32) * 32 padded class bytes, at most kNoAllocScratchBytes
  const size_t rec_bytes = (size_t)ncell * rec_max;
  const size_t rec_span = ((rec_bytes + 255) / 256) * 256;
  const size_t cls_bytes = (size_t)rows * nseg_x * kSegCells;
  if (rec_span + cls_bytes > kNoAllocScratchBytes) {
    set_error("mg_assemble_surplus_noalloc: %lld cells need %zu scratch bytes (ncell*%d rounded up to 256, plus "
              "%lld rows * %d padded class bytes); the limit is %zu",
              (long long)ncell, rec_span + cls_bytes, rec_max, rows, nseg_x * kSegCells, kNoAllocScratchBytes);
    return MG_ERR_INVALID;
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  void* base = nullptr;
  if (!cuda_ok(scratch_address(&base), "scratch address")) return MG_ERR_CUDA;
  uint8_t* rec = (uint8_t*)base;
  uint8_t* cls_pad = rec + rec_span;
  EpsDev F;
  eps_desc_to_dev(*eps, dim, &F);
  // cell-centre eps of the whole grid (the caller's eps_c_out holds n_cells^dim floats)
  if (!cuda_ok(launch_eps_centre(dim, (int)N, &F, 0, eps_c_out, st), "eps centre")) return MG_ERR_CUDA;
  if (s == 1) {   // one sample per cell: the surplus is zero by definition
    if (!cuda_ok(cudaMemsetAsync(cls_out, 0, (size_t)ncell, st), "memset") ||
        !cuda_ok(cudaMemsetAsync(surplus_out, 0, sizeof(float) * ncell * (dim == 3 ? 28 : 6), st), "memset"))
      return MG_ERR_CUDA;
    return MG_OK;
  }
  // the padding class bytes must read as class 0 (the array keeps the last call's contents)
  if (!cuda_ok(cudaMemsetAsync(cls_pad, 0, cls_bytes, st), "memset")) return MG_ERR_CUDA;
  AsmLaunch a{};
  a.dim = dim;
  a.N = (int)N;
  a.s = s;
  a.kind = F.kind;
  a.prec64 = 0;
  a.cell0 = cell0;
  a.ncell = ncell;
  a.eps_host = &F;
  a.hfac = dim == 3 ? 1.0 / (double)N : 1.0;
  a.eps_c = eps_c_out;
  a.out_rec = rec;
  a.out_cls = cls_pad;
  a.nseg_x = nseg_x;
  a.tau = tau > 0 ? tau : 1e-6;
  if (!cuda_ok(launch_assemble(a, st), "assemble")) return MG_ERR_CUDA;
  long long blocks = (ncell + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  if (dim == 3)
    unpack_kernel<3><<<(int)blocks, 256, 0, st>>>((int)N, nseg_x, ncell, rec, cls_pad, cls_out, surplus_out);
  else
    unpack_kernel<2><<<(int)blocks, 256, 0, st>>>((int)N, nseg_x, ncell, rec, cls_pad, cls_out, surplus_out);
  if (!cuda_ok(launched(), "unpack")) return MG_ERR_CUDA;
  return MG_OK;
}
