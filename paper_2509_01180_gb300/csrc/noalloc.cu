// bh_expand_noalloc: the expansion for callers that cannot allocate device memory at call time.
//
// Who needs it: code that runs where cudaMalloc is unavailable or forbidden once work has started --
// a host thread feeding a stream that is being captured into a CUDA graph by someone else, an
// allocator-free real-time loop, or an embedding application that owns all device memory and only
// lends pointers.  bh_expand itself allocates nothing per call either, but it needs the scratch that
// bh_plan_create sized with max_batch; this entry point instead stages the gathered volumes and the
// GEMM output in one fixed array compiled into the library, so its per-call footprint is independent
// of the plan's max_batch.
//
// The scratch is a file-scope __device__ array of kStaticScratchBytes (64 MiB).  Every GPU on which
// the library's module is loaded holds it until the process exits.  Host code cannot use the array's
// name as a device address (it is a host-side stand-in), so the first call on each device looks the
// address up with cudaGetSymbolAddress while that device is current and caches it; make that first
// call before any stream capture.  All calls share the array and it keeps the last call's contents:
// every pass overwrites the rows and columns it reads (including padding), so nothing needs clearing,
// but calls whose work overlaps on the GPU (different streams, or different plans at once) race on it.
#include <mutex>

#include "bh_internal.h"

namespace {

constexpr size_t kStaticScratchBytes = 64ull << 20;
static __device__ __align__(256) unsigned char g_expand_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 128;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

int scratch_address(void** out) {
  int dev = 0;
  BH_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return bh::fail(BH_ERR_UNSUPPORTED, "device ordinal %d", dev);
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_expand_scratch);
    if (e != cudaSuccess || !ptr)
      return bh::fail(BH_ERR_CUDA, "cudaGetSymbolAddress(static expansion scratch): %s", cudaGetErrorString(e));
    g_scratch_ptr[dev] = ptr;
  }
  *out = g_scratch_ptr[dev];
  return BH_OK;
}

}  // namespace

extern "C" int bh_expand_noalloc(bh_plan* p, const float* vols, int B, float* coeffs, void* stream) {
  bh::clear_error();
  const bh::Range range_("bh_expand_noalloc");
  if (!p) return bh::fail(BH_ERR_ARG, "plan is NULL");
  if (B < 0) return bh::fail(BH_ERR_ARG, "B=%d", B);
  if (B == 0) return BH_OK;
  if (!vols || !coeffs) return bh::fail(BH_ERR_ARG, "vols or coeffs is NULL");
  // the plan's tables and tensor maps live on its own device; the scratch looked up below must be that
  // device's copy of the array
  {
    int st = bh::check_plan_device(p);
    if (st == BH_OK) st = bh::check_expansion_plan(p);
    if (st != BH_OK) return st;
  }
  // bytes per row of the 128-row M tile: the volume's 8 parity-class projections over the fundamental voxels
  // (FP32, or BF16 hi + lo) + the real GEMM output (FP32)
  const size_t row_bytes = (size_t)8 * p->VF_pad * 4 + (size_t)p->Nb_pad * 4;
  const size_t tile_rows = bh::kGemmBM;
  // 256 bytes are held back for the alignment of the GEMM-output region
  int rows_cap = (int)((kStaticScratchBytes - 256) / row_bytes) / (int)tile_rows * (int)tile_rows;
  if (rows_cap < (int)tile_rows)
    return bh::fail(BH_ERR_ARG,
                    "bh_expand_noalloc: one %zu-row pass of this plan (N=%d, Lmax=%d) needs %zu bytes of scratch, "
                    "more than the fixed %zu; use bh_expand",
                    tile_rows, p->N, p->Lmax, tile_rows * row_bytes, kStaticScratchBytes);
  if (rows_cap > B) rows_cap = (int)bh::round_up(B, (int)tile_rows);
  void* base = nullptr;
  int st = scratch_address(&base);
  if (st != BH_OK) return st;
  unsigned char* b = static_cast<unsigned char*>(base);
  const size_t x_bytes = bh::round_up64((int64_t)rows_cap * 8 * p->VF_pad * 4, 256);
  float* c = reinterpret_cast<float*>(b + x_bytes);
  return bh::expand_into(p, vols, nullptr, B, coeffs, b, c, rows_cap, static_cast<cudaStream_t>(stream));
}
