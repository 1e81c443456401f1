// Internal declarations shared by the libbh translation units (not part of the ABI).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <map>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/bh.h"

namespace bh {

// Record a message for bh_last_error() and return `code`.
int fail(int code, const char* fmt, ...);
void clear_error();

// NVTX range spanning a C-ABI call (shown on profiler timelines; a no-op without an attached tool).
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};

// Sphere-normalised associated Legendre functions with the Condon-Shortley phase, P[l * (L+1) + m] for
// 0 <= m <= l <= L (Y_l^m = P_l^m(cos theta) e^{i m phi}); FP64, host.
void legendre_all(int L, double x, double* P);

#define BH_CUDA_TRY(call)                                                                           \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess)                                                                          \
      return ::bh::fail(e_ == cudaErrorMemoryAllocation ? BH_ERR_OOM : BH_ERR_CUDA, "%s: %s (%s:%d)", \
                        #call, cudaGetErrorString(e_), __FILE__, __LINE__);                         \
  } while (0)

#define BH_CHECK_LAUNCH()                                                                           \
  do {                                                                                              \
    cudaError_t e_ = cudaGetLastError();                                                            \
    if (e_ != cudaSuccess)                                                                          \
      return ::bh::fail(BH_ERR_CUDA, "kernel launch: %s (%s:%d)", cudaGetErrorString(e_), __FILE__, \
                        __LINE__);                                                                  \
  } while (0)

constexpr int kMaxL = 64;
constexpr int kMaxDevices = 128;

// Ordinal of the current CUDA device in *dev (BH_ERR_CUDA if the runtime cannot say, BH_ERR_UNSUPPORTED
// beyond kMaxDevices).
inline int current_device(int* dev) {
  BH_CUDA_TRY(cudaGetDevice(dev));
  if (*dev < 0 || *dev >= kMaxDevices) return fail(BH_ERR_UNSUPPORTED, "device ordinal %d", *dev);
  return BH_OK;
}

// Kernel attributes set by cudaFuncSetAttribute belong to the device that was current at the call, so the
// record of what was already raised is kept per device.  ensure_smem raises a kernel's dynamic shared-memory
// limit only when a larger size is requested on this device, so that launches recorded into a CUDA graph
// after a first (warm-up) call make no attribute calls.
struct SmemAttr {
  std::atomic<int> have[kMaxDevices] = {};
};
template <typename K>
int ensure_smem(K kernel, SmemAttr& attr, size_t smem) {
  int dev = 0;
  const int st = current_device(&dev);
  if (st != BH_OK) return st;
  if ((int)smem <= attr.have[dev].load()) return BH_OK;
  BH_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  BH_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
  attr.have[dev].store((int)smem);
  return BH_OK;
}

inline int round_up(int x, int m) { return (x + m - 1) / m * m; }
inline int64_t round_up64(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// Coefficient layout passed by value to kernels: off[l] = first slot of degree l, K[l] = roots kept.
struct Layout {
  int Lmax;
  int Nb;
  int off[kMaxL + 2];
  int K[kMaxL + 1];
};

// GEMM tiling of the expansion (tensor-core and FP32 forms).
constexpr int kGemmBM = 128;
constexpr int kGemmBN = 128;  // every parity class of table rows is padded to a multiple of the N tile
constexpr int kGemmBK = 64;
constexpr int kPadV = 64;     // the fundamental voxels are padded to a multiple of the K block

// Octant folding of the expansion GEMM: table rows come class by class (8 parity classes), N tiles
// [ntile_end[c-1], ntile_end[c]) belong to class c, and class c's projected volumes are the rows
// [c rows, (c+1) rows) of the X operand.  rows = 0 turns the mapping off (one plain GEMM).
struct ClassMap {
  int ntile_end[8];
  int rows;
};
__host__ __device__ inline int class_of_ntile(const ClassMap& cm, int nt) {
  int c = 0;
  while (c < 7 && nt >= cm.ntile_end[c]) ++c;
  return c;
}

}  // namespace bh

struct bh_plan {
  int device = -1;
  int N = 0, Lmax = 0, mode = 0, max_batch = 0;
  bool match_only = false;          // BH_PLAN_MATCH_ONLY: no expansion table or scratch
  double lam_max = 0;
  int V = 0, Nb = 0, Nb_pad = 0, M_cap = 0;  // in-ball voxels, coefficients, padded table rows, rows/pass
  int VF = 0, VF_pad = 0;                     // fundamental voxels (x, y, z >= 0) = the GEMM's K
  bh::ClassMap cls{};                         // N tiles of each parity class (rows set per launch)
  std::vector<int> K, offs;         // per degree
  std::vector<double> lam, cst;     // lambda_lk, c_lk flattened by degree
  bh::Layout layout{};

  int* d_fund = nullptr;            // [VF] fundamental voxel coordinates x | y << 10 | z << 20
  int2* d_slot = nullptr;           // [Nb] real-GEMM columns feeding each complex slot (signed, 1-based)
  float* d_T32 = nullptr;           // [Nb_pad][VF_pad] basis table by parity class, FP32 mode
  __nv_bfloat16* d_Thi = nullptr;   // [Nb_pad][VF_pad] BF16 hi part
  __nv_bfloat16* d_Tlo = nullptr;   // [Nb_pad][VF_pad] BF16 lo part
  float* d_X32 = nullptr;           // [8][M_cap][VF_pad] projected volumes per class (FP32 mode)
  __nv_bfloat16* d_Xhi = nullptr;   // [8][M_cap][VF_pad] projected volumes, hi part
  __nv_bfloat16* d_Xlo = nullptr;   // [8][M_cap][VF_pad] lo part
  float* d_C = nullptr;             // [ksplit_max][M_cap][Nb_pad] real GEMM output (per K split)
  int* d_err = nullptr;             // device status word written by bounded waits
  float* d_P = nullptr;             // orbit-table scale P_l(m,n), layout [m][l][n] for l <= Lmax
  float* d_lbin = nullptr;          // 0.5 log2 C(2m, m+n) at [m][m+n], row stride 2 kMaxL + 1
  double2* d_coef64 = nullptr;      // (B_l, g_l) of the rescaled d recursion in FP64, same layout (FP64 re-scoring)
  double* d_lbin64 = nullptr;       // FP64 copy of d_lbin
  int gemm_bn = 128;                // N tile of the tensor-core GEMM
  int num_sms = 152;                // SMs of the device (split-K sizing)
  int ksplit_max = 1;               // K splits the GEMM-output scratch holds
  CUtensorMap tm_xhi, tm_xlo, tm_thi, tm_tlo;  // TMA descriptors (BF16 mode)
  struct AlignVariant {
    int group, starts_per_thread, dealing;
  };
  std::map<std::pair<int, int>, AlignVariant> align_group;  // autotuned ascent variant by (band, S)
  std::map<std::pair<int, int>, AlignVariant> newton_group;        // autotuned Newton variant (lanes per start, dealing)
};

namespace bh {
// A plan's tables live on the device it was created on; calls that read them must run with that device
// current (BH_ERR_ARG otherwise, before anything is enqueued).
inline int check_plan_device(const bh_plan* p) {
  int dev = 0;
  const int st = current_device(&dev);
  if (st != BH_OK) return st;
  if (dev != p->device) return fail(BH_ERR_ARG, "plan lives on device %d, current device is %d", p->device, dev);
  return BH_OK;
}
// Calls that expand volumes need the plan's basis table.
inline int check_expansion_plan(const bh_plan* p) {
  if (p->match_only) return fail(BH_ERR_ARG, "the plan was created with BH_PLAN_MATCH_ONLY (no expansion table)");
  return BH_OK;
}
// expand.cu
int upload_table(bh_plan* p, const std::vector<double>& radial, int n_r2, const std::vector<double>& angular,
                 const std::vector<int>& vox_r2, const std::vector<int2>& colinfo, double h3);
int make_tensor_maps(bh_plan* p);
int set_gemm_bn(bh_plan* p, int bn);
int expand_shifted(bh_plan* p, const float* vols, int B, const int3* d_shifts, int nshift, float* coeffs,
                   cudaStream_t stream);
// Expansion through caller scratch; volume b is vols + b N^3, or vptr[b] when vptr (a device array of B
// addresses) is given.
int expand_into(bh_plan* p, const float* vols, const float* const* vptr, int B, float* coeffs, void* scratch_x,
                float* scratch_c, int rows_cap, cudaStream_t stream);
// C[M][N] = A[M][K] B[N][K]^T, FP32 (M, N multiples of 128, K of 16)
int sgemm_nt(const float* A, const float* B, float* C, int M, int N, int K, cudaStream_t stream);
// align.cu
int align_init_constants();
}  // namespace bh

// Common-region norm of the missing-wedge constrained correlation (bh_wedge_create): pseudo-coefficients
// with one radial index per degree, so that the orbit-table evaluation of Eq. 2 yields
// Dn(R) = |T(0)|^2 + Re sum_l sum_{m,m'} q_lm w_lm' D^l_{mm'}(R).
struct bh_wedge {
  int device = -1;
  int L = 0;
  double half_angle = 0.0;
  bh::Layout layout{};          // K_l = 1, off_l = l^2, Lmax of the plan (indexes the plan's P table)
  float2* d_t = nullptr;        // [(L+1)^2] conj(q_lm), |T(0)|^2 / w_00 added at l = 0
  float2* d_w = nullptr;        // [(L+1)^2] w_lm
  std::vector<double> q, w;     // host FP64 copies, interleaved (re, im), [(L+1)^2]
  double c0 = 0.0;
};
