// Expansion of voxel volumes into ball-harmonic coefficients (Sec. II-A, expansion display) as a dense
// voxel-by-basis contraction:  C[b][j] = sum_v X[b][v] T[j][v],  X = in-ball voxels of volume b,
// T = real-form basis table (one row per coefficient slot, h^3 folded in; see plan.cpp).
//
// Two arithmetic forms:
//   BH_MODE_FP32        plain FP32 FFMA GEMM (128x128 tiles, 8x8 per thread).
//   BH_MODE_BF16_SPLIT  5th-generation tensor cores: tcgen05.mma kind::f16 with BF16 operands staged by
//                       TMA (128-byte swizzle) through an mbarrier pipeline and an FP32 accumulator in
//                       TMEM.  X = Xh + Xl and T = Th + Tl are split into BF16 hi/lo parts and the three
//                       products Xh*Th + Xh*Tl + Xl*Th accumulate into the same tile (the Xl*Tl term,
//                       ~2^-16 relative, is dropped).
// The GEMM runs over the fundamental voxels only (octant folding, see plan.cpp): each volume is first
// projected onto the 8 parity classes (k_project), and the table rows of class c are contracted with the
// class-c projection, so one launch computes 8 block products of one eighth of the voxels each.
// The real GEMM columns are then combined into complex coefficients [b][l][k][m+l].
#include <cstdio>

#include "bh_internal.h"

namespace bh {
namespace {

// ---------------------------------------------------------------- basis table (FP64 -> storage form)
// Row j (a table column of the GEMM, class by class) at fundamental voxel v; padding rows (colinfo -1) and
// padding voxels are zero.
__global__ void k_build_table(const double* __restrict__ radial, int n_r2, const double* __restrict__ angular,
                              const int* __restrict__ vox_r2, const int2* __restrict__ colinfo, double h3, int V,
                              int V_pad, float* __restrict__ T32, __nv_bfloat16* __restrict__ Thi,
                              __nv_bfloat16* __restrict__ Tlo) {
  const int j = blockIdx.y;
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= V_pad) return;
  double val = 0.0;
  const int2 ci = colinfo[j];
  if (ci.x >= 0 && v < V) val = h3 * radial[(size_t)ci.x * n_r2 + vox_r2[v]] * angular[(size_t)ci.y * V + v];
  const size_t o = (size_t)j * V_pad + v;
  if (T32) T32[o] = (float)val;
  if (Thi) {
    const __nv_bfloat16 hi = __double2bfloat16(val);
    Thi[o] = hi;
    Tlo[o] = __double2bfloat16(val - (double)__bfloat162float(hi));
  }
}

// ---------------------------------------------------------------- octant projection (+ hi/lo split)
// Row b of class c (X rows c * cls_rows + b) at fundamental voxel u = (x, y, z >= 0):
//   G_c(u) = 2^{-zeros(u)} sum_{s in {0..7}} (-1)^{popcount(c & s)} f(image_s(u)),
// image_s flipping the sign of axis i when bit i of s is set; a fast Walsh-Hadamard transform over the 8
// images (three butterfly stages), then the scale (coincident images on a zero coordinate counted once).
// kPtr: volume b starts at vptr[b] (a table of B addresses, e.g. request buffers in host memory that the
// device reads coherently).  shift (optional): f is read at image + shift, zero outside the box (the shift
// search's f_s(x) = f(x + s)); rows then index (volume, shift) pairs, r = b * nshift + j.
__device__ __forceinline__ void store_classes(float (&g)[8], size_t o, size_t cls_stride, float* __restrict__ X32,
                                              __nv_bfloat16* __restrict__ Xhi, __nv_bfloat16* __restrict__ Xlo) {
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const size_t oc = o + (size_t)c * cls_stride;
    if (X32) X32[oc] = g[c];
    if (Xhi) {
      const __nv_bfloat16 hi = __float2bfloat16_rn(g[c]);
      Xhi[oc] = hi;
      Xlo[oc] = __float2bfloat16_rn(g[c] - __bfloat162float(hi));
    }
  }
}

__device__ __forceinline__ void walsh8(float (&g)[8], int zeros) {
#pragma unroll
  for (int bit = 1; bit < 8; bit <<= 1)
#pragma unroll
    for (int s = 0; s < 8; ++s)
      if (!(s & bit)) {
        const float a = g[s], b = g[s | bit];
        g[s] = a + b;
        g[s | bit] = a - b;
      }
  const float sc = zeros == 0 ? 1.f : zeros == 1 ? 0.5f : zeros == 2 ? 0.25f : 0.125f;
#pragma unroll
  for (int c = 0; c < 8; ++c) g[c] *= sc;
}

template <bool kPtr>
__global__ void k_project(const float* __restrict__ vols, const float* const* __restrict__ vptr, int B, int N,
                          const int* __restrict__ fund, int VF, int VF_pad, size_t cls_stride,
                          float* __restrict__ X32, __nv_bfloat16* __restrict__ Xhi, __nv_bfloat16* __restrict__ Xlo) {
  const int b = blockIdx.y;
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= VF_pad) return;
  float g[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  int zeros = 0;
  if (b < B && u < VF) {
    const float* vb = kPtr ? vptr[b] : vols + (size_t)b * N * N * N;
    const int pk = __ldg(fund + u), h = N / 2;
    const int x = pk & 1023, y = (pk >> 10) & 1023, z = pk >> 20;
    zeros = (x == 0) + (y == 0) + (z == 0);
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const int ix = h + ((s & 1) ? -x : x), iy = h + ((s & 2) ? -y : y), iz = h + ((s & 4) ? -z : z);
      g[s] = __ldg(vb + ((size_t)iz * N + iy) * N + ix);
    }
    walsh8(g, zeros);
  }
  store_classes(g, (size_t)b * VF_pad + u, cls_stride, X32, Xhi, Xlo);
}

// Projection of shifted volumes: row rr of this pass is pair r = row0 + rr = (volume r / nshift, shift r % nshift).
__global__ void k_project_shifted(const float* __restrict__ vols, int B, int N, const int* __restrict__ fund,
                                  const int3* __restrict__ shifts, int nshift, int row0, int rows, int VF, int VF_pad,
                                  size_t cls_stride, float* __restrict__ X32, __nv_bfloat16* __restrict__ Xhi,
                                  __nv_bfloat16* __restrict__ Xlo) {
  const int rr = blockIdx.y;
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= VF_pad) return;
  float g[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  const int r = row0 + rr;
  if (rr < rows && u < VF) {
    const int bvol = r / nshift, j = r % nshift;
    if (bvol < B) {
      const float* vb = vols + (size_t)bvol * N * N * N;
      const int pk = __ldg(fund + u), h = N / 2;
      const int x = pk & 1023, y = (pk >> 10) & 1023, z = pk >> 20;
      const int3 sh = shifts[j];
#pragma unroll
      for (int s = 0; s < 8; ++s) {
        const int ix = h + ((s & 1) ? -x : x) + sh.x, iy = h + ((s & 2) ? -y : y) + sh.y,
                  iz = h + ((s & 4) ? -z : z) + sh.z;
        const bool in = ix >= 0 && ix < N && iy >= 0 && iy < N && iz >= 0 && iz < N;
        g[s] = in ? __ldg(vb + ((size_t)iz * N + iy) * N + ix) : 0.f;
      }
      walsh8(g, (x == 0) + (y == 0) + (z == 0));
    }
  }
  store_classes(g, (size_t)rr * VF_pad + u, cls_stride, X32, Xhi, Xlo);
}

// ---------------------------------------------------------------- real columns -> complex coefficients
// slot[s] = (re source, im source), 1-based column index with sign, 0 = zero.
// With split-K the GEMM leaves `splits` partial products `split_stride` floats apart; they are summed
// here in split order (deterministic).
__global__ void k_to_complex(const float* __restrict__ C, int ldc, int B, int Nb, const int2* __restrict__ slot,
                             float2* __restrict__ out, int splits, size_t split_stride) {
  const int b = blockIdx.y;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B || s >= Nb) return;
  const int2 src = slot[s];
  float re = 0.f, im = 0.f;
  for (int z = 0; z < splits; ++z) {
    const float* row = C + (size_t)z * split_stride + (size_t)b * ldc;
    if (src.x > 0) re += row[src.x - 1]; else if (src.x < 0) re -= row[-src.x - 1];
    if (src.y > 0) im += row[src.y - 1]; else if (src.y < 0) im -= row[-src.y - 1];
  }
  out[(size_t)b * Nb + s] = make_float2(re, im);
}

// The same, one CTA per row: the row's split partial sums are added (in split order) into shared memory with
// coalesced 16-byte loads (ldc and split_stride are multiples of 4 floats), then the complex coefficients are
// formed from shared memory.  Bitwise equal to k_to_complex (a negated sum equals the sum of the negated terms).
__global__ void __launch_bounds__(256) k_to_complex_rows(const float* __restrict__ C, int ldc, int Nb,
                                                         const int2* __restrict__ slot, float2* __restrict__ out,
                                                         int splits, size_t split_stride) {
  extern __shared__ float4 row4[];
  const float* row = reinterpret_cast<const float*>(row4);
  const int b = blockIdx.x;
  const int n4 = ldc / 4;
#pragma unroll 4
  for (int c = threadIdx.x; c < n4; c += blockDim.x) {
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int z = 0; z < splits; ++z) {
      const float4 t = reinterpret_cast<const float4*>(C + (size_t)z * split_stride + (size_t)b * ldc)[c];
      v.x += t.x;
      v.y += t.y;
      v.z += t.z;
      v.w += t.w;
    }
    row4[c] = v;
  }
  __syncthreads();
  for (int s = threadIdx.x; s < Nb; s += blockDim.x) {
    const int2 src = slot[s];
    const float re = src.x > 0 ? row[src.x - 1] : (src.x < 0 ? -row[-src.x - 1] : 0.f);
    const float im = src.y > 0 ? row[src.y - 1] : (src.y < 0 ? -row[-src.y - 1] : 0.f);
    out[(size_t)b * Nb + s] = make_float2(re, im);
  }
}

// ---------------------------------------------------------------- plain FP32 GEMM, both operands K-major
// C[M][N] = A[M][K] * B[N][K]^T; M % 128 == 0, N % 128 == 0, K % 16 == 0.
constexpr int SG_BM = 128, SG_BN = 128, SG_BK = 16, SG_PAD = 4;

__global__ void __launch_bounds__(256) k_sgemm_nt(const float* __restrict__ A, const float* __restrict__ Bm,
                                                  float* __restrict__ C, int M, int N, int K, int k_split,
                                                  size_t split_stride, ClassMap cm) {
  // split z of the grid covers K range [z k_split, min(K, (z+1) k_split)) and writes C + z split_stride
  const int kbeg = blockIdx.z * k_split;
  const int kend = min(K, kbeg + k_split);
  C += (size_t)blockIdx.z * split_stride;
  __shared__ __align__(16) float As[SG_BK][SG_BM + SG_PAD];
  __shared__ __align__(16) float Bs[SG_BK][SG_BN + SG_PAD];
  const int tid = threadIdx.x;
  const int m0 = blockIdx.x * SG_BM, n0 = blockIdx.y * SG_BN;  // M fastest: CTAs in flight share table panels
  const int lr = tid >> 2, lk = (tid & 3) * 4;  // loader: rows lr and lr+64, k columns lk..lk+3
  const int tx = tid & 15, ty = tid >> 4;
  // octant folding: the A rows of this N tile's parity class (cm.rows = 0: a plain GEMM)
  const int arow0 = (cm.rows ? class_of_ntile(cm, blockIdx.y) * cm.rows : 0) + m0;
  const float* Ap0 = A + (size_t)(arow0 + lr) * K + kbeg + lk;
  const float* Ap1 = Ap0 + (size_t)64 * K;
  const float* Bp0 = Bm + (size_t)(n0 + lr) * K + kbeg + lk;
  const float* Bp1 = Bp0 + (size_t)64 * K;
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
  float4 a0 = __ldg(reinterpret_cast<const float4*>(Ap0)), a1 = __ldg(reinterpret_cast<const float4*>(Ap1));
  float4 b0 = __ldg(reinterpret_cast<const float4*>(Bp0)), b1 = __ldg(reinterpret_cast<const float4*>(Bp1));
  const int klen = kend - kbeg;
  for (int k0 = 0; k0 < klen; k0 += SG_BK) {
    __syncthreads();
    As[lk + 0][lr] = a0.x; As[lk + 1][lr] = a0.y; As[lk + 2][lr] = a0.z; As[lk + 3][lr] = a0.w;
    As[lk + 0][lr + 64] = a1.x; As[lk + 1][lr + 64] = a1.y; As[lk + 2][lr + 64] = a1.z; As[lk + 3][lr + 64] = a1.w;
    Bs[lk + 0][lr] = b0.x; Bs[lk + 1][lr] = b0.y; Bs[lk + 2][lr] = b0.z; Bs[lk + 3][lr] = b0.w;
    Bs[lk + 0][lr + 64] = b1.x; Bs[lk + 1][lr + 64] = b1.y; Bs[lk + 2][lr + 64] = b1.z; Bs[lk + 3][lr + 64] = b1.w;
    __syncthreads();
    if (k0 + SG_BK < klen) {  // prefetch the next K block into registers while computing this one
      a0 = __ldg(reinterpret_cast<const float4*>(Ap0 + k0 + SG_BK));
      a1 = __ldg(reinterpret_cast<const float4*>(Ap1 + k0 + SG_BK));
      b0 = __ldg(reinterpret_cast<const float4*>(Bp0 + k0 + SG_BK));
      b1 = __ldg(reinterpret_cast<const float4*>(Bp1 + k0 + SG_BK));
    }
#pragma unroll
    for (int kk = 0; kk < SG_BK; ++kk) {
      const float4 ra0 = *reinterpret_cast<const float4*>(&As[kk][ty * 4]);
      const float4 ra1 = *reinterpret_cast<const float4*>(&As[kk][64 + ty * 4]);
      const float4 rb0 = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4]);
      const float4 rb1 = *reinterpret_cast<const float4*>(&Bs[kk][64 + tx * 4]);
      const float ra[8] = {ra0.x, ra0.y, ra0.z, ra0.w, ra1.x, ra1.y, ra1.z, ra1.w};
      const float rb[8] = {rb0.x, rb0.y, rb0.z, rb0.w, rb1.x, rb1.y, rb1.z, rb1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(ra[i], rb[j], acc[i][j]);
    }
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int row = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4);
    float* crow = C + (size_t)row * N + n0;
    *reinterpret_cast<float4*>(crow + tx * 4) = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
    *reinterpret_cast<float4*>(crow + 64 + tx * 4) = make_float4(acc[i][4], acc[i][5], acc[i][6], acc[i][7]);
  }
}

}  // namespace

// C[M][N] = A[M][K] B[N][K]^T in FP32 on the caller's stream (M, N multiples of 128, K of 16).
int sgemm_nt(const float* A, const float* Bm, float* C, int M, int N, int K, cudaStream_t stream) {
  if (M % SG_BM || N % SG_BN || K % SG_BK || M <= 0 || N <= 0 || K <= 0)
    return fail(BH_ERR_ARG, "sgemm_nt: M=%d N=%d K=%d not tile multiples", M, N, K);
  k_sgemm_nt<<<dim3(M / SG_BM, N / SG_BN, 1), 256, 0, stream>>>(A, Bm, C, M, N, K, K, 0, ClassMap{});
  BH_CHECK_LAUNCH();
  return BH_OK;
}

namespace {
// ---------------------------------------------------------------- tcgen05 / TMA / mbarrier primitives
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on an mbarrier phase: gives up after ~2 s of device time, records `code` in *err.
constexpr uint64_t kWaitLimitNs = 2000000000ull;
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err, int code) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  for (uint32_t i = 1;; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 255u) == 0u && globaltimer_ns() - t0 > kWaitLimitNs) {
      atomicExch(err, code);
      return false;
    }
  }
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* tm, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld_32x32b_x32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void tmem_st_32x32b_x32(uint32_t taddr, const uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
      "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
      "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
      "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]),
      "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]),
      "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
      : "memory");
}
__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major tile with 128-byte rows and the 128-byte swizzle:
// start address >> 4 at bits [0,14), leading byte offset (unused for this layout) = 16 B at [16,30),
// stride byte offset = 1024 B (one 8-row swizzle atom) at [32,46), descriptor version 1 at [46,48),
// layout SWIZZLE_128B = 2 at [61,64).  Tiles are 1024-byte aligned, so the base offset is 0.
__device__ __forceinline__ uint64_t sdesc_k_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)(16u >> 4) << 16;
  d |= (uint64_t)(1024u >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptor, kind::f16: D = F32 (bits [4,6) = 1), A = B = BF16 (bits [7,10) and [10,13) = 1),
// both K-major (bits 15, 16 = 0), N >> 3 at [17,23), M >> 4 at [24,29).
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Tensor-core GEMM with FP32 promotion of the accumulator.  Additions into the tcgen05 accumulator in
// TMEM truncate, so their error grows with the number of accumulate steps (3 K/16 per output, ~2.6e4 at
// a 64^3 box); here every KCHUNK K-blocks the MMA issuer switches to the other of two TMEM accumulators
// (started afresh), and the four epilogue warps add each finished chunk into an FP32 running sum held in
// a third TMEM region (tcgen05.ld, FP32 add in registers, tcgen05.st), then hand the buffer back.
//   warp 4 lane 0: TMA producer (3-stage ring of A hi/lo and B hi/lo tiles, 128-byte swizzle)
//   warp 5 lane 0: MMA issuer (three tcgen05.mma per 16-wide K step: hi*hi, hi*lo, lo*hi)
//   warps 0-3:     epilogue (warp w owns TMEM lanes and tile rows 32w..32w+31)
constexpr int PBN = 128, PST = 3, KCHUNK = 16;
struct PCfg {
  static constexpr int BM = kGemmBM, BK = kGemmBK;
  static constexpr uint32_t A_BYTES = BM * BK * 2, B_BYTES = PBN * BK * 2;
  static constexpr uint32_t STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
  static constexpr size_t SMEM = (size_t)PST * STAGE_BYTES + 1024;
  // TMEM columns: accumulators [0, PBN) and [PBN, 2 PBN), FP32 running sum [2 PBN, 3 PBN)
  static constexpr uint32_t TMEM_COLS = 512;
  static constexpr uint32_t SUM_COL = 2 * PBN;
};

__global__ void __launch_bounds__(192, 1)
    k_gemm_tc_promoted(const __grid_constant__ CUtensorMap tmAh, const __grid_constant__ CUtensorMap tmAl,
                       const __grid_constant__ CUtensorMap tmBh, const __grid_constant__ CUtensorMap tmBl,
                       float* __restrict__ C, int ldc, int num_kb_total, int kb_split, size_t split_stride,
                       int* __restrict__ err, ClassMap cm) {
  // split z of the grid covers K blocks [z kb_split, min(total, (z+1) kb_split)) and writes C + z split_stride
  const int kb_first = blockIdx.z * kb_split;
  const int num_kb = min(num_kb_total - kb_first, kb_split);
  C += (size_t)blockIdx.z * split_stride;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t full_bar[PST], empty_bar[PST], accf_bar[2], acce_bar[2];
  __shared__ uint32_t tmem_base_sh;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // M tiles vary fastest across the grid, so the CTAs in flight share table (B) panels, the operand
  // larger than L2, while the gathered volumes (A) stay L2-resident
  const int m0 = blockIdx.x * PCfg::BM, n0 = blockIdx.y * PBN;
  // octant folding: this N tile's parity class reads the projected volumes of that class (A rows)
  const int arow0 = (cm.rows ? class_of_ntile(cm, blockIdx.y) * cm.rows : 0) + m0;
  const int nchunks = (num_kb + KCHUNK - 1) / KCHUNK;
  auto sA_hi = [&](int s) { return smem + (size_t)s * PCfg::STAGE_BYTES; };
  auto sA_lo = [&](int s) { return smem + (size_t)s * PCfg::STAGE_BYTES + PCfg::A_BYTES; };
  auto sB_hi = [&](int s) { return smem + (size_t)s * PCfg::STAGE_BYTES + 2 * PCfg::A_BYTES; };
  auto sB_lo = [&](int s) { return smem + (size_t)s * PCfg::STAGE_BYTES + 2 * PCfg::A_BYTES + PCfg::B_BYTES; };

  if (threadIdx.x == 0) {
    for (int s = 0; s < PST; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accf_bar[b], 1);
      mbar_init(&acce_bar[b], 128);
    }
    mbar_fence_init();
  }
  if (warp == 0) {
    tmem_alloc(&tmem_base_sh, PCfg::TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tmem_base_sh;

  if (warp == 4) {
    if (lane == 0) {
      // ---------------- TMA producer
      int kb = 0;
      for (; kb < num_kb; ++kb) {
        const int s = kb % PST;
        const uint32_t ph = (uint32_t)(kb / PST) & 1u;
        if (!mbar_wait(&empty_bar[s], ph ^ 1u, err, 111)) break;
        mbar_arrive_expect_tx(&full_bar[s], PCfg::STAGE_BYTES);
        const int kx = (kb_first + kb) * PCfg::BK;
        tma_load_2d(sA_hi(s), &tmAh, kx, arow0, &full_bar[s]);
        tma_load_2d(sA_lo(s), &tmAl, kx, arow0, &full_bar[s]);
        tma_load_2d(sB_hi(s), &tmBh, kx, n0, &full_bar[s]);
        tma_load_2d(sB_lo(s), &tmBl, kx, n0, &full_bar[s]);
      }
      if (kb < num_kb)  // gave up: let the copies already issued land before the CTA leaves (bounded)
        for (int j = (kb >= PST ? kb - PST : 0); j < kb; ++j)
          mbar_wait(&full_bar[j % PST], (uint32_t)(j / PST) & 1u, err, 112);
    }
  } else if (warp == 5) {
    if (lane == 0) {
      // ---------------- MMA issuer
      constexpr uint32_t idesc = idesc_bf16_f32(PCfg::BM, PBN);
      bool ok = true;
      for (int c = 0; c < nchunks; ++c) {
        const int buf = c & 1, use = c >> 1;
        if (ok && !mbar_wait(&acce_bar[buf], (uint32_t)(use & 1) ^ 1u, err, 113)) ok = false;
        tc_fence_after();
        const uint32_t tacc = tbase + (uint32_t)(buf * PBN);
        const int kb0 = c * KCHUNK, kb1 = min(num_kb, kb0 + KCHUNK);
        for (int kb = kb0; ok && kb < kb1; ++kb) {
          const int s = kb % PST;
          const uint32_t ph = (uint32_t)(kb / PST) & 1u;
          if (!mbar_wait(&full_bar[s], ph, err, 114)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint64_t ah = sdesc_k_sw128(smem_u32(sA_hi(s))), al = sdesc_k_sw128(smem_u32(sA_lo(s)));
          const uint64_t bh = sdesc_k_sw128(smem_u32(sB_hi(s))), bl = sdesc_k_sw128(smem_u32(sB_lo(s)));
#pragma unroll
          for (int k = 0; k < PCfg::BK / 16; ++k) {
            const uint64_t adv = (uint64_t)(k * 32) >> 4;
            umma_bf16(tacc, ah + adv, bh + adv, idesc, (kb != kb0 || k != 0) ? 1u : 0u);
            umma_bf16(tacc, ah + adv, bl + adv, idesc, 1u);
            umma_bf16(tacc, al + adv, bh + adv, idesc, 1u);
          }
          umma_commit(&empty_bar[s]);
        }
        umma_commit(&accf_bar[buf]);  // chunk finished (or abandoned): the epilogue may read the buffer
      }
    }
  } else {
    // ---------------- epilogue warps 0-3: promote every chunk into the FP32 running sum (TMEM)
    const int row = warp * 32 + lane;
    const uint32_t lanes = (uint32_t)(warp * 32) << 16;
    bool ok = true;
    for (int c = 0; c < nchunks; ++c) {
      const int buf = c & 1, use = c >> 1;
      if (ok) ok = mbar_wait(&accf_bar[buf], (uint32_t)(use & 1), err, 115);
      ok = __all_sync(0xffffffffu, ok);
      tc_fence_after();
      const bool last = (c + 1 == nchunks);
#pragma unroll 1
      for (int cc = 0; cc < PBN / 32; ++cc) {
        uint32_t r[32], t[32];
        tmem_ld_32x32b_x32(tbase + lanes + (uint32_t)(buf * PBN + cc * 32), r);
        if (c > 0) tmem_ld_32x32b_x32(tbase + lanes + PCfg::SUM_COL + (uint32_t)(cc * 32), t);
        tmem_ld_wait();
        if (c > 0) {
#pragma unroll
          for (int i = 0; i < 32; ++i) r[i] = __float_as_uint(__uint_as_float(r[i]) + __uint_as_float(t[i]));
        }
        if (!last) {
          tmem_st_32x32b_x32(tbase + lanes + PCfg::SUM_COL + (uint32_t)(cc * 32), r);
        } else if (ok) {
          float4* dst = reinterpret_cast<float4*>(C + (size_t)(m0 + row) * ldc + n0 + cc * 32);
#pragma unroll
          for (int i = 0; i < 8; ++i)
            dst[i] = make_float4(__uint_as_float(r[4 * i]), __uint_as_float(r[4 * i + 1]), __uint_as_float(r[4 * i + 2]),
                                 __uint_as_float(r[4 * i + 3]));
        }
      }
      tmem_st_wait();
      tc_fence_before();
      mbar_arrive(&acce_bar[buf]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tbase, PCfg::TMEM_COLS);
}

}  // namespace

// ====================================================================== host helpers
int upload_table(bh_plan* p, const std::vector<double>& radial, int n_r2, const std::vector<double>& angular,
                 const std::vector<int>& vox_r2, const std::vector<int2>& colinfo, double h3) {
  double *d_rad = nullptr, *d_ang = nullptr;
  int* d_r2 = nullptr;
  int2* d_ci = nullptr;
  auto cleanup = [&]() {
    cudaFree(d_rad);
    cudaFree(d_ang);
    cudaFree(d_r2);
    cudaFree(d_ci);
  };
#define UT_TRY(call)                                                                                           \
  do {                                                                                                         \
    cudaError_t e_ = (call);                                                                                   \
    if (e_ != cudaSuccess) {                                                                                   \
      cleanup();                                                                                               \
      return fail(e_ == cudaErrorMemoryAllocation ? BH_ERR_OOM : BH_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    }                                                                                                          \
  } while (0)
  UT_TRY(cudaMalloc(&d_rad, sizeof(double) * radial.size()));
  UT_TRY(cudaMalloc(&d_ang, sizeof(double) * angular.size()));
  UT_TRY(cudaMalloc(&d_r2, sizeof(int) * vox_r2.size()));
  UT_TRY(cudaMalloc(&d_ci, sizeof(int2) * colinfo.size()));
  UT_TRY(cudaMemcpy(d_rad, radial.data(), sizeof(double) * radial.size(), cudaMemcpyHostToDevice));
  UT_TRY(cudaMemcpy(d_ang, angular.data(), sizeof(double) * angular.size(), cudaMemcpyHostToDevice));
  UT_TRY(cudaMemcpy(d_r2, vox_r2.data(), sizeof(int) * vox_r2.size(), cudaMemcpyHostToDevice));
  UT_TRY(cudaMemcpy(d_ci, colinfo.data(), sizeof(int2) * colinfo.size(), cudaMemcpyHostToDevice));
  dim3 grid((p->VF_pad + 255) / 256, p->Nb_pad);
  k_build_table<<<grid, 256>>>(d_rad, n_r2, d_ang, d_r2, d_ci, h3, p->VF, p->VF_pad, p->d_T32, p->d_Thi,
                               p->d_Tlo);
  UT_TRY(cudaGetLastError());
  UT_TRY(cudaDeviceSynchronize());
#undef UT_TRY
  cleanup();
  return BH_OK;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn get_encode() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(ptr);
  }
  return fn;
}

static int encode_bf16_2d(CUtensorMap* tm, const void* base, uint64_t inner, uint64_t outer, uint32_t box_inner,
                          uint32_t box_outer) {
  auto enc = get_encode();
  if (!enc) return fail(BH_ERR_CUDA, "cuTensorMapEncodeTiled entry point unavailable");
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {inner * 2};
  cuuint32_t box[2] = {box_inner, box_outer};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(BH_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return BH_OK;
}

int make_tensor_maps(bh_plan* p) {
  // Operands are K-major: inner dimension = VF_pad (multiple of 64), boxes 64 x rows; the projected volumes
  // are 8 class blocks of M_cap rows.
  int st;
  if ((st = encode_bf16_2d(&p->tm_xhi, p->d_Xhi, p->VF_pad, 8ull * p->M_cap, kGemmBK, kGemmBM)) != BH_OK) return st;
  if ((st = encode_bf16_2d(&p->tm_xlo, p->d_Xlo, p->VF_pad, 8ull * p->M_cap, kGemmBK, kGemmBM)) != BH_OK) return st;
  if ((st = encode_bf16_2d(&p->tm_thi, p->d_Thi, p->VF_pad, p->Nb_pad, kGemmBK, p->gemm_bn)) != BH_OK) return st;
  if ((st = encode_bf16_2d(&p->tm_tlo, p->d_Tlo, p->VF_pad, p->Nb_pad, kGemmBK, p->gemm_bn)) != BH_OK) return st;
  return BH_OK;
}

int set_gemm_bn(bh_plan* p, int bn) {
  if (bn != 128) return fail(BH_ERR_ARG, "GEMM N tile %d: the promoted tensor-core GEMM uses 128", bn);
  if (p->mode != BH_MODE_BF16_SPLIT || p->gemm_bn == bn) {
    p->gemm_bn = bn;
    return BH_OK;
  }
  p->gemm_bn = bn;
  return make_tensor_maps(p);
}

// K splits for a pass of Mp rows: enough CTAs for about two waves over the SMs when the output tiles
// alone are few, each split keeping at least 32 K-blocks (two promotion chunks), at most the plan's
// scratch allows.
// Split-K count of a pass: one GEMM CTA is resident per SM, so take the fewest splits whose last wave of
// CTAs is at least 90 % full (else the fullest), keeping at least 32 K-blocks per split.
static int choose_splits(const bh_plan* p, int Mp) {
  const int tiles = (Mp / kGemmBM) * (p->Nb_pad / kGemmBN);
  const int num_kb = p->VF_pad / kGemmBK;
  const int smax = std::max(1, std::min(p->ksplit_max, num_kb / 32));
  int best = 1;
  double best_eff = 0.0;
  for (int s = 1; s <= smax; ++s) {
    const double waves = (double)tiles * s / p->num_sms;
    const double eff = waves / std::ceil(waves);
    if (eff >= 0.9) return s;
    if (eff > best_eff + 1e-9) {
      best_eff = eff;
      best = s;
    }
  }
  return best;
}

// Complex coefficients of `rows` GEMM rows (split partial sums added in order).
static int launch_to_complex(const bh_plan* p, const float* C, int rows, float* coeffs, int splits, size_t stride,
                             cudaStream_t stream) {
  const size_t row_bytes = (size_t)p->Nb_pad * sizeof(float);
  if (row_bytes <= 200 * 1024) {
    static SmemAttr attr;
    const int st = ensure_smem(k_to_complex_rows, attr, row_bytes);
    if (st != BH_OK) return st;
    k_to_complex_rows<<<rows, 256, row_bytes, stream>>>(C, p->Nb_pad, p->Nb, p->d_slot, reinterpret_cast<float2*>(coeffs),
                                                        splits, stride);
  } else {
    dim3 g2((p->Nb + 255) / 256, rows);
    k_to_complex<<<g2, 256, 0, stream>>>(C, p->Nb_pad, rows, p->Nb, p->d_slot, reinterpret_cast<float2*>(coeffs),
                                         splits, stride);
  }
  BH_CHECK_LAUNCH();
  return BH_OK;
}

// K splits that hold work for a GEMM of `splits` requested splits (the last ones may be empty).
static int used_splits(const bh_plan* p, int splits) {
  if (p->mode == BH_MODE_FP32) {
    const int ks = round_up((p->VF_pad + splits - 1) / splits, SG_BK);
    return (p->VF_pad + ks - 1) / ks;
  }
  const int nkb = p->VF_pad / kGemmBK;
  const int kbs = round_up((nkb + splits - 1) / splits, KCHUNK);
  return (nkb + kbs - 1) / kbs;
}

// The folded GEMM of Mp rows: X holds 8 class blocks of cls_rows rows (X32, or the tensor maps of its BF16
// hi/lo parts), C gets `splits` partial products split_stride floats apart.
static int launch_gemm(bh_plan* p, const float* X32, const CUtensorMap& tm_hi, const CUtensorMap& tm_lo, float* C,
                       int Mp, int splits, int cls_rows, size_t split_stride, cudaStream_t stream) {
  ClassMap cm = p->cls;
  cm.rows = cls_rows;
  if (p->mode == BH_MODE_FP32) {
    const int k_split = round_up((p->VF_pad + splits - 1) / splits, SG_BK);
    dim3 grid(Mp / SG_BM, p->Nb_pad / SG_BN, (p->VF_pad + k_split - 1) / k_split);  // every split has K work
    k_sgemm_nt<<<grid, 256, 0, stream>>>(X32, p->d_T32, C, Mp, p->Nb_pad, p->VF_pad, k_split, split_stride, cm);
    BH_CHECK_LAUNCH();
    return BH_OK;
  }
  const int num_kb = p->VF_pad / kGemmBK;
  const int kb_split = round_up((num_kb + splits - 1) / splits, KCHUNK);
  static SmemAttr attr;
  const int st = ensure_smem(k_gemm_tc_promoted, attr, PCfg::SMEM);
  if (st != BH_OK) return st;
  dim3 grid(Mp / kGemmBM, p->Nb_pad / PBN, (num_kb + kb_split - 1) / kb_split);
  k_gemm_tc_promoted<<<grid, 192, PCfg::SMEM, stream>>>(tm_hi, tm_lo, p->tm_thi, p->tm_tlo, C, p->Nb_pad, num_kb,
                                                      kb_split, split_stride, p->d_err, cm);
  BH_CHECK_LAUNCH();
  return BH_OK;
}

// Octant projection of Bc volumes into class blocks of cls_rows rows (from vols, or from the address table
// vptr).
static int launch_project(const bh_plan* p, const float* vols, const float* const* vptr, int Bc, int Mp, float* X32,
                          __nv_bfloat16* Xhi, __nv_bfloat16* Xlo, int cls_rows, cudaStream_t stream) {
  dim3 g1((p->VF_pad + 255) / 256, Mp);
  const size_t cls_stride = (size_t)cls_rows * p->VF_pad;
  if (vptr)
    k_project<true><<<g1, 256, 0, stream>>>(nullptr, vptr, Bc, p->N, p->d_fund, p->VF, p->VF_pad, cls_stride, X32, Xhi,
                                            Xlo);
  else
    k_project<false><<<g1, 256, 0, stream>>>(vols, nullptr, Bc, p->N, p->d_fund, p->VF, p->VF_pad, cls_stride, X32,
                                             Xhi, Xlo);
  BH_CHECK_LAUNCH();
  return BH_OK;
}

// Expansion through caller-provided scratch (used by the entry point that allocates nothing and by the
// serving batches): the same kernels as bh_expand, with the projected volumes (8 class blocks of rows_cap
// rows) and the real GEMM output placed in `scratch_x` / `scratch_c`, `rows_cap` rows (a multiple of the
// 128-row M tile) per pass.  Tensor maps of the projected volumes are encoded for the given scratch on
// every call (host-side encoding, no allocation).
int expand_into(bh_plan* p, const float* vols, const float* const* vptr, int B, float* coeffs, void* scratch_x,
                float* scratch_c, int rows_cap, cudaStream_t stream) {
  const long long N3 = (long long)p->N * p->N * p->N;
  float* X32 = nullptr;
  __nv_bfloat16 *Xhi = nullptr, *Xlo = nullptr;
  CUtensorMap tm_hi{}, tm_lo{};
  if (p->mode == BH_MODE_FP32) {
    X32 = static_cast<float*>(scratch_x);
  } else {
    Xhi = static_cast<__nv_bfloat16*>(scratch_x);
    Xlo = Xhi + (size_t)8 * rows_cap * p->VF_pad;
    int st;
    if ((st = encode_bf16_2d(&tm_hi, Xhi, p->VF_pad, 8ull * rows_cap, kGemmBK, kGemmBM)) != BH_OK) return st;
    if ((st = encode_bf16_2d(&tm_lo, Xlo, p->VF_pad, 8ull * rows_cap, kGemmBK, kGemmBM)) != BH_OK) return st;
  }
  for (int b0 = 0; b0 < B; b0 += rows_cap) {
    const int Bc = std::min(rows_cap, B - b0);
    const int Mp = round_up(Bc, kGemmBM);
    int st = launch_project(p, vptr ? nullptr : vols + (size_t)b0 * N3, vptr ? vptr + b0 : nullptr, Bc, Mp, X32, Xhi,
                            Xlo, rows_cap, stream);
    if (st == BH_OK) st = launch_gemm(p, X32, tm_hi, tm_lo, scratch_c, Mp, 1, rows_cap, 0, stream);
    if (st == BH_OK) st = launch_to_complex(p, scratch_c, Bc, coeffs + (size_t)b0 * p->Nb * 2, 1, 0, stream);
    if (st != BH_OK) return st;
  }
  return BH_OK;
}

// Expansion of every (volume, shift) pair into coeffs [b][shift][Nb], through the plan's scratch.
int expand_shifted(bh_plan* p, const float* vols, int B, const int3* d_shifts, int nshift, float* coeffs,
                   cudaStream_t stream) {
  const int total = B * nshift;
  const size_t stride = (size_t)p->M_cap * p->Nb_pad;
  for (int r0 = 0; r0 < total; r0 += p->max_batch) {
    const int rows = std::min(p->max_batch, total - r0);
    const int Mp = round_up(rows, kGemmBM);
    dim3 g1((p->VF_pad + 255) / 256, Mp);
    k_project_shifted<<<g1, 256, 0, stream>>>(vols, B, p->N, p->d_fund, d_shifts, nshift, r0, rows, p->VF, p->VF_pad,
                                              (size_t)p->M_cap * p->VF_pad, p->d_X32, p->d_Xhi, p->d_Xlo);
    BH_CHECK_LAUNCH();
    const int splits = choose_splits(p, Mp);
    int st = launch_gemm(p, p->d_X32, p->tm_xhi, p->tm_xlo, p->d_C, Mp, splits, p->M_cap, stride, stream);
    if (st != BH_OK) return st;
    st = launch_to_complex(p, p->d_C, rows, coeffs + (size_t)r0 * p->Nb * 2, used_splits(p, splits), stride, stream);
    if (st != BH_OK) return st;
  }
  return BH_OK;
}

}  // namespace bh

using namespace bh;

namespace bh {
namespace {
// Probe of the bounded mbarrier wait used by the tensor-core pipeline: one thread waits on a phase that
// nothing completes; after the wait's time limit it records `code` in the error word and returns, as a
// stalled GEMM pipeline would.
__global__ void k_wait_probe(int* err, int code) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
    mbar_wait(&bar, 0u, err, code);
  }
}
}  // namespace
}  // namespace bh

extern "C" int bh_plan_status(bh_plan* p) {
  clear_error();
  if (!p) return fail(BH_ERR_ARG, "plan is NULL");
  int code = 0;
  BH_CUDA_TRY(cudaMemcpy(&code, p->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (code == 0) return BH_OK;
  BH_CUDA_TRY(cudaMemset(p->d_err, 0, sizeof(int)));
  return fail(BH_ERR_TIMEOUT, "a device wait gave up (site %d); the results of the plan's work since the last "
              "status check are invalid", code);
}

extern "C" int bh_plan_probe_wait(bh_plan* p, void* stream) {
  clear_error();
  if (!p) return fail(BH_ERR_ARG, "plan is NULL");
  {
    const int st = check_plan_device(p);
    if (st != BH_OK) return st;
  }
  bh::k_wait_probe<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(p->d_err, 199);
  BH_CHECK_LAUNCH();
  return BH_OK;
}

extern "C" int bh_expand(bh_plan* p, const float* vols, int B, float* coeffs, void* stream_) {
  clear_error();
  const bh::Range range_("bh_expand");
  if (!p) return fail(BH_ERR_ARG, "plan is NULL");
  if (B < 0) return fail(BH_ERR_ARG, "B=%d", B);
  if (B == 0) return BH_OK;
  if (!vols || !coeffs) return fail(BH_ERR_ARG, "vols or coeffs is NULL");
  {
    int st = check_plan_device(p);
    if (st == BH_OK) st = check_expansion_plan(p);
    if (st != BH_OK) return st;
  }
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  const long long N3 = (long long)p->N * p->N * p->N;
  const size_t stride = (size_t)p->M_cap * p->Nb_pad;
  for (int b0 = 0; b0 < B; b0 += p->max_batch) {
    const int Bc = std::min(p->max_batch, B - b0);
    const int Mp = round_up(Bc, kGemmBM);
    int st = launch_project(p, vols + (size_t)b0 * N3, nullptr, Bc, Mp, p->d_X32, p->d_Xhi, p->d_Xlo, p->M_cap,
                            stream);
    if (st != BH_OK) return st;
    const int splits = choose_splits(p, Mp);
    st = launch_gemm(p, p->d_X32, p->tm_xhi, p->tm_xlo, p->d_C, Mp, splits, p->M_cap, stride, stream);
    if (st != BH_OK) return st;
    st = launch_to_complex(p, p->d_C, Bc, coeffs + (size_t)b0 * p->Nb * 2, used_splits(p, splits), stride, stream);
    if (st != BH_OK) return st;
  }
  return BH_OK;
}
