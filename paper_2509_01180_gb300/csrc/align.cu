// Rotational cross-correlation of Eq. 2 at s = 0, its closed-form gradient, and the multi-start
// gradient ascent with frequency marching of Sec. II-C, for many subtomograms in one launch.
//
// Score of a rotation R (quaternion q):  S(R) = Re sum_{l<=L} sum_{m,n} xi^l_{mn} D^l_{mn}(R),
// xi^l_{mn} = sum_k conj(t_klm) f_kln.  With R = Rz(alpha) Ry(beta) Rz(gamma),
// D^l_{mn} = e^{-i m alpha} d^l_{mn}(beta) e^{-i n gamma}, so
//   S = sum_{m,n} Re( e^{-i(m alpha + n gamma)} sum_{l >= max|m|,|n|} d^l_{mn}(beta) xi^l_{mn} ).
// Each (m,n) pair is one l-recursion; the GPU never forms D.
//
// Folding (real volumes, so xi^l_{-m,-n} = (-1)^{m+n} conj(xi^l_{mn})), and d^l_{nm} = (-1)^{m-n} d^l_{mn}:
// the four pairs (m,n), (n,m), (-m,-n), (-n,-m) share one recursion, and (-m,-n) contributes what
// (m,n) contributes.  An "orbit" (m,n) with m >= |n| therefore carries two slots (m,n) and (n,m) with
// weights 2 (1 for (0,0), slot (n,m) dropped on the diagonals n = +-m).  Row m of the shared-memory
// table holds, for l = m..Lb and n = -m..m (n fastest), the float4 P_l (w1 xi_mn, w2 (-1)^{m-n} xi_nm).
//
// d^l_{mn}(beta) for l >= m >= |n| obeys the three-term recursion in l
//   d^l = A_l (cos beta - B_l) d^{l-1} - C_l d^{l-2},
//   A_l = l(2l-1)/u_l, B_l = m n /(l(l-1)), C_l = l u_{l-1} / ((l-1) u_l), u_l = sqrt((l^2-m^2)(l^2-n^2)),
// from the closed form d^m_{mn} = (-1)^{m-n} sqrt(C(2m, m+n)) cos(beta/2)^{m+n} sin(beta/2)^{m-n}.
// Writing d^l = P_l e^l with P_l = prod_{j=m+1..l} j(2j-1)/u_j (independent of beta, folded into the
// table) turns it into a recursion with rational coefficients and no square root:
//   e^l = (cos beta - B_l) e^{l-1} - g_l e^{l-2},  g_l = ((l-1)^2-m^2)((l-1)^2-n^2) / ((l-1)^2 (2l-1)(2l-3)),
// and its beta-derivative  e'^l = (cos beta - B_l) e'^{l-1} - sin beta e^{l-1} - g_l e'^{l-2}.
// The Euler angles never appear explicitly: cos(beta/2) = |(w,z)|, sin(beta/2) = |(x,y)|,
// e^{i(alpha+gamma)/2} = (w + i z)/cos(beta/2), e^{i(alpha-gamma)/2} = (y - i x)/sin(beta/2).
//
// Gradient along right perturbations R exp(eps J_i) (body axes): from dS/dalpha, dS/dbeta, dS/dgamma
// with the ZYZ body angular velocity  omega = alpha'(-sb cg, sb sg, cb) + beta'(sg, cg, 0) + gamma'(0,0,1):
//   g_z = dS/dgamma,  g_x sg + g_y cg = dS/dbeta,  g_x cg - g_y sg = (cos beta dS/dgamma - dS/dalpha)/sin beta.
// (At sin beta -> 0 the last line loses FP32 precision as eps/|sin beta|; exactly at 0 it is taken as 0.)
//
// Work split: one CTA per subtomogram; lane group of G threads per start; within a row m the 2m+1
// orbits are dealt round-robin to the G lanes, which reduce their partial sums by xor-shuffles.  (The
// lanes of a warp step through the rows in lockstep, so a row costs the warp its longest lane whatever
// the dealing; only the FP64 re-score, whose starts span several warps, deals by flat orbit index.)
#include <algorithm>
#include <atomic>
#include <cmath>
#include <memory>
#include <mutex>
#include <vector>

#include "bh_internal.h"

namespace bh {
namespace {

constexpr int kBinStride = 2 * kMaxL + 1;

// Per-band constants of the rescaled recursion, read with a warp-uniform index (every lane of a warp
// steps through the same l): l >= 2: (1/(l(l-1)), 1/((l-1)^2 (2l-1)(2l-3)), (l-1)^2, l(l+1)); below:
// (0, 0, 0, l(l+1)).
__constant__ float4 c_ecoef[kMaxL + 4];  // two spare entries: the loops fetch the next pair of bands ahead

constexpr int kMaxStages = 8;
static_assert(kMaxStages == BH_MAX_STAGES, "schedule rows of the C ABI");
constexpr int kMaxThreads = 512;  // threads per CTA (S * G rounded up to a warp)

struct AlignArgs {
  Layout lay;
  const float2* tmpl;
  const int* tmpl_index;
  int n_templates;
  const float2* sub;
  int B;
  const float4* starts;  // [B][S] rotations (align) or evaluation rotations (score)
  int S;
  int nstages;
  int stages[kMaxStages];
  int steps;
  int Lb;  // band of the shared-memory table (the largest band any subtomogram of the launch uses)
  const int* stage_table;  // [B][kMaxStages + 1] (count, bands) per subtomogram, or NULL: stages[] for all
  const float* P;       // [orbit table of band Lmax] P_l(m,n) = prod_{j=m+1..l} j(2j-1)/u_j
  const float* lbin;    // [m][m+n] 0.5 log2 C(2m, m+n), row stride 2 kMaxL + 1
  float4* quat_out;
  float* score_out;
  float4* start_quat_out;
  float* start_score_out;
  float* grad_out;  // score kernel: [B][S][3]
  float* hess_out;  // score kernel: [B][S][6] (xx, xy, xz, yy, yz, zz) or NULL
  double* score64_out;  // refine kernel: [B] FP64 score of the selected start (may be NULL)
};

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cpow(float2 a, int k) {
  float2 r = make_float2(1.f, 0.f);
  for (int i = 0; i < k; ++i) r = cmul(r, a);
  return r;
}

// Entries before row m of an orbit table of band Lb: sum_{j<m} (2j+1)(Lb-j+1).
__host__ __device__ __forceinline__ int tab_base(int m, int Lb) {
  return (Lb + 1) * m * m - ((m - 1) * m * (2 * m - 1) / 3 + (m - 1) * m / 2);
}

__device__ __forceinline__ float4 qnormalize(float4 q) {
  const float r = rsqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
  return make_float4(q.x * r, q.y * r, q.z * r, q.w * r);
}

// Hamilton product a*b of quaternions stored (w, x, y, z) in (x, y, z, w) of a float4.
__device__ __forceinline__ float4 qmul(float4 a, float4 b) {
  return make_float4(a.x * b.x - a.y * b.y - a.z * b.z - a.w * b.w, a.x * b.y + a.y * b.x + a.z * b.w - a.w * b.z,
                     a.x * b.z - a.y * b.w + a.z * b.x + a.w * b.y, a.x * b.w + a.y * b.z - a.z * b.y + a.w * b.x);
}

// Orbit table of one subtomogram (see header comment) for l <= Lb.
__device__ void build_table(float4* __restrict__ tab, const Layout& lay, const float2* __restrict__ tmpl,
                            const float2* __restrict__ sub, const float* __restrict__ P, int Lb, int tid, int nth) {
  const int nent = tab_base(Lb + 1, Lb);
  for (int e = tid; e < nent; e += nth) {
    int m = 0;
    while (tab_base(m + 1, Lb) <= e) ++m;
    const int w = 2 * m + 1;
    const int rem = e - tab_base(m, Lb);
    const int l = m + rem / w, n = rem % w - m;
    const int K = lay.K[l], off = lay.off[l], wl = 2 * l + 1;
    const bool two = (m > 0) && (n != m) && (n != -m);
    // four radial indices per iteration, so that eight (sixteen) L2 loads are in flight per thread: at
    // large bands few warps share an SM and the build is bound by load latency
    float2 x1 = make_float2(0.f, 0.f), x2 = make_float2(0.f, 0.f);
    const float2* tp = tmpl + off + l;
    const float2* fp = sub + off + l;
    int k = 0;
    for (; k + 4 <= K; k += 4) {
      float2 tm[4], fn[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        tm[u] = __ldg(tp + (k + u) * wl + m);
        fn[u] = __ldg(fp + (k + u) * wl + n);
      }
      float2 tn[4], fm[4];
      if (two) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          tn[u] = __ldg(tp + (k + u) * wl + n);
          fm[u] = __ldg(fp + (k + u) * wl + m);
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        x1.x += tm[u].x * fn[u].x + tm[u].y * fn[u].y;
        x1.y += tm[u].x * fn[u].y - tm[u].y * fn[u].x;
        if (two) {
          x2.x += tn[u].x * fm[u].x + tn[u].y * fm[u].y;
          x2.y += tn[u].x * fm[u].y - tn[u].y * fm[u].x;
        }
      }
    }
    for (; k < K; ++k) {
      const float2 tm = __ldg(tp + k * wl + m), fn = __ldg(fp + k * wl + n);
      x1.x += tm.x * fn.x + tm.y * fn.y;
      x1.y += tm.x * fn.y - tm.y * fn.x;
      if (two) {
        const float2 tn = __ldg(tp + k * wl + n), fm = __ldg(fp + k * wl + m);
        x2.x += tn.x * fm.x + tn.y * fm.y;
        x2.y += tn.x * fm.y - tn.y * fm.x;
      }
    }
    const float pl = __ldg(P + tab_base(m, lay.Lmax) + (l - m) * w + (n + m));
    const float w1 = ((m == 0) ? 1.f : 2.f) * pl;
    const float w2 = two ? (((m - n) & 1) ? -2.f : 2.f) * pl : 0.f;
    tab[e] = make_float4(w1 * x1.x, w1 * x1.y, w2 * x2.x, w2 * x2.y);
  }
}

struct Eval {
  float S, gx, gy, gz;
};

// g_l = ((l-1)^2 - m^2)((l-1)^2 - n^2) / ((l-1)^2 (2l-1)(2l-3)) of the rescaled recursion for orbit (m, n), from
// k = c_ecoef[l] (k.z = (l-1)^2, k.y = the inverse denominator), sq2 = m^2 + n^2 and pq2 = m^2 n^2: the
// numerator a (a - sq2) + pq2 is an integer below 2^24 for l <= 45, exact in FP32, so the one rounding is at the scale
// (the same value as the two-factor product, in three operations instead of four).
__device__ __forceinline__ float gcoef(float4 k, float sq2, float pq2) { return fmaf(k.z, k.z - sq2, pq2) * k.y; }

// Score and body-frame gradient (FP32) of C rotations at once (C starts of one subtomogram) at band L, from
// the orbit table of band Lb >= L.  Every lane of a G-group returns the same (bitwise) results.  For C > 1
// the evaluation is shared: (C starts of one subtomogram): each orbit-step loads the
// table entry, the per-band constants and the rational coefficient g once and advances C independent
// recursions, so the shared part of the step is paid once per C starts and every thread carries C
// independent FMA chains.  With T = 2 the same rotations are scored against a second table of the same
// band (tab2; out[j * T + 1]): the d-recursion, seeds and phases -- functions of the rotation only -- are
// computed once and only the accumulations against the table entries are repeated.  Results for each
// table are bitwise those of a separate evaluation (the same operations in the same order).
template <int G, int C, int T = 1>
__device__ void eval_rotations(const float4* __restrict__ tab, const float4* __restrict__ tab2, int Lb, int L,
                               const float4 (&q)[C], int qg, const float* __restrict__ lbin, Eval (&out)[C * T]) {
  static_assert(T == 1 || T == 2, "one or two tables");
  float xb[C], sinb[C], lcc[C], lss[C], rcs[C], rsc[C];
  float2 es[C], ed[C], R1[C], R2[C], Ed2[C], Uq[C], Wrow[C];
#pragma unroll
  for (int j = 0; j < C; ++j) {
    const float w = q[j].x, x = q[j].y, y = q[j].z, z = q[j].w;
    const float cb = sqrtf(w * w + z * z), sb = sqrtf(x * x + y * y);
    es[j] = cb > 0.f ? make_float2(w / cb, z / cb) : make_float2(1.f, 0.f);
    ed[j] = sb > 0.f ? make_float2(y / sb, -x / sb) : make_float2(1.f, 0.f);
    xb[j] = (cb - sb) * (cb + sb);
    sinb[j] = 2.f * cb * sb;
    const float cbc = fmaxf(cb, 1e-30f), sbc = fmaxf(sb, 1e-30f);
    lcc[j] = log2f(cbc);
    lss[j] = log2f(sbc);
    rcs[j] = cbc / sbc;
    rsc[j] = sbc / cbc;
    const float2 Es = cconj(es[j]);
    const float2 EsG = cpow(Es, G), edG = cpow(ed[j], G);
    // along a lane's orbits in a row (n += G) the two phases are geometric with ratios R1, R2
    R1[j] = cmul(EsG, edG);
    R2[j] = cmul(EsG, cconj(edG));
    const float2 Ed = cconj(ed[j]);
    Ed2[j] = cmul(Ed, Ed);
    Uq[j] = cpow(Es, qg);
    Wrow[j] = cpow(ed[j], qg);
  }
  constexpr int CT = C * T;  // accumulator sets: start j, table k at j * T + k
  float S[CT], Sa[CT], Sb[CT], Sg[CT];
#pragma unroll
  for (int j = 0; j < CT; ++j) S[j] = Sa[j] = Sb[j] = Sg[j] = 0.f;
  for (int m = 0; m <= L; ++m) {
    const int w = 2 * m + 1;
    const float4* rowp = tab + tab_base(m, Lb);
    const float4* rowp2 = (T == 2) ? tab2 + tab_base(m, Lb) : rowp;
    const float fm2 = (float)(m * m);
    float2 P1[C], P2[C];
    // row sums: Re z1 + Re z2, Im z1, Im z2, n Im z1, n Im z2, and the beta-derivative part
    float rS[CT], rI1[CT], rI2[CT], rN1[CT], rN2[CT], rB[CT];
#pragma unroll
    for (int j = 0; j < C; ++j) {
      P1[j] = cmul(Uq[j], Wrow[j]);
      P2[j] = cmul(Uq[j], cconj(Wrow[j]));
    }
#pragma unroll
    for (int i = 0; i < CT; ++i) rS[i] = rI1[i] = rI2[i] = rN1[i] = rN2[i] = rB[i] = 0.f;
    for (int n = qg - m; n <= m; n += G) {
      const float lb = __ldg(lbin + m * kBinStride + m + n);
      const float fa = (float)(m + n), fd = (float)(m - n), fn = (float)n;
      const bool odd = (m - n) & 1;
      float e1[C], e2[C], p1[C], p2[C];
      float a1r[CT], a1i[CT], a2r[CT], a2i[CT], b1r[CT], b1i[CT], b2r[CT], b2i[CT];
      const float4* ep = rowp + (n + m);
      const float4* ep2 = rowp2 + (n + m);
      float4 xv[T];
      xv[0] = *ep;
      if (T == 2) xv[T - 1] = *ep2;
#pragma unroll
      for (int j = 0; j < C; ++j) {
        float d = exp2f(lb + fa * lcc[j] + fd * lss[j]);
        d = odd ? -d : d;
        const float dp = 0.5f * d * (fd * rcs[j] - fa * rsc[j]);
#pragma unroll
        for (int k = 0; k < T; ++k) {
          const int i = j * T + k;
          a1r[i] = d * xv[k].x; a1i[i] = d * xv[k].y; a2r[i] = d * xv[k].z; a2i[i] = d * xv[k].w;
          b1r[i] = dp * xv[k].x; b1i[i] = dp * xv[k].y; b2r[i] = dp * xv[k].z; b2i[i] = dp * xv[k].w;
        }
        e1[j] = d; e2[j] = 0.f; p1[j] = dp; p2[j] = 0.f;
      }
      const float mn = (float)(m * n), fn2 = (float)(n * n);
      const float sq2 = fm2 + fn2, pq2 = fm2 * fn2;  // m^2 + n^2, m^2 n^2
      // one step of band l for start j: (E1, E2, P1, P2) -> (EN, PN), accumulated against every table's X
#define BH_STEP(J, EN, PN, E1, E2, P1, P2, K, G_, X)                                 \
  {                                                                                \
    const float t_ = fmaf(-mn, (K).x, xb[J]);                                      \
    EN = fmaf(t_, E1, -(G_) * E2);                                                 \
    PN = fmaf(t_, P1, -fmaf(sinb[J], E1, (G_) * P2));                              \
    _Pragma("unroll") for (int k_ = 0; k_ < T; ++k_) {                             \
      const int i_ = (J) * T + k_;                                                 \
      a1r[i_] = fmaf(EN, (X)[k_].x, a1r[i_]); a1i[i_] = fmaf(EN, (X)[k_].y, a1i[i_]); \
      a2r[i_] = fmaf(EN, (X)[k_].z, a2r[i_]); a2i[i_] = fmaf(EN, (X)[k_].w, a2i[i_]); \
      b1r[i_] = fmaf(PN, (X)[k_].x, b1r[i_]); b1i[i_] = fmaf(PN, (X)[k_].y, b1i[i_]); \
      b2r[i_] = fmaf(PN, (X)[k_].z, b2r[i_]); b2i[i_] = fmaf(PN, (X)[k_].w, b2i[i_]); \
    }                                                                              \
  }
      int l = m + 1;
      for (; l + 1 <= L; l += 2) {  // two bands per iteration: no register rotation, half the loop overhead
        const float4 k0 = c_ecoef[l], k1 = c_ecoef[l + 1];
        float4 x0[T], x1[T];
        x0[0] = ep[w];
        x1[0] = ep[2 * w];
        if (T == 2) {
          x0[T - 1] = ep2[w];
          x1[T - 1] = ep2[2 * w];
          ep2 += 2 * w;
        }
        ep += 2 * w;
        const float g0 = gcoef(k0, sq2, pq2);
        const float g1 = gcoef(k1, sq2, pq2);
#pragma unroll
        for (int j = 0; j < C; ++j) {
          float ea, pa, eb, pb;
          BH_STEP(j, ea, pa, e1[j], e2[j], p1[j], p2[j], k0, g0, x0);
          BH_STEP(j, eb, pb, ea, e1[j], pa, p1[j], k1, g1, x1);
          e2[j] = ea; e1[j] = eb; p2[j] = pa; p1[j] = pb;
        }
      }
      if (l <= L) {
        const float4 k0 = c_ecoef[l];
        float4 x0[T];
        x0[0] = ep[w];
        if (T == 2) x0[T - 1] = ep2[w];
        const float g0 = gcoef(k0, sq2, pq2);
#pragma unroll
        for (int j = 0; j < C; ++j) {
          float ea, pa;
          BH_STEP(j, ea, pa, e1[j], e2[j], p1[j], p2[j], k0, g0, x0);
        }
      }
#undef BH_STEP
#pragma unroll
      for (int j = 0; j < C; ++j) {
#pragma unroll
        for (int k = 0; k < T; ++k) {
          const int i = j * T + k;
          const float z1r = P1[j].x * a1r[i] - P1[j].y * a1i[i], z1i = P1[j].x * a1i[i] + P1[j].y * a1r[i];
          const float z2r = P2[j].x * a2r[i] - P2[j].y * a2i[i], z2i = P2[j].x * a2i[i] + P2[j].y * a2r[i];
          rS[i] += z1r + z2r;
          rI1[i] += z1i;
          rI2[i] += z2i;
          rN1[i] = fmaf(fn, z1i, rN1[i]);
          rN2[i] = fmaf(fn, z2i, rN2[i]);
          rB[i] += (P1[j].x * b1r[i] - P1[j].y * b1i[i]) + (P2[j].x * b2r[i] - P2[j].y * b2i[i]);
        }
        P1[j] = cmul(P1[j], R1[j]);
        P2[j] = cmul(P2[j], R2[j]);
      }
    }
    const float fm = (float)m;
#pragma unroll
    for (int j = 0; j < C; ++j) {
#pragma unroll
      for (int k = 0; k < T; ++k) {
        const int i = j * T + k;
        S[i] += rS[i];
        Sa[i] += fm * rI1[i] + rN2[i];
        Sg[i] += rN1[i] + fm * rI2[i];
        Sb[i] += rB[i];
      }
      Wrow[j] = cmul(Wrow[j], Ed2[j]);
    }
  }
#pragma unroll
  for (int j = 0; j < C; ++j) {
    const float2 eg = cmul(es[j], cconj(ed[j]));
#pragma unroll
    for (int k = 0; k < T; ++k) {
      const int i = j * T + k;
#pragma unroll
      for (int o = 1; o < G; o <<= 1) {
        S[i] += __shfl_xor_sync(0xffffffffu, S[i], o);
        Sa[i] += __shfl_xor_sync(0xffffffffu, Sa[i], o);
        Sb[i] += __shfl_xor_sync(0xffffffffu, Sb[i], o);
        Sg[i] += __shfl_xor_sync(0xffffffffu, Sg[i], o);
      }
      const float Q = (sinb[j] > 1e-30f) ? (xb[j] * Sg[i] - Sa[i]) / sinb[j] : 0.f;
      out[i].S = S[i];
      out[i].gx = Sb[i] * eg.y + Q * eg.x;
      out[i].gy = Sb[i] * eg.x - Q * eg.y;
      out[i].gz = Sg[i];
    }
  }
}

// Row m of the flat orbit index o = m^2 + m + n (0 <= o < 2^22).
__device__ __forceinline__ int orbit_row(int o) {
  int m = (int)sqrtf((float)o);
  m -= (m * m > o) ? 1 : 0;
  m += ((m + 1) * (m + 1) <= o) ? 1 : 0;
  return m;
}

// z^k, 0 <= k < 2^7, by binary exponentiation (the phases of a lane's first orbit, and the rare jumps of a
// lane over more than one row).
__device__ __forceinline__ float2 cpow_bin(float2 z, int k) {
  float2 r = make_float2(1.f, 0.f);
  while (k > 0) {
    if (k & 1) r = cmul(r, z);
    z = cmul(z, z);
    k >>= 1;
  }
  return r;
}

// The evaluation of eval_rotations (T = 1) with the orbits dealt in flat order across rows: orbit
// o = m^2 + m + n, 0 <= o < (L+1)^2, goes to lane o mod G of the group, so consecutive rounds ("chunks") of G
// orbits straddle row boundaries instead of leaving lanes idle at the end of every row (a row of 2m+1
// orbits dealt to G lanes idles G - ((2m+1) mod G) lanes for the whole row).  The lanes of a chunk run one
// l-loop from the chunk's lowest row: a lane whose row starts later has a zero recursion state until its
// own l = m, where its closed-form seed is injected (a select), so its extra steps add zeros.  Per-orbit
// phases e^{-i(m alpha + n gamma)} and e^{-i(n alpha + m gamma)} follow the lane from orbit to orbit:
// within a row they advance by the ratios R1, R2 of an n-step of G, and on a step into the next row
// (m, n) -> (m+1, n + G - 2m - 2) by the extra factors Ed^2 e^{i gamma (2m+1)} and ed^2 e^{i alpha (2m+1)},
// themselves advanced by e^{2i gamma}, e^{2i alpha} per row; a jump over several rows (only while 2m+3 < G)
// recomputes them by binary powers.  The sums over (m, n) are not factored by row, so results differ from
// eval_rotations by rounding only.
template <int G, int C>
__device__ void eval_flat(const float4* __restrict__ tab, int Lb, int L, const float4 (&q)[C], int qg,
                          const float* __restrict__ lbin, Eval (&out)[C]) {
  float xb[C], sinb[C], lcc[C], lss[C], rcs[C], rsc[C];
  float2 es[C], ed[C], R1[C], R2[C], E2g[C], E2a[C], P1[C], P2[C], U1[C], U2[C];
  const int norb = (L + 1) * (L + 1);
  int m = orbit_row(qg), n = qg - m * m - m;  // the lane's orbit (m, n); it is live while m <= L
  int rowbase = tab_base(m, Lb);              // first table entry of row m
#pragma unroll
  for (int j = 0; j < C; ++j) {
    const float w = q[j].x, x = q[j].y, y = q[j].z, z = q[j].w;
    const float cb = sqrtf(w * w + z * z), sb = sqrtf(x * x + y * y);
    es[j] = cb > 0.f ? make_float2(w / cb, z / cb) : make_float2(1.f, 0.f);
    ed[j] = sb > 0.f ? make_float2(y / sb, -x / sb) : make_float2(1.f, 0.f);
    xb[j] = (cb - sb) * (cb + sb);
    sinb[j] = 2.f * cb * sb;
    const float cbc = fmaxf(cb, 1e-30f), sbc = fmaxf(sb, 1e-30f);
    lcc[j] = log2f(cbc);
    lss[j] = log2f(sbc);
    rcs[j] = cbc / sbc;
    rsc[j] = sbc / cbc;
    const float2 Es = cconj(es[j]), Ed = cconj(ed[j]);
    const float2 EsG = cpow(Es, G), edG = cpow(ed[j], G);
    R1[j] = cmul(EsG, edG);
    R2[j] = cmul(EsG, cconj(edG));
    const float2 eig = cmul(es[j], Ed), eia = cmul(es[j], ed[j]);  // e^{i gamma}, e^{i alpha}
    E2g[j] = cmul(eig, eig);
    E2a[j] = cmul(eia, eia);
    const float2 pa = cpow_bin(Es, m + n);
    P1[j] = cmul(pa, cpow_bin(Ed, m - n));
    P2[j] = cmul(pa, cpow_bin(ed[j], m - n));
    U1[j] = cmul(cmul(Ed, Ed), cpow_bin(eig, 2 * m + 1));
    U2[j] = cmul(cmul(ed[j], ed[j]), cpow_bin(eia, 2 * m + 1));
  }
  float S[C], Sa[C], Sb[C], Sg[C];
#pragma unroll
  for (int j = 0; j < C; ++j) S[j] = Sa[j] = Sb[j] = Sg[j] = 0.f;
  int m_lo = 0, m_hi = 0;  // rows of the chunk's first and last orbits (the same for every lane)
  for (int c0 = 0; c0 < norb; c0 += G) {
    while ((m_lo + 1) * (m_lo + 1) <= c0) ++m_lo;
    const int last = min(c0 + G, norb) - 1;
    while ((m_hi + 1) * (m_hi + 1) <= last) ++m_hi;
    const bool live = m <= L;
    const int wl = live ? 2 * m + 1 : 0;
    const float4* ep0 = tab + (live ? rowbase + (n + m) : 0);
    const float lb = live ? __ldg(lbin + m * kBinStride + m + n) : 0.f;
    const float fa = (float)(m + n), fd = (float)(m - n), fn = (float)n, fm = (float)m;
    const bool odd = (m - n) & 1;
    const float mn = (float)(m * n), fm2 = (float)(m * m), fn2 = (float)(n * n);
    const float sq2 = fm2 + fn2, pq2 = fm2 * fn2;  // m^2 + n^2, m^2 n^2
    float e1[C], e2[C], p1[C], p2[C], ds[C], dps[C];
    float a1r[C], a1i[C], a2r[C], a2i[C], b1r[C], b1i[C], b2r[C], b2i[C];
#pragma unroll
    for (int j = 0; j < C; ++j) {
      float d = live ? exp2f(lb + fa * lcc[j] + fd * lss[j]) : 0.f;
      d = odd ? -d : d;
      ds[j] = d;
      dps[j] = 0.5f * d * (fd * rcs[j] - fa * rsc[j]);
      e1[j] = e2[j] = p1[j] = p2[j] = 0.f;
      a1r[j] = a1i[j] = a2r[j] = a2i[j] = b1r[j] = b1i[j] = b2r[j] = b2i[j] = 0.f;
    }
#define BH_FSTEP(J, EN, PN, E1, E2, P1_, P2_, K, G_, X)                                \
  {                                                                                 \
    const float t_ = fmaf(-mn, (K).x, xb[J]);                                       \
    EN = fmaf(t_, E1, -(G_) * E2);                                                  \
    PN = fmaf(t_, P1_, -fmaf(sinb[J], E1, (G_) * P2_));                             \
  }
#define BH_FACC(J, EN, PN, X)                                                       \
  {                                                                                 \
    a1r[J] = fmaf(EN, (X).x, a1r[J]); a1i[J] = fmaf(EN, (X).y, a1i[J]);             \
    a2r[J] = fmaf(EN, (X).z, a2r[J]); a2i[J] = fmaf(EN, (X).w, a2i[J]);             \
    b1r[J] = fmaf(PN, (X).x, b1r[J]); b1i[J] = fmaf(PN, (X).y, b1i[J]);             \
    b2r[J] = fmaf(PN, (X).z, b2r[J]); b2i[J] = fmaf(PN, (X).w, b2i[J]);             \
  }
    if (m_lo == m_hi) {  // one row: every live lane starts at l = m_lo with its seed (dead lanes: d = 0)
      const float4 X = ep0[0];
#pragma unroll
      for (int j = 0; j < C; ++j) {
        e1[j] = ds[j];
        p1[j] = dps[j];
        BH_FACC(j, ds[j], dps[j], X);
      }
    }
    // l = m_lo .. m_hi over two or more rows: each lane's orbit starts at its own row m (seed injected
    // there; zeros before)
    for (int l = m_lo; l <= m_hi && m_lo < m_hi; ++l) {
      const float4 X = ep0[(max(l, m) - m) * wl];
      const float4 k0 = c_ecoef[l];
      const float g0 = gcoef(k0, sq2, pq2);
      const bool start = (l == m);
#pragma unroll
      for (int j = 0; j < C; ++j) {
        float en, pn;
        BH_FSTEP(j, en, pn, e1[j], e2[j], p1[j], p2[j], k0, g0, X);
        en = start ? ds[j] : en;
        pn = start ? dps[j] : pn;
        BH_FACC(j, en, pn, X);
        e2[j] = e1[j]; e1[j] = en; p2[j] = p1[j]; p1[j] = pn;
      }
    }
    // l = m_hi+1 .. L: every live lane is inside its orbit
    // two bands per iteration, the next pair's constants fetched one iteration ahead; then a last single step
    const float4* ep = ep0 + (m_hi + 1 - m) * wl;
    int l = m_hi + 1;
    float4 k0 = c_ecoef[l], k1 = c_ecoef[l + 1];
    for (; l + 1 <= L; l += 2) {
      const float4 x0 = ep[0], x1 = ep[wl];
      ep += 2 * wl;
      const float4 kn0 = c_ecoef[l + 2], kn1 = c_ecoef[l + 3];
      const float g0 = gcoef(k0, sq2, pq2), g1 = gcoef(k1, sq2, pq2);
#pragma unroll
      for (int j = 0; j < C; ++j) {
        float ea, pa, eb, pb;
        BH_FSTEP(j, ea, pa, e1[j], e2[j], p1[j], p2[j], k0, g0, x0);
        BH_FACC(j, ea, pa, x0);
        BH_FSTEP(j, eb, pb, ea, e1[j], pa, p1[j], k1, g1, x1);
        BH_FACC(j, eb, pb, x1);
        e2[j] = ea; e1[j] = eb; p2[j] = pa; p1[j] = pb;
      }
      k0 = kn0;
      k1 = kn1;
    }
    if (l <= L) {
      const float4 x0 = ep[0];
      const float g0 = gcoef(k0, sq2, pq2);
#pragma unroll
      for (int j = 0; j < C; ++j) {
        float ea, pa;
        BH_FSTEP(j, ea, pa, e1[j], e2[j], p1[j], p2[j], k0, g0, x0);
        BH_FACC(j, ea, pa, x0);
      }
    }
#undef BH_FSTEP
#undef BH_FACC
    // the orbit's terms: S += Re z1 + Re z2, dS/dalpha += m Im z1 + n Im z2, dS/dgamma += n Im z1 + m Im z2,
    // dS/dbeta += Re y1 + Re y2 (z = phase x xi-sum, y = phase x derivative sum)
#pragma unroll
    for (int j = 0; j < C; ++j) {
      const float z1r = P1[j].x * a1r[j] - P1[j].y * a1i[j], z1i = P1[j].x * a1i[j] + P1[j].y * a1r[j];
      const float z2r = P2[j].x * a2r[j] - P2[j].y * a2i[j], z2i = P2[j].x * a2i[j] + P2[j].y * a2r[j];
      S[j] += z1r + z2r;
      Sa[j] = fmaf(fm, z1i, fmaf(fn, z2i, Sa[j]));
      Sg[j] = fmaf(fn, z1i, fmaf(fm, z2i, Sg[j]));
      Sb[j] += (P1[j].x * b1r[j] - P1[j].y * b1i[j]) + (P2[j].x * b2r[j] - P2[j].y * b2i[j]);
    }
    // the lane's next orbit, G further in flat order: n advances by G (phases by R1, R2); each wrap into
    // the next row, (m, n) -> (m+1, n - 2m - 2), multiplies them by the row factors U1, U2, which then
    // advance by e^{2i gamma}, e^{2i alpha}
    n += G;
#pragma unroll
    for (int j = 0; j < C; ++j) {
      P1[j] = cmul(P1[j], R1[j]);
      P2[j] = cmul(P2[j], R2[j]);
    }
    while (n > m) {
      n -= 2 * m + 2;
      rowbase += (2 * m + 1) * (Lb - m + 1);
      ++m;
#pragma unroll
      for (int j = 0; j < C; ++j) {
        P1[j] = cmul(P1[j], U1[j]);
        P2[j] = cmul(P2[j], U2[j]);
        U1[j] = cmul(U1[j], E2g[j]);
        U2[j] = cmul(U2[j], E2a[j]);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < C; ++j) {
    const float2 eg = cmul(es[j], cconj(ed[j]));
#pragma unroll
    for (int s = 1; s < G; s <<= 1) {
      S[j] += __shfl_xor_sync(0xffffffffu, S[j], s);
      Sa[j] += __shfl_xor_sync(0xffffffffu, Sa[j], s);
      Sb[j] += __shfl_xor_sync(0xffffffffu, Sb[j], s);
      Sg[j] += __shfl_xor_sync(0xffffffffu, Sg[j], s);
    }
    const float Q = (sinb[j] > 1e-30f) ? (xb[j] * Sg[j] - Sa[j]) / sinb[j] : 0.f;
    out[j].S = S[j];
    out[j].gx = Sb[j] * eg.y + Q * eg.x;
    out[j].gy = Sb[j] * eg.x - Q * eg.y;
    out[j].gz = Sg[j];
  }
}

template <int G>
__device__ __forceinline__ Eval eval_one(const float4* __restrict__ tab, int Lb, int L, float4 q, int qg,
                                         const float* __restrict__ lbin) {
  const float4 qq[1] = {q};
  Eval e[1];
  eval_rotations<G, 1>(tab, nullptr, Lb, L, qq, qg, lbin, e);
  return e[0];
}

struct EvalH {
  float S, gx, gy, gz;
  float hxx, hxy, hxz, hyy, hyz, hzz;  // symmetric body-frame Hessian
};

// The Hessian evaluations' common end: the group's sums over its G lanes, then the body-frame gradient and
// the symmetrised body-frame Hessian from the Euler-angle sums (S, its first derivatives Sa, Sb, Sg, the second
// ones Saa, Sab, Sag, Sbg, Sgg, and Sk, SL for the second beta derivative).
template <int G>
__device__ EvalH finish_hess(float S, float Sa, float Sb, float Sg, float Saa, float Sab, float Sag, float Sbg,
                             float Sgg, float Sk, float SL, float2 es, float2 ed, float xb, float sinb) {
#pragma unroll
  for (int o = 1; o < G; o <<= 1) {
    S += __shfl_xor_sync(0xffffffffu, S, o);
    Sa += __shfl_xor_sync(0xffffffffu, Sa, o);
    Sb += __shfl_xor_sync(0xffffffffu, Sb, o);
    Sg += __shfl_xor_sync(0xffffffffu, Sg, o);
    Saa += __shfl_xor_sync(0xffffffffu, Saa, o);
    Sab += __shfl_xor_sync(0xffffffffu, Sab, o);
    Sag += __shfl_xor_sync(0xffffffffu, Sag, o);
    Sbg += __shfl_xor_sync(0xffffffffu, Sbg, o);
    Sgg += __shfl_xor_sync(0xffffffffu, Sgg, o);
    Sk += __shfl_xor_sync(0xffffffffu, Sk, o);
    SL += __shfl_xor_sync(0xffffffffu, SL, o);
  }
  const float2 eg = cmul(es, cconj(ed));  // (cos gamma, sin gamma)
  const float cG = eg.x, sG = eg.y;
  EvalH r;
  r.S = S;
  if (!(sinb > 1e-4f)) {  // Euler chart singular: gradient only along gamma, no curvature information
    const float Q = 0.f;
    r.gx = Sb * sG + Q * cG;
    r.gy = Sb * cG - Q * sG;
    r.gz = Sg;
    r.hxx = r.hxy = r.hxz = r.hyy = r.hyz = r.hzz = 0.f;
    return r;
  }
  const float isb = 1.f / sinb, isb2 = isb * isb;
  const float Q = (xb * Sg - Sa) * isb;
  r.gx = Sb * sG + Q * cG;
  r.gy = Sb * cG - Q * sG;
  r.gz = Sg;
  const float Sbb = -xb * isb * Sb + Sk * isb2 - SL;
  // X_i = v_i . (d_alpha, d_beta, d_gamma); X_i X_j S = v_i^T E v_j + (b_i d_beta v_j + c_i d_gamma v_j) . grad
  const float v[3][3] = {{-cG * isb, sG, xb * cG * isb}, {sG * isb, cG, -xb * sG * isb}, {0.f, 0.f, 1.f}};
  const float dbv[3][3] = {{cG * xb * isb2, 0.f, -cG * isb2}, {-sG * xb * isb2, 0.f, sG * isb2}, {0.f, 0.f, 0.f}};
  const float dgv[3][3] = {{v[1][0], v[1][1], v[1][2]}, {-v[0][0], -v[0][1], -v[0][2]}, {0.f, 0.f, 0.f}};
  const float E[3][3] = {{Saa, Sab, Sag}, {Sab, Sbb, Sbg}, {Sag, Sbg, Sgg}};
  const float gr[3] = {Sa, Sb, Sg};
  float XX[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    float Ev[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) Ev[k] = E[k][0] * v[i][0] + E[k][1] * v[i][1] + E[k][2] * v[i][2];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      float t = v[j][0] * Ev[0] + v[j][1] * Ev[1] + v[j][2] * Ev[2];
#pragma unroll
      for (int k = 0; k < 3; ++k) t = fmaf(v[i][1] * dbv[j][k] + v[i][2] * dgv[j][k], gr[k], t);
      XX[i][j] = t;
    }
  }
  r.hxx = XX[0][0];
  r.hyy = XX[1][1];
  r.hzz = XX[2][2];
  r.hxy = 0.5f * (XX[0][1] + XX[1][0]);
  r.hxz = 0.5f * (XX[0][2] + XX[2][0]);
  r.hyz = 0.5f * (XX[1][2] + XX[2][1]);
  return r;
}

// Score, body-frame gradient and Hessian (FP32) of one rotation at band L (Newton steps, Sec. III).  The
// evaluation follows eval_rotations with C = 1 and adds the second Euler-angle derivatives: along alpha and
// gamma the orbit terms only pick up factors of m and n; the second beta derivative comes from the Wigner
// d equation d'' = -cot(b) d' - [l(l+1) - (m^2 + n^2 - 2mn cos b)/sin^2 b] d, which needs one more sum,
// Lambda = sum_l l(l+1) e_l X_l, per orbit.  The body-frame Hessian is the symmetrised X_i X_j S of the
// vector fields X_i of the gradient.
template <int G>
__device__ EvalH eval_hess(const float4* __restrict__ tab, int Lb, int L, float4 q, int qg,
                           const float* __restrict__ lbin) {
  const float w = q.x, x = q.y, y = q.z, z = q.w;
  const float cb = sqrtf(w * w + z * z), sb = sqrtf(x * x + y * y);
  const float2 es = cb > 0.f ? make_float2(w / cb, z / cb) : make_float2(1.f, 0.f);
  const float2 ed = sb > 0.f ? make_float2(y / sb, -x / sb) : make_float2(1.f, 0.f);
  const float xb = (cb - sb) * (cb + sb), sinb = 2.f * cb * sb;
  const float cbc = fmaxf(cb, 1e-30f), sbc = fmaxf(sb, 1e-30f);
  const float lcc = log2f(cbc), lss = log2f(sbc), rcs = cbc / sbc, rsc = sbc / cbc;
  const float2 Es = cconj(es);
  const float2 EsG = cpow(Es, G), edG = cpow(ed, G);
  const float2 R1 = cmul(EsG, edG), R2 = cmul(EsG, cconj(edG));
  const float2 Ed = cconj(ed);
  const float2 Ed2 = cmul(Ed, Ed);
  const float2 Uq = cpow(Es, qg);
  float2 Wrow = cpow(ed, qg);
  float S = 0.f, Sa = 0.f, Sb = 0.f, Sg = 0.f;
  float Saa = 0.f, Sab = 0.f, Sag = 0.f, Sbg = 0.f, Sgg = 0.f, Sk = 0.f, SL = 0.f;
  for (int m = 0; m <= L; ++m) {
    const int wd = 2 * m + 1;
    const float4* rowp = tab + tab_base(m, Lb);
    const float fm2 = (float)(m * m), fm = (float)m;
    float2 P1 = cmul(Uq, Wrow), P2 = cmul(Uq, cconj(Wrow));
    float rS = 0.f, rI1 = 0.f, rI2 = 0.f, rN1 = 0.f, rN2 = 0.f, rB = 0.f;
    float hU1 = 0.f, hU2 = 0.f, hUn1 = 0.f, hUn2 = 0.f, hUnn1 = 0.f, hUnn2 = 0.f;
    float hY1 = 0.f, hY2 = 0.f, hYn1 = 0.f, hYn2 = 0.f, hL = 0.f;
    for (int n = qg - m; n <= m; n += G) {
      const float lb = __ldg(lbin + m * kBinStride + m + n);
      const float fa = (float)(m + n), fd = (float)(m - n), fn = (float)n;
      const float4* ep = rowp + (n + m);
      const float4 xv = *ep;
      float d = exp2f(lb + fa * lcc + fd * lss);
      d = ((m - n) & 1) ? -d : d;
      const float dp = 0.5f * d * (fd * rcs - fa * rsc);
      const float ll0 = (float)(m * (m + 1));
      float a1r = d * xv.x, a1i = d * xv.y, a2r = d * xv.z, a2i = d * xv.w;
      float b1r = dp * xv.x, b1i = dp * xv.y, b2r = dp * xv.z, b2i = dp * xv.w;
      float q1r = ll0 * a1r, q1i = ll0 * a1i, q2r = ll0 * a2r, q2i = ll0 * a2i;
      float e1 = d, e2 = 0.f, p1 = dp, p2 = 0.f;
      const float mn = (float)(m * n), fn2 = (float)(n * n);
      for (int l = m + 1; l <= L; ++l) {
        const float4 k0 = c_ecoef[l];
        ep += wd;
        const float4 X = *ep;
        const float g0 = (k0.z - fm2) * (k0.z - fn2) * k0.y;
        const float t_ = fmaf(-mn, k0.x, xb);
        const float en = fmaf(t_, e1, -g0 * e2);
        const float pn = fmaf(t_, p1, -fmaf(sinb, e1, g0 * p2));
        a1r = fmaf(en, X.x, a1r); a1i = fmaf(en, X.y, a1i); a2r = fmaf(en, X.z, a2r); a2i = fmaf(en, X.w, a2i);
        b1r = fmaf(pn, X.x, b1r); b1i = fmaf(pn, X.y, b1i); b2r = fmaf(pn, X.z, b2r); b2i = fmaf(pn, X.w, b2i);
        const float el = k0.w * en;
        q1r = fmaf(el, X.x, q1r); q1i = fmaf(el, X.y, q1i); q2r = fmaf(el, X.z, q2r); q2i = fmaf(el, X.w, q2i);
        e2 = e1; e1 = en; p2 = p1; p1 = pn;
      }
      const float z1r = P1.x * a1r - P1.y * a1i, z1i = P1.x * a1i + P1.y * a1r;
      const float z2r = P2.x * a2r - P2.y * a2i, z2i = P2.x * a2i + P2.y * a2r;
      const float y1r = P1.x * b1r - P1.y * b1i, y1i = P1.x * b1i + P1.y * b1r;
      const float y2r = P2.x * b2r - P2.y * b2i, y2i = P2.x * b2i + P2.y * b2r;
      rS += z1r + z2r;
      rI1 += z1i;
      rI2 += z2i;
      rN1 = fmaf(fn, z1i, rN1);
      rN2 = fmaf(fn, z2i, rN2);
      rB += y1r + y2r;
      hU1 += z1r;
      hU2 += z2r;
      hUn1 = fmaf(fn, z1r, hUn1);
      hUn2 = fmaf(fn, z2r, hUn2);
      hUnn1 = fmaf(fn2, z1r, hUnn1);
      hUnn2 = fmaf(fn2, z2r, hUnn2);
      hY1 += y1i;
      hY2 += y2i;
      hYn1 = fmaf(fn, y1i, hYn1);
      hYn2 = fmaf(fn, y2i, hYn2);
      hL += (P1.x * q1r - P1.y * q1i) + (P2.x * q2r - P2.y * q2i);
      P1 = cmul(P1, R1);
      P2 = cmul(P2, R2);
    }
    S += rS;
    Sa += fm * rI1 + rN2;
    Sg += rN1 + fm * rI2;
    Sb += rB;
    Saa -= fm2 * hU1 + hUnn2;
    Sgg -= hUnn1 + fm2 * hU2;
    Sag -= fm * (hUn1 + hUn2);
    Sab += fm * hY1 + hYn2;
    Sbg += hYn1 + fm * hY2;
    Sk += fm2 * (hU1 + hU2) + (hUnn1 + hUnn2) - 2.f * xb * fm * (hUn1 + hUn2);
    SL += hL;
    Wrow = cmul(Wrow, Ed2);
  }
  return finish_hess<G>(S, Sa, Sb, Sg, Saa, Sab, Sag, Sbg, Sgg, Sk, SL, es, ed, xb, sinb);
}

// eval_hess with the orbits dealt in flat order across rows (as eval_flat, one start per group): orbit
// o = m^2 + m + n goes to lane o mod G, a round of G orbits runs one l-loop from its lowest row with each lane's
// seed injected at its own l = m, and the lane's phases follow it from orbit to orbit.  The Euler-angle sums
// are accumulated per orbit with the orbit's own (m, n) factors (eval_hess adds them per row first), so the
// two differ by rounding only.
template <int G>
__device__ EvalH eval_hess_flat(const float4* __restrict__ tab, int Lb, int L, float4 q, int qg,
                                const float* __restrict__ lbin) {
  const float w = q.x, x = q.y, y = q.z, z = q.w;
  const float cb = sqrtf(w * w + z * z), sb = sqrtf(x * x + y * y);
  const float2 es = cb > 0.f ? make_float2(w / cb, z / cb) : make_float2(1.f, 0.f);
  const float2 ed = sb > 0.f ? make_float2(y / sb, -x / sb) : make_float2(1.f, 0.f);
  const float xb = (cb - sb) * (cb + sb), sinb = 2.f * cb * sb;
  const float cbc = fmaxf(cb, 1e-30f), sbc = fmaxf(sb, 1e-30f);
  const float lcc = log2f(cbc), lss = log2f(sbc), rcs = cbc / sbc, rsc = sbc / cbc;
  const float2 Es = cconj(es), Ed = cconj(ed);
  const float2 EsG = cpow(Es, G), edG = cpow(ed, G);
  const float2 R1 = cmul(EsG, edG), R2 = cmul(EsG, cconj(edG));
  const float2 eig = cmul(es, Ed), eia = cmul(es, ed);  // e^{i gamma}, e^{i alpha}
  const float2 E2g = cmul(eig, eig), E2a = cmul(eia, eia);
  const int norb = (L + 1) * (L + 1);
  int m = orbit_row(qg), n = qg - m * m - m;  // the lane's orbit (m, n); it is live while m <= L
  int rowbase = tab_base(m, Lb);
  const float2 pa = cpow_bin(Es, m + n);
  float2 P1 = cmul(pa, cpow_bin(Ed, m - n)), P2 = cmul(pa, cpow_bin(ed, m - n));
  float2 U1 = cmul(cmul(Ed, Ed), cpow_bin(eig, 2 * m + 1)), U2 = cmul(cmul(ed, ed), cpow_bin(eia, 2 * m + 1));
  float S = 0.f, Sa = 0.f, Sb = 0.f, Sg = 0.f;
  float Saa = 0.f, Sab = 0.f, Sag = 0.f, Sbg = 0.f, Sgg = 0.f, Sk = 0.f, SL = 0.f;
  int m_lo = 0, m_hi = 0;  // rows of the round's first and last orbits (the same for every lane)
  for (int c0 = 0; c0 < norb; c0 += G) {
    while ((m_lo + 1) * (m_lo + 1) <= c0) ++m_lo;
    const int last = min(c0 + G, norb) - 1;
    while ((m_hi + 1) * (m_hi + 1) <= last) ++m_hi;
    const bool live = m <= L;
    const int wl = live ? 2 * m + 1 : 0;
    const float4* ep0 = tab + (live ? rowbase + (n + m) : 0);
    const float lb = live ? __ldg(lbin + m * kBinStride + m + n) : 0.f;
    const float fa = (float)(m + n), fd = (float)(m - n), fn = (float)n, fm = (float)m;
    const float mn = (float)(m * n), fm2 = (float)(m * m), fn2 = (float)(n * n);
    const float sq2 = fm2 + fn2, pq2 = fm2 * fn2;
    float d = live ? exp2f(lb + fa * lcc + fd * lss) : 0.f;
    d = ((m - n) & 1) ? -d : d;
    const float dp = 0.5f * d * (fd * rcs - fa * rsc);
    float e1 = 0.f, e2 = 0.f, p1 = 0.f, p2 = 0.f;
    float a1r = 0.f, a1i = 0.f, a2r = 0.f, a2i = 0.f, b1r = 0.f, b1i = 0.f, b2r = 0.f, b2i = 0.f;
    float q1r = 0.f, q1i = 0.f, q2r = 0.f, q2i = 0.f;
#define BH_HSTEP(X, K, G_, INJECT)                                                           \
  {                                                                                          \
    const float t_ = fmaf(-mn, (K).x, xb);                                                   \
    float en = fmaf(t_, e1, -(G_) * e2);                                                     \
    float pn = fmaf(t_, p1, -fmaf(sinb, e1, (G_) * p2));                                     \
    if (INJECT) {                                                                            \
      en = (l == m) ? d : en;                                                                \
      pn = (l == m) ? dp : pn;                                                               \
    }                                                                                        \
    a1r = fmaf(en, (X).x, a1r); a1i = fmaf(en, (X).y, a1i);                                  \
    a2r = fmaf(en, (X).z, a2r); a2i = fmaf(en, (X).w, a2i);                                  \
    b1r = fmaf(pn, (X).x, b1r); b1i = fmaf(pn, (X).y, b1i);                                  \
    b2r = fmaf(pn, (X).z, b2r); b2i = fmaf(pn, (X).w, b2i);                                  \
    const float el = (K).w * en;                                                             \
    q1r = fmaf(el, (X).x, q1r); q1i = fmaf(el, (X).y, q1i);                                  \
    q2r = fmaf(el, (X).z, q2r); q2i = fmaf(el, (X).w, q2i);                                  \
    e2 = e1; e1 = en; p2 = p1; p1 = pn;                                                      \
  }
    // l = m_lo .. m_hi: each lane's orbit starts at its own row m (seed injected there; zeros before)
    for (int l = m_lo; l <= m_hi; ++l) {
      const float4 X = ep0[(max(l, m) - m) * wl];
      const float4 k0 = c_ecoef[l];
      const float g0 = gcoef(k0, sq2, pq2);
      BH_HSTEP(X, k0, g0, true);
    }
    // l = m_hi+1 .. L: every live lane is inside its orbit
    const float4* ep = ep0 + (m_hi + 1 - m) * wl;
    for (int l = m_hi + 1; l <= L; ++l) {
      const float4 X = *ep;
      ep += wl;
      const float4 k0 = c_ecoef[l];
      const float g0 = gcoef(k0, sq2, pq2);
      BH_HSTEP(X, k0, g0, false);
    }
#undef BH_HSTEP
    const float z1r = P1.x * a1r - P1.y * a1i, z1i = P1.x * a1i + P1.y * a1r;
    const float z2r = P2.x * a2r - P2.y * a2i, z2i = P2.x * a2i + P2.y * a2r;
    const float y1r = P1.x * b1r - P1.y * b1i, y1i = P1.x * b1i + P1.y * b1r;
    const float y2r = P2.x * b2r - P2.y * b2i, y2i = P2.x * b2i + P2.y * b2r;
    const float zr = z1r + z2r;
    S += zr;
    Sa = fmaf(fm, z1i, fmaf(fn, z2i, Sa));
    Sg = fmaf(fn, z1i, fmaf(fm, z2i, Sg));
    Sb += y1r + y2r;
    Saa -= fmaf(fm2, z1r, fn2 * z2r);
    Sgg -= fmaf(fn2, z1r, fm2 * z2r);
    Sag = fmaf(-mn, zr, Sag);
    Sab = fmaf(fm, y1i, fmaf(fn, y2i, Sab));
    Sbg = fmaf(fn, y1i, fmaf(fm, y2i, Sbg));
    Sk = fmaf(fmaf(-2.f * xb, mn, sq2), zr, Sk);
    SL += (P1.x * q1r - P1.y * q1i) + (P2.x * q2r - P2.y * q2i);
    // the lane's next orbit, G further in flat order (as in eval_flat)
    n += G;
    P1 = cmul(P1, R1);
    P2 = cmul(P2, R2);
    while (n > m) {
      n -= 2 * m + 2;
      rowbase += (2 * m + 1) * (Lb - m + 1);
      ++m;
      P1 = cmul(P1, U1);
      P2 = cmul(P2, U2);
      U1 = cmul(U1, E2g);
      U2 = cmul(U2, E2a);
    }
  }
  return finish_hess<G>(S, Sa, Sb, Sg, Saa, Sab, Sag, Sbg, Sgg, Sk, SL, es, ed, xb, sinb);
}

__device__ __forceinline__ const float2* template_row(const AlignArgs& a, int p) {
  if (!a.tmpl_index) return a.tmpl;
  int t = a.tmpl_index[p];
  t = t < 0 ? 0 : (t >= a.n_templates ? a.n_templates - 1 : t);
  return a.tmpl + (size_t)t * a.lay.Nb;
}

// Marching schedule of subtomogram p into shared memory: sched[0] = number of bands, sched[1..] the bands.
// From the per-subtomogram table when the launch has one -- each band clamped to 1..a.Lb and kept only if
// it exceeds the previous one, so that a malformed row can neither index past the shared-memory table
// (sized for a.Lb) nor stall the marching; an empty row falls back to the launch's own schedule -- else the
// launch's schedule.  Ends with a barrier.
__device__ void load_schedule(const AlignArgs& a, int p, int* sched) {
  if (threadIdx.x == 0) {
    int n = 0;
    if (a.stage_table) {
      const int* row = a.stage_table + (size_t)p * (kMaxStages + 1);
      const int cnt = min(max(row[0], 0), kMaxStages);
      int last = 0;
      for (int i = 0; i < cnt; ++i) {
        const int L = min(max(row[1 + i], 1), a.Lb);
        if (L > last) {
          sched[1 + n++] = L;
          last = L;
        }
      }
    }
    if (n == 0) {
      for (int i = 0; i < a.nstages; ++i) sched[1 + i] = a.stages[i];
      n = a.nstages;
    }
    sched[0] = n;
  }
  __syncthreads();
}

// Minimum resident CTAs per SM requested from the compiler for a block of NT threads.  Small blocks (one
// or two warps) keep 8 resident CTAs (shared memory holds 7 orbit tables of band 16); larger blocks are
// used when the table is large and few CTAs fit, so they get at least 128 registers per thread.
__host__ __device__ constexpr int min_blocks(int NT) { return NT <= 64 ? 8 : NT <= 128 ? 4 : NT <= 256 ? 2 : 1; }
// Kernels that carry C starts per thread need about 180 registers at C = 2: a CTA of NT threads is given
// up to 255 (at least 8 warps' worth of register file per SM), so that the launch bound does not force
// spills; residency then follows from registers and the orbit tables' shared memory.
__host__ __device__ constexpr int min_blocks_c(int NT, int C) {
  return C == 1 ? min_blocks(NT) : (NT <= 32 ? 8 : NT <= 64 ? 4 : NT <= 128 ? 2 : 1);
}

// Multi-start marching ascent; one CTA per subtomogram, blockDim = NT = roundup(S*G, 32).
template <int G, int NT>
__global__ void __launch_bounds__(NT, min_blocks(NT)) k_align(const AlignArgs a) {
  extern __shared__ float4 smem_tab[];
  const int p = blockIdx.x;
  __shared__ int sched[kMaxStages + 1];
  load_schedule(a, p, sched);
  const int Lb = sched[sched[0]];
  const int s = threadIdx.x / G, qg = threadIdx.x % G;
  const bool active = s < a.S;
  const int se = active ? s : s % a.S;  // lanes past the last start shadow a real one and write nothing
  build_table(smem_tab, a.lay, template_row(a, p), a.sub + (size_t)p * a.lay.Nb, a.P, Lb, threadIdx.x,
              blockDim.x);
  __syncthreads();

  float4 q = qnormalize(a.starts[(size_t)p * a.S + se]);
  Eval cur;
  cur.S = 0.f;
  cur.gx = cur.gy = cur.gz = 0.f;
  for (int st = 0; st < sched[0]; ++st) {
    const int L = sched[1 + st];
    const float hmax = 3.14159265358979f / (float)L;
    float h = 0.5f * hmax;
    cur = eval_one<G>(smem_tab, Lb, L, q, qg, a.lbin);
    for (int t = 0; t < a.steps; ++t) {
      const float gn = sqrtf(cur.gx * cur.gx + cur.gy * cur.gy + cur.gz * cur.gz);
      const bool stop = !(gn > 1e-12f * fabsf(cur.S));
      const float inv = stop ? 0.f : 1.f / gn;
      float sh, ch;
      sincosf(stop ? 0.f : 0.5f * h, &sh, &ch);
      const float4 dq = make_float4(ch, sh * cur.gx * inv, sh * cur.gy * inv, sh * cur.gz * inv);
      const float4 qt = qnormalize(qmul(q, dq));
      const Eval tr = eval_one<G>(smem_tab, Lb, L, qt, qg, a.lbin);
      if (!stop) {
        if (tr.S > cur.S) {
          q = qt;
          cur = tr;
          h = fminf(1.5f * h, hmax);
        } else {
          h *= 0.5f;
        }
      }
    }
  }
  __syncthreads();  // the table is no longer read: reuse shared memory for the selection
  float* sS = reinterpret_cast<float*>(smem_tab);
  float4* sQ = reinterpret_cast<float4*>(sS + ((a.S + 3) & ~3));
  if (active && qg == 0) {
    sS[s] = cur.S;
    sQ[s] = q;
    if (a.start_quat_out) a.start_quat_out[(size_t)p * a.S + s] = q;
    if (a.start_score_out) a.start_score_out[(size_t)p * a.S + s] = cur.S;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int best = 0;
    for (int j = 1; j < a.S; ++j)
      if (sS[j] > sS[best]) best = j;
    a.quat_out[p] = sQ[best];
    a.score_out[p] = sS[best];
  }
}

// Score and gradient at given rotations; one CTA per subtomogram.
template <int G>
__global__ void __launch_bounds__(512, 1) k_score(const AlignArgs a, int L) {
  extern __shared__ float4 smem_tab[];
  const int p = blockIdx.x;
  const int s = threadIdx.x / G, qg = threadIdx.x % G;
  const bool active = s < a.S;
  const int se = active ? s : s % a.S;
  build_table(smem_tab, a.lay, template_row(a, p), a.sub + (size_t)p * a.lay.Nb, a.P, a.Lb, threadIdx.x,
              blockDim.x);
  __syncthreads();
  const float4 q = qnormalize(a.starts[(size_t)p * a.S + se]);
  const Eval r = eval_one<G>(smem_tab, a.Lb, L, q, qg, a.lbin);
  if (active && qg == 0) {
    a.score_out[(size_t)p * a.S + s] = r.S;
    if (a.grad_out) {
      float* g = a.grad_out + ((size_t)p * a.S + s) * 3;
      g[0] = r.gx;
      g[1] = r.gy;
      g[2] = r.gz;
    }
  }
}

// Score, gradient and Hessian at given rotations; one CTA per subtomogram.
template <int G>
__global__ void __launch_bounds__(512, 1) k_score_hess(const AlignArgs a, int L) {
  extern __shared__ float4 smem_tab[];
  const int p = blockIdx.x;
  const int s = threadIdx.x / G, qg = threadIdx.x % G;
  const bool active = s < a.S;
  const int se = active ? s : s % a.S;
  build_table(smem_tab, a.lay, template_row(a, p), a.sub + (size_t)p * a.lay.Nb, a.P, a.Lb, threadIdx.x,
              blockDim.x);
  __syncthreads();
  const EvalH r = eval_hess<G>(smem_tab, a.Lb, L, qnormalize(a.starts[(size_t)p * a.S + se]), qg, a.lbin);
  if (active && qg == 0) {
    const size_t o = (size_t)p * a.S + s;
    a.score_out[o] = r.S;
    if (a.grad_out) {
      a.grad_out[o * 3 + 0] = r.gx;
      a.grad_out[o * 3 + 1] = r.gy;
      a.grad_out[o * 3 + 2] = r.gz;
    }
    if (a.hess_out) {
      float* h = a.hess_out + o * 6;
      h[0] = r.hxx; h[1] = r.hxy; h[2] = r.hxz; h[3] = r.hyy; h[4] = r.hyz; h[5] = r.hzz;
    }
  }
}

// Newton direction d = -H^{-1} g when -H is positive definite (Cholesky pivots > 0), else the gradient step
// h0 g/|g|; clipped to length hmax.  Returns the length of d.
__device__ __forceinline__ float newton_dir(const EvalH& e, float gn, float h0, float hmax, float d[3]) {
  bool pd = false;
  const float a11 = -e.hxx;
  if (a11 > 0.f) {
    const float l11 = sqrtf(a11), l21 = -e.hxy / l11, l31 = -e.hxz / l11;
    const float a22 = -e.hyy - l21 * l21;
    if (a22 > 0.f) {
      const float l22 = sqrtf(a22), l32 = (-e.hyz - l31 * l21) / l22;
      const float a33 = -e.hzz - l31 * l31 - l32 * l32;
      if (a33 > 0.f) {
        pd = true;
        const float l33 = sqrtf(a33);
        // (-H) d = g:  L y = g, L^T d = y
        const float y1 = e.gx / l11, y2 = (e.gy - l21 * y1) / l22, y3 = (e.gz - l31 * y1 - l32 * y2) / l33;
        d[2] = y3 / l33;
        d[1] = (y2 - l32 * d[2]) / l22;
        d[0] = (y1 - l21 * d[1] - l31 * d[2]) / l11;
      }
    }
  }
  if (!pd) {
    const float sc = gn > 0.f ? h0 / gn : 0.f;
    d[0] = sc * e.gx;
    d[1] = sc * e.gy;
    d[2] = sc * e.gz;
  }
  float dn = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  if (dn > hmax) {
    const float sc = hmax / dn;
    d[0] *= sc;
    d[1] *= sc;
    d[2] *= sc;
    dn = hmax;
  }
  return dn;
}

// Damped Newton iteration with frequency marching (Sec. III); one CTA per subtomogram, NT = roundup(S*G, 32);
// the orbits dealt by rows (D = 1, eval_hess) or in flat order (D = 2, eval_hess_flat).
template <int G, int NT, int D>
__global__ void __launch_bounds__(NT, min_blocks(NT)) k_newton(const AlignArgs a) {
  extern __shared__ float4 smem_tab[];
  const int p = blockIdx.x;
  __shared__ int sched[kMaxStages + 1];
  load_schedule(a, p, sched);
  const int Lb = sched[sched[0]];
  const int s = threadIdx.x / G, qg = threadIdx.x % G;
  const bool active = s < a.S;
  const int se = active ? s : s % a.S;
  build_table(smem_tab, a.lay, template_row(a, p), a.sub + (size_t)p * a.lay.Nb, a.P, Lb, threadIdx.x,
              blockDim.x);
  __syncthreads();
  float4 q = qnormalize(a.starts[(size_t)p * a.S + se]);
  EvalH cur;
  cur.S = 0.f;
  for (int st = 0; st < sched[0]; ++st) {
    const int L = sched[1 + st];
    const float hmax = 3.14159265358979f / (float)L, h0 = 0.5f * hmax;
    float lam = 1.f;
    cur = D == 2 ? eval_hess_flat<G>(smem_tab, Lb, L, q, qg, a.lbin) : eval_hess<G>(smem_tab, Lb, L, q, qg, a.lbin);
    for (int t = 0; t < a.steps; ++t) {
      const float gn = sqrtf(cur.gx * cur.gx + cur.gy * cur.gy + cur.gz * cur.gz);
      const bool stop = !(gn > 1e-12f * fabsf(cur.S));
      float d[3];
      const float dl = newton_dir(cur, gn, h0, hmax, d);  // |d| before damping
      const float dn = lam * dl;                          // rotation angle of the trial step
      const float inv = (stop || !(dl > 0.f)) ? 0.f : 1.f / dl;
      float sh, ch;
      sincosf(stop ? 0.f : 0.5f * dn, &sh, &ch);
      const float4 dq = make_float4(ch, sh * d[0] * inv, sh * d[1] * inv, sh * d[2] * inv);
      const float4 qt = qnormalize(qmul(q, dq));
      const EvalH tr =
          D == 2 ? eval_hess_flat<G>(smem_tab, Lb, L, qt, qg, a.lbin) : eval_hess<G>(smem_tab, Lb, L, qt, qg, a.lbin);
      if (!stop) {
        if (tr.S > cur.S) {
          q = qt;
          cur = tr;
          lam = fminf(1.f, 2.f * lam);
        } else {
          lam *= 0.5f;
        }
      }
    }
  }
  __syncthreads();
  float* sS = reinterpret_cast<float*>(smem_tab);
  float4* sQ = reinterpret_cast<float4*>(sS + ((a.S + 3) & ~3));
  if (active && qg == 0) {
    sS[s] = cur.S;
    sQ[s] = q;
    if (a.start_quat_out) a.start_quat_out[(size_t)p * a.S + s] = q;
    if (a.start_score_out) a.start_score_out[(size_t)p * a.S + s] = cur.S;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int best = 0;
    for (int j = 1; j < a.S; ++j)
      if (sS[j] > sS[best]) best = j;
    a.quat_out[p] = sQ[best];
    a.score_out[p] = sS[best];
  }
}

// Constrained ascent (missing wedge, Sec. II-B): the ascent's step rule on C(R) = S(R) / sqrt(Dn(R)), the
// common-region norm Dn evaluated like Eq. 2 from a second orbit table built from the wedge's
// pseudo-coefficients (one radial index per degree; the same for every subtomogram of the template) at
// each stage's band, like the score.  (Evaluating it at the wedge's full band in every stage measured
// worse: 1.92 against 1.81 degrees median on the 32^3 batch, and slower.)
__device__ __forceinline__ Eval constrained(const Eval& s, const Eval& d) {
  const float dn = fmaxf(d.S, 1e-30f);
  const float r = rsqrtf(dn);
  const float k = 0.5f * s.S * r / dn;
  Eval c;
  c.S = s.S * r;
  c.gx = s.gx * r - k * d.gx;
  c.gy = s.gy * r - k * d.gy;
  c.gz = s.gz * r - k * d.gz;
  return c;
}

// C(R) and its gradient from one pass over the orbits that scores R against the subtomogram's table and
// the wedge norm's table together.
template <int G>
__device__ __forceinline__ Eval eval_constrained(const float4* __restrict__ tab, const float4* __restrict__ tabw, int Lb,
                                                 int L, float4 q, int qg, const float* __restrict__ lbin) {
  const float4 qq[1] = {q};
  Eval e[2];
  eval_rotations<G, 1, 2>(tab, tabw, Lb, L, qq, qg, lbin, e);
  return constrained(e[0], e[1]);
}

template <int G, int NT>
__global__ void __launch_bounds__(NT, min_blocks(NT)) k_align_wedge(const AlignArgs a, const Layout wlay,
                                                                    const float2* __restrict__ wt,
                                                                    const float2* __restrict__ ww) {
  extern __shared__ float4 smem_tab[];
  const int p = blockIdx.x;
  __shared__ int sched[kMaxStages + 1];
  load_schedule(a, p, sched);
  const int Lb = sched[sched[0]];
  float4* tabw = smem_tab + tab_base(Lb + 1, Lb);
  const int s = threadIdx.x / G, qg = threadIdx.x % G;
  const bool active = s < a.S;
  const int se = active ? s : s % a.S;
  build_table(smem_tab, a.lay, template_row(a, p), a.sub + (size_t)p * a.lay.Nb, a.P, Lb, threadIdx.x,
              blockDim.x);
  build_table(tabw, wlay, wt, ww, a.P, Lb, threadIdx.x, blockDim.x);
  __syncthreads();
  float4 q = qnormalize(a.starts[(size_t)p * a.S + se]);
  Eval cur;
  cur.S = 0.f;
  cur.gx = cur.gy = cur.gz = 0.f;
  for (int st = 0; st < sched[0]; ++st) {
    const int L = sched[1 + st];
    const float hmax = 3.14159265358979f / (float)L;
    float h = 0.5f * hmax;
    cur = eval_constrained<G>(smem_tab, tabw, Lb, L, q, qg, a.lbin);
    for (int t = 0; t < a.steps; ++t) {
      const float gn = sqrtf(cur.gx * cur.gx + cur.gy * cur.gy + cur.gz * cur.gz);
      const bool stop = !(gn > 1e-12f * fabsf(cur.S));
      const float inv = stop ? 0.f : 1.f / gn;
      float sh, ch;
      sincosf(stop ? 0.f : 0.5f * h, &sh, &ch);
      const float4 dq = make_float4(ch, sh * cur.gx * inv, sh * cur.gy * inv, sh * cur.gz * inv);
      const float4 qt = qnormalize(qmul(q, dq));
      const Eval tr = eval_constrained<G>(smem_tab, tabw, Lb, L, qt, qg, a.lbin);
      if (!stop) {
        if (tr.S > cur.S) {
          q = qt;
          cur = tr;
          h = fminf(1.5f * h, hmax);
        } else {
          h *= 0.5f;
        }
      }
    }
  }
  __syncthreads();
  float* sS = reinterpret_cast<float*>(smem_tab);
  float4* sQ = reinterpret_cast<float4*>(sS + ((a.S + 3) & ~3));
  if (active && qg == 0) {
    sS[s] = cur.S;
    sQ[s] = q;
    if (a.start_quat_out) a.start_quat_out[(size_t)p * a.S + s] = q;
    if (a.start_score_out) a.start_score_out[(size_t)p * a.S + s] = cur.S;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int best = 0;
    for (int j = 1; j < a.S; ++j)
      if (sS[j] > sS[best]) best = j;
    a.quat_out[p] = sQ[best];
    a.score_out[p] = sS[best];
  }
}

// Marching ascent with C starts per thread: CTA of NT = roundup(S/C * G, 32) threads per subtomogram.
template <int G, int C, int NT>
__global__ void __launch_bounds__(NT, min_blocks_c(NT, C)) k_align_c(const AlignArgs a) {
  extern __shared__ float4 smem_tab[];
  const int p = blockIdx.x;
  __shared__ int sched[kMaxStages + 1];
  load_schedule(a, p, sched);
  const int Lb = sched[sched[0]];
  const int chunk = threadIdx.x / G, qg = threadIdx.x % G;
  const int nchunks = a.S / C;
  const bool active = chunk < nchunks;
  const int ce = active ? chunk : chunk % nchunks;
  build_table(smem_tab, a.lay, template_row(a, p), a.sub + (size_t)p * a.lay.Nb, a.P, Lb, threadIdx.x,
              blockDim.x);
  __syncthreads();
  float4 q[C];
  Eval cur[C];
  float h[C];
#pragma unroll
  for (int j = 0; j < C; ++j) {
    q[j] = qnormalize(a.starts[(size_t)p * a.S + ce * C + j]);
    cur[j].S = cur[j].gx = cur[j].gy = cur[j].gz = 0.f;
  }
  for (int st = 0; st < sched[0]; ++st) {
    const int L = sched[1 + st];
    const float hmax = 3.14159265358979f / (float)L;
#pragma unroll
    for (int j = 0; j < C; ++j) h[j] = 0.5f * hmax;
    eval_rotations<G, C>(smem_tab, nullptr, Lb, L, q, qg, a.lbin, cur);
    for (int t = 0; t < a.steps; ++t) {
      float4 qt[C];
      bool stop[C];
#pragma unroll
      for (int j = 0; j < C; ++j) {
        const float gn = sqrtf(cur[j].gx * cur[j].gx + cur[j].gy * cur[j].gy + cur[j].gz * cur[j].gz);
        stop[j] = !(gn > 1e-12f * fabsf(cur[j].S));
        const float inv = stop[j] ? 0.f : 1.f / gn;
        float sh, ch;
        sincosf(stop[j] ? 0.f : 0.5f * h[j], &sh, &ch);
        const float4 dq = make_float4(ch, sh * cur[j].gx * inv, sh * cur[j].gy * inv, sh * cur[j].gz * inv);
        qt[j] = qnormalize(qmul(q[j], dq));
      }
      Eval tr[C];
      eval_rotations<G, C>(smem_tab, nullptr, Lb, L, qt, qg, a.lbin, tr);
#pragma unroll
      for (int j = 0; j < C; ++j) {
        if (!stop[j]) {
          if (tr[j].S > cur[j].S) {
            q[j] = qt[j];
            cur[j] = tr[j];
            h[j] = fminf(1.5f * h[j], hmax);
          } else {
            h[j] *= 0.5f;
          }
        }
      }
    }
  }
  __syncthreads();
  float* sS = reinterpret_cast<float*>(smem_tab);
  float4* sQ = reinterpret_cast<float4*>(sS + ((a.S + 3) & ~3));
  if (active && qg == 0) {
#pragma unroll
    for (int j = 0; j < C; ++j) {
      const int s = chunk * C + j;
      sS[s] = cur[j].S;
      sQ[s] = q[j];
      if (a.start_quat_out) a.start_quat_out[(size_t)p * a.S + s] = q[j];
      if (a.start_score_out) a.start_score_out[(size_t)p * a.S + s] = cur[j].S;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int best = 0;
    for (int j = 1; j < a.S; ++j)
      if (sS[j] > sS[best]) best = j;
    a.quat_out[p] = sQ[best];
    a.score_out[p] = sS[best];
  }
}

// Marching ascent with the orbits dealt in flat order (eval_flat), C starts per thread; CTA of
// NT = roundup(S/C * G, 32) threads per subtomogram.
template <int G, int C, int NT>
__global__ void __launch_bounds__(NT, min_blocks_c(NT, C)) k_align_flat(const AlignArgs a) {
  extern __shared__ float4 smem_tab[];
  const int p = blockIdx.x;
  __shared__ int sched[kMaxStages + 1];
  load_schedule(a, p, sched);
  const int Lb = sched[sched[0]];
  const int chunk = threadIdx.x / G, qg = threadIdx.x % G;
  const int nchunks = a.S / C;
  const bool active = chunk < nchunks;
  const int ce = active ? chunk : chunk % nchunks;
  build_table(smem_tab, a.lay, template_row(a, p), a.sub + (size_t)p * a.lay.Nb, a.P, Lb, threadIdx.x,
              blockDim.x);
  __syncthreads();
  float4 q[C];
  Eval cur[C];
  float h[C];
#pragma unroll
  for (int j = 0; j < C; ++j) {
    q[j] = qnormalize(a.starts[(size_t)p * a.S + ce * C + j]);
    cur[j].S = cur[j].gx = cur[j].gy = cur[j].gz = 0.f;
  }
  for (int st = 0; st < sched[0]; ++st) {
    const int L = sched[1 + st];
    const float hmax = 3.14159265358979f / (float)L;
#pragma unroll
    for (int j = 0; j < C; ++j) h[j] = 0.5f * hmax;
    eval_flat<G, C>(smem_tab, Lb, L, q, qg, a.lbin, cur);
    for (int t = 0; t < a.steps; ++t) {
      float4 qt[C];
      bool stop[C];
#pragma unroll
      for (int j = 0; j < C; ++j) {
        const float gn = sqrtf(cur[j].gx * cur[j].gx + cur[j].gy * cur[j].gy + cur[j].gz * cur[j].gz);
        stop[j] = !(gn > 1e-12f * fabsf(cur[j].S));
        const float inv = stop[j] ? 0.f : 1.f / gn;
        float sh, ch;
        sincosf(stop[j] ? 0.f : 0.5f * h[j], &sh, &ch);
        const float4 dq = make_float4(ch, sh * cur[j].gx * inv, sh * cur[j].gy * inv, sh * cur[j].gz * inv);
        qt[j] = qnormalize(qmul(q[j], dq));
      }
      Eval tr[C];
      eval_flat<G, C>(smem_tab, Lb, L, qt, qg, a.lbin, tr);
#pragma unroll
      for (int j = 0; j < C; ++j) {
        if (!stop[j]) {
          if (tr[j].S > cur[j].S) {
            q[j] = qt[j];
            cur[j] = tr[j];
            h[j] = fminf(1.5f * h[j], hmax);
          } else {
            h[j] *= 0.5f;
          }
        }
      }
    }
  }
  __syncthreads();
  float* sS = reinterpret_cast<float*>(smem_tab);
  float4* sQ = reinterpret_cast<float4*>(sS + ((a.S + 3) & ~3));
  if (active && qg == 0) {
#pragma unroll
    for (int j = 0; j < C; ++j) {
      const int s = chunk * C + j;
      sS[s] = cur[j].S;
      sQ[s] = q[j];
      if (a.start_quat_out) a.start_quat_out[(size_t)p * a.S + s] = q[j];
      if (a.start_score_out) a.start_score_out[(size_t)p * a.S + s] = cur[j].S;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int best = 0;
    for (int j = 1; j < a.S; ++j)
      if (sS[j] > sS[best]) best = j;
    a.quat_out[p] = sQ[best];
    a.score_out[p] = sS[best];
  }
}

// ---------------------------------------------------------------------------- energy per degree
// E_l = sum_{m,m'} |xi^l_{mm'}|^2 (Fig. 1's energy ratio is built from these): one CTA per
// (subtomogram, degree), threads over (m, m') pairs, FP64 block sum.
__global__ void __launch_bounds__(256) k_energy(Layout lay, const float2* __restrict__ tmpl,
                                                const int* __restrict__ tmpl_index, int n_templates,
                                                const float2* __restrict__ sub, int L, float* __restrict__ energy) {
  const int p = blockIdx.x, l = blockIdx.y;
  const float2* t = tmpl;
  if (tmpl_index) {
    int ti = tmpl_index[p];
    ti = ti < 0 ? 0 : (ti >= n_templates ? n_templates - 1 : ti);
    t += (size_t)ti * lay.Nb;
  }
  const float2* f = sub + (size_t)p * lay.Nb;
  const int w = 2 * l + 1, K = lay.K[l], off = lay.off[l];
  double acc = 0.0;
  for (int i = threadIdx.x; i < w * w; i += blockDim.x) {
    const int m = i / w, n = i % w;
    double xr = 0.0, xi = 0.0;
    for (int k = 0; k < K; ++k) {
      const float2 a = __ldg(t + off + k * w + m), b = __ldg(f + off + k * w + n);
      xr += (double)a.x * b.x + (double)a.y * b.y;
      xi += (double)a.x * b.y - (double)a.y * b.x;
    }
    acc += xr * xr + xi * xi;
  }
  __shared__ double red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) energy[(size_t)p * (L + 1) + l] = (float)red[0];
}

// ---------------------------------------------------------------------------- band choice (energy ratio)
// Marching bands per subtomogram from the energy ratio of Fig. 1: E_l = sum_{m,m'} |xi^l_{mm'}|^2 for
// l <= Lc (xi^l_{mm'} = sum_k conj(t_klm) f_klm' summed in FP32, |xi|^2 and the sums over (m, m') in FP64,
// per-warp partial sums added in warp order, so the result does not depend on timing), then
// Ratio(L) = sum_{l>L} E_l / sum_{l<=Lc} E_l and band j = the smallest L >= L_min with Ratio(L) <= tau_j;
// a band equal to the previous one is written once.  One CTA per subtomogram.
struct BandRule {
  int n;                    // thresholds, 1..kMaxStages
  int L_min;                // lowest band, >= 1
  double tau[kMaxStages];   // decreasing
};

constexpr int kBandThreads = 256;

__global__ void __launch_bounds__(kBandThreads) k_choose_bands(Layout lay, const float2* __restrict__ tmpl,
                                                               const int* __restrict__ tmpl_index, int n_templates,
                                                               const float2* __restrict__ sub, int Lc, BandRule rule,
                                                               int* __restrict__ stage_table,
                                                               float* __restrict__ energy_out) {
  __shared__ double part[kBandThreads / 32][kMaxL + 1];
  const int p = blockIdx.x;
  const float2* t = tmpl;
  if (tmpl_index) {
    int ti = tmpl_index[p];
    ti = ti < 0 ? 0 : (ti >= n_templates ? n_templates - 1 : ti);
    t += (size_t)ti * lay.Nb;
  }
  const float2* f = sub + (size_t)p * lay.Nb;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  for (int l = 0; l <= Lc; ++l) {
    const int w = 2 * l + 1, K = lay.K[l], off = lay.off[l];
    double acc = 0.0;
    for (int i = threadIdx.x; i < w * w; i += kBandThreads) {
      const int m = i / w, n = i % w;
      float xr = 0.f, xi = 0.f;
      for (int k = 0; k < K; ++k) {
        const float2 a = __ldg(t + off + k * w + m), b = __ldg(f + off + k * w + n);
        xr = fmaf(a.x, b.x, fmaf(a.y, b.y, xr));
        xi = fmaf(a.x, b.y, fmaf(-a.y, b.x, xi));
      }
      acc += (double)xr * xr + (double)xi * xi;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) part[warp][l] = acc;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double E[kMaxL + 1];
    double tot = 0.0;
    for (int l = 0; l <= Lc; ++l) {
      double e = 0.0;
      for (int v = 0; v < kBandThreads / 32; ++v) e += part[v][l];
      E[l] = e;
      tot += e;
      if (energy_out) energy_out[(size_t)p * (Lc + 1) + l] = (float)e;
    }
    // Ratio(L) = sum_{l>L} E_l / total, the tail summed from the highest degree down
    double ratio[kMaxL + 1];
    double tail = 0.0;
    ratio[Lc] = 0.0;
    for (int L = Lc - 1; L >= 0; --L) {
      tail += E[L + 1];
      ratio[L] = tot > 0.0 ? tail / tot : 0.0;
    }
    int* row = stage_table + (size_t)p * (kMaxStages + 1);
    int n = 0, last = 0;
    for (int j = 0; j < rule.n; ++j) {
      int Lj = Lc;  // Ratio(Lc) = 0 always qualifies
      for (int L = rule.L_min; L <= Lc; ++L)
        if (ratio[L] <= rule.tau[j]) {
          Lj = L;
          break;
        }
      if (Lj > last) {
        row[1 + n++] = Lj;
        last = Lj;
      }
    }
    row[0] = n;
  }
}

// ---------------------------------------------------------------------------- FP64 re-scoring
// The same evaluation with the d-recursion, its coefficients, the seeds and the phases in FP64, each orbit's
// chain sum in compensated FP32 pairs and the sums over orbits in FP64 (the shared-memory table stays FP32:
// P_l xi^l rounded once per entry).  Used to re-score the best starts at the last band and select among them.
struct Cx64 {
  double x, y;
};
__device__ __forceinline__ Cx64 cm64(Cx64 a, Cx64 b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__device__ __forceinline__ Cx64 cj64(Cx64 a) { return {a.x, -a.y}; }

__device__ __forceinline__ Cx64 cpow64(Cx64 a, int k) {  // a^k, k >= 0, by binary exponentiation
  Cx64 r{1.0, 0.0};
  while (k > 0) {
    if (k & 1) r = cm64(r, a);
    a = cm64(a, a);
    k >>= 1;
  }
  return r;
}

// Half-angle phases of a rotation (FP64): es = e^{i(alpha+gamma)/2}, ed = e^{i(alpha-gamma)/2}.
struct Rot64 {
  Cx64 es, ed;
  double xb, lcc, lss;
};
__device__ __forceinline__ Rot64 rot64(float4 qf) {
  double w = qf.x, x = qf.y, y = qf.z, z = qf.w;
  const double nq = 1.0 / sqrt(w * w + x * x + y * y + z * z);
  w *= nq; x *= nq; y *= nq; z *= nq;
  const double cb = sqrt(w * w + z * z), sb = sqrt(x * x + y * y);
  Rot64 r;
  r.es = cb > 0.0 ? Cx64{w / cb, z / cb} : Cx64{1.0, 0.0};
  r.ed = sb > 0.0 ? Cx64{y / sb, -x / sb} : Cx64{1.0, 0.0};
  r.xb = (cb - sb) * (cb + sb);
  r.lcc = log2(fmax(cb, 1e-300));
  r.lss = log2(fmax(sb, 1e-300));
  return r;
}

// v (FP64) as hi + lo with hi, lo FP32, formed with integer operations (no FP64 instruction): hi keeps the
// sign, exponent and leading 24 significand bits of v (truncation); lo is the remaining 29 significand bits
// of v as an integer, converted to FP32 (rounded to 24 bits) and scaled by their place value, so that
// |v - hi - lo| <= 2^-48 |v|.  hi = lo = 0 for |v| < 2^-74 (lo's scale would leave the FP32 normal range;
// such terms are below 2^-74 of a table entry), and for values at or above 2^128 (not reached).
__device__ __forceinline__ void split64(double v, float& hi, float& lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const unsigned int h = (unsigned int)(b >> 32), sgn = h & 0x80000000u;
  const int E = (int)((h >> 20) & 0x7FFu);  // FP64 biased exponent: |v| in [2^(E-1023), 2^(E-1022))
  const bool ok = E >= 949 && E < 1151;     // 2^-74 <= |v| < 2^128
  const unsigned int fb = sgn | ((unsigned int)(E - 896) << 23) | ((h & 0xFFFFFu) << 3) | ((unsigned int)b >> 29);
  const float r = (float)((unsigned int)b & 0x1FFFFFFFu);       // the low 29 significand bits, < 2^29
  const float scale = __uint_as_float(sgn | ((unsigned int)(E - 948) << 23));  // +-2^(E - 1075), normal
  hi = ok ? __uint_as_float(fb) : 0.f;
  lo = ok ? r * scale : 0.f;
}
// FP32 to FP64 by integer operations (FP32 subnormals, below 2^-126, give 0).
__device__ __forceinline__ double f2d(float f) {
  const unsigned int u = __float_as_uint(f);
  const unsigned int e = (u >> 23) & 0xFFu;
  const unsigned long long b = ((unsigned long long)(u & 0x80000000u) << 32) |
                               ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)(u & 0x7FFFFFu) << 29);
  return e ? __longlong_as_double((long long)b) : 0.0;
}
// s + c += (hi + lo) x, compensated: hi x is split exactly into p + pe (FMA), p is added to s with an
// error-free two-sum, and the two-sum's error, pe and lo x go to the correction c.
__device__ __forceinline__ void acc_ff(float& s, float& c, float hi, float lo, float x) {
  const float p = hi * x;
  const float pe = fmaf(hi, x, -p);
  const float t = s + p;
  const float z = t - s;
  const float err = (s - (t - z)) + (p - z);
  s = t;
  c = fmaf(lo, x, c + (err + pe));
}

// FP64 score of one rotation at band L, NL lanes per rotation (NL > 32: several warps; the caller adds the
// per-warp partial sums).  Orbits are dealt by their flat index: lane q takes (m, n) with
// m^2 + m + n = q mod NL, so rows shorter than NL still spread over all lanes.  The lane's first orbit in
// row m is n = j - m, j = (q - m^2) mod NL, with phases A^j conj(ed)^{2m} and Bc^j ed^{2m}; A^j and Bc^j
// (j < NL) come from per-rotation power tables in shared memory.  Returns the warp's partial sum.
template <int NL>
__device__ double score_rotation64(const float4* __restrict__ tab, int Lb, int L, const Rot64& r, int q,
                                   const double2* __restrict__ Apow, const double2* __restrict__ Bpow,
                                   const double2* __restrict__ coef, const double* __restrict__ lbin, int Lmax) {
  const Cx64 Es = cj64(r.es), Ed = cj64(r.ed), Ed2 = cm64(Ed, Ed);
  const Cx64 R1 = cpow64(cm64(Es, r.ed), NL), R2 = cpow64(cm64(Es, Ed), NL);
  Cx64 Cm{1.0, 0.0};
  double S = 0.0;
  for (int m = 0; m <= L; ++m) {
    const int w2 = 2 * m + 1;
    const float4* rowp = tab + tab_base(m, Lb);
    const double2* crow = coef + tab_base(m, Lmax);
    int j = (q - m * m) % NL;
    j += j < 0 ? NL : 0;
    const double2 ap = Apow[j], bp = Bpow[j];
    Cx64 P1 = cm64(Cx64{ap.x, ap.y}, Cm), P2 = cm64(Cx64{bp.x, bp.y}, cj64(Cm));
    for (int n = j - m; n <= m; n += NL) {
      double d = exp2(lbin[m * kBinStride + m + n] + (double)(m + n) * r.lcc + (double)(m - n) * r.lss);
      d = ((m - n) & 1) ? -d : d;
      const float4* ep = rowp + (n + m);
      const double2* kp = crow + (n + m);
      // the chain's sums a = sum_l e^l x^l: the recursion in FP64, each term accumulated in compensated FP32
      // (s + c; the split of e^l loses 2^-48 of it, the sum about 2^-43 of the terms' magnitudes, far below the
      // table's FP32 rounding), without FP64 conversions and multiply-adds of the FP32 table entries
      float4 xv = *ep;
      float s1r, s1i, s2r, s2i, c1r = 0.f, c1i = 0.f, c2r = 0.f, c2i = 0.f;
      {
        float hi, lo;
        split64(d, hi, lo);
        s1r = s1i = s2r = s2i = 0.f;
        acc_ff(s1r, c1r, hi, lo, xv.x);
        acc_ff(s1i, c1i, hi, lo, xv.y);
        acc_ff(s2r, c2r, hi, lo, xv.z);
        acc_ff(s2i, c2i, hi, lo, xv.w);
      }
      double e1 = d, e2 = 0.0;
      for (int l = m + 1; l <= L; ++l) {
        ep += w2;
        kp += w2;
        const double2 k = __ldg(kp);
        const double en = fma(r.xb - k.x, e1, -k.y * e2);
        e2 = e1;
        e1 = en;
        xv = *ep;
        float hi, lo;
        split64(en, hi, lo);
        acc_ff(s1r, c1r, hi, lo, xv.x);
        acc_ff(s1i, c1i, hi, lo, xv.y);
        acc_ff(s2r, c2r, hi, lo, xv.z);
        acc_ff(s2i, c2i, hi, lo, xv.w);
      }
      const double a1r = f2d(s1r) + f2d(c1r), a1i = f2d(s1i) + f2d(c1i);
      const double a2r = f2d(s2r) + f2d(c2r), a2i = f2d(s2i) + f2d(c2i);
      S += (P1.x * a1r - P1.y * a1i) + (P2.x * a2r - P2.y * a2i);
      P1 = cm64(P1, R1);
      P2 = cm64(P2, R2);
    }
    Cm = cm64(Cm, Ed2);
  }
#pragma unroll
  for (int o = 1; o < (NL < 32 ? NL : 32); o <<= 1) S += __shfl_xor_sync(0xffffffffu, S, o);
  return S;
}

// Top-K re-scoring in FP64 at the last band (optional): the K starts with the largest FP32 final score
// (ties: lowest index) are re-evaluated with the d-recursion, seeds and phases in FP64, the chain sums in
// compensated FP32 pairs (score_rotation64; the table's
// xi stays the FP32 product; the rational recursion coefficients come from the plan's FP64 table), and
// the subtomogram's result is the best of them on the FP64 score.  One CTA of K * NL threads per
// subtomogram; shared memory: the orbit table, then the per-start power tables A^j, Bc^j (j < NL).
constexpr int kMaxRefine = 64;

template <int NL>
__global__ void __launch_bounds__(512, 1) k_refine64(const AlignArgs a, int Lmax_band, int K, const double2* coef64,
                                                     const double* lbin64) {
  extern __shared__ float4 smem_tab[];
  __shared__ int top[kMaxRefine];
  __shared__ double part[kMaxRefine];  // [start][warp of the start] partial sums; K * max(1, NL/32) <= 64
  constexpr int W = NL > 32 ? NL / 32 : 1;
  const int p = blockIdx.x;
  // the band of the re-score: the subtomogram's last marching band with a per-subtomogram schedule, else
  // the launch's band
  __shared__ int sched[kMaxStages + 1];
  load_schedule(a, p, sched);
  const int L = a.stage_table ? sched[sched[0]] : Lmax_band;
  const int Lb = L;
  const int ntab = tab_base(Lb + 1, Lb);
  double2* Apow = reinterpret_cast<double2*>(smem_tab + ntab);
  double2* Bpow = Apow + (size_t)K * NL;
  build_table(smem_tab, a.lay, template_row(a, p), a.sub + (size_t)p * a.lay.Nb, a.P, Lb, threadIdx.x,
              blockDim.x);
  if (threadIdx.x == 0) {
    const float* sc = a.start_score_out + (size_t)p * a.S;
    for (int k = 0; k < K; ++k) {
      int best = -1;
      for (int j = 0; j < a.S; ++j) {
        bool taken = false;
        for (int i = 0; i < k; ++i) taken |= (top[i] == j);
        if (!taken && (best < 0 || sc[j] > sc[best])) best = j;
      }
      top[k] = best;
    }
  }
  __syncthreads();
  const int s = threadIdx.x / NL, q = threadIdx.x % NL;
  const bool active = s < K;
  const int se = active ? s : s % K;  // lanes past the last start shadow a real one and write nothing
  const Rot64 r = rot64(a.start_quat_out[(size_t)p * a.S + top[se]]);
  if (active) {
    const Cx64 Es = cj64(r.es);
    const Cx64 Ap = cpow64(cm64(Es, r.ed), q), Bp = cpow64(cm64(Es, cj64(r.ed)), q);
    Apow[(size_t)s * NL + q] = make_double2(Ap.x, Ap.y);
    Bpow[(size_t)s * NL + q] = make_double2(Bp.x, Bp.y);
  }
  __syncthreads();
  const double S = score_rotation64<NL>(smem_tab, Lb, L, r, q, Apow + (size_t)se * NL, Bpow + (size_t)se * NL,
                                        coef64, lbin64, a.lay.Lmax);
  if (active && (q & 31) == 0) part[s * W + q / 32] = S;
  __syncthreads();
  if (threadIdx.x == 0) {
    int best = 0;
    double sbest = 0.0;
    for (int k = 0; k < K; ++k) {
      double sk = 0.0;
      for (int w = 0; w < W; ++w) sk += part[k * W + w];
      if (k == 0 || sk > sbest || (sk == sbest && top[k] < top[best])) {
        best = k;
        sbest = sk;
      }
    }
    a.quat_out[p] = a.start_quat_out[(size_t)p * a.S + top[best]];
    a.score_out[p] = (float)sbest;
    if (a.score64_out) a.score64_out[p] = sbest;
  }
}

size_t table_bytes(int Lb) { return (size_t)tab_base(Lb + 1, Lb) * sizeof(float4); }

template <int G, int NT>
int launch_align_nt(const AlignArgs& a, size_t smem, cudaStream_t stream) {
  static SmemAttr have;
  int st = ensure_smem(k_align<G, NT>, have, smem);
  if (st != BH_OK) return st;
  k_align<G, NT><<<a.B, NT, smem, stream>>>(a);
  BH_CHECK_LAUNCH();
  return BH_OK;
}

template <int G>
int launch_align_g(const AlignArgs& a, bool score_only, int L, cudaStream_t stream) {
  const int threads = round_up(a.S * G, 32);
  const size_t sel = (size_t)((a.S + 3) & ~3) * sizeof(float) + (size_t)a.S * sizeof(float4);
  const size_t smem = std::max(table_bytes(a.Lb), score_only ? (size_t)16 : sel);
  if (smem > 232448) return fail(BH_ERR_UNSUPPORTED, "orbit table for band %d needs %zu B of shared memory", a.Lb, smem);
  if (score_only) {
    static SmemAttr have;
    int st = ensure_smem(k_score<G>, have, smem);
    if (st != BH_OK) return st;
    k_score<G><<<a.B, threads, smem, stream>>>(a, L);
    BH_CHECK_LAUNCH();
    return BH_OK;
  }
  switch (threads) {
    case 32: return launch_align_nt<G, 32>(a, smem, stream);
    case 64: return launch_align_nt<G, 64>(a, smem, stream);
    case 96:
    case 128: return launch_align_nt<G, 128>(a, smem, stream);
    case 160:
    case 192:
    case 224:
    case 256: return launch_align_nt<G, 256>(a, smem, stream);
    default: return launch_align_nt<G, 512>(a, smem, stream);
  }
}

template <int G, int NT>
int launch_align_c2_nt(const AlignArgs& a, size_t smem, cudaStream_t stream) {
  static SmemAttr have;
  int st = ensure_smem(k_align_c<G, 2, NT>, have, smem);
  if (st != BH_OK) return st;
  k_align_c<G, 2, NT><<<a.B, NT, smem, stream>>>(a);
  BH_CHECK_LAUNCH();
  return BH_OK;
}

template <int G>
int launch_align_c2_g(const AlignArgs& a, cudaStream_t stream) {
  const int threads = round_up((a.S / 2) * G, 32);
  const size_t sel = (size_t)((a.S + 3) & ~3) * sizeof(float) + (size_t)a.S * sizeof(float4);
  const size_t smem = std::max(table_bytes(a.Lb), sel);
  if (smem > 232448) return fail(BH_ERR_UNSUPPORTED, "orbit table for band %d needs %zu B of shared memory", a.Lb, smem);
  switch (threads) {
    case 32: return launch_align_c2_nt<G, 32>(a, smem, stream);
    case 64: return launch_align_c2_nt<G, 64>(a, smem, stream);
    case 96:
    case 128: return launch_align_c2_nt<G, 128>(a, smem, stream);
    case 160:
    case 192:
    case 224:
    case 256: return launch_align_c2_nt<G, 256>(a, smem, stream);
    default: return launch_align_c2_nt<G, 512>(a, smem, stream);
  }
}

template <int G, int C, int NT>
int launch_align_flat_nt(const AlignArgs& a, size_t smem, cudaStream_t stream) {
  static SmemAttr have;
  int st = ensure_smem(k_align_flat<G, C, NT>, have, smem);
  if (st != BH_OK) return st;
  k_align_flat<G, C, NT><<<a.B, NT, smem, stream>>>(a);
  BH_CHECK_LAUNCH();
  return BH_OK;
}

template <int G, int C>
int launch_align_flat_gc(const AlignArgs& a, cudaStream_t stream) {
  const int threads = round_up((a.S / C) * G, 32);
  const size_t sel = (size_t)((a.S + 3) & ~3) * sizeof(float) + (size_t)a.S * sizeof(float4);
  const size_t smem = std::max(table_bytes(a.Lb), sel);
  if (smem > 232448) return fail(BH_ERR_UNSUPPORTED, "orbit table for band %d needs %zu B of shared memory", a.Lb, smem);
  switch (threads) {
    case 32: return launch_align_flat_nt<G, C, 32>(a, smem, stream);
    case 64: return launch_align_flat_nt<G, C, 64>(a, smem, stream);
    case 96:
    case 128: return launch_align_flat_nt<G, C, 128>(a, smem, stream);
    case 160:
    case 192:
    case 224:
    case 256: return launch_align_flat_nt<G, C, 256>(a, smem, stream);
    default: return launch_align_flat_nt<G, C, 512>(a, smem, stream);
  }
}

// Flat orbit dealing (eval_flat): G lanes per group of C starts (S a multiple of C).
int launch_align_flat(const AlignArgs& a, int G, int C, cudaStream_t stream) {
  if (a.S % C) return fail(BH_ERR_ARG, "%d starts per thread need S divisible by it (S=%d)", C, a.S);
  if (C == 1) {
    switch (G) {
      case 4: return launch_align_flat_gc<4, 1>(a, stream);
      case 8: return launch_align_flat_gc<8, 1>(a, stream);
      case 16: return launch_align_flat_gc<16, 1>(a, stream);
      default: break;
    }
  } else if (C == 2) {
    switch (G) {
      case 4: return launch_align_flat_gc<4, 2>(a, stream);
      case 8: return launch_align_flat_gc<8, 2>(a, stream);
      case 16: return launch_align_flat_gc<16, 2>(a, stream);
      default: break;
    }
  }
  return fail(BH_ERR_ARG, "flat dealing: group %d with %d starts per thread not in {4,8,16} x {1,2}", G, C);
}

// Two starts per thread (S even): G lanes per pair of starts.
int launch_align_c2(const AlignArgs& a, int G, cudaStream_t stream) {
  if (a.S % 2) return fail(BH_ERR_ARG, "two starts per thread need an even S (S=%d)", a.S);
  switch (G) {
    case 2: return launch_align_c2_g<2>(a, stream);
    case 4: return launch_align_c2_g<4>(a, stream);
    case 8: return launch_align_c2_g<8>(a, stream);
    case 16: return launch_align_c2_g<16>(a, stream);
    default: return fail(BH_ERR_ARG, "group %d not in {2,4,8,16} for two starts per thread", G);
  }
}

int launch_align(const AlignArgs& a, int G, bool score_only, int L, cudaStream_t stream) {
  switch (G) {
    case 1: return launch_align_g<1>(a, score_only, L, stream);
    case 2: return launch_align_g<2>(a, score_only, L, stream);
    case 4: return launch_align_g<4>(a, score_only, L, stream);
    case 8: return launch_align_g<8>(a, score_only, L, stream);
    case 16: return launch_align_g<16>(a, score_only, L, stream);
    default: return fail(BH_ERR_ARG, "group %d not in {1,2,4,8,16}", G);
  }
}

template <int G, int NT, int D>
int launch_newton_nt(const AlignArgs& a, size_t smem, cudaStream_t stream) {
  static SmemAttr have;
  int st = ensure_smem(k_newton<G, NT, D>, have, smem);
  if (st != BH_OK) return st;
  k_newton<G, NT, D><<<a.B, NT, smem, stream>>>(a);
  BH_CHECK_LAUNCH();
  return BH_OK;
}

template <int G, int D>
int launch_newton_g(const AlignArgs& a, bool score_only, int L, cudaStream_t stream) {
  const int threads = round_up(a.S * G, 32);
  const size_t sel = (size_t)((a.S + 3) & ~3) * sizeof(float) + (size_t)a.S * sizeof(float4);
  const size_t smem = std::max(table_bytes(a.Lb), score_only ? (size_t)16 : sel);
  if (smem > 232448) return fail(BH_ERR_UNSUPPORTED, "orbit table for band %d needs %zu B of shared memory", a.Lb, smem);
  if (score_only) {
    static SmemAttr have;
    int st = ensure_smem(k_score_hess<G>, have, smem);
    if (st != BH_OK) return st;
    k_score_hess<G><<<a.B, threads, smem, stream>>>(a, L);
    BH_CHECK_LAUNCH();
    return BH_OK;
  }
  switch (threads) {
    case 32: return launch_newton_nt<G, 32, D>(a, smem, stream);
    case 64: return launch_newton_nt<G, 64, D>(a, smem, stream);
    case 96:
    case 128: return launch_newton_nt<G, 128, D>(a, smem, stream);
    case 160:
    case 192:
    case 224:
    case 256: return launch_newton_nt<G, 256, D>(a, smem, stream);
    default: return launch_newton_nt<G, 512, D>(a, smem, stream);
  }
}

// Newton iteration (or, score_only, the score/gradient/Hessian evaluation at band L, always row-dealt) with G
// lanes per start; D = 1 deals the orbits by rows, D = 2 in flat order (G in {8, 16, 32}).
int launch_newton(const AlignArgs& a, int G, int D, bool score_only, int L, cudaStream_t stream) {
  if (D == 2 && !score_only) {
    switch (G) {
      case 8: return launch_newton_g<8, 2>(a, false, L, stream);
      case 16: return launch_newton_g<16, 2>(a, false, L, stream);
      case 32: return launch_newton_g<32, 2>(a, false, L, stream);
      default: return fail(BH_ERR_ARG, "flat dealing of the Newton kernel: group %d not in {8,16,32}", G);
    }
  }
  switch (G) {
    case 1: return launch_newton_g<1, 1>(a, score_only, L, stream);
    case 2: return launch_newton_g<2, 1>(a, score_only, L, stream);
    case 4: return launch_newton_g<4, 1>(a, score_only, L, stream);
    case 8: return launch_newton_g<8, 1>(a, score_only, L, stream);
    case 16: return launch_newton_g<16, 1>(a, score_only, L, stream);
    case 32: return launch_newton_g<32, 1>(a, score_only, L, stream);
    default: return fail(BH_ERR_ARG, "group %d not in {1,2,4,8,16,32}", G);
  }
}

template <int G, int NT>
int launch_wedge_nt(const AlignArgs& a, const bh_wedge* w, size_t smem, cudaStream_t stream) {
  static SmemAttr have;
  int st = ensure_smem(k_align_wedge<G, NT>, have, smem);
  if (st != BH_OK) return st;
  k_align_wedge<G, NT><<<a.B, NT, smem, stream>>>(a, w->layout, w->d_t, w->d_w);
  BH_CHECK_LAUNCH();
  return BH_OK;
}

template <int G>
int launch_wedge_g(const AlignArgs& a, const bh_wedge* w, cudaStream_t stream) {
  const int threads = round_up(a.S * G, 32);
  const size_t sel = (size_t)((a.S + 3) & ~3) * sizeof(float) + (size_t)a.S * sizeof(float4);
  const size_t smem = std::max(2 * table_bytes(a.Lb), sel);
  if (smem > 232448) return fail(BH_ERR_UNSUPPORTED, "two orbit tables of band %d need %zu B of shared memory", a.Lb, smem);
  switch (threads) {
    case 32: return launch_wedge_nt<G, 32>(a, w, smem, stream);
    case 64: return launch_wedge_nt<G, 64>(a, w, smem, stream);
    case 96:
    case 128: return launch_wedge_nt<G, 128>(a, w, smem, stream);
    case 160:
    case 192:
    case 224:
    case 256: return launch_wedge_nt<G, 256>(a, w, smem, stream);
    default: return launch_wedge_nt<G, 512>(a, w, smem, stream);
  }
}

// Constrained ascent with G lanes per start.
int launch_wedge(const AlignArgs& a, const bh_wedge* w, int G, cudaStream_t stream) {
  switch (G) {
    case 1: return launch_wedge_g<1>(a, w, stream);
    case 2: return launch_wedge_g<2>(a, w, stream);
    case 4: return launch_wedge_g<4>(a, w, stream);
    case 8: return launch_wedge_g<8>(a, w, stream);
    case 16: return launch_wedge_g<16>(a, w, stream);
    default: return fail(BH_ERR_ARG, "group %d not in {1,2,4,8,16}", G);
  }
}

template <int NL>
int launch_refine_nl(const AlignArgs& a, int L, int K, const bh_plan* p, cudaStream_t stream) {
  const int threads = round_up(K * NL, 32);
  const size_t smem = table_bytes(a.Lb) + 2 * (size_t)K * NL * sizeof(double2);
  if (smem > 232448) return fail(BH_ERR_UNSUPPORTED, "FP64 re-score for band %d needs %zu B of shared memory", a.Lb, smem);
  static SmemAttr have;
  int st = ensure_smem(k_refine64<NL>, have, smem);
  if (st != BH_OK) return st;
  k_refine64<NL><<<a.B, threads, smem, stream>>>(a, L, K, p->d_coef64, p->d_lbin64);
  BH_CHECK_LAUNCH();
  return BH_OK;
}

// FP64 work needs many warps in flight (GB300's FP64 pipe is narrow and deep): one CTA per subtomogram
// holds the K re-scored starts with up to 128 lanes (four warps) each, 512 threads when K allows.
int launch_refine(const AlignArgs& a, int L, int K, const bh_plan* p, cudaStream_t stream) {
  int NL = 1;
  while (NL < 128 && K * NL * 2 <= kMaxThreads) NL *= 2;
  switch (NL) {
    case 1: return launch_refine_nl<1>(a, L, K, p, stream);
    case 2: return launch_refine_nl<2>(a, L, K, p, stream);
    case 4: return launch_refine_nl<4>(a, L, K, p, stream);
    case 8: return launch_refine_nl<8>(a, L, K, p, stream);
    case 16: return launch_refine_nl<16>(a, L, K, p, stream);
    case 32: return launch_refine_nl<32>(a, L, K, p, stream);
    case 64: return launch_refine_nl<64>(a, L, K, p, stream);
    default: return launch_refine_nl<128>(a, L, K, p, stream);
  }
}

// Default lanes per start (before autotuning): about 512 resident threads per SM, given how many orbit
// tables of band Lb fit in an SM's 227 KB of shared memory (at most 8 CTAs).
int default_group(int S, int Lb, int tables = 1) {
  const int ctas = std::max(1, std::min(8, (int)(232448 / std::max<size_t>(1, tables * table_bytes(Lb)))));
  const int want = std::max(32, 512 / ctas);
  int G = 1;
  while (G < 16 && S * G < want && round_up(S * G * 2, 32) <= kMaxThreads) G *= 2;
  return G;
}

// Default lanes per start of the Newton kernel: about 256 resident threads per SM (its evaluation holds
// more state per lane than the ascent's, measured best at one warp per CTA for band 16), up to a full
// warp per start (few candidate starts on a large orbit table would otherwise leave an SM idle).
int default_group_newton(int S, int Lb) {
  const int ctas = std::max(1, std::min(8, (int)(232448 / std::max<size_t>(1, table_bytes(Lb)))));
  const int want = std::max(32, 256 / ctas);
  int G = 1;
  while (G < 32 && S * G < want && round_up(S * G * 2, 32) <= kMaxThreads) G *= 2;
  return G;
}

}  // namespace

int align_init_constants() {
  static std::mutex mu;
  static bool done[128] = {};
  int dev = 0;
  BH_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  if (dev >= 0 && dev < 128 && done[dev]) return BH_OK;
  float4 ec[kMaxL + 4];
  for (int l = 0; l < kMaxL + 4; ++l) {
    if (l < 2) {
      ec[l] = make_float4(0.f, 0.f, 0.f, (float)(l * (l + 1)));
    } else {
      const double a = (double)(l - 1) * (l - 1);
      ec[l] = make_float4((float)(1.0 / ((double)l * (l - 1))), (float)(1.0 / (a * (2.0 * l - 1.0) * (2.0 * l - 3.0))),
                          (float)a, (float)(l * (l + 1)));
    }
  }
  BH_CUDA_TRY(cudaMemcpyToSymbol(c_ecoef, ec, sizeof(ec)));
  if (dev >= 0 && dev < 128) done[dev] = true;
  return BH_OK;
}

}  // namespace bh

using namespace bh;

static int check_common(const bh_plan* p, const float* tmpl, const float* sub, int B, const float* quats, int S) {
  if (!p) return fail(BH_ERR_ARG, "plan is NULL");
  if (B < 0) return fail(BH_ERR_ARG, "B=%d", B);
  if (S < 1 || S > kMaxThreads) return fail(BH_ERR_ARG, "S=%d outside 1..%d", S, kMaxThreads);
  if (B > 0 && (!tmpl || !sub || !quats)) return fail(BH_ERR_ARG, "NULL input array");
  return check_plan_device(p);
}

extern "C" int bh_score_grad(const bh_plan* p, const float* tmpl, const float* sub, int B, const float* quats, int S,
                             int L, float* score, float* grad, void* stream) {
  clear_error();
  const bh::Range range_("bh_score_grad");
  int st = check_common(p, tmpl, sub, B, quats, S);
  if (st != BH_OK) return st;
  if (L < 0 || L > p->Lmax) return fail(BH_ERR_ARG, "L=%d outside 0..%d", L, p->Lmax);
  if (B == 0) return BH_OK;
  if (!score) return fail(BH_ERR_ARG, "score is NULL");
  AlignArgs a{};
  a.lay = p->layout;
  a.tmpl = reinterpret_cast<const float2*>(tmpl);
  a.sub = reinterpret_cast<const float2*>(sub);
  a.B = B;
  a.starts = reinterpret_cast<const float4*>(quats);
  a.S = S;
  a.Lb = L;
  a.P = p->d_P;
  a.lbin = p->d_lbin;
  a.score_out = score;
  a.grad_out = grad;
  int G = default_group(S, L);
  return launch_align(a, G, true, L, static_cast<cudaStream_t>(stream));
}

extern "C" int bh_score_hess(const bh_plan* p, const float* tmpl, const float* sub, int B, const float* quats, int S,
                             int L, float* score, float* grad, float* hess, void* stream) {
  clear_error();
  const bh::Range range_("bh_score_hess");
  int st = check_common(p, tmpl, sub, B, quats, S);
  if (st != BH_OK) return st;
  if (L < 0 || L > p->Lmax) return fail(BH_ERR_ARG, "L=%d outside 0..%d", L, p->Lmax);
  if (B == 0) return BH_OK;
  if (!score) return fail(BH_ERR_ARG, "score is NULL");
  AlignArgs a{};
  a.lay = p->layout;
  a.tmpl = reinterpret_cast<const float2*>(tmpl);
  a.sub = reinterpret_cast<const float2*>(sub);
  a.B = B;
  a.starts = reinterpret_cast<const float4*>(quats);
  a.S = S;
  a.Lb = L;
  a.P = p->d_P;
  a.lbin = p->d_lbin;
  a.score_out = score;
  a.grad_out = grad;
  a.hess_out = hess;
  return launch_newton(a, default_group(S, L), 1, true, L, static_cast<cudaStream_t>(stream));
}

extern "C" int bh_wedge_norm(const bh_plan* p, const bh_wedge* w, const float* quats, int S, int L, float* dn,
                             float* grad, void* stream) {
  clear_error();
  const bh::Range range_("bh_wedge_norm");
  if (!p || !w) return fail(BH_ERR_ARG, "plan or wedge is NULL");
  if (S < 1 || S > kMaxThreads) return fail(BH_ERR_ARG, "S=%d outside 1..%d", S, kMaxThreads);
  if (L < 0 || L > w->L) return fail(BH_ERR_ARG, "L=%d outside 0..%d (wedge band)", L, w->L);
  if (w->layout.Lmax != p->Lmax) return fail(BH_ERR_ARG, "wedge prepared for another plan");
  if (!quats || !dn) return fail(BH_ERR_ARG, "NULL array");
  if (int st = check_plan_device(p); st != BH_OK) return st;
  AlignArgs a{};
  a.lay = w->layout;
  a.tmpl = w->d_t;
  a.sub = w->d_w;
  a.B = 1;
  a.starts = reinterpret_cast<const float4*>(quats);
  a.S = S;
  a.Lb = L;
  a.P = p->d_P;
  a.lbin = p->d_lbin;
  a.score_out = dn;
  a.grad_out = grad;
  return launch_align(a, default_group(S, L), true, L, static_cast<cudaStream_t>(stream));
}

extern "C" int bh_align_batch(const bh_plan* p, const float* tmpl, const float* sub, int B, const float* starts, int S,
                              const int* stages, int nstages, int steps, float* quat_out, float* score_out,
                              const bh_align_opts* opts, void* stream) {
  clear_error();
  const bh::Range range_("bh_align_batch");
  int st = check_common(p, tmpl, sub, B, starts, S);
  if (st != BH_OK) return st;
  if (!stages || nstages < 1 || nstages > kMaxStages) return fail(BH_ERR_ARG, "nstages=%d outside 1..%d", nstages, kMaxStages);
  for (int i = 0; i < nstages; ++i) {
    if (stages[i] < 1 || stages[i] > p->Lmax) return fail(BH_ERR_ARG, "stage band %d outside 1..%d", stages[i], p->Lmax);
    if (i > 0 && stages[i] <= stages[i - 1]) return fail(BH_ERR_ARG, "stage bands must increase");
  }
  if (steps < 0 || steps > 100000) return fail(BH_ERR_ARG, "steps=%d outside 0..100000", steps);
  if (B == 0) return BH_OK;
  if (!quat_out || !score_out) return fail(BH_ERR_ARG, "quat_out or score_out is NULL");
  AlignArgs a{};
  a.lay = p->layout;
  a.tmpl = reinterpret_cast<const float2*>(tmpl);
  a.sub = reinterpret_cast<const float2*>(sub);
  a.B = B;
  a.starts = reinterpret_cast<const float4*>(starts);
  a.S = S;
  a.nstages = nstages;
  for (int i = 0; i < nstages; ++i) a.stages[i] = stages[i];
  a.steps = steps;
  a.Lb = stages[nstages - 1];
  a.P = p->d_P;
  a.lbin = p->d_lbin;
  a.quat_out = reinterpret_cast<float4*>(quat_out);
  a.score_out = score_out;
  int G = 0, C = 0, D = 0;
  if (opts) {
    if (opts->tmpl_index) {
      if (opts->n_templates < 1) return fail(BH_ERR_ARG, "n_templates=%d with tmpl_index", opts->n_templates);
      a.tmpl_index = opts->tmpl_index;
      a.n_templates = opts->n_templates;
    }
    a.start_quat_out = reinterpret_cast<float4*>(opts->start_quat_out);
    a.start_score_out = opts->start_score_out;
    a.stage_table = opts->stage_table;
    G = opts->group;
    C = opts->starts_per_thread;
    D = opts->dealing;
    if (C < 0 || C > 2) return fail(BH_ERR_ARG, "starts_per_thread=%d not in {0,1,2}", C);
    if (D < 0 || D > 2) return fail(BH_ERR_ARG, "dealing=%d not in {0,1,2}", D);
    if (opts->refine_fp64 < 0 || opts->refine_fp64 > kMaxRefine)
      return fail(BH_ERR_ARG, "refine_fp64=%d outside 0..%d", opts->refine_fp64, kMaxRefine);
    if (opts->refine_fp64 > 0 && (!opts->start_quat_out || !opts->start_score_out))
      return fail(BH_ERR_ARG, "refine_fp64 needs start_quat_out and start_score_out");
  }
  if (G == 0) {
    auto it = p->align_group.find({a.Lb, S});
    if (it != p->align_group.end()) {
      G = it->second.group;
      if (C == 0) C = it->second.starts_per_thread;
      if (D == 0) D = it->second.dealing;
    } else {
      G = default_group(S, a.Lb);
    }
  }
  if (C == 0) C = 1;
  if (D == 0) D = 1;
  if (opts && opts->wedge) {
    const bh_wedge* w = opts->wedge;
    if (opts->newton || opts->starts_per_thread > 1)
      return fail(BH_ERR_ARG, "the constrained ascent runs the ascent's step rule with one start per group");
    if (opts->tmpl_index) return fail(BH_ERR_ARG, "the constrained ascent takes one template");
    if (w->L < a.Lb) return fail(BH_ERR_ARG, "wedge prepared to band %d, stages reach %d", w->L, a.Lb);
    if (w->layout.Lmax != p->Lmax) return fail(BH_ERR_ARG, "wedge prepared for another plan");
    if (opts->group == 0) G = default_group(S, a.Lb, 2);  // two orbit tables per CTA
    if (round_up(S * G, 32) > kMaxThreads)
      return fail(BH_ERR_ARG, "S*group = %d exceeds %d threads", S * G, kMaxThreads);
    st = launch_wedge(a, w, G, static_cast<cudaStream_t>(stream));
  } else if (opts && opts->newton) {
    if (opts->starts_per_thread > 1) return fail(BH_ERR_ARG, "Newton steps run one start per thread group");
    int DN = opts->dealing;
    if (opts->group == 0) {
      auto it = p->newton_group.find({a.Lb, S});
      if (it != p->newton_group.end()) {
        G = it->second.group;
        if (DN == 0) DN = it->second.dealing;
      } else {
        G = default_group_newton(S, a.Lb);
      }
    }
    if (DN == 0) DN = 1;
    if (round_up(S * G, 32) > kMaxThreads)
      return fail(BH_ERR_ARG, "S*group = %d exceeds %d threads", S * G, kMaxThreads);
    st = launch_newton(a, G, DN, false, 0, static_cast<cudaStream_t>(stream));
  } else if (D == 2) {
    if (round_up((S / C) * G, 32) > kMaxThreads)
      return fail(BH_ERR_ARG, "S/%d*group = %d exceeds %d threads", C, (S / C) * G, kMaxThreads);
    st = launch_align_flat(a, G, C, static_cast<cudaStream_t>(stream));
  } else if (C == 2) {
    if (round_up((S / 2) * G, 32) > kMaxThreads)
      return fail(BH_ERR_ARG, "S/2*group = %d exceeds %d threads", (S / 2) * G, kMaxThreads);
    st = launch_align_c2(a, G, static_cast<cudaStream_t>(stream));
  } else {
    if (round_up(S * G, 32) > kMaxThreads)
      return fail(BH_ERR_ARG, "S*group = %d exceeds %d threads", S * G, kMaxThreads);
    st = launch_align(a, G, false, 0, static_cast<cudaStream_t>(stream));
  }
  if (st != BH_OK || !opts || opts->refine_fp64 == 0) return st;
  return launch_refine(a, a.Lb, std::min(opts->refine_fp64, S), p, static_cast<cudaStream_t>(stream));
}

extern "C" int bh_refine_fp64(const bh_plan* p, const float* tmpl, const float* sub, int B, const float* start_quat,
                              const float* start_score, int S, int L, int K, const int* tmpl_index, int n_templates,
                              const int* stage_table, float* quat_out, float* score_out, double* score64_out,
                              void* stream) {
  clear_error();
  const bh::Range range_("bh_refine_fp64");
  int st = check_common(p, tmpl, sub, B, start_quat, S);
  if (st != BH_OK) return st;
  if (L < (stage_table ? 1 : 0) || L > p->Lmax) return fail(BH_ERR_ARG, "L=%d outside 0..%d", L, p->Lmax);
  if (K < 1 || K > kMaxRefine || K > S) return fail(BH_ERR_ARG, "K=%d outside 1..min(%d, S=%d)", K, kMaxRefine, S);
  if (tmpl_index && n_templates < 1) return fail(BH_ERR_ARG, "n_templates=%d with tmpl_index", n_templates);
  if (B == 0) return BH_OK;
  if (!start_score || !quat_out || !score_out) return fail(BH_ERR_ARG, "NULL array");
  AlignArgs a{};
  a.lay = p->layout;
  a.tmpl = reinterpret_cast<const float2*>(tmpl);
  a.sub = reinterpret_cast<const float2*>(sub);
  a.tmpl_index = tmpl_index;
  a.n_templates = tmpl_index ? n_templates : 0;
  a.B = B;
  a.S = S;
  a.Lb = L;
  a.nstages = 1;  // the band of subtomograms whose table row is empty
  a.stages[0] = L;
  a.stage_table = stage_table;
  a.P = p->d_P;
  a.lbin = p->d_lbin;
  a.start_quat_out = reinterpret_cast<float4*>(const_cast<float*>(start_quat));
  a.start_score_out = const_cast<float*>(start_score);
  a.quat_out = reinterpret_cast<float4*>(quat_out);
  a.score_out = score_out;
  a.score64_out = score64_out;
  return launch_refine(a, L, K, p, static_cast<cudaStream_t>(stream));
}

extern "C" int bh_autotune(bh_plan* p, int B, int S, const int* stages, int nstages, int steps, bh_tune_result* out) {
  clear_error();
  const bh::Range range_("bh_autotune");
  if (!p) return fail(BH_ERR_ARG, "plan is NULL");
  if (B < 1 || B > (1 << 20)) return fail(BH_ERR_ARG, "B=%d", B);
  if (S < 1 || S > kMaxThreads) return fail(BH_ERR_ARG, "S=%d", S);
  if (!stages || nstages < 1 || nstages > kMaxStages) return fail(BH_ERR_ARG, "nstages=%d", nstages);
  const int Lb = stages[nstages - 1];
  if (Lb < 1 || Lb > p->Lmax) return fail(BH_ERR_ARG, "band %d", Lb);
  if (int rc = check_plan_device(p); rc != BH_OK) return rc;
  cudaStream_t st;
  BH_CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  cudaEvent_t e0, e1;
  BH_CUDA_TRY(cudaEventCreate(&e0));
  BH_CUDA_TRY(cudaEventCreate(&e1));
  float *coef = nullptr, *tmpl = nullptr, *starts = nullptr, *quat = nullptr, *score = nullptr, *vols = nullptr;
  const size_t N3 = (size_t)p->N * p->N * p->N;
  auto cleanup = [&]() {
    cudaStreamSynchronize(st);
    cudaFree(coef); cudaFree(tmpl); cudaFree(starts); cudaFree(quat); cudaFree(score); cudaFree(vols);
    cudaEventDestroy(e0); cudaEventDestroy(e1); cudaStreamDestroy(st);
  };
#define AT_TRY(call)                                                                                      \
  do {                                                                                                    \
    cudaError_t e_ = (call);                                                                              \
    if (e_ != cudaSuccess) {                                                                              \
      cleanup();                                                                                          \
      return fail(e_ == cudaErrorMemoryAllocation ? BH_ERR_OOM : BH_ERR_CUDA, "%s: %s", #call,            \
                  cudaGetErrorString(e_));                                                                \
    }                                                                                                     \
  } while (0)
  AT_TRY(cudaMalloc(&coef, (size_t)B * p->Nb * 8));
  AT_TRY(cudaMalloc(&tmpl, (size_t)p->Nb * 8));
  AT_TRY(cudaMalloc(&starts, (size_t)B * S * 16));
  AT_TRY(cudaMalloc(&quat, (size_t)B * 16));
  AT_TRY(cudaMalloc(&score, (size_t)B * 4));
  // value-independent timing: every byte 0x3C (float ~0.0115, never denormal)
  AT_TRY(cudaMemsetAsync(coef, 0x3C, (size_t)B * p->Nb * 8, st));
  AT_TRY(cudaMemsetAsync(tmpl, 0x3C, (size_t)p->Nb * 8, st));
  AT_TRY(cudaMemsetAsync(starts, 0x3C, (size_t)B * S * 16, st));
  int best_g = 0, best_c = 1, best_d = 1;
  float best_ms = 1e30f;
  // (lanes, starts per thread, dealing: 1 by rows, 2 flat)
  const int cand[][3] = {{1, 1, 1}, {2, 1, 1}, {4, 1, 1}, {8, 1, 1}, {16, 1, 1}, {2, 2, 1}, {4, 2, 1}, {8, 2, 1},
                         {16, 2, 1}, {4, 1, 2}, {8, 1, 2}, {16, 1, 2}, {4, 2, 2}, {8, 2, 2}, {16, 2, 2}};
  for (const auto& gc : cand) {
    const int G = gc[0], C = gc[1], Dv = gc[2];
    if (C == 2 && (S % 2)) continue;
    if (round_up((S / C) * G, 32) > kMaxThreads) continue;
    bh_align_opts o{};
    o.group = G;
    o.starts_per_thread = C;
    o.dealing = Dv;
    int rc = BH_OK;
    for (int it = 0; it < 2 && rc == BH_OK; ++it)
      rc = bh_align_batch(p, tmpl, coef, B, starts, S, stages, nstages, steps, quat, score, &o, st);
    if (rc != BH_OK) continue;
    AT_TRY(cudaEventRecord(e0, st));
    for (int it = 0; it < 3; ++it) bh_align_batch(p, tmpl, coef, B, starts, S, stages, nstages, steps, quat, score, &o, st);
    AT_TRY(cudaEventRecord(e1, st));
    AT_TRY(cudaEventSynchronize(e1));
    float ms = 0.f;
    AT_TRY(cudaEventElapsedTime(&ms, e0, e1));
    ms /= 3.f;
    if (ms < best_ms) {
      best_ms = ms;
      best_g = G;
      best_c = C;
      best_d = Dv;
    }
  }
  if (best_g == 0) {
    cleanup();
    return fail(BH_ERR_UNSUPPORTED, "no alignment variant runs for S=%d band %d", S, Lb);
  }
  p->align_group[{Lb, S}] = {best_g, best_c, best_d};
  int best_bn = 0;
  float best_ems = 0.f;
  if (p->mode == BH_MODE_BF16_SPLIT && !p->match_only) {
    AT_TRY(cudaMalloc(&vols, (size_t)B * N3 * 4));
    AT_TRY(cudaMemsetAsync(vols, 0x3C, (size_t)B * N3 * 4, st));
    best_ems = 1e30f;
    for (int bn : {128}) {
      int rc = set_gemm_bn(p, bn);
      for (int it = 0; it < 2 && rc == BH_OK; ++it) rc = bh_expand(p, vols, B, coef, st);
      if (rc != BH_OK) continue;
      AT_TRY(cudaEventRecord(e0, st));
      for (int it = 0; it < 3; ++it) bh_expand(p, vols, B, coef, st);
      AT_TRY(cudaEventRecord(e1, st));
      AT_TRY(cudaEventSynchronize(e1));
      float ms = 0.f;
      AT_TRY(cudaEventElapsedTime(&ms, e0, e1));
      ms /= 3.f;
      if (ms < best_ems) {
        best_ems = ms;
        best_bn = bn;
      }
    }
    int rc = set_gemm_bn(p, best_bn ? best_bn : 128);
    if (rc != BH_OK) {
      cleanup();
      return rc;
    }
  }
#undef AT_TRY
  cleanup();
  if (out) {
    out->align_group = best_g;
    out->align_starts_per_thread = best_c;
    out->align_dealing = best_d;
    out->align_ms = best_ms;
    out->gemm_bn = best_bn;
    out->expand_ms = best_ems;
  }
  return BH_OK;
}

extern "C" int bh_autotune_newton(bh_plan* p, int B, int S, const int* stages, int nstages, int steps,
                                  bh_tune_result* out) {
  clear_error();
  const bh::Range range_("bh_autotune_newton");
  if (!p) return fail(BH_ERR_ARG, "plan is NULL");
  if (B < 1 || B > (1 << 20)) return fail(BH_ERR_ARG, "B=%d", B);
  if (S < 1 || S > kMaxThreads) return fail(BH_ERR_ARG, "S=%d", S);
  if (!stages || nstages < 1 || nstages > kMaxStages) return fail(BH_ERR_ARG, "nstages=%d", nstages);
  const int Lb = stages[nstages - 1];
  if (Lb < 1 || Lb > p->Lmax) return fail(BH_ERR_ARG, "band %d", Lb);
  if (int rc = check_plan_device(p); rc != BH_OK) return rc;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float *coef = nullptr, *tmpl = nullptr, *starts = nullptr, *quat = nullptr, *score = nullptr;
  auto cleanup = [&]() {
    if (st) cudaStreamSynchronize(st);
    cudaFree(coef); cudaFree(tmpl); cudaFree(starts); cudaFree(quat); cudaFree(score);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
  };
  auto cuda_fail = [&](cudaError_t e, const char* what) {
    cleanup();
    return fail(e == cudaErrorMemoryAllocation ? BH_ERR_OOM : BH_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
  };
  cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaMalloc(&coef, (size_t)B * p->Nb * 8);
  if (e == cudaSuccess) e = cudaMalloc(&tmpl, (size_t)p->Nb * 8);
  if (e == cudaSuccess) e = cudaMalloc(&starts, (size_t)B * S * 16);
  if (e == cudaSuccess) e = cudaMalloc(&quat, (size_t)B * 16);
  if (e == cudaSuccess) e = cudaMalloc(&score, (size_t)B * 4);
  // every iteration evaluates its trial rotation whatever the data, so constant bytes time it faithfully
  if (e == cudaSuccess) e = cudaMemsetAsync(coef, 0x3C, (size_t)B * p->Nb * 8, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(tmpl, 0x3C, (size_t)p->Nb * 8, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(starts, 0x3C, (size_t)B * S * 16, st);
  if (e != cudaSuccess) return cuda_fail(e, "autotune setup");
  int best_g = 0, best_d = 1;
  float best_ms = 1e30f;
  struct Cand {
    int G, D;
  };
  for (const Cand c : {Cand{1, 1}, Cand{2, 1}, Cand{4, 1}, Cand{8, 1}, Cand{16, 1}, Cand{32, 1}, Cand{8, 2},
                       Cand{16, 2}, Cand{32, 2}}) {
    const int G = c.G;
    if (round_up(S * G, 32) > kMaxThreads) continue;
    bh_align_opts o{};
    o.group = G;
    o.dealing = c.D;
    o.newton = 1;
    int rc = BH_OK;
    for (int it = 0; it < 2 && rc == BH_OK; ++it)
      rc = bh_align_batch(p, tmpl, coef, B, starts, S, stages, nstages, steps, quat, score, &o, st);
    if (rc != BH_OK) continue;
    e = cudaEventRecord(e0, st);
    for (int it = 0; it < 3 && e == cudaSuccess; ++it)
      bh_align_batch(p, tmpl, coef, B, starts, S, stages, nstages, steps, quat, score, &o, st);
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) return cuda_fail(e, "autotune timing");
    ms /= 3.f;
    if (ms < best_ms) {
      best_ms = ms;
      best_g = G;
      best_d = c.D;
    }
  }
  cleanup();
  if (best_g == 0) return fail(BH_ERR_UNSUPPORTED, "no Newton variant runs for S=%d band %d", S, Lb);
  p->newton_group[{Lb, S}] = bh_plan::AlignVariant{best_g, 1, best_d};
  if (out) {
    *out = bh_tune_result{};
    out->align_group = best_g;
    out->align_starts_per_thread = 1;
    out->align_dealing = best_d;
    out->align_ms = best_ms;
  }
  return BH_OK;
}

extern "C" int bh_energy(const bh_plan* p, const float* tmpl, const float* sub, int B, int L, const int* tmpl_index,
                         int n_templates, float* energy, void* stream) {
  clear_error();
  const bh::Range range_("bh_energy");
  if (!p) return fail(BH_ERR_ARG, "plan is NULL");
  if (B < 0 || L < 0 || L > p->Lmax) return fail(BH_ERR_ARG, "B=%d L=%d", B, L);
  if (B == 0) return BH_OK;
  if (!tmpl || !sub || !energy) return fail(BH_ERR_ARG, "NULL array");
  if (tmpl_index && n_templates < 1) return fail(BH_ERR_ARG, "n_templates=%d", n_templates);
  if (int st = check_plan_device(p); st != BH_OK) return st;
  if (B > 65535 * 1024) return fail(BH_ERR_ARG, "B=%d too large", B);
  dim3 grid(B, L + 1);
  k_energy<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(p->layout, reinterpret_cast<const float2*>(tmpl),
                                                                 tmpl_index, n_templates,
                                                                 reinterpret_cast<const float2*>(sub), L, energy);
  BH_CHECK_LAUNCH();
  return BH_OK;
}

// ---------------------------------------------------------------------------- shift search
namespace bh {
namespace {
__global__ void k_repeat_starts(const float4* __restrict__ starts, int B, int S, int nshift, float4* __restrict__ out) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t total = (size_t)B * nshift * S;
  if (i >= total) return;
  const size_t s = i % S, r = i / S, b = r / nshift;
  out[i] = starts[b * S + s];
}

// Best shift per subtomogram by final score (exact ties: lowest shift index).
__global__ void k_select_shift(const float4* __restrict__ quat, const float* __restrict__ score, int B, int nshift,
                               int* __restrict__ shift_out, float4* __restrict__ quat_out, float* __restrict__ score_out) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  int best = 0;
  for (int j = 1; j < nshift; ++j)
    if (score[(size_t)b * nshift + j] > score[(size_t)b * nshift + best]) best = j;
  shift_out[b] = best;
  quat_out[b] = quat[(size_t)b * nshift + best];
  score_out[b] = score[(size_t)b * nshift + best];
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
}  // namespace
}  // namespace bh

extern "C" int bh_choose_bands(const bh_plan* p, const float* tmpl, const float* sub, int B, int L,
                               const int* tmpl_index, int n_templates, const double* thresholds, int n_thresholds,
                               int L_min, int* stage_table, float* energy, void* stream) {
  clear_error();
  const bh::Range range_("bh_choose_bands");
  if (!p) return fail(BH_ERR_ARG, "plan is NULL");
  if (B < 0 || L < 1 || L > p->Lmax) return fail(BH_ERR_ARG, "B=%d L=%d (band 1..%d)", B, L, p->Lmax);
  if (!thresholds || n_thresholds < 1 || n_thresholds > kMaxStages)
    return fail(BH_ERR_ARG, "n_thresholds=%d outside 1..%d", n_thresholds, kMaxStages);
  if (L_min < 1 || L_min > L) return fail(BH_ERR_ARG, "L_min=%d outside 1..%d", L_min, L);
  BandRule rule{};
  rule.n = n_thresholds;
  rule.L_min = L_min;
  for (int j = 0; j < n_thresholds; ++j) {
    const double t = thresholds[j];
    if (!(t > 0.0 && t < 1.0)) return fail(BH_ERR_ARG, "threshold %d = %g outside (0, 1)", j, t);
    if (j > 0 && !(t < thresholds[j - 1])) return fail(BH_ERR_ARG, "thresholds must decrease");
    rule.tau[j] = t;
  }
  if (tmpl_index && n_templates < 1) return fail(BH_ERR_ARG, "n_templates=%d", n_templates);
  if (int st = check_plan_device(p); st != BH_OK) return st;
  if (B == 0) return BH_OK;
  if (!tmpl || !sub || !stage_table) return fail(BH_ERR_ARG, "NULL array");
  k_choose_bands<<<B, kBandThreads, 0, static_cast<cudaStream_t>(stream)>>>(
      p->layout, reinterpret_cast<const float2*>(tmpl), tmpl_index, n_templates, reinterpret_cast<const float2*>(sub),
      L, rule, stage_table, energy);
  BH_CHECK_LAUNCH();
  return BH_OK;
}

extern "C" size_t bh_align_shifts_workspace(const bh_plan* p, int B, int nshift, int S) {
  if (!p || B < 0 || nshift < 1 || S < 1) return 0;
  const size_t R = (size_t)B * nshift;
  return align256((size_t)nshift * sizeof(int3)) + align256(R * p->Nb * 8) + align256(R * S * 16) + align256(R * 16) +
         align256(R * 4);
}

extern "C" int bh_align_shifts(bh_plan* p, const float* tmpl, const float* vols, int B, const int* shifts, int nshift,
                               const float* starts, int S, const int* stages, int nstages, int steps, void* workspace,
                               size_t workspace_bytes, int* shift_out, float* quat_out, float* score_out,
                               const bh_align_opts* opts, void* stream_) {
  clear_error();
  const bh::Range range_("bh_align_shifts");
  if (!p) return fail(BH_ERR_ARG, "plan is NULL");
  if (B < 0 || nshift < 1 || nshift > 4096 || S < 1) return fail(BH_ERR_ARG, "B=%d nshift=%d S=%d", B, nshift, S);
  if (int st = check_plan_device(p); st != BH_OK) return st;
  if (int st = check_expansion_plan(p); st != BH_OK) return st;
  if (B == 0) return BH_OK;
  if (!tmpl || !vols || !shifts || !starts || !workspace || !shift_out || !quat_out || !score_out)
    return fail(BH_ERR_ARG, "NULL argument");
  if (opts && (opts->start_quat_out || opts->start_score_out || opts->refine_fp64))
    return fail(BH_ERR_ARG, "per-start outputs and FP64 re-scoring are not available with shifts");
  if ((long long)B * nshift > (1LL << 30)) return fail(BH_ERR_ARG, "B * nshift too large");
  const size_t need = bh_align_shifts_workspace(p, B, nshift, S);
  if (workspace_bytes < need) return fail(BH_ERR_ARG, "workspace of %zu bytes, %zu needed", workspace_bytes, need);
  for (int j = 0; j < nshift; ++j)
    for (int d = 0; d < 3; ++d)
      if (shifts[3 * j + d] <= -p->N || shifts[3 * j + d] >= p->N)
        return fail(BH_ERR_ARG, "shift %d component %d = %d outside the box", j, d, shifts[3 * j + d]);
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  const size_t R = (size_t)B * nshift;
  char* w = static_cast<char*>(workspace);
  int3* d_shifts = reinterpret_cast<int3*>(w);
  w += align256((size_t)nshift * sizeof(int3));
  float* coeffs = reinterpret_cast<float*>(w);
  w += align256(R * p->Nb * 8);
  float4* rep = reinterpret_cast<float4*>(w);
  w += align256(R * S * 16);
  float4* q_all = reinterpret_cast<float4*>(w);
  w += align256(R * 16);
  float* s_all = reinterpret_cast<float*>(w);
  BH_CUDA_TRY(cudaMemcpyAsync(d_shifts, shifts, (size_t)nshift * sizeof(int3), cudaMemcpyHostToDevice, stream));
  int st = expand_shifted(p, vols, B, d_shifts, nshift, coeffs, stream);
  if (st != BH_OK) return st;
  const size_t n = R * S;
  k_repeat_starts<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(reinterpret_cast<const float4*>(starts), B, S, nshift,
                                                                  rep);
  BH_CHECK_LAUNCH();
  st = bh_align_batch(p, tmpl, coeffs, (int)R, reinterpret_cast<const float*>(rep), S, stages, nstages, steps,
                      reinterpret_cast<float*>(q_all), s_all, opts, stream);
  if (st != BH_OK) return st;
  k_select_shift<<<(B + 127) / 128, 128, 0, stream>>>(q_all, s_all, B, nshift, shift_out,
                                                      reinterpret_cast<float4*>(quat_out), score_out);
  BH_CHECK_LAUNCH();
  return BH_OK;
}

// ---------------------------------------------------------------------------- candidate starts (Sec. III)
struct bh_grid {
  int device = 0;
  int n = 0;
  int npow2 = 0;
  int max_nbr = 0;
  long long n_edges = 0;
  double radius = 0.0;
  float4* d_q = nullptr;   // [n] rotations (w, x, y, z) as given
  int* d_off = nullptr;    // [n + 1] CSR offsets of the neighbour lists
  int* d_nbr = nullptr;    // [n_edges] neighbour indices, ascending per grid point
  unsigned* d_pairs = nullptr;  // [n_edges / 2] neighbour pairs i < j packed as (i << 14) | j
  int n_pairs = 0;
  mutable std::mutex mu;
  mutable std::map<int, float4*> coef;  // band L -> [n_pad][Kf4(L)] Wigner coefficients of every rotation
};

namespace bh {
namespace {
constexpr int kGridMax = 16384;  // the sort keys of one subtomogram's grid scores live in shared memory
static_assert(kGridMax <= (1 << 14), "neighbour pairs pack two 14-bit grid indices");
constexpr int kCandThreads = 256;

// |q_i . q_j| >= c, the dot product summed in the order w, x, y, z in FP64 (exact products of floats).  An
// FP32 dot product decides every pair farther than 1e-5 from the threshold (its error is below 1e-6);
// the rest take the FP64 sum, so the relation is exactly the FP64 one.
__device__ __forceinline__ bool within(float4 a, float4 b, double c, float cf) {
  const float d32 = fabsf(fmaf(a.w, b.w, fmaf(a.z, b.z, fmaf(a.y, b.y, a.x * b.x))));
  if (fabsf(d32 - cf) > 1e-5f) return d32 > cf;
  double d = __dmul_rn((double)a.x, (double)b.x);
  d = __dadd_rn(d, __dmul_rn((double)a.y, (double)b.y));
  d = __dadd_rn(d, __dmul_rn((double)a.z, (double)b.z));
  d = __dadd_rn(d, __dmul_rn((double)a.w, (double)b.w));
  return fabs(d) >= c;
}

// Pass 1 (count) and pass 2 (fill, off != NULL) of the neighbour lists; one warp per grid point, lanes
// over j in chunks of 32, ballot compaction keeps each list ascending.
__global__ void k_grid_nbr(const float4* __restrict__ q, int n, double c, const int* __restrict__ off,
                           int* __restrict__ out) {
  const int i = (int)(((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= n) return;  // uniform per warp
  const float4 qi = q[i];
  const float cf = (float)c;
  int cnt = 0;
  int* dst = off ? out + off[i] : nullptr;
  for (int j0 = 0; j0 < n; j0 += 32) {
    const int j = j0 + lane;
    const bool hit = j < n && j != i && within(qi, q[j], c, cf);
    const unsigned m = __ballot_sync(0xffffffffu, hit);
    if (hit && dst) dst[cnt + __popc(m & ((1u << lane) - 1u))] = j;
    cnt += __popc(m);
  }
  if (!off && lane == 0) out[i] = cnt;
}

// Sort key of grid point i: [local-maximum flag : 1][score, order-preserving bits : 32][~i : 31], so that a
// larger key ranks higher (larger score; equal scores: lower index) and local maxima come first.
__device__ __forceinline__ unsigned long long grid_key(float s, int i) {
  unsigned u = __float_as_uint(s);
  u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
  return ((unsigned long long)u << 31) | (unsigned long long)(0x7FFFFFFF - i);
}

struct GridArgs {
  const float4* q;
  int n, npow2;
  int L;
  float4* starts_out;   // [B][S]
  int* index_out;       // [B][S] or NULL
  float* score_out;     // [B][n] or NULL
  const float* scores;  // [B_pad][ld] band-L scores of every grid rotation
  int ld;
  const unsigned* pairs;  // neighbour pairs (i << 14) | j, i < j
  int npairs;
};

constexpr int kSelectRounds = 64;  // up to this many candidates: S rounds of a block-wide argmax; above: sort

// Orbit-table entries of band L padded to a multiple of 4 float4 (the GEMM's K multiple of 16 floats).
__host__ __device__ inline int cand_kf4(int L) { return (tab_base(L + 1, L) + 3) & ~3; }

// Row p < B: the orbit table of band L of subtomogram p (the score's left factor, flattened); padding
// entries and rows p >= B are zero.
__global__ void __launch_bounds__(128) k_cand_tables(const AlignArgs a, int L, int Kf4, float4* __restrict__ X) {
  const int p = blockIdx.x;
  float4* row = X + (size_t)p * Kf4;
  const int nent = p < a.B ? tab_base(L + 1, L) : 0;
  if (p < a.B)
    build_table(row, a.lay, template_row(a, p), a.sub + (size_t)p * a.lay.Nb, a.P, L, threadIdx.x, blockDim.x);
  for (int e = nent + threadIdx.x; e < Kf4; e += blockDim.x) row[e] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// Wigner coefficients of the grid rotations at band L: for rotation i and orbit-table entry (m, l, n) the
// factor e_l (Re P1, -Im P1, Re P2, -Im P2) -- the rescaled d-recursion value of the orbit at degree l
// times the orbit's two phases, as in eval_rotations without the beta derivative -- so that the band-L
// score of a subtomogram, Re sum over entries of P1 e_l (x + iy) + P2 e_l (z + iw), is the dot product of
// its orbit table with row i: a dense contraction over all subtomograms and grid rotations.  One thread
// per rotation; the phases advance along the row (n += 1) by the ratios R1, R2.
__global__ void __launch_bounds__(128) k_grid_coef(const float4* __restrict__ gq, int n, int n_pad, int L, int Kf4,
                                                   const float* __restrict__ lbin, float4* __restrict__ coef) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_pad) return;
  float4* out = coef + (size_t)i * Kf4;
  if (i >= n) {
    for (int e = 0; e < Kf4; ++e) out[e] = make_float4(0.f, 0.f, 0.f, 0.f);
    return;
  }
  const float4 q = qnormalize(gq[i]);
  const float w = q.x, x = q.y, y = q.z, z = q.w;
  const float cb = sqrtf(w * w + z * z), sb = sqrtf(x * x + y * y);
  const float2 es = cb > 0.f ? make_float2(w / cb, z / cb) : make_float2(1.f, 0.f);
  const float2 ed = sb > 0.f ? make_float2(y / sb, -x / sb) : make_float2(1.f, 0.f);
  const float xb = (cb - sb) * (cb + sb);
  const float lcc = log2f(fmaxf(cb, 1e-30f)), lss = log2f(fmaxf(sb, 1e-30f));
  const float2 Es = cconj(es);
  const float2 R1 = cmul(Es, ed), R2 = cmul(Es, cconj(ed));
  const float2 Ed = cconj(ed);
  const float2 Ed2 = cmul(Ed, Ed);
  float2 Wrow = make_float2(1.f, 0.f);
  for (int m = 0; m <= L; ++m) {
    const int wd = 2 * m + 1;
    float4* rowp = out + tab_base(m, L);
    const float fm2 = (float)(m * m);
    float2 P1 = Wrow, P2 = cconj(Wrow);
    for (int nn = -m; nn <= m; ++nn) {
      const float lb = __ldg(lbin + m * kBinStride + m + nn);
      float d = exp2f(lb + (float)(m + nn) * lcc + (float)(m - nn) * lss);
      d = ((m - nn) & 1) ? -d : d;
      float4* ep = rowp + (nn + m);
      *ep = make_float4(d * P1.x, -d * P1.y, d * P2.x, -d * P2.y);
      const float mn = (float)(m * nn), fn2 = (float)(nn * nn);
      float e1 = d, e2 = 0.f;
      for (int l = m + 1; l <= L; ++l) {
        const float4 k0 = c_ecoef[l];
        const float g0 = (k0.z - fm2) * (k0.z - fn2) * k0.y;
        const float en = fmaf(fmaf(-mn, k0.x, xb), e1, -g0 * e2);
        ep += wd;
        *ep = make_float4(en * P1.x, -en * P1.y, en * P2.x, -en * P2.y);
        e2 = e1;
        e1 = en;
      }
      P1 = cmul(P1, R1);
      P2 = cmul(P2, R2);
    }
    Wrow = cmul(Wrow, Ed2);
  }
  for (int e = tab_base(L + 1, L); e < Kf4; ++e) out[e] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// One CTA per subtomogram: the band-L scores of every grid rotation (precomputed by the contraction) as
// rank keys in shared memory, local-maximum flags from the neighbour lists, then the S highest keys,
// either by S rounds of a block-wide argmax (S <= kSelectRounds) or by a bitonic sort of next_pow2(n)
// keys.
__global__ void __launch_bounds__(kCandThreads, 4) k_grid_candidates(const AlignArgs a, const GridArgs g) {
  extern __shared__ unsigned long long key[];
  __shared__ unsigned long long wbest[kCandThreads / 32];
  const int p = blockIdx.x;
  const bool sort = a.S > kSelectRounds;
  const int nkeys = sort ? g.npow2 : g.n;
  for (int i = g.n + threadIdx.x; i < nkeys; i += blockDim.x) key[i] = 0ull;  // padding ranks last
  // global loads in batches of kBatch per thread (coalesced across the block), so that a thread waits
  // about one L2 latency per batch rather than per element
  constexpr int kBatch = 8;
  const float* srow = g.scores + (size_t)p * g.ld;
  for (int i0 = threadIdx.x; i0 < g.n; i0 += kBatch * blockDim.x) {
    float e[kBatch];
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const int i = i0 + u * blockDim.x;
      e[u] = i < g.n ? __ldg(srow + i) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const int i = i0 + u * blockDim.x;
      if (i < g.n) {
        key[i] = grid_key(e[u], i);
        if (g.score_out) g.score_out[(size_t)p * g.n + i] = e[u];
      }
    }
  }
  __syncthreads();
  // local maxima over the neighbour pairs (coalesced 4-byte loads, each pair once): of every pair the
  // lower-ranked point is not a maximum
  unsigned char* notmax = reinterpret_cast<unsigned char*>(key + nkeys);
  for (int i = threadIdx.x; i < g.n; i += blockDim.x) notmax[i] = 0;
  __syncthreads();
  for (int e0 = threadIdx.x; e0 < g.npairs; e0 += kBatch * blockDim.x) {
    unsigned w[kBatch];
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const int e = e0 + u * blockDim.x;
      w[u] = e < g.npairs ? __ldg(g.pairs + e) : 0xFFFFFFFFu;
    }
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      if (w[u] != 0xFFFFFFFFu) {
        const int i = (int)(w[u] >> 14), j = (int)(w[u] & 0x3FFFu);
        notmax[key[i] > key[j] ? j : i] = 1;
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < g.n; i += blockDim.x)
    if (!notmax[i]) key[i] |= 1ull << 63;
  __syncthreads();
  if (!sort) {
    unsigned long long mine = 0ull;
    int pos = -1;
    for (int i = threadIdx.x; i < g.n; i += blockDim.x)
      if (key[i] > mine) {
        mine = key[i];
        pos = i;
      }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int s = 0; s < a.S; ++s) {
      unsigned long long v = mine;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long u = __shfl_xor_sync(0xffffffffu, v, o);
        v = u > v ? u : v;
      }
      if (lane == 0) wbest[warp] = v;
      __syncthreads();
      unsigned long long best = wbest[0];
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w) best = wbest[w] > best ? wbest[w] : best;
      if (threadIdx.x == 0) {
        const int i = 0x7FFFFFFF - (int)(best & 0x7FFFFFFFull);
        g.starts_out[(size_t)p * a.S + s] = g.q[i];
        if (g.index_out) g.index_out[(size_t)p * a.S + s] = i;
      }
      if (pos >= 0 && mine == best) {  // keys are unique: exactly one owner; it drops the key and rescans
        key[pos] = 0ull;
        mine = 0ull;
        pos = -1;
        for (int i = threadIdx.x; i < g.n; i += blockDim.x)
          if (key[i] > mine) {
            mine = key[i];
            pos = i;
          }
      }
      __syncthreads();
    }
    return;
  }
  // bitonic sort, descending
  for (int k = 2; k <= g.npow2; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < (g.npow2 >> 1); t += blockDim.x) {
        const int i = 2 * t - (t & (j - 1)), l = i + j;
        const unsigned long long x = key[i], y = key[l];
        if ((x < y) == ((i & k) == 0)) {
          key[i] = y;
          key[l] = x;
        }
      }
      __syncthreads();
    }
  }
  for (int s = threadIdx.x; s < a.S; s += blockDim.x) {
    const int i = 0x7FFFFFFF - (int)(key[s] & 0x7FFFFFFFull);
    g.starts_out[(size_t)p * a.S + s] = g.q[i];
    if (g.index_out) g.index_out[(size_t)p * a.S + s] = i;
  }
}

size_t grid_smem(int n, int npow2, int S) {
  return (size_t)(S > kSelectRounds ? npow2 : n) * 8 + (size_t)round_up(n, 16);  // rank keys + local-max flags
}
}  // namespace
}  // namespace bh

extern "C" int bh_grid_create(bh_grid** out, const float* quats, int n, double radius) {
  clear_error();
  const bh::Range range_("bh_grid_create");
  if (!out) return fail(BH_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!quats) return fail(BH_ERR_ARG, "quats is NULL");
  if (n < 1 || n > kGridMax) return fail(BH_ERR_ARG, "n=%d outside 1..%d", n, kGridMax);
  if (!(radius >= 0.0 && radius <= 3.141592653589793)) return fail(BH_ERR_ARG, "radius=%g outside [0, pi]", radius);
  for (int i = 0; i < n; ++i) {
    const double w = quats[4 * i], x = quats[4 * i + 1], y = quats[4 * i + 2], z = quats[4 * i + 3];
    const double r2 = w * w + x * x + y * y + z * z;
    if (!std::isfinite(r2) || std::fabs(r2 - 1.0) > 1e-4) return fail(BH_ERR_ARG, "grid rotation %d is not a unit quaternion", i);
  }
  std::unique_ptr<bh_grid, int (*)(bh_grid*)> g(new bh_grid(), bh_grid_destroy);
  BH_CUDA_TRY(cudaGetDevice(&g->device));
  g->n = n;
  g->radius = radius;
  g->npow2 = 32;
  while (g->npow2 < n) g->npow2 <<= 1;
  const double c = std::cos(radius / 2);
  BH_CUDA_TRY(cudaMalloc(&g->d_q, (size_t)n * sizeof(float4)));
  BH_CUDA_TRY(cudaMalloc(&g->d_off, (size_t)(n + 1) * sizeof(int)));
  BH_CUDA_TRY(cudaMemcpy(g->d_q, quats, (size_t)n * sizeof(float4), cudaMemcpyHostToDevice));
  int* d_cnt = nullptr;
  BH_CUDA_TRY(cudaMalloc(&d_cnt, (size_t)n * sizeof(int)));
  const unsigned nbr_blocks = (unsigned)(((size_t)n * 32 + 255) / 256);
  k_grid_nbr<<<nbr_blocks, 256>>>(g->d_q, n, c, nullptr, d_cnt);
  std::vector<int> cnt(n), off(n + 1, 0);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpy(cnt.data(), d_cnt, (size_t)n * sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(d_cnt);
  if (e != cudaSuccess) return fail(BH_ERR_CUDA, "neighbour count: %s", cudaGetErrorString(e));
  for (int i = 0; i < n; ++i) {
    off[i + 1] = off[i] + cnt[i];
    g->max_nbr = std::max(g->max_nbr, cnt[i]);
  }
  g->n_edges = off[n];
  BH_CUDA_TRY(cudaMemcpy(g->d_off, off.data(), (size_t)(n + 1) * sizeof(int), cudaMemcpyHostToDevice));
  BH_CUDA_TRY(cudaMalloc(&g->d_nbr, (size_t)std::max<long long>(1, g->n_edges) * sizeof(int)));
  k_grid_nbr<<<nbr_blocks, 256>>>(g->d_q, n, c, g->d_off, g->d_nbr);
  BH_CHECK_LAUNCH();
  BH_CUDA_TRY(cudaDeviceSynchronize());
  // each neighbour pair once (the relation is symmetric: the same FP64 dot product either way)
  std::vector<int> nbr((size_t)g->n_edges);
  if (g->n_edges)
    BH_CUDA_TRY(cudaMemcpy(nbr.data(), g->d_nbr, (size_t)g->n_edges * sizeof(int), cudaMemcpyDeviceToHost));
  std::vector<unsigned> pairs;
  pairs.reserve((size_t)g->n_edges / 2 + 1);
  for (int i = 0; i < n; ++i)
    for (int e = off[i]; e < off[i + 1]; ++e)
      if (nbr[e] > i) pairs.push_back(((unsigned)i << 14) | (unsigned)nbr[e]);
  g->n_pairs = (int)pairs.size();
  BH_CUDA_TRY(cudaMalloc(&g->d_pairs, std::max<size_t>(1, pairs.size()) * sizeof(unsigned)));
  if (!pairs.empty())
    BH_CUDA_TRY(cudaMemcpy(g->d_pairs, pairs.data(), pairs.size() * sizeof(unsigned), cudaMemcpyHostToDevice));
  *out = g.release();
  return BH_OK;
}

extern "C" int bh_grid_destroy(bh_grid* g) {
  if (!g) return BH_OK;
  for (auto& kv : g->coef) cudaFree(kv.second);
  cudaFree(g->d_pairs);
  cudaFree(g->d_q);
  cudaFree(g->d_off);
  cudaFree(g->d_nbr);
  delete g;
  return BH_OK;
}

extern "C" int bh_grid_info(const bh_grid* g, int* n, int* max_neighbors, long long* n_edges) {
  clear_error();
  if (!g) return fail(BH_ERR_ARG, "grid is NULL");
  if (n) *n = g->n;
  if (max_neighbors) *max_neighbors = g->max_nbr;
  if (n_edges) *n_edges = g->n_edges;
  return BH_OK;
}

extern "C" int bh_grid_neighbors(const bh_grid* g, int* offsets, int* neighbors, long long cap) {
  clear_error();
  if (!g) return fail(BH_ERR_ARG, "grid is NULL");
  if (!offsets || (!neighbors && g->n_edges > 0)) return fail(BH_ERR_ARG, "NULL output");
  if (cap < g->n_edges) return fail(BH_ERR_ARG, "cap %lld < %lld neighbour entries", cap, g->n_edges);
  BH_CUDA_TRY(cudaMemcpy(offsets, g->d_off, (size_t)(g->n + 1) * sizeof(int), cudaMemcpyDeviceToHost));
  if (g->n_edges > 0)
    BH_CUDA_TRY(cudaMemcpy(neighbors, g->d_nbr, (size_t)g->n_edges * sizeof(int), cudaMemcpyDeviceToHost));
  return BH_OK;
}

extern "C" int bh_candidates(const bh_plan* p, const bh_grid* grid, const float* tmpl, const float* sub, int B, int L,
                             const int* tmpl_index, int n_templates, int S, float* starts_out, int* index_out,
                             float* grid_score_out, void* stream) {
  clear_error();
  const bh::Range range_("bh_candidates");
  if (!p || !grid) return fail(BH_ERR_ARG, "plan or grid is NULL");
  if (B < 0) return fail(BH_ERR_ARG, "B=%d", B);
  if (L < 1 || L > p->Lmax) return fail(BH_ERR_ARG, "L=%d outside 1..%d", L, p->Lmax);
  if (S < 1 || S > grid->n) return fail(BH_ERR_ARG, "S=%d outside 1..%d (grid size)", S, grid->n);
  if (int st = check_plan_device(p); st != BH_OK) return st;
  if (tmpl_index && n_templates < 1) return fail(BH_ERR_ARG, "n_templates=%d with tmpl_index", n_templates);
  if (B == 0) return BH_OK;
  if (!tmpl || !sub || !starts_out) return fail(BH_ERR_ARG, "NULL array");
  int dev = 0;
  BH_CUDA_TRY(cudaGetDevice(&dev));
  if (dev != grid->device) return fail(BH_ERR_ARG, "grid lives on device %d, current device is %d", grid->device, dev);
  const size_t smem = grid_smem(grid->n, grid->npow2, S);
  if (smem > 232448) return fail(BH_ERR_ARG, "%d grid points need %zu bytes of shared memory", grid->n, smem);
  AlignArgs a{};
  a.lay = p->layout;
  a.tmpl = reinterpret_cast<const float2*>(tmpl);
  a.tmpl_index = tmpl_index;
  a.n_templates = n_templates;
  a.sub = reinterpret_cast<const float2*>(sub);
  a.B = B;
  a.S = S;
  a.Lb = L;
  a.P = p->d_P;
  a.lbin = p->d_lbin;
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  const int Kf4 = cand_kf4(L), n_pad = round_up(grid->n, 128), B_pad = round_up(B, 128);
  // Wigner coefficients of the grid at band L: built once per (grid, band), on a private stream that is
  // synchronised before use, so that every caller stream sees the finished matrix
  float4* coef = nullptr;
  {
    std::lock_guard<std::mutex> lk(grid->mu);
    auto it = grid->coef.find(L);
    if (it != grid->coef.end()) {
      coef = it->second;
    } else {
      BH_CUDA_TRY(cudaMalloc(&coef, (size_t)n_pad * Kf4 * sizeof(float4)));
      cudaStream_t s2 = nullptr;
      cudaError_t e = cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking);
      if (e == cudaSuccess) {
        k_grid_coef<<<(n_pad + 127) / 128, 128, 0, s2>>>(grid->d_q, grid->n, n_pad, L, Kf4, p->d_lbin, coef);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(s2);
        cudaStreamDestroy(s2);
      }
      if (e != cudaSuccess) {
        cudaFree(coef);
        return fail(BH_ERR_CUDA, "grid coefficients for band %d: %s", L, cudaGetErrorString(e));
      }
      grid->coef[L] = coef;
    }
  }
  // band-L scores of every (subtomogram, grid rotation): orbit tables [B_pad][4 Kf4] times coefficients
  // [n_pad][4 Kf4]^T, one FP32 GEMM
  float4* X = nullptr;
  float* scores = nullptr;
  BH_CUDA_TRY(cudaMallocAsync(&X, (size_t)B_pad * Kf4 * sizeof(float4), cs));
  cudaError_t ea = cudaMallocAsync(&scores, (size_t)B_pad * n_pad * sizeof(float), cs);
  if (ea != cudaSuccess) {
    cudaFreeAsync(X, cs);
    return fail(ea == cudaErrorMemoryAllocation ? BH_ERR_OOM : BH_ERR_CUDA, "candidate scores: %s", cudaGetErrorString(ea));
  }
  k_cand_tables<<<B_pad, 128, 0, cs>>>(a, L, Kf4, X);
  int st = BH_OK;
  cudaError_t el = cudaGetLastError();
  if (el != cudaSuccess) st = fail(BH_ERR_CUDA, "kernel launch: %s", cudaGetErrorString(el));
  if (st == BH_OK) st = sgemm_nt(reinterpret_cast<const float*>(X), reinterpret_cast<const float*>(coef), scores, B_pad, n_pad, 4 * Kf4, cs);
  if (st == BH_OK) {
    GridArgs g{grid->d_q, grid->n, grid->npow2, L,
               reinterpret_cast<float4*>(starts_out), index_out, grid_score_out, scores, n_pad,
               grid->d_pairs, grid->n_pairs};
    static SmemAttr have;
    st = ensure_smem(k_grid_candidates, have, smem);
    if (st == BH_OK) {
      k_grid_candidates<<<B, kCandThreads, smem, cs>>>(a, g);
      el = cudaGetLastError();
      if (el != cudaSuccess) st = fail(BH_ERR_CUDA, "kernel launch: %s", cudaGetErrorString(el));
    }
  }
  cudaFreeAsync(X, cs);
  cudaFreeAsync(scores, cs);
  return st;
}
