// Host side of a plan: FP64 radial data of the ball-harmonic basis (Sec. II-A), the real-form
// basis table, device uploads, error reporting.
//
// Basis (Sec. II-A, unnumbered display): psi_klm = c_lk j_l(lambda_lk r) Y_l^m(theta,phi) chi_[0,1)(r),
// lambda_lk the k-th positive root of j_l, c_lk > 0 normalisation constants.  Here c_lk makes psi
// orthonormal on the unit ball: c_lk = sqrt(2)/|j_{l+1}(lambda_lk)|, because the integral of
// j_l(lambda r)^2 r^2 over [0,1] is j_{l+1}(lambda)^2/2 at a root of j_l.
//
// The expansion f_hat_klm = h^3 sum_v f(x_v) conj(psi_klm(x_v)) of a real volume is computed as a
// real GEMM against a table with one row per coefficient slot (l,k,m):
//   m = 0:  h^3 R_lk(r) Pbar_l^0(cos theta)                 -> Re f_hat_kl0
//   m > 0:  h^3 R_lk(r) Pbar_l^m(cos theta) cos(m phi)      -> Re f_hat_klm
//   m < 0:  -h^3 R_lk(r) Pbar_l^|m|(cos theta) sin(|m| phi) -> Im f_hat_kl|m|
// with R_lk(r) = c_lk j_l(lambda_lk r) and Y_l^m = Pbar_l^m(cos theta) e^{i m phi}; negative orders
// follow from f_hat_{k,l,-m} = (-1)^m conj(f_hat_klm).
//
// Octant folding.  The in-ball voxels (coordinates i - N/2 with squared radius below (N/2)^2) form a set
// symmetric under the reflections x -> -x, y -> -y, z -> -z (the plane i = 0, at -N/2, lies outside the
// ball), and every real-form row is even or odd under each of them: odd in x for m > 0 odd and for m < 0
// with |m| even, odd in y for m < 0, odd in z for l + |m| odd.  So each row belongs to one parity class
// c = (odd in x) + 2 (odd in y) + 4 (odd in z), and sum_v f(v) psi(v) = sum_u psi(u) G_c(u) over the
// fundamental voxels u = (x, y, z >= 0), where G_c(u) = 2^{-zeros(u)} sum over the 8 sign images s u of
// (+-1) f(s u) (the sign odd in the class's odd axes; images that coincide on a zero coordinate counted
// once).  The table holds the rows class by class, each class padded to the GEMM's 128-column tile, over
// the fundamental voxels only: one eighth of the voxels, and so one eighth of the multiply-adds and of the
// table, for the same coefficients up to rounding.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <thread>

#include "bh_internal.h"

namespace bh {

static thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

void clear_error() { g_err.clear(); }

// ------------------------------------------------------------------ spherical Bessel functions
// j_0..j_L at x >= 0.  For x >= L the upward recurrence j_{l+1} = (2l+1)/x j_l - j_{l-1} is stable;
// below that, Miller's downward recurrence from well above max(L, x), normalised against the closed
// forms j_0 = sin x / x or j_1 = sin x / x^2 - cos x / x (whichever is larger in magnitude).
static void sph_bessel_seq(int L, double x, double* j) {
  if (x == 0.0) {
    j[0] = 1.0;
    for (int l = 1; l <= L; ++l) j[l] = 0.0;
    return;
  }
  const double s = std::sin(x), c = std::cos(x);
  const double j0 = s / x;
  const double j1 = s / (x * x) - c / x;
  j[0] = j0;
  if (L == 0) return;
  if (x >= L) {
    j[1] = j1;
    for (int l = 1; l < L; ++l) j[l + 1] = (2.0 * l + 1.0) / x * j[l] - j[l - 1];
    return;
  }
  const int n0 = L + 24 + (int)std::sqrt(40.0 * (L + 1)) + (int)x;
  std::vector<double> f(n0 + 2, 0.0);
  f[n0 + 1] = 0.0;
  f[n0] = 1e-280;
  for (int n = n0; n >= 1; --n) {
    f[n - 1] = (2.0 * n + 1.0) / x * f[n] - f[n + 1];
    if (std::fabs(f[n - 1]) > 1e250) {
      for (int i = n - 1; i <= n0 + 1; ++i) f[i] *= 1e-250;
    }
  }
  const double scale = (std::fabs(j0) >= std::fabs(j1)) ? j0 / f[0] : j1 / f[1];
  for (int l = 0; l <= L; ++l) j[l] = f[l] * scale;
}

static double sph_bessel(int l, double x) {
  std::vector<double> j(l + 1);
  sph_bessel_seq(l, x, j.data());
  return j[l];
}

// Positive roots of j_l up to lambda_max (+1e-9): sign-change scan with step 0.05 starting at
// max(l, 0.5) (the first root exceeds l), then bisection to the last representable bit.
static void bessel_roots(int l, double lam_max, std::vector<double>& out) {
  out.clear();
  const double x0 = (l == 0) ? 0.5 : (double)l;
  const double hi = lam_max + 0.5;
  double xa = x0, fa = sph_bessel(l, xa);
  for (int i = 1;; ++i) {
    const double xb = x0 + 0.05 * i;
    if (xb > hi + 0.05) break;
    const double fb = sph_bessel(l, xb);
    double root = -1.0;
    if (fa == 0.0) {
      root = xa;
    } else if ((fa < 0.0) != (fb < 0.0) && fb != 0.0) {
      double a = xa, b = xb, va = fa;
      for (int it = 0; it < 200 && b - a > 0.0; ++it) {
        const double mid = 0.5 * (a + b);
        if (mid <= a || mid >= b) break;
        const double vm = sph_bessel(l, mid);
        if (vm == 0.0) { a = b = mid; break; }
        if ((vm < 0.0) == (va < 0.0)) { a = mid; va = vm; } else { b = mid; }
      }
      root = 0.5 * (a + b);
    }
    if (root > 0.0 && root <= lam_max + 1e-9) out.push_back(root);
    xa = xb;
    fa = fb;
  }
}

// ------------------------------------------------------------------ real spherical harmonics
// Sphere-normalised associated Legendre functions with the Condon-Shortley phase,
// Pbar_l^m(x) for 0 <= m <= l <= L, stored at P[l*(L+1)+m]:
//   Pbar_0^0 = 1/sqrt(4 pi); Pbar_m^m = -sqrt((2m+1)/(2m)) sqrt(1-x^2) Pbar_{m-1}^{m-1};
//   Pbar_{m+1}^m = sqrt(2m+3) x Pbar_m^m;
//   Pbar_l^m = a_lm (x Pbar_{l-1}^m - Pbar_{l-2}^m / a_{l-1,m}), a_lm = sqrt((4l^2-1)/(l^2-m^2)).
void legendre_all(int L, double x, double* P) {
  const int W = L + 1;
  const double s = std::sqrt(std::fmax(0.0, 1.0 - x * x));
  P[0] = 1.0 / std::sqrt(4.0 * M_PI);
  for (int m = 1; m <= L; ++m) P[m * W + m] = -std::sqrt((2.0 * m + 1.0) / (2.0 * m)) * s * P[(m - 1) * W + m - 1];
  for (int m = 0; m < L; ++m) P[(m + 1) * W + m] = std::sqrt(2.0 * m + 3.0) * x * P[m * W + m];
  for (int m = 0; m <= L; ++m) {
    for (int l = m + 2; l <= L; ++l) {
      const double al = std::sqrt((4.0 * l * l - 1.0) / ((double)l * l - (double)m * m));
      const double alm1 = std::sqrt((4.0 * (l - 1) * (l - 1) - 1.0) / ((double)(l - 1) * (l - 1) - (double)m * m));
      P[l * W + m] = al * (x * P[(l - 1) * W + m] - P[(l - 2) * W + m] / alm1);
    }
  }
}

}  // namespace bh

// ====================================================================== C ABI (host parts)
using namespace bh;

extern "C" const char* bh_last_error(void) { return g_err.c_str(); }

extern "C" const char* bh_status_string(int s) {
  switch (s) {
    case BH_OK: return "BH_OK";
    case BH_PENDING: return "BH_PENDING";
    case BH_ERR_ARG: return "BH_ERR_ARG";
    case BH_ERR_CUDA: return "BH_ERR_CUDA";
    case BH_ERR_OOM: return "BH_ERR_OOM";
    case BH_ERR_BUDGET: return "BH_ERR_BUDGET";
    case BH_ERR_TIMEOUT: return "BH_ERR_TIMEOUT";
    case BH_ERR_BUSY: return "BH_ERR_BUSY";
    case BH_ERR_UNSUPPORTED: return "BH_ERR_UNSUPPORTED";
    default: return "BH_ERR_UNKNOWN";
  }
}

extern "C" int bh_version(void) { return 10000; }

static int compute_roots(int Lmax, double lam_max, std::vector<int>& K, std::vector<double>& lam,
                         std::vector<double>& cst) {
  K.assign(Lmax + 1, 0);
  lam.clear();
  cst.clear();
  std::vector<std::vector<double>> per(Lmax + 1);
  std::vector<std::thread> th;
  const int nth = std::max(1, std::min<int>(Lmax + 1, (int)std::thread::hardware_concurrency()));
  for (int t = 0; t < nth; ++t)
    th.emplace_back([&, t] {
      for (int l = t; l <= Lmax; l += nth) bessel_roots(l, lam_max, per[l]);
    });
  for (auto& x : th) x.join();
  for (int l = 0; l <= Lmax; ++l) {
    K[l] = (int)per[l].size();
    for (double r : per[l]) {
      lam.push_back(r);
      cst.push_back(std::sqrt(2.0) / std::fabs(sph_bessel(l + 1, r)));
    }
  }
  return BH_OK;
}

extern "C" int bh_basis_roots(int Lmax, double lambda_max, int* K, double* lambda, double* c, int cap) {
  clear_error();
  if (Lmax < 0 || Lmax > kMaxL) return fail(BH_ERR_ARG, "Lmax %d outside 0..%d", Lmax, kMaxL);
  if (!(lambda_max > 0.0) || lambda_max > 1e4) return fail(BH_ERR_ARG, "lambda_max %g outside (0, 1e4]", lambda_max);
  if (!K) return fail(BH_ERR_ARG, "K is NULL");
  std::vector<int> k;
  std::vector<double> lam, cst;
  compute_roots(Lmax, lambda_max, k, lam, cst);
  for (int l = 0; l <= Lmax; ++l) K[l] = k[l];
  if ((int)lam.size() > cap) return fail(BH_ERR_ARG, "capacity %d < %zu roots", cap, lam.size());
  if (!lambda || !c) return fail(BH_ERR_ARG, "lambda or c is NULL");
  for (size_t i = 0; i < lam.size(); ++i) {
    lambda[i] = lam[i];
    c[i] = cst[i];
  }
  return BH_OK;
}

static void free_plan(bh_plan* p) {
  if (!p) return;
  cudaFree(p->d_fund);
  cudaFree(p->d_slot);
  cudaFree(p->d_T32);
  cudaFree(p->d_Thi);
  cudaFree(p->d_Tlo);
  cudaFree(p->d_X32);
  cudaFree(p->d_Xhi);
  cudaFree(p->d_Xlo);
  cudaFree(p->d_C);
  cudaFree(p->d_err);
  cudaFree(p->d_P);
  cudaFree(p->d_lbin);
  cudaFree(p->d_coef64);
  cudaFree(p->d_lbin64);
  delete p;
}

extern "C" int bh_plan_create(bh_plan** out, const bh_plan_opts* o) {
  clear_error();
  const bh::Range range_("bh_plan_create");
  if (!out || !o) return fail(BH_ERR_ARG, "NULL argument");
  *out = nullptr;
  if (o->N < 4 || o->N > 256 || (o->N % 2)) return fail(BH_ERR_ARG, "N=%d must be even in 4..256", o->N);
  if (o->Lmax < 0 || o->Lmax > kMaxL) return fail(BH_ERR_ARG, "Lmax=%d outside 0..%d", o->Lmax, kMaxL);
  if (o->mode != BH_MODE_FP32 && o->mode != BH_MODE_BF16_SPLIT) return fail(BH_ERR_ARG, "mode=%d", o->mode);
  const double lam_max = (o->lambda_max > 0.0) ? o->lambda_max : M_PI * o->N / 2.0;
  if (lam_max > 1e4) return fail(BH_ERR_ARG, "lambda_max %g too large", lam_max);
  const int max_batch = (o->max_batch > 0) ? o->max_batch : 512;
  if (max_batch > (1 << 20)) return fail(BH_ERR_ARG, "max_batch %d too large", max_batch);
  if (o->flags & ~BH_PLAN_MATCH_ONLY) return fail(BH_ERR_ARG, "flags=%d", o->flags);
  const bool match_only = (o->flags & BH_PLAN_MATCH_ONLY) != 0;

  int dev = 0;
  BH_CUDA_TRY(cudaGetDevice(&dev));
  cudaDeviceProp prop;
  BH_CUDA_TRY(cudaGetDeviceProperties(&prop, dev));
  if (prop.major != 10 || prop.minor != 3)
    return fail(BH_ERR_UNSUPPORTED, "device %d is sm_%d%d; libbh is built for sm_103a (GB300)", dev, prop.major,
                prop.minor);
  int st = align_init_constants();
  if (st != BH_OK) return st;

  bh_plan* p = new bh_plan();
  p->device = dev;
  p->N = o->N;
  p->Lmax = o->Lmax;
  p->mode = o->mode;
  p->max_batch = max_batch;
  p->lam_max = lam_max;
  p->match_only = match_only;

  // ---- index set (FP64 roots and constants)
  compute_roots(p->Lmax, lam_max, p->K, p->lam, p->cst);
  p->offs.assign(p->Lmax + 2, 0);
  for (int l = 0; l <= p->Lmax; ++l) p->offs[l + 1] = p->offs[l] + p->K[l] * (2 * l + 1);
  p->Nb = p->offs[p->Lmax + 1];
  if (p->Nb == 0) {
    free_plan(p);
    return fail(BH_ERR_ARG, "empty index set (lambda_max %g below the first root)", lam_max);
  }
  p->layout.Lmax = p->Lmax;
  p->layout.Nb = p->Nb;
  for (int l = 0; l <= p->Lmax + 1; ++l) p->layout.off[l] = p->offs[l];
  for (int l = 0; l <= p->Lmax; ++l) p->layout.K[l] = p->K[l];

  // ---- voxels of the ball (counted) and its fundamental voxels x, y, z >= 0 (z-major order)
  const int N = p->N, h = N / 2;
  std::vector<int> fund, vox_r2;
  std::vector<int> vx, vy, vz;
  p->V = 0;
  for (int z = -h; z < h; ++z)
    for (int y = -h; y < h; ++y)
      for (int x = -h; x < h; ++x) p->V += (x * x + y * y + z * z < h * h) ? 1 : 0;
  for (int z = 0; z < h; ++z)
    for (int y = 0; y < h; ++y)
      for (int x = 0; x < h; ++x) {
        const int r2 = x * x + y * y + z * z;
        if (r2 < h * h) {
          fund.push_back(x | (y << 10) | (z << 20));
          vox_r2.push_back(r2);
          vx.push_back(x);
          vy.push_back(y);
          vz.push_back(z);
        }
      }
  p->VF = (int)fund.size();
  p->VF_pad = round_up(p->VF, kPadV);
  p->M_cap = round_up(max_batch, kGemmBM);

  // ---- radial table R[lk][r2] = c_lk j_l(lambda_lk sqrt(r2)/h), r2 = 0..h^2-1 (expansion plans only)
  const int n_r2 = match_only ? 0 : h * h;
  int nlk = 0;
  for (int l = 0; l <= p->Lmax; ++l) nlk += p->K[l];
  std::vector<double> radial((size_t)nlk * n_r2);
  {
    std::vector<int> lk_l(nlk);
    for (int l = 0, i = 0; l <= p->Lmax; ++l)
      for (int k = 0; k < p->K[l]; ++k) lk_l[i++] = l;
    std::vector<std::thread> th;
    const int nth = std::max(1u, std::thread::hardware_concurrency());
    for (int t = 0; t < nth; ++t)
      th.emplace_back([&, t] {
        std::vector<double> j(p->Lmax + 2);
        for (int i = t; i < nlk; i += nth) {
          const int l = lk_l[i];
          for (int r2 = 0; r2 < n_r2; ++r2) {
            const double x = p->lam[i] * std::sqrt((double)r2) / h;
            sph_bessel_seq(l, x, j.data());
            radial[(size_t)i * n_r2 + r2] = p->cst[i] * j[l];
          }
        }
      });
    for (auto& x : th) x.join();
  }

  // ---- angular table A[lm][v], lm = l^2 + l + m (real form, see header comment)
  const int nlm = (p->Lmax + 1) * (p->Lmax + 1);
  std::vector<double> angular(match_only ? 0 : (size_t)nlm * p->VF);
  if (!match_only) {
    std::vector<std::thread> th;
    const int nth = std::max(1u, std::thread::hardware_concurrency());
    const int L = p->Lmax;
    for (int t = 0; t < nth; ++t)
      th.emplace_back([&, t] {
        std::vector<double> P((L + 1) * (L + 1));
        for (int v = t; v < p->VF; v += nth) {
          const double x = vx[v], y = vy[v], z = vz[v];
          const double r = std::sqrt(x * x + y * y + z * z), rho = std::sqrt(x * x + y * y);
          const double ct = (r > 0) ? z / r : 1.0;
          const double cphi = (rho > 0) ? x / rho : 1.0, sphi = (rho > 0) ? y / rho : 0.0;
          legendre_all(L, ct, P.data());
          double cm = 1.0, sm = 0.0;  // cos(m phi), sin(m phi)
          for (int m = 0; m <= L; ++m) {
            for (int l = m; l <= L; ++l) {
              const double pl = P[l * (L + 1) + m];
              const int base = l * l + l;
              if (m == 0) {
                angular[(size_t)base * p->VF + v] = pl;
              } else {
                angular[(size_t)(base + m) * p->VF + v] = pl * cm;
                angular[(size_t)(base - m) * p->VF + v] = -pl * sm;
              }
            }
            const double cn = cm * cphi - sm * sphi, sn = sm * cphi + cm * sphi;
            cm = cn;
            sm = sn;
          }
        }
      });
    for (auto& x : th) x.join();
  }

  // ---- table rows (real form) grouped by parity class, and the complex sources of every slot
  std::vector<int> row_class(p->Nb), row_col(p->Nb);
  int class_count[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int l = 0; l <= p->Lmax; ++l)
    for (int k = 0; k < p->K[l]; ++k)
      for (int m = -l; m <= l; ++m) {
        const int s = p->offs[l] + k * (2 * l + 1) + m + l, mu = m < 0 ? -m : m;
        const int odd_x = (m >= 0) ? (mu & 1) : !(mu & 1), odd_y = m < 0, odd_z = (l + mu) & 1;
        row_class[s] = odd_x | (odd_y << 1) | (odd_z << 2);
        row_col[s] = class_count[row_class[s]]++;
      }
  int class_base[8];
  for (int c = 0, base = 0; c < 8; ++c) {
    class_base[c] = base;
    base += round_up(class_count[c], kGemmBN);
    p->cls.ntile_end[c] = base / kGemmBN;
  }
  p->Nb_pad = p->cls.ntile_end[7] * kGemmBN;
  for (int s = 0; s < p->Nb; ++s) row_col[s] += class_base[row_class[s]];
  std::vector<int2> colinfo(p->Nb_pad, make_int2(-1, -1));  // padding columns stay zero
  std::vector<int2> slot(p->Nb);
  for (int l = 0, lk = 0; l <= p->Lmax; ++l) {
    for (int k = 0; k < p->K[l]; ++k, ++lk) {
      const int base = p->offs[l] + k * (2 * l + 1);
      for (int m = -l; m <= l; ++m) {
        const int s = base + m + l;
        colinfo[row_col[s]] = make_int2(lk, l * l + l + m);
        const int mu = m < 0 ? -m : m;
        const int pos = row_col[base + l + mu], neg = row_col[base + l - mu];
        if (m == 0) {
          slot[s] = make_int2(pos + 1, 0);
        } else if (m > 0) {
          slot[s] = make_int2(pos + 1, neg + 1);
        } else {
          const int sg = (mu & 1) ? -1 : 1;
          slot[s] = make_int2(sg * (pos + 1), -sg * (neg + 1));
        }
      }
    }
  }

  // ---- device allocations and uploads
#define PLAN_TRY(call)            \
  do {                            \
    int st_ = (call);             \
    if (st_ != BH_OK) {           \
      free_plan(p);               \
      return st_;                 \
    }                             \
  } while (0)
  auto cuda_ok = [&](cudaError_t e, const char* what) -> int {
    if (e == cudaSuccess) return BH_OK;
    return fail(e == cudaErrorMemoryAllocation ? BH_ERR_OOM : BH_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
  };
  PLAN_TRY(cuda_ok(cudaMalloc(&p->d_fund, sizeof(int) * p->VF), "cudaMalloc fund"));
  PLAN_TRY(cuda_ok(cudaMemcpy(p->d_fund, fund.data(), sizeof(int) * p->VF, cudaMemcpyHostToDevice), "upload fund"));
  PLAN_TRY(cuda_ok(cudaMalloc(&p->d_slot, sizeof(int2) * p->Nb), "cudaMalloc slot"));
  PLAN_TRY(cuda_ok(cudaMemcpy(p->d_slot, slot.data(), sizeof(int2) * p->Nb, cudaMemcpyHostToDevice), "upload slot"));
  PLAN_TRY(cuda_ok(cudaMalloc(&p->d_err, sizeof(int)), "cudaMalloc err"));
  PLAN_TRY(cuda_ok(cudaMemset(p->d_err, 0, sizeof(int)), "memset err"));
  const size_t tab_elems = (size_t)p->Nb_pad * p->VF_pad;
  const size_t x_elems = (size_t)8 * p->M_cap * p->VF_pad;  // [class][row][fundamental voxel]
  if (match_only) {
    // no table, gathered volumes or GEMM output
  } else if (p->mode == BH_MODE_FP32) {
    PLAN_TRY(cuda_ok(cudaMalloc(&p->d_T32, sizeof(float) * tab_elems), "cudaMalloc table"));
    PLAN_TRY(cuda_ok(cudaMalloc(&p->d_X32, sizeof(float) * x_elems), "cudaMalloc X"));
  } else {
    PLAN_TRY(cuda_ok(cudaMalloc(&p->d_Thi, sizeof(__nv_bfloat16) * tab_elems), "cudaMalloc table hi"));
    PLAN_TRY(cuda_ok(cudaMalloc(&p->d_Tlo, sizeof(__nv_bfloat16) * tab_elems), "cudaMalloc table lo"));
    PLAN_TRY(cuda_ok(cudaMalloc(&p->d_Xhi, sizeof(__nv_bfloat16) * x_elems), "cudaMalloc X hi"));
    PLAN_TRY(cuda_ok(cudaMalloc(&p->d_Xlo, sizeof(__nv_bfloat16) * x_elems), "cudaMalloc X lo"));
  }
  // split-K capacity: about two waves over the SMs for a single 128-row pass, at most 8 splits
  p->num_sms = prop.multiProcessorCount;
  {
    const int tiles = p->Nb_pad / 128;
    p->ksplit_max = std::max(1, std::min(8, (2 * p->num_sms + tiles - 1) / tiles));
  }
  if (!match_only)
    PLAN_TRY(cuda_ok(cudaMalloc(&p->d_C, sizeof(float) * (size_t)p->ksplit_max * p->M_cap * p->Nb_pad),
                     "cudaMalloc C"));
  // ---- scale of the rescaled Wigner-d recursion: P_l(m,n) = prod_{j=m+1..l} j(2j-1)/sqrt((j^2-m^2)(j^2-n^2)),
  //      rows m = 0..Lmax, each [l = m..Lmax][n = -m..m]
  {
    std::vector<float> P;
    for (int m = 0; m <= p->Lmax; ++m) {
      std::vector<double> cur(2 * m + 1, 1.0);
      for (int l = m; l <= p->Lmax; ++l) {
        for (int n = -m; n <= m; ++n) {
          if (l > m)
            cur[n + m] *= (double)l * (2.0 * l - 1.0) /
                          std::sqrt(((double)l * l - (double)m * m) * ((double)l * l - (double)n * n));
          P.push_back((float)cur[n + m]);
        }
      }
    }
    PLAN_TRY(cuda_ok(cudaMalloc(&p->d_P, sizeof(float) * P.size()), "cudaMalloc P"));
    PLAN_TRY(cuda_ok(cudaMemcpy(p->d_P, P.data(), sizeof(float) * P.size(), cudaMemcpyHostToDevice), "upload P"));
    // coefficients of the rescaled recursion e^l = (cos beta - B_l) e^{l-1} - g_l e^{l-2}:
    //   B_l = m n / (l (l-1)),  g_l = ((l-1)^2 - m^2)((l-1)^2 - n^2) / ((l-1)^2 (2l-1)(2l-3))  (0 at l < 2)
    std::vector<double2> co64;
    co64.reserve(P.size());
    for (int m = 0; m <= p->Lmax; ++m)
      for (int l = m; l <= p->Lmax; ++l)
        for (int n = -m; n <= m; ++n) {
          double B = 0.0, g = 0.0;
          if (l >= 2) {
            const double a = (double)(l - 1) * (l - 1);
            B = (double)m * n / ((double)l * (l - 1));
            g = (a - (double)m * m) * (a - (double)n * n) / (a * (2.0 * l - 1.0) * (2.0 * l - 3.0));
          }
          co64.push_back(make_double2(B, g));
        }
    // 0.5 log2 C(2m, j), j = m + n
    const int stride = 2 * kMaxL + 1;
    std::vector<float> lb((size_t)(kMaxL + 1) * stride, 0.f);
    std::vector<double> lb64((size_t)(kMaxL + 1) * stride, 0.0);
    for (int m = 0; m <= kMaxL; ++m)
      for (int j = 0; j <= 2 * m; ++j) {
        lb64[(size_t)m * stride + j] =
            0.5 * (std::lgamma(2.0 * m + 1.0) - std::lgamma(j + 1.0) - std::lgamma(2.0 * m - j + 1.0)) / std::log(2.0);
        lb[(size_t)m * stride + j] = (float)lb64[(size_t)m * stride + j];
      }
    PLAN_TRY(cuda_ok(cudaMalloc(&p->d_lbin, sizeof(float) * lb.size()), "cudaMalloc lbin"));
    PLAN_TRY(cuda_ok(cudaMemcpy(p->d_lbin, lb.data(), sizeof(float) * lb.size(), cudaMemcpyHostToDevice), "upload lbin"));
    PLAN_TRY(cuda_ok(cudaMalloc(&p->d_coef64, sizeof(double2) * co64.size()), "cudaMalloc coef64"));
    PLAN_TRY(cuda_ok(cudaMemcpy(p->d_coef64, co64.data(), sizeof(double2) * co64.size(), cudaMemcpyHostToDevice),
                     "upload coef64"));
    PLAN_TRY(cuda_ok(cudaMalloc(&p->d_lbin64, sizeof(double) * lb64.size()), "cudaMalloc lbin64"));
    PLAN_TRY(cuda_ok(cudaMemcpy(p->d_lbin64, lb64.data(), sizeof(double) * lb64.size(), cudaMemcpyHostToDevice),
                     "upload lbin64"));
  }
  const double hv = 2.0 / N;
  if (!match_only) {
    PLAN_TRY(upload_table(p, radial, n_r2, angular, vox_r2, colinfo, hv * hv * hv));
    if (p->mode == BH_MODE_BF16_SPLIT) PLAN_TRY(make_tensor_maps(p));
  }
  PLAN_TRY(cuda_ok(cudaDeviceSynchronize(), "plan build"));
#undef PLAN_TRY
  *out = p;
  return BH_OK;
}

extern "C" int bh_plan_destroy(bh_plan* p) {
  clear_error();
  if (!p) return BH_OK;
  cudaDeviceSynchronize();
  free_plan(p);
  return BH_OK;
}

extern "C" int bh_plan_layout(const bh_plan* p, int* Nb, int* V, int* offsets) {
  clear_error();
  if (!p) return fail(BH_ERR_ARG, "plan is NULL");
  if (Nb) *Nb = p->Nb;
  if (V) *V = p->V;
  if (offsets)
    for (int l = 0; l <= p->Lmax + 1; ++l) offsets[l] = p->offs[l];
  return BH_OK;
}

extern "C" int bh_plan_gemm(const bh_plan* p, int* K, int* N) {
  clear_error();
  if (!p) return fail(BH_ERR_ARG, "plan is NULL");
  if (K) *K = p->VF_pad;
  if (N) *N = p->Nb_pad;
  return BH_OK;
}

extern "C" int bh_plan_info(const bh_plan* p, bh_plan_opts* o) {
  clear_error();
  if (!p || !o) return fail(BH_ERR_ARG, "NULL argument");
  o->N = p->N;
  o->Lmax = p->Lmax;
  o->lambda_max = p->lam_max;
  o->mode = p->mode;
  o->max_batch = p->max_batch;
  o->flags = p->match_only ? BH_PLAN_MATCH_ONLY : 0;
  return BH_OK;
}
