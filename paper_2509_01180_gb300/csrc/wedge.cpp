// Missing-wedge constrained correlation (Sec. II-B: the correlation is measured only in the region of
// Fourier space that both volumes sample): host preparation of the common-region norm, FP64.
//
// The subtomogram samples the Fourier directions |k_z| <= tan(a) |k_x| (tilt axis y, beam z, half-angle
// a); the template is complete.  Rotating the subtomogram by R rotates that region, W_R(k) = W(R^{-1} k),
// and the constrained score is C(R) = S(R) / sqrt(Dn(R)) with Dn(R) = ||W_R t||^2.  On the voxel grid,
// with W replaced by its spherical-harmonic expansion truncated at band L,
//   Dn(R) = |T(0)|^2 + sum_{0 < |k| < N/2} W_L(R^{-1} k/|k|) |T(k)|^2
//         = |T(0)|^2 + Re sum_{l<=L} sum_{m,m'} q_lm w_lm' D^l_{mm'}(R),
//   q_lm = sum_k Y_l^m(k/|k|) |T(k)|^2,   w_lm = integral over the sphere of W conj(Y_l^m),
// T the unnormalised DFT of the template restricted to the ball.  That is Eq. 2 with one radial index per
// degree: template pseudo-coefficients conj(q_lm) (|T(0)|^2 / w_00 added at l = 0) and subtomogram
// pseudo-coefficients w_lm, both with the symmetry of real functions, so the alignment kernels evaluate
// Dn and its gradient with their orbit tables.
//
// w_lm: for x = cos(theta) the sampled azimuths are |cos phi| >= |cot theta| / tan(a), two arcs whose
// phi integral is closed-form; the x integral is taken in phi0 = arccos(|cot theta| / tan(a)), in which
// the integrand is smooth (Gauss-Legendre with 96 nodes).  Only even l and even m survive.
#include <algorithm>
#include <cmath>
#include <complex>
#include <memory>
#include <thread>
#include <vector>

#include "bh_internal.h"

namespace bh {
namespace {

using cd = std::complex<double>;

// Gauss-Legendre nodes and weights on [-1, 1] (Newton iteration on P_n from the three-term recurrence).
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.resize(n);
  w.resize(n);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// In-place DFT along one axis (0 = x, fastest; 1 = y; 2 = z) of an N^3 array, e^{-2 pi i k n / N}.
void dft_axis(std::vector<cd>& v, int N, int axis, int nthreads) {
  std::vector<cd> tw(N);
  for (int j = 0; j < N; ++j) tw[j] = std::polar(1.0, -2.0 * M_PI * j / N);
  const size_t stride = axis == 0 ? 1 : (axis == 1 ? (size_t)N : (size_t)N * N);
  const int lines = N * N;
  auto work = [&](int t0, int t1) {
    std::vector<cd> in(N);
    for (int li = t0; li < t1; ++li) {
      const int a = li / N, b = li % N;
      size_t base;
      if (axis == 0) base = ((size_t)a * N + b) * N;
      else if (axis == 1) base = (size_t)a * N * N + b;
      else base = (size_t)a * N + b;
      for (int n = 0; n < N; ++n) in[n] = v[base + n * stride];
      for (int k = 0; k < N; ++k) {
        cd s = 0.0;
        for (int n = 0; n < N; ++n) s += in[n] * tw[(size_t)k * n % N];
        v[base + k * stride] = s;
      }
    }
  };
  std::vector<std::thread> th;
  const int per = (lines + nthreads - 1) / nthreads;
  for (int t = 0; t < nthreads; ++t) {
    const int t0 = t * per, t1 = std::min(lines, t0 + per);
    if (t0 < t1) th.emplace_back(work, t0, t1);
  }
  for (auto& x : th) x.join();
}

}  // namespace
}  // namespace bh

using namespace bh;

extern "C" int bh_wedge_destroy(bh_wedge* w) {
  if (!w) return BH_OK;
  cudaFree(w->d_t);
  cudaFree(w->d_w);
  delete w;
  return BH_OK;
}

extern "C" int bh_wedge_create(const bh_plan* p, const float* tvol, double half_angle_deg, int L, bh_wedge** out) {
  clear_error();
  const bh::Range range_("bh_wedge_create");
  if (!out) return fail(BH_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!p || !tvol) return fail(BH_ERR_ARG, "plan or template is NULL");
  if (L < 0 || L > p->Lmax) return fail(BH_ERR_ARG, "L=%d outside 0..%d", L, p->Lmax);
  if (!(half_angle_deg > 0.0 && half_angle_deg < 90.0))
    return fail(BH_ERR_ARG, "half_angle_deg=%g outside (0, 90)", half_angle_deg);
  const int N = p->N, h = N / 2;
  const size_t N3 = (size_t)N * N * N;
  std::unique_ptr<bh_wedge, int (*)(bh_wedge*)> wd(new bh_wedge(), bh_wedge_destroy);
  wd->device = p->device;
  wd->L = L;
  wd->half_angle = half_angle_deg;
  const int nthreads = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));

  // DFT of the template restricted to the ball (voxel (x, y, z) inside when |(x,y,z) - N/2|^2 < (N/2)^2)
  std::vector<cd> v(N3, 0.0);
  for (int z = 0; z < N; ++z)
    for (int y = 0; y < N; ++y)
      for (int x = 0; x < N; ++x) {
        const long r2 = (long)(x - h) * (x - h) + (long)(y - h) * (y - h) + (long)(z - h) * (z - h);
        if (r2 < (long)h * h) {
          const size_t i = ((size_t)z * N + y) * N + x;
          v[i] = (double)tvol[i];
        }
      }
  for (int a = 0; a < 3; ++a) dft_axis(v, N, a, nthreads);
  wd->c0 = std::norm(v[0]);

  // q_lm = sum over 0 < |k| < N/2 of Y_l^m(k/|k|) |T(k)|^2 for m >= 0; per-thread partial sums added in order
  const int W = L + 1;
  const int nq = W * W;  // [l][m] with m <= l used
  std::vector<std::vector<cd>> part(nthreads, std::vector<cd>(nq, 0.0));
  auto qwork = [&](int t, int z0, int z1) {
    std::vector<double> P((size_t)W * W);
    std::vector<cd>& acc = part[t];
    for (int zi = z0; zi < z1; ++zi)
      for (int yi = 0; yi < N; ++yi)
        for (int xi = 0; xi < N; ++xi) {
          const int kz = zi < h ? zi : zi - N, ky = yi < h ? yi : yi - N, kx = xi < h ? xi : xi - N;
          const long r2 = (long)kx * kx + (long)ky * ky + (long)kz * kz;
          if (r2 == 0 || r2 >= (long)h * h) continue;
          const double r = std::sqrt((double)r2), rho = std::sqrt((double)kx * kx + (double)ky * ky);
          const cd eiphi = rho > 0.0 ? cd(kx / rho, ky / rho) : cd(1.0, 0.0);
          const double pw = std::norm(v[((size_t)zi * N + yi) * N + xi]);
          legendre_all(L, kz / r, P.data());
          cd e = 1.0;
          for (int m = 0; m <= L; ++m) {
            const cd em = e * pw;
            for (int l = m; l <= L; ++l) acc[(size_t)l * W + m] += P[(size_t)l * W + m] * em;
            e *= eiphi;
          }
        }
  };
  {
    std::vector<std::thread> th;
    const int per = (N + nthreads - 1) / nthreads;
    for (int t = 0; t < nthreads; ++t) {
      const int z0 = t * per, z1 = std::min(N, z0 + per);
      if (z0 < z1) th.emplace_back(qwork, t, z0, z1);
    }
    for (auto& x : th) x.join();
  }
  std::vector<cd> qlm(nq, 0.0);
  for (int t = 0; t < nthreads; ++t)
    for (int i = 0; i < nq; ++i) qlm[i] += part[t][i];

  // w_lm by Gauss-Legendre in phi0 on [0, pi/2] (upper hemisphere, doubled)
  std::vector<double> gx, gw;
  gauss_legendre(96, gx, gw);
  const double Ta = std::tan(half_angle_deg * M_PI / 180.0);
  std::vector<double> wlm(nq, 0.0), P((size_t)W * W);
  for (int i = 0; i < 96; ++i) {
    const double phi0 = (gx[i] + 1.0) * (M_PI / 4.0), wq = gw[i] * (M_PI / 4.0);
    const double c = std::cos(phi0), den = 1.0 + Ta * Ta * c * c;
    const double x = Ta * c / std::sqrt(den), jac = Ta * std::sin(phi0) / (den * std::sqrt(den));
    legendre_all(L, x, P.data());
    for (int l = 0; l <= L; l += 2)
      for (int m = 0; m <= l; m += 2) {
        const double Phi = m == 0 ? 4.0 * phi0 : 4.0 * std::sin(m * phi0) / m;
        wlm[(size_t)l * W + m] += 2.0 * wq * P[(size_t)l * W + m] * Phi * jac;
      }
  }

  if (!(wlm[0] > 0.0)) return fail(BH_ERR_ARG, "the wedge samples no direction");
  // pseudo-coefficients in the K_l = 1 layout: slot l^2 + m + l
  const int nb = W * W;
  wd->q.assign(2 * (size_t)nb, 0.0);
  wd->w.assign(2 * (size_t)nb, 0.0);
  std::vector<float2> ht(nb), hw(nb);
  for (int l = 0; l <= L; ++l)
    for (int m = -l; m <= l; ++m) {
      const int am = m < 0 ? -m : m;
      const double sg = (m < 0 && (am & 1)) ? -1.0 : 1.0;
      cd q = qlm[(size_t)l * W + am];
      if (m < 0) q = sg * std::conj(q);  // q_{l,-m} = (-1)^m conj(q_lm) (real |T|^2)
      const double wv = sg * wlm[(size_t)l * W + am];  // w real: w_{l,-m} = (-1)^m w_lm
      const int s = l * l + m + l;
      wd->q[2 * s] = q.real();
      wd->q[2 * s + 1] = q.imag();
      wd->w[2 * s] = wv;
      cd tq = std::conj(q);
      if (l == 0) tq += wd->c0 / wv;
      ht[s] = make_float2((float)tq.real(), (float)tq.imag());
      hw[s] = make_float2((float)wv, 0.f);
    }

  Layout& lay = wd->layout;
  lay = Layout{};
  lay.Lmax = p->Lmax;
  lay.Nb = nb;
  for (int l = 0; l <= kMaxL + 1; ++l) lay.off[l] = std::min(l, L + 1) * std::min(l, L + 1);
  for (int l = 0; l <= kMaxL; ++l) lay.K[l] = l <= L ? 1 : 0;
  int dev = 0;
  BH_CUDA_TRY(cudaGetDevice(&dev));
  if (dev != p->device) return fail(BH_ERR_ARG, "plan lives on device %d, current device is %d", p->device, dev);
  BH_CUDA_TRY(cudaMalloc(&wd->d_t, (size_t)nb * sizeof(float2)));
  BH_CUDA_TRY(cudaMalloc(&wd->d_w, (size_t)nb * sizeof(float2)));
  BH_CUDA_TRY(cudaMemcpy(wd->d_t, ht.data(), (size_t)nb * sizeof(float2), cudaMemcpyHostToDevice));
  BH_CUDA_TRY(cudaMemcpy(wd->d_w, hw.data(), (size_t)nb * sizeof(float2), cudaMemcpyHostToDevice));
  *out = wd.release();
  return BH_OK;
}

extern "C" int bh_wedge_coeffs(const bh_wedge* w, double* q, double* wl, double* c0) {
  clear_error();
  if (!w) return fail(BH_ERR_ARG, "wedge is NULL");
  if (q) std::copy(w->q.begin(), w->q.end(), q);
  if (wl) std::copy(w->w.begin(), w->w.end(), wl);
  if (c0) *c0 = w->c0;
  return BH_OK;
}
