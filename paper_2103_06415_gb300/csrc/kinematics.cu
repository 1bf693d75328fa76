// Prescribed flapping kinematics of DRIVEN plates (Sec. 5.1), evaluated on the host once per step and
// uploaded ahead of the steps as a table the FSI kernels index by step number.
//
//   X1(t) = (A0/2) G_t(f t)/max G_t C(f t),  alpha1(t) = -beta G_r(f t)/max G_r,
//   G_t(tau) = int_0^tau tanh(sigma_t cos(2 pi u)) du,  G_r(tau) = tanh(sigma_r cos(2 pi tau)),
//   C(tau) = (tanh(8 tau - 2) + tanh 2)/(1 + tanh 2).
// The integrand of G_t has zero mean over a period, so G_t is periodic and only the fractional part of
// tau is integrated, by 16-point Gauss-Legendre quadrature on 16 equal panels (the integrand is analytic;
// its poles lie at least asinh(pi/(2 sigma_t))/(2 pi) from the real axis).
#include <cmath>
#include <vector>
#include "../../include/ibfsi_ops.h"
#include "internal.h"

namespace {

constexpr int kGauss = 16, kPanels = 16;

// nodes and weights of Gauss-Legendre quadrature on [-1, 1]: roots of P_n by Newton's method from the
// classical cosine estimate, weights 2 / ((1 - x^2) P_n'(x)^2)
struct GaussRule {
  double x[kGauss], w[kGauss];
  GaussRule() {
    const int n = kGauss;
    for (int i = 0; i < n; ++i) {
      double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
      double dp = 1.0;
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
};

const GaussRule& rule() {
  static const GaussRule r;
  return r;
}

double shape_t(double sigma, double tau) {
  const double frac = tau - std::floor(tau);
  if (frac <= 0.0) return 0.0;
  const GaussRule& g = rule();
  const double hp = frac / kPanels;
  double sum = 0.0;
  for (int p = 0; p < kPanels; ++p) {
    const double mid = (p + 0.5) * hp;
    double part = 0.0;
    for (int k = 0; k < kGauss; ++k) {
      const double u = mid + 0.5 * hp * g.x[k];
      part += g.w[k] * std::tanh(sigma * std::cos(2.0 * M_PI * u));
    }
    sum += 0.5 * hp * part;
  }
  return sum;
}

bool params_ok(const double* k) {
  for (int i = 0; i < 5; ++i)
    if (!std::isfinite(k[i])) return false;
  return k[0] >= 0.0 && k[2] > 0.0 && k[3] > 0.0 && k[4] > 0.0;
}

}  // namespace

bool flapping_params_ok(const double* k) { return params_ok(k); }

void flapping_state(const double* k, double t, double* out) {
  const double a0 = k[0], beta = k[1], st = k[2], sr = k[3], f = k[4];
  const double tau = f * t, w = 2.0 * M_PI;
  const double sn = std::sin(w * tau), cs = std::cos(w * tau);
  const double gt_max = shape_t(st, 0.25);
  const double g0 = shape_t(st, tau);
  const double tt = std::tanh(st * cs);
  const double g1 = tt, g2 = -w * st * sn * (1.0 - tt * tt);
  const double th2 = std::tanh(2.0), z = 8.0 * tau - 2.0, tz = std::tanh(z), sech2 = 1.0 - tz * tz;
  const double c0 = (tz + th2) / (1.0 + th2), c1 = 8.0 * sech2 / (1.0 + th2), c2 = -128.0 * sech2 * tz / (1.0 + th2);
  const double ax = 0.5 * a0 / gt_max;
  out[0] = ax * g0 * c0;
  out[1] = f * ax * (g1 * c0 + g0 * c1);
  out[2] = f * f * ax * (g2 * c0 + 2.0 * g1 * c1 + g0 * c2);
  const double tr = std::tanh(sr * cs), s2 = 1.0 - tr * tr, du = -w * sr * sn;
  const double r0 = tr, r1 = s2 * du, r2 = -w * w * sr * cs * s2 - 2.0 * s2 * tr * du * du;
  const double ar = -beta / std::tanh(sr);
  out[3] = ar * r0;
  out[4] = f * ar * r1;
  out[5] = f * f * ar * r2;
}

// kinematics of the steps first .. first + n - 1 (each at its end time t_{n+1}) into the device table
// ([kin_cap][n_bodies][6], slot = step mod kin_cap); n <= kin_cap.  Pageable source: the call returns once
// the values are staged, and the copy is ordered on the context stream before the steps that read them.
fsi_status upload_kinematics(fsi_ctx* c, long long first, int n) {
  if (!c->d_kin || n <= 0) return FSI_OK;
  const int nbod = c->n_bodies;
  std::vector<double> buf((size_t)n * nbod * 6, 0.0);
  for (int k = 0; k < n; ++k) {
    const double t = (double)(first + k + 1) * c->g.dt;
    for (int bi = 0; bi < nbod; ++bi)
      if (c->bodies[bi].type == FSI_BODY_DRIVEN) flapping_state(c->bodies[bi].kin, t, &buf[((size_t)k * nbod + bi) * 6]);
  }
  // the slots may wrap around the end of the table: at most two copies
  const long long s0 = first % c->kin_cap;
  const int n1 = (int)std::min<long long>(n, c->kin_cap - s0);
  FSI_CUDA_TRY(cudaMemcpyAsync(c->d_kin + (size_t)s0 * nbod * 6, buf.data(), (size_t)n1 * nbod * 6 * 8,
                               cudaMemcpyHostToDevice, c->stream));
  if (n1 < n)
    FSI_CUDA_TRY(cudaMemcpyAsync(c->d_kin, buf.data() + (size_t)n1 * nbod * 6, (size_t)(n - n1) * nbod * 6 * 8,
                                 cudaMemcpyHostToDevice, c->stream));
  return FSI_OK;
}

extern "C" fsi_status fsi_op_flapping_kinematics(const double* params, double t, double* out) {
  if (!params || !out || !std::isfinite(t) || !params_ok(params)) return FSI_ERR_INVALID_ARG;
  flapping_state(params, t, out);
  return FSI_OK;
}
