// Host set-up of a deformable body (Sec. 2.1 Eq. beam, App. A), FP64: the initial shape, the reference
// chords of the first step and the initial acceleration.  The element is the corotational Euler-Bernoulli
// beam of beam.cuh; here only its end forces are needed.
#include <cmath>
#include <vector>
#include "internal.h"

namespace {

// End forces of one element from its end nodes (x, y, theta); psi measured from the undeformed direction.
void element_forces(double L0, double ka, double kb, double ca0, double sa0, const double pa[3], const double pb[3],
                    double fa[3], double fb[3]) {
  const double dx = pb[0] - pa[0], dy = pb[1] - pa[1];
  const double L = std::hypot(dx, dy);
  const double c = dx / L, s = dy / L;
  const double psi = std::atan2(-dx * sa0 + dy * ca0, dx * ca0 + dy * sa0);
  const double tba = pa[2] - psi, tbb = pb[2] - psi;
  const double N = ka * (L - L0);
  const double Ma = kb * (2.0 * tba + tbb), Mb = kb * (tba + 2.0 * tbb);
  const double Q = (Ma + Mb) / L;
  fa[0] = -(N * c + Q * s);
  fa[1] = Q * c - N * s;
  fa[2] = Ma;
  fb[0] = -fa[0];
  fb[1] = -fa[1];
  fb[2] = Mb;
}

}  // namespace

// chi, zeta, zdot: 3 (n - 1) values each; ref: 3 (n - 1) values (psi, c, s per element).
// The flag starts at rest in the inextensible shape whose slope angle is tip (2 s/L - s^2/L^2) (zero at the
// clamp, tip at the free end): node rotations take that angle at the node, each chord the angle at its
// midpoint, so no element is stretched.  zeta = 0; zetadot balances the internal force (no fluid load at
// t = 0, no gravity).  Returns the tip displacement normal to the undeformed flag.
double beam_initial_state(const BodyHost& h, double ds, double tip, double* chi, double* zeta, double* zdot,
                          double* ref) {
  const int ne = h.n - 1;
  const double len = ne * ds;
  const double ca0 = std::cos(h.theta0), sa0 = std::sin(h.theta0);
  auto slope = [&](double sp) { return tip * (2.0 * sp / len - (sp / len) * (sp / len)); };
  double x = h.hx, y = h.hy;
  for (int e = 0; e < ne; ++e) {
    const double a = h.theta0 + slope((e + 0.5) * ds);
    x += ds * std::cos(a);
    y += ds * std::sin(a);
    chi[3 * e] = x;
    chi[3 * e + 1] = y;
    chi[3 * e + 2] = slope((e + 1) * ds);
  }
  const double ka = h.ea / ds, kb = 2.0 * h.ei / ds;
  std::vector<double> r(3 * ne, 0.0);
  for (int e = 0; e < ne; ++e) {
    const double pa[3] = {e == 0 ? h.hx : chi[3 * (e - 1)], e == 0 ? h.hy : chi[3 * (e - 1) + 1],
                          e == 0 ? 0.0 : chi[3 * (e - 1) + 2]};
    const double pb[3] = {chi[3 * e], chi[3 * e + 1], chi[3 * e + 2]};
    double fa[3], fb[3];
    element_forces(ds, ka, kb, ca0, sa0, pa, pb, fa, fb);
    for (int k = 0; k < 3; ++k) {
      if (e > 0) r[3 * (e - 1) + k] += fa[k];
      r[3 * e + k] += fb[k];
    }
    const double dx = pb[0] - pa[0], dy = pb[1] - pa[1], L = std::hypot(dx, dy);
    ref[3 * e] = std::atan2(-dx * sa0 + dy * ca0, dx * ca0 + dy * sa0);
    ref[3 * e + 1] = dx / L;
    ref[3 * e + 2] = dy / L;
  }
  for (int i = 0; i < ne; ++i) {
    const double mt = h.mu * ds * (i == ne - 1 ? 0.5 : 1.0), mr = mt * ds * ds / 12.0;
    for (int k = 0; k < 3; ++k) {
      zeta[3 * i + k] = 0.0;
      zdot[3 * i + k] = -r[3 * i + k] / (k < 2 ? mt : mr);
    }
  }
  const double tx = chi[3 * (ne - 1)] - (h.hx + len * ca0), ty = chi[3 * (ne - 1) + 1] - (h.hy + len * sa0);
  return -tx * sa0 + ty * ca0;
}
