// Force history analysis (host): drag and lift coefficients and the vortex
// shedding frequency (Strouhal number) from the hydrodynamic force the
// Newton steps report, F_fluid = -int_Gamma lambda (Section 5.3: the fluid
// force is the integral of the Lagrange multiplier; Section 6: force
// coefficients and the shedding frequency of the cylinder wake).
#include <algorithm>
#include <cmath>
#include <vector>

#include "viv_internal.h"

using namespace viv;

namespace {

// trapezoidal time average of v over samples [i0, n)
double time_mean(const double* t, const std::vector<double>& v, int64_t i0, int64_t n) {
  double s = 0;
  for (int64_t i = i0 + 1; i < n; ++i) s += 0.5 * (v[i] + v[i - 1]) * (t[i] - t[i - 1]);
  return s / (t[n - 1] - t[i0]);
}

}  // namespace

extern "C" vivStatus viv_force_analysis(const double* t, const double* Fx, const double* Fy, int64_t n, double rho,
                                        double U, double D, double t_start, vivForceStats* out) {
  try {
    VIV_CHECK(t && Fx && Fy && out, VIV_ERR_ARG, "NULL argument");
    VIV_CHECK(rho > 0 && U > 0 && D > 0, VIV_ERR_ARG, "rho, U and D must be positive");
    for (int64_t i = 1; i < n; ++i) VIV_CHECK(t[i] > t[i - 1], VIV_ERR_ARG, "times must increase");
    int64_t i0 = 0;
    while (i0 < n && t[i0] < t_start) ++i0;
    const int64_t m = n - i0;
    VIV_CHECK(m >= 8, VIV_ERR_ARG, "fewer than 8 samples after t_start");
    const double q = 0.5 * rho * U * U * D;   // dynamic pressure times the reference length
    std::vector<double> cd(n), cl(n);
    for (int64_t i = 0; i < n; ++i) {
      cd[i] = Fx[i] / q;
      cl[i] = Fy[i] / q;
    }
    vivForceStats r{};
    r.samples = m;
    r.cd_mean = time_mean(t, cd, i0, n);
    r.cl_mean = time_mean(t, cl, i0, n);
    double cdmin = cd[i0], cdmax = cd[i0], clmin = cl[i0], clmax = cl[i0], s2 = 0;
    for (int64_t i = i0; i < n; ++i) {
      cdmin = std::min(cdmin, cd[i]);
      cdmax = std::max(cdmax, cd[i]);
      clmin = std::min(clmin, cl[i]);
      clmax = std::max(clmax, cl[i]);
    }
    for (int64_t i = i0 + 1; i < n; ++i) {
      const double a = cl[i] - r.cl_mean, b = cl[i - 1] - r.cl_mean;
      s2 += 0.5 * (a * a + b * b) * (t[i] - t[i - 1]);
    }
    r.cd_amp = 0.5 * (cdmax - cdmin);
    r.cl_amp = 0.5 * (clmax - clmin);
    r.cl_rms = std::sqrt(s2 / (t[n - 1] - t[i0]));
    // dominant frequency of the lift: the lift minus its mean, linearly
    // resampled on m uniform times, Hann-windowed, zero-padded to 8 m and
    // transformed; the largest magnitude away from zero frequency, refined by
    // a parabola through the log-magnitudes of the peak and its neighbours
    const double T = t[n - 1] - t[i0], h = T / (double)(m - 1);
    std::vector<double> g(m);
    int64_t j = i0;
    const double pi = 3.14159265358979323846;
    for (int64_t k = 0; k < m; ++k) {
      const double tk = t[i0] + h * (double)k;
      while (j + 1 < n - 1 && t[j + 1] < tk) ++j;
      const double a = (tk - t[j]) / (t[j + 1] - t[j]);
      const double v = (1 - a) * cl[j] + a * cl[j + 1] - r.cl_mean;
      g[k] = v * (0.5 - 0.5 * std::cos(2 * pi * (double)k / (double)(m - 1)));
    }
    const int64_t P = 8 * m, nf = P / 2;
    std::vector<double> mag(nf + 1);
    for (int64_t f = 0; f <= nf; ++f) {
      double re = 0, im = 0;
      const double w = -2 * pi * (double)f / (double)P;
      for (int64_t k = 0; k < m; ++k) {
        re += g[k] * std::cos(w * (double)k);
        im += g[k] * std::sin(w * (double)k);
      }
      mag[f] = std::sqrt(re * re + im * im);
    }
    int64_t best = 1;
    for (int64_t f = 2; f < nf; ++f)
      if (mag[f] > mag[best]) best = f;
    double shift = 0;
    if (best > 0 && best < nf && mag[best - 1] > 0 && mag[best + 1] > 0) {
      const double a = std::log(mag[best - 1]), b = std::log(mag[best]), c = std::log(mag[best + 1]);
      const double den = a - 2 * b + c;
      if (den < 0) shift = 0.5 * (a - c) / den;
    }
    r.frequency = ((double)best + shift) / ((double)P * h);
    r.strouhal = r.frequency * D / U;
    *out = r;
  } catch (const Error& e) {
    set_error(e.msg);
    return e.status;
  }
  return VIV_OK;
}
