"""Force coefficients and shedding frequency of a force history (test
infrastructure; plain numpy).

The fluid force on the cylinder is the integral of the Lagrange multiplier,
F = -int_Gamma lambda (Section 5.3); Section 6 studies the drag and lift
coefficients C = F / (rho U^2 D / 2) and the vortex-shedding frequency of the
wake (Strouhal number St = f D / U).  The reading taken here: time averages
are trapezoidal over the samples at or after t_start; the frequency is the
peak of the spectrum of the lift minus its mean, resampled linearly on as many
uniform times, Hann-windowed, zero-padded eightfold, and refined by a
parabola through the log-magnitudes of the peak bin and its neighbours.
Pinned by sinusoids of known frequency, mean, amplitude and RMS.
"""
from __future__ import annotations

import numpy as np


def force_analysis(t, F, rho=1.0, U=1.0, D=1.0, t_start=0.0):
    t = np.asarray(t, dtype=np.float64)
    F = np.asarray(F, dtype=np.float64)
    q = 0.5 * rho * U * U * D
    sel = t >= t_start
    ts, cd, cl = t[sel], F[sel, 0] / q, F[sel, 1] / q
    T = ts[-1] - ts[0]
    cd_mean = np.trapezoid(cd, ts) / T
    cl_mean = np.trapezoid(cl, ts) / T
    cl_rms = np.sqrt(np.trapezoid((cl - cl_mean) ** 2, ts) / T)
    m = len(ts)
    h = T / (m - 1)
    tk = ts[0] + h * np.arange(m)
    g = (np.interp(tk, ts, cl) - cl_mean) * (0.5 - 0.5 * np.cos(2 * np.pi * np.arange(m) / (m - 1)))
    P = 8 * m
    mag = np.abs(np.fft.rfft(g, n=P))
    k = 1 + int(np.argmax(mag[1:P // 2]))
    a, b, c = np.log(mag[k - 1]), np.log(mag[k]), np.log(mag[k + 1])
    shift = 0.5 * (a - c) / (a - 2 * b + c) if (a - 2 * b + c) < 0 else 0.0
    f = (k + shift) / (P * h)
    return dict(cd_mean=cd_mean, cd_amp=0.5 * (cd.max() - cd.min()), cl_mean=cl_mean,
                cl_amp=0.5 * (cl.max() - cl.min()), cl_rms=cl_rms, frequency=f, strouhal=f * D / U,
                samples=m)
