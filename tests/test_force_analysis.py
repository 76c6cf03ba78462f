"""Force coefficients and Strouhal number of a force history: the oracle
against closed forms, and the library's viv_force_analysis (host code, no
GPU) against the oracle."""
import numpy as np
import pytest

from oracle.analysis import force_analysis


def _signal(seed=0, n=4000, T=60.0, f=0.21):
    rng = np.random.default_rng(seed)
    t = np.sort(rng.uniform(0.0, T, n))          # uneven steps, as with adaptive dt
    F = np.stack([0.5 * (1.3 + 0.04 * np.sin(2 * np.pi * 2 * f * t)), 0.5 * 0.7 * np.sin(2 * np.pi * f * t + 0.4)], 1)
    return t, F


def test_oracle_recovers_closed_forms():
    """A lift 0.7 sin(2 pi f t) and a drag 1.3 + 0.04 sin(4 pi f t) in units of
    rho U^2 D / 2: mean 1.3 and half range 0.04 for the drag, half range 0.7,
    RMS 0.7 / sqrt 2 and frequency f for the lift (over about 12 periods)."""
    t, F = _signal()
    r = force_analysis(t, F, t_start=2.0)
    assert abs(r["cd_mean"] - 1.3) < 2e-3 and abs(r["cd_amp"] - 0.04) < 1e-4
    assert abs(r["cl_amp"] - 0.7) < 1e-4 and abs(r["cl_rms"] - 0.7 / np.sqrt(2)) < 5e-3
    assert abs(r["strouhal"] - 0.21) < 2e-4
    # scaling: St = f D / U and C = F / (rho U^2 D / 2)
    r2 = force_analysis(t, F * 4.0, rho=1.0, U=2.0, D=1.0, t_start=2.0)
    assert abs(r2["strouhal"] - 0.105) < 1e-4 and abs(r2["cl_amp"] - 0.7) < 1e-4


def test_library_matches_oracle():
    from paper_2609_31477_b300 import build, viv
    build.build()
    viv.load()
    t, F = _signal(seed=3)
    F = F + 1e-3 * np.random.default_rng(4).standard_normal(F.shape)
    a = viv.force_analysis(t, F, rho=1.2, U=1.1, D=0.9, t_start=5.0)
    b = force_analysis(t, F, rho=1.2, U=1.1, D=0.9, t_start=5.0)
    for k in ("cd_mean", "cd_amp", "cl_mean", "cl_amp", "cl_rms", "frequency", "strouhal"):
        assert abs(a[k] - b[k]) <= 1e-9 * max(1.0, abs(b[k])), (k, a[k], b[k])
    assert a["samples"] == b["samples"]
    with pytest.raises(viv.VivError):
        viv.force_analysis(t[:5], F[:5])
