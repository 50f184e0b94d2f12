"""Pins of the AMA error model (oracle/ama.py, eqs. ama1-ama3) on synthetic
measurements with a known correlation structure, and the library's host
implementation (qcd_ama_error_model) against the oracle.

Model: O_appx^g = a z + b e_g (a common part z shared by all positions and
an independent part e_g per position), O^f = O_appx^f + c d_f, all unit
normal.  Then corr(O^f, O_appx^f) = s / sqrt(s^2 + c^2) with s^2 = a^2 + b^2,
corr(O_appx^g, O_appx^g') = a^2 / s^2, so
    Delta r = (1/N_org - 1/N_G)(1 - s / sqrt(s^2 + c^2)),
    R = (N_G - 1)/N_G * a^2 / s^2,
and the variance of the AMA estimate (1/N_org) sum_f c d_f + mean_g O_appx^g
is c^2/N_org + a^2 + b^2/N_G exactly, against Var O^f = s^2 + c^2."""
import numpy as np
import pytest

from oracle import ama


def _sample(n_conf, n_org, n_g, a, b, c, seed):
    rng = np.random.default_rng(seed)
    z = rng.standard_normal((n_conf, 1))
    appx = a * z + b * rng.standard_normal((n_conf, n_g))
    exact = appx[:, :n_org] + c * rng.standard_normal((n_conf, n_org))
    return exact, appx[:, :n_org].copy(), appx


@pytest.mark.parametrize("a,b,c,n_org,n_g", [(0.0, 1.0, 0.3, 1, 8), (0.5, 1.0, 0.2, 2, 16), (1.0, 0.5, 0.0, 1, 4)])
def test_error_model_closed_form(a, b, c, n_org, n_g):
    n_conf = 40000
    exact, appx_org, appx = _sample(n_conf, n_org, n_g, a, b, c, seed=7)
    dr, R, model, measured = ama.error_model(exact, appx_org, appx)
    s = np.hypot(a, b)
    dr_ref = (1 / n_org - 1 / n_g) * (1 - s / np.hypot(s, c))
    R_ref = (n_g - 1) / n_g * a * a / (s * s)
    meas_ref = np.sqrt((c * c / n_org + a * a + b * b / n_g) / (s * s + c * c))
    tol = 4.0 / np.sqrt(n_conf)            # a few standard errors of a sample correlation
    assert abs(dr - dr_ref) < tol and abs(R - R_ref) < tol * 2, (dr, dr_ref, R, R_ref)
    assert abs(measured - meas_ref) < 3 * tol, (measured, meas_ref)
    if c == 0.0:
        assert dr == pytest.approx(0.0, abs=1e-12)      # perfect approximation: no bias-correction noise


def test_error_model_matches_library():
    """The library's host implementation against the oracle formula."""
    from paper_1605_00564_gb300 import build
    from paper_1605_00564_gb300.qcd import ama_error_model
    build.build()
    exact, appx_org, appx = _sample(500, 3, 12, 0.7, 1.0, 0.4, seed=11)
    ref = ama.error_model(exact, appx_org, appx)
    got = ama_error_model(exact, appx_org, appx)
    for k, r in zip(("dr", "R", "model", "measured"), ref):
        assert abs(got[k] - r) <= 1e-12 * max(1.0, abs(r)), (k, got[k], r)
