"""Pins of the oracle's Feynman-Hellmann derivatives: the trilinear form with
equal propagators is the nucleon correlator, and the forward-mode derivatives
agree with central finite differences in m0 and lambda (h = 1e-4)."""
import numpy as np
import pytest

from oracle import nucleon
from oracle.gradient import FHCorrelator, project_time, trilinear
from paper_1605_00564_gb300 import synth


def test_trilinear_equal_slots_is_the_correlator():
    rng = np.random.default_rng(8)
    S = rng.standard_normal((2, 1, 1, 2, 4, 3, 4, 3)) + 1j * rng.standard_normal((2, 1, 1, 2, 4, 3, 4, 3))
    assert np.abs(trilinear(S, S, S) - nucleon.wick_contract(S)).max() < 1e-12 * np.abs(S).max() ** 3


@pytest.fixture(scope="module")
def fh():
    dims = (6, 2, 2, 2)
    U = synth.gauge_field(dims, 0.3, 91)
    return FHCorrelator(U, m0=0.2, csw=1.3, src=(1, 0, 0, 0))


def test_mass_derivative_finite_difference(fh):
    h = 1e-4
    dm, _ = fh.derivatives()
    cp = FHCorrelator(fh.U, fh.m0 + h, fh.csw, fh.src).correlator()
    cm = FHCorrelator(fh.U, fh.m0 - h, fh.csw, fh.src).correlator()
    fd = (cp - cm) / (2 * h)
    assert np.abs(dm - fd).max() < 1e-6 * np.abs(dm).max()


def test_lambda_derivative_finite_difference(fh):
    h = 1e-4
    _, dl = fh.derivatives()
    fd = (fh.correlator(lam=h) - fh.correlator(lam=-h)) / (2 * h)
    assert np.abs(dl - fd).max() < 1e-6 * max(np.abs(dl).max(), 1e-12)
    assert np.abs(dl).max() > 0
