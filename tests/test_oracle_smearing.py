"""Pins of the oracle's smearing (oracle/smearing.py).

* SU(3) projection: unitary, unit determinant, the identity on SU(3), and
  invariant under a positive rescaling.
* APE smearing: a pure-gauge field U_k(x) = g(x) g(x+k)^+ is a fixed point
  (every staple equals the link itself, so V = (1 + 4 alpha) U); gauge
  covariance under a random SU(3) transformation; time links untouched.
* Gaussian smearing: on the free field it is diagonal in spatial momentum
  with eigenvalue ((1 + 2 kappa sum_k cos p_k) / (1 + 6 kappa))^N (FFT closed
  form); gauge covariance; the operator is Hermitian; it acts within a
  time-slice.
"""
import numpy as np

from oracle import smearing
from paper_1605_00564_gb300 import synth

DIMS = (4, 4, 4, 6)   # T, X, Y, Z


def _gauge_transform(U, g):
    out = U.copy()
    for mu, ax in enumerate((0, 3, 2, 1)):
        gf = np.roll(g, -1, axis=ax)
        out[..., mu, :, :] = g @ U[..., mu, :, :] @ np.conj(np.swapaxes(gf, -1, -2))
    return out


def test_project_su3():
    U = synth.gauge_field(DIMS, 0.7, 1)[..., 1, :, :]
    W = smearing.project_su3(U)
    assert np.abs(W - U).max() < 1e-13
    assert np.abs(smearing.project_su3(2.5 * U) - U).max() < 1e-13
    rng = np.random.default_rng(0)
    V = rng.standard_normal(U.shape) + 1j * rng.standard_normal(U.shape)
    P = smearing.project_su3(V)
    eye = np.eye(3)
    assert np.abs(np.conj(np.swapaxes(P, -1, -2)) @ P - eye).max() < 1e-13
    assert np.abs(np.linalg.det(P) - 1).max() < 1e-13


def test_ape_pure_gauge_fixed_point_and_covariance():
    g = synth.random_su3_field(DIMS, 5)
    one = synth.unit_gauge(DIMS)
    Upure = _gauge_transform(one, g)
    S = smearing.ape_smear(Upure, 0.6, 3)
    assert np.abs(S - Upure).max() < 1e-12
    U = synth.gauge_field(DIMS, 0.5, 6)
    S = smearing.ape_smear(U, 0.45, 2)
    assert np.abs(S[..., 0, :, :] - U[..., 0, :, :]).max() == 0.0          # time links untouched
    assert np.abs(S - U).max() > 1e-2
    Sg = smearing.ape_smear(_gauge_transform(U, g), 0.45, 2)
    assert np.abs(Sg - _gauge_transform(S, g)).max() < 1e-12


def test_gaussian_free_field_closed_form():
    U = synth.unit_gauge(DIMS)
    T, X, Y, Z = DIMS
    psi = synth.random_spinor(DIMS, 3)
    kappa, n = 0.25, 5
    out = smearing.gaussian_smear(U, psi, kappa, n)
    # spatial axes of the (T, Z, Y, X) array: 1, 2, 3
    pz = 2 * np.pi * np.fft.fftfreq(Z)[:, None, None]
    py = 2 * np.pi * np.fft.fftfreq(Y)[None, :, None]
    px = 2 * np.pi * np.fft.fftfreq(X)[None, None, :]
    lam = ((1 + 2 * kappa * (np.cos(px) + np.cos(py) + np.cos(pz))) / (1 + 6 * kappa)) ** n
    ref = np.fft.ifftn(np.fft.fftn(psi, axes=(1, 2, 3)) * lam[None, :, :, :, None, None], axes=(1, 2, 3))
    assert np.abs(out - ref).max() < 1e-13


def test_gaussian_covariance_hermiticity_locality():
    U = smearing.ape_smear(synth.gauge_field(DIMS, 0.5, 7), 0.5, 1)
    g = synth.random_su3_field(DIMS, 8)
    a, b = synth.random_spinor(DIMS, 9), synth.random_spinor(DIMS, 10)
    K = lambda V, f: smearing.gaussian_smear(V, f, 0.3, 3)
    ga = np.einsum("...ab,...sb->...sa", g, a)
    assert np.abs(K(_gauge_transform(U, g), ga) - np.einsum("...ab,...sb->...sa", g, K(U, a))).max() < 1e-13
    assert abs(np.vdot(a, K(U, b)) - np.vdot(K(U, a), b)) < 1e-12 * abs(np.vdot(a, K(U, b)))
    e = np.zeros_like(a)
    e[2] = a[2]
    out = K(U, e)
    assert np.abs(out[[0, 1, 3]]).max() == 0.0
    mats = smearing.timeslice_matrices(U, 0.3, 3)
    flat = out[2][..., 0, :].reshape(-1)
    assert np.abs(mats[2] @ e[2][..., 0, :].reshape(-1) - flat).max() < 1e-13
