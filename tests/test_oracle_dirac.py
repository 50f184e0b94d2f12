"""Pins of the oracle's Wilson-clover operator against facts that do not come
from the oracle itself: the Clifford algebra, the free-field operator in
momentum space, gamma_5-hermiticity, gauge covariance, and a constant abelian
field strength whose clover term is known in closed form."""
import numpy as np
import pytest

from oracle import dirac
from oracle.dirac import GAMMA, GAMMA5, Operator, inner
from paper_1605_00564_gb300 import synth


def test_clifford_algebra_and_gamma5():
    for mu in range(4):
        assert np.allclose(GAMMA[mu], GAMMA[mu].conj().T)
        for nu in range(4):
            ac = GAMMA[mu] @ GAMMA[nu] + GAMMA[nu] @ GAMMA[mu]
            assert np.allclose(ac, 2.0 * (mu == nu) * np.eye(4))
    # chiral basis: gamma_5 = g0 g1 g2 g3 = diag(1, 1, -1, -1)
    assert np.allclose(GAMMA5, np.diag([1, 1, -1, -1]))
    for mu in range(4):
        for nu in range(4):
            s = dirac.sigma(mu, nu)
            assert np.allclose(s, s.conj().T)
            assert np.allclose(s @ GAMMA5, GAMMA5 @ s)


def _free_momentum_apply(psi, kappa, bc_t, inverse=False):
    """D(p) psi(p) with D(p) = (1 - 2 kappa sum cos p) + 2 i kappa sum g_mu sin p_mu,
    or its inverse written out in closed form, via FFT; antiperiodic time is a
    half-integer momentum shift pi/T."""
    T, Z, Y, X = psi.shape[:4]
    t = np.arange(T)
    twist = np.exp(1j * np.pi * t / T) if bc_t == -1 else np.ones(T)
    phi = psi * np.conj(twist)[:, None, None, None, None, None]
    ph = np.fft.fftn(phi, axes=(0, 1, 2, 3))
    p0 = 2 * np.pi * np.fft.fftfreq(T) + (np.pi / T if bc_t == -1 else 0.0)
    p3 = 2 * np.pi * np.fft.fftfreq(Z)
    p2 = 2 * np.pi * np.fft.fftfreq(Y)
    p1 = 2 * np.pi * np.fft.fftfreq(X)
    P = np.meshgrid(p0, p3, p2, p1, indexing="ij")
    mom = (P[0], P[3], P[2], P[1])       # p_mu for mu = t, x, y, z
    a = 1.0 - 2.0 * kappa * sum(np.cos(p) for p in mom)
    s = [2.0 * kappa * np.sin(p) for p in mom]
    slash = sum(s[m][..., None, None] * GAMMA[m] for m in range(4))
    if not inverse:
        Dp = a[..., None, None] * np.eye(4) + 1j * slash
    else:
        den = a ** 2 + sum(x ** 2 for x in s)
        Dp = (a[..., None, None] * np.eye(4) - 1j * slash) / den[..., None, None]
    out = np.einsum("...rs,...sa->...ra", Dp, ph)
    out = np.fft.ifftn(out, axes=(0, 1, 2, 3))
    return out * twist[:, None, None, None, None, None]


@pytest.mark.parametrize("bc_t", [-1, 1])
def test_free_field_matches_momentum_space(bc_t):
    dims = (8, 4, 6, 4)
    U = synth.unit_gauge(dims)
    op = Operator(U, kappa=0.124, csw=1.7, bc_t=bc_t)
    assert np.abs(op.C).max() == 0.0          # F = 0 at U = 1
    psi = synth.random_spinor(dims, 7)
    ref = _free_momentum_apply(psi, 0.124, bc_t)
    assert np.abs(op.D(psi) - ref).max() < 1e-13


def test_free_propagator_closed_form():
    from oracle.solve import gcr
    dims = (8, 4, 4, 4)
    op = Operator(synth.unit_gauge(dims), kappa=0.115, csw=1.0, bc_t=-1)
    src = synth.point_source(dims, (0, 0, 0, 0), 2, 1)
    S_ref = _free_momentum_apply(src, 0.115, -1, inverse=True)
    S, it, res = gcr(op, src, tol=1e-13)
    assert res < 1e-12
    assert np.abs(S - S_ref).max() / np.abs(S_ref).max() < 1e-11


def test_gamma5_hermiticity_and_adjoint():
    dims = (4, 4, 4, 4)
    op = Operator(synth.gauge_field(dims, 0.3, 11), kappa=0.13, csw=1.9)
    a = synth.random_spinor(dims, 1)
    b = synth.random_spinor(dims, 2)
    lhs = inner(a, dirac.gamma5(op.D(b)))
    rhs = inner(dirac.gamma5(op.D(a)), b)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    # the explicit adjoint agrees with (a, D b) = (D^+ a, b)
    assert abs(inner(a, op.D(b)) - inner(op.Ddag(a), b)) < 1e-12 * abs(lhs)
    # clover term Hermitian and block-diagonal in chirality
    C = op.C
    assert np.abs(C - np.conj(np.swapaxes(C, -1, -2))).max() < 1e-15
    g5 = np.kron(GAMMA5, np.eye(3))
    assert np.abs(C @ g5 - g5 @ C).max() < 1e-15
    assert np.abs(C).max() > 1e-2


def test_gauge_covariance():
    dims = (4, 4, 4, 6)
    U = synth.gauge_field(dims, 0.4, 3)
    Om = synth.random_su3_field(dims, 4)
    Ug = np.empty_like(U)
    for mu in range(4):
        Ug[..., mu, :, :] = Om @ U[..., mu, :, :] @ np.conj(np.swapaxes(dirac.link_at(Om, {mu: 1}), -1, -2))
    psi = synth.random_spinor(dims, 5)
    op, opg = Operator(U, 0.13, 1.9), Operator(Ug, 0.13, 1.9)
    lhs = opg.D(np.einsum("...ab,...sb->...sa", Om, psi))
    rhs = np.einsum("...ab,...sb->...sa", Om, op.D(psi))
    assert np.abs(lhs - rhs).max() < 1e-13


@pytest.mark.parametrize("mu,nu", [(1, 2), (0, 3), (2, 0)])
def test_clover_constant_abelian_field(mu, nu):
    """All (mu,nu) plaquettes equal diag(exp(i q phi)), so F_{mu nu} = i sin(q phi)
    and the site-diagonal part of D is 1 - kappa c_sw sigma_{mu nu} (x) diag(sin q phi)."""
    dims = (4, 4, 4, 4)
    U, phi = synth.constant_field_gauge(dims, mu, nu, 1)
    kappa, csw = 0.125, 1.3
    op = Operator(U, kappa, csw)
    expect = np.eye(12) - kappa * csw * np.kron(dirac.sigma(mu, nu), np.diag(np.sin(np.array([1.0, -1.0, 0.0]) * phi)))
    y = (1, 2, 3, 0)                      # (t, x, y, z)
    blk = np.zeros((12, 12), dtype=complex)
    for j in range(12):
        e = synth.point_source(dims, y, j // 3, j % 3)
        blk[:, j] = op.D(e)[y[0], y[3], y[2], y[1]].reshape(-1)
    assert np.abs(blk - expect).max() < 1e-14
