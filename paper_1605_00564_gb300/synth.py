"""Seeded synthetic inputs: gauge fields, sources, gauge transformations.

This module is the one place where inputs are made.  Both the CUDA path
(through the binding) and the CPU oracle read the bytes produced here; it
holds none of the solver's or the contraction's arithmetic.

Conventions shared with the C-ABI (include/qcd.h):

* ``dims = (T, X, Y, Z)``; numpy arrays are shaped ``(T, Z, Y, X, ...)`` so
  that a C-order flatten gives the canonical site index
  ``((t*LZ + z)*LY + y)*LX + x`` (x fastest).
* Gauge field: ``(T, Z, Y, X, 4, 3, 3)`` complex128, ``U[..., mu, a, b]`` is
  the link from x to x + mu-hat, mu = 0 time, 1 x, 2 y, 3 z.
* Spinor: ``(T, Z, Y, X, 4, 3)`` complex128 (spin, colour); a batch of n
  right-hand sides is ``(n, T, Z, Y, X, 4, 3)``.

The paper's ensembles (CLS N_f = 2, Table 1) are not available, so the gauge
fields are the seeded stand-in ``U = exp(i eps H)`` with H a random traceless
Hermitian 3x3 matrix with Gaussian entries, one independent draw per link.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "lattice_shape", "gauge_field", "unit_gauge", "constant_field_gauge",
    "random_spinor", "point_source", "point_sources", "random_su3_field",
    "ama_source_shifts", "CONFIGS",
]

# Workloads used by the tests and the benchmark, named by what they are.
# (dims T,X,Y,Z; eps; csw; kappa; gauge seed)
CONFIGS = {
    "small_8c16":      dict(dims=(16, 8, 8, 8),   eps=0.30, csw=1.0, kappa=0.1300, seed=160500564),
    "prod_32c64":      dict(dims=(64, 32, 32, 32), eps=0.15, csw=1.9, kappa=0.1360, seed=160500565),
    # same field at kappa = 0.1300: at 0.1360 this synthetic field needs ~600
    # SAP-GCR outer iterations for a 1e-10 solve (beyond the O(100) the
    # workload is specified with); 0.1300 needs ~150
    "prod_32c64_k130": dict(dims=(64, 32, 32, 32), eps=0.15, csw=1.9, kappa=0.1300, seed=160500565),
    "batch2_24c48":    dict(dims=(48, 24, 24, 24), eps=0.15, csw=1.9, kappa=0.1355, seed=160500566),
    # same field at kappa = 0.1300, as for 32^3x64: at 0.1355 the 1e-10 solves
    # need ~390 SAP-GCR iterations on this field, at 0.1300 ~130
    "batch2_24c48_k130": dict(dims=(48, 24, 24, 24), eps=0.15, csw=1.9, kappa=0.1300, seed=160500566),
    "defl_48c96":      dict(dims=(96, 48, 48, 48), eps=0.12, csw=1.9, kappa=0.1362, seed=160500567),
}


def lattice_shape(dims):
    """numpy lattice shape (T, Z, Y, X) for dims = (T, X, Y, Z)."""
    T, X, Y, Z = (int(d) for d in dims)
    return (T, Z, Y, X)


def _rng(seed, stream):
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed) & 0xFFFFFFFFFFFF, int(stream)])))


def _expi_hermitian(H, eps):
    """exp(i eps H) for a stack of Hermitian 3x3 matrices (eigendecomposition)."""
    w, v = np.linalg.eigh(H)
    U = (v * np.exp(1j * eps * w)[..., None, :]) @ np.conj(np.swapaxes(v, -1, -2))
    return _reunitarise(U)


def _reunitarise(U):
    """Project a stack of near-SU(3) matrices back onto SU(3): Gram-Schmidt on
    rows 0 and 1, row 2 = conj(row0 x row1) (unit determinant)."""
    r0 = U[..., 0, :]
    r0 = r0 / np.linalg.norm(r0, axis=-1, keepdims=True)
    r1 = U[..., 1, :]
    r1 = r1 - np.sum(np.conj(r0) * r1, axis=-1, keepdims=True) * r0
    r1 = r1 / np.linalg.norm(r1, axis=-1, keepdims=True)
    r2 = np.conj(np.cross(r0, r1))
    return np.stack([r0, r1, r2], axis=-2)


def gauge_field(dims, eps, seed):
    """Seeded links U_mu(x) = exp(i eps H), H = (A + A^dag)/2 - tr/3, A_ij with
    independent N(0,1) real and imaginary parts.  One RNG stream per
    timeslice, so the field is generated slice by slice with bounded memory."""
    T, Z, Y, X = lattice_shape(dims)
    U = np.empty((T, Z, Y, X, 4, 3, 3), dtype=np.complex128)
    eye = np.eye(3)
    for t in range(T):
        g = _rng(seed, t)
        a = g.standard_normal((Z, Y, X, 4, 3, 3, 2))
        A = a[..., 0] + 1j * a[..., 1]
        H = 0.5 * (A + np.conj(np.swapaxes(A, -1, -2)))
        H = H - (np.trace(H, axis1=-2, axis2=-1).real / 3.0)[..., None, None] * eye
        U[t] = _expi_hermitian(H, eps)
    return U


def unit_gauge(dims):
    """Free field U_mu(x) = 1."""
    T, Z, Y, X = lattice_shape(dims)
    U = np.zeros((T, Z, Y, X, 4, 3, 3), dtype=np.complex128)
    U[..., :, :, :] = np.eye(3)
    return U


def constant_field_gauge(dims, mu, nu, n_flux, colour_charges=(1.0, -1.0, 0.0)):
    """Abelian background with a constant plaquette angle in the (mu, nu) plane.

    Links U_nu(x) = diag(exp(i q_a phi x_mu)) for the nu direction, with
    phi = 2 pi n_flux / (L_mu L_nu) chosen so that the field is periodic; all
    other links are 1 except U_mu at x_mu = L_mu - 1, which carries the
    compensating phase exp(-i q_a phi L_mu x_nu).  Every plaquette
    U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag then equals
    diag(exp(i q_a phi)) everywhere.  Returns (U, phi).
    """
    T, Z, Y, X = lattice_shape(dims)
    L = {0: T, 1: X, 2: Y, 3: Z}
    axis = {0: 0, 1: 3, 2: 2, 3: 1}
    phi = 2.0 * np.pi * n_flux / (L[mu] * L[nu])
    q = np.asarray(colour_charges, dtype=float)
    U = unit_gauge(dims)
    shp = (T, Z, Y, X)
    xmu = np.indices(shp)[axis[mu]]
    xnu = np.indices(shp)[axis[nu]]
    ph_nu = np.exp(1j * q[None, :] * (phi * xmu.reshape(-1))[:, None]).reshape(shp + (3,))
    U[..., nu, :, :] = 0
    for a in range(3):
        U[..., nu, a, a] = ph_nu[..., a]
    edge = xmu == L[mu] - 1
    ph_mu = np.exp(-1j * q[None, :] * (phi * L[mu] * xnu.reshape(-1))[:, None]).reshape(shp + (3,))
    for a in range(3):
        U[..., mu, a, a] = np.where(edge, ph_mu[..., a], 1.0)
    return U, phi


def random_spinor(dims, seed, nrhs=None):
    """Gaussian complex spinor field(s), unit-variance real and imaginary parts."""
    shp = lattice_shape(dims) + (4, 3)
    if nrhs is not None:
        shp = (int(nrhs),) + shp
    g = _rng(seed, 1 << 20)
    a = g.standard_normal(shp + (2,))
    return a[..., 0] + 1j * a[..., 1]


def point_source(dims, src, spin, colour):
    """delta(x - src) delta_{alpha,spin} delta_{a,colour}; src = (t, x, y, z)."""
    s = np.zeros(lattice_shape(dims) + (4, 3), dtype=np.complex128)
    t, x, y, z = src
    s[t, z, y, x, spin, colour] = 1.0
    return s


def point_sources(dims, src):
    """The 12 spin-colour point sources at src, ordered rhs = spin*3 + colour."""
    out = np.zeros((12,) + lattice_shape(dims) + (4, 3), dtype=np.complex128)
    t, x, y, z = src
    for al in range(4):
        for a in range(3):
            out[al * 3 + a, t, z, y, x, al, a] = 1.0
    return out


def random_su3_field(dims, seed):
    """Haar-random SU(3) matrix per site (QR of a complex Gaussian matrix with
    the phase of R's diagonal divided out, then determinant fixed)."""
    shp = lattice_shape(dims)
    g = _rng(seed, 1 << 21)
    a = g.standard_normal(shp + (3, 3, 2))
    A = a[..., 0] + 1j * a[..., 1]
    Q, R = np.linalg.qr(A)
    d = np.diagonal(R, axis1=-2, axis2=-1)
    Q = Q * (d / np.abs(d))[..., None, :]
    det = np.linalg.det(Q)
    Q = Q / (det ** (1.0 / 3.0))[..., None, None]
    return _reunitarise(Q)


def ama_source_shifts(dims, n_g, block=(4, 4, 4, 4)):
    """n_g source positions (t, x, y, z) for the AMA translations.

    The translations must map the SAP domains Omega and Omega* (the black and
    the white blocks) onto themselves: every component is a multiple of the
    block extent and the shift measured in blocks has an even sum.  Here each
    component is a multiple of twice the block extent: t = 2 b_t i mod T and
    x, y, z alternate between 0 and the largest multiple of 2 b below half the
    extent (bits 0, 1, 2 of i).  For T = 64, L = 32 and 4^4 blocks this gives
    t = 8 i and x, y, z in {0, 16}.
    """
    T, X, Y, Z = (int(d) for d in dims)
    bt, bx, by, bz = (int(b) for b in block)

    def half(L, b):
        return (L // 2) // (2 * b) * (2 * b)

    hx, hy, hz = half(X, bx), half(Y, by), half(Z, bz)
    out = []
    for i in range(n_g):
        out.append(((2 * bt * i) % T, hx * (i & 1), hy * ((i >> 1) & 1), hz * ((i >> 2) & 1)))
    return out
