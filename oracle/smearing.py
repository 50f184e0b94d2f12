"""Oracle: smeared sources and sinks (Sec. 2.3: Gaussian smearing of the
quark fields at source and sink, with APE-smeared gauge links in the
Laplacian), plain numpy FP64.

Test infrastructure only (see ``oracle/__init__``).

The paper fixes the method by citation and takes its parameters from earlier
work, so the parameters are inputs here.  Readings:

* APE smearing of the spatial links (k = 1, 2, 3), one step:
      V_k(x) = U_k(x) + alpha sum_{j spatial, j != k} [ U_j(x) U_k(x+j) U_j(x+k)^+
                                                      + U_j(x-j)^+ U_k(x-j) U_j(x-j+k) ]
      U'_k(x) = Proj_SU(3) V_k(x),
  applied n times; the time links are not used.  Proj_SU(3) takes the unitary
  factor W of the polar decomposition V = W (V^+ V)^(1/2) (from the singular
  value decomposition V = A S B^+, W = A B^+) and divides out the phase of its
  determinant with the principal cube root: W det(W)^(-1/3).
* Gaussian smearing of a field (spatial hops on one time-slice, colour
  matrices only, spin untouched), one step:
      psi'(x) = [ psi(x) + kappa_G sum_{k=1..3} ( U_k(x) psi(x+k) + U_k(x-k)^+ psi(x-k) ) ] / (1 + 6 kappa_G),
  applied N times with the APE-smeared links (periodic in space).  The
  operator is Hermitian, so a smeared sink is the same operator acting on the
  sink index of the propagator.
"""
from __future__ import annotations

import numpy as np

from .dirac import AXIS

SPATIAL = (1, 2, 3)


def _dag(M):
    return np.conj(np.swapaxes(M, -1, -2))


def _shift(field, mu, n):
    """field(x + n mu-hat), periodic (n = +1 or -1)."""
    return np.roll(field, -n, axis=AXIS[mu])


def project_su3(V):
    """Unitary polar factor of each 3x3 matrix, divided by the principal cube
    root of its determinant."""
    A, _, Bh = np.linalg.svd(V)
    W = A @ Bh
    det = np.linalg.det(W)
    return W * np.exp(-1j * np.angle(det) / 3.0)[..., None, None]


def ape_smear(U, alpha, n):
    """APE-smeared links: spatial links smeared n times, time links unchanged."""
    U = U.copy()
    for _ in range(n):
        new = U.copy()
        for k in SPATIAL:
            V = U[..., k, :, :].copy()
            for j in SPATIAL:
                if j == k:
                    continue
                Uj, Uk = U[..., j, :, :], U[..., k, :, :]
                # forward staple U_j(x) U_k(x+j) U_j(x+k)^+
                V = V + alpha * (Uj @ _shift(Uk, j, 1) @ _dag(_shift(Uj, k, 1)))
                # backward staple U_j(x-j)^+ U_k(x-j) U_j(x-j+k)
                Ujm = _shift(Uj, j, -1)
                V = V + alpha * (_dag(Ujm) @ _shift(Uk, j, -1) @ _shift(_shift(Uj, j, -1), k, 1))
            new[..., k, :, :] = project_su3(V)
        U = new
    return U


def hop3(U, psi):
    """sum_k U_k(x) psi(x+k) + U_k(x-k)^+ psi(x-k) on every site (colour only)."""
    out = np.zeros_like(psi)
    for k in SPATIAL:
        Uk = U[..., k, :, :]
        out = out + np.einsum("...ab,...sb->...sa", Uk, _shift(psi, k, 1))
        out = out + np.einsum("...ba,...sb->...sa", np.conj(_shift(Uk, k, -1)), _shift(psi, k, -1))
    return out


def gaussian_smear(U, psi, kappa_g, n):
    """(1 + kappa_g H)^n / (1 + 6 kappa_g)^n applied to psi [T, Z, Y, X, 4, 3]."""
    for _ in range(n):
        psi = (psi + kappa_g * hop3(U, psi)) / (1.0 + 6.0 * kappa_g)
    return psi


def timeslice_matrices(U, kappa_g, n):
    """The Gaussian smearing operator as one dense matrix per time-slice,
    K_t [3 L3, 3 L3] acting on (site of the time-slice, colour), spin
    untouched: column j of K_t is the smearing of the unit vector j (built
    from ``gaussian_smear`` itself, no other formula)."""
    T, Z, Y, X = U.shape[:4]
    L3 = Z * Y * X
    mats = np.zeros((T, 3 * L3, 3 * L3), dtype=np.complex128)
    for j in range(3 * L3):
        e = np.zeros((T, Z, Y, X, 4, 3), dtype=np.complex128)
        site, col = divmod(j, 3)
        z, r = divmod(site, Y * X)
        y, x = divmod(r, X)
        e[:, z, y, x, 0, col] = 1.0                        # the same unit vector on every time-slice
        out = gaussian_smear(U, e, kappa_g, n)[..., 0, :]  # spin 0 carries it; spin is untouched
        mats[:, :, j] = out.reshape(T, 3 * L3)
    return mats
