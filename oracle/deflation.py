"""Oracle: local deflation of Sec. 2.2 (FP64, numpy).

Test infrastructure only (see ``oracle/__init__``).

* The deflation subspace has dimension N = N_s N_b: N_s global fields are
  restricted to each of the N_b blocks and orthonormalised on every block by
  Gram-Schmidt, so each deflation field phi_k^b lives on one block.
* The global fields approximate low modes: starting from random fields (an
  input here), each round applies the SAP approximation M_SAP of D^-1 to
  every field (inverse iteration) and re-orthonormalises on the blocks.
* Little Dirac operator (eq. little): A_{(b,k),(b',l)} = (phi_k^b, D phi_l^b').
* Projectors: P_L = 1 - D Phi A^-1 Phi^+,  P_R = 1 - Phi A^-1 Phi^+ D, with
  P_L D = D P_R; the deflated solution (eq. deflsoln) is
  psi = chi + Phi A^-1 Phi^+ eta with P_L D chi = P_L eta.
* Preconditioner used with deflation (the low-mode solve plus SAP on the
  projected residual): M rho = Phi A^-1 Phi^+ rho + M_SAP(P_L rho).

Storage: ``phi`` has shape (N_s, T, Z, Y, X, 4, 3); its restriction to block
b is the set {phi_k^b}.  Little vectors are arrays (N_b, N_s), index
(b, k) <-> b * N_s + k.
"""
from __future__ import annotations

import numpy as np

from .sap import block_index


class Deflation:
    def __init__(self, op, block):
        self.op = op
        self.dims = op.dims
        self.block = tuple(block)
        self.bidx = block_index(self.dims, self.block)
        self.nb = int(self.bidx.max()) + 1
        self._flat = self.bidx.reshape(-1)

    # per-block inner products ------------------------------------------------
    def block_inner(self, a, b):
        """(a, b) restricted to every block: array (N_b,) complex."""
        v = np.sum(np.conj(a) * b, axis=(-2, -1)).reshape(-1)
        re = np.bincount(self._flat, weights=v.real, minlength=self.nb)
        im = np.bincount(self._flat, weights=v.imag, minlength=self.nb)
        return re + 1j * im

    def _per_site(self, coef):
        """Broadcast a per-block coefficient (N_b,) to a field-shaped factor."""
        return coef[self.bidx][..., None, None]

    def block_gram_schmidt(self, fields):
        """Orthonormalise the N_s fields on every block (modified Gram-Schmidt
        in the order k = 0, 1, ...)."""
        out = []
        for f in fields:
            v = f.copy()
            for q in out:
                v = v - self._per_site(self.block_inner(q, v)) * q
            n = np.sqrt(np.real(self.block_inner(v, v)))
            out.append(v / self._per_site(n))
        return np.stack(out)

    def subspace(self, init_fields, sap, n_inv):
        """Deflation fields from random init_fields: block Gram-Schmidt, then
        n_inv rounds of (M_SAP on every field, block Gram-Schmidt)."""
        phi = self.block_gram_schmidt(init_fields)
        for _ in range(n_inv):
            phi = self.block_gram_schmidt(np.stack([sap.apply(f) for f in phi]))
        self.phi = phi
        return phi

    # little vectors -------------------------------------------------------------
    def project(self, v):
        """Phi^+ v: c[b, k] = (phi_k^b, v)."""
        return np.stack([self.block_inner(p, v) for p in self.phi], axis=1)

    def prolong(self, c):
        """Phi c = sum_{b,k} c[b, k] phi_k^b."""
        out = np.zeros_like(self.phi[0])
        for k, p in enumerate(self.phi):
            out = out + self._per_site(c[:, k]) * p
        return out

    def little_dirac(self):
        """Dense A[(b,k), (b',l)] = (phi_k^b, D phi_l^b') from its definition:
        D applied to every single-block deflation field."""
        ns, nb = self.phi.shape[0], self.nb
        A = np.zeros((nb * ns, nb * ns), dtype=np.complex128)
        for bp in range(nb):
            m = (self.bidx == bp)[..., None, None]
            for l in range(ns):
                w = self.op.D(self.phi[l] * m)
                A[:, bp * ns + l] = self.project(w).reshape(-1)
        self.A = A
        return A

    def little_solve(self, c):
        return np.linalg.solve(self.A, c.reshape(-1)).reshape(c.shape)

    # projectors and the deflated preconditioner ---------------------------------
    def low_mode(self, v):
        """Phi A^-1 Phi^+ v."""
        return self.prolong(self.little_solve(self.project(v)))

    def P_L(self, v):
        return v - self.op.D(self.low_mode(v))

    def P_R(self, v):
        return v - self.low_mode(self.op.D(v))

    def precondition(self, rho, sap):
        """M rho = Phi A^-1 Phi^+ rho + M_SAP(P_L rho)."""
        return self.low_mode(rho) + sap.apply(self.P_L(rho))
