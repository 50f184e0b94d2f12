"""Oracle: Schwarz alternating procedure (SAP) of Sec. 2.2 (FP64, numpy).

Test infrastructure only (see ``oracle/__init__``).

The lattice is divided into rectangular blocks arranged as a checkerboard:
Omega holds the blocks whose block coordinates sum to an even number
("black", colour 0), Omega* the others ("white", colour 1).  With 1_Omega the
projection onto the sites of Omega,

    D_Omega = 1_Omega D 1_Omega          (block-diagonal, Dirichlet boundaries)
    D_dOmega* = 1_Omega* D 1_Omega       (terms through which Omega* points
                                          receive contributions from Omega)

One SAP cycle maps psi -> (1 - K D) psi + K eta with
K = D_Omega^-1 + D_Omega*^-1 - D_Omega*^-1 D_dOmega* D_Omega^-1, and n_cy cycles
from psi = 0 give M_SAP = K sum_{nu < n_cy} (1 - D K)^nu.

In the residual form used here a half-cycle solves the block equations on
one colour, adds the block solution delta to psi and subtracts D delta
(the full operator) from the residual rho = eta - D psi.  The block solves
are either exact (dense LU per block, ``nmr=None``) or ``nmr`` steps of the
minimal-residual iteration started from zero on each block:
p = D_Lambda r, alpha = (p, r)/(p, p), x += alpha r, r -= alpha p.
The block-size, cycle count and MR-step count are the method's tunables.
"""
from __future__ import annotations

import numpy as np

from .dirac import AXIS


def block_coords(dims, block):
    """Per-site block coordinates (nt, nx, ny, nz) as a tuple of (T,Z,Y,X) arrays."""
    T, X, Y, Z = dims
    for L, b in zip(dims, block):
        if L % b:
            raise ValueError("block size must divide the lattice")
    idx = np.indices((T, Z, Y, X))
    return tuple(idx[AXIS[mu]] // block[mu] for mu in range(4))


def colour_mask(dims, block, colour):
    """True on the sites of blocks of the given colour (0 = Omega, 1 = Omega*)."""
    nb = [L // b for L, b in zip(dims, block)]
    if any(n % 2 for n in nb):
        raise ValueError("the checkerboard needs an even number of blocks per direction")
    bc = block_coords(dims, block)
    return (sum(bc) % 2) == colour


def block_index(dims, block):
    """Per-site block number, lexicographic in (t, z, y, x) block coordinates."""
    T, X, Y, Z = dims
    bt, bx, by, bz = block_coords(dims, block)
    nx, ny, nz = X // block[1], Y // block[2], Z // block[3]
    return ((bt * nz + bz) * ny + by) * nx + bx


def _restrict(mask, psi):
    return psi * mask[..., None, None]


def D_colour(op, mask, psi):
    """D_Lambda psi for all blocks of one colour: 1_c D 1_c psi."""
    return _restrict(mask, op.D(_restrict(mask, psi)))


def _block_sum(bidx, nblk, v):
    """Per-block sums of a complex per-site scalar field."""
    f = bidx.reshape(-1)
    re = np.bincount(f, weights=np.real(v).reshape(-1), minlength=nblk)
    im = np.bincount(f, weights=np.imag(v).reshape(-1), minlength=nblk)
    return re + 1j * im


def mr_block_solve(op, mask, bidx, nblk, rho, nmr):
    """nmr minimal-residual steps from zero on every block of one colour
    (each block with its own step length).  Returns (x, r) with r the
    block residual rho - D_Lambda x on those blocks."""
    x = np.zeros_like(rho)
    r = _restrict(mask, rho)
    for _ in range(nmr):
        p = D_colour(op, mask, r)
        pr = _block_sum(bidx, nblk, np.sum(np.conj(p) * r, axis=(-2, -1)))
        pp = _block_sum(bidx, nblk, np.sum(np.abs(p) ** 2, axis=(-2, -1))).real
        alpha = np.where(pp > 0, pr / np.where(pp > 0, pp, 1.0), 0.0)
        a = alpha[bidx][..., None, None] * mask[..., None, None]
        x = x + a * r
        r = r - a * p
    return x, r


class SAP:
    """SAP with either exact block solves (``nmr=None``; dense LU per colour,
    small lattices only) or ``nmr`` MR steps per block."""

    def __init__(self, op, block, ncy, nmr=None):
        self.op = op
        self.dims = op.dims
        self.block = tuple(block)
        self.ncy = int(ncy)
        self.nmr = nmr
        self.masks = [colour_mask(self.dims, self.block, c) for c in (0, 1)]
        self.bidx = block_index(self.dims, self.block)
        self.nblk = int(self.bidx.max()) + 1
        self._inv = None

    # exact block inverses (dense) ---------------------------------------
    def _dense_inverses(self):
        if self._inv is None:
            from .solve import dense_matrix
            M = dense_matrix(self.op)
            self._M = M
            inv = []
            for c in (0, 1):
                sel = np.repeat(self.masks[c].reshape(-1), 12)
                idx = np.nonzero(sel)[0]
                inv.append((idx, np.linalg.inv(M[np.ix_(idx, idx)])))
            self._inv = inv
        return self._inv

    def block_solve(self, colour, rho):
        """Approximate (or exact) D_c^-1 rho on the blocks of one colour."""
        if self.nmr is None:
            idx, inv = self._dense_inverses()[colour]
            out = np.zeros(rho.size, dtype=np.complex128)
            out[idx] = inv @ rho.reshape(-1)[idx]
            return out.reshape(rho.shape)
        x, _ = mr_block_solve(self.op, self.masks[colour], self.bidx, self.nblk, rho, self.nmr)
        return x

    def cycle(self, psi, rho):
        """One SAP cycle in residual form: black blocks, then white blocks."""
        for c in (0, 1):
            delta = self.block_solve(c, rho)
            psi = psi + delta
            rho = rho - self.op.D(delta)
        return psi, rho

    def apply(self, eta):
        """M_SAP eta: n_cy cycles starting from psi = 0."""
        psi = np.zeros_like(eta)
        rho = eta.copy()
        for _ in range(self.ncy):
            psi, rho = self.cycle(psi, rho)
        return psi

    # the paper's matrices, for the exact-block identities ------------------
    def kernel_matrix(self):
        """K = D_O^-1 + D_O*^-1 - D_O*^-1 D_dO* D_O^-1 as a dense matrix."""
        inv = self._dense_inverses()
        n = self._M.shape[0]
        Dinv = []
        for idx, iv in inv:
            m = np.zeros((n, n), dtype=np.complex128)
            m[np.ix_(idx, idx)] = iv
            Dinv.append(m)
        P0 = np.repeat(self.masks[0].reshape(-1), 12).astype(float)
        P1 = np.repeat(self.masks[1].reshape(-1), 12).astype(float)
        D_dOs = P1[:, None] * self._M * P0[None, :]
        return Dinv[0] + Dinv[1] - Dinv[1] @ D_dOs @ Dinv[0]

    def msap_matrix(self):
        """M_SAP = K sum_{nu < n_cy} (1 - D K)^nu as a dense matrix."""
        K = self.kernel_matrix()
        n = K.shape[0]
        X = np.eye(n) - self._M @ K
        S = np.eye(n, dtype=np.complex128)
        P = np.eye(n, dtype=np.complex128)
        for _ in range(1, self.ncy):
            P = P @ X
            S = S + P
        return K @ S
