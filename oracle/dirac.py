"""Oracle: the O(a)-improved Wilson-clover Dirac operator (FP64, numpy).

Test infrastructure only (see ``oracle/__init__``).

The paper states the problem as the Dirac equation D psi = eta for
O(a)-improved Wilson quarks (Sec. 1 and Sec. 2.2) and leaves the operator's
normalisation, gamma basis and clover formula to the cited literature.  The
readings taken here are:

* kappa normalisation::

    (D psi)(x) = psi(x)
               - kappa sum_mu [ (1 - g_mu) U_mu(x)        psi(x + mu)
                              + (1 + g_mu) U_mu(x - mu)^+ psi(x - mu) ]
               + i kappa c_sw sum_{mu<nu} sigma_{mu nu} F_{mu nu}(x) psi(x)

  which is 2 kappa times the Wilson operator in lattice units with
  (i/4) c_sw sum_{mu,nu} sigma F, kappa = 1 / (2 m0 + 8).
* chiral Euclidean basis with Hermitian gammas, mu = 0 is time,
  gamma_5 = g0 g1 g2 g3 = diag(1, 1, -1, -1); sigma_{mu nu} = (i/2)[g_mu, g_nu].
* F_{mu nu}(x) = (Q_{mu nu}(x) - Q_{mu nu}(x)^+) / 8 with Q the sum of the
  four plaquette leaves in the (mu, nu) plane that touch x (no trace
  subtraction); leaves use the raw links.
* periodic in space, antiperiodic in time: a hop that crosses the boundary
  between t = T - 1 and t = 0 carries a factor ``bc_t`` (-1).
"""
from __future__ import annotations

import numpy as np

# --------------------------------------------------------------------------
# Dirac algebra
# --------------------------------------------------------------------------
_I2 = np.eye(2, dtype=np.complex128)
_Z2 = np.zeros((2, 2), dtype=np.complex128)
PAULI = (
    np.array([[0, 1], [1, 0]], dtype=np.complex128),
    np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    np.array([[1, 0], [0, -1]], dtype=np.complex128),
)


def _blocks(a, b, c, d):
    return np.block([[a, b], [c, d]])


GAMMA = (
    _blocks(_Z2, -_I2, -_I2, _Z2),
    _blocks(_Z2, -1j * PAULI[0], 1j * PAULI[0], _Z2),
    _blocks(_Z2, -1j * PAULI[1], 1j * PAULI[1], _Z2),
    _blocks(_Z2, -1j * PAULI[2], 1j * PAULI[2], _Z2),
)
GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]
ID4 = np.eye(4, dtype=np.complex128)


def sigma(mu, nu):
    """sigma_{mu nu} = (i/2) [gamma_mu, gamma_nu]."""
    return 0.5j * (GAMMA[mu] @ GAMMA[nu] - GAMMA[nu] @ GAMMA[mu])


# numpy axis of direction mu in a (T, Z, Y, X) lattice array
AXIS = (0, 3, 2, 1)


def dims_of(U):
    T, Z, Y, X = U.shape[:4]
    return (T, X, Y, Z)


# --------------------------------------------------------------------------
# Lattice shifts
# --------------------------------------------------------------------------
def link_at(field, disp):
    """field(x + disp) with periodic wrap; disp maps direction -> integer step.
    Used for gauge links (the time boundary sign belongs to the hop only)."""
    out = field
    for mu, n in disp.items():
        if n:
            out = np.roll(out, -n, axis=AXIS[mu])
    return out


def spinor_fwd(psi, mu, bc_t):
    """psi(x + mu), with the time-boundary factor on the hop from T-1 to 0."""
    out = np.roll(psi, -1, axis=AXIS[mu])
    if mu == 0 and bc_t != 1:
        out = out.copy()
        out[-1] *= bc_t
    return out


def spinor_bwd(psi, mu, bc_t):
    """psi(x - mu), with the time-boundary factor on the hop from 0 to T-1."""
    out = np.roll(psi, 1, axis=AXIS[mu])
    if mu == 0 and bc_t != 1:
        out = out.copy()
        out[0] *= bc_t
    return out


def colour_mul(U, psi):
    """(U psi)_{s a} = sum_b U_{a b} psi_{s b} per site."""
    return np.einsum("...ab,...sb->...sa", U, psi)


def colour_mul_dag(U, psi):
    """(U^+ psi)_{s a} = sum_b conj(U_{b a}) psi_{s b} per site."""
    return np.einsum("...ba,...sb->...sa", np.conj(U), psi)


def spin_mul(G, psi):
    """(G psi)_{r a} = sum_s G_{r s} psi_{s a} per site."""
    return np.einsum("rs,...sa->...ra", G, psi)


# --------------------------------------------------------------------------
# Clover term
# --------------------------------------------------------------------------
def _dag(M):
    return np.conj(np.swapaxes(M, -1, -2))


def clover_leaves(U, mu, nu):
    """Q_{mu nu}(x): sum of the four plaquettes in the (mu, nu) plane with a
    corner at x, each traversed counter-clockwise starting at x."""
    Umu, Unu = U[..., mu, :, :], U[..., nu, :, :]
    L1 = Umu @ link_at(Unu, {mu: 1}) @ _dag(link_at(Umu, {nu: 1})) @ _dag(Unu)
    L2 = (Unu @ _dag(link_at(Umu, {mu: -1, nu: 1})) @ _dag(link_at(Unu, {mu: -1}))
          @ link_at(Umu, {mu: -1}))
    L3 = (_dag(link_at(Umu, {mu: -1})) @ _dag(link_at(Unu, {mu: -1, nu: -1}))
          @ link_at(Umu, {mu: -1, nu: -1}) @ link_at(Unu, {nu: -1}))
    L4 = (_dag(link_at(Unu, {nu: -1})) @ link_at(Umu, {nu: -1})
          @ link_at(Unu, {mu: 1, nu: -1}) @ _dag(Umu))
    return L1 + L2 + L3 + L4


def field_strength(U, mu, nu):
    """F_{mu nu}(x) = (Q_{mu nu} - Q_{mu nu}^+) / 8 (anti-Hermitian)."""
    Q = clover_leaves(U, mu, nu)
    return (Q - _dag(Q)) / 8.0


def clover_field(U, kappa, csw):
    """Per-site 12x12 matrix C(x) = i kappa c_sw sum_{mu<nu} sigma_{mu nu} (x) F_{mu nu}(x),
    index (spin, colour) -> 3*spin + colour.  Hermitian, commutes with gamma_5."""
    shp = U.shape[:4]
    C = np.zeros(shp + (12, 12), dtype=np.complex128)
    for mu in range(4):
        for nu in range(mu + 1, 4):
            F = field_strength(U, mu, nu)
            s = sigma(mu, nu)
            C += np.einsum("rs,...ab->...rasb", s, F).reshape(shp + (12, 12))
    return 1j * kappa * csw * C


# --------------------------------------------------------------------------
# The operator
# --------------------------------------------------------------------------
def apply_clover(C, psi):
    shp = psi.shape
    v = psi.reshape(shp[:4] + (12,))
    return np.einsum("...ij,...j->...i", C, v).reshape(shp)


def hopping(U, psi, bc_t, dagger=False):
    """H psi = sum_mu [(1 - g_mu) U_mu(x) psi(x+mu) + (1 + g_mu) U_mu(x-mu)^+ psi(x-mu)];
    the adjoint exchanges the two projectors."""
    out = np.zeros_like(psi)
    for mu in range(4):
        Umu = U[..., mu, :, :]
        fwd = colour_mul(Umu, spinor_fwd(psi, mu, bc_t))
        bwd = colour_mul_dag(link_at(Umu, {mu: -1}), spinor_bwd(psi, mu, bc_t))
        pm, pp = ID4 - GAMMA[mu], ID4 + GAMMA[mu]
        if dagger:
            pm, pp = pp, pm
        out += spin_mul(pm, fwd) + spin_mul(pp, bwd)
    return out


def apply_D(U, C, psi, kappa, bc_t=-1, dagger=False):
    """D psi (or D^+ psi) for one spinor field psi of shape (T, Z, Y, X, 4, 3).
    C is the clover field from ``clover_field`` (already scaled by kappa c_sw)."""
    Cd = _dag(C) if dagger else C
    return psi + apply_clover(Cd, psi) - kappa * hopping(U, psi, bc_t, dagger)


class Operator:
    """Bundle of (U, kappa, c_sw, bc_t) with its clover field; ``D(psi)``
    applies the operator to one field or a batch (leading axis)."""

    def __init__(self, U, kappa, csw, bc_t=-1):
        self.U = U
        self.kappa = float(kappa)
        self.csw = float(csw)
        self.bc_t = int(bc_t)
        self.C = clover_field(U, kappa, csw)
        self.dims = dims_of(U)

    def D(self, psi, dagger=False):
        if psi.ndim == 7:
            return np.stack([self.D(p, dagger) for p in psi])
        return apply_D(self.U, self.C, psi, self.kappa, self.bc_t, dagger)

    def Ddag(self, psi):
        return self.D(psi, dagger=True)


def gamma5(psi):
    return spin_mul(GAMMA5, psi)


def inner(a, b):
    """(a, b) = sum_x a(x)^+ b(x)."""
    return np.vdot(a.reshape(-1), b.reshape(-1))


def norm(a):
    return float(np.sqrt(np.real(inner(a, a))))
