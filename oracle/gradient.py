"""Oracle: derivatives of the nucleon two-point function with respect to the
bare quark mass and a Feynman-Hellmann coupling (FP64, numpy).

Test infrastructure only (see ``oracle/__init__``).

Wilson normalisation: D_w = (4 + m0) - H/2 + c_sw (i/4) sum sigma F, so the
kappa-normalised operator of ``dirac`` is D = 2 kappa D_w with
kappa = 1 / (2 m0 + 8), and the point-to-all propagator in Wilson
normalisation is S = D_w^-1 = 2 kappa D^-1.

The axial coupling lambda adds lambda * g3 g5 at every site to the u-quark
operator and -lambda * g3 g5 to the d-quark operator (isovector zero-momentum
insertion of A_3, the current of R_A in Sec. 2.3).  dS/dtheta = -S (dD/dtheta) S
with dD_w/dm0 = 1 and dD_w/dlambda = +-g3 g5.

The correlator with distinct u and d propagators is the trilinear form
F(S_a, S_b, S_c): S_a is the propagator of the u quark of the diquark, S_b
that of the d quark, S_c that of the third quark (the two Wick terms differ
in which u-bar each u meets).  Derivatives are taken by differentiating each
slot in turn with dS from extra solves (forward mode, from the definition).
"""
from __future__ import annotations

import itertools

import numpy as np

from .dirac import GAMMA, GAMMA5, Operator, spin_mul
from .nucleon import EPS, G_SINK, G_SRC, P_MINUS, P_PLUS, _perm_sign, propagator_matrix
from .solve import gcr

G3G5 = GAMMA[3] @ GAMMA5


def kappa_of(m0):
    return 1.0 / (2.0 * m0 + 8.0)


def trilinear(Sa, Sb, Sc):
    """G[..., alpha, alpha'] = sum of the Wick terms with the diquark u quark
    propagating by Sa, the d quark by Sb and the third quark by Sc; the second
    term exchanges the u-bar partners (sign from the fermion permutation)."""
    quarks = [("u", "a", "B"), ("d", "b", "C"), ("u", "c", "A")]
    antiq = [("d", "e", "F"), ("u", "d", "E"), ("u", "f", "D")]
    slot = {0: Sa, 1: Sb, 2: Sc}
    total = 0.0
    for perm in itertools.permutations(range(3)):
        if any(quarks[i][0] != antiq[perm[i]][0] for i in range(3)):
            continue
        order = []
        for i in range(3):
            order += [i, 3 + perm[i]]
        sign = _perm_sign(order)
        terms, ops = [], []
        for i in range(3):
            q, aq = quarks[i], antiq[perm[i]]
            terms.append("..." + q[2] + q[1] + aq[2] + aq[1])
            ops.append(slot[i])
        spec = "abc,def,BC,FE," + ",".join(terms) + "->...AD"
        total = total + sign * np.einsum(spec, EPS, EPS, G_SINK, G_SRC, *ops, optimize=True)
    return total


def project_time(G, t0, bc_t=-1):
    """C[parity, t_rel] from G[T, Z, Y, X, 4, 4] as in nucleon.two_point."""
    Gt = G.sum(axis=(1, 2, 3))
    T = Gt.shape[0]
    out = np.zeros((2, T), dtype=np.complex128)
    for t in range(T):
        trel = (t - t0) % T
        sgn = bc_t ** 3 if t < t0 else 1.0
        out[0, trel] = sgn * np.trace(P_PLUS @ Gt[t])
        out[1, trel] = sgn * np.trace(P_MINUS @ Gt[t])
    return out


class FHCorrelator:
    """C(t; m0, lambda) and its derivatives at the given point, for a point source."""

    def __init__(self, U, m0, csw, src, bc_t=-1, tol=1e-13):
        self.U, self.m0, self.csw, self.src, self.bc_t, self.tol = U, m0, csw, src, bc_t, tol
        self.kappa = kappa_of(m0)
        self.op = Operator(U, self.kappa, csw, bc_t)
        from paper_1605_00564_gb300 import synth
        self.eta = synth.point_sources(self.op.dims, src)

    def _Dinv_wilson(self, rhs, lam_sign=0.0, lam=0.0):
        """Solve D_w x = rhs column by column (x = 2 kappa D^-1 rhs) with the
        optional lambda term: (D + 2 kappa lam_sign lam g3g5) x' = rhs, x = 2 kappa x'."""
        k2 = 2.0 * self.kappa
        if lam == 0.0:
            op = self.op
        else:
            base = self.op

            class _Op:
                dims = base.dims

                def D(_, psi, dagger=False):
                    return base.D(psi, dagger) + k2 * lam_sign * lam * spin_mul(G3G5, psi)
            op = _Op()
        return np.stack([k2 * gcr(op, r, tol=self.tol)[0] for r in rhs])

    def correlator(self, lam=0.0):
        Su = propagator_matrix(self._Dinv_wilson(self.eta, +1.0, lam))
        Sd = propagator_matrix(self._Dinv_wilson(self.eta, -1.0, lam)) if lam != 0.0 else Su
        return project_time(trilinear(Su, Sd, Su), self.src[0], self.bc_t)

    def derivatives(self):
        """(dC/dm0, dC/dlambda) at lambda = 0 from dS = -S (dD_w) S."""
        prop = self._Dinv_wilson(self.eta)                      # S columns, Wilson normalisation
        S = propagator_matrix(prop)
        dS_m = propagator_matrix(-self._Dinv_wilson(prop))      # -S (1) S
        g = np.stack([spin_mul(G3G5, p) for p in prop])
        dS_l = propagator_matrix(-self._Dinv_wilson(g))         # -S (g3g5) S  (u; d has the opposite sign)
        t0 = self.src[0]
        dm = project_time(trilinear(dS_m, S, S) + trilinear(S, dS_m, S) + trilinear(S, S, dS_m), t0, self.bc_t)
        dl = project_time(trilinear(dS_l, S, S) - trilinear(S, dS_l, S) + trilinear(S, S, dS_l), t0, self.bc_t)
        return dm, dl
