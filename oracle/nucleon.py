"""Oracle: nucleon two-point function and the AMA estimator (FP64, numpy).

Test infrastructure only (see ``oracle/__init__``).

Interpolator (eq. Nop):  N_alpha = eps^{abc} (u^a^T G d^b) u^c_alpha with
G = C gamma_5 and C = gamma_0 gamma_2 (satisfies C g_mu C^-1 = -g_mu^T in the
chiral basis used here).  The conjugate follows from N-bar = N^+ gamma_0:
N-bar_alpha' = eps^{a'b'c'} (d-bar^b' G' u-bar^a'^T) u-bar^c'_alpha' with
G' = gamma_0 G^+ gamma_0^T.

The correlator G_{alpha alpha'}(x) = <N_alpha(x) N-bar_alpha'(x0)> is the sum
of all Wick contractions <q q-bar> -> S = D^-1 with the sign of the fermion
permutation; ``wick_contract`` enumerates them programmatically (two terms
for u = d, which differ in which u-bar each u meets).  ``matrix_form`` is
the same sum written by hand as spin-matrix products, an independent check.

Projections (Sec. 2.3): P+- = (1 +- gamma_0)/2; C_+-(t) = sum_x tr[P+- G(x,t)]
at zero momentum.  Times are re-referenced to the source, t -> (t - t0) mod T,
and a sink time that wrapped past T picks up (-1)^3 from the three
antiperiodic quark propagators.  The overall sign is fixed so that the
free-field forward correlator C_+(t) is positive.

AMA (eqs. caa1, caa2):  O_AMA = O_rest + (1/N_G) sum_g O_appx^g,
O_rest = (1/N_org) sum_f [O^f - O_appx^f].
"""
from __future__ import annotations

import itertools

import numpy as np

from .dirac import GAMMA, GAMMA5

CHARGE_C = GAMMA[0] @ GAMMA[2]
G_SINK = CHARGE_C @ GAMMA5
G_SRC = GAMMA[0] @ G_SINK.conj().T @ GAMMA[0].T
P_PLUS = 0.5 * (np.eye(4) + GAMMA[0])
P_MINUS = 0.5 * (np.eye(4) - GAMMA[0])

EPS = np.zeros((3, 3, 3))
for _p in itertools.permutations(range(3)):
    EPS[_p] = np.linalg.det(np.eye(3)[list(_p)])

# overall sign of the correlator, fixed by free-field positivity of C_+
OVERALL_SIGN = 1.0


def propagator_matrix(prop):
    """prop[rhs = 3 alpha' + a', T, Z, Y, X, alpha, a] -> S[T, Z, Y, X, alpha, a, alpha', a']."""
    n = prop.shape[0]
    assert n == 12
    S = np.moveaxis(prop.reshape((4, 3) + prop.shape[1:]), (0, 1), (-2, -1))
    return S


def _perm_sign(order):
    inv = 0
    for i in range(len(order)):
        for j in range(i + 1, len(order)):
            inv += order[i] > order[j]
    return -1.0 if inv % 2 else 1.0


def wick_contract(S):
    """G[T,Z,Y,X, alpha, alpha'] by explicit enumeration of the Wick
    contractions of N_alpha(x) N-bar_alpha'(x0) with u = d (one propagator)."""
    # fields in operator order: sink  u(a,beta) d(b,gamma) u(c,alpha)
    #                          source d-bar(b',gamma') u-bar(a',beta') u-bar(c',alpha')
    quarks = [("u", "a", "B"), ("d", "b", "C"), ("u", "c", "A")]
    antiq = [("d", "e", "F"), ("u", "d", "E"), ("u", "f", "D")]   # b'->e,g'->F; a'->d,b'->E; c'->f,a'->D
    pos_q = [0, 1, 2]
    pos_aq = [3, 4, 5]
    total = 0.0
    for perm in itertools.permutations(range(3)):
        if any(quarks[i][0] != antiq[perm[i]][0] for i in range(3)):
            continue
        order = []
        for i in range(3):
            order += [pos_q[i], pos_aq[perm[i]]]
        sign = _perm_sign(order)
        # S index letters: site..., spin_sink, col_sink, spin_src, col_src
        terms = []
        for i in range(3):
            q, aq = quarks[i], antiq[perm[i]]
            terms.append("..." + q[2] + q[1] + aq[2] + aq[1])
        spec = "abc,def,BC,FE," + ",".join(terms) + "->...AD"
        total = total + sign * np.einsum(spec, EPS, EPS, G_SINK, G_SRC, S, S, S, optimize=True)
    return OVERALL_SIGN * total


def matrix_form(S):
    """The same correlator written as spin-matrix products:
    G = eps eps' { S^{cc'} tr[S^{aa'T} G S^{bb'} G'] - S^{ca'} G'^T S^{bb'T} G^T S^{ac'} }."""
    Sm = S  # [..., alpha, a, alpha', a']
    out = np.zeros(S.shape[:4] + (4, 4), dtype=np.complex128)
    for a, b, c in itertools.permutations(range(3)):
        e1 = EPS[a, b, c]
        for ap, bp, cp in itertools.permutations(range(3)):
            e = e1 * EPS[ap, bp, cp]
            Saa = Sm[..., :, a, :, ap]
            Sbb = Sm[..., :, b, :, bp]
            Scc = Sm[..., :, c, :, cp]
            Sca = Sm[..., :, c, :, ap]
            Sac = Sm[..., :, a, :, cp]
            tr = np.einsum("...ji,jk,...kl,li->...", Saa, G_SINK, Sbb, G_SRC)
            t1 = Scc * tr[..., None, None]
            t2 = Sca @ G_SRC.T @ np.swapaxes(Sbb, -1, -2) @ G_SINK.T @ Sac
            out += e * (t1 - t2)
    return OVERALL_SIGN * out


def two_point(prop, t0, bc_t=-1, contraction=wick_contract):
    """C[parity, t] (parity 0: P+, 1: P-) for times relative to the source
    time t0, from the 12-component point-source propagator ``prop``."""
    S = propagator_matrix(prop)
    G = contraction(S)
    Gt = G.sum(axis=(1, 2, 3))                      # zero momentum: sum over z, y, x
    T = Gt.shape[0]
    out = np.zeros((2, T), dtype=np.complex128)
    for t in range(T):
        trel = (t - t0) % T
        sgn = bc_t ** 3 if t < t0 else 1.0
        out[0, trel] = sgn * np.trace(P_PLUS @ Gt[t])
        out[1, trel] = sgn * np.trace(P_MINUS @ Gt[t])
    return out


def ama_combine(appx, exact, appx_at_exact):
    """O_AMA = (1/N_org) sum_f [O^f - O_appx^f] + (1/N_G) sum_g O_appx^g.

    appx: [N_G, ...] sloppy observables over the translations g;
    exact, appx_at_exact: [N_org, ...] exact and sloppy observables at the
    translations f used for the bias correction."""
    appx = np.asarray(appx)
    rest = np.mean(np.asarray(exact) - np.asarray(appx_at_exact), axis=0)
    return rest + np.mean(appx, axis=0)
