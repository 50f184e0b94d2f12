"""Oracle: nucleon three-point functions with the isovector insertions of the
axial, scalar and tensor charges (Sec. 2.3, eqs. R_A, R_S, R_T), FP64 numpy.

Test infrastructure only (see ``oracle/__init__``).

The three-point function with the sink at time t_s, the operator at time t
and the point source at x0 (zero momentum at sink and operator):

    C3_O(t, t_s) = sum_{x, y}  tr[ P < N(x, t_s) O(y, t) N-bar(x0) > ],
    O = u-bar Gamma u - d-bar Gamma d,

Gamma = g3 g5 (A_3, with P = P53+ = P+ g5 g3), 1 (S, with P = P+) or
sigma_12 (T_12, with P = P53+).  With u = d degenerate only the connected
Wick contractions remain for the isovector combination: every propagator of
flavour f from the source to the sink is replaced in turn by the propagator
through the operator,

    S(x, x0)  ->  K(x) = sum_{y at t} S(x, y) Gamma S(y, x0),

so with the two-point function's trilinear form F(S_a, S_b, S_c) (u quark of
the diquark, d quark, third u quark; ``gradient.trilinear``)

    C3_u = F(K, S, S) + F(S, S, K),   C3_d = F(S, K, S),   C3 = C3_u - C3_d.

``three_point`` evaluates this definition literally from the all-to-all
propagator S(x, y) of a tiny lattice (a dense inverse): no sequential source,
no gamma_5 trick.  Normalisation: S = D^-1 of the kappa-normalised operator of
``dirac`` (the three-point function of Wilson-normalised propagators is
(2 kappa)^4 times this, the two-point function (2 kappa)^3 times
``nucleon.two_point``).  Backward-propagating nucleon: sink at t0 - t_s with
P- and P53- = P- g5 g3 (the paper averages the two directions).  Times are
re-referenced to the source exactly as for the two-point function
(``nucleon.two_point``): t_rel = (t - t0) mod T, and a sink whose absolute
time is earlier than the source's (reached forward from t0 only across the
time boundary) multiplies the result by bc_t^3, so that C3 / C2 pairs
values of one convention.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from .dirac import GAMMA, GAMMA5, sigma
from .gradient import trilinear
from .nucleon import P_MINUS, P_PLUS
from .solve import dense_matrix

G3G5 = GAMMA[3] @ GAMMA5
SIGMA12 = sigma(1, 2)
ID4 = np.eye(4, dtype=np.complex128)

# (name, Gamma, projector of the forward nucleon, projector of the backward nucleon)
INSERTIONS = (
    ("A3", G3G5, P_PLUS @ GAMMA5 @ GAMMA[3], P_MINUS @ GAMMA5 @ GAMMA[3]),
    ("S", ID4, P_PLUS, P_MINUS),
    ("T12", SIGMA12, P_PLUS @ GAMMA5 @ GAMMA[3], P_MINUS @ GAMMA5 @ GAMMA[3]),
)


def sink_time(T, t0, t_sep, direction):
    """Absolute sink time and whether the boundary sign applies (the sink's
    absolute time is earlier than the source's, as in nucleon.two_point)."""
    ts = (t0 + direction * t_sep) % T
    return ts, int(ts < t0)


class AllToAll:
    """The all-to-all propagator S(x, y) = D^-1 of a tiny lattice (LU of the
    dense operator), with sites in the canonical order and spinor index
    3 spin + colour."""

    def __init__(self, op):
        self.op = op
        self.dims = op.dims
        self.shape = op.U.shape[:4]
        self.V = int(np.prod(self.shape))
        self.lu = scipy.linalg.lu_factor(dense_matrix(op))

    def columns(self, site):
        """S(., site) as a 12V x 12 matrix (the 12 point sources at site)."""
        n = 12 * self.V
        E = np.zeros((n, 12), dtype=np.complex128)
        E[12 * site + np.arange(12), np.arange(12)] = 1.0
        return scipy.linalg.lu_solve(self.lu, E)

    def rows(self, sites):
        """S(x, .) for the given sites: (len(sites), 12, 12V), from D^T y = e_x."""
        n = 12 * self.V
        idx = (12 * np.asarray(sites)[:, None] + np.arange(12)[None, :]).reshape(-1)
        E = np.zeros((n, idx.size), dtype=np.complex128)
        E[idx, np.arange(idx.size)] = 1.0
        R = scipy.linalg.lu_solve(self.lu, E, trans=1).T          # rows of D^-1
        return R.reshape(len(sites), 12, n)


def site_index(dims, x):
    """Canonical site index of x = (t, x, y, z), dims = (T, X, Y, Z)."""
    T, X, Y, Z = dims
    t, xx, y, z = x
    return ((t * Z + z) * Y + y) * X + xx


def _smear_sink_side(Kt, A):
    """Apply a time-slice smearing matrix Kt [3 L3, 3 L3] (site, colour) to
    the sink index of A [L3, 12, n] (rows: site of the time-slice, spin
    colour); spin untouched."""
    L3, _, n = A.shape
    B = A.reshape(L3, 4, 3, n).transpose(1, 0, 2, 3).reshape(4, 3 * L3, n)
    B = np.einsum("ij,sjn->sin", Kt, B)
    return B.reshape(4, L3, 3, n).transpose(1, 0, 2, 3).reshape(L3, 12, n)


def three_point(op, src, t_sep, direction=+1, bc_t=-1, a2a=None, smear=None):
    """C3[insertion, t_rel] for the insertions of ``INSERTIONS`` (isovector
    u - d), sink at t0 + direction * t_sep.  Returns (C3 (3, T) complex,
    the two-point function tr[P+- G] at the sink: the ratios' denominator).

    smear = (K, ) with K the per-time-slice Gaussian smearing matrices of
    ``smearing.timeslice_matrices``: smeared source and sink, i.e. every
    source-to-sink propagator is K S K and the propagator through the
    operator is (K S)(x, y) Gamma (S K)(y, x0)."""
    dims = op.dims
    T = dims[0]
    a2a = a2a or AllToAll(op)
    L3 = a2a.V // T
    t0 = src[0]
    ts, wraps = sink_time(T, t0, t_sep, direction)
    sign = float(bc_t) ** 3 if wraps else 1.0
    s0 = site_index(dims, src)
    if smear is None:
        S0 = a2a.columns(s0)                               # (12V, 12): S(y, x0)
    else:
        # the 12 smeared point sources K delta_{x0}: on the source time-slice only
        K = smear[0]
        E = np.zeros((12 * a2a.V, 12), dtype=np.complex128)
        loc = s0 - t0 * L3
        for al in range(4):
            for a in range(3):
                col = K[t0][:, 3 * loc + a].reshape(L3, 3)             # (site, colour) of the time-slice
                for z in range(L3):
                    E[12 * (t0 * L3 + z) + 3 * al + np.arange(3), 3 * al + a] = col[z]
        S0 = scipy.linalg.lu_solve(a2a.lu, E)              # (S K)(y, x0)
    sink_sites = np.arange(ts * L3, (ts + 1) * L3)
    Srow = a2a.rows(sink_sites)                            # (L3, 12, 12V): S(x, y)
    S0s = S0.reshape(a2a.V, 12, 12)[sink_sites]            # (S K)(x, x0) at the sink
    if smear is not None:
        Srow = _smear_sink_side(smear[0][ts], Srow)        # (K S)(x, y)
        S0s = _smear_sink_side(smear[0][ts], S0s)          # (K S K)(x, x0)

    def to_mat(block):                                     # (n, 12, 12) -> (n, 4, 3, 4, 3)
        return block.reshape(block.shape[0], 4, 3, 4, 3)

    S_sink = to_mat(S0s)
    out = np.zeros((len(INSERTIONS), T), dtype=np.complex128)
    G2 = trilinear(S_sink, S_sink, S_sink).sum(axis=0)
    c2 = sign * np.trace((P_PLUS if direction > 0 else P_MINUS) @ G2)
    for k, (name, Gam, Pf, Pb) in enumerate(INSERTIONS):
        P = Pf if direction > 0 else Pb
        GS = np.kron(Gam, np.eye(3)) @ S0.reshape(a2a.V, 12, 12)     # (Gamma S)(y, x0) per site y
        for t in range(T):
            ys = np.arange(t * L3, (t + 1) * L3)
            # K(x) = sum_{y at t} S(x, y) Gamma S(y, x0)
            cols = (12 * ys[:, None] + np.arange(12)[None, :]).reshape(-1)
            K = np.einsum("xik,kj->xij", Srow[:, :, cols], GS[ys].reshape(-1, 12))
            K = to_mat(K)
            Gu = trilinear(K, S_sink, S_sink) + trilinear(S_sink, S_sink, K)
            Gd = trilinear(S_sink, K, S_sink)
            out[k, (t - t0) % T] = sign * np.trace(P @ (Gu - Gd).sum(axis=0))
    return out, c2


def two_point_flavoured(op, src, t_sep, direction, P, shift_u=None, shift_d=None, bc_t=-1):
    """tr[P G] at the sink for u and d propagators of modified operators
    D + theta_f Gamma_f at every site (shift_f = (theta_f, Gamma_f) or None),
    each solved from the dense matrix: the insertions summed over all times
    are -d/dtheta of this two-point function."""
    dims = op.dims
    T = dims[0]
    ts, wraps = sink_time(T, src[0], t_sep, direction)
    sign = float(bc_t) ** 3 if wraps else 1.0
    M = dense_matrix(op)
    V = M.shape[0] // 12
    L3 = V // T
    s0 = site_index(dims, src)
    E = np.zeros((12 * V, 12), dtype=np.complex128)
    E[12 * s0 + np.arange(12), np.arange(12)] = 1.0

    def prop(shift):
        A = M.copy()
        if shift is not None:
            coupling, Gam = shift
            A = A + coupling * np.kron(np.eye(V), np.kron(Gam, np.eye(3)))
        S = np.linalg.solve(A, E).reshape(V, 12, 12)[ts * L3:(ts + 1) * L3]
        return S.reshape(L3, 4, 3, 4, 3)

    Su, Sd = prop(shift_u), prop(shift_d)
    G = trilinear(Su, Sd, Su).sum(axis=0)
    return sign * np.trace(P @ G)
