"""Pins of the oracle's three-point functions (oracle/threept.py).

The insertion of Gamma on the quark lines of flavour f, summed over every
operator time, is minus the derivative of the two-point function with
respect to a coupling theta that adds theta Gamma to that flavour's operator
(dS/dtheta = -S Gamma S, from the Dirac equation): central finite
differences of two-point functions from independent dense solves.  This
fixes the gamma structure of each insertion (A_3 = g3 g5, S = 1,
T_12 = sigma_12), the projectors, the flavour slots of the contraction and
the isovector sign; the per-time values follow from the definition.
"""
import numpy as np
import pytest

from oracle import threept
from oracle.dirac import Operator
from paper_1605_00564_gb300 import synth

DIMS = (4, 2, 2, 2)


@pytest.fixture(scope="module")
def setup():
    U = synth.gauge_field(DIMS, 0.5, 4242)
    op = Operator(U, 0.115, 1.3, -1)
    return op, threept.AllToAll(op)


@pytest.mark.parametrize("direction,t_sep", [(+1, 2), (-1, 3)])
def test_insertions_sum_to_minus_derivative(setup, direction, t_sep):
    op, a2a = setup
    src = (1, 1, 0, 1)
    c3, c2 = threept.three_point(op, src, t_sep, direction, a2a=a2a)
    h = 1e-4
    for k, (name, Gam, Pf, Pb) in enumerate(threept.INSERTIONS):
        P = Pf if direction > 0 else Pb

        def c2_at(th):
            return threept.two_point_flavoured(op, src, t_sep, direction, P, shift_u=(th, Gam), shift_d=(-th, Gam))
        deriv = (c2_at(h) - c2_at(-h)) / (2 * h)
        total = c3[k].sum()
        assert abs(total + deriv) < 1e-6 * max(abs(deriv), 1e-3), (name, total, -deriv)
        assert abs(total) > 1e-4, name                       # a non-trivial check


def test_flavours_separately(setup):
    """u and d insertions on their own (scalar), against the same identity
    with the coupling on one flavour only."""
    op, a2a = setup
    src = (0, 0, 1, 0)
    t_sep = 2
    P = threept.P_PLUS
    h = 1e-4
    cu = threept.two_point_flavoured
    du = (cu(op, src, t_sep, 1, P, shift_u=(h, np.eye(4))) - cu(op, src, t_sep, 1, P, shift_u=(-h, np.eye(4)))) / (2 * h)
    dd = (cu(op, src, t_sep, 1, P, shift_d=(h, np.eye(4))) - cu(op, src, t_sep, 1, P, shift_d=(-h, np.eye(4)))) / (2 * h)
    c3, _ = threept.three_point(op, src, t_sep, 1, a2a=a2a)
    # the isovector scalar is -(du - dd)
    assert abs(c3[1].sum() + (du - dd)) < 1e-6 * abs(du - dd)
    assert abs(du) > 1e-6 and abs(dd) > 1e-6                # both flavours contribute


def test_two_point_matches_nucleon_module(setup):
    """The ratios' denominator equals nucleon.two_point at the sink time."""
    from oracle import nucleon
    op, a2a = setup
    src = (1, 0, 0, 0)
    for direction, t_sep in ((1, 2), (-1, 2)):
        _, c2 = threept.three_point(op, src, t_sep, direction, a2a=a2a)
        prop = a2a.columns(threept.site_index(op.dims, src)).T.reshape((12,) + op.U.shape[:4] + (4, 3))
        ref = nucleon.two_point(prop, src[0])
        trel = (direction * t_sep) % op.dims[0]
        assert abs(c2 - ref[0 if direction > 0 else 1, trel]) < 1e-12 * abs(c2)


def test_smeared_source_and_sink(setup):
    """With Gaussian smearing at source and sink the insertion sum rule holds
    for the smeared correlators (the coupling acts between the smearings),
    and K = 1 (kappa_G = 0) reproduces the point correlators."""
    from oracle import smearing
    op, a2a = setup
    src = (1, 0, 1, 1)
    t_sep = 2
    Uape = smearing.ape_smear(op.U, 0.5, 2)
    K = smearing.timeslice_matrices(Uape, 0.3, 2)
    c3, c2 = threept.three_point(op, src, t_sep, 1, a2a=a2a, smear=(K,))
    p3, p2 = threept.three_point(op, src, t_sep, 1, a2a=a2a)
    assert abs(c2 - p2) > 1e-3 * abs(p2)                          # smearing changes the correlator
    K0 = smearing.timeslice_matrices(Uape, 0.0, 2)
    z3, z2 = threept.three_point(op, src, t_sep, 1, a2a=a2a, smear=(K0,))
    assert np.abs(z3 - p3).max() < 1e-12 * np.abs(p3).max() and abs(z2 - p2) < 1e-12 * abs(p2)
    # sum rule with smeared source and sink: -d/dtheta of the smeared two-point function
    from oracle.solve import dense_matrix
    M = dense_matrix(op)
    V = M.shape[0] // 12
    T = op.dims[0]
    L3 = V // T
    big = np.zeros((12 * V, 12 * V), dtype=complex)     # K on every time-slice, spin untouched
    for t in range(T):
        for al in range(4):
            idx = 12 * (t * L3 + np.arange(L3))[:, None] + 3 * al + np.arange(3)[None, :]
            idx = idx.reshape(-1)
            big[np.ix_(idx, idx)] = K[t]
    s0 = threept.site_index(op.dims, src)
    E = np.zeros((12 * V, 12), dtype=complex)
    E[12 * s0 + np.arange(12), np.arange(12)] = 1.0
    ts = (src[0] + t_sep) % T
    Gam = threept.INSERTIONS[1][1]
    P = threept.P_PLUS
    h = 1e-4

    def c2_at(th):
        shift = th * np.kron(np.eye(V), np.kron(Gam, np.eye(3)))
        Su = (big @ np.linalg.solve(M + shift, big @ E)).reshape(V, 12, 12)[ts * L3:(ts + 1) * L3]
        Sd = (big @ np.linalg.solve(M - shift, big @ E)).reshape(V, 12, 12)[ts * L3:(ts + 1) * L3]
        shp = (L3, 4, 3, 4, 3)
        return np.trace(P @ threept.trilinear(Su.reshape(shp), Sd.reshape(shp), Su.reshape(shp)).sum(axis=0))
    deriv = (c2_at(h) - c2_at(-h)) / (2 * h)
    assert abs(c3[1].sum() + deriv) < 1e-6 * abs(deriv)
    assert abs(c2 - c2_at(0.0)) < 1e-12 * abs(c2)
