"""Pins of the oracle's nucleon contraction and AMA estimator."""
import numpy as np

from oracle import nucleon
from oracle.dirac import GAMMA, Operator
from oracle.solve import gcr
from paper_1605_00564_gb300 import synth


def test_charge_conjugation():
    C = nucleon.CHARGE_C
    for mu in range(4):
        assert np.allclose(C @ GAMMA[mu] @ np.linalg.inv(C), -GAMMA[mu].T)
    assert np.allclose(nucleon.G_SINK, -nucleon.G_SINK.T)      # C g5 antisymmetric


def test_two_contraction_forms_agree_on_any_propagator():
    rng = np.random.default_rng(4)
    S = rng.standard_normal((2, 1, 2, 1, 4, 3, 4, 3)) + 1j * rng.standard_normal((2, 1, 2, 1, 4, 3, 4, 3))
    a = nucleon.wick_contract(S)
    b = nucleon.matrix_form(S)
    assert np.abs(a - b).max() < 1e-12 * np.abs(a).max()


def test_colour_singlet_closed_form():
    """For S = delta^{aa'} M with a fixed spin matrix M the colour sums are
    eps eps' delta delta delta = 6 and eps^{abc} eps^{cba} = -6, so
    G = 6 [M tr(M^T G M G') + M G'^T M^T G^T M]."""
    rng = np.random.default_rng(5)
    M = rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4))
    S = np.einsum("ij,ab->iajb", M, np.eye(3))[None, None, None, None]
    G = nucleon.wick_contract(S)[0, 0, 0, 0]
    Gs, Gp = nucleon.G_SINK, nucleon.G_SRC
    ref = 6 * (M * np.trace(M.T @ Gs @ M @ Gp) + M @ Gp.T @ M.T @ Gs.T @ M)
    assert np.abs(G - ref).max() < 1e-12 * np.abs(ref).max()


def test_free_field_correlator_positive_and_decaying():
    dims = (8, 4, 4, 4)
    op = Operator(synth.unit_gauge(dims), 0.12, 1.0)
    src = (2, 0, 0, 0)
    prop = np.stack([gcr(op, s, tol=1e-12)[0] for s in synth.point_sources(dims, src)])
    c = nucleon.two_point(prop, src[0])
    assert np.abs(c.imag).max() < 1e-12 * np.abs(c.real).max()
    fwd = c[0].real[: dims[0] // 2 + 1]
    assert np.all(fwd > 0) and np.all(np.diff(fwd) < 0)
    # the backward nucleon appears with the opposite parity projection
    bwd = -c[1].real[::-1][: dims[0] // 2]
    assert np.all(bwd[:-1] > 0)


def test_translation_covariance_exact_solves():
    """A translated source on the translated gauge field gives the same
    correlator (delta_c = 0 for exact solves)."""
    dims = (8, 4, 4, 4)
    U = synth.gauge_field(dims, 0.3, 31)
    g = (4, 2, 0, 2)
    Ush = np.roll(U, shift=(g[0], g[3], g[2], g[1]), axis=(0, 1, 2, 3))
    c = []
    for Uf, src in ((U, (0, 0, 0, 0)), (Ush, g)):
        op = Operator(Uf, 0.12, 1.0)
        prop = np.stack([gcr(op, s, tol=1e-13)[0] for s in synth.point_sources(dims, src)])
        c.append(nucleon.two_point(prop, src[0]))
    # antiperiodic time: shifting by 4 in t changes the wrapped-segment signs consistently
    assert np.abs(c[0] - c[1]).max() < 1e-9 * np.abs(c[0]).max()


def test_ama_algebra():
    rng = np.random.default_rng(6)
    appx = rng.standard_normal((8, 2, 16))
    exact = rng.standard_normal((1, 2, 16))
    # sloppy == exact: AMA reduces to the plain average over translations
    assert np.allclose(nucleon.ama_combine(appx, appx[:1], appx[:1]), appx.mean(0))
    # bias correction with N_org = 2
    out = nucleon.ama_combine(appx, np.stack([exact[0], exact[0] + 1]), appx[:2])
    ref = appx.mean(0) + 0.5 * ((exact[0] - appx[0]) + (exact[0] + 1 - appx[1]))
    assert np.allclose(out, ref)
