"""Smeared sources and sinks on the GPU against the oracle (oracle/smearing.py,
oracle/threept.py), through the C-ABI.

Bounds: APE links 1e-13 per entry (FP64, Newton polar iteration against the
SVD polar factor; measured 4.6e-15), Gaussian smearing 1e-13 element-wise
(FP64 stencil; measured 3.5e-15), smeared two- and three-point functions
from exact (1e-12) solves 1e-10 per time-slice relative to
max(|C(t)|, rms C) (measured 4.3e-12)."""
import numpy as np
import pytest

from gpu_util import elem_err, record, to_dev, to_host
from paper_1605_00564_gb300 import synth

pytestmark = pytest.mark.gpu

DIMS = (8, 4, 4, 4)
ALPHA, N_APE, KAPPA_G, N_GAUSS = 0.5, 3, 0.25, 4


@pytest.fixture(scope="module")
def setup():
    from oracle import smearing
    from oracle.dirac import Operator
    from paper_1605_00564_gb300.qcd import Lattice
    U = synth.gauge_field(DIMS, 0.4, 2718)
    kappa, csw = 0.12, 1.3
    lat = Lattice(DIMS)
    lat.load_gauge(U, csw, kappa, -1)
    lat.set_params(block=(4, 2, 2, 2), ncy=5, nmr=4, nkv=16, precision="f32", dfl=0)
    lat.smear_links(ALPHA, N_APE)
    yield lat, Operator(U, kappa, csw, -1), U, smearing.ape_smear(U, ALPHA, N_APE)
    lat.close()


def test_ape_links(setup):
    lat, op, U, Uape = setup
    got = to_host(lat.smeared_links())
    assert record("ape_links", float(np.abs(got - Uape).max())) < 1e-13
    assert np.abs(got[..., 0, :, :] - U[..., 0, :, :]).max() == 0.0


def test_gaussian_smearing(setup):
    from oracle import smearing
    lat, op, U, Uape = setup
    lat.set_smearing(KAPPA_G, N_GAUSS)
    psi = synth.random_spinor(DIMS, 5, nrhs=3)
    out = to_host(lat.smear_gaussian(to_dev(psi)))
    ref = np.stack([smearing.gaussian_smear(Uape, p, KAPPA_G, N_GAUSS) for p in psi])
    assert record("gaussian_smear", elem_err(out, ref)) < 1e-13


@pytest.mark.parametrize("t_sep,direction", [(3, 1), (3, -1)])
def test_smeared_two_and_three_point(setup, t_sep, direction):
    from oracle import smearing, threept
    lat, op, U, Uape = setup
    lat.set_smearing(KAPPA_G, N_GAUSS)
    src = (4, 2, 0, 2)
    try:
        r = lat.ama_nucleon([src], 1, sloppy_tol=1e-3, exact_tol=1e-12, t_sep=t_sep, direction=direction)
    finally:
        lat.set_smearing(0.0, 0)
    K = smearing.timeslice_matrices(Uape, KAPPA_G, N_GAUSS)
    ref3, ref2 = threept.three_point(op, src, t_sep, direction, a2a=threept.AllToAll(op), smear=(K,))
    c3, c2 = r["c3_all"][1], r["c2_all"][1]                      # the exact position
    for k, name in enumerate(("A3", "S", "T12")):
        floor = np.sqrt(np.mean(np.abs(ref3[k]) ** 2))
        e = float(np.max(np.abs(c3[k] - ref3[k]) / np.maximum(np.abs(ref3[k]), floor)))
        assert record("smeared_3pt_%s_d%d" % (name, direction), e) < 1e-10, (name, e)
    trel = (direction * t_sep) % DIMS[0]
    got2 = c2[0 if direction > 0 else 1, trel]
    assert record("smeared_2pt_d%d" % direction, abs(got2 - ref2) / abs(ref2)) < 1e-10
