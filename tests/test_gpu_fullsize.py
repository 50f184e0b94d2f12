"""Parity at the benchmark's size and launch configuration: 32^3x64, kappa 0.1300,
c_sw 1.9, SAP 4^4 blocks, n_cy 5, n_mr 4, FP16 block copies, nkv 16.  The oracle
applies its operator to whole fields (a few seconds each) and contracts sampled
timeslices.  Bounds as in test_gpu_parity (element-wise operator, per-timeslice
contraction)."""
import numpy as np
import pytest

from gpu_util import elem_err, record, timeslice_err, to_dev, to_host
from paper_1605_00564_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def big():
    from oracle.dirac import Operator
    from paper_1605_00564_gb300.qcd import Lattice
    cfg = synth.CONFIGS["prod_32c64_k130"]
    U = synth.gauge_field(cfg["dims"], cfg["eps"], cfg["seed"])
    lat = Lattice(cfg["dims"])
    lat.load_gauge(U, cfg["csw"], cfg["kappa"], -1)
    lat.set_params(block=(4, 4, 4, 4), ncy=5, nmr=4, nkv=16, precision="f32", sap_half=1, dfl=0,
                   restart_drop=1e-5, max_outer=4000)
    yield lat, Operator(U, cfg["kappa"], cfg["csw"], -1)
    lat.close()


def test_dirac_fullsize(big):
    """One RHS (lexicographic runs) and two RHS (z-slab traversal order)."""
    lat, op = big
    psi = synth.random_spinor(lat.dims, 81, nrhs=2)
    ref = np.stack([op.D(p) for p in psi])
    edge = [0, lat.T - 1]
    for prec, tol in (("f64", 1e-13), ("f32", 5e-6)):
        for n in (1, 2):
            out = to_host(lat.apply_dirac(to_dev(psi[:n]), precision=prec))
            assert record("dirac_fullsize_%s_n%d" % (prec, n), elem_err(out, ref[:n])) < tol
            assert elem_err(out[:, edge], ref[:n, edge]) < tol


@pytest.mark.parametrize("tol,basis_half", [(1e-10, 0), (1e-3, 0), (1e-3, 1)])
def test_solve_fullsize(big, tol, basis_half):
    """A point source at full size: far from it the SAP's block residuals and the
    Krylov images reach FP32 denormals, which the MR step length and the FP16
    encoding of chi_k must survive."""
    lat, op = big
    src = synth.point_source(lat.dims, (8, 16, 0, 0), 2, 1)
    lat.set_params(basis_half=basis_half)
    try:
        psi, st = lat.solve(to_dev(src[None]), tol)
    finally:
        lat.set_params(basis_half=0)
    res = np.linalg.norm(src - op.D(to_host(psi)[0])) / np.linalg.norm(src)
    assert st[0]["status"] == "QCD_OK" and res <= tol * 1.1, res


def test_contraction_fullsize_sampled(big):
    from oracle import nucleon
    lat, op = big
    rng = np.random.default_rng(9)
    prop = (rng.standard_normal(lat.spinor_shape(12) + (2,)) @ np.array([1, 1j])).astype(np.complex128)
    src = (8, 16, 0, 0)
    out = lat.nucleon_2pt(to_dev(prop), src, precision="f64")
    for t in (8, 9, 40, 3):                            # sampled timeslices, incl. one wrapped past T
        S = nucleon.propagator_matrix(prop[:, t:t + 1])
        G = nucleon.wick_contract(S).sum(axis=(1, 2, 3))[0]
        trel = (t - src[0]) % lat.T
        sgn = -1.0 if t < src[0] else 1.0
        ref = sgn * np.array([np.trace(nucleon.P_PLUS @ G), np.trace(nucleon.P_MINUS @ G)])
        assert record("contract_fullsize_t%d" % t, timeslice_err(out[:, trel], ref)) <= 1e-12
