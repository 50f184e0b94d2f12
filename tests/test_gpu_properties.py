"""Properties of the CUDA path that hold at any size, and its failure paths.

* batched = single: a right-hand side solved inside a batch gives the same bits as
  solved alone (every kernel and reduction works per RHS in a fixed order);
* translation covariance of the sloppy correlator (the paper's covariance test,
  Sec. 3.1): a source shifted by a translation that maps each SAP domain onto
  itself (an even number of blocks), on the correspondingly shifted gauge field,
  gives the same correlator up to rounding, while a shift that exchanges Omega and
  Omega* or does not map blocks onto blocks changes the sloppy solution at the
  level of the solver tolerance;
* failure paths (made on the host): zero source, NaN source, max_outer = 1,
  invalid arguments.
"""
import numpy as np
import pytest

from gpu_util import make_lattice, record, to_dev, to_host
from paper_1605_00564_gb300 import synth
from paper_1605_00564_gb300.qcd import QcdError

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def small():
    return make_lattice("small_8c16")


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_dirac_batched_equals_single(small, prec):
    """One RHS and a batch of five launch different grids; each RHS of the
    batch gives the same bits as alone."""
    lat, _, _ = small
    psi = synth.random_spinor(lat.dims, 72, nrhs=5)
    for dagger in (False, True):
        out_b = to_host(lat.apply_dirac(to_dev(psi), dagger=dagger, precision=prec))
        for r in (0, 4):
            out_s = to_host(lat.apply_dirac(to_dev(psi[r:r + 1]), dagger=dagger, precision=prec))[0]
            assert np.array_equal(out_s, out_b[r])


def test_batched_equals_single(small):
    lat, op, _ = small
    lat.set_params(block=(4, 4, 4, 4), ncy=5, nmr=4, nkv=16, precision="f32", sap_half=1, dfl=0)
    eta = synth.random_spinor(lat.dims, 71, nrhs=3)
    psi_b, st_b = lat.solve(to_dev(eta), 1e-8)
    psi_b = to_host(psi_b)
    for r in range(3):
        psi_s, st_s = lat.solve(to_dev(eta[r:r + 1]), 1e-8)
        assert st_s[0]["outer_iters"] == st_b[r]["outer_iters"]
        assert np.array_equal(to_host(psi_s)[0], psi_b[r])


def _sloppy_corr(U, src, tol=1e-3):
    from paper_1605_00564_gb300.qcd import Lattice
    cfg = synth.CONFIGS["small_8c16"]
    lat = Lattice(cfg["dims"])
    lat.load_gauge(U, cfg["csw"], cfg["kappa"], -1)
    lat.set_params(block=(4, 4, 4, 4), ncy=5, nmr=4, nkv=16, precision="f32", sap_half=1, dfl=0)
    psi, _ = lat.solve(to_dev(synth.point_sources(cfg["dims"], src)), tol)
    c = lat.nucleon_2pt(psi, src, precision="f64")
    lat.close()
    return c


def test_translation_covariance_block_preserving():
    cfg = synth.CONFIGS["small_8c16"]
    U = synth.gauge_field(cfg["dims"], cfg["eps"], cfg["seed"])
    c0 = _sloppy_corr(U, (0, 0, 0, 0))

    def delta(g):
        Ug = np.roll(U, shift=(g[0], g[3], g[2], g[1]), axis=(0, 1, 2, 3))
        cg = _sloppy_corr(Ug, g)
        return (np.abs(cg[0] - c0[0]) / np.abs(c0[0]))[:8].max()

    # shift by (2, 1, 0, 1) blocks: Omega -> Omega, Omega* -> Omega*
    # measured: 0 (the shifted problem gives the same bits at t < 8)
    d_even = record("covariance_d_even", delta((8, 4, 0, 4)))
    assert d_even < 1e-12, d_even
    # shift by (1, 1, 0, 1) blocks exchanges Omega and Omega*: M_SAP changes
    d_odd = record("covariance_d_odd", delta((4, 4, 0, 4)))
    # shift by one site: the blocks are not mapped onto blocks
    d_site = record("covariance_d_site", delta((1, 0, 0, 0)))
    # measured 9.3e-3 and 2.7e-3: the sloppy solution differs at the level of its tolerance
    assert d_odd > 1e-5 and d_site > 1e-5, (d_even, d_odd, d_site)


def test_failure_paths(small):
    lat, op, _ = small
    lat.set_params(block=(4, 4, 4, 4), ncy=5, nmr=4, nkv=16, precision="f32", sap_half=1, dfl=0, max_outer=2000)
    # zero source: psi = 0, converged
    psi, st = lat.solve(to_dev(np.zeros(lat.spinor_shape(1), dtype=complex)), 1e-8)
    assert st[0]["status"] == "QCD_OK" and np.abs(to_host(psi)).max() == 0
    # NaN in the source: non-finite status for that RHS only
    eta = synth.random_spinor(lat.dims, 72, nrhs=2)
    eta[1, 0, 0, 0, 0, 0, 0] = np.nan
    psi, st = lat.solve(to_dev(eta), 1e-8, check=False)
    assert st[0]["status"] == "QCD_OK" and st[1]["status"] == "QCD_ERR_NONFINITE"
    with pytest.raises(QcdError) as e:
        lat.solve(to_dev(eta), 1e-8)
    assert e.value.status == 6
    # max_outer = 1: not converged, best iterate returned (residual below 1)
    lat.set_params(max_outer=1)
    psi, st = lat.solve(to_dev(eta[:1]), 1e-12, allow_not_converged=True)
    assert st[0]["status"] == "QCD_ERR_NOT_CONVERGED" and 0 < st[0]["true_rel_residual"] < 1
    lat.set_params(max_outer=2000)
    # argument errors, reported before any launch
    with pytest.raises(QcdError) as e:
        lat.set_params(block=(3, 4, 4, 4))
    assert e.value.status == 1
    with pytest.raises(QcdError):
        lat.solve(to_dev(eta[:1]), 2.0)
    with pytest.raises(QcdError):
        lat.ama_nucleon_2pt([(1, 0, 0, 0)], 1, 1e-3, 1e-10)   # source not block-aligned
    with pytest.raises(QcdError):
        lat.ama_nucleon_2pt([(0, 0, 0, 0), (4, 0, 0, 0)], 1, 1e-3, 1e-10)   # odd block shift
