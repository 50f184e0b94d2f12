"""Three-point functions on the GPU (sequential propagators through the
sink) against the oracle's literal definition (dense all-to-all propagator,
oracle/threept.py), per operator time and insertion, through the C-ABI.

Bound: |C3(t) - C3_oracle(t)| <= 1e-10 max(|C3_oracle(t)|, rms_t C3_oracle)
for solves to 1e-12 (the forward propagator and the 24 sequential ones; the
error of a solution is about cond(D) times its residual; measured 1.6e-12)."""
import numpy as np
import pytest

from gpu_util import record, to_dev, to_host
from paper_1605_00564_gb300 import synth

pytestmark = pytest.mark.gpu

DIMS = (8, 4, 4, 4)


@pytest.fixture(scope="module")
def setup():
    from oracle import threept
    from oracle.dirac import Operator
    from paper_1605_00564_gb300.qcd import Lattice
    U = synth.gauge_field(DIMS, 0.4, 31337)
    kappa, csw = 0.12, 1.3
    op = Operator(U, kappa, csw, -1)
    lat = Lattice(DIMS)
    lat.load_gauge(U, csw, kappa, -1)
    lat.set_params(block=(4, 2, 2, 2), ncy=5, nmr=4, nkv=16, precision="f32", dfl=0)
    yield lat, op, threept.AllToAll(op)
    lat.close()


def _err(c, ref):
    floor = np.sqrt(np.mean(np.abs(ref) ** 2))
    return float(np.max(np.abs(c - ref) / np.maximum(np.abs(ref), floor)))


@pytest.mark.parametrize("src,t_sep,direction", [((1, 1, 2, 3), 3, 1), ((6, 0, 1, 1), 4, 1), ((2, 3, 0, 0), 3, -1)])
def test_three_point_matches_oracle(setup, src, t_sep, direction):
    from oracle import threept
    lat, op, a2a = setup
    eta = to_dev(synth.point_sources(DIMS, src))
    prop, st = lat.solve(eta, 1e-12)
    c3, st3 = lat.nucleon_3pt(prop, src, t_sep, direction, tol=1e-12)
    assert all(s["status"] == "QCD_OK" for s in st3)
    ref, c2 = threept.three_point(op, src, t_sep, direction, a2a=a2a)
    for k, name in enumerate(("A3", "S", "T12")):
        e = record("threept_%s_d%d_ts%d" % (name, direction, t_sep), _err(c3[k], ref[k]))
        assert e < 1e-10, (name, e)
    # the ratios' denominator from the library's two-point function
    c2_gpu = lat.nucleon_2pt(prop, src, precision="f64")[0 if direction > 0 else 1, (direction * t_sep) % DIMS[0]]
    assert abs(c2_gpu - c2) < 1e-9 * abs(c2)


def test_three_point_argument_errors(setup):
    from paper_1605_00564_gb300.qcd import QcdError
    lat, op, _ = setup
    prop = to_dev(np.zeros((12,) + synth.lattice_shape(DIMS) + (4, 3), dtype=complex))
    for kw in (dict(t_sep=0, direction=1), dict(t_sep=DIMS[0], direction=1), dict(t_sep=2, direction=0)):
        with pytest.raises(QcdError) as e:
            lat.nucleon_3pt(prop, (0, 0, 0, 0), **kw)
        assert e.value.status == 1
