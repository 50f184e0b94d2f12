"""The differentiable correlator at the size of the differentiable-solve
workload: 24^3x48, kappa 0.1355 (m0 = 1 / (2 kappa) - 4), c_sw 1.9, a point
source, SAP 4^4 blocks.  The oracle cannot solve at this size, so:

* dL/dm0 from the adjoint solves is checked against a central finite
  difference of the GPU correlator (h = 1e-4).  The weights sit on the first
  time-slices, where the third derivative that sets the O(h^2) error is small;
  the solves stop at 1e-11, which puts the finite difference's rounding near
  1e-7 relative.  Bound 1e-5, as on the small lattice.
* dL/dlambda has no finite-difference counterpart on the GPU (the operator
  carries no lambda term); it is checked through translation covariance: the
  same source shifted by a translation that maps the SAP domains onto
  themselves, on the shifted gauge field, gives the same gradients up to the
  order of the lattice-wide sums (bound 1e-9 relative).  The small-lattice
  test pins both gradients against the oracle."""
import numpy as np
import pytest

from paper_1605_00564_gb300 import synth

pytestmark = pytest.mark.gpu

DIMS = (48, 24, 24, 24)
KAPPA, CSW = 0.1355, 1.9
TOL = 1e-11


def _grads(lat, U, src, w):
    import torch
    from paper_1605_00564_gb300.qcd import nucleon_fh
    m0 = 1.0 / (2.0 * KAPPA) - 4.0
    m = torch.tensor(m0, dtype=torch.float64, requires_grad=True)
    lam = torch.tensor(0.0, dtype=torch.float64, requires_grad=True)
    C = nucleon_fh(m, lam, lat, U, CSW, src, TOL)
    L = (torch.from_numpy(w) * C[0, :, 0]).sum()
    L.backward()
    return float(L.detach()), m.grad.item(), lam.grad.item()


def test_fh_gradients_24c48():
    import torch
    from paper_1605_00564_gb300.qcd import Lattice, nucleon_fh
    cfg = synth.CONFIGS["batch2_24c48"]
    U = synth.gauge_field(DIMS, cfg["eps"], cfg["seed"])
    lat = Lattice(DIMS, stream=torch.cuda.Stream())
    lat.load_gauge(U, CSW, KAPPA, -1)
    lat.set_params(block=(4, 4, 4, 4), ncy=5, nmr=4, nkv=16, precision="f32", sap_half=1, dfl=0, max_outer=4000)
    w = np.zeros(DIMS[0])
    w[1:7] = np.random.default_rng(31).standard_normal(6)
    src = (0, 0, 0, 0)
    L0, gm, gl = _grads(lat, U, src, w)
    assert np.isfinite(gm) and np.isfinite(gl) and abs(gm) > 0 and abs(gl) > 0
    # central finite difference in m0
    h = 1e-4
    m0 = 1.0 / (2.0 * KAPPA) - 4.0
    Lp = float((torch.from_numpy(w) * nucleon_fh(m0 + h, 0.0, lat, U, CSW, src, TOL)[0, :, 0]).sum())
    Lm = float((torch.from_numpy(w) * nucleon_fh(m0 - h, 0.0, lat, U, CSW, src, TOL)[0, :, 0]).sum())
    fd = (Lp - Lm) / (2 * h)
    assert abs(fd - gm) < 1e-5 * abs(gm), (fd, gm)
    # translation by (2, 1, 0, 1) blocks: Omega -> Omega, Omega* -> Omega*
    g = (8, 4, 0, 4)
    Ug = np.roll(U, shift=(g[0], g[3], g[2], g[1]), axis=(0, 1, 2, 3))
    L1, gm1, gl1 = _grads(lat, Ug, g, w)
    assert abs(L1 - L0) < 1e-9 * abs(L0), (L1, L0)
    assert abs(gm1 - gm) < 1e-9 * abs(gm), (gm1, gm)
    assert abs(gl1 - gl) < 1e-9 * abs(gl), (gl1, gl)
    lat.close()
