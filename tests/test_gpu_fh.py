"""Differentiable nucleon correlator: the GPU adjoint gradients (through
torch.autograd and the C-ABI) against the oracle's forward-mode derivatives
(themselves pinned by finite differences), and a GPU central finite
difference in m0.  Tolerances: gradients 1e-7 relative (solves at 1e-12);
finite difference 1e-5 (h = 1e-4, second-order error)."""
import numpy as np
import pytest

from paper_1605_00564_gb300 import synth

pytestmark = pytest.mark.gpu


def test_fh_gradients_match_oracle():
    import torch
    from oracle.gradient import FHCorrelator
    from paper_1605_00564_gb300.qcd import Lattice, nucleon_fh
    dims = (8, 4, 4, 4)
    U = synth.gauge_field(dims, 0.3, 91)
    m0, csw, src = 0.2, 1.3, (1, 0, 0, 0)
    lat = Lattice(dims)
    lat.load_gauge(U, csw, 1.0 / (2 * m0 + 8), -1)
    lat.set_params(block=(4, 2, 2, 2), ncy=5, nmr=4, nkv=16, precision="f32", dfl=0)
    w = np.random.default_rng(12).standard_normal(dims[0])
    m = torch.tensor(m0, dtype=torch.float64, requires_grad=True)
    lam = torch.tensor(0.0, dtype=torch.float64, requires_grad=True)
    C = nucleon_fh(m, lam, lat, U, csw, src, 1e-12)
    L = (torch.from_numpy(w) * C[0, :, 0]).sum()
    L.backward()
    o = FHCorrelator(U, m0, csw, src)
    c_ref = o.correlator()
    assert np.abs(C.detach().numpy()[..., 0] + 1j * C.detach().numpy()[..., 1] - c_ref).max() < 1e-9 * np.abs(c_ref).max()
    dm, dl = o.derivatives()
    gm, gl = float(np.sum(w * dm[0].real)), float(np.sum(w * dl[0].real))
    assert abs(m.grad.item() - gm) < 1e-7 * abs(gm), (m.grad.item(), gm)
    assert abs(lam.grad.item() - gl) < 1e-7 * max(abs(gl), 1e-30), (lam.grad.item(), gl)
    # central finite difference in m0 on the GPU
    h = 1e-4
    Lp = float((torch.from_numpy(w) * nucleon_fh(m0 + h, 0.0, lat, U, csw, src, 1e-12)[0, :, 0]).sum())
    Lm = float((torch.from_numpy(w) * nucleon_fh(m0 - h, 0.0, lat, U, csw, src, 1e-12)[0, :, 0]).sum())
    assert abs((Lp - Lm) / (2 * h) - gm) < 1e-5 * abs(gm)
    lat.close()
