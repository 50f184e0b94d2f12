"""The allocation-free contraction entry point, qcd_nucleon_2pt_noalloc.

It exists for callers that cannot allocate device memory at the point of
the call (inside a stream capture, under their own device allocator or a
fixed arena).  The test calls it twice in a row through the C-ABI on the
same propagator and checks both results against qcd_nucleon_2pt, with the
tolerances of the contraction parity tests (FP64 1e-12, FP32 2e-5 of
max |C|).  The two calls share the library's fixed scratch array; the
second must not see leftovers of the first.  This file is collected last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 2e-5)])
def test_noalloc_matches_contraction(prec, tol):
    import torch
    from paper_1605_00564_gb300 import synth
    from paper_1605_00564_gb300.qcd import Lattice, nucleon_2pt_noalloc

    dims = (16, 8, 8, 8)
    lat = Lattice(dims)
    lat.load_gauge(synth.unit_gauge(dims), 1.0, 0.12, -1)
    rng = np.random.default_rng(11)
    src = (5, 4, 0, 4)
    results = []
    for call in range(2):
        prop = rng.standard_normal(lat.spinor_shape(12) + (2,)) @ np.array([1, 1j])
        pd = torch.from_numpy(prop).cuda()
        ref = lat.nucleon_2pt(pd, src, precision=prec)
        corr = torch.full((2, dims[0], 2), float("nan"), dtype=torch.float64, device="cuda")
        nucleon_2pt_noalloc(dims, pd, src, corr, precision=prec)
        torch.cuda.synchronize()
        out = corr.cpu().numpy()
        out = out[..., 0] + 1j * out[..., 1]
        assert np.all(np.isfinite(out))
        assert np.abs(out - ref).max() <= tol * np.abs(ref).max(), (call, np.abs(out - ref).max())
        results.append(out)
    assert np.abs(results[0] - results[1]).max() > 0      # two different propagators
    lat.close()
