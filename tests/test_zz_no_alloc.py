"""The allocation-free contraction entry point, qcd_nucleon_2pt_noalloc.

It exists for callers that cannot allocate device memory at the point of
the call (inside a stream capture, under their own device allocator or a
fixed arena).  The tests call it through the C-ABI:

* twice in a row on two different propagators, each result checked timeslice
  by timeslice against the oracle's contraction (oracle.nucleon.two_point)
  and against the context-based qcd_nucleon_2pt, with the tolerances of the
  contraction parity tests (FP64 1e-13, FP32 5e-6 of |C(t)| per timeslice);
  the two calls share the library's fixed scratch array, so the second must
  not see leftovers of the first;
* on lattices whose spatial volume has 32 as a factor (one full CTA of 32
  sites) and 8 as its largest power-of-two factor (6^3: CTAs of 8 sites,
  48 working threads in two warps);
* inside a CUDA-graph capture after a warm-up call, the graph replayed on a
  new propagator copied into the captured buffer.

This file is collected last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _per_timeslice_err(out, ref):
    return float((np.abs(out - ref) / np.abs(ref)).max())


def _random_prop(shape, rng):
    return rng.standard_normal(shape + (2,)) @ np.array([1, 1j])


@pytest.mark.parametrize("dims", [(16, 8, 8, 8), (8, 6, 6, 6)])
@pytest.mark.parametrize("prec,tol", [("f64", 1e-13), ("f32", 5e-6)])
def test_noalloc_matches_oracle(dims, prec, tol):
    import torch
    from oracle import nucleon
    from paper_1605_00564_gb300 import synth
    from paper_1605_00564_gb300.qcd import Lattice, nucleon_2pt_noalloc

    lat = Lattice(dims)
    lat.load_gauge(synth.unit_gauge(dims), 1.0, 0.12, -1)
    rng = np.random.default_rng(11)
    src = (5 % dims[0], 4 % dims[1], 0, 2)
    results = []
    for call in range(2):
        prop = _random_prop(lat.spinor_shape(12), rng)
        pd = torch.from_numpy(prop).cuda()
        ref = nucleon.two_point(prop, src[0])
        ctx = lat.nucleon_2pt(pd, src, precision=prec)
        corr = torch.full((2, dims[0], 2), float("nan"), dtype=torch.float64, device="cuda")
        nucleon_2pt_noalloc(dims, pd, src, corr, precision=prec)
        torch.cuda.synchronize()
        out = corr.cpu().numpy()
        out = out[..., 0] + 1j * out[..., 1]
        assert np.all(np.isfinite(out))
        assert _per_timeslice_err(out, ref) <= tol, (call, _per_timeslice_err(out, ref))
        assert _per_timeslice_err(out, ctx) <= tol, (call, _per_timeslice_err(out, ctx))
        results.append(out)
    assert np.abs(results[0] - results[1]).max() > 0      # two different propagators
    lat.close()


def test_noalloc_graph_capture_replay():
    """Warm-up call, then a second call captured into a CUDA graph on a side
    stream; replaying the graph after copying a new propagator into the
    captured input buffer gives that propagator's correlator."""
    import torch
    from oracle import nucleon
    from paper_1605_00564_gb300.qcd import nucleon_2pt_noalloc

    dims = (8, 6, 6, 6)
    rng = np.random.default_rng(12)
    shape = (12,) + (dims[0], dims[3], dims[2], dims[1], 4, 3)
    src = (3, 0, 2, 4)
    buf = torch.from_numpy(_random_prop(shape, rng)).cuda()
    corr = torch.zeros((2, dims[0], 2), dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        nucleon_2pt_noalloc(dims, buf, src, corr, precision="f64", stream=s)      # warm-up (device set-up)
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        nucleon_2pt_noalloc(dims, buf, src, corr, precision="f64", stream=s)
    for k in range(2):
        prop = _random_prop(shape, rng)
        buf.copy_(torch.from_numpy(prop))
        corr.fill_(float("nan"))
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        out = corr.cpu().numpy()
        out = out[..., 0] + 1j * out[..., 1]
        ref = nucleon.two_point(prop, src[0])
        assert _per_timeslice_err(out, ref) <= 1e-13, (k, _per_timeslice_err(out, ref))


def test_noalloc_rejects_oversize():
    """Lattices beyond the fixed scratch are refused before any launch."""
    import torch
    from paper_1605_00564_gb300.qcd import QcdError, nucleon_2pt_noalloc
    dummy = torch.zeros(2, dtype=torch.complex128, device="cuda")
    corr = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(QcdError) as e:
        nucleon_2pt_noalloc((128, 64, 64, 64), dummy, (0, 0, 0, 0), corr)   # 33.5 M sites
    assert e.value.status == 1
    with pytest.raises(QcdError) as e:
        nucleon_2pt_noalloc((2048, 2048, 2048, 2048), dummy, (0, 0, 0, 0), corr)   # volume >= 2^31
    assert e.value.status == 1
