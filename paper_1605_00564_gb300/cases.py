"""Small, self-contained runs of single kernels of the library, sized for
profiling one kernel at a time (a few hundred MB on the device, larger than
L2 where DRAM figures matter).

    python -m paper_1605_00564_gb300.cases dslash      # FP32 Dslash, 32^3x64, 1 RHS, 3 launches
    python -m paper_1605_00564_gb300.cases dslash12    # FP32 Dslash, 32^3x64, 12 RHS, 3 launches
    python -m paper_1605_00564_gb300.cases sap         # SAP sweeps, 16^3x32, 12 RHS, FP16 block copies
    python -m paper_1605_00564_gb300.cases sap32       # same with FP32 block copies
    python -m paper_1605_00564_gb300.cases sap_32c64   # SAP sweeps at 32^3x64, 12 RHS (DRAM counters only)
    python -m paper_1605_00564_gb300.cases deflation   # deflation setup + one deflated sloppy solve, 16^3x32
    python -m paper_1605_00564_gb300.cases contract    # nucleon contraction, 16^3x32
    python -m paper_1605_00564_gb300.cases gcr         # sloppy SAP-GCR solve, 16^3x32, 12 RHS, nkv 8, FP16 chi_k
    python -m paper_1605_00564_gb300.cases gcr32       # same with FP32 chi_k
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _lattice(dims, eps=0.15, csw=1.9, kappa=0.136, seed=7):
    from paper_1605_00564_gb300 import synth
    from paper_1605_00564_gb300.qcd import Lattice
    lat = Lattice(dims)
    lat.load_gauge(synth.gauge_field(dims, eps, seed), csw, kappa, -1)
    return lat


def dslash(nrhs=1):
    import torch
    lat = _lattice((64, 32, 32, 32))
    psi = torch.randn(lat.spinor_shape(nrhs), dtype=torch.complex128, device="cuda")
    for _ in range(3):
        lat.apply_dirac(psi, precision="f32")


def sap(half=1):
    import torch
    lat = _lattice((32, 16, 16, 16))
    psi = torch.randn(lat.spinor_shape(12), dtype=torch.complex128, device="cuda")
    lat.set_params(block=(4, 4, 4, 4), ncy=1, nmr=4, sap_half=half)
    for _ in range(2):
        lat.apply_sap(psi)


def sap_32c64():
    import torch
    lat = _lattice((64, 32, 32, 32), kappa=0.13)
    psi = torch.randn(lat.spinor_shape(12), dtype=torch.complex128, device="cuda")
    lat.set_params(block=(4, 4, 4, 4), ncy=1, nmr=4, sap_half=1)
    for _ in range(2):
        lat.apply_sap(psi)


def deflation():
    import torch
    from paper_1605_00564_gb300 import synth
    lat = _lattice((32, 16, 16, 16))
    lat.set_params(block=(4, 4, 4, 4), sap_half=1, dfl=1)
    lat.deflation_setup(torch.from_numpy(synth.random_spinor(lat.dims, 3, nrhs=12)).cuda(), 2)
    eta = torch.from_numpy(synth.point_sources(lat.dims, (0, 0, 0, 0))).cuda()
    lat.solve(eta, 1e-3)


def contract():
    import torch
    lat = _lattice((32, 16, 16, 16))
    prop = torch.randn(lat.spinor_shape(12), dtype=torch.complex128, device="cuda")
    for prec in ("f64", "f32"):
        lat.nucleon_2pt(prop, (0, 0, 0, 0), precision=prec)


def gcr(basis_half=1):
    import torch
    from paper_1605_00564_gb300 import synth
    lat = _lattice((32, 16, 16, 16), kappa=0.13)
    lat.set_params(block=(4, 4, 4, 4), ncy=5, nmr=4, nkv=8, sap_half=1, dfl=0, basis_half=basis_half)
    eta = torch.from_numpy(synth.point_sources(lat.dims, (0, 0, 0, 0))).cuda()
    lat.solve(eta, 1e-3)


CASES = {"dslash": dslash, "dslash12": lambda: dslash(12), "sap": sap, "sap32": lambda: sap(0), "sap_32c64": sap_32c64,
         "deflation": deflation, "contract": contract, "gcr": gcr, "gcr32": lambda: gcr(0)}

if __name__ == "__main__":
    import torch
    from paper_1605_00564_gb300 import build
    build.build()
    CASES[sys.argv[1]]()
    torch.cuda.synchronize()
    print("ok", sys.argv[1])
