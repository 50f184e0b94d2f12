"""Helpers shared by the GPU tests: move seeded inputs to the device and
bring results back for comparison with the oracle."""
import numpy as np

from paper_1605_00564_gb300 import synth


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def to_host(t):
    return t.detach().cpu().numpy()


def rel(a, b):
    return float(np.linalg.norm((a - b).reshape(-1)) / np.linalg.norm(b.reshape(-1)))


def make_lattice(name_or_dims, eps=None, csw=None, kappa=None, seed=None, bc_t=-1):
    """(Lattice, oracle Operator, U) for a named workload or explicit parameters."""
    from oracle.dirac import Operator
    from paper_1605_00564_gb300.qcd import Lattice
    if isinstance(name_or_dims, str):
        cfg = synth.CONFIGS[name_or_dims]
        dims, eps, csw, kappa, seed = cfg["dims"], cfg["eps"], cfg["csw"], cfg["kappa"], cfg["seed"]
    else:
        dims = name_or_dims
    U = synth.gauge_field(dims, eps, seed)
    lat = Lattice(dims)
    lat.load_gauge(U, csw, kappa, bc_t)
    return lat, Operator(U, kappa, csw, bc_t), U
