"""Helpers shared by the GPU tests: move seeded inputs to the device, bring
results back, and compare them with the oracle element by element.

``elem_err(a, b)`` is the largest per-element error
``|a_i - b_i| / max(|b_i|, rms(b))``: relative to the element itself, with
the field's root-mean-square magnitude as the floor for elements near zero
(an absolute error of the size of the rounding of the typical element).
Each parity test states its bound next to the assertion.  ``face_mask``
selects the sites on a block face (the sites that receive the boundary term
of the Schwarz procedure), so a defect confined to the faces is checked on
its own.  With the environment variable QCD_PARITY_LOG set to a file path,
every measured error is appended there as a JSON line (the values behind the
bounds).
"""
import json
import os

import numpy as np

from paper_1605_00564_gb300 import synth


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def to_host(t):
    return t.detach().cpu().numpy()


def rel(a, b):
    """Norm-wise relative error ||a - b|| / ||b|| (the form of the solver tolerances)."""
    return float(np.linalg.norm((a - b).reshape(-1)) / np.linalg.norm(b.reshape(-1)))


def elem_err(a, b):
    """max_i |a_i - b_i| / max(|b_i|, rms(b))."""
    a = np.asarray(a).reshape(-1)
    b = np.asarray(b).reshape(-1)
    floor = float(np.sqrt(np.mean(np.abs(b) ** 2)))
    if floor == 0.0:
        return float(np.abs(a).max()) if a.size else 0.0
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), floor)))


def face_mask(dims, block):
    """Boolean (T, Z, Y, X): True on sites with a block-local coordinate 0 or
    b_mu - 1 in some direction mu (dims and block as (T, X, Y, Z))."""
    T, X, Y, Z = dims
    t, z, y, x = np.indices((T, Z, Y, X))
    m = np.zeros((T, Z, Y, X), dtype=bool)
    for c, b in ((t, block[0]), (x, block[1]), (y, block[2]), (z, block[3])):
        lc = c % b
        m |= (lc == 0) | (lc == b - 1)
    return m


def elem_err_faces(a, b, dims, block):
    """elem_err restricted to the block-face sites (floor: rms over all of b).
    a, b: (..., T, Z, Y, X, 4, 3)."""
    m = face_mask(dims, block)
    floor = float(np.sqrt(np.mean(np.abs(b) ** 2)))
    af, bf = np.asarray(a)[..., m, :, :], np.asarray(b)[..., m, :, :]
    return float(np.max(np.abs(af - bf) / np.maximum(np.abs(bf), floor)))


def timeslice_err(c, ref):
    """max_t |C(t) - C_ref(t)| / |C_ref(t)| over both parities: each timeslice
    relative to itself, so late timeslices count as much as early ones."""
    c, ref = np.asarray(c), np.asarray(ref)
    return float(np.max(np.abs(c - ref) / np.abs(ref)))


def record(name, value):
    """Append a measured error to the file named by QCD_PARITY_LOG (if set)."""
    path = os.environ.get("QCD_PARITY_LOG")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps({"test": name, "value": float(value)}) + "\n")
    return value


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


def _oracle_gcr_worker(args):
    from oracle.dirac import Operator
    from oracle.solve import gcr
    U, kappa, csw, bc_t, eta, tol = args
    return gcr(Operator(U, kappa, csw, bc_t), eta, tol=tol)[0]


def oracle_solve_many(U, kappa, csw, bc_t, etas, tol=1e-13):
    """The oracle's GCR solutions of several sources, one process per source
    (a 'spawn' pool, safe after CUDA has been initialised in this process)."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    n = len(etas)
    workers = max(1, min(n, os.cpu_count() or 1))
    # one thread per worker process: the workers are the parallelism
    keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in keys}
    os.environ.update({k: "1" for k in keys})
    try:
        with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
            return np.stack(list(ex.map(_oracle_gcr_worker, [(U, kappa, csw, bc_t, e, tol) for e in etas])))
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
