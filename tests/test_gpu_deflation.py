"""Local deflation on the GPU vs the oracle, through the C-ABI.

Tolerances:
  subspace, no inverse iteration     1e-5 per block-normalised field (FP32 Gram-Schmidt)
  subspace after 2 SAP rounds        2e-3 (FP32 SAP + Gram-Schmidt vs FP64)
  little Dirac operator              2e-5 of max |A| (FP32 GEMM over a block)
  little solve (m = 32 steps)        residual <= 1e-3 against the dense A
  deflated exact solve               oracle residual <= 1.1e-10
"""
import numpy as np
import pytest

from gpu_util import make_lattice, rel, to_dev, to_host
from paper_1605_00564_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def small():
    return make_lattice("small_8c16")


def _oracle_dfl(op, block, phi=None):
    from oracle.deflation import Deflation
    d = Deflation(op, block)
    if phi is not None:
        d.phi = phi
    return d


def _dense_from_parts(A, dims, block):
    """Dense little matrix from the [b][9][k][l] parts (neighbour parts summed)."""
    nbd = [dims[m] // block[m] for m in range(4)]
    nb, ns = A.shape[0], A.shape[2]
    D = np.zeros((nb * ns, nb * ns), dtype=complex)
    for b in range(nb):
        bx = b % nbd[1]; r = b // nbd[1]; by = r % nbd[2]; r //= nbd[2]; bz = r % nbd[3]; bt = r // nbd[3]
        bc = [bt, bx, by, bz]
        D[b * ns:(b + 1) * ns, b * ns:(b + 1) * ns] += A[b, 0]
        for mu in range(4):
            for sgn, part in ((1, 1 + 2 * mu), (-1, 2 + 2 * mu)):
                cc = list(bc)
                cc[mu] = (cc[mu] + sgn) % nbd[mu]
                bp = ((cc[0] * nbd[3] + cc[3]) * nbd[2] + cc[2]) * nbd[1] + cc[1]
                D[b * ns:(b + 1) * ns, bp * ns:(bp + 1) * ns] += A[b, part]
    return D


@pytest.mark.parametrize("block", [(4, 4, 4, 4), (4, 2, 4, 2)])
def test_subspace_gram_schmidt(small, block):
    lat, op, _ = small
    lat.set_params(block=block, ncy=4, nmr=4, sap_half=0)
    init = synth.random_spinor(lat.dims, 51, nrhs=6)
    lat.deflation_setup(to_dev(init), 0)
    phi = to_host(lat.deflation_fields())
    ref = _oracle_dfl(op, block).block_gram_schmidt(init)
    assert rel(phi, ref) < 1e-5


def test_subspace_inverse_iteration(small):
    from oracle.sap import SAP
    lat, op, _ = small
    block = (4, 4, 4, 4)
    lat.set_params(block=block, ncy=4, nmr=4, sap_half=0)
    init = synth.random_spinor(lat.dims, 52, nrhs=4)
    lat.deflation_setup(to_dev(init), 2)
    phi = to_host(lat.deflation_fields())
    ref = _oracle_dfl(op, block).subspace(init, SAP(op, block, ncy=4, nmr=4), 2)
    assert rel(phi, ref) < 2e-3


@pytest.mark.parametrize("dims,block", [(None, (4, 4, 4, 4)), ((16, 8, 8, 8), (2, 2, 2, 4))])
def test_little_dirac_operator(small, dims, block):
    if dims is None:
        lat, op, _ = small
    else:
        lat, op, _ = make_lattice(dims, eps=0.3, csw=1.5, kappa=0.127, seed=53)
    lat.set_params(block=block, ncy=4, nmr=4, sap_half=0)
    init = synth.random_spinor(lat.dims, 54, nrhs=4)
    lat.deflation_setup(to_dev(init), 1)
    phi = to_host(lat.deflation_fields())
    d = _oracle_dfl(op, block, phi)
    Aref = d.little_dirac()
    A = _dense_from_parts(lat.deflation_little_matrix(), lat.dims, block)
    assert np.abs(A - Aref).max() < 2e-5 * np.abs(Aref).max()
    # the little operator on a random little vector (mode 0) agrees with the dense one
    v = np.random.default_rng(5).standard_normal((2, d.nb, 4)) * (1 + 0.5j)
    out = lat.deflation_little(v, 0)
    ref = np.stack([(Aref @ x.reshape(-1)).reshape(x.shape) for x in v])
    assert rel(out, ref) < 2e-5


def test_little_solve(small):
    lat, op, _ = small
    block = (4, 4, 4, 4)
    lat.set_params(block=block, ncy=4, nmr=4, sap_half=0)
    init = synth.random_spinor(lat.dims, 55, nrhs=6)
    lat.deflation_setup(to_dev(init), 2)
    A = _dense_from_parts(lat.deflation_little_matrix(), lat.dims, block)
    v = np.random.default_rng(6).standard_normal((3, A.shape[0] // 6, 6)) * (1 - 0.3j)
    x = lat.deflation_little(v, 1, m=32)
    for i in range(3):
        r = np.linalg.norm(A @ x[i].reshape(-1) - v[i].reshape(-1)) / np.linalg.norm(v[i])
        assert r < 1e-3


@pytest.mark.parametrize("half,gen", [(0, 0), (1, 0), (1, 4)])
def test_deflated_solve(small, half, gen):
    """gen > 0: subspace rounds after the first use gen iterations of the deflated solver."""
    lat, op, _ = small
    lat.set_params(block=(4, 4, 4, 4), ncy=5, nmr=4, nkv=16, precision="f32", sap_half=half, dfl=0,
                   dfl_gen_iters=gen)
    src = synth.point_sources(lat.dims, (0, 0, 0, 0))
    eta = to_dev(src)
    _, st0 = lat.solve(eta, 1e-10)
    lat.deflation_setup(to_dev(synth.random_spinor(lat.dims, 56, nrhs=8)), 3)
    phi = to_host(lat.deflation_fields())
    from oracle.deflation import Deflation
    d = Deflation(op, (4, 4, 4, 4))
    for k in range(8):               # block orthonormal whatever the generation scheme
        for l in range(8):
            g = d.block_inner(phi[k], phi[l])
            assert np.abs(g - (1.0 if k == l else 0.0)).max() < 1e-5
    lat.set_params(dfl=1, dfl_little_iters=16)
    psi, st = lat.solve(eta, 1e-10)
    psi = to_host(psi)
    for r in range(12):
        res = np.linalg.norm(src[r] - op.D(psi[r])) / np.linalg.norm(src[r])
        assert st[r]["status"] == "QCD_OK" and res <= 1.1e-10, (r, res)
    assert sum(s["outer_iters"] for s in st) < sum(s["outer_iters"] for s in st0)
