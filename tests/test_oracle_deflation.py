"""Pins of the oracle's local deflation (Sec. 2.2): the projector identities
P_L D = D P_R and Phi^+ P_L = 0, block orthonormality of the deflation
fields, the nearest-neighbour sparsity of the little Dirac operator, the
exactness of the low-mode solve on D span(Phi), and that deflation improves
the preconditioned operator."""
import numpy as np
import pytest

from oracle.deflation import Deflation
from oracle.dirac import Operator, norm
from oracle.sap import SAP
from paper_1605_00564_gb300 import synth


@pytest.fixture(scope="module")
def dfl():
    dims = (8, 4, 4, 4)
    op = Operator(synth.gauge_field(dims, 0.3, 41), kappa=0.128, csw=1.5)
    block = (4, 2, 2, 2)
    sap = SAP(op, block, ncy=4, nmr=4)
    d = Deflation(op, block)
    init = synth.random_spinor(dims, 42, nrhs=4)
    d.subspace(init, sap, n_inv=2)
    d.little_dirac()
    return d, sap


def test_block_orthonormal(dfl):
    d, _ = dfl
    ns = d.phi.shape[0]
    for k in range(ns):
        for l in range(ns):
            g = d.block_inner(d.phi[k], d.phi[l])
            assert np.abs(g - (1.0 if k == l else 0.0)).max() < 1e-12


def test_projector_identities(dfl):
    d, _ = dfl
    v = synth.random_spinor(d.dims, 43)
    # P_L D = D P_R
    assert norm(d.P_L(d.op.D(v)) - d.op.D(d.P_R(v))) < 1e-11 * norm(v)
    # Phi^+ P_L = 0 and P_R Phi = 0
    assert np.abs(d.project(d.P_L(v))).max() < 1e-11 * norm(v)
    c = np.random.default_rng(1).standard_normal((d.nb, d.phi.shape[0])) + 0j
    assert norm(d.P_R(d.prolong(c))) < 1e-11 * norm(d.prolong(c))


def test_little_dirac_structure(dfl):
    """A couples a block only to itself and its 8 nearest neighbours."""
    d, _ = dfl
    ns = d.phi.shape[0]
    nbl = [d.dims[m] // d.block[m] for m in range(4)]     # blocks per direction (t, x, y, z)

    def coords(b):
        nx, ny, nz = nbl[1], nbl[2], nbl[3]
        bx, r = b % nx, b // nx
        by, r = r % ny, r // ny
        bz, bt = r % nz, r // nz
        return np.array([bt, bx, by, bz])

    for b in range(d.nb):
        for bp in range(d.nb):
            diff = (coords(b) - coords(bp)) % np.array(nbl)
            steps = [min(x, n - x) for x, n in zip(diff, nbl)]
            blk = d.A[b * ns:(b + 1) * ns, bp * ns:(bp + 1) * ns]
            if sum(steps) > 1:
                assert np.abs(blk).max() == 0.0


def test_low_mode_solve_exact_on_D_span(dfl):
    """eta = D Phi c is solved by the low-mode part alone (eq. deflsoln with chi = 0)."""
    d, _ = dfl
    c = np.random.default_rng(2).standard_normal((d.nb, d.phi.shape[0])) * (1 + 1j)
    x = d.prolong(c)
    eta = d.op.D(x)
    assert norm(d.low_mode(eta) - x) < 1e-10 * norm(x)
    assert norm(d.P_L(eta)) < 1e-10 * norm(eta)


def test_deflation_improves_preconditioner(dfl):
    """One application of the deflated preconditioner leaves a smaller residual
    than SAP alone for a source dominated by the deflation subspace."""
    d, sap = dfl
    rng = np.random.default_rng(3)
    eta = d.op.D(d.prolong(rng.standard_normal((d.nb, d.phi.shape[0])) + 0j)) + 1e-2 * synth.random_spinor(d.dims, 44)
    r_sap = norm(eta - d.op.D(sap.apply(eta)))
    r_dfl = norm(eta - d.op.D(d.precondition(eta, sap)))
    assert r_dfl < r_sap
