"""Pins of the oracle's solvers and SAP: the solution of D psi = eta against a
library dense LU on a 2^4 lattice, and the SAP cycle / M_SAP polynomial
against the paper's matrix formulas built from dense block inverses."""
import numpy as np
import pytest

from oracle.dirac import Operator, norm
from oracle import sap as osap
from oracle.solve import cgne, dense_matrix, dense_solve, gcr, true_residual
from paper_1605_00564_gb300 import synth


@pytest.fixture(scope="module")
def op2():
    dims = (2, 2, 2, 2)
    return Operator(synth.gauge_field(dims, 0.5, 21), kappa=0.125, csw=1.9)


def test_dense_2x4_solution(op2):
    eta = synth.random_spinor(op2.dims, 3)
    x_dense = dense_solve(op2, eta)
    x_gcr, it, res = gcr(op2, eta, tol=1e-13)
    assert res <= 1e-13
    assert norm(x_gcr - x_dense) / norm(x_dense) < 1e-11
    x_cg, it, res = cgne(op2, eta, tol=1e-12)
    assert res <= 1e-12
    assert norm(x_cg - x_dense) / norm(x_dense) < 1e-10


def test_dense_matrix_adjoint(op2):
    M = dense_matrix(op2)
    Md = dense_matrix(op2, dagger=True)
    assert np.abs(Md - M.conj().T).max() < 1e-15
    g5 = np.kron(np.eye(16), np.kron(np.diag([1, 1, -1, -1]), np.eye(3)))
    assert np.abs(g5 @ M @ g5 - M.conj().T).max() < 1e-14


@pytest.fixture(scope="module")
def sap_exact():
    dims = (4, 4, 4, 4)
    op = Operator(synth.gauge_field(dims, 0.3, 5), kappa=0.125, csw=1.5)
    return osap.SAP(op, (2, 2, 2, 2), ncy=3, nmr=None)


def test_colouring():
    dims = (8, 4, 4, 4)
    m0 = osap.colour_mask(dims, (4, 2, 2, 2), 0)
    m1 = osap.colour_mask(dims, (4, 2, 2, 2), 1)
    assert m0.sum() == m1.sum() == m0.size // 2 and not np.any(m0 & m1)
    with pytest.raises(ValueError):
        osap.colour_mask((12, 4, 4, 4), (4, 2, 2, 2), 0)       # 3 blocks in t


def test_sap_cycle_equals_kernel(sap_exact):
    """One cycle from psi = 0 gives K eta with K = D_O^-1 + D_O*^-1 - D_O*^-1 D_dO* D_O^-1."""
    s = sap_exact
    eta = synth.random_spinor(s.dims, 8)
    psi, rho = s.cycle(np.zeros_like(eta), eta.copy())
    K = s.kernel_matrix()
    ref = (K @ eta.reshape(-1)).reshape(eta.shape)
    assert norm(psi - ref) / norm(ref) < 1e-12
    assert norm(rho - (eta - s.op.D(psi))) / norm(eta) < 1e-13
    # Omega* blocks are solved exactly in the last half-cycle: residual vanishes there
    assert np.abs(rho[s.masks[1]]).max() < 1e-12


def test_msap_polynomial(sap_exact):
    """n_cy cycles from zero give M_SAP = K sum_{nu<n_cy} (1 - D K)^nu."""
    s = sap_exact
    eta = synth.random_spinor(s.dims, 9)
    ref = (s.msap_matrix() @ eta.reshape(-1)).reshape(eta.shape)
    out = s.apply(eta)
    assert norm(out - ref) / norm(ref) < 1e-11
    # the preconditioner is a contraction of the residual here
    assert norm(eta - s.op.D(out)) < 0.2 * norm(eta)


def test_mr_converges_to_exact_block_solve(sap_exact):
    s = sap_exact
    eta = synth.random_spinor(s.dims, 10)
    exact = s.block_solve(0, eta)
    x, r = osap.mr_block_solve(s.op, s.masks[0], s.bidx, s.nblk, eta, 150)
    assert norm(x - exact) / norm(exact) < 1e-9
    # block residual is what is left of rho on the block
    m = s.masks[0]
    assert norm(r - (eta * m[..., None, None] - osap.D_colour(s.op, m, x))) < 1e-12 * norm(eta)


def test_mr_residual_monotone_per_block():
    dims = (8, 4, 4, 4)
    op = Operator(synth.gauge_field(dims, 0.3, 6), kappa=0.13, csw=1.0)
    blk = (4, 2, 2, 2)
    m = osap.colour_mask(dims, blk, 1)
    bidx = osap.block_index(dims, blk)
    nb = int(bidx.max()) + 1
    eta = synth.random_spinor(dims, 12)
    prev = None
    for n in range(0, 6):
        _, r = osap.mr_block_solve(op, m, bidx, nb, eta, n)
        per = np.bincount(bidx.reshape(-1), weights=np.sum(np.abs(r) ** 2, axis=(-2, -1)).reshape(-1), minlength=nb)
        if prev is not None:
            assert np.all(per <= prev * (1 + 1e-13))
        prev = per


def test_mr_sap_is_good_preconditioner():
    dims = (8, 4, 4, 4)
    op = Operator(synth.gauge_field(dims, 0.3, 7), kappa=0.13, csw=1.0)
    s = osap.SAP(op, (4, 2, 2, 2), ncy=5, nmr=4)
    eta = synth.random_spinor(dims, 13)
    psi = s.apply(eta)
    assert true_residual(op, psi, eta) < 0.5
