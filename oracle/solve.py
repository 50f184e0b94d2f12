"""Oracle: plain solvers for D psi = eta (FP64, numpy).

Test infrastructure only (see ``oracle/__init__``).

The method (SAP-preconditioned, deflated GCR, Sec. 2.2) reaches the solution
of the Dirac equation D psi = eta to a tolerance faster; the solution itself
has a plain definition, which these unpreconditioned solvers compute:

* ``gcr``   - restarted generalised conjugate residual on D psi = eta;
* ``cgne``  - conjugate gradient on D^+ D psi = D^+ eta;
* ``dense_matrix`` / ``dense_solve`` - the operator as an explicit matrix
  (tiny lattices only) and a library LU solve.

The tolerance is relative: ||eta - D psi|| / ||eta||.
"""
from __future__ import annotations

import numpy as np

from .dirac import inner, norm


def true_residual(op, psi, eta):
    """||eta - D psi|| / ||eta|| in FP64."""
    return norm(eta - op.D(psi)) / norm(eta)


def gcr(op, eta, tol=1e-13, nkv=24, max_iter=20000, psi0=None):
    """Restarted GCR for D psi = eta.  Returns (psi, iterations, rel_residual).

    Within a cycle the search directions p_k have images q_k = D p_k made
    orthonormal by Gram-Schmidt; psi and the residual are updated along each.
    The residual is recomputed from the definition at every restart."""
    psi = np.zeros_like(eta) if psi0 is None else psi0.copy()
    eta_n = norm(eta)
    r = eta - op.D(psi)
    it = 0
    while it < max_iter:
        ps, qs = [], []
        for _ in range(nkv):
            p = r.copy()
            q = op.D(p)
            for pj, qj in zip(ps, qs):
                c = inner(qj, q)
                q = q - c * qj
                p = p - c * pj
            nq = norm(q)
            p, q = p / nq, q / nq
            ps.append(p)
            qs.append(q)
            a = inner(q, r)
            psi = psi + a * p
            r = r - a * q
            it += 1
            if norm(r) <= tol * eta_n or it >= max_iter:
                break
        r = eta - op.D(psi)
        if norm(r) <= tol * eta_n:
            break
    return psi, it, norm(r) / eta_n


def cgne(op, eta, tol=1e-13, max_iter=50000, psi0=None):
    """CG on the normal equations D^+ D psi = D^+ eta, stopped on the residual
    of the original system.  Returns (psi, iterations, rel_residual)."""
    psi = np.zeros_like(eta) if psi0 is None else psi0.copy()
    eta_n = norm(eta)
    r = op.Ddag(eta - op.D(psi))
    p = r.copy()
    rr = np.real(inner(r, r))
    it = 0
    while it < max_iter:
        Ap = op.D(p)
        alpha = rr / np.real(inner(Ap, Ap))
        psi = psi + alpha * p
        r = r - alpha * op.Ddag(Ap)
        rr_new = np.real(inner(r, r))
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
        if it % 10 == 0 and true_residual(op, psi, eta) <= tol:
            break
    return psi, it, true_residual(op, psi, eta)


def dense_matrix(op, dagger=False):
    """The operator as a (12 V) x (12 V) matrix, column j = D e_j."""
    shp = op.U.shape[:4] + (4, 3)
    n = int(np.prod(shp))
    M = np.empty((n, n), dtype=np.complex128)
    e = np.zeros(n, dtype=np.complex128)
    for j in range(n):
        e[:] = 0
        e[j] = 1
        M[:, j] = op.D(e.reshape(shp), dagger).reshape(-1)
    return M


def dense_solve(op, eta):
    M = dense_matrix(op)
    return np.linalg.solve(M, eta.reshape(-1)).reshape(eta.shape)
