"""Thin Python binding of the C-ABI in include/qcd.h (ctypes).

Argument marshalling only: every step of the computation runs in the CUDA
library ``libqcd_gb300.so``.  Device buffers are torch tensors (complex128,
canonical layouts); the context is bound to a torch CUDA stream.  If the
library is missing the import of this module still works, but creating a
``Lattice`` raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libqcd_gb300.so")

PREC = {"f64": 0, "f32": 1}

STATUS = {
    0: "QCD_OK", 1: "QCD_ERR_ARG", 2: "QCD_ERR_CUDA", 3: "QCD_ERR_OOM", 4: "QCD_ERR_NOT_CONVERGED",
    5: "QCD_ERR_BREAKDOWN", 6: "QCD_ERR_NONFINITE", 7: "QCD_ERR_TIMEOUT", 8: "QCD_ERR_STATE",
}

# every symbol include/qcd.h declares
EXPORTS = (
    "qcd_status_string", "qcd_last_error", "qcd_create", "qcd_destroy", "qcd_load_gauge",
    "qcd_default_params", "qcd_set_params", "qcd_apply_dirac", "qcd_apply_sap", "qcd_solve",
    "qcd_nucleon_2pt", "qcd_ama_nucleon_2pt", "qcd_get_clover", "qcd_profile_enable", "qcd_profile_read",
    "qcd_deflation_setup", "qcd_deflation_fields", "qcd_deflation_little_matrix", "qcd_deflation_little",
    "qcd_nucleon_2pt_noalloc", "qcd_autotune", "qcd_fh_forward", "qcd_fh_gradient", "qcd_solve_multi",
    "qcd_nucleon_3pt", "qcd_ama_nucleon", "qcd_ama_error_model", "qcd_smear_links", "qcd_set_smearing",
    "qcd_smear_gaussian", "qcd_get_smeared_links",
)


class QcdError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


class SolverParams(ctypes.Structure):
    _fields_ = [
        ("block", ctypes.c_int * 4), ("ncy", ctypes.c_int), ("nmr", ctypes.c_int), ("nkv", ctypes.c_int),
        ("max_outer", ctypes.c_int), ("restart_drop", ctypes.c_double), ("precision", ctypes.c_int),
        ("rhs_tile", ctypes.c_int), ("sap_half", ctypes.c_int), ("dfl", ctypes.c_int),
        ("dfl_little_iters", ctypes.c_int), ("dfl_gen_iters", ctypes.c_int), ("graphs", ctypes.c_int),
        ("basis_half", ctypes.c_int), ("resid_f32_tol", ctypes.c_double),
    ]


class AmaParams(ctypes.Structure):
    _fields_ = [("n_exact", ctypes.c_int), ("sloppy_tol", ctypes.c_double), ("exact_tol", ctypes.c_double),
                ("n_iter_2pt", ctypes.c_int), ("n_iter_3pt", ctypes.c_int), ("t_sep", ctypes.c_int),
                ("direction", ctypes.c_int)]


class KernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("launches", ctypes.c_int), ("ms", ctypes.c_double),
                ("bytes", ctypes.c_double), ("flops", ctypes.c_double)]


class RhsStats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("outer_iters", ctypes.c_int), ("restarts", ctypes.c_int),
                ("true_rel_residual", ctypes.c_double)]

    def as_dict(self):
        return {"status": STATUS.get(self.status, self.status), "outer_iters": self.outer_iters,
                "restarts": self.restarts, "true_rel_residual": self.true_rel_residual}


_lib = None


def load_library(path=LIB_PATH):
    """Load libqcd_gb300.so and declare the signatures; raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libqcd_gb300.so not found at %s: run __graft_entry__.build() first "
                           "(the library has no CPU fallback)" % path)
    L = ctypes.CDLL(path)
    vp, ip, dp, i, d = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double), \
        ctypes.c_int, ctypes.c_double
    L.qcd_status_string.restype = ctypes.c_char_p
    L.qcd_status_string.argtypes = [i]
    L.qcd_last_error.restype = ctypes.c_char_p
    L.qcd_last_error.argtypes = []
    L.qcd_create.argtypes = [ctypes.POINTER(vp), ip, vp]
    L.qcd_destroy.argtypes = [vp]
    L.qcd_destroy.restype = None
    L.qcd_load_gauge.argtypes = [vp, vp, i, d, d, i]
    L.qcd_default_params.argtypes = [ctypes.POINTER(SolverParams)]
    L.qcd_default_params.restype = None
    L.qcd_set_params.argtypes = [vp, ctypes.POINTER(SolverParams)]
    L.qcd_apply_dirac.argtypes = [vp, vp, vp, i, i, i]
    L.qcd_apply_sap.argtypes = [vp, vp, vp, i, i]
    L.qcd_solve.argtypes = [vp, vp, vp, i, dp, ctypes.POINTER(RhsStats)]
    L.qcd_nucleon_2pt.argtypes = [vp, vp, ip, dp, i]
    L.qcd_nucleon_3pt.argtypes = [vp, vp, ip, i, i, d, dp, ctypes.POINTER(RhsStats)]
    L.qcd_ama_nucleon.argtypes = [vp, ip, i, ctypes.POINTER(AmaParams), dp, dp, dp, dp, ctypes.POINTER(RhsStats)]
    L.qcd_ama_error_model.argtypes = [dp, dp, dp, i, i, i, dp]
    L.qcd_smear_links.argtypes = [vp, d, i]
    L.qcd_set_smearing.argtypes = [vp, d, i]
    L.qcd_smear_gaussian.argtypes = [vp, vp, vp, i]
    L.qcd_get_smeared_links.argtypes = [vp, vp]
    L.qcd_ama_nucleon_2pt.argtypes = [vp, ip, i, i, d, d, dp, dp, ctypes.POINTER(RhsStats)]
    L.qcd_get_clover.argtypes = [vp, vp]
    L.qcd_nucleon_2pt_noalloc.argtypes = [ip, i, vp, ip, vp, i, vp]
    L.qcd_autotune.argtypes = [vp, vp, i, d, ctypes.c_char_p, ctypes.POINTER(SolverParams)]
    L.qcd_fh_forward.argtypes = [vp, ip, d, vp, dp, ctypes.POINTER(RhsStats)]
    L.qcd_solve_multi.argtypes = [ctypes.POINTER(vp), i, ctypes.POINTER(vp), ctypes.POINTER(vp), ip,
                                  ctypes.POINTER(dp), ctypes.POINTER(ctypes.POINTER(RhsStats))]
    L.qcd_fh_gradient.argtypes = [vp, vp, ip, dp, d, dp, ctypes.POINTER(RhsStats)]
    L.qcd_deflation_setup.argtypes = [vp, vp, i, i]
    L.qcd_deflation_fields.argtypes = [vp, vp]
    L.qcd_deflation_little_matrix.argtypes = [vp, dp]
    L.qcd_deflation_little.argtypes = [vp, dp, dp, i, i, i]
    L.qcd_profile_enable.argtypes = [vp, i]
    L.qcd_profile_read.argtypes = [vp, ctypes.POINTER(KernelTime), i, ip]
    for name in EXPORTS:
        if name not in ("qcd_status_string", "qcd_last_error", "qcd_destroy", "qcd_default_params"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(status, allow=()):
    if status != 0 and status not in allow:
        raise QcdError(status, _lib.qcd_last_error().decode(errors="replace"))
    return status


def _dev_ptr(t):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()):
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def nucleon_2pt_noalloc(dims, prop, src, corr, precision="f64", time_bc=-1, stream=None):
    """Enqueue the allocation-free contraction: prop (CUDA complex128, 12 spinors,
    canonical) -> corr (CUDA float64 tensor of 2*T*2 values, written in place).
    The library allocates nothing; the caller owns both buffers."""
    import torch
    L = load_library()
    s = stream if stream is not None else torch.cuda.current_stream()
    _check(L.qcd_nucleon_2pt_noalloc((ctypes.c_int * 4)(*dims), int(time_bc), _dev_ptr(prop),
                                     (ctypes.c_int * 4)(*src), _dev_ptr(corr), PREC[precision],
                                     ctypes.c_void_p(s.cuda_stream)))
    return corr


def ama_error_model(exact, appx_org, appx):
    """Error model of the AMA estimator (eqs. ama1-ama3) computed by the
    library: exact, appx_org [n_conf, n_org], appx [n_conf, n_g] (real).
    Returns {dr, R, model, measured}."""
    L = load_library()
    e = np.ascontiguousarray(exact, dtype=np.float64)
    a0 = np.ascontiguousarray(appx_org, dtype=np.float64)
    a = np.ascontiguousarray(appx, dtype=np.float64)
    out = np.zeros(4)
    dpp = lambda x: x.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    _check(L.qcd_ama_error_model(dpp(e), dpp(a0), dpp(a), e.shape[0], e.shape[1], a.shape[1], dpp(out)))
    return {"dr": out[0], "R": out[1], "model": out[2], "measured": out[3]}


class Lattice:
    """A lattice context: dims = (T, X, Y, Z)."""

    def __init__(self, dims, stream=None):
        import torch
        L = load_library()
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the Wilson-clover library runs on the GPU only")
        self.dims = tuple(int(x) for x in dims)
        self.T, self.X, self.Y, self.Z = self.dims
        self.V = self.T * self.X * self.Y * self.Z
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._ctx = ctypes.c_void_p()
        _check(L.qcd_create(ctypes.byref(self._ctx), (ctypes.c_int * 4)(*self.dims),
                            ctypes.c_void_p(self.stream.cuda_stream)))
        self.params = SolverParams()
        L.qcd_default_params(ctypes.byref(self.params))
        self.time_bc = -1

    # ----------------------------------------------------------------------
    def _after_torch(self):
        """The library works on self.stream; tensors handed to it were written on
        torch's current stream (e.g. the zero-filled solution of solve): make
        self.stream wait for that work before the call."""
        import torch
        cur = torch.cuda.current_stream()
        if cur != self.stream:
            self.stream.wait_stream(cur)

    def _before_torch(self):
        """Results the library wrote on self.stream: make torch's current stream
        wait for them (calls that return to the host have synchronised already)."""
        import torch
        cur = torch.cuda.current_stream()
        if cur != self.stream:
            cur.wait_stream(self.stream)

    def close(self):
        if self._ctx:
            _lib.qcd_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def spinor_shape(self, nrhs=None):
        s = (self.T, self.Z, self.Y, self.X, 4, 3)
        return s if nrhs is None else (nrhs,) + s

    # ----------------------------------------------------------------------
    def load_gauge(self, U, csw, kappa, time_bc=-1):
        """U: numpy complex128 (host) or torch complex128 CUDA tensor, shape (T,Z,Y,X,4,3,3)."""
        import torch
        self.time_bc = int(time_bc)
        if isinstance(U, torch.Tensor):
            U = U.contiguous()
            self._after_torch()
            st = _lib.qcd_load_gauge(self._ctx, _dev_ptr(U), 1, float(csw), float(kappa), int(time_bc))
        else:
            U = np.ascontiguousarray(U, dtype=np.complex128)
            st = _lib.qcd_load_gauge(self._ctx, U.ctypes.data_as(ctypes.c_void_p), 0, float(csw), float(kappa),
                                     int(time_bc))
        _check(st)

    def set_params(self, **kw):
        p = SolverParams()
        ctypes.memmove(ctypes.byref(p), ctypes.byref(self.params), ctypes.sizeof(p))
        for k, v in kw.items():
            if k == "block":
                p.block = (ctypes.c_int * 4)(*v)
            elif k == "precision":
                p.precision = PREC[v] if isinstance(v, str) else int(v)
            else:
                setattr(p, k, v)
        _check(_lib.qcd_set_params(self._ctx, ctypes.byref(p)))
        self.params = p

    # ----------------------------------------------------------------------
    def apply_dirac(self, psi, dagger=False, precision="f64"):
        import torch
        psi = psi.contiguous()
        n = psi.shape[0] if psi.dim() == 7 else 1
        out = torch.empty_like(psi)
        self._after_torch()
        _check(_lib.qcd_apply_dirac(self._ctx, _dev_ptr(psi), _dev_ptr(out), n, int(bool(dagger)), PREC[precision]))
        self._before_torch()
        return out

    def apply_sap(self, eta, precision="f32"):
        import torch
        eta = eta.contiguous()
        n = eta.shape[0] if eta.dim() == 7 else 1
        out = torch.empty_like(eta)
        self._after_torch()
        _check(_lib.qcd_apply_sap(self._ctx, _dev_ptr(eta), _dev_ptr(out), n, PREC[precision]))
        self._before_torch()
        return out

    def autotune(self, eta, tol, cache_path=None):
        """Pick SAP block shape, block-copy precision, nkv and rhs_tile by timing solves of eta."""
        eta = eta.contiguous()
        n = eta.shape[0] if eta.dim() == 7 else 1
        best = SolverParams()
        cp = cache_path.encode() if cache_path else None
        self._after_torch()
        _check(_lib.qcd_autotune(self._ctx, _dev_ptr(eta), n, float(tol), cp, ctypes.byref(best)))
        self.params = best
        return {"block": list(best.block), "sap_half": best.sap_half, "nkv": best.nkv, "rhs_tile": best.rhs_tile}

    def solve(self, eta, tol, psi0=None, allow_not_converged=False, check=True):
        """Solve D psi = eta; returns (psi, [stats dict per RHS]).  check=False returns
        whatever the per-RHS statuses are instead of raising."""
        import torch
        eta = eta.contiguous()
        n = eta.shape[0] if eta.dim() == 7 else 1
        psi = torch.zeros_like(eta) if psi0 is None else psi0.clone().contiguous()
        tols = (ctypes.c_double * n)(*([float(tol)] * n if np.isscalar(tol) else [float(x) for x in tol]))
        stats = (RhsStats * n)()
        self._after_torch()
        st = _lib.qcd_solve(self._ctx, _dev_ptr(eta), _dev_ptr(psi), n, tols, stats)
        self._before_torch()
        if check:
            _check(st, allow=(4,) if allow_not_converged else ())
        return psi, [s.as_dict() for s in stats]

    def nucleon_2pt(self, prop, src, precision="f64"):
        """C[parity, t] (complex, host numpy) from a 12-spinor point-source propagator."""
        prop = prop.contiguous()
        out = np.zeros((2, self.T, 2), dtype=np.float64)
        self._after_torch()
        _check(_lib.qcd_nucleon_2pt(self._ctx, _dev_ptr(prop), (ctypes.c_int * 4)(*src),
                                    out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), PREC[precision]))
        return out[..., 0] + 1j * out[..., 1]

    def nucleon_3pt(self, prop, src, t_sep, direction=1, tol=1e-10, allow_not_converged=False):
        """Isovector three-point functions C3[insertion (A_3, S, T_12), t] (host
        numpy complex) from the 12-spinor point-source propagator prop, sink at
        src_t + direction * t_sep; returns (C3, stats of the 24 sequential solves)."""
        prop = prop.contiguous()
        out = np.zeros((3, self.T, 2), dtype=np.float64)
        stats = (RhsStats * 24)()
        self._after_torch()
        st = _lib.qcd_nucleon_3pt(self._ctx, _dev_ptr(prop), (ctypes.c_int * 4)(*src), int(t_sep), int(direction),
                                  float(tol), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), stats)
        _check(st, allow=(4,) if allow_not_converged else ())
        return out[..., 0] + 1j * out[..., 1], [s.as_dict() for s in stats]

    def ama_nucleon(self, srcs, n_exact, sloppy_tol=1e-3, exact_tol=1e-10, n_iter_2pt=0, n_iter_3pt=0, t_sep=0,
                    direction=1, allow_not_converged=False):
        """AMA two- (and with t_sep, three-) point functions; returns a dict with
        c2_ama [2, T], c2_all [n, 2, T], c3_ama [3, T], c3_all [n, 3, T] (complex
        numpy; the 3pt entries only with t_sep) and stats (list per solve)."""
        srcs = np.ascontiguousarray(np.asarray(srcs, dtype=np.int32).reshape(-1, 4))
        ns = srcs.shape[0]
        nj = ns + int(n_exact)
        p = AmaParams(int(n_exact), float(sloppy_tol), float(exact_tol), int(n_iter_2pt), int(n_iter_3pt), int(t_sep),
                      int(direction))
        c2a = np.zeros((2, self.T, 2))
        c2 = np.zeros((nj, 2, self.T, 2))
        c3a = np.zeros((3, self.T, 2))
        c3 = np.zeros((nj, 3, self.T, 2))
        stats = (RhsStats * (nj * (12 + (24 if t_sep else 0))))()
        dpp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        st = _lib.qcd_ama_nucleon(self._ctx, srcs.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), ns, ctypes.byref(p),
                                  dpp(c2a), dpp(c3a), dpp(c2), dpp(c3), stats)
        _check(st, allow=(4,) if allow_not_converged else ())
        cx = lambda a: a[..., 0] + 1j * a[..., 1]
        out = {"c2_ama": cx(c2a), "c2_all": cx(c2), "stats": [s.as_dict() for s in stats]}
        if t_sep:
            out.update({"c3_ama": cx(c3a), "c3_all": cx(c3)})
        return out

    def ama_nucleon_2pt(self, srcs, n_exact, sloppy_tol, exact_tol, allow_not_converged=False):
        """AMA nucleon two-point function; returns (ama[2,T], all[n_src+n_exact,2,T], stats)."""
        srcs = np.ascontiguousarray(np.asarray(srcs, dtype=np.int32).reshape(-1, 4))
        ns = srcs.shape[0]
        ama = np.zeros((2, self.T, 2))
        allc = np.zeros((ns + n_exact, 2, self.T, 2))
        stats = (RhsStats * (12 * (ns + n_exact)))()
        st = _lib.qcd_ama_nucleon_2pt(self._ctx, srcs.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), ns,
                                      int(n_exact), float(sloppy_tol), float(exact_tol),
                                      ama.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                      allc.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), stats)
        _check(st, allow=(4,) if allow_not_converged else ())
        return ama[..., 0] + 1j * ama[..., 1], allc[..., 0] + 1j * allc[..., 1], [s.as_dict() for s in stats]

    def profile(self, on=True):
        """Start (clearing old records) or stop recording kernel times."""
        _check(_lib.qcd_profile_enable(self._ctx, int(bool(on))))

    def profile_read(self):
        """{family: {launches, ms, bytes, flops}} since the last read; clears the records."""
        buf = (KernelTime * 16)()
        n = ctypes.c_int()
        _check(_lib.qcd_profile_read(self._ctx, buf, 16, ctypes.byref(n)))
        return {buf[k].name.decode(): {"launches": buf[k].launches, "ms": buf[k].ms, "bytes": buf[k].bytes,
                                       "flops": buf[k].flops} for k in range(n.value)}

    # ----------------------------------------------------------------------
    def deflation_setup(self, init, n_inv):
        """Build the deflation subspace from init (CUDA complex128, (ns,)+spinor shape)."""
        init = init.contiguous()
        self._after_torch()
        _check(_lib.qcd_deflation_setup(self._ctx, _dev_ptr(init), int(init.shape[0]), int(n_inv)))
        self.dfl_ns = int(init.shape[0])

    def deflation_fields(self):
        import torch
        out = torch.empty(self.spinor_shape(self.dfl_ns), dtype=torch.complex128, device="cuda")
        self._after_torch()
        _check(_lib.qcd_deflation_fields(self._ctx, _dev_ptr(out)))
        self._before_torch()
        return out

    def n_blocks(self):
        b = list(self.params.block)
        return (self.T // b[0]) * (self.X // b[1]) * (self.Y // b[2]) * (self.Z // b[3])

    def deflation_little_matrix(self):
        """A as numpy complex [block][9][ns][ns]."""
        nb, ns = self.n_blocks(), self.dfl_ns
        out = np.zeros((nb, 9, ns, ns, 2))
        _check(_lib.qcd_deflation_little_matrix(self._ctx, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return out[..., 0] + 1j * out[..., 1]

    def deflation_little(self, v, mode, m=16):
        """mode 0: A v; mode 1: m-step approximation of A^-1 v.  v: numpy complex [n, block, ns]."""
        v = np.ascontiguousarray(v, dtype=np.complex128)
        n = v.shape[0]
        out = np.zeros(v.shape + (2,))
        vin = np.ascontiguousarray(np.stack([v.real, v.imag], axis=-1))
        _check(_lib.qcd_deflation_little(self._ctx, vin.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                         out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), n, int(mode), int(m)))
        return out[..., 0] + 1j * out[..., 1]

    # ----------------------------------------------------------------------
    def fh_forward(self, src, tol):
        """(S in Wilson normalisation [CUDA, 12 spinors], C as numpy float64 [2, T, 2])."""
        import torch
        prop = torch.empty(self.spinor_shape(12), dtype=torch.complex128, device="cuda")
        corr = np.zeros((2, self.T, 2))
        stats = (RhsStats * 12)()
        self._after_torch()
        _check(_lib.qcd_fh_forward(self._ctx, (ctypes.c_int * 4)(*src), float(tol), _dev_ptr(prop),
                                   corr.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), stats))
        return prop, corr

    def fh_gradient(self, prop, src, gcorr, tol):
        """(dL/dm0, dL/dlambda) for the upstream gradient gcorr [2, T, 2] of C."""
        g = np.ascontiguousarray(gcorr, dtype=np.float64)
        grad = np.zeros(2)
        stats = (RhsStats * 24)()
        self._after_torch()
        _check(_lib.qcd_fh_gradient(self._ctx, _dev_ptr(prop.contiguous()), (ctypes.c_int * 4)(*src),
                                    g.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), float(tol),
                                    grad.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), stats))
        return float(grad[0]), float(grad[1])

    def smear_links(self, alpha, n_ape):
        """APE-smear the spatial links (kept in the context)."""
        _check(_lib.qcd_smear_links(self._ctx, float(alpha), int(n_ape)))

    def set_smearing(self, kappa_g, n_gauss):
        """Gaussian source and sink smearing for ama_nucleon (n_gauss = 0: point)."""
        _check(_lib.qcd_set_smearing(self._ctx, float(kappa_g), int(n_gauss)))

    def smear_gaussian(self, psi):
        """K psi for a CUDA complex128 tensor of spinors (canonical layout)."""
        import torch
        psi = psi.contiguous()
        n = psi.shape[0] if psi.dim() == 7 else 1
        out = torch.empty_like(psi)
        self._after_torch()
        _check(_lib.qcd_smear_gaussian(self._ctx, _dev_ptr(psi), _dev_ptr(out), n))
        self._before_torch()
        return out

    def smeared_links(self):
        """The APE-smeared gauge field as a CUDA complex128 tensor (T, Z, Y, X, 4, 3, 3)."""
        import torch
        out = torch.empty((self.T, self.Z, self.Y, self.X, 4, 3, 3), dtype=torch.complex128, device="cuda")
        self._after_torch()
        _check(_lib.qcd_get_smeared_links(self._ctx, _dev_ptr(out)))
        self._before_torch()
        return out

    def get_clover(self):
        """A(x) as a CUDA complex128 tensor [V, 2, 6, 6]."""
        import torch
        out = torch.empty((self.V, 2, 6, 6), dtype=torch.complex128, device="cuda")
        self._after_torch()
        _check(_lib.qcd_get_clover(self._ctx, _dev_ptr(out)))
        self._before_torch()
        return out


def solve_multi(lattices, etas, tol):
    """Solve D psi = eta on several lattices in one call (their kernels overlap
    on the GPU); every lattice needs its own non-default stream."""
    import torch
    L = load_library()
    n = len(lattices)
    etas = [e.contiguous() for e in etas]
    psis = [torch.zeros_like(e) for e in etas]
    nr = [e.shape[0] if e.dim() == 7 else 1 for e in etas]
    tols = [(ctypes.c_double * k)(*([float(tol)] * k)) for k in nr]
    stats = [(RhsStats * k)() for k in nr]
    VP = ctypes.c_void_p
    for lat in lattices:
        lat._after_torch()
    st = L.qcd_solve_multi((VP * n)(*[l._ctx for l in lattices]), n, (VP * n)(*[e.data_ptr() for e in etas]),
                           (VP * n)(*[p.data_ptr() for p in psis]), (ctypes.c_int * n)(*nr),
                           (ctypes.POINTER(ctypes.c_double) * n)(*[ctypes.cast(t, ctypes.POINTER(ctypes.c_double)) for t in tols]),
                           (ctypes.POINTER(RhsStats) * n)(*[ctypes.cast(s, ctypes.POINTER(RhsStats)) for s in stats]))
    _check(st)
    return psis, [[s.as_dict() for s in ss] for ss in stats]


def _nucleon_fh_class():
    import torch

    class NucleonFH(torch.autograd.Function):
        """Point-source nucleon two-point function C (float64 [2, T, 2]: parity,
        time, re/im) as a function of the bare mass m0 and the axial
        Feynman-Hellmann coupling lambda (at lambda = 0).  forward: 12 solves and
        the contraction; backward: the adjoint (gamma_5) solves, all in the
        library."""

        @staticmethod
        def forward(ctx, m0, lam, lattice, U, csw, src, tol):
            if float(lam) != 0.0:
                raise ValueError("the derivative is taken at lambda = 0")
            kappa = 1.0 / (2.0 * float(m0) + 8.0)
            lattice.load_gauge(U, csw, kappa, lattice.time_bc)
            prop, corr = lattice.fh_forward(src, tol)
            ctx.lattice, ctx.prop, ctx.src, ctx.tol = lattice, prop, tuple(src), tol
            return torch.from_numpy(corr)

        @staticmethod
        def backward(ctx, g):
            dm, dl = ctx.lattice.fh_gradient(ctx.prop, ctx.src, g.detach().cpu().numpy(), ctx.tol)
            return (torch.tensor(dm, dtype=torch.float64), torch.tensor(dl, dtype=torch.float64),
                    None, None, None, None, None)

    return NucleonFH


def nucleon_fh(m0, lam, lattice, U, csw, src, tol=1e-12):
    """Differentiable C(m0, lambda) (see NucleonFH)."""
    return _nucleon_fh_class().apply(m0, lam, lattice, U, csw, src, tol)
