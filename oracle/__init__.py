"""FP64 CPU oracle for MB-SCB transient slab S_N transport (arXiv 2305.13555).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  It shares
no code with the CUDA implementation in ``paper_2305_13555_gb300``; the only
module both sides read is ``workloads`` (seeded input generators, no method
arithmetic).

Contents
  * ``gauss_legendre``      -- S_N quadrature (Sec. 2, "Gauss Legendre quadrature").
  * ``oci_iteration``       -- one one-cell-inversion iteration: per-cell dense
                               (A - S) Psi = c solved by LU (Sec. "One-Cell Inversion").
  * ``si_iteration``        -- one source iteration: per-ordinate 4x4 sweeps
                               (Sec. "Source Iteration (SI)").
  * ``run``                 -- the time-step driver for either scheme.
  * ``be_oci_iteration``, ``be_si_iteration``, ``run_be`` -- the same for the
                               backward-Euler scheme (the disabled section).
  * ``oracle.brute``        -- whole-problem dense solve assembled directly from
                               the SCB-MB balance equations (tiny slabs).
  * ``oracle.nn``           -- FP64 plain-loop 1-D CNN forward/backward.

Layouts follow ``oci_oracle.c``: ordinates ascending in mu; psi [J][N][4] with
components (k,L) (k,R) (k+1/2,L) (k+1/2,R); psi_edge [J][N][2]; phi [J][4].
"""
import ctypes

import numpy as np

from . import build as _build

BC_VACUUM, BC_REFLECT, BC_INCIDENT = 0, 1, 2
OCI, SI = 0, 1

_BC_NAMES = {"vacuum": BC_VACUUM, "reflect": BC_REFLECT, "reflecting": BC_REFLECT,
             "incident": BC_INCIDENT}


class _Problem(ctypes.Structure):
    _fields_ = [
        ("n_cells", ctypes.c_int32), ("n_ord", ctypes.c_int32),
        ("dx", ctypes.c_void_p), ("sigma_t", ctypes.c_void_p), ("sigma_s", ctypes.c_void_p),
        ("q", ctypes.c_void_p),
        ("v", ctypes.c_double), ("dt", ctypes.c_double),
        ("bc_left", ctypes.c_int32), ("bc_right", ctypes.c_int32),
        ("psi_bc_left", ctypes.c_void_p), ("psi_bc_right", ctypes.c_void_p),
    ]


_lib = None


def load_library(path):
    """Load an oracle shared library built from ``oci_oracle.c`` (the default
    one, or a deliberately altered copy in the sensitivity tests)."""
    lib = ctypes.CDLL(path)
    dp = ctypes.c_void_p
    lib.oracle_gauss_legendre.argtypes = [ctypes.c_int32, dp, dp]
    lib.oracle_oci_iteration.argtypes = [ctypes.POINTER(_Problem), dp, dp, dp, dp]
    lib.oracle_si_iteration.argtypes = [ctypes.POINTER(_Problem), dp, dp, dp, dp, dp]
    lib.oracle_run.argtypes = [ctypes.POINTER(_Problem), ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                               ctypes.c_int32, ctypes.c_int32, dp, dp, dp, dp, ctypes.c_int32]
    lib.oracle_be_run.argtypes = lib.oracle_run.argtypes
    lib.oracle_be_oci_iteration.argtypes = [ctypes.POINTER(_Problem), dp, dp, dp, dp]
    lib.oracle_be_si_iteration.argtypes = [ctypes.POINTER(_Problem), dp, dp, dp, dp, dp]
    lib.oracle_max_threads.restype = ctypes.c_int
    return lib


def _load(lib=None):
    global _lib
    if lib is not None:
        return lib
    if _lib is None:
        _lib = load_library(_build.build())
    return _lib


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _bc_code(x):
    return _BC_NAMES[x] if isinstance(x, str) else int(x)


class Problem:
    """Holds contiguous FP64 copies of a problem dict (see ``workloads``) and the
    ctypes struct pointing at them."""

    def __init__(self, prob: dict):
        J, N = int(prob["n_cells"]), int(prob["n_ord"])
        self.J, self.N = J, N
        self.dx = _f64(prob["dx"], (J,))
        self.sigma_t = _f64(prob["sigma_t"], (J,))
        self.sigma_s = _f64(prob["sigma_s"], (J,))
        q = prob.get("q")
        self.q = np.zeros((J, 4)) if q is None else _f64(q, (J, 4))
        bl, br = prob.get("psi_bc_left"), prob.get("psi_bc_right")
        self.bcl = None if bl is None else _f64(bl, (N // 2, 2))
        self.bcr = None if br is None else _f64(br, (N // 2, 2))
        self.s = _Problem(J, N, _ptr(self.dx).value, _ptr(self.sigma_t).value, _ptr(self.sigma_s).value,
                          _ptr(self.q).value, float(prob["v"]), float(prob["dt"]),
                          _bc_code(prob.get("bc_left", 0)), _bc_code(prob.get("bc_right", 0)),
                          None if self.bcl is None else _ptr(self.bcl).value,
                          None if self.bcr is None else _ptr(self.bcr).value)
        p0 = prob.get("psi0")
        self.psi0 = np.zeros((J, N, 2)) if p0 is None else _f64(p0, (J, N, 2))


def _as_problem(prob):
    return prob if isinstance(prob, Problem) else Problem(prob)


def gauss_legendre(n: int, lib=None):
    """Nodes (ascending) and weights of the n-point Gauss-Legendre rule on [-1, 1]."""
    mu, w = np.zeros(n), np.zeros(n)
    if _load(lib).oracle_gauss_legendre(n, _ptr(mu), _ptr(w)):
        raise ValueError("n must be >= 1")
    return mu, w


def oci_iteration(prob, psi_edge, psi_in, lib=None):
    """One OCI iteration from iterate ``psi_in`` [J][N][4]; returns (psi_out, phi)."""
    p = _as_problem(prob)
    pe, pi = _f64(psi_edge, (p.J, p.N, 2)), _f64(psi_in, (p.J, p.N, 4))
    po, ph = np.zeros((p.J, p.N, 4)), np.zeros((p.J, 4))
    err = _load(lib).oracle_oci_iteration(ctypes.byref(p.s), _ptr(pe), _ptr(pi), _ptr(po), _ptr(ph))
    if err:
        raise RuntimeError(f"oracle_oci_iteration failed ({err})")
    return po, ph


def si_iteration(prob, psi_edge, phi_in, psi_in, lib=None):
    """One SI iteration with lagged scalar flux ``phi_in`` [J][4]; ``psi_in``
    supplies a lagged reflecting right face.  Returns (psi_out, phi)."""
    p = _as_problem(prob)
    pe, fi, pi = _f64(psi_edge, (p.J, p.N, 2)), _f64(phi_in, (p.J, 4)), _f64(psi_in, (p.J, p.N, 4))
    po, ph = np.zeros((p.J, p.N, 4)), np.zeros((p.J, 4))
    err = _load(lib).oracle_si_iteration(ctypes.byref(p.s), _ptr(pe), _ptr(fi), _ptr(pi), _ptr(po), _ptr(ph))
    if err:
        raise RuntimeError(f"oracle_si_iteration failed ({err})")
    return po, ph


def be_oci_iteration(prob, psi_prev, psi_in, lib=None):
    """One backward-Euler OCI iteration from iterate ``psi_in`` [J][N][2] with
    psi^{n-1} = ``psi_prev``; returns (psi_out [J][N][2], phi [J][2])."""
    p = _as_problem(prob)
    pp, pi = _f64(psi_prev, (p.J, p.N, 2)), _f64(psi_in, (p.J, p.N, 2))
    po, ph = np.zeros((p.J, p.N, 2)), np.zeros((p.J, 2))
    err = _load(lib).oracle_be_oci_iteration(ctypes.byref(p.s), _ptr(pp), _ptr(pi), _ptr(po), _ptr(ph))
    if err:
        raise RuntimeError(f"oracle_be_oci_iteration failed ({err})")
    return po, ph


def be_si_iteration(prob, psi_prev, phi_in, psi_in, lib=None):
    """One backward-Euler SI iteration with lagged scalar flux ``phi_in`` [J][2]
    (``psi_in`` supplies a lagged reflecting right face)."""
    p = _as_problem(prob)
    pp, fi, pi = _f64(psi_prev, (p.J, p.N, 2)), _f64(phi_in, (p.J, 2)), _f64(psi_in, (p.J, p.N, 2))
    po, ph = np.zeros((p.J, p.N, 2)), np.zeros((p.J, 2))
    err = _load(lib).oracle_be_si_iteration(ctypes.byref(p.s), _ptr(pp), _ptr(fi), _ptr(pi), _ptr(po), _ptr(ph))
    if err:
        raise RuntimeError(f"oracle_be_si_iteration failed ({err})")
    return po, ph


def run(prob, method=OCI, n_steps=1, tol=1e-10, max_iter=10000, commit_unconverged=False,
        psi_edge=None, n_threads=0, lib=None):
    """March ``n_steps`` steps.  Returns dict with psi_edge [J][N][2] (last
    committed), phi_steps [n_steps][J][4], iters, resid and status (0 ok,
    4 not converged, 5 NaN)."""
    p = _as_problem(prob)
    if isinstance(method, str):
        method = {"oci": OCI, "si": SI}[method.lower()]
    pe = (p.psi0 if psi_edge is None else _f64(psi_edge, (p.J, p.N, 2))).copy()
    phs = np.zeros((n_steps, p.J, 4))
    its = np.zeros(n_steps, dtype=np.int32)
    res = np.zeros(n_steps)
    st = _load(lib).oracle_run(ctypes.byref(p.s), int(method), int(n_steps), float(tol), int(max_iter),
                            int(bool(commit_unconverged)), _ptr(pe), _ptr(phs),
                            its.ctypes.data_as(ctypes.c_void_p), _ptr(res), int(n_threads))
    if st not in (0, 4, 5):
        raise RuntimeError(f"oracle_run failed ({st})")
    return {"psi_edge": pe, "phi_steps": phs, "iters": its, "resid": res, "status": st}


def run_be(prob, method=OCI, n_steps=1, tol=1e-10, max_iter=10000, commit_unconverged=False,
           psi=None, n_threads=0, lib=None):
    """Backward-Euler variant (one time level per step, Sigma_hat = Sigma +
    1/(v dt), source psi^{n-1}/(v dt); the source at the new time is Q_{k+1/2}).
    Returns psi [J][N][2] (last committed step), phi_steps [n_steps][J][2],
    iters, resid, status.  The initial psi is prob's psi0 (or ``psi``)."""
    p = _as_problem(prob)
    if isinstance(method, str):
        method = {"oci": OCI, "si": SI}[method.lower()]
    ps = (p.psi0 if psi is None else _f64(psi, (p.J, p.N, 2))).copy()
    phs = np.zeros((n_steps, p.J, 2))
    its = np.zeros(n_steps, dtype=np.int32)
    res = np.zeros(n_steps)
    st = _load(lib).oracle_be_run(ctypes.byref(p.s), int(method), int(n_steps), float(tol), int(max_iter),
                                  int(bool(commit_unconverged)), _ptr(ps), _ptr(phs),
                                  its.ctypes.data_as(ctypes.c_void_p), _ptr(res), int(n_threads))
    if st not in (0, 4, 5):
        raise RuntimeError(f"oracle_be_run failed ({st})")
    return {"psi": ps, "phi_steps": phs, "iters": its, "resid": res, "status": st}


def max_threads() -> int:
    return int(_load().oracle_max_threads())
