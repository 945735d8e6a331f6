"""GB300 (sm_103a) one-cell inversion for transient slab S_N transport.

Thin Python binding of the C ABI declared in ``include/oci.h`` (arguments are
marshalled here; every step of the method runs in the library's CUDA kernels).
The functions carry the C names: ``oci_create``, ``oci_step``, ``si_step``,
``oci_fluxes`` ... and ``Solver`` wraps a handle for convenience.

Importing this package loads ``_build/liboci_gb300.so``; it raises if the
library has not been built (``python -m paper_2305_13555_gb300.build``) --
there is no CPU fallback.
"""
import ctypes
import os

import numpy as np

from . import build as _build

OCI_OK, OCI_EINVAL, OCI_ENOMEM, OCI_ECUDA, OCI_ENOTCONV, OCI_ENAN, OCI_ETIMEOUT, OCI_ESTATE, OCI_ESKIPPED = range(9)
OCI_BC_VACUUM, OCI_BC_REFLECT, OCI_BC_INCIDENT = 0, 1, 2
OCI_FP64, OCI_FP32, OCI_FP32_BF16HALO = 0, 1, 2
OCI_HALO_FP32, OCI_HALO_BF16 = 0, 1
OCI_GUESS_PREVIOUS, OCI_GUESS_EXTRAPOLATE = 0, 1
OCI_SOLVER_WOODBURY, OCI_SOLVER_DENSE = 0, 1
OCI_SWEEP_MARCH, OCI_SWEEP_SCAN = 0, 1
OCI_TIME_MB, OCI_TIME_BE = 0, 1
_SCHEME = {"mb": OCI_TIME_MB, "be": OCI_TIME_BE}
_SWEEP = {"march": OCI_SWEEP_MARCH, "scan": OCI_SWEEP_SCAN}
_SOLVER = {"woodbury": OCI_SOLVER_WOODBURY, "dense": OCI_SOLVER_DENSE}
_BC = {"vacuum": OCI_BC_VACUUM, "reflect": OCI_BC_REFLECT, "reflecting": OCI_BC_REFLECT,
       "incident": OCI_BC_INCIDENT}
_PREC = {"fp64": OCI_FP64, "f64": OCI_FP64, "double": OCI_FP64, "fp32": OCI_FP32, "f32": OCI_FP32,
         "float": OCI_FP32, "fp32_bf16halo": OCI_FP32_BF16HALO}
_HALO = {"fp32": OCI_HALO_FP32, "bf16": OCI_HALO_BF16}
_GUESS = {"previous": OCI_GUESS_PREVIOUS, "extrapolate": OCI_GUESS_EXTRAPOLATE}


class OciProblem(ctypes.Structure):
    _fields_ = [
        ("n_cells", ctypes.c_int32), ("n_ord", ctypes.c_int32),
        ("dx", ctypes.c_void_p), ("sigma_t", ctypes.c_void_p), ("sigma_s", ctypes.c_void_p),
        ("q", ctypes.c_void_p), ("v", ctypes.c_double), ("dt", ctypes.c_double),
        ("bc_left", ctypes.c_int32), ("bc_right", ctypes.c_int32),
        ("psi_bc_left", ctypes.c_void_p), ("psi_bc_right", ctypes.c_void_p), ("psi0", ctypes.c_void_p),
        ("precision", ctypes.c_int32), ("max_iter", ctypes.c_int32), ("tol", ctypes.c_double),
        ("cuda_stream", ctypes.c_void_p),
    ]


class OciStats(ctypes.Structure):
    _fields_ = [
        ("iters", ctypes.c_int32), ("status", ctypes.c_int32), ("residual", ctypes.c_double),
        ("seconds", ctypes.c_double), ("committed", ctypes.c_int32), ("nn_accepts", ctypes.c_int32),
        ("nn_rejects", ctypes.c_int32), ("refined", ctypes.c_int32), ("launches", ctypes.c_int32),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


# Every entry point declared in include/oci.h, with its ctypes signature.
_VP, _I32, _D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_double
SIGNATURES = {
    "oci_create": (ctypes.c_int, [ctypes.POINTER(OciProblem), ctypes.POINTER(ctypes.c_void_p)]),
    "oci_destroy": (None, [_VP]),
    "oci_set_source": (ctypes.c_int, [_VP, _VP]),
    "oci_set_iteration": (ctypes.c_int, [_VP, _D, _I32, _I32]),
    "oci_set_stream": (ctypes.c_int, [_VP, _VP]),
    "oci_set_solver": (ctypes.c_int, [_VP, _I32]),
    "oci_set_sweep": (ctypes.c_int, [_VP, _I32]),
    "oci_set_time_scheme": (ctypes.c_int, [_VP, _I32]),
    "oci_set_halo": (ctypes.c_int, [_VP, _I32]),
    "oci_set_guess": (ctypes.c_int, [_VP, _I32]),
    "oci_step_async": (ctypes.c_int, [_VP]),
    "oci_step_wait": (ctypes.c_int, [_VP, _VP]),
    "oci_run_steps": (ctypes.c_int, [_VP, _I32, _VP, _VP, _VP, _VP]),
    "oci_fluxes_async": (ctypes.c_int, [_VP, _VP]),
    "oci_sync": (ctypes.c_int, [_VP]),
    "oci_set_wait_limits": (ctypes.c_int, [_VP, ctypes.c_uint32, _I32]),
    "oci_step": (ctypes.c_int, [_VP, ctypes.POINTER(OciStats)]),
    "si_step": (ctypes.c_int, [_VP, ctypes.POINTER(OciStats)]),
    "oci_fluxes": (ctypes.c_int, [_VP, _VP]),
    "oci_fluxes_device": (ctypes.c_int, [_VP, _VP]),
    "oci_get_state": (ctypes.c_int, [_VP, _VP]),
    "oci_set_state": (ctypes.c_int, [_VP, _VP]),
    "oci_query": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP]),
    "oci_profile_iterations": (ctypes.c_int, [_VP, _I32, ctypes.POINTER(ctypes.c_double)]),
    "oci_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "oci_dd_begin": (ctypes.c_int, [_VP]),
    "oci_dd_export": (ctypes.c_int, [_VP, _VP, _VP]),
    "oci_dd_import": (ctypes.c_int, [_VP, _VP, _VP]),
    "oci_dd_iterate": (ctypes.c_int, [_VP, _VP]),
    "oci_dd_decide": (ctypes.c_int, [_VP, _VP, _VP, ctypes.POINTER(OciStats)]),
    "oci_nn_attach": (ctypes.c_int, [_VP, _VP, _I32, _I32]),
    "oci_nn_static_features": (ctypes.c_int, [_VP, _VP, _VP]),
    # include/oci_nn.h
    "oci_nn_param_count": (ctypes.c_int32, []),
    "oci_nn_workspace_bytes": (ctypes.c_size_t, [_I32, _I32]),
    "oci_nn_features": (ctypes.c_int, [_VP, _VP, _VP, _VP, _I32, _I32, _VP, _VP, _VP]),
    "oci_nn_targets": (ctypes.c_int, [_VP, _VP, _VP, _I32, _I32, _VP, _VP]),
    "oci_nn_forward": (ctypes.c_int, [_VP, _VP, _I32, _I32, _VP, _VP, ctypes.c_size_t, _VP]),
    "oci_nn_predict": (ctypes.c_int, [_VP, _VP, _VP, _I32, _I32, _VP, _VP]),
    "oci_nn_loss_grad": (ctypes.c_int, [_VP, _VP, _VP, _I32, _I32, _VP, ctypes.POINTER(ctypes.c_double), _VP,
                                        ctypes.c_size_t, _VP]),
    "oci_nn_train_step": (ctypes.c_int, [_VP, _VP, _VP, _I32, ctypes.c_float, _VP, _VP, _I32, _I32,
                                         ctypes.POINTER(ctypes.c_double), _VP, ctypes.c_size_t, _VP]),
    "oci_nn_forward_noalloc": (ctypes.c_int, [_VP, _VP, _I32, _VP, _VP]),
    "oci_nn_train": (ctypes.c_int, [_VP, _VP, _VP]),
    "oci_last_cuda_error": (ctypes.c_char_p, [_VP]),
}

LIB_PATH = _build.LIB
_lib = None


def load_library(path: str = None):
    """Load the C-ABI library (raises if it has not been built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"CUDA library {p} is missing: build it with paper_2305_13555_gb300.build.build()")
    lib = ctypes.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


class OciError(RuntimeError):
    def __init__(self, code, msg=""):
        self.code = code
        super().__init__(f"{msg}: status {code} ({oci_strerror(code)})")


def oci_strerror(code: int) -> str:
    return load_library().oci_strerror(int(code)).decode()


def _f64(a, shape):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(shape))


def _ptr(a):
    return None if a is None else a.ctypes.data


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return None


def oci_create(prob: dict, precision="fp64", tol=None, max_iter=100000, stream=None):
    """Create a handle from a problem dict (see ``workloads``); returns an int handle."""
    J, N = int(prob["n_cells"]), int(prob["n_ord"])
    keep = {
        "dx": _f64(prob["dx"], (J,)), "sigma_t": _f64(prob["sigma_t"], (J,)),
        "sigma_s": _f64(prob["sigma_s"], (J,)),
        "q": None if prob.get("q") is None else _f64(prob["q"], (J, 4)),
        "bl": None if prob.get("psi_bc_left") is None else _f64(prob["psi_bc_left"], (N // 2, 2)),
        "br": None if prob.get("psi_bc_right") is None else _f64(prob["psi_bc_right"], (N // 2, 2)),
        "psi0": None if prob.get("psi0") is None else _f64(prob["psi0"], (J, N, 2)),
    }
    bcl, bcr = prob.get("bc_left", 0), prob.get("bc_right", 0)
    s = OciProblem(J, N, _ptr(keep["dx"]), _ptr(keep["sigma_t"]), _ptr(keep["sigma_s"]), _ptr(keep["q"]),
                   float(prob["v"]), float(prob["dt"]),
                   _BC[bcl] if isinstance(bcl, str) else int(bcl), _BC[bcr] if isinstance(bcr, str) else int(bcr),
                   _ptr(keep["bl"]), _ptr(keep["br"]), _ptr(keep["psi0"]),
                   _PREC[precision] if isinstance(precision, str) else int(precision), int(max_iter),
                   float(prob.get("tol", 1e-8) if tol is None else tol),
                   stream if stream is not None else _current_stream())
    h = ctypes.c_void_p()
    rc = load_library().oci_create(ctypes.byref(s), ctypes.byref(h))
    if rc != OCI_OK:
        raise OciError(rc, "oci_create")
    return h.value


def oci_destroy(h):
    load_library().oci_destroy(h)


def _check(rc, what, h=None):
    if rc != OCI_OK:
        extra = ""
        if rc == OCI_ECUDA and h is not None:
            extra = " " + load_library().oci_last_cuda_error(h).decode()
        raise OciError(rc, what + extra)


def oci_set_source(h, q):
    q = np.ascontiguousarray(q, dtype=np.float64)
    _check(load_library().oci_set_source(h, _ptr(q)), "oci_set_source", h)


def oci_set_iteration(h, tol, max_iter, commit_unconverged=False):
    _check(load_library().oci_set_iteration(h, float(tol), int(max_iter), int(bool(commit_unconverged))),
           "oci_set_iteration", h)


def oci_set_stream(h, stream):
    _check(load_library().oci_set_stream(h, stream), "oci_set_stream", h)


def oci_set_solver(h, solver):
    """OCI_SOLVER_WOODBURY (default) or OCI_SOLVER_DENSE (see oci.h); also "woodbury" / "dense"."""
    solver = _SOLVER.get(solver, solver)
    _check(load_library().oci_set_solver(h, int(solver)), "oci_set_solver", h)


def oci_set_sweep(h, sweep):
    """OCI_SWEEP_MARCH (default) or OCI_SWEEP_SCAN for si_step (see oci.h); also "march" / "scan"."""
    sweep = _SWEEP.get(sweep, sweep)
    _check(load_library().oci_set_sweep(h, int(sweep)), "oci_set_sweep", h)


def oci_set_wait_limits(h, poll_limit=0, barrier_shortfall=0):
    """Bounded-wait diagnostics (see oci.h): grid-barrier poll limit, missing arrivals."""
    _check(load_library().oci_set_wait_limits(h, int(poll_limit), int(barrier_shortfall)), "oci_set_wait_limits", h)


def oci_set_time_scheme(h, scheme):
    """OCI_TIME_MB (default) or OCI_TIME_BE (see oci.h); also "mb" / "be"."""
    scheme = _SCHEME.get(scheme, scheme)
    _check(load_library().oci_set_time_scheme(h, int(scheme)), "oci_set_time_scheme", h)


def oci_set_halo(h, halo):
    """OCI_HALO_FP32 (default) or OCI_HALO_BF16 for the OCI iteration's face buffers (see oci.h);
    also "fp32" / "bf16"."""
    halo = _HALO.get(halo, halo)
    _check(load_library().oci_set_halo(h, int(halo)), "oci_set_halo", h)


def oci_set_guess(h, guess):
    """OCI_GUESS_PREVIOUS (default) or OCI_GUESS_EXTRAPOLATE: the next step's
    initial iterate (see oci.h); also "previous" / "extrapolate"."""
    guess = _GUESS.get(guess, guess)
    _check(load_library().oci_set_guess(h, int(guess)), "oci_set_guess", h)


def oci_step(h):
    """One OCI time step; returns (status, stats dict).  Raises only on
    OCI_EINVAL / OCI_ECUDA; convergence failures come back as the status."""
    st = OciStats()
    rc = load_library().oci_step(h, ctypes.byref(st))
    if rc in (OCI_EINVAL, OCI_ECUDA, OCI_ENOMEM):
        _check(rc, "oci_step", h)
    return rc, st.as_dict()


def oci_step_async(h):
    """Enqueue one OCI step and return at once (see oci.h); raises on any error,
    OCI_ESTATE included (a step already pending, or a handle whose step needs the host)."""
    _check(load_library().oci_step_async(h), "oci_step_async", h)


def oci_step_wait(h):
    """Wait for the step oci_step_async enqueued; returns (status, stats dict) as oci_step."""
    st = OciStats()
    rc = load_library().oci_step_wait(h, ctypes.byref(st))
    if rc in (OCI_EINVAL, OCI_ECUDA, OCI_ENOMEM, OCI_ESTATE):
        _check(rc, "oci_step_wait", h)
    return rc, st.as_dict()


def oci_run_steps(h, n, q=None, phi=None):
    """n steps in one call (see oci.h): q [n][J][4] float64 sources or None (keep
    the current one), phi [n][J][4] float64 to receive each step's moments or
    None; both ideally page-locked.  Returns (status, steps committed, list of
    per-step stats dicts)."""
    for a in (q, phi):
        if a is not None and not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]):
            raise ValueError("q and phi must be C-contiguous float64 arrays")
    stats = (OciStats * max(n, 1))()
    done = ctypes.c_int32()
    rc = load_library().oci_run_steps(h, int(n), None if q is None else _ptr(q), None if phi is None else _ptr(phi),
                                      stats, ctypes.byref(done))
    if rc in (OCI_EINVAL, OCI_ECUDA, OCI_ENOMEM, OCI_ESTATE):
        _check(rc, "oci_run_steps", h)
    return rc, done.value, [stats[k].as_dict() for k in range(n)]


def oci_fluxes_async(h, out):
    """Enqueue the copy of the published moments into out ([J][4] float64, ideally
    page-locked); out is complete after the next oci_step_wait or oci_sync."""
    if not (isinstance(out, np.ndarray) and out.dtype == np.float64 and out.flags["C_CONTIGUOUS"]):
        raise ValueError("out must be a C-contiguous float64 array")
    _check(load_library().oci_fluxes_async(h, _ptr(out)), "oci_fluxes_async", h)


def oci_sync(h):
    _check(load_library().oci_sync(h), "oci_sync", h)


def si_step(h):
    st = OciStats()
    rc = load_library().si_step(h, ctypes.byref(st))
    if rc in (OCI_EINVAL, OCI_ECUDA, OCI_ENOMEM):
        _check(rc, "si_step", h)
    return rc, st.as_dict()


def oci_query(h):
    J, N = ctypes.c_int32(), ctypes.c_int32()
    _check(load_library().oci_query(h, ctypes.byref(J), ctypes.byref(N), None, None), "oci_query", h)
    mu, w = np.zeros(N.value), np.zeros(N.value)
    _check(load_library().oci_query(h, None, None, _ptr(mu), _ptr(w)), "oci_query", h)
    return J.value, N.value, mu, w


def oci_fluxes(h, out=None):
    J = oci_query(h)[0]
    out = np.zeros((J, 4)) if out is None else out
    _check(load_library().oci_fluxes(h, _ptr(out)), "oci_fluxes", h)
    return out


def oci_fluxes_device(h, dptr):
    _check(load_library().oci_fluxes_device(h, dptr), "oci_fluxes_device", h)


def oci_profile_iterations(h, n_iter):
    """Mean device seconds per launch of the OCI iteration kernel (see oci.h)."""
    sec = ctypes.c_double()
    _check(load_library().oci_profile_iterations(h, int(n_iter), ctypes.byref(sec)), "oci_profile_iterations", h)
    return sec.value


def oci_get_state(h):
    J, N, _, _ = oci_query(h)
    out = np.zeros((J, N, 2))
    _check(load_library().oci_get_state(h, _ptr(out)), "oci_get_state", h)
    return out


def oci_set_state(h, psi):
    psi = np.ascontiguousarray(psi, dtype=np.float64)
    _check(load_library().oci_set_state(h, _ptr(psi)), "oci_set_state", h)


def oci_dd_begin(h):
    _check(load_library().oci_dd_begin(h), "oci_dd_begin", h)


def oci_dd_export(h, out_left, out_right):
    """Outgoing cut fluxes into device tensors [N/2][2] of the handle's storage dtype (or None)."""
    _check(load_library().oci_dd_export(h, _dp(out_left), _dp(out_right)), "oci_dd_export", h)


def oci_dd_import(h, in_left, in_right):
    """Incident cut fluxes from device tensors [N/2][2] (or None: keep the face's own condition)."""
    _check(load_library().oci_dd_import(h, _dp(in_left), _dp(in_right)), "oci_dd_import", h)


def oci_dd_iterate(h):
    """One iteration of the sub-domain; returns its (sum dphi^2, sum phi^2)."""
    sums = np.zeros(2)
    _check(load_library().oci_dd_iterate(h, _ptr(sums)), "oci_dd_iterate", h)
    return sums


def oci_dd_decide(h, total):
    """The step's decision from the global sums: (done, status, stats)."""
    t = np.ascontiguousarray(total, dtype=np.float64)
    done = ctypes.c_int32()
    st = OciStats()
    rc = load_library().oci_dd_decide(h, _ptr(t), ctypes.byref(done), ctypes.byref(st))
    if rc not in (OCI_OK, OCI_ENOTCONV, OCI_ENAN):
        _check(rc, "oci_dd_decide", h)
    return bool(done.value), rc, st.as_dict()


class Solver:
    """Owns one handle.  ``step()`` / ``si_step()`` advance one time step."""

    def __init__(self, prob, precision="fp64", tol=None, max_iter=100000, stream=None, solver="woodbury",
                 sweep="march", scheme="mb", halo="fp32", guess="previous"):
        self.prob = prob
        self.h = oci_create(prob, precision, tol, max_iter, stream)
        try:
            if halo != "fp32":
                oci_set_halo(self.h, halo)
            if solver != "woodbury":
                oci_set_solver(self.h, solver)
            if sweep != "march":
                oci_set_sweep(self.h, sweep)
            if scheme != "mb":
                oci_set_time_scheme(self.h, scheme)
            if guess != "previous":
                oci_set_guess(self.h, guess)
        except Exception:
            self.close()
            raise

    def step(self, method="oci"):
        return (oci_step if method == "oci" else si_step)(self.h)

    def fluxes(self):
        return oci_fluxes(self.h)

    def get_state(self):
        return oci_get_state(self.h)

    def set_state(self, psi):
        oci_set_state(self.h, psi)

    def set_source(self, q):
        oci_set_source(self.h, q)

    def set_iteration(self, tol, max_iter, commit_unconverged=False):
        oci_set_iteration(self.h, tol, max_iter, commit_unconverged)

    def close(self):
        if self.h:
            oci_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ learned guess
# Thin wrappers of include/oci_nn.h taking torch CUDA tensors (device pointers).

def _dp(t):
    return None if t is None else t.data_ptr()


def _stream(stream):
    if stream is not None:
        return stream
    return _current_stream()


OCI_NN_OFF, OCI_NN_GUESS, OCI_NN_GUESS_CORRECT, OCI_NN_GUESS_ADAPTIVE = 0, 1, 2, 3


def oci_nn_attach(h, params, mode=OCI_NN_GUESS, k_corr=50):
    """Attach trained parameters (host float32 array) to a handle (see oci.h)."""
    p = None if params is None else np.ascontiguousarray(np.asarray(params, dtype=np.float32))
    _check(load_library().oci_nn_attach(h, None if p is None else p.ctypes.data, int(mode), int(k_corr)),
           "oci_nn_attach", h)


def oci_nn_static_features(h, stat, qfeat):
    _check(load_library().oci_nn_static_features(h, _dp(stat), _dp(qfeat)), "oci_nn_static_features", h)


def oci_nn_param_count():
    return int(load_library().oci_nn_param_count())


def oci_nn_workspace_bytes(batch, n_cells):
    return int(load_library().oci_nn_workspace_bytes(int(batch), int(n_cells)))


def oci_nn_features(phi1, phi2, stat, qfeat, inp, scale, stream=None):
    B, J = phi1.shape[0], phi1.shape[1]
    _check(load_library().oci_nn_features(_dp(phi1), _dp(phi2), _dp(stat), _dp(qfeat), B, J, _dp(inp), _dp(scale),
                                          _stream(stream)), "oci_nn_features")


def oci_nn_targets(phin, phi1, scale, tgt, stream=None):
    B, J = phin.shape[0], phin.shape[1]
    _check(load_library().oci_nn_targets(_dp(phin), _dp(phi1), _dp(scale), B, J, _dp(tgt), _stream(stream)),
           "oci_nn_targets")


def oci_nn_forward(params, inp, out, workspace, stream=None):
    B, J = inp.shape[0], inp.shape[2]
    _check(load_library().oci_nn_forward(_dp(params), _dp(inp), B, J, _dp(out), _dp(workspace),
                                         workspace.numel() * workspace.element_size(), _stream(stream)),
           "oci_nn_forward")


def oci_nn_predict(phi1, out, scale, phat, stream=None):
    B, J = phi1.shape[0], phi1.shape[1]
    _check(load_library().oci_nn_predict(_dp(phi1), _dp(out), _dp(scale), B, J, _dp(phat), _stream(stream)),
           "oci_nn_predict")


def oci_nn_loss_grad(params, inp, tgt, grad, workspace, stream=None):
    B, J = inp.shape[0], inp.shape[2]
    loss = ctypes.c_double()
    _check(load_library().oci_nn_loss_grad(_dp(params), _dp(inp), _dp(tgt), B, J, _dp(grad), ctypes.byref(loss),
                                           _dp(workspace), workspace.numel() * workspace.element_size(),
                                           _stream(stream)), "oci_nn_loss_grad")
    return loss.value


def oci_nn_train_step(params, m, v, step, lr, inp, tgt, workspace, want_loss=True, stream=None):
    B, J = inp.shape[0], inp.shape[2]
    loss = ctypes.c_double()
    _check(load_library().oci_nn_train_step(_dp(params), _dp(m), _dp(v), int(step), float(lr), _dp(inp), _dp(tgt),
                                            B, J, ctypes.byref(loss) if want_loss else None, _dp(workspace),
                                            workspace.numel() * workspace.element_size(), _stream(stream)),
           "oci_nn_train_step")
    return loss.value if want_loss else None



class OciNNTrainCfg(ctypes.Structure):
    _fields_ = [
        ("n_traj", ctypes.c_int32), ("n_steps", ctypes.c_int32), ("n_cells", ctypes.c_int32),
        ("phi", ctypes.c_void_p), ("stat", ctypes.c_void_p), ("qfeat", ctypes.c_void_p),
        ("epochs", ctypes.c_int32), ("batch", ctypes.c_int32), ("lr", ctypes.c_float), ("val_frac", ctypes.c_float),
        ("seed", ctypes.c_uint64), ("init_params", ctypes.c_void_p), ("stream", ctypes.c_void_p),
    ]


class OciNNTrainStats(ctypes.Structure):
    _fields_ = [
        ("epochs_done", ctypes.c_int32), ("steps_done", ctypes.c_int32), ("n_train", ctypes.c_int32),
        ("n_val", ctypes.c_int32), ("train_loss", ctypes.c_double), ("val_loss", ctypes.c_double),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def oci_nn_train(phi, stat, qfeat, weights_out, epochs=20, batch=32, lr=1e-3, val_frac=0.05, seed=0,
                 init_params=None, stream=None):
    """The library's training procedure (oci_nn_train in oci_nn.h) on device
    tensors phi [T][S+1][J][4] (float64), stat [T][J][4], qfeat [T][J] (float32);
    writes the trained parameters into the device tensor weights_out and
    returns the run's statistics."""
    T, S1, J = phi.shape[0], phi.shape[1], phi.shape[2]
    cfg = OciNNTrainCfg(T, S1 - 1, J, _dp(phi), _dp(stat), _dp(qfeat), int(epochs), int(batch), float(lr),
                        float(val_frac), int(seed) & ((1 << 64) - 1), _dp(init_params), _stream(stream))
    st = OciNNTrainStats()
    _check(load_library().oci_nn_train(ctypes.byref(cfg), _dp(weights_out), ctypes.byref(st)), "oci_nn_train")
    return st.as_dict()
