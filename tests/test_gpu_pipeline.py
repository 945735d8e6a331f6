"""Pipelined stepping through the C ABI (oci_step_async / oci_step_wait, the
next step's source staged on the copy stream while a step runs, the moments
copied out by oci_fluxes_async while the next step runs): the same iteration
counts and bit-identical moments as the synchronous calls, for time-dependent
sources, both precisions and a stalled FP32 step that needs the refinement."""
import numpy as np
import pytest

import paper_2305_13555_gb300 as pkg
import workloads
from paper_2305_13555_gb300 import learned

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2305_13555_gb300 import build
    build.build()
    pkg.load_library()


def _pinned(shape):
    import torch
    return torch.zeros(shape, dtype=torch.float64).pin_memory().numpy()


def _sources(prob, n):
    J = prob["n_cells"]
    q = np.asarray(prob["q"], dtype=np.float64).reshape(J, 4)
    return [q * (1.0 + 0.25 * k) + 0.1 * k for k in range(n)]


def _synchronous(prob, prec, qs):
    phis, its = [], []
    with pkg.Solver(prob, precision=prec, tol=1e-8 if prec == "fp32" else 1e-10) as s:
        for q in qs:
            s.set_source(q)
            rc, st = s.step()
            assert rc == pkg.OCI_OK, (rc, st)
            phis.append(s.fluxes())
            its.append((st["iters"], st["refined"]))
    return phis, its


def _pipelined(prob, prec, qs):
    n, J = len(qs), prob["n_cells"]
    q_pin = [_pinned((J, 4)) for _ in range(2)]
    bufs = [_pinned((J, 4)) for _ in range(2)]
    phis, its = [None] * n, []
    with pkg.Solver(prob, precision=prec, tol=1e-8 if prec == "fp32" else 1e-10) as s:
        q_pin[0][:] = qs[0]
        pkg.oci_set_source(s.h, q_pin[0])
        pkg.oci_step_async(s.h)
        for k in range(n):
            if k + 1 < n:
                q_pin[(k + 1) % 2][:] = qs[k + 1]
                pkg.oci_set_source(s.h, q_pin[(k + 1) % 2])  # staged while step k runs
            rc, st = pkg.oci_step_wait(s.h)
            assert rc == pkg.OCI_OK, (rc, st)
            its.append((st["iters"], st["refined"]))
            if k >= 1:
                phis[k - 1] = bufs[(k - 1) % 2].copy()  # complete: the copy stream was drained
            pkg.oci_fluxes_async(s.h, bufs[k % 2])
            if k + 1 < n:
                pkg.oci_step_async(s.h)
        pkg.oci_sync(s.h)
        phis[n - 1] = bufs[(n - 1) % 2].copy()
    return phis, its


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_pipelined_steps_match_synchronous_steps(prec):
    prob = workloads.hetero(seed=7, J=20000, N=64, n_steps=6, bc_left="reflect", bc_right="vacuum")
    qs = _sources(prob, 6)
    ref_phi, ref_its = _synchronous(prob, prec, qs)
    phi, its = _pipelined(prob, prec, qs)
    assert its == ref_its
    for a, b in zip(phi, ref_phi):
        assert np.array_equal(a, b)


def test_pipelined_stalled_step_is_refined(monkeypatch):
    monkeypatch.setenv("OCI_STALL_FLOOR", "1e-3")
    monkeypatch.setenv("OCI_STALL_ITERS", "-1")
    prob = workloads.hetero(seed=5, J=5000, N=16, n_steps=3, bc_left="reflect", bc_right="vacuum")
    qs = _sources(prob, 3)
    ref_phi, ref_its = _synchronous(prob, "fp32", qs)
    phi, its = _pipelined(prob, "fp32", qs)
    assert all(r == 1 for _, r in its) and its == ref_its
    for a, b in zip(phi, ref_phi):
        assert np.array_equal(a, b)


def test_pipeline_guards():
    prob = workloads.config2(N=32, c=0.9, dx=0.1, J=4096, n_steps=2)
    with pkg.Solver(prob, precision="fp32") as s:
        with pytest.raises(pkg.OciError):
            pkg.oci_step_wait(s.h)  # nothing pending
        pkg.oci_step_async(s.h)
        rc, _ = pkg.oci_step(s.h)
        assert rc == pkg.OCI_ESTATE
        with pytest.raises(pkg.OciError):
            pkg.oci_step_async(s.h)
        with pytest.raises(pkg.OciError):
            s.set_state(np.zeros((4096, 32, 2)))
        with pytest.raises(pkg.OciError):
            s.set_iteration(1e-8, 100)
        rc, st = pkg.oci_step_wait(s.h)
        assert rc == pkg.OCI_OK and st["iters"] > 0
        rc, _ = s.step()  # synchronous again
        assert rc == pkg.OCI_OK
        pkg.oci_nn_attach(s.h, learned.init_params(seed=1), pkg.OCI_NN_GUESS, 20)
        with pytest.raises(pkg.OciError):
            pkg.oci_step_async(s.h)  # the learned guess decides on the host
