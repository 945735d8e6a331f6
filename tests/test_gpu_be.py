"""GPU parity of the backward-Euler time scheme (oci_set_time_scheme(OCI_TIME_BE))
against the FP64 oracle's BE OCI (dense 2N x 2N solve per cell): FP64 to 1e-12
at a fixed iteration count and with the oracle's iteration counts at
convergence; FP32 within the FP32 bound of the MB tests."""
import numpy as np
import pytest

import oracle
import paper_2305_13555_gb300 as pkg
import workloads

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32_TOL = 2e-6


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2305_13555_gb300 import build
    build.build()
    pkg.load_library()


def _rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(b).max(), 1e-300)


def _be_fixed(prob, n_iter, n_steps, precision="fp64"):
    phis = []
    with pkg.Solver(prob, precision=precision, scheme="be") as s:
        s.set_iteration(0.0, n_iter, commit_unconverged=True)
        for _ in range(n_steps):
            rc, st = s.step()
            assert rc == pkg.OCI_ENOTCONV and st["iters"] == n_iter and st["committed"] == 1, (rc, st)
            f = s.fluxes()
            assert np.array_equal(f[:, :2], f[:, 2:])
            phis.append(f[:, :2])
        state = s.get_state()
    return np.array(phis), state


BCS = [("vacuum", "vacuum"), ("reflect", "vacuum"), ("incident", "reflect"), ("reflect", "reflect"),
       ("vacuum", "incident")]


@pytest.mark.parametrize("bcl,bcr", BCS)
def test_be_fixed_iterations_fp64_boundaries(bcl, bcr):
    prob = workloads.random_small(seed=61, J=37, N=8, bc_left=bcl, bc_right=bcr)
    ref = oracle.run_be(prob, "oci", 3, tol=0.0, max_iter=3, commit_unconverged=True)
    phis, state = _be_fixed(prob, 3, 3)
    assert _rel(phis, ref["phi_steps"]) < FP64_TOL
    assert _rel(state, ref["psi"]) < FP64_TOL


@pytest.mark.parametrize("N,J", [(2, 300), (16, 77), (64, 45), (128, 21)])
def test_be_fixed_iterations_fp64_layouts(N, J):
    prob = workloads.random_small(seed=700 + N, J=J, N=N, bc_left="reflect", bc_right="incident")
    ref = oracle.run_be(prob, "oci", 2, tol=0.0, max_iter=4, commit_unconverged=True)
    phis, state = _be_fixed(prob, 4, 2)
    assert _rel(phis, ref["phi_steps"]) < FP64_TOL
    assert _rel(state, ref["psi"]) < FP64_TOL


def test_be_converged_config1_fp64():
    prob = workloads.config1()
    ref = oracle.run_be(prob, "oci", prob["n_steps"], tol=prob["tol"], max_iter=100000)
    assert ref["status"] == 0
    with pkg.Solver(prob, precision="fp64", scheme="be") as s:
        for k in range(prob["n_steps"]):
            rc, st = s.step()
            assert rc == pkg.OCI_OK, (rc, st)
            assert st["iters"] == ref["iters"][k]
            assert _rel(s.fluxes()[:, :2], ref["phi_steps"][k]) < FP64_TOL


def test_be_infinite_medium_fp64():
    J, N, st, c, v, dt, Q = 300, 16, 1.0, 0.5, 1.0, 0.1, 1.0
    prob = workloads.homogeneous(J, N, sigma_t=st, c=c, dx=0.3, v=v, dt=dt, q=Q, bc_left="reflect",
                                 bc_right="reflect", n_steps=4, tol=1e-13)
    sa, tau, phi = st * (1 - c), 1.0 / (v * dt), 0.0
    with pkg.Solver(prob, precision="fp64", tol=1e-13, scheme="be") as s:
        for _ in range(4):
            rc, stt = s.step()
            assert rc == pkg.OCI_OK
            phi = (Q + tau * phi) / (sa + tau)
            assert np.abs(s.fluxes() - phi).max() < 1e-11


def test_be_fp32_within_bound():
    prob = workloads.hetero(seed=5, J=4000, N=32, n_steps=3, dt=0.02)
    ref = oracle.run_be(prob, "oci", 3, tol=1e-11, max_iter=100000)
    with pkg.Solver(prob, precision="fp32", tol=1e-8, scheme="be") as s:
        for k in range(3):
            rc, st = s.step()
            assert rc == pkg.OCI_OK, (rc, st)
            assert _rel(s.fluxes()[:, :2], ref["phi_steps"][k]) < FP32_TOL


def test_be_and_mb_switch_on_one_handle():
    """The state carries over: MB steps, then BE steps, agree with a handle
    that ran the same sequence; si_step is refused under BE."""
    prob = workloads.random_small(seed=13, J=50, N=8, bc_left="reflect", bc_right="vacuum")
    ref_state = None
    with pkg.Solver(prob, precision="fp64", tol=1e-12) as s:
        s.step()
        mb_state = s.get_state()
        pkg.oci_set_time_scheme(s.h, "be")
        rc, st = s.step()
        assert rc == pkg.OCI_OK
        ref_state = s.get_state()
        with pytest.raises(pkg.OciError):
            s.step("si")
        pkg.oci_set_time_scheme(s.h, "mb")
        rc, st = s.step()
        assert rc == pkg.OCI_OK
    r = oracle.run_be(prob, "oci", 1, tol=1e-14, max_iter=100000, psi=mb_state)
    assert _rel(ref_state, r["psi"]) < 1e-10
