"""OCI_GUESS_EXTRAPOLATE (oci_set_guess): the next step's initial iterate is
the linear extrapolation in time through the last two end-of-step fluxes.
Parity: a fixed number of iterations per step from that iterate, against the
oracle's OCI iteration started from the same iterate built here on the host
(first step: the end-of-step flux of the initial state, as without it);
FP64 to 1e-12, FP32 (the persistent loop, which commits in the same launch)
to the FP32 bound.  Then the property it is for: the same converged answer in
fewer iterations on a slowly converging transient."""
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


def _oracle_extrapolated(prob, n_iter, n_steps):
    """n_iter OCI iterations per step; Psi^(0) of step k > 1 = (pe + d/2, pe + d)
    with d = pe - pe_prev, the last two committed end-of-step fluxes."""
    J, N = prob["n_cells"], prob["n_ord"]
    pe = np.asarray(oracle.run(prob, "oci", 0)["psi_edge"]).reshape(J, N, 2).copy()
    pe_prev, phis = None, []
    for _ in range(n_steps):
        if pe_prev is None:
            psi = np.concatenate([pe, pe], axis=2)
        else:
            d = pe - pe_prev
            psi = np.concatenate([pe + 0.5 * d, pe + d], axis=2)
        for _ in range(n_iter):
            psi, phi = oracle.oci_iteration(prob, pe, psi)
        pe_prev, pe = pe, psi[:, :, 2:4].copy()
        phis.append(phi)
    return np.array(phis), pe


def _gpu_fixed(prob, n_iter, n_steps, precision):
    phis = []
    with pkg.Solver(prob, precision=precision, guess="extrapolate") as s:
        s.set_iteration(0.0, n_iter, commit_unconverged=True)
        for _ in range(n_steps):
            rc, st = s.step()
            assert rc == pkg.OCI_ENOTCONV and st["iters"] == n_iter and st["committed"] == 1, (rc, st)
            phis.append(s.fluxes())
        return np.array(phis), s.get_state()


@pytest.mark.parametrize("N,J,bcl,bcr", [(8, 200, "reflect", "incident"), (16, 77, "vacuum", "reflect"),
                                         (64, 45, "incident", "vacuum"), (128, 21, "reflect", "reflect")])
def test_extrapolated_iterate_fp64_matches_oracle(N, J, bcl, bcr):
    prob = workloads.random_small(seed=300 + N, J=J, N=N, bc_left=bcl, bc_right=bcr)
    ref_phi, ref_pe = _oracle_extrapolated(prob, 3, 4)
    phis, state = _gpu_fixed(prob, 3, 4, "fp64")
    assert _rel(phis, ref_phi) < FP64_TOL
    assert _rel(state, ref_pe) < FP64_TOL


def test_extrapolated_iterate_fp32_loop_matches_oracle():
    prob = workloads.random_small(seed=5, J=500, N=64, bc_left="reflect", bc_right="vacuum")
    ref_phi, ref_pe = _oracle_extrapolated(prob, 4, 3)
    phis, state = _gpu_fixed(prob, 4, 3, "fp32")
    assert _rel(phis, ref_phi) < FP32_TOL
    assert _rel(state, ref_pe) < FP32_TOL


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 1e-8)])
def test_extrapolation_keeps_the_answer_and_saves_iterations(precision, tol):
    """A thin, highly scattering transient (sigma_t dx 0.01-0.1, c 0.9-0.999,
    dt 0.02, 4096 cells, S_16): the converged fluxes of every step agree with
    the previous-flux start within what the tolerance leaves, and steps 3-8
    take fewer iterations in total."""
    n = 8
    prob = workloads.config5_deploy(9, J=4096, N=16, n_steps=n)
    out = {}
    for guess in ("previous", "extrapolate"):
        its, phis = [], []
        with pkg.Solver(prob, precision=precision, tol=tol, max_iter=100000, guess=guess) as s:
            for _ in range(n):
                rc, st = s.step()
                assert rc == pkg.OCI_OK, (guess, rc, st)
                its.append(st["iters"])
                phis.append(s.fluxes())
        out[guess] = (np.array(its), np.array(phis))
    (ip, pp), (ie, pe) = out["previous"], out["extrapolate"]
    print(precision, "iterations previous", ip.tolist(), "extrapolated", ie.tolist())
    assert _rel(pe, pp) < (1e-7 if precision == "fp64" else 2e-5)
    assert ie[2:].sum() < 0.9 * ip[2:].sum()


def test_set_guess_rejects_unknown_modes():
    prob = workloads.random_small(seed=1, J=16, N=4)
    with pkg.Solver(prob) as s:
        assert pkg.load_library().oci_set_guess(s.h, 2) == pkg.OCI_EINVAL
        pkg.oci_set_guess(s.h, pkg.OCI_GUESS_EXTRAPOLATE)
        pkg.oci_set_guess(s.h, "previous")


def test_learned_guess_on_the_extrapolated_iterate_keeps_the_answer():
    """The lift of a (random) network's prediction onto the extrapolated
    iterate: every step converges, to the answer of the plain start."""
    from paper_2305_13555_gb300 import learned
    n = 5
    prob = workloads.config5_deploy(11, J=4096, N=16, n_steps=n)
    phis = {}
    for guess, nn in (("previous", False), ("extrapolate", True)):
        with pkg.Solver(prob, precision="fp64", tol=1e-10, max_iter=100000, guess=guess) as s:
            if nn:
                pkg.oci_nn_attach(s.h, learned.init_params(seed=3), pkg.OCI_NN_GUESS, 50)
            out = []
            for _ in range(n):
                rc, st = s.step()
                assert rc == pkg.OCI_OK, (guess, rc, st)
                out.append(s.fluxes())
            phis[guess] = np.array(out)
    assert _rel(phis["extrapolate"], phis["previous"]) < 1e-7


@pytest.mark.parametrize("bcl,bcr", [("reflect", "vacuum"), ("vacuum", "reflect")])
def test_si_steps_after_extrapolated_commits_keep_the_answer(bcl, bcr):
    """OCI and SI steps alternating on a handle with the extrapolated start (an
    SI step starts from the committed moments and, at a reflecting right face,
    the extrapolated face it lags; its own commit leaves the end-of-step flux):
    every step converges to the answer of the same sequence without it."""
    n = 6
    prob = workloads.random_small(seed=41, J=300, N=16, bc_left=bcl, bc_right=bcr)
    out = {}
    for guess in ("previous", "extrapolate"):
        phis = []
        with pkg.Solver(prob, precision="fp64", tol=1e-11, guess=guess) as s:
            for k in range(n):
                rc, st = s.step("si" if k % 2 else "oci")
                assert rc == pkg.OCI_OK, (guess, k, rc, st)
                phis.append(s.fluxes())
        out[guess] = np.array(phis)
    assert _rel(out["extrapolate"], out["previous"]) < 1e-8


def test_extrapolated_iterate_full_size_fp64_and_fp32():
    """65536 cells, S_64 (the benchmark's launch configuration; FP32: the
    persistent loop that ends the step, extrapolating in its ring-streamed
    commit): two steps of two fixed iterations against the oracle's iteration
    from the host-built extrapolated iterate, on every output."""
    prob = workloads.config2(N=64, c=0.9, dx=0.1, J=65536, n_steps=2)
    ref_phi, ref_pe = _oracle_extrapolated(prob, 2, 2)
    phis, state = _gpu_fixed(prob, 2, 2, "fp64")
    assert _rel(phis, ref_phi) < FP64_TOL
    assert _rel(state, ref_pe) < FP64_TOL
    phis, state = _gpu_fixed(prob, 2, 2, "fp32")
    assert _rel(phis, ref_phi) < FP32_TOL
    assert _rel(state, ref_pe) < FP32_TOL


def _oracle_si_extrapolated(prob, n_iter, n_steps):
    """n_iter SI iterations per step; from step 2 on the iterate is extrapolated
    in time: the faces as in _oracle_extrapolated and the scalar flux the SI
    iteration starts from, e + (e - e_old)/2 (step average) and e + (e - e_old)
    (end), e / e_old the last two published end-of-step moments."""
    J, N = prob["n_cells"], prob["n_ord"]
    _, w = np.polynomial.legendre.leggauss(N)
    pe = np.asarray(oracle.run(prob, "si", 0)["psi_edge"]).reshape(J, N, 2).copy()
    e_prev = np.einsum("n,jnc->jc", w, pe)  # published end moments of the initial state
    pe_prev, e_old, phis = None, None, []
    for _ in range(n_steps):
        if pe_prev is None:
            psi = np.concatenate([pe, pe], axis=2)
            phi = np.einsum("n,jnc->jc", w, psi)
        else:
            d = pe - pe_prev
            psi = np.concatenate([pe + 0.5 * d, pe + d], axis=2)
            de = e_prev - e_old
            phi = np.concatenate([e_prev + 0.5 * de, e_prev + de], axis=1)
        for _ in range(n_iter):
            psi, phi = oracle.si_iteration(prob, pe, phi, psi)
        pe_prev, pe = pe, psi[:, :, 2:4].copy()
        e_old, e_prev = e_prev, phi[:, 2:4].copy()
        phis.append(phi)
    return np.array(phis), pe


@pytest.mark.parametrize("N,bcl,bcr", [(16, "reflect", "vacuum"), (16, "vacuum", "reflect"), (16, "incident", "reflect"),
                                       (2, "reflect", "reflect"), (4, "vacuum", "reflect"), (64, "reflect", "incident")])
def test_extrapolated_si_iterate_fp64_matches_oracle(N, bcl, bcr):
    """Also one and two lanes per cell (S_2, S_4), where a lane publishes
    several moments of its cell, and 32 (S_64)."""
    prob = workloads.random_small(seed=55 + N, J=150, N=N, bc_left=bcl, bc_right=bcr)
    ref_phi, ref_pe = _oracle_si_extrapolated(prob, 3, 4)
    phis = []
    with pkg.Solver(prob, precision="fp64", guess="extrapolate") as s:
        s.set_iteration(0.0, 3, commit_unconverged=True)
        for _ in range(4):
            rc, st = s.step("si")
            assert rc == pkg.OCI_ENOTCONV and st["iters"] == 3 and st["committed"] == 1, (rc, st)
            phis.append(s.fluxes())
        state = s.get_state()
    assert _rel(np.array(phis), ref_phi) < FP64_TOL
    assert _rel(state, ref_pe) < FP64_TOL
