"""GPU parity of the dense per-material inverse variant of OCI
(oci_set_solver(OCI_SOLVER_DENSE): (A - S)^{-1} formed once per material, one
GEMM per material per iteration) against the FP64 oracle, whose OCI iteration
factorises the same dense cell system (LU with partial pivoting).  FP64: 1e-12
relative, same iteration counts.  FP32: against the FP32 Woodbury kernels at
a fixed iteration count, within the FP32 bound of the Woodbury tests."""
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


def _run_fixed(prob, n_iter, n_steps, precision="fp64", solver="dense"):
    phis = []
    with pkg.Solver(prob, precision=precision, solver=solver) as s:
        s.set_iteration(0.0, n_iter, commit_unconverged=True)
        for _ in range(n_steps):
            rc, st = s.step()
            assert rc == pkg.OCI_ENOTCONV and st["iters"] == n_iter and st["committed"] == 1, (rc, st)
            phis.append(s.fluxes())
        state = s.get_state()
    return np.array(phis), state


# (N, J, boundaries): ragged cell counts, every boundary kind, several materials
CASES = [(2, 33, "reflect", "incident"), (8, 77, "vacuum", "vacuum"), (16, 45, "incident", "reflect"),
         (32, 21, "reflect", "reflect"), (64, 9, "vacuum", "incident")]


@pytest.mark.parametrize("N,J,bcl,bcr", CASES)
def test_dense_fixed_iterations_fp64(N, J, bcl, bcr):
    prob = workloads.random_small(seed=300 + N, J=J, N=N, bc_left=bcl, bc_right=bcr)
    ref = oracle.run(prob, "oci", 2, tol=0.0, max_iter=4, commit_unconverged=True)
    phis, state = _run_fixed(prob, 4, 2)
    assert _rel(phis, ref["phi_steps"]) < FP64_TOL
    assert _rel(state, ref["psi_edge"]) < FP64_TOL


def test_dense_converged_config1_fp64():
    prob = workloads.config1()
    ref = oracle.run(prob, "oci", prob["n_steps"], tol=prob["tol"], max_iter=100000)
    assert ref["status"] == 0
    with pkg.Solver(prob, precision="fp64", solver="dense") as s:
        for k in range(prob["n_steps"]):
            rc, st = s.step()
            assert rc == pkg.OCI_OK, (rc, st)
            assert st["iters"] == ref["iters"][k]
            assert _rel(s.fluxes(), ref["phi_steps"][k]) < FP64_TOL
        assert _rel(s.get_state(), ref["psi_edge"]) < FP64_TOL


def test_dense_matches_woodbury_heterogeneous_fp64():
    """Several materials (columns grouped per material, one GEMM each)."""
    prob = workloads.hetero(seed=11, J=3000, N=16, n_steps=2)
    out = {}
    for solver in ("woodbury", "dense"):
        with pkg.Solver(prob, precision="fp64", tol=1e-10, solver=solver) as s:
            its = []
            for _ in range(2):
                rc, st = s.step()
                assert rc == pkg.OCI_OK, (solver, rc, st)
                its.append(st["iters"])
            out[solver] = (its, s.fluxes(), s.get_state())
    assert out["dense"][0] == out["woodbury"][0]
    assert _rel(out["dense"][1], out["woodbury"][1]) < FP64_TOL
    assert _rel(out["dense"][2], out["woodbury"][2]) < FP64_TOL


def test_dense_config3_s128_fp64():
    """The S_128 slab (512 x 512 inverse): dense and Woodbury agree, sampled
    cells against the oracle's per-cell solve at the same iterate count."""
    prob = workloads.config3(n_steps=1)
    ref_w, _ = _run_fixed(prob, 3, 1, solver="woodbury")
    dense, _ = _run_fixed(prob, 3, 1, solver="dense")
    assert _rel(dense, ref_w) < FP64_TOL


def test_dense_fixed_iterations_fp32_vs_woodbury():
    prob = workloads.random_small(seed=77, J=500, N=32, bc_left="reflect", bc_right="vacuum")
    w, _ = _run_fixed(prob, 6, 2, precision="fp32", solver="woodbury")
    d, _ = _run_fixed(prob, 6, 2, precision="fp32", solver="dense")
    assert _rel(d, w) < FP32_TOL


def test_dense_invalid_solver():
    prob = workloads.random_small(seed=1, J=8, N=4)
    with pkg.Solver(prob) as s:
        with pytest.raises(pkg.OciError):
            pkg.oci_set_solver(s.h, 7)
