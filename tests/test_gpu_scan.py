"""GPU parity of the parallel-prefix SI sweep (oci_set_sweep(OCI_SWEEP_SCAN))
against the FP64 oracle's sequential SI sweep.  The scan evaluates the same
recurrence with a different association order, so FP64 agrees to rounding
(1e-12 relative) at a fixed iteration count and gives the oracle's iteration
counts at convergence; FP32 agrees with the FP32 march within the FP32 bound.
Cell counts span several 2048-cell segments with a ragged last segment."""
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


def _si_fixed(prob, n_iter, n_steps, precision="fp64", sweep="scan"):
    phis = []
    with pkg.Solver(prob, precision=precision, sweep=sweep) as s:
        s.set_iteration(0.0, n_iter, commit_unconverged=True)
        for _ in range(n_steps):
            rc, st = s.step("si")
            assert rc == pkg.OCI_ENOTCONV and st["iters"] == n_iter and st["committed"] == 1, (rc, st)
            phis.append(s.fluxes())
        state = s.get_state()
    return np.array(phis), state


BCS = [("vacuum", "vacuum"), ("reflect", "vacuum"), ("incident", "reflect"), ("reflect", "reflect"),
       ("vacuum", "incident")]


@pytest.mark.parametrize("bcl,bcr", BCS)
def test_scan_fixed_iterations_fp64_boundaries(bcl, bcr):
    prob = workloads.random_small(seed=41, J=4500, N=4, bc_left=bcl, bc_right=bcr)
    ref = oracle.run(prob, "si", 2, tol=0.0, max_iter=3, commit_unconverged=True)
    phis, state = _si_fixed(prob, 3, 2)
    assert _rel(phis, ref["phi_steps"]) < FP64_TOL
    assert _rel(state, ref["psi_edge"]) < FP64_TOL


@pytest.mark.parametrize("N,J", [(2, 2049), (8, 300), (16, 6000), (64, 2100)])
def test_scan_fixed_iterations_fp64_layouts(N, J):
    prob = workloads.random_small(seed=500 + N, J=J, N=N, bc_left="reflect", bc_right="incident")
    ref = oracle.run(prob, "si", 2, tol=0.0, max_iter=3, commit_unconverged=True)
    phis, state = _si_fixed(prob, 3, 2)
    assert _rel(phis, ref["phi_steps"]) < FP64_TOL
    assert _rel(state, ref["psi_edge"]) < FP64_TOL


def test_scan_converged_config1_fp64():
    prob = workloads.config1()
    ref = oracle.run(prob, "si", prob["n_steps"], tol=prob["tol"], max_iter=100000)
    assert ref["status"] == 0
    with pkg.Solver(prob, precision="fp64", sweep="scan") as s:
        for k in range(prob["n_steps"]):
            rc, st = s.step("si")
            assert rc == pkg.OCI_OK, (rc, st)
            assert st["iters"] == ref["iters"][k]
            assert _rel(s.fluxes(), ref["phi_steps"][k]) < FP64_TOL


def test_scan_matches_march_fp32_full_size():
    """The 65536-cell S_64 slab: 32 segments per chain."""
    prob = workloads.config2(64, 0.9, 0.1, J=65536, n_steps=1)
    march, _ = _si_fixed(prob, 3, 1, precision="fp32", sweep="march")
    scan, _ = _si_fixed(prob, 3, 1, precision="fp32", sweep="scan")
    assert _rel(scan, march) < FP32_TOL


def test_scan_and_march_switch_on_one_handle():
    prob = workloads.hetero(seed=3, J=5000, N=8, n_steps=3)
    with pkg.Solver(prob, precision="fp64", tol=1e-10) as a, pkg.Solver(prob, precision="fp64", tol=1e-10) as b:
        for sweep in ("scan", "march", "scan"):
            pkg.oci_set_sweep(a.h, sweep)
            ra, sa = a.step("si")
            rb, sb = b.step("si")
            assert ra == rb == pkg.OCI_OK and sa["iters"] == sb["iters"]
            assert _rel(a.fluxes(), b.fluxes()) < FP64_TOL
