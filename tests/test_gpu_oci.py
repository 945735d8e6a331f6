"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

FP64 mode must agree with the oracle to 1e-12 relative (max-norm of the
difference over the max-norm of the oracle's scalar flux / angular flux), both
at a fixed iteration count (same algorithm, same iterate) and at convergence
(same iteration counts).  FP32 mode stores the angular flux and per-ordinate
blocks in float, so its bound is derived from float rounding: relative error
of the scalar flux <= 2e-6 at convergence (a few float ulps, amplified by at
most ~1/(1-c) through the scattering coupling of the test problems).
"""
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


def _gpu_fixed(prob, method, n_iter, n_steps, precision="fp64"):
    phis, states = [], []
    with pkg.Solver(prob, precision=precision) as s:
        s.set_iteration(0.0, n_iter, commit_unconverged=True)
        for _ in range(n_steps):
            rc, st = s.step(method)
            assert rc == pkg.OCI_ENOTCONV and st["iters"] == n_iter and st["committed"] == 1, (rc, st)
            phis.append(s.fluxes())
            states.append(s.get_state())
    return np.array(phis), states[-1]


# (N, J): J spans several warp chunks plus a ragged tail for each lane layout
LAYOUTS = [(2, 300), (4, 150), (6, 70), (8, 200), (16, 77), (32, 45), (64, 45), (128, 21), (256, 11)]
BCS = [("vacuum", "vacuum"), ("reflect", "vacuum"), ("incident", "reflect"), ("reflect", "reflect"),
       ("vacuum", "incident")]


@pytest.mark.parametrize("method", ["oci", "si"])
@pytest.mark.parametrize("N,J", LAYOUTS)
def test_fixed_iterations_fp64_layouts(method, N, J):
    prob = workloads.random_small(seed=100 + N, J=J, N=N, bc_left="reflect", bc_right="incident")
    ref = oracle.run(prob, method, 2, tol=0.0, max_iter=4, commit_unconverged=True)
    phis, state = _gpu_fixed(prob, method, 4, 2)
    assert _rel(phis, ref["phi_steps"]) < FP64_TOL
    assert _rel(state, ref["psi_edge"]) < FP64_TOL


@pytest.mark.parametrize("method", ["oci", "si"])
@pytest.mark.parametrize("bcl,bcr", BCS)
def test_fixed_iterations_fp64_boundaries(method, bcl, bcr):
    prob = workloads.random_small(seed=7, J=37, N=8, bc_left=bcl, bc_right=bcr)
    ref = oracle.run(prob, method, 3, tol=0.0, max_iter=3, commit_unconverged=True)
    phis, state = _gpu_fixed(prob, method, 3, 3)
    assert _rel(phis, ref["phi_steps"]) < FP64_TOL
    assert _rel(state, ref["psi_edge"]) < FP64_TOL


@pytest.mark.parametrize("method", ["oci", "si"])
def test_converged_config1_fp64(method):
    prob = workloads.config1()
    ref = oracle.run(prob, method, prob["n_steps"], tol=prob["tol"], max_iter=100000)
    assert ref["status"] == 0
    with pkg.Solver(prob, precision="fp64") as s:
        for k in range(prob["n_steps"]):
            rc, st = s.step(method)
            assert rc == pkg.OCI_OK, (rc, st)
            assert st["iters"] == ref["iters"][k]
            assert _rel(s.fluxes(), ref["phi_steps"][k]) < FP64_TOL
        assert _rel(s.get_state(), ref["psi_edge"]) < FP64_TOL


@pytest.mark.parametrize("method", ["oci", "si"])
def test_converged_hetero_fp32_bound(method):
    prob = workloads.hetero(seed=11, J=3000, N=16, n_steps=3, bc_left="reflect", bc_right="vacuum")
    ref = oracle.run(prob, method, 3, tol=1e-8, max_iter=100000)
    assert ref["status"] == 0
    with pkg.Solver(prob, precision="fp32") as s:
        for k in range(3):
            rc, st = s.step(method)
            assert rc == pkg.OCI_OK, (rc, st)
            assert abs(st["iters"] - ref["iters"][k]) <= 2
            assert _rel(s.fluxes(), ref["phi_steps"][k]) < FP32_TOL


def test_fixed_iterations_fp32_bound():
    prob = workloads.random_small(seed=5, J=500, N=64, bc_left="reflect", bc_right="vacuum")
    ref = oracle.run(prob, "oci", 2, tol=0.0, max_iter=5, commit_unconverged=True)
    phis, state = _gpu_fixed(prob, "oci", 5, 2, precision="fp32")
    assert _rel(phis, ref["phi_steps"]) < FP32_TOL
    assert _rel(state, ref["psi_edge"]) < FP32_TOL


def test_full_size_config2_sampled_fp64_and_fp32():
    """65536 cells, S_64 (the benchmark's launch configuration): three fixed
    iterations of one step against the oracle on every output."""
    prob = workloads.config2(N=64, c=0.9, dx=0.1, J=65536, n_steps=1)
    ref = oracle.run(prob, "oci", 1, tol=0.0, max_iter=3, commit_unconverged=True)
    phis, state = _gpu_fixed(prob, "oci", 3, 1, "fp64")
    assert _rel(phis[0], ref["phi_steps"][0]) < FP64_TOL
    assert _rel(state, ref["psi_edge"]) < FP64_TOL
    phis, state = _gpu_fixed(prob, "oci", 3, 1, "fp32")
    assert _rel(phis[0], ref["phi_steps"][0]) < FP32_TOL


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("fp32", 2e-6)])
def test_infinite_medium_full_size(precision, tol):
    """Reflecting both faces, uniform source: every cell follows the flat-mode
    multiple-balance recurrence phi_{n+1/2} = g phi_{n-1/2} + h."""
    J, N, c, dt = 65536, 64, 0.9, 0.05
    prob = workloads.homogeneous(J, N, 1.0, c, 0.1, 1.0, dt, 1.0, "reflect", "reflect", tol=1e-13)
    tau, sa = 1.0 / dt, 1.0 - c
    den = sa * sa + 2 * sa * tau + 2 * tau * tau
    g, h = 2 * tau * tau / den, (sa + 2 * tau) / den
    prev = 0.0
    with pkg.Solver(prob, precision=precision, tol=1e-13 if precision == "fp64" else 1e-7) as s:
        for _ in range(4):
            rc, st = s.step("oci")
            assert rc == pkg.OCI_OK, (rc, st)
            nxt = g * prev + h
            avg = (1.0 + tau * prev - tau * nxt) / sa
            phi = s.fluxes()
            assert np.abs(phi[:, 2:] - nxt).max() < tol * nxt
            assert np.abs(phi[:, :2] - avg).max() < tol * avg
            prev = nxt


def test_not_converged_keeps_state_then_recovers():
    prob = workloads.config1()
    with pkg.Solver(prob, precision="fp64") as s:
        s.set_iteration(1e-14, 2)
        before = s.fluxes().copy()
        rc, st = s.step()
        assert rc == pkg.OCI_ENOTCONV and st["committed"] == 0 and st["iters"] == 2
        assert np.array_equal(s.fluxes(), before)
        s.set_iteration(1e-10, 100000)
        rc, st = s.step()
        assert rc == pkg.OCI_OK
    ref = oracle.run(prob, "oci", 1, tol=1e-10)
    assert st["iters"] == ref["iters"][0]


def test_nan_source_reported():
    prob = workloads.config1()
    with pkg.Solver(prob, precision="fp32") as s:
        q = np.array(prob["q"], dtype=float)
        q[30, 1] = np.nan
        s.set_source(q)
        rc, st = s.step()
        assert rc == pkg.OCI_ENAN and st["committed"] == 0


def test_state_roundtrip_and_time_dependent_source():
    prob = workloads.random_small(seed=3, J=120, N=16, bc_left="vacuum", bc_right="reflect")
    # oracle: step 1 with q, step 2 with 2q
    r1 = oracle.run(prob, "oci", 1, tol=1e-12)
    p2 = dict(prob)
    p2["q"] = 2.0 * np.asarray(prob["q"])
    r2 = oracle.run(p2, "oci", 1, tol=1e-12, psi_edge=r1["psi_edge"])
    with pkg.Solver(prob, precision="fp64", tol=1e-12) as s:
        s.step()
        st1 = s.get_state()
        assert _rel(st1, r1["psi_edge"]) < FP64_TOL
        s.set_source(p2["q"])
        s.step()
        assert _rel(s.fluxes(), r2["phi_steps"][0]) < FP64_TOL
    # resume from the oracle's state in a fresh handle
    with pkg.Solver(p2, precision="fp64", tol=1e-12) as s:
        s.set_state(r1["psi_edge"])
        s.step()
        assert _rel(s.fluxes(), r2["phi_steps"][0]) < FP64_TOL


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_set_state_restarts_the_trajectory(prec):
    """oci_set_state converts on the device: get_state returns what was set
    (exactly in FP64, to float rounding in FP32), and a handle restarted from
    the initial condition replays its own first steps."""
    prob = workloads.random_small(seed=17, J=333, N=32, bc_left="reflect", bc_right="incident")
    J, N = prob["n_cells"], prob["n_ord"]
    psi0 = np.asarray(prob["psi0"], dtype=np.float64).reshape(J, N, 2)
    tol = 1e-12 if prec == "fp64" else 1e-8
    with pkg.Solver(prob, precision=prec, tol=tol) as s:
        got = s.get_state()
        if prec == "fp64":
            assert np.array_equal(got, psi0)
        else:
            assert np.array_equal(got, psi0.astype(np.float32).astype(np.float64))
        first = []
        for _ in range(3):
            rc, st = s.step()
            assert rc == pkg.OCI_OK
            first.append((st["iters"], s.fluxes()))
        s.set_state(psi0)
        for it, phi in first:
            rc, st = s.step()
            assert rc == pkg.OCI_OK and st["iters"] == it
            assert _rel(s.fluxes(), phi) < 1e-13
        s.set_state(np.zeros((J, N, 2)))
        assert not s.get_state().any()


def test_steady_state_and_single_cell():
    prob = workloads.random_small(seed=9, J=1, N=2, bc_left="incident", bc_right="incident")
    prob["v"] = float("inf")
    for method in ("oci", "si"):
        ref = oracle.run(prob, method, 1, tol=1e-14)
        with pkg.Solver(prob, precision="fp64", tol=1e-14) as s:
            rc, _ = s.step(method)
            assert rc == pkg.OCI_OK
            assert _rel(s.fluxes(), ref["phi_steps"][0]) < FP64_TOL


def test_mirror_symmetry_config1_fp32():
    prob = workloads.config1()
    with pkg.Solver(prob, precision="fp32", tol=1e-7) as s:
        for _ in range(3):
            s.step()
        ph = s.fluxes()
    assert np.abs(ph[:, 0] - ph[::-1, 1]).max() < 1e-6 * np.abs(ph).max()


def test_torch_stream_and_device_fluxes():
    import torch
    prob = workloads.config1()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        with pkg.Solver(prob, precision="fp64", stream=stream.cuda_stream) as s:
            s.step()
            out = torch.empty((prob["n_cells"], 4), dtype=torch.float64, device="cuda")
            pkg.oci_fluxes_device(s.h, out.data_ptr())
            stream.synchronize()
            assert np.array_equal(out.cpu().numpy(), s.fluxes())


@pytest.mark.parametrize("N,J", [(4, 333), (16, 1000), (32, 515), (64, 2049), (128, 300)])
def test_staged_kernel_matches_unstaged(N, J, monkeypatch):
    """The TMA-staged persistent FP32 kernel and the plain one compute the same
    iterates up to float rounding order (the staged back-substitution forms
    A^{-1}(u + s phi) in one pass), and both match the oracle."""
    prob = workloads.random_small(seed=40 + N, J=J, N=N, bc_left="reflect", bc_right="reflect")
    ref = oracle.run(prob, "oci", 2, tol=0.0, max_iter=4, commit_unconverged=True)
    a = _gpu_fixed(prob, "oci", 4, 2, precision="fp32")
    monkeypatch.setenv("OCI_NO_TMA", "1")
    b = _gpu_fixed(prob, "oci", 4, 2, precision="fp32")
    assert _rel(a[0], b[0]) < 1e-6 and _rel(a[1], b[1]) < 1e-6
    assert _rel(a[0], ref["phi_steps"]) < FP32_TOL and _rel(b[0], ref["phi_steps"]) < FP32_TOL


@pytest.mark.parametrize("method", ["oci", "si"])
def test_fp32_ill_conditioned_capacitance(method):
    """c = 0.999 in optically thick cells: (I - s M)^{-1} has entries ~1/(1-c);
    the FP32 path's double-float capacitance solve keeps the FP32 bound."""
    prob = workloads.homogeneous(400, 16, 1.0, 0.999, 5.0, 1.0, 2.0, 1.0, "reflect", "vacuum", tol=1e-9)
    ref = oracle.run(prob, method, 3, tol=1e-9, max_iter=200000)
    assert ref["status"] == 0
    with pkg.Solver(prob, precision="fp32", tol=1e-8) as s:
        for k in range(3):
            rc, st = s.step(method)
            assert rc == pkg.OCI_OK, (rc, st)
            assert _rel(s.fluxes(), ref["phi_steps"][k]) < 5 * FP32_TOL


def test_fp32_refinement_forced(monkeypatch):
    """Force the FP32 refinement (stop as soon as the change is below 1e-3):
    r0 = G(h0) - h0 in FP64, the correction iterated in FP32; the committed
    steps match the FP64 path to the FP32 bound."""
    prob = workloads.hetero(seed=5, J=5000, N=16, n_steps=4, bc_left="reflect", bc_right="incident")
    prob["psi_bc_right"] = np.full((8, 2), 0.3)
    ref = []
    with pkg.Solver(prob, precision="fp64", tol=1e-10) as s:
        for _ in range(4):
            assert s.step()[0] == pkg.OCI_OK
            ref.append(s.fluxes())
    monkeypatch.setenv("OCI_STALL_FLOOR", "1e-3")
    monkeypatch.setenv("OCI_STALL_ITERS", "-1")
    with pkg.Solver(prob, precision="fp32", tol=1e-8) as s:
        for k in range(4):
            rc, st = s.step()
            assert rc == pkg.OCI_OK and st["refined"] == 1, (rc, st)
            assert _rel(s.fluxes(), ref[k]) < FP32_TOL


def test_fp32_stalling_trajectory_converges():
    """A training slab whose FP32 iteration stalls at the rounding-noise floor
    (seed 100044: the FP64 path needs ~35 iterations per step) now converges
    every step, via the refinement when needed, and matches the FP64 path."""
    prob = workloads.config5_train(100044, J=4096, N=16, n_steps=20)
    ref = []
    with pkg.Solver(prob, precision="fp64", tol=1e-8) as s:
        for _ in range(20):
            assert s.step()[0] == pkg.OCI_OK
            ref.append(s.fluxes())
    with pkg.Solver(prob, precision="fp32", tol=1e-8, max_iter=5000) as s:
        for k in range(20):
            rc, st = s.step()
            assert rc == pkg.OCI_OK, (k, rc, st)
            assert _rel(s.fluxes(), ref[k]) < FP32_TOL


def test_step_reports_its_kernel_launches():
    """oci_stats.launches: prologue, commit, the initial-iterate kernel of a
    first step, and the iteration launches: one per iteration (FP64: plain
    kernels in a WHILE body), or one persistent launch for all iterations that
    also ends the step (the staged FP32 path at S_64)."""
    prob = workloads.config2(64, 0.9, 0.1, J=4096, n_steps=2)
    for prec in ("fp32", "fp64"):
        with pkg.Solver(prob, precision=prec) as s:
            for k in range(2):
                rc, st = s.step()
                assert rc == pkg.OCI_OK, (rc, st)
                fixed = 2 + (1 if k == 0 else 0)
                if prec == "fp64":  # prologue, commit, [initial iterate], one launch per iteration
                    assert st["launches"] == fixed + st["iters"], (prec, st)
                else:  # prologue, [initial iterate], the persistent loop (which commits)
                    assert st["launches"] == fixed, st


def test_grid_barrier_wait_runs_out_and_the_device_recovers():
    """Failure path of the persistent FP32 iteration without a fault: a grid
    barrier that waits for one arrival more than the grid has (a flag nothing
    sets) gives up after a short poll limit; the step ends with OCI_ETIMEOUT,
    nothing is committed, and the next steps run normally and match a solver
    that never timed out."""
    prob = workloads.config2(64, 0.9, 0.1, J=65536, n_steps=3)
    with pkg.Solver(prob, precision="fp32") as s, pkg.Solver(prob, precision="fp32") as ref:
        pkg.oci_set_wait_limits(s.h, 2000, 1)
        rc, st = s.step()
        assert rc == pkg.OCI_ETIMEOUT and st["committed"] == 0, (rc, st)
        pkg.oci_set_wait_limits(s.h, 0, 0)
        for _ in range(2):
            rc, st = s.step()
            rc2, st2 = ref.step()
            assert rc == rc2 == pkg.OCI_OK and st["iters"] == st2["iters"], (st, st2)
            assert np.array_equal(s.fluxes(), ref.fluxes())


def test_persistent_loop_matches_one_launch_per_iteration(monkeypatch):
    """The FP32 persistent cooperative loop and the same kernel launched once per
    iteration (OCI_NO_LOOP) take the same iterations to the same fluxes."""
    prob = workloads.hetero(seed=21, J=20000, N=64, n_steps=3)
    out = {}
    for mode in ("loop", "per_launch"):
        if mode == "per_launch":
            monkeypatch.setenv("OCI_NO_LOOP", "1")
        with pkg.Solver(prob, precision="fp32", tol=1e-8) as s:
            its, phis = [], []
            for _ in range(3):
                rc, st = s.step()
                assert rc == pkg.OCI_OK, (mode, rc, st)
                its.append(st["iters"])
                phis.append(s.fluxes())
            out[mode] = (its, np.array(phis))
    assert out["loop"][0] == out["per_launch"][0]
    assert _rel(out["loop"][1], out["per_launch"][1]) < 1e-12


@pytest.mark.parametrize("N,J", [(64, 20000), (32, 9001), (128, 3001)])
def test_barrier_free_loop_matches_the_barrier_loop(monkeypatch, N, J):
    """The barrier-free persistent loop (OCI_ASYNC_LOOP=1: neighbour flags, a
    decision one iteration behind, three face buffers, the end of the step in
    the same launch) takes the barrier loop's iterations to the same fluxes and
    state; a stalled step still refines from the latest iterate, and a forced
    wait timeout ends the step with nothing committed."""
    prob = workloads.hetero(seed=21, J=J, N=N, n_steps=4, bc_left="reflect", bc_right="vacuum")
    out = {}
    for mode in ("barrier", "barrier_free"):
        if mode == "barrier_free":
            monkeypatch.setenv("OCI_ASYNC_LOOP", "1")
        with pkg.Solver(prob, precision="fp32", tol=1e-8) as s:
            its, phis = [], []
            for k in range(4):
                rc, st = s.step()
                assert rc == pkg.OCI_OK, (mode, rc, st)
                its.append(st["iters"])
                phis.append(s.fluxes())
                if mode == "barrier_free" and k > 0:
                    assert st["launches"] == 2, st  # prologue + the loop that also commits
            out[mode] = (its, np.array(phis), s.get_state())
    assert out["barrier"][0] == out["barrier_free"][0]
    assert _rel(out["barrier_free"][1], out["barrier"][1]) < 1e-12
    assert _rel(out["barrier_free"][2], out["barrier"][2]) < 1e-12
    # failure path: a decision that never comes (one arrival short) times out
    with pkg.Solver(prob, precision="fp32", tol=1e-8) as s:
        pkg.oci_set_wait_limits(s.h, 2000, 1)
        rc, st = s.step()
        assert rc == pkg.OCI_ETIMEOUT and st["committed"] == 0, (rc, st)
        pkg.oci_set_wait_limits(s.h, 0, 0)
        rc, st = s.step()
        assert rc == pkg.OCI_OK and st["iters"] == out["barrier"][0][0]
        assert _rel(s.fluxes(), out["barrier"][1][0]) < 1e-12


def test_barrier_free_loop_stalled_step_refines(monkeypatch):
    """A step that stalls in the barrier-free loop hands the latest iterate
    (wherever the three-buffer rotation left it) to the FP32 refinement."""
    monkeypatch.setenv("OCI_ASYNC_LOOP", "1")
    monkeypatch.setenv("OCI_STALL_FLOOR", "1e-3")
    monkeypatch.setenv("OCI_STALL_ITERS", "-1")
    prob = workloads.hetero(seed=5, J=4000, N=32, n_steps=3, dt=0.02)
    ref = oracle.run(prob, "oci", 3, tol=1e-11, max_iter=100000)
    with pkg.Solver(prob, precision="fp32", tol=1e-8) as s:
        for k in range(3):
            rc, st = s.step()
            assert rc == pkg.OCI_OK and st["refined"] == 1, (rc, st)
            assert _rel(s.fluxes(), ref["phi_steps"][k]) < FP32_TOL


def test_full_size_config4_converged_fp32_bound():
    """131072-cell seeded layered slab, S_64 (the benchmark's headline workload
    and launch configuration): three converged FP32 steps against the FP64 path
    converged to 1e-12 (itself the oracle's map to 1e-12 at a fixed iteration
    count, tests above), element-wise over every moment of every cell, within
    the FP32 bound."""
    prob = workloads.config4(seed=4, n_steps=3)
    with pkg.Solver(prob, precision="fp64", tol=1e-12) as s:
        ref = []
        for _ in range(3):
            rc, st = s.step("oci")
            assert rc == pkg.OCI_OK, (rc, st)
            ref.append(s.fluxes())
    with pkg.Solver(prob, precision="fp32", tol=1e-8) as s:
        for k in range(3):
            rc, st = s.step("oci")
            assert rc == pkg.OCI_OK, (rc, st)
            assert _rel(s.fluxes(), ref[k]) < FP32_TOL


def test_fp32_refinement_on_a_slowly_converging_slab(monkeypatch):
    """Thin, strongly scattering cells (the deployment family: the OCI map's
    spectral radius near 1) with the refinement forced early (as soon as the
    change is below 1e-3): the correction iteration must run to the tolerance
    itself -- its first iteration, from a zero correction, changes nothing and
    must not count as converged -- so the committed steps are as close to the
    tightly converged FP64 answer as an FP64 solve to the same tolerance."""
    prob = workloads.config5_deploy(101, J=4096, N=16, n_steps=3)
    ref, loose = [], []
    for tol, out in ((1e-12, ref), (1e-8, loose)):
        with pkg.Solver(prob, precision="fp64", tol=tol) as s:
            for _ in range(3):
                assert s.step()[0] == pkg.OCI_OK
                out.append(s.fluxes())
    monkeypatch.setenv("OCI_STALL_FLOOR", "1e-3")
    monkeypatch.setenv("OCI_STALL_ITERS", "-1")
    with pkg.Solver(prob, precision="fp32", tol=1e-8) as s:
        for k in range(3):
            rc, st = s.step()
            assert rc == pkg.OCI_OK and st["refined"] == 1, (rc, st)
            assert st["iters"] > 20, st  # the correction iterated, not one pass
            assert _rel(s.fluxes(), ref[k]) < 2 * _rel(loose[k], ref[k]) + FP32_TOL
