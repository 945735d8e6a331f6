"""oci_run_steps: n steps in one call with the next step queued before the
host waits for the current one.  Its results must be those of n rounds of
oci_set_source / oci_step / oci_fluxes on a second handle, bit for bit (the
same kernels on the same inputs): on a slab that never stalls, on one whose
FP32 steps all stall and are refined on the host (the queued step is held,
then enqueued again), and when a step does not commit (later steps not run,
the handle keeps that step's source).  Also the one-at-a-time form of handles
that cannot queue (FP64)."""
import numpy as np
import pytest

import paper_2305_13555_gb300 as pkg
import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2305_13555_gb300 import build
    build.build()
    pkg.load_library()


def _sources(prob, n, seed):
    g = np.random.default_rng(seed)
    q0 = np.asarray(prob["q"], dtype=np.float64).reshape(prob["n_cells"], 4)
    return np.ascontiguousarray(np.stack([q0 * g.uniform(0.5, 1.5) for _ in range(n)]))


def _sequential(prob, q, precision, n, **kw):
    phis, its, refined = [], [], []
    with pkg.Solver(prob, precision=precision, tol=1e-8, **kw) as s:
        for k in range(n):
            pkg.oci_set_source(s.h, q[k])
            rc, st = s.step()
            assert rc == pkg.OCI_OK, (k, rc, st)
            phis.append(s.fluxes())
            its.append(st["iters"])
            refined.append(st["refined"])
        return np.array(phis), its, refined, s.get_state()


def _batched(prob, q, precision, n, **kw):
    J = prob["n_cells"]
    phi = np.full((n, J, 4), np.nan)
    with pkg.Solver(prob, precision=precision, tol=1e-8, **kw) as s:
        rc, done, stats = pkg.oci_run_steps(s.h, n, q, phi)
        return rc, done, stats, phi, s.get_state()


@pytest.mark.parametrize("precision,guess,halo", [("fp32", "previous", "fp32"), ("fp64", "previous", "fp32"),
                                                  ("fp32", "extrapolate", "fp32"), ("fp32", "previous", "bf16")])
def test_run_steps_equals_one_step_at_a_time(precision, guess, halo):
    """Queued (FP32 loop), and one at a time (FP64; the BF16-halo phase)."""
    n = 6
    prob = workloads.hetero(seed=21, J=20000, N=64, n_steps=n)
    q = _sources(prob, n, 1)
    ref_phi, ref_its, _, ref_state = _sequential(prob, q, precision, n, guess=guess, halo=halo)
    rc, done, stats, phi, state = _batched(prob, q, precision, n, guess=guess, halo=halo)
    assert rc == pkg.OCI_OK and done == n
    assert [st["iters"] for st in stats] == ref_its
    assert np.array_equal(phi, ref_phi)
    assert np.array_equal(state, ref_state)
    if precision == "fp32" and halo == "fp32":  # queued: prologue, the loop that commits, the source scaling (+ the first guess)
        assert [st["launches"] for st in stats] == [4] + [3] * (n - 1), stats


def test_run_steps_refines_stalled_steps_and_reruns_the_held_one(monkeypatch):
    """Every FP32 step stalls (the stall floor forced to 1e-3) and is refined on
    the host while the step behind it waits held: same fluxes, state and
    iteration counts as one step at a time."""
    monkeypatch.setenv("OCI_STALL_FLOOR", "1e-3")
    monkeypatch.setenv("OCI_STALL_ITERS", "-1")
    n = 4
    prob = workloads.config5_deploy(101, J=4096, N=64, n_steps=n)
    q = _sources(prob, n, 2)
    ref_phi, ref_its, ref_ref, ref_state = _sequential(prob, q, "fp32", n)
    assert all(ref_ref), ref_ref
    rc, done, stats, phi, state = _batched(prob, q, "fp32", n)
    assert rc == pkg.OCI_OK and done == n
    assert [st["refined"] for st in stats] == [1] * n
    assert [st["iters"] for st in stats] == ref_its
    assert np.array_equal(phi, ref_phi)
    assert np.array_equal(state, ref_state)


def test_run_steps_stops_at_a_step_that_does_not_commit():
    """Step 2's source is NaN: it ends with OCI_ENAN uncommitted, step 3 (queued
    behind it) does nothing, later ones are skipped; the state is that after
    step 1, and the handle keeps step 2's source, as after oci_set_source and a
    failed oci_step."""
    n = 4
    prob = workloads.hetero(seed=22, J=20000, N=64, n_steps=n)
    q = _sources(prob, n, 3)
    q[1, 100, 0] = np.nan
    rc, done, stats, phi, state = _batched(prob, q, "fp32", n)
    assert rc == pkg.OCI_ENAN and done == 1
    assert stats[0]["status"] == pkg.OCI_OK and stats[1]["status"] == pkg.OCI_ENAN and stats[1]["committed"] == 0
    assert [st["status"] for st in stats[2:]] == [pkg.OCI_ESKIPPED] * (n - 2)
    with pkg.Solver(prob, precision="fp32", tol=1e-8) as s:
        pkg.oci_set_source(s.h, q[0])
        assert s.step()[0] == pkg.OCI_OK
        assert np.array_equal(phi[0], s.fluxes())
        assert np.array_equal(state, s.get_state())
    # the handle's source is step 2's: a further step fails the same way
    with pkg.Solver(prob, precision="fp32", tol=1e-8) as s:
        rc, done, stats = pkg.oci_run_steps(s.h, 2, q[:2].copy())
        assert rc == pkg.OCI_ENAN and done == 1
        assert s.step()[0] == pkg.OCI_ENAN


def test_run_steps_without_sources_keeps_the_current_one():
    n = 3
    prob = workloads.hetero(seed=23, J=20000, N=64, n_steps=n)
    q = np.ascontiguousarray(np.stack([np.asarray(prob["q"], dtype=np.float64).reshape(-1, 4)] * n))
    ref_phi, ref_its, _, _ = _sequential(prob, q, "fp32", n)
    J = prob["n_cells"]
    phi = np.zeros((n, J, 4))
    with pkg.Solver(prob, precision="fp32", tol=1e-8) as s:
        rc, done, stats = pkg.oci_run_steps(s.h, n, None, phi)
    assert rc == pkg.OCI_OK and done == n and np.array_equal(phi, ref_phi)
    assert [st["iters"] for st in stats] == ref_its
