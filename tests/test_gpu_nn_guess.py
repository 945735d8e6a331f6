"""The learned guess inside the OCI step.

The network only moves the initial iterate (and, in corrector mode, later
iterates, with a safeguard that restores the saved iterate when the residual
rises); the iteration still runs to the same tolerance.  So with ANY network
-- here an untrained one -- the converged moments must equal plain OCI's to the
convergence tolerance, and the oracle's.
"""
import numpy as np
import pytest

import oracle
import paper_2305_13555_gb300 as pkg
import workloads
from paper_2305_13555_gb300 import learned

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2305_13555_gb300 import build
    build.build()
    pkg.load_library()


def _run(prob, prec, mode, params, steps, tol, k=20):
    out, stats = [], []
    with pkg.Solver(prob, precision=prec, tol=tol) as s:
        if mode:
            pkg.oci_nn_attach(s.h, params, mode, k)
        for _ in range(steps):
            rc, st = s.step()
            assert rc == pkg.OCI_OK, (rc, st)
            out.append(s.fluxes())
            stats.append(st)
    return np.array(out), stats


@pytest.mark.parametrize("mode", [pkg.OCI_NN_GUESS, pkg.OCI_NN_GUESS_CORRECT])
@pytest.mark.parametrize("prec,tol,bound", [("fp64", 1e-12, 1e-9), ("fp32", 1e-8, 2e-6)])
def test_untrained_network_keeps_the_answer(mode, prec, tol, bound):
    prob = workloads.hetero(seed=21, J=3000, N=16, n_steps=4, tau_range=(0.01, 0.1), c_range=(0.9, 0.999),
                            bc_left="reflect", bc_right="vacuum")
    params = learned.init_params(seed=3)
    plain, _ = _run(prob, prec, 0, None, 4, tol)
    nn, stats = _run(prob, prec, mode, params, 4, tol, k=15)
    ref = oracle.run(prob, "oci", 4, tol=1e-12, max_iter=200000)
    scale = np.abs(ref["phi_steps"]).max()
    assert np.abs(nn - plain).max() / scale < bound
    assert np.abs(nn - ref["phi_steps"]).max() / scale < bound
    assert all(st["nn_accepts"] >= 1 for st in stats)
    if mode == pkg.OCI_NN_GUESS:
        assert all(st["nn_rejects"] == 0 for st in stats)


def test_set_state_restarts_the_network_history():
    """After oci_set_state the network's two previous steps are the new state's
    moments, so a restart from the initial condition replays the guessed steps."""
    prob = workloads.hetero(seed=21, J=3000, N=16, n_steps=4, tau_range=(0.01, 0.1), c_range=(0.9, 0.999),
                            bc_left="reflect", bc_right="vacuum")
    J, N = prob["n_cells"], prob["n_ord"]
    params = learned.init_params(seed=3)
    with pkg.Solver(prob, precision="fp32", tol=1e-8) as s:
        pkg.oci_nn_attach(s.h, params, pkg.OCI_NN_GUESS, 20)
        first = []
        for _ in range(3):
            rc, st = s.step()
            assert rc == pkg.OCI_OK and st["nn_accepts"] == 1
            first.append((st["iters"], s.fluxes()))
        s.set_state(np.zeros((J, N, 2)))
        for it, phi in first:
            rc, st = s.step()
            assert rc == pkg.OCI_OK and st["iters"] == it, (st, it)
            assert np.abs(s.fluxes() - phi).max() <= 1e-12 * np.abs(phi).max()


def test_attach_validation():
    prob = workloads.config1()
    with pkg.Solver(prob) as s:
        with pytest.raises(pkg.OciError):
            pkg.oci_nn_attach(s.h, None, pkg.OCI_NN_GUESS, 10)
        with pytest.raises(pkg.OciError):
            pkg.oci_nn_attach(s.h, learned.init_params(), 7, 10)
        with pytest.raises(pkg.OciError):
            pkg.oci_nn_attach(s.h, learned.init_params(), pkg.OCI_NN_GUESS_CORRECT, 0)
        pkg.oci_nn_attach(s.h, None, pkg.OCI_NN_OFF, 1)


def test_trajectory_generation_and_short_training():
    data = learned.trajectories(range(7, 15), J=512, N=8, n_steps=6)
    assert data["phi"].shape == (8, 7, 512, 4)
    assert (data["iters"] > 0).all()
    p1, st1 = learned.train(data, epochs=1, batch=4, lr=2e-3, log=None, val_frac=0.2)
    p, st = learned.train(data, epochs=6, batch=4, lr=2e-3, log=None, val_frac=0.2)
    assert st["epochs_done"] == 6 and st["steps_done"] == 6 * (st["n_train"] // 4)
    assert st["val_loss"] < st1["val_loss"]
    assert np.isfinite(p).all()
