"""What the trained network (paper_2305_13555_gb300/data/cnn_weights.npy,
trained by paper_2305_13555_gb300.learned on 2000 OCI trajectories of 4096-cell
S_16 slabs) gains over plain OCI on a thin-cell deployment slab: fewer
iterations per converged step, and an answer as close to a tightly converged
FP64 solve as plain OCI's at the same tolerance."""
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


def _steps(prob, W, n, precision="fp32", tol=1e-8):
    its, phis = [], []
    with pkg.Solver(prob, precision=precision, tol=tol, max_iter=50000) as s:
        if W is not None:
            pkg.oci_nn_attach(s.h, W, pkg.OCI_NN_GUESS, 50)
        for _ in range(n):
            rc, st = s.step()
            assert rc == pkg.OCI_OK, (rc, st)
            its.append(st["iters"])
            phis.append(s.fluxes())
    return np.array(its), np.array(phis)


def _rel_l2(a, ref):
    return np.sqrt(((a - ref) ** 2).sum(axis=(1, 2)) / (ref ** 2).sum(axis=(1, 2)))


def test_trained_guess_saves_iterations_on_thin_cells():
    W = learned.load_weights()
    n = 6
    prob = workloads.config5_deploy(8, J=131072, N=64, n_steps=n)
    plain_it, plain_phi = _steps(prob, None, n)
    nn_it, nn_phi = _steps(prob, W, n)
    _, ref_phi = _steps(prob, None, n, precision="fp64", tol=1e-12)
    e_plain, e_nn = _rel_l2(plain_phi, ref_phi), _rel_l2(nn_phi, ref_phi)
    print("iterations plain", plain_it.tolist(), "with learned guess", nn_it.tolist())
    print("relative L2 error vs FP64 at 1e-12: plain", e_plain.tolist(), "learned", e_nn.tolist())
    assert nn_it.sum() < 0.85 * plain_it.sum()
    # Both stop on the same residual ||dphi|| / ||phi|| < 1e-8.  The error left
    # behind is that residual over (1 - rho); 175 iterations from O(1) to 1e-8
    # put rho near 0.9, i.e. errors of order 1e-7.  The guess must not make it
    # worse than plain OCI's by more than that order.
    assert np.all(e_plain < 1e-5)
    assert np.all(e_nn < np.maximum(3 * e_plain, 3e-7))


def test_adaptive_guess_falls_back_where_the_guess_does_not_pay():
    """OCI_NN_GUESS_ADAPTIVE: after two plain lead-in steps and its plain /
    guessed / guessed / plain trial it keeps the guess on the slabs where the
    guess saves iterations and drops it on those where it costs iterations
    (seeds 8 and 7, 9, 10 of the deployment family); every step still converges."""
    W = learned.load_weights()
    n = 9
    for seed, keep in ((8, True), (7, False), (9, False), (10, False)):
        prob = workloads.config5_deploy(seed, J=131072, N=64, n_steps=n)
        plain_it, _ = _steps(prob, None, n)
        its = []
        with pkg.Solver(prob, precision="fp32", tol=1e-8, max_iter=50000) as s:
            pkg.oci_nn_attach(s.h, W, pkg.OCI_NN_GUESS_ADAPTIVE, 50)
            for k in range(n):
                rc, st = s.step()
                assert rc == pkg.OCI_OK, (rc, st)
                its.append(st["iters"])
                guessed = k in (3, 4) or (k >= 6 and keep)
                assert st["nn_accepts"] == (1 if guessed else 0), (seed, k, st)
        print("seed", seed, "plain", plain_it.tolist(), "adaptive", its)
        if keep:
            assert sum(its[6:]) < 0.85 * sum(plain_it[6:].tolist())
        else:  # back on the plain path (states equal to within the tolerance)
            assert all(abs(a - b) <= 5 for a, b in zip(its[6:], plain_it[6:].tolist())), (its, plain_it)
