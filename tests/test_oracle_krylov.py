"""Why OCI is not wrapped in GMRES (Krylov acceleration of the OCI map): on the
whole-problem system of one time step (oracle.brute, assembled from the
balance equations), OCI is block Jacobi over cells, and GMRES preconditioned by
it -- i.e. GMRES whose operator is the OCI map -- needs about as many
applications of that map as plain OCI needs iterations on the deployment
family's thin, highly scattering cells: one application moves information one
cell, and no Krylov combination of k applications reaches further than k
cells.  Each GMRES iteration also pays the orthogonalisation, so on the GPU it
could only be slower.  CPU only (scipy's GMRES as a library step)."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import workloads
from oracle import brute


def _counts(prob, tol=1e-8, restart=30):
    J, N = prob["n_cells"], prob["n_ord"]
    M, rhs = brute.step_system(prob, np.zeros((J, N, 2)))
    M = sp.csr_matrix(M)
    nb = 4 * N
    blocks = [M[j * nb:(j + 1) * nb, j * nb:(j + 1) * nb].toarray() for j in range(J)]
    Dinv = sp.csr_matrix(sp.block_diag([np.linalg.inv(b) for b in blocks]))
    R = M - sp.csr_matrix(sp.block_diag(blocks))
    x = np.zeros_like(rhs)
    n_oci = 0
    while n_oci < 20000:  # OCI: every cell solved from its neighbours' previous iterate
        xn = Dinv @ (rhs - R @ x)
        n_oci += 1
        done = np.linalg.norm(xn - x) < tol * np.linalg.norm(xn)
        x = xn
        if done:
            break
    A = spla.LinearOperator(M.shape, matvec=lambda v: Dinv @ (M @ v))
    n_gm = [0]
    xg, info = spla.gmres(A, Dinv @ rhs, rtol=0.1 * tol, restart=restart, maxiter=5000,
                          callback=lambda r: n_gm.__setitem__(0, n_gm[0] + 1), callback_type="pr_norm")
    x_ref = spla.spsolve(M.tocsc(), rhs)
    return n_oci, n_gm[0], x, xg, x_ref


@pytest.mark.parametrize("seed", [8, 9])
def test_gmres_on_the_oci_map_does_not_save_applications(seed):
    prob = workloads.config5_deploy(seed, J=256, N=16, n_steps=1)
    prob["bc_left"] = prob["bc_right"] = "vacuum"
    n_oci, n_gm, x, xg, x_ref = _counts(prob)
    scale = np.linalg.norm(x_ref)
    assert np.linalg.norm(x - x_ref) < 1e-6 * scale and np.linalg.norm(xg - x_ref) < 1e-6 * scale
    assert n_oci >= 50  # a slowly converging step of the deployment family
    assert n_gm >= 0.9 * n_oci, (n_oci, n_gm)
