"""Why OCI is not wrapped in GMRES (Krylov acceleration of the OCI map): on the
whole-problem system of one time step (oracle.brute, assembled from the
balance equations), OCI is block Jacobi over cells, and GMRES preconditioned by
it -- i.e. GMRES whose operator is the OCI map -- needs about as many
applications of that map as plain OCI needs iterations on the deployment
family's thin, highly scattering cells: one application moves information one
cell, and no Krylov combination of k applications reaches further than k
cells.  Each GMRES iteration also pays the orthogonalisation, so on the GPU it
could only be slower.  Where OCI itself is slow for another reason -- thick,
highly scattering cells in steady state, S_64 -- GMRES does cut the
applications 2-5x, but on a bandwidth-bound device the Krylov basis traffic
(each basis vector a third of an OCI iteration's bytes, read twice per
GMRES iteration) costs as much as it saves at every restart size; and the
transient configurations converge in a handful of iterations.  CPU only
(scipy's GMRES as a library step)."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle
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


# ------------------------------------------------- S_64, thick and low-c cells
# Matrix-free on the oracle's own OCI iteration (the whole-problem matrix of a
# 256-cell S_64 slab would not fit): the map G(psi) of one iteration is affine,
# so the step's solution solves (I - B) psi = G(0) with B psi = G(psi) - G(0),
# and GMRES whose operator is I - B applies G once per iteration.

def _map_counts(prob, restarts, tol=1e-8):
    J, N = prob["n_cells"], prob["n_ord"]
    P = oracle.Problem(prob)
    pe = np.zeros((J, N, 2))
    n = J * N * 4
    _, w = np.polynomial.legendre.leggauss(N)
    calls = [0]

    def G(v):
        calls[0] += 1
        return oracle.oci_iteration(P, pe, v.reshape(J, N, 4))[0].ravel()

    g0 = G(np.zeros(n))
    x, phi, n_oci = np.zeros(n), np.zeros((J, 4)), 0
    while n_oci < 20000:  # plain OCI to a relative change of phi below tol
        xn = G(x)
        n_oci += 1
        phin = np.einsum("n,jnc->jc", w, xn.reshape(J, N, 4))
        done = np.linalg.norm(phin - phi) < tol * np.linalg.norm(phin)
        x, phi = xn, phin
        if done:
            break
    A = spla.LinearOperator((n, n), matvec=lambda v: v - (G(v) - g0))
    out = {}
    for m in restarts:
        calls[0] = 0
        xg, info = spla.gmres(A, g0, rtol=0.1 * tol, restart=m, maxiter=20000)
        assert info == 0
        phig = np.einsum("n,jnc->jc", w, xg.reshape(J, N, 4))
        assert np.abs(phig - phi).max() < 1e-5 * np.abs(phi).max()
        out[m] = calls[0]
    return n_oci, out


def _gpu_cost(apps, m):
    """Modelled device cost of GMRES(m) in OCI-iteration equivalents: one OCI
    application moves 24 B per cell-ordinate (FP32), a Krylov vector of the
    incident-flux halo 8 B (two FP32 words), and classical Gram-Schmidt reads
    each of the (on average (m + 1) / 2) basis vectors twice per iteration."""
    return apps * (1.0 + 2.0 * (m + 1) / 2.0 * 8.0 / 24.0)


def test_gmres_on_the_oci_map_thick_high_c_s64_saves_applications_not_bandwidth():
    """Steady state (v -> infinity), c = 0.99, 10 mfp cells, S_64: GMRES on the
    OCI map needs 2-4x fewer applications than plain OCI, but its basis
    traffic eats the saving on a bandwidth-bound device at every restart size."""
    prob = dict(workloads.homogeneous(256, 64, 1.0, 0.99, 10.0, 1.0, 0.05, 1.0, "vacuum", "vacuum"), v=float("inf"))
    n_oci, gm = _map_counts(prob, (5, 30))
    assert n_oci >= 60
    assert gm[30] < 0.5 * n_oci and gm[5] < 0.6 * n_oci, (n_oci, gm)
    for m, apps in gm.items():
        assert _gpu_cost(apps, m) > 0.9 * n_oci, (m, apps, n_oci)


def test_gmres_on_the_oci_map_transient_s64_saves_nothing():
    """The transient configurations (dt = 0.05, 1/(v dt) = 20 per mfp) converge
    in a handful of OCI iterations; GMRES needs at least as many applications."""
    prob = workloads.homogeneous(256, 64, 1.0, 0.99, 1.0, 1.0, 0.05, 1.0, "vacuum", "vacuum")
    n_oci, gm = _map_counts(prob, (30,))
    assert n_oci <= 10 and gm[30] >= n_oci, (n_oci, gm)


# ------------------------------------------- extrapolating the iterate itself
def _extrapolated_counts(prob, k, tol=1e-8, warm=3, smax=50.0, max_it=3000):
    """OCI iterations to tol from the previous step's flux, with (k > 0) the
    iterate extrapolated every k iterations along its last change by the
    estimated ratio rho of successive changes (the sign-aware least-squares
    estimate <dx_l, dx_{l-1}> / |dx_{l-1}|^2, used once two estimates agree to
    1 %): x <- x + rho / (1 - rho) dx, the classical removal of a dominant
    error mode (exact when one real mode dominates)."""
    J, N = prob["n_cells"], prob["n_ord"]
    P = oracle.Problem(prob)
    pe = np.asarray(oracle.run(prob, "oci", 0)["psi_edge"]).reshape(J, N, 2)
    for _ in range(warm):  # a few steps in, where the deployment steps are
        pe = oracle.run(prob, "oci", 1, tol=1e-12, psi_edge=pe)["psi_edge"].reshape(J, N, 2)
    _, w = np.polynomial.legendre.leggauss(N)
    x = np.concatenate([pe, pe], axis=2)
    phi = np.einsum("n,jnc->jc", w, x)
    dprev, rhos, it, applied = None, [], 0, 0
    while it < max_it:
        xn, phin = oracle.oci_iteration(P, pe, x)
        it += 1
        done = np.linalg.norm(phin - phi) < tol * np.linalg.norm(phin)
        dx = xn - x
        x, phi = xn, phin
        if done:
            break
        if dprev is not None:
            rhos.append(float(np.vdot(dx, dprev) / np.vdot(dprev, dprev)))
        dprev = dx
        if k and it % k == 0 and len(rhos) >= 2 and abs(rhos[-1] - rhos[-2]) < 0.01 * abs(rhos[-1]) \
                and abs(rhos[-1]) < 0.999:
            r = rhos[-1]
            x = x + max(min(r / (1 - r), smax), -0.5) * dx
            applied += 1
            dprev, rhos = None, []
    return it, applied


def test_extrapolating_the_oci_iterate_saves_little_on_thin_scattering_cells():
    """Why there is no residual-driven corrector: on the deployment family's
    thin, highly scattering cells the OCI error is not one slowly decaying
    mode that an estimate from the last changes could remove -- the
    extrapolation applies and the count barely moves (seed 101, 512 cells,
    S_16: 169 iterations plain, 150-165 with it)."""
    prob = workloads.config5_deploy(101, J=512, N=16, n_steps=10)
    n_plain, _ = _extrapolated_counts(prob, 0)
    n_ext, applied = _extrapolated_counts(prob, 10)
    assert n_plain >= 150 and applied >= 1
    assert n_ext > 0.85 * n_plain, (n_plain, n_ext, applied)
