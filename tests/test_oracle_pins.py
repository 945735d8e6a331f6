"""Pins for the FP64 oracle against facts fixed by the paper and the mathematics.

Each check comes from somewhere other than the oracle's own formulas:
  * Gauss-Legendre rule         -> numpy's leggauss (library routine);
  * converged OCI and SI        -> whole-problem dense solve assembled from the
                                   balance equations (oracle.brute), which the
                                   paper states both schemes converge to
                                   (Sec. "GPU Implementations": same solutions
                                   within the convergence criteria);
  * infinite medium             -> closed-form multiple-balance recurrence for
                                   the flat mode (derived from Eqs. 2-3);
  * particle balance            -> sum of Eqs. scb-mb-a..d over cells/ordinates;
  * mirror symmetry, c = 0 SI, second order in space and time (Sec. "Higher-
    order methods": SCB and MB are second-order accurate), spectral-radius
    trends (Sec. "One-Cell Inversion (OCI)", Fig. 1 text).
"""
import numpy as np
import pytest

import oracle
import workloads
from oracle import brute


# ----------------------------------------------------------------- quadrature

@pytest.mark.parametrize("n", [2, 4, 8, 16, 32, 64, 128, 256])
def test_gauss_legendre_matches_numpy(n):
    mu, w = oracle.gauss_legendre(n)
    m2, w2 = np.polynomial.legendre.leggauss(n)
    assert np.max(np.abs(mu - m2)) < 1e-14
    assert np.max(np.abs(w - w2)) < 1e-13
    assert abs(w.sum() - 2.0) < 1e-13   # the 1/2 of Eq. 1 implies sum w = 2
    assert np.all(np.diff(mu) > 0)


# ------------------------------------------------ converged = whole-problem solve

BC_CASES = [("vacuum", "vacuum"), ("reflect", "vacuum"), ("vacuum", "reflect"), ("incident", "incident"),
            ("reflect", "incident"), ("incident", "reflect"), ("reflect", "reflect")]


@pytest.mark.parametrize("method", ["oci", "si"])
@pytest.mark.parametrize("bcl,bcr", BC_CASES)
@pytest.mark.parametrize("N", [2, 4, 8])
def test_converged_equals_brute_force(method, bcl, bcr, N):
    p = workloads.random_small(seed=10 + N, J=6, N=N, bc_left=bcl, bc_right=bcr)
    pe_b, ph_b = brute.run(p, 3)
    r = oracle.run(p, method, 3, tol=1e-14, max_iter=20000)
    assert r["status"] == 0
    scale = np.abs(ph_b).max()
    assert np.abs(r["phi_steps"] - ph_b).max() / scale < 1e-12
    assert np.abs(r["psi_edge"] - pe_b).max() / np.abs(pe_b).max() < 1e-12


def test_oci_and_si_agree_thin_cells():
    p = workloads.random_small(seed=3, J=8, N=8, bc_left="reflect", bc_right="vacuum")
    p["dx"][:] = 0.02
    r1 = oracle.run(p, "oci", 2, tol=1e-14, max_iter=100000)
    r2 = oracle.run(p, "si", 2, tol=1e-14, max_iter=100000)
    pe_b, ph_b = brute.run(p, 2)
    assert r1["status"] == 0 and r2["status"] == 0
    for r in (r1, r2):
        assert np.abs(r["phi_steps"] - ph_b).max() / np.abs(ph_b).max() < 1e-11


def test_steady_state_limit_brute_force():
    """v -> infinity drops the time terms (the paper's steady-state calculations)."""
    p = workloads.random_small(seed=5, J=5, N=4, bc_left="incident", bc_right="vacuum", with_psi0=False)
    p["v"] = float("inf")
    pe_b, ph_b = brute.run(p, 1)
    for m in ("oci", "si"):
        r = oracle.run(p, m, 1, tol=1e-14, max_iter=20000)
        assert np.abs(r["phi_steps"] - ph_b).max() / np.abs(ph_b).max() < 1e-12


# ------------------------------------------------------------ closed forms

def _infinite_medium(sigma=1.0, c=0.5, v=1.0, dt=0.1, Q=1.0, J=6, N=4):
    p = workloads.homogeneous(J, N, sigma, c, 0.3, v, dt, Q, "reflect", "reflect")
    return p


def _mb_recurrence(sigma, c, v, dt, Q, n):
    """Flat-mode multiple balance: tau = 1/(v dt), Sa = sigma (1-c);
    phi_{n+1/2} = g phi_{n-1/2} + h, phi_n = (Q + tau phi_{n-1/2} - tau phi_{n+1/2}) / Sa."""
    tau, sa = 1.0 / (v * dt), sigma * (1.0 - c)
    den = sa * sa + 2 * sa * tau + 2 * tau * tau
    g, h = 2 * tau * tau / den, (sa + 2 * tau) * Q / den
    edge, avg, prev = [], [], 0.0
    for _ in range(n):
        nxt = g * prev + h
        avg.append((Q + tau * prev - tau * nxt) / sa)
        edge.append(nxt)
        prev = nxt
    return np.array(avg), np.array(edge)


@pytest.mark.parametrize("method", ["oci", "si"])
@pytest.mark.parametrize("c", [0.5, 0.9])
def test_infinite_medium_recurrence(method, c):
    p = _infinite_medium(c=c)
    r = oracle.run(p, method, 10, tol=1e-15, max_iter=5000)
    avg, edge = _mb_recurrence(1.0, c, 1.0, 0.1, 1.0, 10)
    ph = r["phi_steps"]
    for comp, ref in ((0, avg), (1, avg), (2, edge), (3, edge)):
        assert np.abs(ph[:, :, comp] - ref[:, None]).max() < 1e-12 * ref.max()


def test_infinite_medium_worked_values():
    # Sigma = 1, c = 0.5, v = 1, dt = 0.1, Q = 1: values of the recurrence above
    # evaluated once by hand (g = 0.9512485136741974).
    p = _infinite_medium(c=0.5)
    r = oracle.run(p, "oci", 10, tol=1e-15, max_iter=5000)
    ph = r["phi_steps"]
    assert abs(ph[0, 0, 2] - 0.09750297265160524) < 1e-14
    assert abs(ph[1, 0, 2] - 0.19025253046526064) < 1e-14
    assert abs(ph[2, 0, 2] - 0.27848040947943936) < 1e-14
    assert abs(ph[0, 0, 0] - 0.049940546967895294) < 1e-14
    assert abs(ph[9, 3, 3] - 0.7866952227018651) < 1e-13


def test_time_second_order():
    """Flat mode against the continuous solution phi(t) = Q/Sa (1 - exp(-Sa v t)):
    halving dt cuts the error about 4x (MB is second order, Sec. Higher-order)."""
    errs = []
    for dt in (0.2, 0.1, 0.05):
        n = int(round(1.0 / dt))
        p = _infinite_medium(c=0.5, dt=dt, J=3, N=2)
        r = oracle.run(p, "oci", n, tol=1e-15, max_iter=5000)
        exact = 1.0 / 0.5 * (1 - np.exp(-0.5 * 1.0))
        errs.append(abs(r["phi_steps"][-1, 0, 2] - exact))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.5 < r1 < 4.5 and 3.5 < r2 < 4.5, errs


def test_space_second_order():
    """Steady pure absorber, unit incident flux on the left (exact psi = exp(-x/mu)):
    the transmitted flux and the cell averages (psi_L + psi_R)/2 converge at second
    order (SCB is second-order accurate, Sec. Higher-order methods)."""
    X, N = 2.0, 4
    mu, _ = np.polynomial.legendre.leggauss(N)
    e_exit, e_avg = [], []
    for J in (20, 40, 80, 160):
        dx = X / J
        p = workloads.homogeneous(J, N, 1.0, 0.0, dx, float("inf"), 1.0, 0.0, "incident", "vacuum")
        p["psi_bc_left"] = np.ones((N // 2, 2))
        r = oracle.run(p, "oci", 1, tol=1e-15, max_iter=100000)
        x = np.arange(J) * dx
        ee = ea = 0.0
        for m in range(N // 2, N):
            avg = mu[m] / dx * (np.exp(-x / mu[m]) - np.exp(-(x + dx) / mu[m]))
            num = 0.5 * (r["psi_edge"][:, m, 0] + r["psi_edge"][:, m, 1])
            ea = max(ea, np.abs(num - avg).max())
            ee = max(ee, abs(r["psi_edge"][-1, m, 1] - np.exp(-X / mu[m])))
        e_exit.append(ee)
        e_avg.append(ea)
    r_exit = [e_exit[i] / e_exit[i + 1] for i in range(3)]
    r_avg = [e_avg[i] / e_avg[i + 1] for i in range(3)]
    assert all(3.6 < r < 4.4 for r in r_exit), (e_exit, r_exit)
    assert 3.3 < r_avg[-1] < 4.4 and r_avg[-1] > r_avg[0], (e_avg, r_avg)


# ---------------------------------------------------------------- invariants

def _converged_psi(p, psi_edge, tol=1e-15):
    """Iterate OCI to convergence from Psi^(0); returns converged Psi [J][N][4]."""
    J, N = p["n_cells"], p["n_ord"]
    pe = np.asarray(psi_edge).reshape(J, N, 2)
    psi = np.concatenate([pe, pe], axis=2)
    phi_old = None
    for _ in range(20000):
        psi, phi = oracle.oci_iteration(p, pe, psi)
        if phi_old is not None and np.linalg.norm(phi - phi_old) <= tol * np.linalg.norm(phi):
            break
        phi_old = phi
    return psi


@pytest.mark.parametrize("bcl,bcr", [("incident", "vacuum"), ("reflect", "incident"), ("vacuum", "vacuum")])
def test_particle_balance(bcl, bcr):
    """Summing Eqs. scb-mb-a+b (and c+d) over ordinates (weights w) and cells,
    streaming telescopes to the net boundary current."""
    p = workloads.random_small(seed=21, J=7, N=8, bc_left=bcl, bc_right=bcr)
    J, N, P = 7, 8, 4
    mu, w = np.polynomial.legendre.leggauss(N)
    pe = np.asarray(p["psi0"])
    psi = _converged_psi(p, pe)
    phi = np.einsum("n,jnc->jc", w, psi)
    phip = np.einsum("n,jnc->jc", w, pe)
    dx, st, ss, q = p["dx"], p["sigma_t"], p["sigma_s"], p["q"]
    sa = st - ss
    tau = 1.0 / (p["v"] * p["dt"])

    def edge_flux(t):
        cL, cR = (0, 1) if t == 0 else (2, 3)
        right = np.zeros(N); left = np.zeros(N)
        for m in range(N):
            if mu[m] > 0:
                right[m] = psi[J - 1, m, cR]
                left[m] = {"reflect": psi[0, N - 1 - m, cL],
                           "incident": p["psi_bc_left"][m - P, t], "vacuum": 0.0}[bcl]
            else:
                left[m] = psi[0, m, cL]
                right[m] = {"reflect": psi[J - 1, N - 1 - m, cR],
                            "incident": p["psi_bc_right"][P - 1 - m, t], "vacuum": 0.0}[bcr]
        return np.sum(w * mu * (right - left))

    bal_k = np.sum(dx / 2 * ((phi[:, 2] - phip[:, 0] + phi[:, 3] - phip[:, 1]) * tau
                             + sa * (phi[:, 0] + phi[:, 1]) - q[:, 0] - q[:, 1])) + edge_flux(0)
    bal_h = np.sum(dx / 2 * (2 * tau * (phi[:, 2] - phi[:, 0] + phi[:, 3] - phi[:, 1])
                             + sa * (phi[:, 2] + phi[:, 3]) - q[:, 2] - q[:, 3])) + edge_flux(1)
    scale = np.sum(dx * np.abs(q).sum(1))
    assert abs(bal_k) < 1e-11 * scale and abs(bal_h) < 1e-11 * scale


@pytest.mark.parametrize("method", ["oci", "si"])
def test_mirror_symmetry_config1(method):
    p = workloads.config1()
    r = oracle.run(p, method, 10, tol=1e-13, max_iter=20000)
    assert r["status"] == 0
    ph = r["phi_steps"]
    assert np.abs(ph[:, :, 0] - ph[:, ::-1, 1]).max() < 1e-11 * np.abs(ph).max()
    assert np.abs(ph[:, :, 2] - ph[:, ::-1, 3]).max() < 1e-11 * np.abs(ph).max()


def test_si_pure_absorber_converges_in_one_sweep():
    p = workloads.random_small(seed=8, J=9, N=8, bc_left="incident", bc_right="incident")
    p["sigma_s"][:] = 0.0
    r = oracle.run(p, "si", 2, tol=1e-300, max_iter=2, commit_unconverged=True)
    # iteration 2 reproduces iteration 1 exactly: relative change 0
    assert r["resid"][0] == 0.0 and r["resid"][1] == 0.0


def test_fixed_iteration_driver_matches_manual_iterations():
    p = workloads.random_small(seed=9, J=5, N=4, bc_left="reflect", bc_right="incident")
    r = oracle.run(p, "oci", 1, tol=0.0, max_iter=3, commit_unconverged=True)
    pe = p["psi0"]
    psi = np.concatenate([pe, pe], axis=2)
    for _ in range(3):
        psi, phi = oracle.oci_iteration(p, pe, psi)
    assert np.array_equal(r["phi_steps"][0], phi)
    assert np.array_equal(r["psi_edge"], psi[:, :, 2:4])


# ------------------------------------------------------------ spectral radii

def _oci_iteration_matrix(p):
    J, N = p["n_cells"], p["n_ord"]
    n = J * N * 4
    pe = np.zeros((J, N, 2))
    B = np.zeros((n, n))
    for i in range(n):
        e = np.zeros(n); e[i] = 1.0
        B[:, i] = oracle.oci_iteration(p, pe, e.reshape(J, N, 4))[0].ravel()
    return B


def _si_iteration_matrix(p):
    J, N = p["n_cells"], p["n_ord"]
    nf, npsi = J * 4, J * N * 4
    pe = np.zeros((J, N, 2))
    B = np.zeros((nf + npsi, nf + npsi))
    for i in range(nf + npsi):
        e = np.zeros(nf + npsi); e[i] = 1.0
        po, ph = oracle.si_iteration(p, pe, e[:nf].reshape(J, 4), e[nf:].reshape(J, N, 4))
        B[:nf, i] = ph.ravel(); B[nf:, i] = po.ravel()
    return B


def _rho(B):
    return np.max(np.abs(np.linalg.eigvals(B)))


def test_spectral_radius_trends():
    """S_4, steady state, infinite medium via reflecting boundaries (Fig. 1 text):
    rho_OCI falls as the cell optical thickness grows and rises with c; rho_SI
    depends on c and, for slabs many mean free paths thick, hardly on the cell
    thickness, approaching the textbook infinite-medium value c.  (The lagged
    reflecting right face adds slow modes in thin slabs, so rho_SI >= c.)"""
    J, N = 20, 4
    rho_oci, rho_si = {}, {}
    for c in (0.5, 0.9):
        for sdx in (0.1, 1.0, 10.0):
            p = workloads.homogeneous(J, N, 1.0, c, sdx, float("inf"), 1.0, 0.0, "reflect", "reflect")
            rho_oci[c, sdx] = _rho(_oci_iteration_matrix(p))
            rho_si[c, sdx] = _rho(_si_iteration_matrix(p))
    for c in (0.5, 0.9):
        assert rho_oci[c, 0.1] > rho_oci[c, 1.0] > rho_oci[c, 10.0]
        for sdx in (0.1, 1.0, 10.0):
            assert rho_si[c, sdx] >= c - 1e-10
        assert abs(rho_si[c, 1.0] - c) < 0.05 and abs(rho_si[c, 10.0] - c) < 0.05
        assert abs(rho_si[c, 1.0] - rho_si[c, 10.0]) < 0.03
    for sdx in (0.1, 1.0, 10.0):
        assert rho_oci[0.9, sdx] > rho_oci[0.5, sdx]
        assert rho_si[0.9, sdx] > rho_si[0.5, sdx]
    assert rho_oci[0.5, 10.0] < 0.2 and rho_oci[0.9, 0.1] > 0.9
