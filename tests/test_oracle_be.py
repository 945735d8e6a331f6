"""Pins of the backward-Euler oracle (the paper's disabled section "Backward
Euler transient implementation": Sigma_hat = Sigma + 1/(v dt), the previous
step's angular flux as a source).  CPU only."""
import numpy as np
import pytest

import oracle
import workloads
from oracle import brute

BCS = [("vacuum", "vacuum"), ("reflect", "vacuum"), ("incident", "reflect"), ("reflect", "reflect"),
       ("vacuum", "incident")]


@pytest.mark.parametrize("bcl,bcr", BCS)
@pytest.mark.parametrize("N", [2, 4, 8])
def test_be_oci_and_si_converge_to_the_whole_problem_solve(bcl, bcr, N):
    """Both iterations reach the dense solve of all cells' SCB balances with
    Sigma_hat, assembled from the balance equations (not from A^+/A^-)."""
    prob = workloads.random_small(seed=40 + N, J=7, N=N, bc_left=bcl, bc_right=bcr)
    psi0 = np.asarray(prob["psi0"]).reshape(7, N, 2)
    _, ref = brute.be_run(prob, 3, psi0=psi0)
    for method in ("oci", "si"):
        r = oracle.run_be(prob, method, 3, tol=1e-14, max_iter=20000)
        assert r["status"] == 0
        assert np.abs(r["phi_steps"] - ref).max() < 1e-12 * np.abs(ref).max()


def test_be_infinite_medium_recurrence():
    """Reflecting slab, uniform material and source, psi0 = 0: every step is
    the exact BE recurrence (Sigma_a + 1/(v dt)) phi^n = Q + phi^{n-1}/(v dt)."""
    J, N, st, c, v, dt, Q = 9, 8, 1.0, 0.5, 1.0, 0.1, 1.0
    prob = workloads.homogeneous(J, N, sigma_t=st, c=c, dx=0.3, v=v, dt=dt, q=Q, bc_left="reflect",
                                 bc_right="reflect", n_steps=6, tol=1e-14)
    r = oracle.run_be(prob, "oci", 6, tol=1e-14, max_iter=10000)
    sa, tau = st * (1 - c), 1.0 / (v * dt)
    phi = 0.0
    for n in range(6):
        phi = (Q + tau * phi) / (sa + tau)
        assert np.abs(r["phi_steps"][n] - phi).max() < 1e-12
    # hand value of the first step: Q / (Sigma_a + 1/(v dt)) = 1 / 10.5
    assert abs(r["phi_steps"][0, 0, 0] - 1.0 / 10.5) < 1e-13


def test_be_particle_balance():
    """Summing the corner balances over ordinates and cells: production,
    absorption and storage against the leakage through both faces."""
    prob = workloads.random_small(seed=9, J=11, N=8, bc_left="incident", bc_right="vacuum")
    J, N = 11, 8
    psi0 = np.asarray(prob["psi0"]).reshape(J, N, 2)
    r = oracle.run_be(prob, "oci", 1, tol=1e-14, max_iter=20000)
    psi = r["psi"]
    mu, w = np.polynomial.legendre.leggauss(N)
    dx = np.asarray(prob["dx"])
    sa = np.asarray(prob["sigma_t"]) - np.asarray(prob["sigma_s"])
    q = np.asarray(prob["q"]).reshape(J, 4)
    tau = 1.0 / (prob["v"] * prob["dt"])
    phi = np.einsum("n,jnc->jc", w, psi)
    phi0 = np.einsum("n,jnc->jc", w, psi0)
    vol = np.sum((dx / 2)[:, None] * (tau * (phi - phi0) + sa[:, None] * phi - q[:, 2:4]))
    # leakage: outgoing minus incoming angular current at both faces
    P = N // 2
    bl = np.asarray(prob["psi_bc_left"]).reshape(P, 2)[:, 1]
    right = sum(w[m] * mu[m] * psi[J - 1, m, 1] for m in range(P, N))
    left_out = sum(w[m] * abs(mu[m]) * psi[0, m, 0] for m in range(P))
    left_in = sum(w[m] * mu[m] * bl[m - P] for m in range(P, N))
    assert abs(vol + right + left_out - left_in) < 1e-12 * (abs(vol) + abs(left_in))


def test_be_is_first_order_in_time():
    """Flat mode: phi(t) -> Q/Sigma_a (1 - exp(-Sigma_a v t)); BE's per-step
    factor 1/(1 + z) (z = Sigma_a v dt) makes the error at fixed t halve with dt."""
    st, c, v, Q, T = 1.0, 0.5, 1.0, 1.0, 0.4
    sa = st * (1 - c)
    errs = []
    for n in (4, 8, 16):
        dt = T / n
        prob = workloads.homogeneous(5, 4, sigma_t=st, c=c, dx=0.5, v=v, dt=dt, q=Q, bc_left="reflect",
                                     bc_right="reflect", n_steps=n, tol=1e-14)
        r = oracle.run_be(prob, "oci", n, tol=1e-14, max_iter=10000)
        exact = Q / sa * (1 - np.exp(-sa * v * T))
        errs.append(abs(r["phi_steps"][-1, 0, 0] - exact))
    assert 1.8 < errs[0] / errs[1] < 2.2 and 1.8 < errs[1] / errs[2] < 2.2


def _wall(c, dt, N=8):
    """The BE example of the paper's disabled section: a 10 cm wall, Sigma =
    0.5 /cm, dx = 0.5 cm, v = 2 cm/s, no flux inside, constant isotropic
    incident flux 1 at x = 0, vacuum at x = L (S_8 is a reading)."""
    J, P = 20, N // 2
    return {"n_cells": J, "n_ord": N, "dx": np.full(J, 0.5), "sigma_t": np.full(J, 0.5),
            "sigma_s": np.full(J, 0.5 * c), "q": np.zeros((J, 4)), "v": 2.0, "dt": dt,
            "bc_left": "incident", "bc_right": "vacuum", "psi_bc_left": np.ones((P, 2)), "psi_bc_right": None,
            "psi0": np.zeros((J, N, 2))}


@pytest.mark.parametrize("c", [0.5, 0.9, 0.99])
def test_be_oci_gains_on_si_as_the_time_step_shrinks(c):
    """The section's observation (its figure is missing, so trends only): the
    ratio N_SI / N_OCI of iterations to 1e-9 rises as dt shrinks, below 1 for
    long steps and above 1 for short enough ones."""
    ratios = []
    for dt in (10.0, 1.0, 0.1, 0.01, 0.001):
        p = _wall(c, dt)
        n_oci = oracle.run_be(p, "oci", 1, tol=1e-9, max_iter=100000)["iters"][0]
        n_si = oracle.run_be(p, "si", 1, tol=1e-9, max_iter=100000)["iters"][0]
        ratios.append(n_si / n_oci)
    assert all(b >= a for a, b in zip(ratios, ratios[1:])), ratios
    assert ratios[0] < 1.0 < ratios[-1], ratios
