"""Plant plausible mistakes in copies of the C oracle and check the pins catch them.

Each mutant is compiled from a text-edited copy of ``oracle/oci_oracle.c`` in a
temporary directory (the oracle itself carries no mutation switches) and run
against the checks of test_oracle_pins: the whole-problem solve assembled from
the balance equations, numpy's Gauss-Legendre rule, and the infinite-medium
recurrence.  A mutant that still passes them would mean the pins are blind to
that kind of error.
"""
import os

import numpy as np
import pytest

import oracle
import workloads
from oracle import brute
from oracle import build as obuild

SRC = os.path.join(os.path.dirname(obuild.__file__), "oci_oracle.c")

MUTANTS = {
    # c^- sign of the incident term (time-average, right corner)
    "c_minus_sign": ("cm[1] = dx / 4.0 * Q[1] + e * pR - mu[m] * ink;",
                     "cm[1] = dx / 4.0 * Q[1] + e * pR + mu[m] * ink;"),
    # dropped time-edge term in c^+
    "c_plus_drop_time": ("cm[0] = dx / 4.0 * Q[0] + e * pL + mu[m] * ink;",
                         "cm[0] = dx / 4.0 * Q[0] + mu[m] * ink;"),
    # wrong sign of the lower streaming coupling in A^+/A^-
    "A_offdiag_sign": ("        -h,  d,    0.0,   e,", "        h,  d,    0.0,   e,"),
    # transposed scattering weight index (w_m instead of w_n)
    "S_weight_index": ("M[(size_t)(4 * m + i) * n4 + 4 * n + i] -= s * w[n];",
                       "M[(size_t)(4 * m + i) * n4 + 4 * n + i] -= s * w[m];"),
    # dt instead of dt/2 in the end-of-step equation (E = dx/(v dt) halved)
    "E_factor": ("const double E = dx / (v * dt);       /* dx / (v dt)   */",
                 "const double E = dx / (2.0 * v * dt); /* dx / (v dt)   */"),
    # SI: reflecting left face picks the same ordinate instead of its mirror
    "si_reflect_index": ("ink = psi_out[ix_psi(0, N - 1 - m, 0, N)];", "ink = psi_out[ix_psi(0, m - 1, 0, N)];"),
    # SI: scattering source lagged on the wrong moment
    "si_phi_moment": ("b[2] = dx / 4.0 * (ss * ph[2] + Q[2]) + mu * inh;",
                      "b[2] = dx / 4.0 * (ss * ph[0] + Q[2]) + mu * inh;"),
    # quadrature weights normalised to 1 instead of 2
    "gl_weight_norm": ("double wi = 2.0 / ((1.0 - x * x) * dp * dp);", "double wi = 1.0 / ((1.0 - x * x) * dp * dp);"),
    # upwind closure taken from the wrong corner of the upstream cell
    "upwind_corner": ("if (j > 0) return psi[ix_psi(j - 1, m, cR, N)];", "if (j > 0) return psi[ix_psi(j - 1, m, cL, N)];"),
    # OCI as forward Gauss-Seidel over cells: the mu > 0 incident flux read from the
    # left neighbour's new iterate (cells taken in order on one thread), not iterate l
    "oci_gauss_seidel": [
        ("const double ink = incident(p, mu, psi_in, j, m, 0);",
         "const double ink = incident(p, mu, (mu[m] > 0.0 && j > 0) ? psi_out : psi_in, j, m, 0);"),
        ("const double inh = incident(p, mu, psi_in, j, m, 1);",
         "const double inh = incident(p, mu, (mu[m] > 0.0 && j > 0) ? psi_out : psi_in, j, m, 1);"),
        ("#pragma omp parallel\n        {\n            double *c = malloc(sizeof(double) * (size_t)n4);\n"
         "#pragma omp for schedule(static)\n",
         "        {\n            double *c = malloc(sizeof(double) * (size_t)n4);\n"),
    ],
    # SI: reflecting left face lagged (iterate l) instead of the current sweep's mu < 0 flux
    "si_reflect_left_lagged": [
        ("ink = psi_out[ix_psi(0, N - 1 - m, 0, N)];", "ink = psi_in[ix_psi(0, N - 1 - m, 0, N)];"),
        ("inh = psi_out[ix_psi(0, N - 1 - m, 2, N)];", "inh = psi_in[ix_psi(0, N - 1 - m, 2, N)];"),
    ],
}


def _build_mutant(tmp_path, name):
    edits = MUTANTS[name]
    src = open(SRC).read()
    for old, new in ([edits] if isinstance(edits, tuple) else edits):
        assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
        src = src.replace(old, new)
    path = tmp_path / f"{name}.c"
    path.write_text(src)
    lib = obuild.build(force=True, src=str(path), out=str(tmp_path / f"lib{name}.so"))
    return oracle.load_library(lib)


def _map_fails(p, lib):
    """One OCI and one SI iteration from a random iterate against the splittings
    of the whole-problem matrix (the pins of test_oracle_map)."""
    J, N = int(p["n_cells"]), int(p["n_ord"])
    pe = np.asarray(p["psi0"]).reshape(J, N, 2)
    parts, b = brute.step_parts(p, pe)
    psi_l = np.random.default_rng(1).uniform(-0.5, 1.5, (J, N, 4))
    _, w = np.polynomial.legendre.leggauss(N)
    D = parts["own"] + parts["scatter"]
    R = parts["neighbour"] + parts["reflect_left"] + parts["reflect_right"]
    want = np.linalg.solve(D, b - R @ psi_l.ravel())
    got, _ = oracle.oci_iteration(p, pe, psi_l, lib=lib)
    if np.abs(got.ravel() - want).max() > 1e-12 * np.abs(want).max():
        return True
    L = parts["own"] + parts["neighbour"] + parts["reflect_left"]
    want = np.linalg.solve(L, b - (parts["scatter"] + parts["reflect_right"]) @ psi_l.ravel())
    got, _ = oracle.si_iteration(p, pe, np.einsum("n,jnc->jc", w, psi_l), psi_l, lib=lib)
    return bool(np.abs(got.ravel() - want).max() > 1e-12 * np.abs(want).max())


def _pins_fail(lib):
    """True if any pin detects the mutant."""
    mu, w = oracle.gauss_legendre(8, lib=lib)
    m2, w2 = np.polynomial.legendre.leggauss(8)
    if np.abs(mu - m2).max() > 1e-12 or np.abs(w - w2).max() > 1e-12:
        return True
    for bcl, bcr in (("reflect", "incident"), ("incident", "reflect")):
        p = workloads.random_small(seed=77, J=5, N=4, bc_left=bcl, bc_right=bcr)
        if _map_fails(p, lib):
            return True
        pe_b, ph_b = brute.run(p, 2)
        for method in ("oci", "si"):
            r = oracle.run(p, method, 2, tol=1e-13, max_iter=5000, lib=lib)
            if r["status"] != 0:
                return True
            if np.abs(r["phi_steps"] - ph_b).max() > 1e-9 * np.abs(ph_b).max():
                return True
    return False


def test_unmutated_copy_passes(tmp_path):
    src = open(SRC).read()
    path = tmp_path / "same.c"
    path.write_text(src)
    lib = oracle.load_library(obuild.build(force=True, src=str(path), out=str(tmp_path / "libsame.so")))
    assert not _pins_fail(lib)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    lib = _build_mutant(tmp_path, name)
    assert _pins_fail(lib), f"planted mistake {name} passed every pin"


# Planted mistakes in the backward-Euler part, caught by the BE pins (the
# whole-problem BE solve from the balance equations).
BE_MUTANTS = {
    # 1/(v dt) left out of Sigma_hat
    "be_sigma_hat": ("assemble_B_m(mu[m], dx, sig_hat, b);", "assemble_B_m(mu[m], dx, st, b);"),
    # previous-step source with the full-cell factor dx/(v dt)
    "be_edge_factor": ("const double e = dx / (2.0 * p->v * p->dt);\n    const double *Q = p->q + (size_t)j * 4;\n    c2[0]",
                       "const double e = dx / (p->v * p->dt);\n    const double *Q = p->q + (size_t)j * 4;\n    c2[0]"),
    # SI: outgoing corner of a mu < 0 cell taken from the wrong side
    "be_si_outgoing": ("in = mu[m] > 0.0 ? c2[1] : c2[0];  /* outgoing corner */",
                       "in = mu[m] > 0.0 ? c2[1] : c2[1];  /* outgoing corner */"),
}


def _be_pins_fail(lib):
    for bcl, bcr in (("reflect", "incident"), ("incident", "reflect")):
        p = workloads.random_small(seed=78, J=5, N=4, bc_left=bcl, bc_right=bcr)
        _, ph_b = brute.be_run(p, 2, psi0=np.asarray(p["psi0"]).reshape(5, 4, 2))
        for method in ("oci", "si"):
            r = oracle.run_be(p, method, 2, tol=1e-13, max_iter=5000, lib=lib)
            if r["status"] != 0 or np.abs(r["phi_steps"] - ph_b).max() > 1e-9 * np.abs(ph_b).max():
                return True
    return False


def test_unmutated_copy_passes_be_pins(tmp_path):
    path = tmp_path / "same_be.c"
    path.write_text(open(SRC).read())
    lib = oracle.load_library(obuild.build(force=True, src=str(path), out=str(tmp_path / "libsame_be.so")))
    assert not _be_pins_fail(lib)


@pytest.mark.parametrize("name", sorted(BE_MUTANTS))
def test_be_mutant_is_caught(tmp_path, name):
    old, new = BE_MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new))
    lib = oracle.load_library(obuild.build(force=True, src=str(path), out=str(tmp_path / f"lib{name}.so")))
    assert _be_pins_fail(lib), f"planted mistake {name} passed every BE pin"


@pytest.mark.parametrize("name", ["oci_gauss_seidel", "si_reflect_left_lagged"])
def test_map_mutants_keep_the_fixed_point(tmp_path, name):
    """These two mistakes change only the order of the iteration, not where it
    converges: the converged-solution pins alone pass them, and only the
    one-iteration map pin catches them."""
    lib = _build_mutant(tmp_path, name)
    for bcl, bcr in (("reflect", "incident"), ("incident", "reflect")):
        p = workloads.random_small(seed=77, J=5, N=4, bc_left=bcl, bc_right=bcr)
        _, ph_b = brute.run(p, 2)
        for method in ("oci", "si"):
            r = oracle.run(p, method, 2, tol=1e-13, max_iter=5000, lib=lib)
            assert r["status"] == 0
            assert np.abs(r["phi_steps"] - ph_b).max() <= 1e-9 * np.abs(ph_b).max()
    assert any(_map_fails(workloads.random_small(seed=77, J=5, N=4, bc_left=l, bc_right=r), lib)
               for l, r in (("reflect", "incident"), ("incident", "reflect")))
