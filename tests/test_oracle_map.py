"""Pins for the oracle's one-iteration maps (not only their fixed point).

The converged-solution pins (test_oracle_pins) fix where OCI and SI end up, but
a scheme that reads a neighbour's already-updated iterate (Gauss-Seidel instead
of block Jacobi) or lags a face the paper keeps current ends up at the same
place.  The GPU fixed-iteration parity tests compare iterates, so the map
itself needs a pin.

Both maps are splittings of the one whole-problem matrix of a time step, which
``oracle.brute.step_parts`` assembles straight from the balance equations
(Eqs. scb-mb-a..d), independently of ``oci_oracle.c``:

  * OCI (Sec. "One-Cell Inversion (OCI)": every cell solved with its incident
    fluxes from iterate l): keep each cell's own block implicit -- streaming,
    collision, time and scattering -- and lag every coupling that leaves the
    cell's unknowns, i.e. the neighbours' corners and the reflecting faces
    (the mirror ordinate of a reflecting face is also read from iterate l):
        D psi^{l+1} = b - R psi^l,  D = own + scatter,
        R = neighbour + reflect_left + reflect_right.
  * SI (Sec. "Source Iteration (SI)": sweeps along each ordinate with the
    scattering source from the previous iterate; mu < 0 swept first, so a
    reflecting left face takes the current sweep and a reflecting right face
    iterate l):
        L psi^{l+1} = b - (scatter + reflect_right) psi^l,
        L = own + neighbour + reflect_left.
"""
import numpy as np
import pytest

import oracle
import workloads
from oracle import brute

BC_CASES = [("vacuum", "vacuum"), ("reflect", "vacuum"), ("vacuum", "reflect"), ("incident", "incident"),
            ("reflect", "incident"), ("incident", "reflect"), ("reflect", "reflect")]


def _random_iterate(seed, J, N):
    return np.random.default_rng(seed).uniform(-0.5, 1.5, (J, N, 4))


def _oci_map(parts, b, psi_l):
    D = parts["own"] + parts["scatter"]
    R = parts["neighbour"] + parts["reflect_left"] + parts["reflect_right"]
    return np.linalg.solve(D, b - R @ psi_l.ravel())


def _si_map(parts, b, psi_l):
    L = parts["own"] + parts["neighbour"] + parts["reflect_left"]
    lag = parts["scatter"] + parts["reflect_right"]
    return np.linalg.solve(L, b - lag @ psi_l.ravel())


@pytest.mark.parametrize("bcl,bcr", BC_CASES)
@pytest.mark.parametrize("N", [2, 4, 8])
def test_oci_iteration_is_the_block_jacobi_splitting(bcl, bcr, N):
    J = 5
    p = workloads.random_small(seed=40 + N, J=J, N=N, bc_left=bcl, bc_right=bcr)
    pe = np.asarray(p["psi0"]).reshape(J, N, 2)
    parts, b = brute.step_parts(p, pe)
    psi_l = _random_iterate(N, J, N)
    want = _oci_map(parts, b, psi_l).reshape(J, N, 4)
    got, phi = oracle.oci_iteration(p, pe, psi_l)
    scale = np.abs(want).max()
    assert np.abs(got - want).max() / scale < 1e-13
    _, w = np.polynomial.legendre.leggauss(N)
    assert np.abs(phi - np.einsum("n,jnc->jc", w, want)).max() / np.abs(phi).max() < 1e-13


@pytest.mark.parametrize("bcl,bcr", BC_CASES)
@pytest.mark.parametrize("N", [2, 4, 8])
def test_si_iteration_is_the_lagged_scattering_splitting(bcl, bcr, N):
    J = 5
    p = workloads.random_small(seed=60 + N, J=J, N=N, bc_left=bcl, bc_right=bcr)
    pe = np.asarray(p["psi0"]).reshape(J, N, 2)
    parts, b = brute.step_parts(p, pe)
    psi_l = _random_iterate(100 + N, J, N)
    _, w = np.polynomial.legendre.leggauss(N)
    phi_l = np.einsum("n,jnc->jc", w, psi_l)
    want = _si_map(parts, b, psi_l).reshape(J, N, 4)
    got, _ = oracle.si_iteration(p, pe, phi_l, psi_l)
    assert np.abs(got - want).max() / np.abs(want).max() < 1e-13


def test_parts_sum_to_the_whole_problem_and_couple_as_labelled():
    """The splitting is exhaustive, and each part couples only what its name
    says: own + scatter stay inside a cell's 4N unknowns, neighbour entries sit
    one cell off the diagonal, reflecting entries only in cell 0 / J-1."""
    J, N = 4, 4
    p = workloads.random_small(seed=5, J=J, N=N, bc_left="reflect", bc_right="reflect")
    pe = np.asarray(p["psi0"]).reshape(J, N, 2)
    parts, b = brute.step_parts(p, pe)
    M, b2 = brute.step_system(p, pe)
    assert np.array_equal(b, b2)
    assert np.allclose(sum(parts.values()), M, rtol=0, atol=1e-15)
    n = 4 * N
    cell = np.arange(J * n) // n
    for name, A in parts.items():
        r, c = np.nonzero(A)
        assert len(r) > 0, name
        if name in ("own", "scatter"):
            assert np.all(cell[r] == cell[c]), name
        elif name == "neighbour":
            assert np.all(np.abs(cell[r] - cell[c]) == 1)
        elif name == "reflect_left":
            assert np.all(cell[r] == 0) and np.all(cell[c] == 0)
        else:
            assert np.all(cell[r] == J - 1) and np.all(cell[c] == J - 1)


def test_gauss_seidel_order_differs_from_the_pinned_map():
    """Sanity of the pin itself: a map that reads the left neighbour's new
    iterate (forward Gauss-Seidel over cells) gives a different iterate, so the
    comparison above can tell the two orders apart."""
    J, N = 5, 4
    p = workloads.random_small(seed=9, J=J, N=N, bc_left="vacuum", bc_right="vacuum")
    pe = np.asarray(p["psi0"]).reshape(J, N, 2)
    parts, b = brute.step_parts(p, pe)
    psi_l = _random_iterate(3, J, N).ravel()
    nb = parts["neighbour"]
    lower = np.tril(nb)   # couplings to cell j-1 (mu > 0 upstream)
    D = parts["own"] + parts["scatter"]
    gs = np.linalg.solve(D + lower, b - (nb - lower) @ psi_l)
    jac = _oci_map(parts, b, psi_l.reshape(J, N, 4))
    assert np.abs(gs - jac).max() > 1e-3 * np.abs(jac).max()


# ------------------------------------------------------------ backward Euler

@pytest.mark.parametrize("bcl,bcr", BC_CASES)
@pytest.mark.parametrize("N", [2, 4, 8])
def test_be_iterations_are_the_same_splittings(bcl, bcr, N):
    """The backward-Euler scheme (the paper's disabled section) iterates the
    same way: OCI lags the neighbour and reflecting couplings, SI the
    scattering source and the reflecting right face."""
    J = 5
    p = workloads.random_small(seed=80 + N, J=J, N=N, bc_left=bcl, bc_right=bcr)
    pp = np.asarray(p["psi0"]).reshape(J, N, 2)
    parts, b = brute.be_step_parts(p, pp)
    psi_l = np.random.default_rng(N).uniform(-0.5, 1.5, (J, N, 2))
    want = _oci_map(parts, b, psi_l).reshape(J, N, 2)
    got, _ = oracle.be_oci_iteration(p, pp, psi_l)
    assert np.abs(got - want).max() / np.abs(want).max() < 1e-13
    _, w = np.polynomial.legendre.leggauss(N)
    want = _si_map(parts, b, psi_l).reshape(J, N, 2)
    got, _ = oracle.be_si_iteration(p, pp, np.einsum("n,jnc->jc", w, psi_l), psi_l)
    assert np.abs(got - want).max() / np.abs(want).max() < 1e-13
