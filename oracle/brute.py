"""Whole-problem dense solve of one MB-SCB time step (tiny slabs only).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

This is the plain definition of the result both iterative schemes converge to:
every equation of the SCB-MB discretisation (Eqs. scb-mb-a..d of Sec. "Derivation
of MB-SCB") is written as a row of one dense linear system over all 4NJ unknowns
of a time step, with the two spatial closures -- the midpoint average and the
upstream cell-edge flux -- substituted **unlagged**, and the boundary conditions
of Eq. 1 (prescribed, vacuum, or reflecting: incident = mirror ordinate's
outgoing at that face).  The system is assembled straight from the balance
equations, not from the A^+/A^- matrices, so it is an independent route to the
same discrete solution.  numpy's Gauss-Legendre rule and dense solver are used as
library steps.

Unknown ordering: u(j, m, c) = (j*N + m)*4 + c, c in (k,L) (k,R) (k+1/2,L) (k+1/2,R),
ordinates ascending in mu.
"""
import numpy as np

BC_VACUUM, BC_REFLECT, BC_INCIDENT = 0, 1, 2
_BC_NAMES = {"vacuum": 0, "reflect": 1, "reflecting": 1, "incident": 2}


def _bc(x):
    return _BC_NAMES[x] if isinstance(x, str) else int(x)


def step_parts(prob, psi_edge):
    """Assemble one time step's whole-problem system from psi_{k-1/2} = psi_edge
    [J][N][2], with the matrix split by the kind of coupling each entry makes:

      "own"           the cell's own streaming, collision and time terms, with
                      the upstream closure where the upstream corner lies in the
                      same cell (mu > 0 at the right face, mu < 0 at the left);
      "scatter"       the isotropic scattering entries, Delta x Sigma_s w_n / 4
                      on the same corner and time moment of every ordinate;
      "neighbour"     the upstream closure that reads the adjacent cell's
                      corner (mu > 0 from cell j-1, mu < 0 from cell j+1);
      "reflect_left", "reflect_right"
                      a reflecting face's closure: the mirror ordinate's
                      outgoing corner of cell 0 or cell J-1.

    Returns (parts, rhs); the whole-problem matrix is the sum of the parts.  The
    iteration schemes are splittings of this one matrix (Sec. "One-Cell
    Inversion (OCI)": each cell solved with its neighbours' fluxes from the
    previous iterate; Sec. "Source Iteration (SI)": sweeps with the scattering
    source from the previous iterate), so the parts let a test build each
    scheme's iteration map without the oracle's code."""
    J, N = int(prob["n_cells"]), int(prob["n_ord"])
    P = N // 2
    mu, w = np.polynomial.legendre.leggauss(N)
    dx = np.asarray(prob["dx"], float)
    sig = np.asarray(prob["sigma_t"], float)
    sigs = np.asarray(prob["sigma_s"], float)
    q = np.zeros((J, 4)) if prob.get("q") is None else np.asarray(prob["q"], float).reshape(J, 4)
    v, dt = float(prob["v"]), float(prob["dt"])
    inv_v = 0.0 if np.isinf(v) else 1.0 / v
    bcl, bcr = _bc(prob.get("bc_left", 0)), _bc(prob.get("bc_right", 0))
    psl = None if prob.get("psi_bc_left") is None else np.asarray(prob["psi_bc_left"], float).reshape(P, 2)
    psr = None if prob.get("psi_bc_right") is None else np.asarray(prob["psi_bc_right"], float).reshape(P, 2)
    pe = np.asarray(psi_edge, float).reshape(J, N, 2)

    n = 4 * N * J
    parts = {k: np.zeros((n, n)) for k in ("own", "scatter", "neighbour", "reflect_left", "reflect_right")}
    M = parts["own"]
    b = np.zeros(n)

    def u(j, m, c):
        return (j * N + m) * 4 + c

    def add_edge(row, coef, j, m, t, side):
        """Add coef * (upstream edge flux of ordinate m, time moment t) on the
        `side` ('left' = j-1/2, 'right' = j+1/2) face of cell j."""
        cL, cR = (0, 1) if t == 0 else (2, 3)
        if side == "right":
            if mu[m] > 0:
                M[row, u(j, m, cR)] += coef
            elif j + 1 < J:
                parts["neighbour"][row, u(j + 1, m, cL)] += coef
            elif bcr == BC_REFLECT:
                parts["reflect_right"][row, u(J - 1, N - 1 - m, cR)] += coef
            elif bcr == BC_INCIDENT and psr is not None:
                b[row] -= coef * psr[P - 1 - m, t]
        else:
            if mu[m] < 0:
                M[row, u(j, m, cL)] += coef
            elif j > 0:
                parts["neighbour"][row, u(j - 1, m, cR)] += coef
            elif bcl == BC_REFLECT:
                parts["reflect_left"][row, u(0, N - 1 - m, cL)] += coef
            elif bcl == BC_INCIDENT and psl is not None:
                b[row] -= coef * psl[m - P, t]

    def add_scatter(row, j, c):
        for k in range(N):
            parts["scatter"][row, u(j, k, c)] -= dx[j] / 4 * sigs[j] * w[k]

    for j in range(J):
        h = dx[j] / 2.0
        for m in range(N):
            mm = mu[m]
            # (a): left half, time average
            r = u(j, m, 0)
            M[r, u(j, m, 2)] += h * inv_v / dt
            b[r] += h * inv_v / dt * pe[j, m, 0]
            M[r, u(j, m, 0)] += mm / 2 + h * sig[j]
            M[r, u(j, m, 1)] += mm / 2
            add_edge(r, -mm, j, m, 0, "left")
            add_scatter(r, j, 0)
            b[r] += h / 2 * q[j, 0]
            # (b): right half, time average
            r = u(j, m, 1)
            M[r, u(j, m, 3)] += h * inv_v / dt
            b[r] += h * inv_v / dt * pe[j, m, 1]
            add_edge(r, mm, j, m, 0, "right")
            M[r, u(j, m, 0)] -= mm / 2
            M[r, u(j, m, 1)] += -mm / 2 + h * sig[j]
            add_scatter(r, j, 1)
            b[r] += h / 2 * q[j, 1]
            # (c): left half, end of step (time derivative over dt/2)
            r = u(j, m, 2)
            M[r, u(j, m, 2)] += h * inv_v / (dt / 2) + mm / 2 + h * sig[j]
            M[r, u(j, m, 0)] -= h * inv_v / (dt / 2)
            M[r, u(j, m, 3)] += mm / 2
            add_edge(r, -mm, j, m, 1, "left")
            add_scatter(r, j, 2)
            b[r] += h / 2 * q[j, 2]
            # (d): right half, end of step
            r = u(j, m, 3)
            M[r, u(j, m, 3)] += h * inv_v / (dt / 2) - mm / 2 + h * sig[j]
            M[r, u(j, m, 1)] -= h * inv_v / (dt / 2)
            M[r, u(j, m, 2)] -= mm / 2
            add_edge(r, mm, j, m, 1, "right")
            add_scatter(r, j, 3)
            b[r] += h / 2 * q[j, 3]
    return parts, b


def step_system(prob, psi_edge):
    """Assemble (M, rhs) for one time step from psi_{k-1/2} = psi_edge [J][N][2]:
    every balance equation as one row, both closures unlagged."""
    parts, b = step_parts(prob, psi_edge)
    return sum(parts.values()), b


def solve_step(prob, psi_edge):
    """Exact discrete solution of one step: returns (psi [J][N][4], phi [J][4])."""
    J, N = int(prob["n_cells"]), int(prob["n_ord"])
    M, b = step_system(prob, psi_edge)
    psi = np.linalg.solve(M, b).reshape(J, N, 4)
    _, w = np.polynomial.legendre.leggauss(N)
    phi = np.einsum("n,jnc->jc", w, psi)
    return psi, phi


def run(prob, n_steps, psi_edge=None):
    """March n_steps exact steps; returns (psi_edge_final [J][N][2], phi_steps [n_steps][J][4])."""
    J, N = int(prob["n_cells"]), int(prob["n_ord"])
    pe = np.zeros((J, N, 2)) if psi_edge is None else np.array(psi_edge, float).reshape(J, N, 2)
    if psi_edge is None and prob.get("psi0") is not None:
        pe = np.array(prob["psi0"], float).reshape(J, N, 2)
    phis = []
    for _ in range(n_steps):
        psi, phi = solve_step(prob, pe)
        pe = psi[:, :, 2:4].copy()
        phis.append(phi)
    return pe, np.array(phis)


def be_step_parts(prob, psi_prev):
    """Assemble one backward-Euler step from psi^{n-1} = psi_prev [J][N][2]:
    per cell, ordinate and half-cell the SCB balance
    mu (psi_out_face - psi_in_face) + Sigma_hat dx/2 psi_corner
        = dx/2 [Sigma_s/2 phi_corner + Q/2 + psi^{n-1}_corner/(v dt)],
    Sigma_hat = Sigma + 1/(v dt), with the midpoint value (psi_L + psi_R)/2 at
    x_j and the upstream corner at the cell edges (unlagged), Q = Q_{k+1/2}.
    Unknown u(j, m, c) = (j*N + m)*2 + c, c in (L, R).  The matrix comes split
    into the same parts as ``step_parts`` (own, scatter, neighbour,
    reflect_left, reflect_right); returns (parts, rhs)."""
    J, N = int(prob["n_cells"]), int(prob["n_ord"])
    P = N // 2
    mu, w = np.polynomial.legendre.leggauss(N)
    dx = np.asarray(prob["dx"], float)
    sig = np.asarray(prob["sigma_t"], float)
    sigs = np.asarray(prob["sigma_s"], float)
    q = np.zeros((J, 4)) if prob.get("q") is None else np.asarray(prob["q"], float).reshape(J, 4)
    v, dt = float(prob["v"]), float(prob["dt"])
    inv_vdt = 0.0 if np.isinf(v) else 1.0 / (v * dt)
    bcl, bcr = _bc(prob.get("bc_left", 0)), _bc(prob.get("bc_right", 0))
    psl = None if prob.get("psi_bc_left") is None else np.asarray(prob["psi_bc_left"], float).reshape(P, 2)
    psr = None if prob.get("psi_bc_right") is None else np.asarray(prob["psi_bc_right"], float).reshape(P, 2)
    pp = np.asarray(psi_prev, float).reshape(J, N, 2)
    n = 2 * N * J
    parts = {k: np.zeros((n, n)) for k in ("own", "scatter", "neighbour", "reflect_left", "reflect_right")}
    M = parts["own"]
    b = np.zeros(n)

    def u(j, m, c):
        return (j * N + m) * 2 + c

    def add_face(row, coef, j, m, side):
        """coef * (flux of ordinate m on the `side` face of cell j, upstream value)."""
        if side == "left":
            if mu[m] < 0:
                M[row, u(j, m, 0)] += coef
            elif j > 0:
                parts["neighbour"][row, u(j - 1, m, 1)] += coef
            elif bcl == BC_REFLECT:
                parts["reflect_left"][row, u(0, N - 1 - m, 0)] += coef
            elif bcl == BC_INCIDENT and psl is not None:
                b[row] -= coef * psl[m - P, 1]
        else:
            if mu[m] > 0:
                M[row, u(j, m, 1)] += coef
            elif j + 1 < J:
                parts["neighbour"][row, u(j + 1, m, 0)] += coef
            elif bcr == BC_REFLECT:
                parts["reflect_right"][row, u(J - 1, N - 1 - m, 1)] += coef
            elif bcr == BC_INCIDENT and psr is not None:
                b[row] -= coef * psr[P - 1 - m, 1]

    for j in range(J):
        h = dx[j] / 2.0
        sh = sig[j] + inv_vdt
        for m in range(N):
            mm = mu[m]
            for c, side in ((0, "left"), (1, "right")):
                r = u(j, m, c)
                # mu (psi_mid - psi_left_face) or mu (psi_right_face - psi_mid)
                sgn = 1.0 if c == 0 else -1.0
                M[r, u(j, m, 0)] += sgn * mm / 2
                M[r, u(j, m, 1)] += sgn * mm / 2
                add_face(r, -sgn * mm, j, m, side)
                M[r, u(j, m, c)] += h * sh
                for k in range(N):
                    parts["scatter"][r, u(j, k, c)] -= h / 2 * sigs[j] * w[k]
                b[r] += h / 2 * q[j, 2 + c] + h * inv_vdt * pp[j, m, c]
    return parts, b


def be_step_system(prob, psi_prev):
    """(M, rhs) of one backward-Euler step (the sum of ``be_step_parts``)."""
    parts, b = be_step_parts(prob, psi_prev)
    return sum(parts.values()), b


def be_solve_step(prob, psi_prev):
    M, b = be_step_system(prob, psi_prev)
    J, N = int(prob["n_cells"]), int(prob["n_ord"])
    return np.linalg.solve(M, b).reshape(J, N, 2)


def be_run(prob, n_steps, psi0=None):
    """Dense BE steps; returns (psi [J][N][2], phi_steps [n][J][2])."""
    J, N = int(prob["n_cells"]), int(prob["n_ord"])
    _, w = np.polynomial.legendre.leggauss(N)
    psi = np.zeros((J, N, 2)) if psi0 is None else np.asarray(psi0, float).reshape(J, N, 2).copy()
    phis = []
    for _ in range(n_steps):
        psi = be_solve_step(prob, psi)
        phis.append(np.einsum("n,jnc->jc", w, psi))
    return psi, np.array(phis)
