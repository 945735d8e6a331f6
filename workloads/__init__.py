"""Seeded synthetic slab problems shaped like the paper's workloads.

This module only draws and lays out inputs (cell widths, cross sections,
sources, boundary data, initial fluxes); it contains none of the method's
arithmetic and is the one module that both the CUDA path and the oracle read.
All randomness is numpy PCG64 with an explicit seed.

A problem is a plain dict:
  n_cells J, n_ord N (even), dx[J], sigma_t[J], sigma_s[J], q[J][4]
  (Q_{k,L}, Q_{k,R}, Q_{k+1/2,L}, Q_{k+1/2,R}), v, dt,
  bc_left / bc_right in {"vacuum", "reflect", "incident"},
  psi_bc_left / psi_bc_right [N/2][2] or None, psi0 [J][N][2] or None,
  n_steps, tol, plus a "name".

The paper's own workloads stood in for here:
  * the homogeneous slab of the quadrature sweep (Sec. "GPU Explorations Across
    Quadrature Sets": L = 10, Sigma = 2, Q = 0.1, vacuum, 5 steps);
  * the multi-region transient Reed-type problem (Sec. "Transient Reed's
    Problem"), whose geometry is only in a figure; a seeded layered slab
    (``hetero``) takes its place.
"""
import numpy as np

BC = ("vacuum", "reflect", "incident")


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def homogeneous(J, N, sigma_t=1.0, c=0.5, dx=0.1, v=1.0, dt=0.05, q=1.0, bc_left="vacuum",
                bc_right="vacuum", n_steps=1, tol=1e-8, name="homogeneous", q_cells=None):
    """Uniform slab; ``q_cells`` optionally restricts the source to a cell range [a, b)."""
    qa = np.zeros((J, 4))
    if q_cells is None:
        qa[:] = q
    else:
        qa[q_cells[0]:q_cells[1]] = q
    return {
        "name": name, "n_cells": J, "n_ord": N,
        "dx": np.full(J, float(dx)), "sigma_t": np.full(J, float(sigma_t)),
        "sigma_s": np.full(J, float(c * sigma_t)), "q": qa, "v": float(v), "dt": float(dt),
        "bc_left": bc_left, "bc_right": bc_right, "psi_bc_left": None, "psi_bc_right": None,
        "psi0": None, "n_steps": n_steps, "tol": tol,
    }


def config1():
    """64 cells, dx = 0.1 mfp, Sigma = 1, c = 0.5, v = 1, S_8, vacuum both sides,
    Q = 1 on cells 24..39 (0-based), psi0 = 0, dt = 0.1, 10 steps, tol 1e-10."""
    return homogeneous(64, 8, 1.0, 0.5, 0.1, 1.0, 0.1, 1.0, "vacuum", "vacuum", 10, 1e-10,
                       name="slab64_S8_c0.5_dx0.1", q_cells=(24, 40))


def config2(N=64, c=0.9, dx=0.1, J=65536, n_steps=50):
    """Production homogeneous slab: Sigma = 1, dt = 0.05, v = 1, Q = 1,
    reflecting left / vacuum right, tol 1e-8.  Swept over N in {32, 64},
    c in {0.5, 0.9, 0.99}, dx in {0.01, 0.1, 1, 10} mfp."""
    return homogeneous(J, N, 1.0, c, dx, 1.0, 0.05, 1.0, "reflect", "vacuum", n_steps, 1e-8,
                       name=f"slab{J}_S{N}_c{c}_dx{dx}")


def config3(J=16384, n_steps=20):
    """High angle count: S_128, Sigma = 1, c = 0.9, dx = 1 mfp, v = 1, dt = 0.05,
    reflecting left / vacuum right, Q = 1, tol 1e-8."""
    return homogeneous(J, 128, 1.0, 0.9, 1.0, 1.0, 0.05, 1.0, "reflect", "vacuum", n_steps, 1e-8,
                       name=f"slab{J}_S128_c0.9_dx1")


def hetero(seed, J=131072, N=64, n_steps=100, dt=0.02, v=1.0, tau_range=(0.05, 5.0),
           c_range=(0.0, 0.999), log_sigma_range=(-2.0, 2.0), n_layers_range=(8, 32),
           q_max=10.0, tol=1e-8, bc_left="vacuum", bc_right="vacuum", name=None):
    """Seeded layered slab (Reed-type stand-in).

    n_L ~ U{8..32} layers; layer sizes from sorted uniform cut points (each layer
    >= 1 cell); per layer sigma_t = 10^U(-2, 2), c ~ U(0, 0.999), optical cell
    thickness sigma_t * dx ~ U(0.05, 5) (so dx = U / sigma_t); Q ~ U(0, 10) on a
    random half of the layers, else 0.
    """
    g = _rng(seed)
    nl = int(g.integers(n_layers_range[0], n_layers_range[1] + 1))
    nl = min(nl, J)
    cuts = np.sort(g.choice(np.arange(1, J), size=nl - 1, replace=False)) if nl > 1 else np.array([], int)
    bounds = np.concatenate([[0], cuts, [J]])
    st = 10.0 ** g.uniform(log_sigma_range[0], log_sigma_range[1], nl)
    c = g.uniform(c_range[0], c_range[1], nl)
    tau = g.uniform(tau_range[0], tau_range[1], nl)
    src_layers = g.permutation(nl)[: nl // 2]
    qv = np.zeros(nl)
    qv[src_layers] = g.uniform(0.0, q_max, len(src_layers))
    dx = np.empty(J); sig = np.empty(J); sigs = np.empty(J); q = np.zeros((J, 4))
    layer = np.empty(J, dtype=np.int32)
    for i in range(nl):
        a, b = bounds[i], bounds[i + 1]
        dx[a:b] = tau[i] / st[i]
        sig[a:b] = st[i]
        sigs[a:b] = c[i] * st[i]
        q[a:b] = qv[i]
        layer[a:b] = i
    return {
        "name": name or f"hetero{J}_S{N}_seed{seed}", "n_cells": J, "n_ord": N,
        "dx": dx, "sigma_t": sig, "sigma_s": sigs, "q": q, "v": float(v), "dt": float(dt),
        "bc_left": bc_left, "bc_right": bc_right, "psi_bc_left": None, "psi_bc_right": None,
        "psi0": None, "n_steps": n_steps, "tol": tol, "layer": layer,
    }


def config4(seed=4, J=131072, n_steps=100):
    """Heterogeneous seeded slab: 131072 cells, S_64, dt = 0.02, 100 steps, tol 1e-8."""
    return hetero(seed, J=J, N=64, n_steps=n_steps, dt=0.02)


def config5_train(seed, J=4096, N=16, n_steps=50):
    """Training trajectory problem: a config-4-style slab at 4096 cells, S_16."""
    return hetero(seed, J=J, N=N, n_steps=n_steps, dt=0.02, name=f"train{J}_S{N}_seed{seed}")


def config5_deploy(seed, J=131072, N=64, n_steps=200):
    """Deployment problem: thin cells (sigma_t dx ~ U(0.01, 0.1)), c ~ U(0.9, 0.999)."""
    return hetero(seed, J=J, N=N, n_steps=n_steps, dt=0.02, tau_range=(0.01, 0.1), c_range=(0.9, 0.999),
                  name=f"deploy{J}_S{N}_seed{seed}")


def random_small(seed, J=6, N=4, bc_left="vacuum", bc_right="vacuum", v=1.0, dt=0.1, with_psi0=True,
                 with_bc=True, homogeneous_material=False):
    """Tiny random slab for brute-force and parity checks: per-cell random
    materials, sources per time moment and corner, random psi0 and incident data."""
    g = _rng(seed)
    if homogeneous_material:
        dx = np.full(J, g.uniform(0.05, 1.0)); st = np.full(J, g.uniform(0.5, 3.0))
        ss = st * g.uniform(0.0, 0.99)
    else:
        dx = g.uniform(0.05, 1.0, J); st = g.uniform(0.5, 3.0, J); ss = st * g.uniform(0.0, 0.99, J)
    P = N // 2
    return {
        "name": f"small{J}_S{N}_seed{seed}", "n_cells": J, "n_ord": N,
        "dx": dx, "sigma_t": st, "sigma_s": ss, "q": g.uniform(0.0, 2.0, (J, 4)),
        "v": float(v), "dt": float(dt), "bc_left": bc_left, "bc_right": bc_right,
        "psi_bc_left": g.uniform(0.0, 1.0, (P, 2)) if with_bc else None,
        "psi_bc_right": g.uniform(0.0, 1.0, (P, 2)) if with_bc else None,
        "psi0": g.uniform(0.0, 1.0, (J, N, 2)) if with_psi0 else None,
        "n_steps": 3, "tol": 1e-13,
    }
