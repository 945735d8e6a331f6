"""Multi-rank paths on CPU (gloo, world_size 2).

* The benchmark's replica aggregation (max time, summed work over ranks).
* Domain decomposition of OCI: each rank owns a contiguous cell range and per
  iteration exchanges one halo per cut -- the outgoing mu>0 flux of its last
  cell and the outgoing mu<0 flux of its first cell -- then all-reduces the two
  residual sums.  OCI is block Jacobi over cells (Sec. "One-Cell Inversion":
  no communication between cells within an iteration), so the partitioned
  iterates must equal the single-domain ones bit for bit.  The per-rank solve
  is the oracle's OCI iteration with the halo as prescribed incident data.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _init(rank, world, port):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)


def _aggregate_worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    _init(rank, world, port)
    t, u = bench.aggregate(1.0 + rank, 10.0 * (rank + 1), "cpu")
    out[rank] = (t, u)
    dist.destroy_process_group()


def test_replica_aggregation_gloo():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_aggregate_worker, args=(2, port, out), nprocs=2, join=True)
        for r in range(2):
            assert out[r] == (2.0, 30.0)


def _subproblem(prob, a, b, left_bc, right_bc):
    N = prob["n_ord"]
    sub = dict(prob)
    for k in ("dx", "sigma_t", "sigma_s"):
        sub[k] = np.asarray(prob[k])[a:b]
    sub["q"] = np.asarray(prob["q"])[a:b]
    sub["psi0"] = np.asarray(prob["psi0"])[a:b]
    sub["n_cells"] = b - a
    if left_bc is not None:
        sub["bc_left"], sub["psi_bc_left"] = "incident", left_bc
    if right_bc is not None:
        sub["bc_right"], sub["psi_bc_right"] = "incident", right_bc
    return sub


def _dd_worker(rank, world, port, n_iter, out):
    import sys
    sys.path.insert(0, ROOT)
    import oracle
    import workloads
    _init(rank, world, port)
    prob = workloads.random_small(seed=31, J=24, N=8, bc_left="reflect", bc_right="incident")
    J, N, P = prob["n_cells"], prob["n_ord"], prob["n_ord"] // 2
    cut = 11
    a, b = (0, cut) if rank == 0 else (cut, J)
    pe = np.asarray(prob["psi0"])[a:b]
    psi = np.concatenate([pe, pe], axis=2)
    phi_old = np.einsum("n,jnc->jc", np.polynomial.legendre.leggauss(N)[1], psi)
    resid = []
    for _ in range(n_iter):
        # halo of iterate l: [outgoing mu<0 of my first cell (L corner), outgoing mu>0 of my last cell (R corner)]
        mine = np.concatenate([psi[0, P - 1 - np.arange(P)][:, [0, 2]].ravel(),
                               psi[-1, P + np.arange(P)][:, [1, 3]].ravel()])
        halos = [torch.zeros(4 * P, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(halos, torch.from_numpy(mine))
        if rank == 0:
            right = halos[1].numpy()[:2 * P].reshape(P, 2)   # neighbour's first-cell mu<0 flux
            sub = _subproblem(prob, a, b, None, right)
        else:
            left = halos[0].numpy()[2 * P:].reshape(P, 2)    # neighbour's last-cell mu>0 flux
            sub = _subproblem(prob, a, b, left, None)
        psi, phi = oracle.oci_iteration(sub, pe, psi)
        sums = torch.tensor([np.sum((phi - phi_old) ** 2), np.sum(phi ** 2)], dtype=torch.float64)
        dist.all_reduce(sums)
        resid.append(float(np.sqrt(sums[0] / sums[1])))
        phi_old = phi
    out[rank] = (phi, psi, resid)
    dist.destroy_process_group()


def test_domain_decomposed_oci_matches_single_domain():
    import oracle
    import workloads
    n_iter = 6
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_dd_worker, args=(2, port, n_iter, out), nprocs=2, join=True)
        phi = np.concatenate([out[0][0], out[1][0]])
        psi = np.concatenate([out[0][1], out[1][1]])
        resid = out[0][2]
    prob = workloads.random_small(seed=31, J=24, N=8, bc_left="reflect", bc_right="incident")
    pe = np.asarray(prob["psi0"])
    ref = np.concatenate([pe, pe], axis=2)
    ref_resid = []
    phi_old = np.einsum("n,jnc->jc", np.polynomial.legendre.leggauss(8)[1], ref)
    for _ in range(n_iter):
        ref, rphi = oracle.oci_iteration(prob, pe, ref)
        ref_resid.append(np.sqrt(np.sum((rphi - phi_old) ** 2) / np.sum(rphi ** 2)))
        phi_old = rphi
    assert np.array_equal(psi, ref) and np.array_equal(phi, rphi)
    assert np.allclose(resid, ref_resid, rtol=1e-12, atol=0)
