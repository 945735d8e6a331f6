"""Domain decomposition through the C ABI (oci_dd_*): a slab split into cell
ranges, each a handle of its own, exchanging the angular flux crossing each
cut once per iteration and summing two scalars for the convergence test
(Sec. "GPU Implementations": OCI splits over accelerators within an
iteration).  In FP64 every cell's arithmetic is the undivided slab's, so the
results agree with one handle bit for bit: at a fixed iteration count and at
convergence (same iteration counts).  The exchange runs through plain device
copies between two handles on one GPU, and through gloo between two
processes (host copies of the same faces)."""

import numpy as np
import pytest
import torch

import paper_2305_13555_gb300 as pkg
import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2305_13555_gb300 import build
    build.build()
    pkg.load_library()


def _sub(prob, lo, hi):
    """The sub-slab of cells [lo, hi): its own data, a cut (incident, zero data) where it does not end the slab."""
    J, N = prob["n_cells"], prob["n_ord"]
    zeros = np.zeros((N // 2, 2))
    s = dict(prob)
    s["n_cells"] = hi - lo
    for k in ("dx", "sigma_t", "sigma_s", "q"):
        s[k] = np.asarray(prob[k])[lo:hi]
    if prob.get("psi0") is not None:
        s["psi0"] = np.asarray(prob["psi0"]).reshape(J, N, 2)[lo:hi]
    if lo > 0:
        s["bc_left"], s["psi_bc_left"] = "incident", zeros
    if hi < J:
        s["bc_right"], s["psi_bc_right"] = "incident", zeros
    return s


def _dd_steps(prob, cuts, precision, n_steps, tol, max_iter, commit_unconverged=False):
    """March n_steps decomposed steps; returns (phi per step [J][4], final state, iterations per step)."""
    edges = [0] + list(cuts) + [prob["n_cells"]]
    subs = [pkg.Solver(_sub(prob, a, b), precision=precision, tol=tol, max_iter=max_iter)
            for a, b in zip(edges[:-1], edges[1:])]
    dt = torch.float64 if precision == "fp64" else torch.float32
    P = prob["n_ord"] // 2
    outs = [(torch.zeros((P, 2), dtype=dt, device="cuda"), torch.zeros((P, 2), dtype=dt, device="cuda"))
            for _ in subs]
    phis, iters = [], []
    try:
        for s in subs:
            pkg.oci_set_iteration(s.h, tol, max_iter, commit_unconverged)
        for _ in range(n_steps):
            for s in subs:
                pkg.oci_dd_begin(s.h)
            while True:
                for s, (ol, orr) in zip(subs, outs):
                    pkg.oci_dd_export(s.h, ol, orr)
                for i, s in enumerate(subs):
                    pkg.oci_dd_import(s.h, outs[i - 1][1] if i > 0 else None,
                                      outs[i + 1][0] if i + 1 < len(subs) else None)
                total = np.zeros(2)
                for s in subs:
                    total += pkg.oci_dd_iterate(s.h)
                res = [pkg.oci_dd_decide(s.h, total) for s in subs]
                assert len({r[0] for r in res}) == 1
                if res[0][0]:
                    break
            st = res[0][2]
            assert all(r[1] == res[0][1] for r in res)
            iters.append(st["iters"])
            phis.append(np.concatenate([s.fluxes() for s in subs]))
        state = np.concatenate([s.get_state() for s in subs])
    finally:
        for s in subs:
            s.close()
    return np.array(phis), state, iters


def _one_domain(prob, precision, n_steps, tol, max_iter, commit_unconverged=False):
    phis, iters = [], []
    with pkg.Solver(prob, precision=precision, tol=tol, max_iter=max_iter) as s:
        s.set_iteration(tol, max_iter, commit_unconverged)
        for _ in range(n_steps):
            rc, st = s.step("oci")
            iters.append(st["iters"])
            phis.append(s.fluxes())
        return np.array(phis), s.get_state(), iters


@pytest.mark.parametrize("bcl,bcr", [("reflect", "vacuum"), ("incident", "reflect"), ("reflect", "reflect")])
def test_two_subdomains_fp64_bit_identical_fixed_iterations(bcl, bcr):
    prob = workloads.random_small(seed=21, J=300, N=8, bc_left=bcl, bc_right=bcr)
    ref, ref_state, _ = _one_domain(prob, "fp64", 2, 0.0, 6, commit_unconverged=True)
    got, state, iters = _dd_steps(prob, [137], "fp64", 2, 0.0, 6, commit_unconverged=True)
    assert iters == [6, 6]
    assert np.array_equal(got, ref) and np.array_equal(state, ref_state)


def test_three_subdomains_fp64_bit_identical_at_convergence():
    prob = workloads.hetero(seed=5, J=2000, N=16, n_steps=3, bc_left="reflect", bc_right="vacuum")
    ref, ref_state, ref_it = _one_domain(prob, "fp64", 3, 1e-10, 10000)
    got, state, iters = _dd_steps(prob, [613, 1400], "fp64", 3, 1e-10, 10000)
    assert iters == ref_it
    assert np.array_equal(got, ref) and np.array_equal(state, ref_state)


def test_two_subdomains_fp32_within_bound():
    prob = workloads.hetero(seed=6, J=5000, N=64, n_steps=2, bc_left="vacuum", bc_right="reflect")
    ref, _, ref_it = _one_domain(prob, "fp32", 2, 1e-8, 10000)
    got, _, iters = _dd_steps(prob, [2471], "fp32", 2, 1e-8, 10000)
    assert all(abs(a - b) <= 1 for a, b in zip(iters, ref_it))
    assert np.abs(got - ref).max() / np.abs(ref).max() < 2e-6


def _gloo_rank(rank, world, port, prob, cuts, out_path):
    import torch.distributed as dist
    torch.cuda.set_device(0)
    pkg.load_library()
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    edges = [0] + list(cuts) + [prob["n_cells"]]
    P = prob["n_ord"] // 2
    s = pkg.Solver(_sub(prob, edges[rank], edges[rank + 1]), precision="fp64", tol=1e-10, max_iter=10000)
    ol = torch.zeros((P, 2), dtype=torch.float64, device="cuda")
    orr = torch.zeros_like(ol)
    il, ir = torch.zeros_like(ol), torch.zeros_like(ol)
    phis, iters = [], []
    for _ in range(2):
        pkg.oci_dd_begin(s.h)
        while True:
            pkg.oci_dd_export(s.h, ol, orr)
            torch.cuda.synchronize()
            # host exchange of the cut faces: my right outgoing -> right neighbour's left incident
            reqs = []
            recv_l, recv_r = torch.zeros((P, 2), dtype=torch.float64), torch.zeros((P, 2), dtype=torch.float64)
            send_l, send_r = ol.cpu(), orr.cpu()
            if rank + 1 < world:
                reqs.append(dist.isend(send_r, rank + 1))
                reqs.append(dist.irecv(recv_r, rank + 1))
            if rank > 0:
                reqs.append(dist.isend(send_l, rank - 1))
                reqs.append(dist.irecv(recv_l, rank - 1))
            for r in reqs:
                r.wait()
            il.copy_(recv_l)
            ir.copy_(recv_r)
            pkg.oci_dd_import(s.h, il if rank > 0 else None, ir if rank + 1 < world else None)
            total = torch.tensor(pkg.oci_dd_iterate(s.h))
            dist.all_reduce(total)
            done, rc, st = pkg.oci_dd_decide(s.h, total.numpy())
            if done:
                break
        iters.append(st["iters"])
        phis.append(s.fluxes())
    np.savez(out_path, phi=np.array(phis), iters=np.array(iters))
    s.close()
    dist.destroy_process_group()


def test_two_processes_exchange_through_gloo(tmp_path):
    import socket

    import torch.multiprocessing as mp
    prob = workloads.hetero(seed=7, J=1500, N=8, n_steps=2, bc_left="reflect", bc_right="vacuum")
    ref, _, ref_it = _one_domain(prob, "fp64", 2, 1e-10, 10000)
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_gloo_rank, args=(r, 2, port, prob, [700], str(tmp_path / f"r{r}.npz")))
             for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    parts = [np.load(tmp_path / f"r{r}.npz") for r in range(2)]
    assert list(parts[0]["iters"]) == list(parts[1]["iters"]) == ref_it
    got = np.concatenate([parts[0]["phi"], parts[1]["phi"]], axis=1)
    assert np.array_equal(got, ref)
