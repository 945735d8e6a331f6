"""Learned initial guess for the OCI iteration: training data and training loop.

The network (include/oci_nn.h) predicts a time step's converged scalar-flux
moments from the two previous steps' moments and per-cell material / source
inputs.  Its training data are trajectories produced by this library's own OCI
solver on seeded slabs (``workloads.config5_train``); training is one
call of the library's oci_nn_train (minibatches, epochs, schedule and
validation inside the library, on its forward / backward / Adam kernels).
PyTorch only holds device arrays.  The paper has no learned component.

Usage (on a GPU):
    python -m paper_2305_13555_gb300.learned --trajectories 2000 --epochs 20 \
        --out paper_2305_13555_gb300/data/cnn_weights.npy
"""
import argparse
import json
import math
import os
import time

import numpy as np

from . import (OCI_OK, Solver, oci_fluxes_device, oci_nn_features, oci_nn_forward, oci_nn_param_count,
               oci_nn_predict, oci_nn_static_features, oci_nn_workspace_bytes)

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_WEIGHTS = os.path.join(HERE, "data", "cnn_weights.npy")


def trajectories(seeds, J=4096, N=16, n_steps=20, precision="fp64", problem=None):
    """Run the OCI solver on one seeded slab per seed; returns device tensors
    phi [T][n_steps+1][J][4] (float64; index 0 = initial moments), stat
    [T][J][4] and qfeat [T][J] (float32), and the iteration counts."""
    import torch
    import workloads
    problem = problem or (lambda s: workloads.config5_train(s, J=J, N=N, n_steps=n_steps))
    T = len(seeds)
    phi = torch.zeros((T, n_steps + 1, J, 4), dtype=torch.float64, device="cuda")
    stat = torch.zeros((T, J, 4), dtype=torch.float32, device="cuda")
    qfeat = torch.zeros((T, J), dtype=torch.float32, device="cuda")
    iters = np.zeros((T, n_steps), dtype=np.int32)
    for i, seed in enumerate(seeds):
        prob = problem(seed)
        with Solver(prob, precision=precision, tol=1e-8) as s:
            oci_nn_static_features(s.h, stat[i], qfeat[i])
            oci_fluxes_device(s.h, phi[i, 0].data_ptr())
            for n in range(n_steps):
                rc, st = s.step()
                if rc != OCI_OK:
                    raise RuntimeError(f"trajectory seed {seed} step {n}: status {rc}")
                iters[i, n] = st["iters"]
                oci_fluxes_device(s.h, phi[i, n + 1].data_ptr())
    torch.cuda.synchronize()
    return {"phi": phi, "stat": stat, "qfeat": qfeat, "iters": iters}


def init_params(seed=0):
    """He-uniform weights for the ReLU layers, zero biases (layout of oci_nn.h)."""
    g = np.random.default_rng(seed)
    ch = (13, 32, 32, 32, 32, 4)
    out = []
    for ci, co in zip(ch[:-1], ch[1:]):
        bound = math.sqrt(6.0 / (ci * 5))
        out.append(g.uniform(-bound, bound, co * ci * 5))
        out.append(np.zeros(co))
    p = np.concatenate(out).astype(np.float32)
    assert p.size == oci_nn_param_count()
    return p


def extrapolation_params(seed=0):
    """Parameters whose network is exactly linear extrapolation in time,
    out = (phi_{n-1} - phi_{n-2}) / S (so phi_hat = 2 phi_{n-1} - phi_{n-2}),
    with room to learn a correction on top: in layers 1-4, channels 0-7
    carry the positive and negative parts of input channels 4-7 (the
    normalised change of the last step) on the centre tap, channels 8-31
    start He-uniform, and the last layer reads only channels 0-7, so training
    starts from the extrapolation's loss and moves away from it only where
    that lowers the loss."""
    g = np.random.default_rng(seed)
    ch = (13, 32, 32, 32, 32, 4)
    out = []
    for l, (ci, co) in enumerate(zip(ch[:-1], ch[1:])):
        bound = math.sqrt(6.0 / (ci * 5))
        W = g.uniform(-bound, bound, (co, ci, 5))
        if l == 0:
            W[:8] = 0.0
            for c in range(4):
                W[2 * c, 4 + c, 2], W[2 * c + 1, 4 + c, 2] = 1.0, -1.0
        elif l < len(ch) - 2:
            W[:8] = 0.0
            for c in range(8):
                W[c, c, 2] = 1.0
        else:
            W[:] = 0.0
            for c in range(4):
                W[c, 2 * c, 2], W[c, 2 * c + 1, 2] = 1.0, -1.0
        out += [W.ravel(), np.zeros(co)]
    p = np.concatenate(out).astype(np.float32)
    assert p.size == oci_nn_param_count()
    return p


def train(data, epochs=20, batch=32, lr=1e-3, seed=0, params=None, log=print, val_frac=0.05):
    """The library's training procedure (oci_nn_train): minibatch Adam over all
    (trajectory, step) samples with a held-out validation set and a cosine
    learning-rate schedule.  Returns (params, statistics)."""
    import torch
    from . import oci_nn_train
    p0 = torch.tensor(init_params(seed) if params is None else params, device="cuda")
    out = torch.empty_like(p0)
    t0 = time.time()
    st = oci_nn_train(data["phi"], data["stat"], data["qfeat"], out, epochs=epochs, batch=batch, lr=lr,
                      val_frac=val_frac, seed=seed, init_params=p0)
    st["seconds"] = time.time() - t0
    if log:
        log(f"{st['epochs_done']} epochs, {st['steps_done']} steps: train {st['train_loss']:.3e} "
            f"val {st['val_loss']:.3e} ({st['seconds']:.1f} s)")
    return out.cpu().numpy(), st


def predict(params, phi1, phi2, stat, qfeat):
    """Network prediction phat [B][J][4] (float64) for device inputs."""
    import torch
    B, J = phi1.shape[0], phi1.shape[1]
    ws = torch.empty(oci_nn_workspace_bytes(B, J), dtype=torch.uint8, device="cuda")
    inp = torch.empty((B, 13, J), dtype=torch.float32, device="cuda")
    out = torch.empty((B, 4, J), dtype=torch.float32, device="cuda")
    scale = torch.empty(B, dtype=torch.float32, device="cuda")
    phat = torch.empty((B, J, 4), dtype=torch.float64, device="cuda")
    p = torch.as_tensor(params, device="cuda")
    oci_nn_features(phi1, phi2, stat, qfeat, inp, scale)
    oci_nn_forward(p, inp, out, ws)
    oci_nn_predict(phi1, out, scale, phat)
    return phat


def time_inference(params, J, reps=50, warmup=5, stat=None, qfeat=None, stream=None):
    """Device microseconds of the network's parts for one J-cell sample (CUDA
    events on the launching stream, mean of reps after warmup): the input
    features, the forward pass (the BF16 parameter image and the fused
    five-layer tensor-core kernel) and the prediction of the moments.  Random
    moments; static inputs random unless given."""
    import torch
    stream = stream or torch.cuda.current_stream()
    g = torch.Generator(device="cuda").manual_seed(0)
    if stat is None:
        stat = torch.rand((1, J, 4), dtype=torch.float32, device="cuda", generator=g)
    if qfeat is None:
        qfeat = torch.rand((1, J), dtype=torch.float32, device="cuda", generator=g)
    phi1 = torch.rand((1, J, 4), dtype=torch.float64, device="cuda", generator=g)
    phi2 = torch.rand((1, J, 4), dtype=torch.float64, device="cuda", generator=g)
    inp = torch.empty((1, 13, J), dtype=torch.float32, device="cuda")
    out = torch.empty((1, 4, J), dtype=torch.float32, device="cuda")
    sc = torch.empty(1, dtype=torch.float32, device="cuda")
    phat = torch.empty((1, J, 4), dtype=torch.float64, device="cuda")
    ws = torch.empty(oci_nn_workspace_bytes(1, J), dtype=torch.uint8, device="cuda")
    p = torch.as_tensor(params, device="cuda")
    cs = stream.cuda_stream
    res = {}
    for name, fn in (("features", lambda: oci_nn_features(phi1, phi2, stat, qfeat, inp, sc, cs)),
                     ("forward", lambda: oci_nn_forward(p, inp, out, ws, cs)),
                     ("predict", lambda: oci_nn_predict(phi1, out, sc, phat, cs))):
        for _ in range(warmup):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        res[name] = round(e0.elapsed_time(e1) * 1e3 / reps, 2)
    return res


def load_weights(path=DEFAULT_WEIGHTS):
    return np.load(path).astype(np.float32)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--trajectories", type=int, default=2000)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--cells", type=int, default=4096)
    ap.add_argument("--ordinates", type=int, default=16)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed0", type=int, default=100000)
    ap.add_argument("--family", default="config4", choices=["config4", "thin"],
                    help="training slabs: the config-4 family (default) or thin, strongly scattering "
                         "cells like the deployment slabs")
    ap.add_argument("--init", default="extrapolation", choices=["extrapolation", "random"],
                    help="starting parameters: linear extrapolation in time plus free channels "
                         "(extrapolation_params), or He-uniform (init_params)")
    ap.add_argument("--out", default=DEFAULT_WEIGHTS)
    ap.add_argument("--time-inference", type=int, metavar="J", default=0,
                    help="only time the inference of the weights at --out on a J-cell sample and print it")
    a = ap.parse_args()
    import torch
    torch.cuda.set_device(0)
    if a.time_inference:
        from . import load_library
        load_library()
        print(json.dumps(time_inference(load_weights(a.out), a.time_inference)))
        return
    t0 = time.time()
    problem = None
    if a.family == "thin":
        import workloads
        problem = (lambda sd: workloads.hetero(sd, J=a.cells, N=a.ordinates, n_steps=a.steps, dt=0.02,
                                               tau_range=(0.01, 0.1), c_range=(0.9, 0.999)))
    data = trajectories(range(a.seed0, a.seed0 + a.trajectories), J=a.cells, N=a.ordinates, n_steps=a.steps,
                        problem=problem)
    print(f"generated {a.trajectories} trajectories x {a.steps} steps in {time.time() - t0:.1f} s; "
          f"mean OCI iterations per step {data['iters'].mean():.1f}", flush=True)
    p0 = extrapolation_params() if a.init == "extrapolation" else init_params()
    params, hist = train(data, epochs=a.epochs, batch=a.batch, lr=a.lr, params=p0)
    os.makedirs(os.path.dirname(a.out), exist_ok=True)
    np.save(a.out, params)
    print(f"saved {params.size} parameters to {a.out}; final val loss {hist['val_loss']:.3e}")


if __name__ == "__main__":
    main()
