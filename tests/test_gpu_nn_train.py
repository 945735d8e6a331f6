"""oci_nn_train (include/oci_nn.h): the library's whole training procedure --
sample order, train/validation split, cosine schedule, minibatch gather -- is
the documented one: it matches oci_nn_train_step iterated by hand in the order
the header defines (Fisher-Yates passes driven by splitmix64), bit for bit.
The paper has no learned component; the network's gradient and Adam step are
pinned to the FP64 oracle in test_gpu_nn."""
import math

import numpy as np
import pytest
import torch

import paper_2305_13555_gb300 as pkg
from paper_2305_13555_gb300 import learned

pytestmark = pytest.mark.gpu

M64 = (1 << 64) - 1


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2305_13555_gb300 import build
    build.build()
    pkg.load_library()


def splitmix64(x):
    """Vigna's splitmix64 finaliser, as the header states it."""
    z = (x + 0x9E3779B97F4A7C15) & M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def shuffle_round(a, seed, r):
    for i in range(len(a) - 1, 0, -1):
        j = splitmix64((seed + (r << 32) + i) & M64) % (i + 1)
        a[i], a[j] = a[j], a[i]


def _data(T, S, J, seed=0):
    g = np.random.default_rng(seed)
    phi = np.cumsum(g.uniform(0.0, 1.0, (T, S + 1, J, 4)), axis=1)  # growing moments along each trajectory
    stat = g.normal(0.0, 1.0, (T, J, 4)).astype(np.float32)
    qfeat = g.uniform(0.0, 1.0, (T, J)).astype(np.float32)
    return (torch.tensor(phi, device="cuda"), torch.tensor(stat, device="cuda"), torch.tensor(qfeat, device="cuda"))


def _gather(phi, stat, qfeat, ks, S):
    t = torch.tensor([k // S for k in ks], device="cuda")
    n = torch.tensor([k % S + 1 for k in ks], device="cuda")
    return (phi[t, n].contiguous(), phi[t, n - 1].contiguous(), phi[t, torch.clamp(n - 2, min=0)].contiguous(),
            stat[t].contiguous(), qfeat[t].contiguous())


def _inputs(phi, stat, qfeat, ks, S, J):
    B = len(ks)
    phin, phi1, phi2, st, qf = _gather(phi, stat, qfeat, ks, S)
    inp = torch.empty((B, 13, J), dtype=torch.float32, device="cuda")
    tgt = torch.empty((B, 4, J), dtype=torch.float32, device="cuda")
    sc = torch.empty(B, dtype=torch.float32, device="cuda")
    pkg.oci_nn_features(phi1, phi2, st, qf, inp, sc)
    pkg.oci_nn_targets(phin, phi1, sc, tgt)
    return inp, tgt


def test_train_matches_train_step_iterated_by_hand():
    T, S, J, B, epochs, lr, seed, vf = 3, 4, 200, 2, 3, 3e-3, 12345, 0.25
    phi, stat, qfeat = _data(T, S, J)
    p0 = torch.tensor(learned.init_params(seed=2), device="cuda")
    out = torch.empty_like(p0)
    st = pkg.oci_nn_train(phi, stat, qfeat, out, epochs=epochs, batch=B, lr=lr, val_frac=vf, seed=seed,
                          init_params=p0)
    torch.cuda.synchronize()

    n_all = T * S
    n_val = int(math.floor(n_all * np.float32(vf)))
    order = list(range(n_all))
    shuffle_round(order, seed, 0)
    val, tr = order[:n_val], order[n_val:]
    p, m, v = p0.clone(), torch.zeros_like(p0), torch.zeros_like(p0)
    ws = torch.empty(pkg.oci_nn_workspace_bytes(B, J), dtype=torch.uint8, device="cuda")
    step = 0
    for ep in range(epochs):
        shuffle_round(tr, seed, ep + 1)
        lr_ep = float(np.float32(float(np.float32(lr)) * 0.5 * (1.0 + math.cos(math.pi * ep / epochs))))
        for b0 in range(0, len(tr) - B + 1, B):
            inp, tgt = _inputs(phi, stat, qfeat, tr[b0:b0 + B], S, J)
            step += 1
            pkg.oci_nn_train_step(p, m, v, step, lr_ep, inp, tgt, ws, want_loss=False)
    torch.cuda.synchronize()
    assert st["steps_done"] == step == epochs * ((n_all - n_val) // B)
    assert st["n_train"] == n_all - n_val and st["n_val"] == n_val and st["epochs_done"] == epochs
    assert torch.equal(out, p)
    # validation loss of the final parameters, minibatches of min(batch, n_val)
    vb = min(B, n_val)
    wsv = torch.empty(pkg.oci_nn_workspace_bytes(vb, J), dtype=torch.uint8, device="cuda")
    losses = []
    for b0 in range(0, n_val - vb + 1, vb):
        inp, tgt = _inputs(phi, stat, qfeat, val[b0:b0 + vb], S, J)
        losses.append(pkg.oci_nn_loss_grad(p, inp, tgt, None, wsv))
    assert abs(st["val_loss"] - np.mean(losses)) <= 1e-12 * abs(np.mean(losses))


def test_train_reduces_the_loss_from_the_library_initialisation():
    T, S, J = 4, 6, 256
    phi, stat, qfeat = _data(T, S, J, seed=1)
    out = torch.empty(pkg.oci_nn_param_count(), dtype=torch.float32, device="cuda")
    st1 = pkg.oci_nn_train(phi, stat, qfeat, out, epochs=1, batch=4, lr=1e-3, val_frac=0.2, seed=7)
    st30 = pkg.oci_nn_train(phi, stat, qfeat, out, epochs=30, batch=4, lr=1e-3, val_frac=0.2, seed=7)
    assert np.isfinite(st30["val_loss"]) and st30["val_loss"] < st1["val_loss"]
    assert torch.isfinite(out).all()


def test_train_rejects_bad_sizes():
    phi, stat, qfeat = _data(1, 2, 64)
    out = torch.empty(pkg.oci_nn_param_count(), dtype=torch.float32, device="cuda")
    with pytest.raises(pkg.OciError):
        pkg.oci_nn_train(phi, stat, qfeat, out, epochs=1, batch=8)  # 2 samples: not one full minibatch
    with pytest.raises(pkg.OciError):
        pkg.oci_nn_train(phi, stat, qfeat, out, epochs=1, batch=1, val_frac=1.0)
