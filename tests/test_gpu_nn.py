"""GPU kernels of the learned guess against the FP64 CNN oracle (oracle.nn).

Training kernels use BF16-rounded weights with FP32 activations and FP32
accumulation; the oracle is fed the same rounded weights in FP64, so the
remaining difference is FP32 accumulation over at most 32 channels x 5 taps
per layer: 1e-4 relative (to the largest component) for gradients summed over
hundreds of cells.  Inference runs on the tensor cores with every layer's
input rounded to BF16 too (see test_forward_matches_oracle for its bound).
"""
import numpy as np
import pytest
import torch

import paper_2305_13555_gb300 as pkg
from oracle import nn as onn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2305_13555_gb300 import build
    build.build()
    pkg.load_library()


def _bf16_round(theta):
    """Weights rounded to BF16 as the kernels use them; biases stay FP32."""
    t = torch.tensor(theta, dtype=torch.float32)
    out = t.clone()
    o = 0
    for (co, ci, kw), _ in onn.param_shapes():
        n = co * ci * kw
        out[o:o + n] = t[o:o + n].to(torch.bfloat16).to(torch.float32)
        o += n + co
    return out.double().numpy()


def _data(seed, B, J):
    g = np.random.default_rng(seed)
    theta = g.normal(0, 0.15, onn.n_params()).astype(np.float32)
    x = g.normal(0, 1, (B, 13, J)).astype(np.float32)
    t = g.normal(0, 0.5, (B, 4, J)).astype(np.float32)
    return theta, x, t


def test_param_count():
    assert pkg.oci_nn_param_count() == onn.n_params()


def _bf16(a):
    return torch.tensor(a, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()


def _forward_bf16_inputs(theta, x):
    """The oracle's layers with every layer's input rounded to BF16, as the
    tensor-core inference kernels take it (FP64 otherwise)."""
    layers = onn.unflatten(_bf16_round(theta))
    out = []
    for s in range(x.shape[0]):
        h = np.asarray(x[s], dtype=np.float64)
        for li, (W, b) in enumerate(layers):
            z = onn.conv_forward(_bf16(h), W, b)
            h = np.maximum(z, 0.0) if li < len(layers) - 1 else z
        out.append(h)
    return np.array(out)


@pytest.mark.parametrize("B,J", [(1, 7), (2, 300), (3, 129), (1, 240), (1, 241), (2, 479), (1, 4099), (4, 20000)])
def test_forward_matches_oracle(B, J):
    """Inference on the tensor cores (BF16 operands, FP32 accumulation), all
    five layers in one kernel over tiles of 240 cells (sizes below, at and
    across a tile, and more tiles than the persistent grid's CTAs), against
    the oracle fed the same BF16 rounding of weights and layer inputs.  The
    GPU rounds its FP32 sums to BF16 where the oracle rounds FP64 ones, so a
    value within FP32 rounding of a BF16 rounding boundary can land one BF16 ulp
    (2^-8 relative) apart and move the outputs downstream: the bound is a few
    such ulps of the output scale, and the mean error stays at FP32 level."""
    theta, x, _ = _data(1, B, J)
    ws = torch.empty(pkg.oci_nn_workspace_bytes(B, J), dtype=torch.uint8, device="cuda")
    out = torch.empty((B, 4, J), dtype=torch.float32, device="cuda")
    pkg.oci_nn_forward(torch.tensor(theta, device="cuda"), torch.tensor(x, device="cuda"), out, ws)
    torch.cuda.synchronize()
    ref = _forward_bf16_inputs(theta, x)
    err = np.abs(out.cpu().numpy() - ref)
    scale = max(1.0, np.abs(ref).max())
    assert err.max() < 1e-2 * scale
    assert err.mean() < 1e-4 * scale
    # and it is the same network as the FP32-activation form up to that rounding
    ref32, _ = onn.forward(_bf16_round(theta), x.astype(np.float64))
    assert np.abs(out.cpu().numpy() - ref32).max() < 5e-2 * max(1.0, np.abs(ref32).max())


@pytest.mark.parametrize("B,J", [(1, 9), (2, 260)])
def test_loss_grad_matches_oracle(B, J):
    theta, x, t = _data(2, B, J)
    ws = torch.empty(pkg.oci_nn_workspace_bytes(B, J), dtype=torch.uint8, device="cuda")
    grad = torch.empty(pkg.oci_nn_param_count(), dtype=torch.float32, device="cuda")
    loss = pkg.oci_nn_loss_grad(torch.tensor(theta, device="cuda"), torch.tensor(x, device="cuda"),
                                torch.tensor(t, device="cuda"), grad, ws)
    th = _bf16_round(theta)
    out, _ = onn.forward(th, x.astype(np.float64))
    ref_loss = onn.mse(out, t.astype(np.float64))
    ref_grad = onn.backward(th, x.astype(np.float64), t.astype(np.float64))
    assert abs(loss - ref_loss) < 1e-5 * ref_loss
    g = grad.cpu().numpy()
    assert np.abs(g - ref_grad).max() < 1e-4 * np.abs(ref_grad).max()


def test_train_step_adam_matches_oracle():
    B, J = 2, 64
    theta, x, t = _data(3, B, J)
    n = pkg.oci_nn_param_count()
    ws = torch.empty(pkg.oci_nn_workspace_bytes(B, J), dtype=torch.uint8, device="cuda")
    p = torch.tensor(theta, device="cuda")
    m = torch.zeros(n, device="cuda")
    v = torch.zeros(n, device="cuda")
    grad = torch.empty(n, dtype=torch.float32, device="cuda")
    pkg.oci_nn_loss_grad(p, torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda"), grad, ws)
    g = grad.cpu().double().numpy()
    pkg.oci_nn_train_step(p, m, v, 1, 1e-3, torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda"), ws)
    ref, _, _ = onn.adam_step(theta.astype(np.float64), np.zeros(n), np.zeros(n), g, 1)
    assert np.abs(p.cpu().double().numpy() - ref).max() < 1e-6


@pytest.mark.parametrize("B,J", [(1, 1), (2, 50), (3, 5000)])
def test_features_targets_predict_follow_their_definition(B, J):
    """The scale's sums of squares are split over blocks of 2048 elements of
    phi1 (one block below 512 cells, ten at 5000)."""
    g = np.random.default_rng(4)
    phi1 = g.uniform(0, 2, (B, J, 4)); phi2 = g.uniform(0, 2, (B, J, 4)); phin = g.uniform(0, 2, (B, J, 4))
    stat = g.normal(0, 1, (B, J, 4)).astype(np.float32); q = g.uniform(0, 1, (B, J)).astype(np.float32)
    d = lambda a: torch.tensor(a, device="cuda")
    inp = torch.empty((B, 13, J), dtype=torch.float32, device="cuda")
    scale = torch.empty(B, dtype=torch.float32, device="cuda")
    pkg.oci_nn_features(d(phi1), d(phi2), d(stat), d(q), inp, scale)
    tgt = torch.empty((B, 4, J), dtype=torch.float32, device="cuda")
    pkg.oci_nn_targets(d(phin), d(phi1), scale, tgt)
    phat = torch.empty((B, J, 4), dtype=torch.float64, device="cuda")
    pkg.oci_nn_predict(d(phi1), tgt, scale, phat)
    torch.cuda.synchronize()
    S = np.maximum(np.sqrt((phi1 ** 2).mean(axis=(1, 2))), np.sqrt((q.astype(np.float64) ** 2).mean(axis=1)))
    assert np.allclose(scale.cpu().numpy(), S, rtol=1e-6)
    I = inp.cpu().numpy()
    for b in range(B):
        assert np.allclose(I[b, 0:4], (phi1[b] / S[b]).T, rtol=1e-5, atol=1e-6)
        assert np.allclose(I[b, 4:8], ((phi1[b] - phi2[b]) / S[b]).T, rtol=1e-5, atol=1e-6)
        assert np.allclose(I[b, 8:12], stat[b].T)
        assert np.allclose(I[b, 12], q[b] / S[b], rtol=1e-5)
    # predict(targets) reproduces phi_n up to float rounding of the target
    assert np.abs(phat.cpu().numpy() - phin).max() < 1e-6 * np.abs(phin).max()


def test_training_reduces_loss():
    B, J = 4, 256
    g = np.random.default_rng(7)
    x = g.normal(0, 1, (B, 13, J)).astype(np.float32)
    # a target the network can represent: a local linear filter of the inputs
    t = np.stack([0.3 * x[:, 0] - 0.2 * np.roll(x[:, 4], 1, axis=1) + 0.1 * x[:, 9]] * 4, axis=1).astype(np.float32)
    n = pkg.oci_nn_param_count()
    p = torch.tensor(g.normal(0, 0.05, n).astype(np.float32), device="cuda")
    m = torch.zeros(n, device="cuda"); v = torch.zeros(n, device="cuda")
    ws = torch.empty(pkg.oci_nn_workspace_bytes(B, J), dtype=torch.uint8, device="cuda")
    xi, ti = torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda")
    first = pkg.oci_nn_train_step(p, m, v, 1, 3e-3, xi, ti, ws)
    for step in range(2, 301):
        last = pkg.oci_nn_train_step(p, m, v, step, 3e-3, xi, ti, ws, want_loss=(step == 300))
    assert last < 0.05 * first
