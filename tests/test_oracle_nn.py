"""Pins for the FP64 CNN oracle: torch's FP64 conv1d and autograd (library
routines), central finite differences, and torch.optim.Adam."""
import numpy as np
import pytest
import torch

from oracle import nn as onn

CH = (3, 5, 4, 2)   # small network with the same structure (kernel 5, same padding, ReLU between)


def _torch_forward(theta, x, channels):
    layers = onn.unflatten(theta, channels)
    h = x
    for li, (W, b) in enumerate(layers):
        h = torch.nn.functional.conv1d(h, W, b, padding=onn.PAD)
        if li < len(layers) - 1:
            h = torch.relu(h)
    return h


def _setup(seed, B=2, J=11, channels=CH):
    g = np.random.default_rng(seed)
    theta = g.normal(0, 0.4, onn.n_params(channels))
    x = g.normal(0, 1, (B, channels[0], J))
    t = g.normal(0, 1, (B, channels[-1], J))
    return theta, x, t


def test_forward_matches_torch_conv1d():
    theta, x, _ = _setup(1)
    out, _ = onn.forward(theta, x, CH)
    ref = _torch_forward(torch.tensor(theta), torch.tensor(x), CH).numpy()
    assert np.abs(out - ref).max() < 1e-13


def test_full_size_network_forward_matches_torch():
    g = np.random.default_rng(2)
    theta = g.normal(0, 0.1, onn.n_params())
    x = g.normal(0, 1, (1, 13, 40))
    out, _ = onn.forward(theta, x)
    ref = _torch_forward(torch.tensor(theta), torch.tensor(x), onn.CHANNELS).numpy()
    assert out.shape == (1, 4, 40)
    assert np.abs(out - ref).max() < 1e-12


def test_backward_matches_torch_autograd():
    theta, x, t = _setup(3)
    grad = onn.backward(theta, x, t, CH)
    th = torch.tensor(theta, requires_grad=True)
    out = _torch_forward(th, torch.tensor(x), CH)
    loss = torch.mean((out - torch.tensor(t)) ** 2)
    loss.backward()
    assert np.abs(grad - th.grad.numpy()).max() < 1e-12


def test_backward_matches_finite_differences():
    theta, x, t = _setup(4, B=1, J=7)
    grad = onn.backward(theta, x, t, CH)
    h = 1e-6
    idx = np.random.default_rng(5).choice(theta.size, 25, replace=False)
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (onn.mse(onn.forward(tp, x, CH)[0], t) - onn.mse(onn.forward(tm, x, CH)[0], t)) / (2 * h)
        assert abs(fd - grad[i]) < 1e-7 * max(1.0, abs(grad[i]))


def test_adam_matches_torch():
    g = np.random.default_rng(6)
    theta = g.normal(0, 1, 10)
    th = torch.tensor(theta.copy(), requires_grad=True)
    opt = torch.optim.Adam([th], lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    m, v = np.zeros(10), np.zeros(10)
    for step in range(1, 6):
        grad = g.normal(0, 1, 10)
        theta, m, v = onn.adam_step(theta, m, v, grad, step)
        th.grad = torch.tensor(grad)
        opt.step()
    assert np.abs(theta - th.detach().numpy()).max() < 1e-14
