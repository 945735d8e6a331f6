"""FP64 plain-loop oracle of the 1-D convolutional network over cells.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The network (the learned initial guess / corrector of the OCI iteration; the
paper has no learned component, so its form is this implementation's
specification):
  5 convolution layers over the cell index, kernel width 5, zero padding of 2
  cells at both slab ends ("same" length), channels 13 -> 32 -> 32 -> 32 -> 32 -> 4,
  ReLU after the first four layers, none after the last.
  layer l: out[co][x] = b[co] + sum_{ci} sum_{k=0..4} W[co][ci][k] * in[ci][x + k - 2]
Parameters are flattened layer by layer as W (co, ci, k row-major) then b.
Loss: mean over outputs of (out - target)^2 (mean squared error).

Forward and backward are written as explicit loops over (co, ci, k) with numpy
vector operations over the cell index only, so each line can be checked
against the formula above.
"""
import numpy as np

KW = 5
PAD = 2
CHANNELS = (13, 32, 32, 32, 32, 4)


def param_shapes(channels=CHANNELS):
    return [((co, ci, KW), (co,)) for ci, co in zip(channels[:-1], channels[1:])]


def n_params(channels=CHANNELS):
    return sum(co * ci * KW + co for (co, ci, _), _ in param_shapes(channels))


def unflatten(theta, channels=CHANNELS):
    out, o = [], 0
    for (co, ci, kw), _ in param_shapes(channels):
        W = theta[o:o + co * ci * kw].reshape(co, ci, kw); o += co * ci * kw
        b = theta[o:o + co]; o += co
        out.append((W, b))
    return out


def conv_forward(x, W, b):
    """x [ci][J] -> [co][J] for one sample (zero padding at both ends)."""
    co_n, ci_n, kw = W.shape
    J = x.shape[1]
    xp = np.zeros((ci_n, J + 2 * PAD))
    xp[:, PAD:PAD + J] = x
    y = np.zeros((co_n, J))
    for co in range(co_n):
        acc = np.full(J, b[co], dtype=np.float64)
        for ci in range(ci_n):
            for k in range(kw):
                acc += W[co, ci, k] * xp[ci, k:k + J]
        y[co] = acc
    return y


def forward(theta, x, channels=CHANNELS):
    """x [B][13][J] -> (out [B][4][J], activations per layer for backward)."""
    layers = unflatten(np.asarray(theta, dtype=np.float64), channels)
    outs, acts = [], []
    for s in range(x.shape[0]):
        a = [np.asarray(x[s], dtype=np.float64)]
        h = a[0]
        for li, (W, b) in enumerate(layers):
            z = conv_forward(h, W, b)
            h = np.maximum(z, 0.0) if li < len(layers) - 1 else z
            a.append(h)
        outs.append(h)
        acts.append(a)
    return np.array(outs), acts


def mse(out, target):
    return float(np.mean((out - target) ** 2))


def backward(theta, x, target, channels=CHANNELS):
    """Gradient of mse(forward(theta, x), target) with respect to theta (flattened)."""
    layers = unflatten(np.asarray(theta, dtype=np.float64), channels)
    out, acts = forward(theta, x, channels)
    grads = [(np.zeros_like(W), np.zeros_like(b)) for W, b in layers]
    n_out = out.size
    for s in range(x.shape[0]):
        a = acts[s]
        g = 2.0 * (out[s] - target[s]) / n_out          # d loss / d output of the last layer
        for li in range(len(layers) - 1, -1, -1):
            W, b = layers[li]
            co_n, ci_n, kw = W.shape
            if li < len(layers) - 1:
                g = g * (a[li + 1] > 0.0)                 # through the ReLU
            J = g.shape[1]
            inp = a[li]
            xp = np.zeros((ci_n, J + 2 * PAD))
            xp[:, PAD:PAD + J] = inp
            dW, db = grads[li]
            for co in range(co_n):
                db[co] += g[co].sum()
                for ci in range(ci_n):
                    for k in range(kw):
                        dW[co, ci, k] += np.dot(g[co], xp[ci, k:k + J])
            # gradient with respect to this layer's input
            gx = np.zeros((ci_n, J + 2 * PAD))
            for co in range(co_n):
                for ci in range(ci_n):
                    for k in range(kw):
                        gx[ci, k:k + J] += W[co, ci, k] * g[co]
            g = gx[:, PAD:PAD + J]
    flat = []
    for dW, db in grads:
        flat.append(dW.ravel())
        flat.append(db)
    return np.concatenate(flat)


def adam_step(theta, m, v, grad, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba), bias-corrected, returns (theta, m, v)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
