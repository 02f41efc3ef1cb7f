"""FP64 CPU oracle of the learned grid surrogate's network (numpy).

TEST INFRASTRUCTURE ONLY: called by the tests (gradient checks and parity of the CUDA network kernels)
and by nothing on the product path. The surrogate is this project's extension of the method: the
paper has no learned component in its simulator, so there is no passage to cite for the network; each
function states the definition it writes out.

Layout (shared with the CUDA kernels' C-ABI, not their code): activations channels-last (D, H, W, C);
conv weights (27, Cout, Cin) with tap t = (dz * 3 + dy) * 3 + dx for offsets (dz - 1, dy - 1, dx - 1)
along (D, H, W); biases (Cout,).
"""
from __future__ import annotations

import numpy as np

TAPS = [(dz - 1, dy - 1, dx - 1) for dz in range(3) for dy in range(3) for dx in range(3)]


def _shifted(x, o):
    """x[p + o] with zeros outside the array (x: (D, H, W, C), o: offset per spatial axis)."""
    out = np.zeros_like(x)
    src, dst = [], []
    for n, oo in zip(x.shape[:3], o):
        src.append(slice(max(oo, 0), n + min(oo, 0)))
        dst.append(slice(max(-oo, 0), n - max(oo, 0)))
    out[tuple(dst)] = x[tuple(src)]
    return out


def conv3d_forward(x, w, b=None):
    """y[p, co] = b[co] + sum_{t, ci} x[p + o_t, ci] w[t, co, ci]: a 3x3x3 cross-correlation with zero
    padding of one voxel (output size = input size)."""
    x = np.asarray(x, np.float64)
    w = np.asarray(w, np.float64)
    y = np.zeros(x.shape[:3] + (w.shape[1],))
    for t, o in enumerate(TAPS):
        y += _shifted(x, o) @ w[t].T
    if b is not None:
        y += np.asarray(b, np.float64)
    return y


def conv3d_backward_data(dy, w):
    """Adjoint of the forward map in x: dx[q, ci] = sum_t sum_co dy[q - o_t, co] w[t, co, ci]."""
    dy = np.asarray(dy, np.float64)
    w = np.asarray(w, np.float64)
    dx = np.zeros(dy.shape[:3] + (w.shape[2],))
    for t, o in enumerate(TAPS):
        dx += _shifted(dy @ w[t], tuple(-oo for oo in o))
    return dx


def conv3d_backward_weight(x, dy):
    """dw[t, co, ci] = sum_p dy[p, co] x[p + o_t, ci]; db[co] = sum_p dy[p, co]."""
    x = np.asarray(x, np.float64)
    dy = np.asarray(dy, np.float64)
    C_in, C_out = x.shape[3], dy.shape[3]
    dw = np.zeros((27, C_out, C_in))
    dyf = dy.reshape(-1, C_out)
    for t, o in enumerate(TAPS):
        dw[t] = dyf.T @ _shifted(x, o).reshape(-1, C_in)
    return dw, dyf.sum(axis=0)


def relu(x):
    return np.maximum(x, 0.0)


def relu_backward(dy, act):
    """Gradient through y = max(z, 0) given the activation y (zero where y <= 0)."""
    return np.where(np.asarray(act) > 0.0, dy, 0.0)


def net_forward(params, x):
    """The surrogate network: conv -> ReLU -> conv -> ReLU -> conv -> ReLU -> conv (no final ReLU).
    params: list of (w, b) per layer. Returns the activations [x, a1, a2, a3, y]."""
    acts = [np.asarray(x, np.float64)]
    for i, (w, b) in enumerate(params):
        z = conv3d_forward(acts[-1], w, b)
        acts.append(relu(z) if i + 1 < len(params) else z)
    return acts


def mse_loss(pred, target, mask):
    """L = sum over masked voxels and all channels of (pred - target)^2, divided by (masked voxels x C).
    Returns (L, dL/dpred)."""
    pred = np.asarray(pred, np.float64)
    target = np.asarray(target, np.float64)
    m = np.asarray(mask, np.float64)[..., None]
    count = max(float(m.sum()) * pred.shape[-1], 1.0)
    d = (pred - target) * m
    return float((d * d).sum() / count), 2.0 * d / count


def net_backward(params, acts, dy):
    """Gradients of a scalar loss with dL/dy = dy through the network: returns [(dw, db)] per layer."""
    grads = [None] * len(params)
    g = np.asarray(dy, np.float64)
    for i in range(len(params) - 1, -1, -1):
        w, _ = params[i]
        grads[i] = conv3d_backward_weight(acts[i], g)
        if i > 0:
            g = relu_backward(conv3d_backward_data(g, w), acts[i])
    return grads


def adam_step(p, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015) with bias correction, step t >= 1. Returns (p, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
