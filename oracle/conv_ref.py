"""CPU oracle of the learned correction network: 3x3x3 'same' convolutions with ReLU, its backward
pass, the mean-squared-error loss and the Adam update, in plain numpy FP64.

TEST INFRASTRUCTURE ONLY (like the rest of `oracle/`): used by the tests and the smoke check to
verify the CUDA kernels; the product never imports it.

The correction network is not part of the paper (it is a learned flexible-preconditioner stage
added on top of the ILU sweep).  Layout conventions, shared with the CUDA kernels only through
this written definition:
  * a field on an nz x ny x nx grid (x fastest) with C channels is an array [nz, ny, nx, C];
  * a layer's weights W[dz, dy, dx, ci, co] (d = 0, 1, 2 meaning offsets -1, 0, +1) and bias b[co];
  * Y[z, y, x, co] = b[co] + sum_{dz,dy,dx,ci} X[z+dz-1, y+dy-1, x+dx-1, ci] W[dz, dy, dx, ci, co],
    with X = 0 outside the grid (zero 'same' padding);
  * every layer but the last is followed by ReLU.
"""
from __future__ import annotations

import numpy as np


def conv3d(X, W, b):
    """One 3x3x3 'same' convolution, written as the sum over the 27 shifted copies of X."""
    nz, ny, nx, ci = X.shape
    co = W.shape[4]
    P = np.zeros((nz + 2, ny + 2, nx + 2, ci))
    P[1:-1, 1:-1, 1:-1, :] = X
    Y = np.broadcast_to(b, (nz, ny, nx, co)).astype(np.float64).copy()
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                S = P[dz:dz + nz, dy:dy + ny, dx:dx + nx, :]
                Y += S @ W[dz, dy, dx]
    return Y


def forward(X, params):
    """params: list of (W, b).  Returns the list of layer outputs [A_1, ..., A_L] (ReLU applied to
    all but the last) and the pre-activations [Z_1, ..., Z_L]."""
    acts, pre = [], []
    A = X
    for li, (W, b) in enumerate(params):
        Z = conv3d(A, W, b)
        pre.append(Z)
        A = np.maximum(Z, 0.0) if li < len(params) - 1 else Z
        acts.append(A)
    return acts, pre


def conv3d_backward(X, W, dY):
    """Gradients of Y = conv3d(X, W, b) for the upstream gradient dY:
    dW[dz,dy,dx] = sum over voxels of X-shifted^T dY, db = sum of dY, dX = the convolution of dY with
    the spatially flipped, channel-transposed kernel."""
    nz, ny, nx, ci = X.shape
    P = np.zeros((nz + 2, ny + 2, nx + 2, ci))
    P[1:-1, 1:-1, 1:-1, :] = X
    dW = np.zeros_like(W)
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                S = P[dz:dz + nz, dy:dy + ny, dx:dx + nx, :].reshape(-1, ci)
                dW[dz, dy, dx] = S.T @ dY.reshape(-1, dY.shape[-1])
    db = dY.reshape(-1, dY.shape[-1]).sum(axis=0)
    Wf = W[::-1, ::-1, ::-1].transpose(0, 1, 2, 4, 3)
    dX = conv3d(dY, Wf, np.zeros(ci))
    return dX, dW, db


def mse(out, target):
    d = out - target
    return float(np.mean(d * d)), 2.0 * d / d.size


def backward(X, params, dOut):
    """Backpropagation through forward(): returns [(dW, db)] per layer and dX."""
    acts, pre = forward(X, params)
    grads = [None] * len(params)
    dA = dOut
    for li in range(len(params) - 1, -1, -1):
        dZ = dA if li == len(params) - 1 else dA * (pre[li] > 0.0)
        inp = X if li == 0 else acts[li - 1]
        dA, dW, db = conv3d_backward(inp, params[li][0], dZ)
        grads[li] = (dW, db)
    return grads, dA


def adam(p, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba) with bias correction; t counts from 1.  Returns new (p, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def bf16_round(a):
    """Round FP64 values to BF16 (to nearest even, directly from FP64) and widen back; uses the
    C oracle's rounding routine."""
    from . import round_bf16_bits
    bits = round_bf16_bits(np.ravel(a)).astype(np.uint32) << 16
    return bits.view(np.float32).astype(np.float64).reshape(np.shape(a))
