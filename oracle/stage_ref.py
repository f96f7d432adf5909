"""CPU oracle of the learned correction stage's gated step, in plain numpy FP64.

TEST INFRASTRUCTURE ONLY (like the rest of `oracle/`): the tests compare the CUDA stage with it;
the product never imports it.

The stage is not part of the paper.  It is a flexible-preconditioner step added after the ILU
sweep (Eq. 1 gives z1 = U^-1 L^-1 v), defined as follows, in this order:

  1. r1 = v - A z1                                  (the residual the ILU step leaves)
  2. sigma = sqrt(mean(r1^2))                       (RMS; the network sees unit-scale input)
  3. X = [r1 / sigma, aux_scale * aux]              (two channels on the nx x ny x nz grid)
  4. c = sigma * Net(X)                             (the network's output, rescaled)
  5. alpha = <r1, A c> / <A c, A c>                 (the step that minimises ||r1 - alpha A c||)
  6. accept when alpha > 0 and ||r1 - alpha A c|| < rho ||r1||
  7. z = z1 + alpha c when accepted, else z = z1    (the fallback is plain ILU)

When sigma = 0 (z1 already solves A z1 = v) there is nothing to correct and z = z1.  The network
is `conv_ref.forward` on the layers [(W, b)] (3x3x3 'same' convolutions, ReLU between layers), or
any callable X -> output field, so that hand-made nets can pin each step.

`bf16=True` evaluates the network as the tensor-core kernels store it: the weights and every
hidden layer's output rounded to BF16 (to nearest even, directly from FP64), the two input
channels rounded to FP32 first and then to BF16 (the kernels form them in FP32), biases and all
arithmetic in FP64.  The rest of the step is FP64 either way.
"""
from __future__ import annotations

import numpy as np

from . import conv_ref, spmv


def _field(a, dims):
    nx, ny, nz = dims
    return np.asarray(a, dtype=np.float64).reshape(nz, ny, nx)


def network(X, net, bf16=False):
    """Net(X) for X [nz, ny, nx, 2]; returns the output field [nz, ny, nx]."""
    if callable(net):
        return np.asarray(net(X), dtype=np.float64).reshape(X.shape[:3])
    if not bf16:
        acts, _ = conv_ref.forward(X, net)
        return acts[-1][..., 0]
    A = conv_ref.bf16_round(X.astype(np.float32).astype(np.float64))
    for li, (W, b) in enumerate(net):
        Z = conv_ref.conv3d(A, conv_ref.bf16_round(W), b)
        if li < len(net) - 1:
            A = conv_ref.bf16_round(np.maximum(Z, 0.0))
        else:
            A = Z
    return A[..., 0]


def stage_step(A, v, z1, net, aux, dims, rho=0.99, aux_scale=0.5, bf16=False):
    """One application of the stage (steps 1-7 above).  A is the CSR matrix (rowptr, col, val) of
    the n = nx*ny*nz grid unknowns (x fastest), v the vector to precondition, z1 = M^-1 v from
    the ILU step, aux the second input field.  Returns a dict with z and the intermediate values
    (r1, sigma, c, alpha, accepted, reduction = ||r1 - alpha A c|| / ||r1||)."""
    v = np.asarray(v, dtype=np.float64)
    z1 = np.asarray(z1, dtype=np.float64)
    n = v.size
    r1 = v - spmv(A, z1)
    sigma = float(np.sqrt(np.sum(r1 * r1) / n))
    out = {"r1": r1, "sigma": sigma, "c": np.zeros(n), "alpha": 0.0, "accepted": False, "reduction": 1.0}
    if sigma == 0.0:
        out["z"] = z1.copy()
        return out
    X = np.stack([_field(r1 / sigma, dims), _field(aux_scale * np.asarray(aux, dtype=np.float64), dims)], axis=-1)
    c = sigma * network(X, net, bf16).reshape(-1)
    Ac = spmv(A, c)
    AcAc = float(np.dot(Ac, Ac))
    alpha = float(np.dot(r1, Ac)) / AcAc if AcAc > 0.0 else 0.0
    red = float(np.linalg.norm(r1 - alpha * Ac) / np.linalg.norm(r1))
    accepted = alpha > 0.0 and red < rho
    out.update(c=c, alpha=alpha, reduction=red, accepted=accepted)
    out["z"] = z1 + alpha * c if accepted else z1.copy()
    return out


def identity_layers(channel=0, sign=1.0, bias=0.0, C=16):
    """A 2 -> 16 -> 16 -> 16 -> 1 network whose output is sign * X[..., channel] + bias exactly:
    the first layer splits the input into its positive and negative parts (ReLU keeps both), the
    middle layers copy them, the last layer recombines them.  Only centre taps are non-zero, and
    every weight is +-1, so the net is exact in BF16 as well."""
    chans = [(2, C), (C, C), (C, C), (C, 1)]
    layers = []
    for li, (ci, co) in enumerate(chans):
        W = np.zeros((3, 3, 3, ci, co))
        b = np.zeros(co)
        if li == 0:
            W[1, 1, 1, channel, 0] = 1.0
            W[1, 1, 1, channel, 1] = -1.0
        elif li < 3:
            W[1, 1, 1, 0, 0] = 1.0
            W[1, 1, 1, 1, 1] = 1.0
        else:
            W[1, 1, 1, 0, 0] = sign
            W[1, 1, 1, 1, 0] = -sign
            b[0] = bias
        layers.append((W, b))
    return layers
