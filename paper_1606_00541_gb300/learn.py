"""Training of the learned correction stage (orchestration only: every numerical step runs in
libhec's CUDA kernels through the binding).

Data (the spec recipe): crops of the permeability field, each with its own 7-point
finite-volume matrix (Dirichlet at the crop boundary), the ILU(0) preconditioner with FP32
factor values (the one the stage will follow at solve time), seeded right-hand sides v, and
    z1 = M^-1 v,   r1 = v - A z1,   e1 = A^-1 r1 (FP64 FGMRES to 1e-10),
normalized by sigma = RMS(r1): input [r1 / sigma, ln k / 2], target e1 / sigma.  The network is
trained with the mean-squared error and Adam, samples stacked along z in minibatches.
"""
from __future__ import annotations

import ctypes
import time

import numpy as np
import torch

from . import hec, synth

C = 16
LAYER = 27 * C * C + C


def init_params(seed=0, last_scale=0.1):
    """He-normal weights for the used channels (2 -> 16 -> 16 -> 16 -> 1), zero biases, zeros for the
    unused channels; the last layer is scaled down so the initial correction is small."""
    rng = np.random.default_rng(seed)
    p = np.zeros(4 * LAYER, dtype=np.float32)
    chans = [(2, 16), (16, 16), (16, 16), (16, 1)]
    for li, (ci, co) in enumerate(chans):
        W = np.zeros((27, C, C), dtype=np.float32)
        std = np.sqrt(2.0 / (27 * ci)) * (last_scale if li == 3 else 1.0)
        W[:, :ci, :co] = rng.normal(0.0, std, size=(27, ci, co))
        p[li * LAYER: li * LAYER + 27 * C * C] = W.reshape(-1)
    return p


def crop_fields(lnk, m_full, crop, count, seed):
    """`count` seeded crop positions of a crop^3 window in an m_full^3 field (x fastest)."""
    rng = np.random.default_rng(seed)
    k3 = lnk.reshape(m_full, m_full, m_full)  # [z, y, x]
    out = []
    for _ in range(count):
        z, y, x = rng.integers(0, m_full - crop + 1, size=3)
        out.append(np.ascontiguousarray(k3[z:z + crop, y:y + crop, x:x + crop]).reshape(-1))
    return out


def make_pairs(lnk_crops, crop, rhs_per_crop=16, seed=0, aux_scale=0.5, solve_rtol=1e-10, vdt="f32"):
    """Training samples (x [n,16] bf16, target [n] f32) from each crop: see the module docstring."""
    samples = []
    n = crop ** 3
    for ci, lk in enumerate(lnk_crops):
        A = synth.fv7_lognormal(crop, perm=np.exp(lk))
        Ad = [torch.as_tensor(a, device="cuda") for a in A]
        Lh, Uh = hec.ilu_factor(*Ad, k=0)
        L, U = Lh.tensors(), Uh.tensors()
        s = hec.IluSolver(L, U, A=Ad, vdt=vdt, max_nrhs=rhs_per_crop)
        s64 = hec.IluSolver(L, U, A=Ad, vdt="f64", max_nrhs=rhs_per_crop)
        V = torch.as_tensor(synth.uniform_vector(n, seed + 1000 * ci, nrhs=rhs_per_crop), device="cuda")
        Z1 = s.apply(V)
        R1 = hec.spmv(s.A, Z1, V.clone(), alpha=-1.0, beta=1.0)
        E1, info = s64.solve(R1.contiguous(), rtol=solve_rtol, max_iters=4000, raise_on_nonconvergence=False)
        aux = torch.as_tensor(lk, device="cuda")
        for q in range(rhs_per_crop):
            x = torch.empty(n, C, dtype=torch.bfloat16, device="cuda")
            t = torch.empty(n, dtype=torch.float32, device="cuda")
            sig = torch.empty(1, dtype=torch.float64, device="cuda")
            r = R1[:, q].contiguous()
            e = E1[:, q].contiguous()
            hec._check(hec._lib.net_make_sample(ctypes.c_int(n), ctypes.c_void_p(r.data_ptr()),
                                                ctypes.c_void_p(e.data_ptr()), ctypes.c_void_p(aux.data_ptr()),
                                                ctypes.c_double(aux_scale), ctypes.c_void_p(x.data_ptr()),
                                                ctypes.c_void_p(t.data_ptr()), ctypes.c_void_p(sig.data_ptr()),
                                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)),
                       "net_make_sample")
            samples.append((x, t))
    return samples


def train(net, samples, crop, epochs=4, batch=8, lr=1e-3, seed=0, log=None):
    """Adam on minibatches of `batch` samples stacked along z.  Returns the loss history."""
    rng = np.random.default_rng(seed)
    hist = []
    n = crop ** 3
    for ep in range(epochs):
        order = rng.permutation(len(samples))
        for b0 in range(0, len(order) - batch + 1, batch):
            idx = order[b0:b0 + batch]
            X = torch.cat([samples[i][0] for i in idx], dim=0)
            T = torch.cat([samples[i][1] for i in idx], dim=0)
            loss = net.train_step(X, T, (crop, crop, crop * batch), zs=crop, lr=lr)
            hist.append(loss)
        if log:
            log("epoch %d loss %.4e" % (ep, float(np.mean(hist[-max(1, len(order) // batch):]))))
    return hist


def forward_timing(m, reps=10, seed=0):
    """Times the network's forward pass on an m^3 field (random input, seeded initial weights):
    returns (ms per forward, TFLOP/s counting the 16 x 16 channel products of every layer)."""
    net = hec.Net(init_params(seed))
    n = m ** 3
    g = torch.Generator(device="cuda").manual_seed(seed)
    x = torch.zeros(n, C, dtype=torch.bfloat16, device="cuda")
    x[:, :2] = torch.randn(n, 2, device="cuda", generator=g).to(torch.bfloat16)
    for _ in range(2):
        net.forward(x, (m, m, m))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        net.forward(x, (m, m, m))
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    return ms, 4 * n * 27 * C * C * 2 / ms / 1e9


def train_stage(lnk_full, m_full, crop=64, crops=125, rhs_per_crop=16, epochs=4, batch=8, lr=1e-3, seed=0,
                log=None):
    """Generates the pairs and trains a network from scratch; returns (net, info)."""
    t0 = time.perf_counter()
    fields = crop_fields(lnk_full, m_full, crop, crops, seed)
    samples = make_pairs(fields, crop, rhs_per_crop, seed)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    net = hec.Net(init_params(seed))
    hist = train(net, samples, crop, epochs, batch, lr, seed, log)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    return net, dict(pairs=len(samples), crop=crop, data_s=t1 - t0, train_s=t2 - t1, loss_first=hist[0] if hist else None,
                     loss_last=float(np.mean(hist[-10:])) if hist else None, steps=len(hist))


if __name__ == "__main__":
    import argparse

    ap = argparse.ArgumentParser(description="correction-network utilities")
    ap.add_argument("command", choices=["forward"])
    ap.add_argument("--size", type=int, default=128)
    ap.add_argument("--reps", type=int, default=10)
    a = ap.parse_args()
    ms, tf = forward_timing(a.size, a.reps)
    print("forward %d^3: %.3f ms, %.1f TFLOP/s" % (a.size, ms, tf))
