"""The learned correction stage on the GPU: forward, gradients and the Adam step against the FP64
oracle (oracle/conv_ref.py), the stage inside FGMRES (fallback and acceptance), and what a trained
network gains over plain ILU-FGMRES."""
import numpy as np
import pytest
import torch

from oracle import conv_ref
from paper_1606_00541_gb300 import synth

pytestmark = pytest.mark.gpu

C = 16
LAYER = 27 * C * C + C


@pytest.fixture(scope="module")
def hec():
    from paper_1606_00541_gb300 import hec as h
    return h


def params_to_layers(p):
    """Flat FP32 parameters -> oracle layers [(W[dz,dy,dx,ci,co], b)] with the real channel counts."""
    chans = [(2, 16), (16, 16), (16, 16), (16, 1)]
    out = []
    for li, (ci, co) in enumerate(chans):
        blk = p[li * LAYER:(li + 1) * LAYER].astype(np.float64)
        W = blk[:27 * C * C].reshape(3, 3, 3, C, C)[:, :, :, :ci, :co]
        out.append((W, blk[27 * C * C:27 * C * C + co]))
    return out


def bf(a):
    return conv_ref.bf16_round(a)


def rand_input(rng, dims, zs):
    nx, ny, nz = dims
    n = nx * ny * nz
    x = np.zeros((n, C))
    x[:, 0] = rng.normal(size=n)
    x[:, 1] = rng.normal(size=n) * 0.5
    xb = bf(x)
    return xb, torch.as_tensor(xb, dtype=torch.float32, device="cuda").to(torch.bfloat16).contiguous()


def field(a, dims, zs, c):
    """[n, c] -> list of per-sample oracle arrays [zs, ny, nx, c]."""
    nx, ny, nz = dims
    a = a.reshape(nz, ny, nx, -1)[..., :c]
    return [a[s * zs:(s + 1) * zs] for s in range(nz // zs)]


@pytest.mark.parametrize("dims,zs", [((40, 12, 6), 3), ((32, 4, 2), 2), ((70, 9, 5), 5)])
def test_forward_layer_parity(hec, dims, zs):
    from paper_1606_00541_gb300 import learn
    rng = np.random.default_rng(1)
    p = learn.init_params(3, last_scale=1.0)
    net = hec.Net(p)
    layers = params_to_layers(p)
    xb, xd = rand_input(rng, dims, zs)
    out, acts = net.forward(xd, dims, zs=zs, acts=True)
    acts = acts.float().cpu().numpy().astype(np.float64)
    out = out.cpu().numpy().astype(np.float64)
    inp = xb
    cin = [2, 16, 16, 16]
    for li, (W, b) in enumerate(layers):
        Wb = bf(W)  # the kernels use BF16 weights, FP32 biases
        got = field(acts[li], dims, zs, W.shape[-1])
        for s, xs in enumerate(field(inp, dims, zs, cin[li])):
            ref = conv_ref.conv3d(xs, Wb, b.astype(np.float32).astype(np.float64))
            if li < 3:
                ref = np.maximum(ref, 0.0)
            scale = np.max(np.abs(ref)) + 1e-30
            # one BF16 rounding of the output, plus FP32 accumulation-order differences
            assert np.all(np.abs(got[s] - ref) <= 2.0 ** -7 * np.abs(ref) + 1e-5 * scale), (li, s)
            if li == 3:
                o = field(out, dims, zs, 1)[s]
                assert np.max(np.abs(o - ref)) <= 1e-5 * scale
        inp = acts[li]


def test_gradients_and_adam_match_oracle(hec):
    from paper_1606_00541_gb300 import learn
    rng = np.random.default_rng(2)
    dims, zs = (32, 8, 6), 3
    p = learn.init_params(5, last_scale=1.0)
    net = hec.Net(p)
    xb, xd = rand_input(rng, dims, zs)
    n = int(np.prod(dims))
    tgt = rng.normal(size=n).astype(np.float32)
    loss = net.train_step(xd, torch.as_tensor(tgt, device="cuda"), dims, zs=zs, lr=1e-3, update=False)
    _, g = net.params(grads=True)
    # oracle: same BF16 weights and input, FP64 everywhere else
    layers = [(bf(W), b.astype(np.float32).astype(np.float64)) for W, b in params_to_layers(p)]
    nz, ny, nx = dims[2], dims[1], dims[0]
    X = xb.reshape(nz, ny, nx, C)[..., :2]
    T = tgt.astype(np.float64).reshape(nz, ny, nx, 1)
    gsum = [[np.zeros_like(W), np.zeros_like(b)] for W, b in layers]
    lsum = 0.0
    for s in range(nz // zs):
        Xs, Ts = X[s * zs:(s + 1) * zs], T[s * zs:(s + 1) * zs]
        acts, _ = conv_ref.forward(Xs, layers)
        d = acts[-1] - Ts
        lsum += float(np.sum(d * d))
        grads, _ = conv_ref.backward(Xs, layers, 2.0 * d / n)
        for li in range(4):
            gsum[li][0] += grads[li][0]
            gsum[li][1] += grads[li][1]
    assert abs(loss - lsum / n) <= 1e-2 * lsum / n
    # strict oracle: the GPU's own BF16 activations, and BF16 rounding of every data gradient it
    # stores, with FP64 arithmetic otherwise; only accumulation order (and rare rounding flips)
    # remains between the two
    out, acts = net.forward(xd, dims, zs=zs, acts=True)
    acts = acts.float().cpu().numpy().astype(np.float64)
    outn = out.cpu().numpy().astype(np.float64)
    strict = [[np.zeros_like(W), np.zeros_like(b)] for W, b in layers]
    cin = [2, 16, 16, 16]
    cout = [16, 16, 16, 1]
    for s in range(nz // zs):
        sl = slice(s * zs * ny * nx, (s + 1) * zs * ny * nx)
        a_in = [xb[sl]] + [acts[li][sl] for li in range(3)]
        dA = bf((2.0 * (outn[sl] - tgt[sl].astype(np.float64)) / n).astype(np.float32).astype(np.float64))
        dA = dA.reshape(zs, ny, nx, 1)
        for li in range(3, -1, -1):
            dZ = dA if li == 3 else dA * (acts[li][sl].reshape(zs, ny, nx, C)[..., :cout[li]] > 0)
            Ain = a_in[li].reshape(zs, ny, nx, C)[..., :cin[li]]
            dX, dW, db = conv_ref.conv3d_backward(Ain, layers[li][0], dZ)
            strict[li][0] += dW
            strict[li][1] += db
            dA = bf(dX)
    chans = [(2, 16), (16, 16), (16, 16), (16, 1)]
    for li, (ci, co) in enumerate(chans):
        blk = g[li * LAYER:(li + 1) * LAYER].astype(np.float64)
        gW = blk[:27 * C * C].reshape(3, 3, 3, C, C)
        gb = blk[27 * C * C:]
        sW, sb = strict[li]
        assert np.linalg.norm(gW[..., :ci, :co] - sW) <= 2e-3 * np.linalg.norm(sW), li
        assert np.linalg.norm(gb[:co] - sb) <= 2e-3 * np.linalg.norm(sb) + 1e-12, li
        assert np.all(gW[..., ci:, :] == 0) and np.all(gW[..., :, co:] == 0) and np.all(gb[co:] == 0)
        # against the pure FP64 chain the BF16 path drifts by a few percent but points the same way
        rW = gsum[li][0]
        cos = np.sum(gW[..., :ci, :co] * rW) / (np.linalg.norm(gW[..., :ci, :co]) * np.linalg.norm(rW))
        assert cos >= 0.995, (li, cos)
    # one Adam step against the oracle's update from the GPU's own gradients
    net.train_step(xd, torch.as_tensor(tgt, device="cuda"), dims, zs=zs, lr=1e-3, update=True)
    p1, g1 = net.params(grads=True)
    ref, _, _ = conv_ref.adam(p.astype(np.float64), g1.astype(np.float64), 0.0, 0.0, 1, lr=1e-3)
    assert np.max(np.abs(p1 - ref)) <= 1e-6


def test_training_reduces_loss(hec):
    from paper_1606_00541_gb300 import learn
    rng = np.random.default_rng(4)
    dims, zs = (32, 16, 16), 16
    net = hec.Net(learn.init_params(7))
    xb, xd = rand_input(rng, dims, zs)
    # a target the network can represent: a smoothed copy of channel 0
    x0 = xb[:, 0].reshape(16, 16, 32)
    t = (x0 + np.roll(x0, 1, 2) + np.roll(x0, -1, 2)) / 3.0
    T = torch.as_tensor(t.reshape(-1).astype(np.float32), device="cuda")
    losses = [net.train_step(xd, T, dims, zs=zs, lr=3e-3) for _ in range(60)]
    assert losses[-1] < 0.5 * losses[0]


def _fv_problem(m, seed):
    lnk = np.random.default_rng(np.random.PCG64(seed)).normal(0.0, 2.0, size=m ** 3)
    A = synth.fv7_lognormal(m, perm=np.exp(lnk))
    return A, lnk


def test_stage_fallback_and_acceptance(hec):
    from paper_1606_00541_gb300 import learn
    m = 24
    A, lnk = _fv_problem(m, 11)
    n = m ** 3
    Ad = [torch.as_tensor(a, device="cuda") for a in A]
    Lh, Uh = hec.ilu_factor(*Ad, k=0)
    s = hec.IluSolver(Lh.tensors(), Uh.tensors(), A=Ad, vdt="f32")
    b = hec.spmv(s.A, torch.as_tensor(synth.uniform_vector(n, 3), device="cuda"))
    _, plain = s.solve(b, rtol=1e-8)
    net = hec.Net(learn.init_params(1))
    aux = torch.as_tensor(lnk, device="cuda")
    # rho tiny: the correction can never pass the test, so every application falls back to plain ILU
    never = hec.Stage(net, s.A, (m, m, m), aux, rho=1e-12)
    _, info = hec.fgmres_solve(s.A, s.M, b, stage=never, rtol=1e-8)
    st = never.stats()
    assert st["accepted"] == 0 and st["applied"] >= info["iterations"]
    assert info["converged"] and info["iterations"] == plain["iterations"]
    # rho huge: every positive-alpha correction is accepted; the solve still reaches 1e-8
    always = hec.Stage(net, s.A, (m, m, m), aux, rho=1e12)
    x, info2 = hec.fgmres_solve(s.A, s.M, b, stage=always, rtol=1e-8, max_iters=3000)
    assert info2["converged"] and always.stats()["applied"] >= info2["iterations"]
    r = b - hec.spmv(s.A, x)
    assert float(torch.linalg.norm(r) / torch.linalg.norm(b)) <= 1e-8 * (1 + 1e-6)


def test_trained_stage_gain(hec):
    """Trains on crops of one log-normal field and solves on another field of the same statistics:
    reports iterations with and without the stage; the stage must converge and must not need more
    iterations than plain ILU-FGMRES."""
    from paper_1606_00541_gb300 import learn
    m_train, crop, m = 48, 16, 32
    lnk_train = np.random.default_rng(np.random.PCG64(21)).normal(0.0, 2.0, size=m_train ** 3)
    net, tinfo = learn.train_stage(lnk_train, m_train, crop=crop, crops=24, rhs_per_crop=16, epochs=6, batch=8,
                                   lr=2e-3, seed=3)
    assert tinfo["loss_last"] < tinfo["loss_first"]
    A, lnk = _fv_problem(m, 22)
    n = m ** 3
    Ad = [torch.as_tensor(a, device="cuda") for a in A]
    Lh, Uh = hec.ilu_factor(*Ad, k=0)
    s = hec.IluSolver(Lh.tensors(), Uh.tensors(), A=Ad, vdt="f32")
    b = hec.spmv(s.A, torch.as_tensor(synth.uniform_vector(n, 5), device="cuda"))
    _, plain = s.solve(b, rtol=1e-8, max_iters=3000)
    stage = hec.Stage(net, s.A, (m, m, m), torch.as_tensor(lnk, device="cuda"), rho=0.99)
    x, learned = hec.fgmres_solve(s.A, s.M, b, stage=stage, rtol=1e-8, max_iters=3000)
    st = stage.stats()
    print("plain ILU-FGMRES %d iterations; with the learned stage %d iterations (%d of %d corrections accepted); "
          "train loss %.3e -> %.3e" % (plain["iterations"], learned["iterations"], st["accepted"], st["applied"],
                                       tinfo["loss_first"], tinfo["loss_last"]))
    assert learned["converged"]
    assert learned["iterations"] <= plain["iterations"]


def test_stage_apply_matches_its_definition(hec):
    """One stage application against the stage's definition assembled from separate calls: r1 =
    v - A z1, sigma = RMS(r1), c = sigma Net([r1 / sigma, aux / 2]) (the network run on the packed
    sample of net_make_sample), alpha = <r1, Ac> / <Ac, Ac>, z = z1 + alpha c.  The stage reads r1
    and aux directly in its first layer and writes c from its last, so this checks the fused
    input and output paths; an x extent of 37 leaves a ragged 32-wide tile."""
    import ctypes
    from paper_1606_00541_gb300 import learn
    dims = (37, 20, 18)
    n = int(np.prod(dims))
    lnk = np.random.default_rng(np.random.PCG64(31)).normal(0.0, 2.0, size=n)
    nx, ny, nz = dims
    A = synth.fv7_lognormal_box(nx, ny, nz, perm=np.exp(lnk))
    Ad = [torch.as_tensor(a, device="cuda") for a in A]
    Lh, Uh = hec.ilu_factor(*Ad, k=0)
    s = hec.IluSolver(Lh.tensors(), Uh.tensors(), A=Ad, vdt="f32")
    net = hec.Net(learn.init_params(4, last_scale=1.0))
    aux = torch.as_tensor(lnk, device="cuda")
    v = torch.as_tensor(synth.uniform_vector(n, 8), device="cuda")
    z1 = s.apply(v)
    stage = hec.Stage(net, s.A, dims, aux, rho=1e12)
    z = stage.apply(v, z1)
    # the definition, one call at a time
    r1 = hec.spmv(s.A, z1, v.clone(), alpha=-1.0, beta=1.0)
    x = torch.empty(n, C, dtype=torch.bfloat16, device="cuda")
    sig = torch.empty(1, dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    hec._check(hec._lib.net_make_sample(ctypes.c_int(n), ctypes.c_void_p(r1.data_ptr()), None,
                                        ctypes.c_void_p(aux.data_ptr()), ctypes.c_double(0.5),
                                        ctypes.c_void_p(x.data_ptr()), None, ctypes.c_void_p(sig.data_ptr()),
                                        ctypes.c_void_p(st)), "net_make_sample")
    out = net.forward(x, dims)
    c = sig * out.double()
    Ac = hec.spmv(s.A, c)
    alpha = float(torch.dot(r1, Ac) / torch.dot(Ac, Ac))
    assert alpha > 0.0
    zr = z1 + alpha * c
    # the stage takes alpha's inner products with FP32 partial sums: alpha within ~1e-6
    tol = 1e-5 * float(torch.max(torch.abs(alpha * c))) + 1e-12 * float(torch.max(torch.abs(zr)))
    assert float(torch.max(torch.abs(z - zr))) <= tol
    assert stage.stats()["accepted"] == 1
    # the fallback returns z1 itself
    never = hec.Stage(net, s.A, dims, aux, rho=1e-12)
    assert torch.equal(never.apply(v, z1), z1)
