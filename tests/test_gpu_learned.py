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


# shapes: one ragged x tile, and several 128-voxel x tiles (the tcgen05 tile) with ragged x, y
# and z tails, odd sample depths, one-plane samples and samples of several 8-plane z chunks
@pytest.mark.parametrize("tensor_cores", [True, False], ids=["tcgen05", "mma_sync"])
@pytest.mark.parametrize("dims,zs", [((40, 12, 6), 3), ((32, 4, 2), 2), ((70, 9, 5), 5), ((300, 5, 14), 7),
                                     ((129, 3, 4), 1), ((256, 2, 3), 3), ((130, 6, 19), 19)])
def test_forward_layer_parity(hec, dims, zs, tensor_cores):
    from paper_1606_00541_gb300 import learn
    rng = np.random.default_rng(1)
    p = learn.init_params(3, last_scale=1.0)
    net = hec.Net(p)
    net.set_engine(tensor_cores)
    layers = params_to_layers(p)
    xb, xd = rand_input(rng, dims, zs)
    out, acts = net.forward(xd, dims, zs=zs, acts=True)
    net.sync_status()
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


def test_engines_agree(hec):
    """The tcgen05 and mma.sync forward passes add the same BF16 products in FP32 in a different
    order.  The first layer (same input in both) differs by at most one BF16 unit in the last place,
    where the two sums straddle a rounding boundary; the layers after it see inputs that differ in
    those places, so they and the output are compared in norm."""
    from paper_1606_00541_gb300 import learn
    rng = np.random.default_rng(4)
    dims, zs = (200, 20, 24), 24
    net = hec.Net(learn.init_params(7, last_scale=1.0))
    _, xd = rand_input(rng, dims, zs)
    res = []
    for tc in (True, False):
        net.set_engine(tc)
        out, acts = net.forward(xd, dims, zs=zs, acts=True)
        net.sync_status()
        res.append((out.cpu().numpy().astype(np.float64), acts.float().cpu().numpy().astype(np.float64)))
    (o1, a1), (o0, a0) = res
    d = np.abs(a1[0] - a0[0])
    assert np.all(d <= 2.0 ** -7 * np.maximum(np.abs(a1[0]), np.abs(a0[0])) + 1e-6)
    assert np.mean(d > 0) < 0.05
    for li in (1, 2, 3):
        assert np.linalg.norm(a1[li] - a0[li]) <= 2.0 ** -8 * np.linalg.norm(a0[li]), li
    assert np.linalg.norm(o1 - o0) <= 2.0 ** -8 * np.linalg.norm(o0)


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


def test_backward_then_adam_equals_train_step(hec):
    """net_backward followed by net_adam_step is net_train_step: the same loss, gradients and
    updated parameters, bit for bit, over three steps."""
    from paper_1606_00541_gb300 import learn
    rng = np.random.default_rng(9)
    dims, zs = (32, 8, 4), 2
    p = learn.init_params(11, last_scale=1.0)
    a, b = hec.Net(p), hec.Net(p)
    _, xd = rand_input(rng, dims, zs)
    T = torch.as_tensor(rng.normal(size=int(np.prod(dims))).astype(np.float32), device="cuda")
    for _ in range(3):
        la = a.train_step(xd, T, dims, zs=zs, lr=2e-3)
        lb = b.backward(xd, T, dims, zs=zs)
        b.adam_step(lr=2e-3)
        pa, ga = a.params(grads=True)
        pb, gb = b.params(grads=True)
        assert la == lb and np.array_equal(ga, gb) and np.array_equal(pa, pb)


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


def layers_to_params(layers):
    """Oracle layers [(W[dz,dy,dx,ci,co], b)] -> the flat FP32 parameter array of the C ABI (weight
    (tap, ci, co) at (tap*16 + ci)*16 + co, tap = (dz*3 + dy)*3 + dx, then the 16 biases)."""
    p = np.zeros(4 * LAYER, dtype=np.float32)
    for li, (W, b) in enumerate(layers):
        ci, co = W.shape[3], W.shape[4]
        Wf = np.zeros((27, C, C), dtype=np.float32)
        Wf[:, :ci, :co] = W.reshape(27, ci, co)
        p[li * LAYER:li * LAYER + 27 * C * C] = Wf.reshape(-1)
        p[li * LAYER + 27 * C * C:li * LAYER + 27 * C * C + co] = b
    return p


def random_layers(seed, scale=0.3):
    """The identity net of the stage oracle with every weight and bias perturbed by seeded noise
    (He-normal times `scale`, as FP32 values): all 27 taps and 16 channels of every layer carry
    random values, while the output stays close enough to the first input channel that the step
    length alpha is positive."""
    from oracle import stage_ref
    rng = np.random.default_rng(seed)
    out = []
    for W0, b0 in stage_ref.identity_layers():
        ci = W0.shape[3]
        W = W0 + scale * rng.normal(0.0, np.sqrt(2.0 / (27 * ci)), size=W0.shape)
        b = b0 + 0.05 * scale * rng.normal(size=b0.shape)
        out.append((W.astype(np.float32).astype(np.float64), b.astype(np.float32).astype(np.float64)))
    return out


@pytest.mark.parametrize("net_kind", ["identity", "random"])
def test_stage_apply_matches_oracle(hec, net_kind):
    """One stage application (stage_apply through the C ABI) against oracle/stage_ref.stage_step on
    the same inputs: A, v, z1 = the oracle's FP64 ILU(0) apply, the same FP32 weights and the same
    aux field; the oracle evaluates the network BF16-faithfully (weights, inputs and hidden
    activations rounded as the kernels store them, FP64 arithmetic).  An x extent of 37 leaves a
    ragged 32-wide tile.
    - identity net (every weight +-1, output = its first input channel): the network path is exact
      in BF16, so c, alpha and z agree to the FP32 partial sums alpha is taken from (1e-5);
    - perturbed net (identity plus seeded noise on every weight and bias): c differs by
      accumulation order (FP32 against FP64) and the BF16
      rounding flips it causes in the hidden layers, 8 significant bits at worst per value:
      ||c - c_ref|| <= 2^-6 ||c_ref||, alpha within 2^-6, z within 2^-5 ||alpha c||.
    Both with rho = 1e12 (always accepted) and rho = 1e-12 (always the fallback, z = z1 bit for
    bit), and with rho between, the oracle's decision."""
    from oracle import ilu0, ilu_apply, stage_ref
    dims = (37, 20, 18)
    n = int(np.prod(dims))
    lnk = np.random.default_rng(np.random.PCG64(31)).normal(0.0, 2.0, size=n)
    nx, ny, nz = dims
    A = synth.fv7_lognormal_box(nx, ny, nz, perm=np.exp(lnk))
    L, U = ilu0(A)
    v = synth.uniform_vector(n, 8)
    z1 = ilu_apply(L, U, v)
    layers = stage_ref.identity_layers() if net_kind == "identity" else random_layers(41)
    net = hec.Net(layers_to_params(layers))
    Ad = [torch.as_tensor(a, device="cuda") for a in A]
    HA = hec.hec_from_csr(*Ad)
    aux = torch.as_tensor(lnk, device="cuda")
    vd, z1d = torch.as_tensor(v, device="cuda"), torch.as_tensor(z1, device="cuda")
    ref = stage_ref.stage_step(A, v, z1, layers, lnk, dims, rho=1e12, aux_scale=0.5, bf16=True)
    assert ref["alpha"] > 0.0 and ref["accepted"]
    stage = hec.Stage(net, HA, dims, aux, aux_scale=0.5, rho=1e12)
    z = stage.apply(vd, z1d).cpu().numpy()
    assert stage.stats()["accepted"] == 1
    ac = ref["alpha"] * ref["c"]
    if net_kind == "identity":
        assert np.max(np.abs(z - ref["z"])) <= 1e-5 * np.max(np.abs(ac)) + 1e-14 * np.max(np.abs(ref["z"]))
    else:
        c_gpu = (z - z1)  # = alpha_gpu c_gpu
        assert np.linalg.norm(c_gpu - ac) <= 2.0 ** -5 * np.linalg.norm(ac)
        assert abs(np.dot(c_gpu, ac) / np.dot(ac, ac) - 1.0) <= 2.0 ** -6
    print(net_kind, "alpha %.6f reduction %.4f, |z - z_ref| / |alpha c| = %.3e"
          % (ref["alpha"], ref["reduction"], np.linalg.norm(z - ref["z"]) / np.linalg.norm(ac)))
    # the fallback returns z1 itself
    never = hec.Stage(net, HA, dims, aux, aux_scale=0.5, rho=1e-12)
    assert torch.equal(never.apply(vd, z1d), z1d)
    assert not stage_ref.stage_step(A, v, z1, layers, lnk, dims, rho=1e-12, bf16=True)["accepted"]
    # a threshold on either side of the oracle's reduction gives the oracle's decision
    for rho in (ref["reduction"] * 1.05, ref["reduction"] * 0.95):
        st = hec.Stage(net, HA, dims, aux, aux_scale=0.5, rho=rho)
        st.apply(vd, z1d)
        assert bool(st.stats()["accepted"]) == (ref["reduction"] < rho), rho
