"""Pins for the correction-network oracle (oracle/conv_ref.py): the forward convolution against
torch's conv3d on CPU in FP64 (an independent library implementation), a 1x1x1 special case,
the backward pass against central finite differences, and Adam's first step against its closed
form.  CPU only."""
import numpy as np
import pytest

from oracle import conv_ref


def rand_params(rng, chans):
    return [(rng.normal(0, 0.3, (3, 3, 3, a, b)), rng.normal(0, 0.1, b)) for a, b in zip(chans[:-1], chans[1:])]


@pytest.mark.parametrize("shape,ci,co", [((4, 5, 6), 2, 3), ((3, 3, 3), 16, 16), ((1, 2, 7), 3, 1)])
def test_conv3d_matches_torch(shape, ci, co):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    X = rng.normal(size=shape + (ci,))
    W = rng.normal(size=(3, 3, 3, ci, co))
    b = rng.normal(size=co)
    Y = conv_ref.conv3d(X, W, b)
    xt = torch.tensor(X).permute(3, 0, 1, 2).unsqueeze(0)           # (1, ci, z, y, x)
    wt = torch.tensor(W).permute(4, 3, 0, 1, 2)                      # (co, ci, dz, dy, dx)
    ref = torch.nn.functional.conv3d(xt, wt, torch.tensor(b), padding=1)[0].permute(1, 2, 3, 0).numpy()
    assert np.max(np.abs(Y - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


def test_center_tap_is_scaling():
    rng = np.random.default_rng(1)
    X = rng.normal(size=(3, 4, 5, 1))
    W = np.zeros((3, 3, 3, 1, 1))
    W[1, 1, 1, 0, 0] = 2.5
    assert np.array_equal(conv_ref.conv3d(X, W, np.zeros(1)), 2.5 * X)


def test_shift_tap_moves_field_with_zero_padding():
    X = np.arange(2 * 3 * 4, dtype=float).reshape(2, 3, 4, 1)
    W = np.zeros((3, 3, 3, 1, 1))
    W[1, 1, 2, 0, 0] = 1.0  # dx = +1: Y[z,y,x] = X[z,y,x+1]
    Y = conv_ref.conv3d(X, W, np.zeros(1))
    assert np.array_equal(Y[..., :-1, 0], X[..., 1:, 0]) and np.all(Y[..., -1, 0] == 0)


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(2)
    chans = [2, 3, 3, 3, 1]
    params = rand_params(rng, chans)
    X = rng.normal(size=(3, 4, 4, 2))
    T = rng.normal(size=(3, 4, 4, 1))

    def loss(ps, x):
        acts, _ = conv_ref.forward(x, ps)
        return conv_ref.mse(acts[-1], T)[0]

    acts, _ = conv_ref.forward(X, params)
    _, dOut = conv_ref.mse(acts[-1], T)
    grads, dX = conv_ref.backward(X, params, dOut)
    h = 1e-6
    checks = 0
    for li in range(len(params)):
        for which in (0, 1):
            arr = params[li][which]
            flat = arr.reshape(-1)
            for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
                old = flat[idx]
                flat[idx] = old + h
                lp = loss(params, X)
                flat[idx] = old - h
                lm = loss(params, X)
                flat[idx] = old
                fd = (lp - lm) / (2 * h)
                an = grads[li][which].reshape(-1)[idx]
                assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (li, which, idx, fd, an)
                checks += 1
    flat = X.reshape(-1)
    for idx in rng.choice(flat.size, size=6, replace=False):
        old = flat[idx]
        flat[idx] = old + h
        lp = loss(params, X)
        flat[idx] = old - h
        lm = loss(params, X)
        flat[idx] = old
        assert abs((lp - lm) / (2 * h) - dX.reshape(-1)[idx]) <= 1e-6
    assert checks > 20


def test_adam_first_step_closed_form():
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    p1, m, v = conv_ref.adam(p, g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    # after one step m_hat = g and v_hat = g^2: the step is lr * g / (|g| + eps)
    assert np.allclose(p1, p - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)


def test_bf16_round_is_idempotent_and_close():
    x = np.random.default_rng(3).normal(size=200)
    r = conv_ref.bf16_round(x)
    assert np.array_equal(conv_ref.bf16_round(r), r)
    assert np.all(np.abs(r - x) <= 2.0 ** -8 * np.abs(x))  # half a unit in the last of 8 bits
