"""Pins for the learned stage's oracle (oracle/stage_ref.py), each fixed by something other than the
oracle's own formulas: closed forms on hand-made networks, the exact-solve limit, the fallback rules,
and the scale invariance the normalisation gives.  CPU only.

The nets used here are real 2 -> 16 -> 16 -> 16 -> 1 convolution layers (oracle_stage.identity_layers)
that reproduce one input channel exactly, so the pins also check the channel order, the grid layout
(x fastest) and the rescaling by sigma that the network path goes through."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import stage_ref
from paper_1606_00541_gb300 import synth


def _diag(d):
    n = len(d)
    return (np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), np.asarray(d, dtype=np.float64))


def _csr(A):
    return sp.csr_matrix((A[2], A[1], A[0]))


DIMS = (3, 2, 2)  # nx, ny, nz: 12 unknowns


def test_identity_net_closed_form_on_a_diagonal_matrix(orc):
    """Net(X) = X[...,0] gives c = sigma * r1 / sigma = r1, so alpha = sum d r^2 / sum d^2 r^2 and
    z = z1 + alpha r1 (accepted: the reduction is below 1 for a positive diagonal)."""
    rng = np.random.default_rng(0)
    d = rng.uniform(0.5, 3.0, 12)
    A = _diag(d)
    v, z1 = rng.normal(size=12), rng.normal(size=12)
    r = v - d * z1
    alpha = np.sum(d * r * r) / np.sum(d * d * r * r)
    out = stage_ref.stage_step(A, v, z1, stage_ref.identity_layers(), np.zeros(12), DIMS, rho=0.999)
    assert out["accepted"]
    assert abs(out["alpha"] - alpha) <= 1e-14 * alpha
    assert np.allclose(out["z"], z1 + alpha * r, rtol=0, atol=1e-14)
    # the same through the BF16-faithful path with exactly representable data
    v2 = np.array([1.0, -2.0, 0.5, 4.0, -1.0, 2.0, -0.5, 1.0, 3.0, -3.0, 0.25, -0.25])
    z0 = np.zeros(12)
    ones = _diag(np.ones(12))
    o2 = stage_ref.stage_step(ones, v2, z0, stage_ref.identity_layers(), np.zeros(12), DIMS, bf16=True)
    # r1 / sigma is not exactly BF16 here, so only the decision and the step direction are fixed
    assert o2["accepted"] and abs(o2["alpha"] - 1.0) < 2.0 ** -7


def test_negative_alpha_falls_back(orc):
    """Net(X) = -X[...,0] gives c = -r1 and, for an SPD matrix, alpha < 0: the stage returns z1."""
    A = synth.fv7_lognormal(3, seed=1)
    rng = np.random.default_rng(1)
    v, z1 = rng.normal(size=27), rng.normal(size=27)
    out = stage_ref.stage_step(A, v, z1, stage_ref.identity_layers(sign=-1.0), np.zeros(27), (3, 3, 3), rho=1e12)
    assert out["alpha"] < 0.0 and not out["accepted"]
    assert np.array_equal(out["z"], z1)


def test_tiny_rho_falls_back(orc):
    A = synth.fv7_lognormal(3, seed=2)
    rng = np.random.default_rng(2)
    v, z1 = rng.normal(size=27), rng.normal(size=27)
    out = stage_ref.stage_step(A, v, z1, stage_ref.identity_layers(), np.zeros(27), (3, 3, 3), rho=1e-12)
    assert out["alpha"] > 0.0 and not out["accepted"]
    assert np.array_equal(out["z"], z1)


def test_exact_solve_net_gives_the_exact_solution(orc):
    """A 'network' that returns A^-1 applied to its first channel makes c = A^-1 r1, A c = r1,
    alpha = 1, and z = z1 + A^-1 (v - A z1) = A^-1 v, whatever z1 is."""
    m = 5
    A = synth.fv7_lognormal(m, seed=3)
    As = _csr(A).tocsc()
    n = m ** 3
    rng = np.random.default_rng(3)
    v, z1 = rng.normal(size=n), rng.normal(size=n)

    def exact(X):
        return spla.spsolve(As, X[..., 0].reshape(-1))

    out = stage_ref.stage_step(A, v, z1, exact, np.zeros(n), (m, m, m), rho=0.5)
    x = spla.spsolve(As, v)
    assert out["accepted"] and abs(out["alpha"] - 1.0) <= 1e-10
    assert out["reduction"] <= 1e-10
    assert np.max(np.abs(out["z"] - x)) <= 1e-10 * np.max(np.abs(x))


def test_sigma_is_the_rms(orc):
    """Net(X) = X[...,0] + beta on A = I with sum(r1) = 0: c = r1 + sigma beta, and
    alpha = ||r1||^2 / (||r1||^2 + n sigma^2 beta^2), which equals 1 / (1 + beta^2) exactly when
    sigma^2 = ||r1||^2 / n."""
    r = np.array([1.0, -1.0, 2.0, -2.0, 3.0, -3.0, 0.5, -0.5, 1.5, -1.5, 4.0, -4.0])
    A = _diag(np.ones(12))
    for beta in (0.5, 1.0, 3.0):
        out = stage_ref.stage_step(A, r, np.zeros(12), stage_ref.identity_layers(bias=beta), np.zeros(12), DIMS,
                                   rho=1.0)
        assert abs(out["sigma"] - np.sqrt(np.mean(r * r))) <= 1e-15 * out["sigma"]
        assert abs(out["alpha"] - 1.0 / (1.0 + beta * beta)) <= 1e-14


def test_aux_channel_and_its_scale(orc):
    """Net(X) = X[...,1] = aux_scale * aux with aux = r1 gives c = sigma aux_scale r1 and, on A = I,
    z = z1 + r1 exactly for any aux_scale and sigma."""
    rng = np.random.default_rng(4)
    v, z1 = rng.normal(size=12), rng.normal(size=12)
    A = _diag(np.ones(12))
    r1 = v - z1
    for s in (0.5, 2.0):
        out = stage_ref.stage_step(A, v, z1, stage_ref.identity_layers(channel=1), r1, DIMS, rho=0.5, aux_scale=s)
        assert out["accepted"] and out["reduction"] <= 1e-14
        assert abs(out["alpha"] - 1.0 / (s * out["sigma"])) <= 1e-14 * out["alpha"]
        assert np.max(np.abs(out["z"] - (z1 + r1))) <= 1e-14


def test_grid_layout_x_fastest(orc):
    """A net that shifts its input by one cell along x (the dx = +1 tap): c_i = r1_{i+1} within each
    x line and 0 at the line's end, which fixes the flattening order of the grid."""
    nx, ny, nz = 4, 3, 2
    n = nx * ny * nz
    layers = stage_ref.identity_layers()
    W, b = layers[-1]
    W2 = np.zeros_like(W)
    W2[1, 1, 2] = W[1, 1, 1]  # read x + 1 instead of x
    layers[-1] = (W2, b)
    r = np.random.default_rng(5).normal(size=n)
    A = _diag(np.ones(n))
    out = stage_ref.stage_step(A, r, np.zeros(n), layers, np.zeros(n), (nx, ny, nz), rho=10.0)
    c = out["c"].reshape(nz, ny, nx)
    R = r.reshape(nz, ny, nx)
    assert np.allclose(c[..., :-1], R[..., 1:], rtol=0, atol=1e-14) and np.all(c[..., -1] == 0.0)


def test_zero_residual_returns_z1(orc):
    A = _diag(np.full(12, 2.0))
    z1 = np.arange(12.0)
    v = 2.0 * z1
    out = stage_ref.stage_step(A, v, z1, stage_ref.identity_layers(), np.zeros(12), DIMS)
    assert out["sigma"] == 0.0 and not out["accepted"] and np.array_equal(out["z"], z1)


@pytest.mark.parametrize("scale", [1e-3, 7.0])
def test_positive_homogeneity(orc, scale):
    """r1 / sigma does not change when v and z1 are scaled by s > 0, so z scales by s (any net)."""
    rng = np.random.default_rng(6)
    m = 4
    A = synth.fv7_lognormal(m, seed=6)
    n = m ** 3
    layers = [(rng.normal(0, 0.3, (3, 3, 3, a, b)), rng.normal(0, 0.1, b))
              for a, b in [(2, 16), (16, 16), (16, 16), (16, 1)]]
    v, z1, aux = rng.normal(size=n), rng.normal(size=n), rng.normal(size=n)
    o1 = stage_ref.stage_step(A, v, z1, layers, aux, (m, m, m), rho=10.0)
    o2 = stage_ref.stage_step(A, scale * v, scale * z1, layers, aux, (m, m, m), rho=10.0)
    assert o1["accepted"] == o2["accepted"]
    assert np.max(np.abs(o2["z"] - scale * o1["z"])) <= 1e-12 * scale * np.max(np.abs(o1["z"]))
