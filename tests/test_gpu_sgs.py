"""Symmetric Gauss-Seidel on the level-scheduled sweeps (the smoother use of the triangular solver,
Sec. 1) against the oracle's plain loops: the triangles split on the GPU, forward sweep on
(D + L), backward sweep on (D + U), FP64 within 1e-12."""
import numpy as np
import pytest
import torch

import oracle
from paper_1606_00541_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hec():
    from paper_1606_00541_gb300 import hec as h
    return h


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def relmax(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("name", ["fv7_16", "27pt_11", "poisson2d_50"])
def test_triangles_bit_exact(hec, name):
    A = {"fv7_16": lambda: synth.fv7_lognormal(16, seed=4), "27pt_11": lambda: synth.stencil27_jitter(11, seed=2),
         "poisson2d_50": lambda: synth.poisson2d_5pt(50)}[name]()
    rp, ci, v = A
    n = len(rp) - 1
    rows = np.repeat(np.arange(n), np.diff(rp))
    Ad = [dev(a) for a in A]
    for uplo in (0, 1):
        for strict in (False, True):
            keep = (ci < rows if strict else ci <= rows) if uplo == 0 else (ci > rows if strict else ci >= rows)
            T = [t.cpu().numpy() for t in hec.csr_triangle(*Ad, uplo, strict).tensors()]
            ref_rp = np.concatenate([[0], np.cumsum(np.bincount(rows[keep], minlength=n))])
            assert np.array_equal(T[0], ref_rp) and np.array_equal(T[1], ci[keep]) and np.array_equal(T[2], v[keep])


@pytest.mark.parametrize("name,sweeps", [("fv7_16", 3), ("27pt_11", 2), ("poisson2d_50", 4)])
def test_sgs_matches_oracle(hec, name, sweeps):
    A = {"fv7_16": lambda: synth.fv7_lognormal(16, seed=4), "27pt_11": lambda: synth.stencil27_jitter(11, seed=2),
         "poisson2d_50": lambda: synth.poisson2d_5pt(50)}[name]()
    n = len(A[0]) - 1
    b = synth.uniform_vector(n, 1)
    x0 = synth.uniform_vector(n, 2)
    sm = hec.SgsSmoother([dev(a) for a in A])
    x = sm.smooth(dev(x0), dev(b), sweeps).cpu().numpy()
    assert relmax(x, oracle.sgs(A, b, x0, sweeps)) <= 1e-12


def test_sgs_several_rhs(hec):
    A = synth.fv7_lognormal(12, seed=6)
    n = 12 ** 3
    B = synth.uniform_vector(n, 3, nrhs=4)
    sm = hec.SgsSmoother([dev(a) for a in A], max_nrhs=4)
    X = sm.smooth(torch.zeros(n, 4, dtype=torch.float64, device="cuda"), dev(B), 2).cpu().numpy()
    for q in range(4):
        assert relmax(X[:, q], oracle.sgs(A, B[:, q], np.zeros(n), 2)) <= 1e-12


def test_sgs_reduces_the_residual(hec):
    A = synth.poisson3d_7pt(20)
    n = 20 ** 3
    b = synth.uniform_vector(n, 4)
    Ad = [dev(a) for a in A]
    sm = hec.SgsSmoother(Ad)
    HA = hec.hec_from_csr(*Ad)
    bd = dev(b)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    r0 = float(torch.linalg.norm(bd))
    for _ in range(5):
        x = sm.smooth(x, bd, 4)
        r = float(torch.linalg.norm(bd - hec.spmv(HA, x)))
        assert r < r0
        r0 = r
