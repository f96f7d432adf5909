"""GPU ILUT(p, tol) against the oracle's (Sec. 3; Saad's dual threshold): the same operations in
the same order without fused multiply-adds, so pattern and values must be identical, including
the tie-breaking of equal magnitudes (Poisson matrices); exact LU for tol = 0, p = n; the error
paths; and FGMRES with the GPU factors."""
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


def host(csr):
    return [t.cpu().numpy() for t in csr.tensors()]


CASES = [
    ("27pt_jitter_10", lambda: synth.stencil27_jitter(10, seed=1), 10, 1e-3),
    ("fv7_lognormal_12", lambda: synth.fv7_lognormal(12, seed=4), 5, 1e-2),
    ("poisson2d_32_ties", lambda: synth.poisson2d_5pt(32), 3, 0.05),
    ("poisson3d_8_ties", lambda: synth.poisson3d_7pt(8), 4, 1e-2),
    ("random_600", lambda: synth.random_sparse(600, 0.01, 7), 20, 1e-4),
    ("p0_diagonal_only", lambda: synth.fv7_lognormal(6, seed=5), 0, 1e-3),
    ("exact_lu_poisson2d_8", lambda: synth.poisson2d_5pt(8), 64, 0.0),
    ("hand_worked_4x4", lambda: (np.array([0, 3, 6, 9, 12], np.int32),
                                 np.array([0, 1, 2, 0, 1, 3, 0, 1, 2, 1, 2, 3], np.int32),
                                 np.array([4.0, 1.0, 1.0, 2.0, 5.0, 1.0, 0.3, 3.0, 6.0, 1.0, 0.01, 8.0])), 1, 0.01),
]


@pytest.mark.parametrize("name,make,p,tol", CASES, ids=[c[0] for c in CASES])
def test_ilut_matches_oracle_bitwise(hec, name, make, p, tol):
    A = make()
    Lo, Uo = oracle.ilut(A, p, tol)
    Lh, Uh = hec.ilut_factor(*[dev(a) for a in A], p=p, tol=tol)
    L, U = host(Lh), host(Uh)
    for got, ref in ((L, Lo), (U, Uo)):
        assert np.array_equal(got[0], ref[0])
        assert np.array_equal(got[1], ref[1])
        assert np.array_equal(got[2], ref[2])


def test_ilut_exact_lu_reproduces_a(hec):
    A = synth.poisson2d_5pt(8)
    n = len(A[0]) - 1
    Lh, Uh = hec.ilut_factor(*[dev(a) for a in A], p=n, tol=0.0)
    L, U = host(Lh), host(Uh)

    def dense(M):
        D = np.zeros((n, n))
        for i in range(n):
            D[i, M[1][M[0][i]:M[0][i + 1]]] = M[2][M[0][i]:M[0][i + 1]]
        return D
    assert np.max(np.abs(dense(L) @ dense(U) - dense(A))) <= 1e-12


def test_ilut_errors(hec):
    # a zero pivot
    A = (np.array([0, 2, 4], np.int32), np.array([0, 1, 0, 1], np.int32), np.array([0.0, 1.0, 1.0, 1.0]))
    with pytest.raises(hec.HecError):
        hec.ilut_factor(*[dev(a) for a in A], p=2, tol=0.0)
    # a row longer than the largest working list (9000 entries): diagonal rows, then one full row
    n = 9001
    rp = np.concatenate([np.arange(n, dtype=np.int32), [2 * n - 1]]).astype(np.int32)
    ci = np.concatenate([np.arange(n - 1), np.arange(n)]).astype(np.int32)
    v = np.concatenate([np.full(n - 1, 2.0), np.full(n, -1.0)])
    v[-1] = 2.0 * n
    with pytest.raises(hec.HecError):
        hec.ilut_factor(dev(rp), dev(ci), dev(v), p=n, tol=0.0)
    # a dense 300 x 300 matrix fits a larger working list and gives exact LU
    m = 300
    rp = np.arange(0, m * m + 1, m, dtype=np.int32)
    ci = np.tile(np.arange(m, dtype=np.int32), m)
    v = np.full(m * m, -1.0)
    v[np.arange(m) * m + np.arange(m)] = 2.0 * m
    Lo, Uo = oracle.ilut((rp, ci, v), m, 0.0)
    Lh, Uh = hec.ilut_factor(dev(rp), dev(ci), dev(v), p=m, tol=0.0)
    for got, ref in ((host(Lh), Lo), (host(Uh), Uo)):
        assert all(np.array_equal(g, r) for g, r in zip(got, ref))


def test_ilut_preconditioned_fgmres(hec):
    A = synth.stencil27_jitter(16, seed=3)
    Ad = [dev(a) for a in A]
    Lh, Uh = hec.ilut_factor(*Ad, p=10, tol=1e-3)
    s = hec.IluSolver(Lh.tensors(), Uh.tensors(), A=Ad, vdt="f32")
    b = synth.uniform_vector(16 ** 3, 31)
    x, info = s.solve(dev(b), rtol=1e-8)
    r = b - oracle.spmv(A, x.cpu().numpy())
    assert info["converged"] and np.linalg.norm(r) <= 1e-8 * np.linalg.norm(b) * 1.0001


def test_ilut_structural_diagonal_unsorted_and_empty(hec):
    # row 1 stores no diagonal: the structural zero slot receives fill (0 - 0.5 * 1) and the
    # factors equal the oracle's
    A = (np.array([0, 2, 3], np.int32), np.array([0, 1, 0], np.int32), np.array([2.0, 1.0, 1.0]))
    Lo, Uo = oracle.ilut(A, 2, 0.0)
    Lh, Uh = hec.ilut_factor(*[dev(a) for a in A], p=2, tol=0.0)
    for got, ref in ((host(Lh), Lo), (host(Uh), Uo)):
        assert all(np.array_equal(g, r) for g, r in zip(got, ref))
    assert host(Uh)[2][-1] == -0.5
    # a row with descending columns is rejected
    B = (np.array([0, 2, 4], np.int32), np.array([1, 0, 0, 1], np.int32), np.array([1.0, 2.0, 1.0, 2.0]))
    with pytest.raises(hec.HecError):
        hec.ilut_factor(*[dev(a) for a in B], p=2, tol=0.0)
    # the empty matrix
    E = (np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0))
    Lh, Uh = hec.ilut_factor(*[dev(a) for a in E], p=4, tol=1e-3)
    assert all(len(t) == 0 for t in host(Lh)[1:]) and list(host(Uh)[0]) == [0]
