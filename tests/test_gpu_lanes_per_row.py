"""Single-right-hand-side sweeps with several lanes per row (the row's slab slots and tail entries
spread over 2, 4 or 8 lanes, partial sums combined by an xor butterfly) against the oracle's
substitution (Alg. 2): FP64 within 1e-12 for short and long rows, long CSR tails, both triangles,
the ILU apply, and the choice the plan makes by row length."""
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


def factors(kind):
    if kind == "fv7":
        return oracle.ilu0(synth.fv7_lognormal(12, seed=3))
    if kind == "27pt_ilut":
        return oracle.ilut(synth.stencil27_jitter(10, seed=1), 10, 1e-3)
    # random sparse ILUT with long, irregular rows
    return oracle.ilut(synth.random_sparse(1200, 0.01, 5), 40, 1e-5)


@pytest.mark.parametrize("kind", ["fv7", "27pt_ilut", "rand"])
@pytest.mark.parametrize("uplo", [0, 1])
@pytest.mark.parametrize("width", [-1, 3])
@pytest.mark.parametrize("lpr", [1, 2, 4, 8])
def test_lanes_per_row_fp64_parity(hec, kind, uplo, width, lpr):
    L, U = factors(kind)
    T = L if uplo == 0 else U
    n = len(T[0]) - 1
    Td = [dev(a) for a in T]
    lv = hec.sptrsv_analyze(Td[0], Td[1], uplo)
    H = hec.hec_from_csr(*Td, levels=lv, ell_width=width, vdt="f64")
    p = hec.sptrsv_plan_create(H, lv, 1, lanes_per_row=lpr)
    b = synth.uniform_vector(n, 21)
    x = (hec.sptrsv_lower if uplo == 0 else hec.sptrsv_upper)(p, dev(b)).cpu().numpy()
    ref = (oracle.lower_solve if uplo == 0 else oracle.upper_solve)(T, b)
    assert relmax(x, ref) <= 1e-12
    assert hec.hec_sync_status(p) == 0


@pytest.mark.parametrize("lpr", [2, 4, 8])
def test_lanes_per_row_ilu_apply_and_fp32(hec, lpr):
    L, U = factors("27pt_ilut")
    n = len(L[0]) - 1
    r = synth.uniform_vector(n, 22)
    ref = oracle.ilu_apply(L, U, r)
    s = hec.IluSolver([dev(a) for a in L], [dev(a) for a in U], vdt="f64", lanes_per_row=lpr)
    assert relmax(s.apply(dev(r)).cpu().numpy(), ref) <= 1e-12
    s32 = hec.IluSolver([dev(a) for a in L], [dev(a) for a in U], vdt="f32", lanes_per_row=lpr)
    s1 = hec.IluSolver([dev(a) for a in L], [dev(a) for a in U], vdt="f32", lanes_per_row=1)
    # FP32 values and sums: the same result up to FP32 rounding of a different summation order
    assert relmax(s32.apply(dev(r)).cpu().numpy(), s1.apply(dev(r)).cpu().numpy()) <= 1e-5


def test_autotuned_lanes_per_row_and_errors(hec):
    """The autotuner searches lanes per row for one right-hand side; whatever it picks, the sweep
    still matches the oracle.  An unsupported lane count is rejected."""
    for kind in ("fv7", "27pt_ilut"):
        L, _ = factors(kind)
        n = len(L[0]) - 1
        Td = [dev(a) for a in L]
        lv = hec.sptrsv_analyze(Td[0], Td[1], 0)
        H = hec.hec_from_csr(*Td, levels=lv, vdt="f64")
        p = hec.sptrsv_plan_create(H, lv, 1)
        chosen = hec.sptrsv_autotune(p, 1)["lanes_per_row"]
        assert chosen in (1, 2, 4, 8), (kind, chosen)
        b = synth.uniform_vector(n, 23)
        assert relmax(hec.sptrsv_lower(p, dev(b)).cpu().numpy(), oracle.lower_solve(L, b)) <= 1e-12
    with pytest.raises(hec.HecError):
        hec.sptrsv_plan_create(H, lv, 1, lanes_per_row=3)
