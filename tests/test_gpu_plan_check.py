"""sptrsv_plan_check: the device-side check of every index the sweeps follow.  Plans the library
builds pass (global, partitioned, RAS); a plan whose arrays are corrupted on purpose (a column out
of range, a dependency on a row of the same level, a zero diagonal, decreasing tail pointers, a
broken permutation) is reported as OUT_OF_BOUNDS naming the check, and passes again once the
value is restored.  No sweep runs on a corrupted plan: only the check reads it."""
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


def factors(kind):
    if kind == "5pt":
        A = synth.poisson2d_5pt(64)
        return A, oracle.ilu0(A)
    if kind == "fv7":
        A = synth.fv7_lognormal(12, seed=1)
        return A, oracle.ilu0(A)
    if kind == "27pt_ilut":
        A = synth.stencil27_jitter(10, seed=2)
        return A, oracle.ilut(A, 10, 1e-3)
    A = synth.random_sparse(700, 0.01, 3)
    return A, oracle.ilut(A, 40, 1e-4)


def plan(hec, T, uplo, vdt="f64", nrhs=1):
    Td = [dev(a) for a in T]
    lv = hec.sptrsv_analyze(Td[0], Td[1], uplo)
    H = hec.hec_from_csr(*Td, levels=lv, vdt=vdt)
    return hec.sptrsv_plan_create(H, lv, nrhs), H, lv


@pytest.mark.parametrize("kind", ["5pt", "fv7", "27pt_ilut", "rand"])
@pytest.mark.parametrize("vdt", ["f64", "f32", "bf16"])
def test_library_plans_pass(hec, kind, vdt):
    A, (L, U) = factors(kind)
    n = len(A[0]) - 1
    for uplo, T in [(0, L), (1, U)]:
        p, _, _ = plan(hec, T, uplo, vdt, nrhs=16)
        hec.sptrsv_plan_check(p)
        part = np.random.default_rng(5).integers(0, 9, size=n).astype(np.int32)
        hec.sptrsv_plan_partition(p, dev(part), 9, 256)
        hec.sptrsv_plan_check(p)
        hec.sptrsv_plan_partition(p, None, 4, 1024)
        hec.sptrsv_plan_check(p)


def test_ras_plans_pass(hec):
    m = 12
    A = synth.fv7_lognormal(m, seed=6)
    part, ns = synth.box_partition(m, [5, 7])
    s = hec.RasSolver([dev(a) for a in A], dev(part), ns, vdt="f32", max_nrhs=16)
    hec.sptrsv_plan_check(s.pL)
    hec.sptrsv_plan_check(s.pU)


def _raw(hec, ptr, n, dtype, owner):
    """A writable view of a library array (zero-copy)."""
    return hec._view(ptr, n, dtype, owner)


def test_corrupted_plans_are_reported(hec):
    A, (L, U) = factors("fv7")
    n = len(A[0]) - 1
    p, H, lv = plan(hec, L, 0)
    inf = H.info()
    ec = _raw(hec, inf.ell_col, inf.w * inf.ld, torch.int32, H)
    tp = _raw(hec, inf.tptr, n + 1, torch.int32, H)
    tv = _raw(hec, inf.tval, int(inf.tail_nnz), torch.float64, H)
    _, _, _, (lev_p, perm_p, iperm_p, lp_p) = lv._get()
    perm = _raw(hec, perm_p, n, torch.int32, lv)
    lptr = _raw(hec, lp_p, lv.nlev + 1, torch.int32, lv).cpu().numpy()
    # the second row of a middle level (levels there hold many rows, each with a first slab slot)
    lmid = lv.nlev // 2
    r = int(lptr[lmid]) + 1
    assert r < int(lptr[lmid + 1]) and int(ec[r]) >= 0

    def expect(name):
        with pytest.raises(hec.HecError) as e:
            hec.sptrsv_plan_check(p)
        assert hec.STATUS_NAMES[e.value.status] == "OUT_OF_BOUNDS" and name in str(e.value), str(e.value)

    cases = [(ec, r, n + 3, "HEC factor"),                # a column out of range
             (ec, r, r - 1, "HEC factor"),                 # a row of the same level
             (tv, int(tp[r + 1]) - 1, 0.0, "HEC factor"),  # a zero diagonal
             (tp, r, int(tp[r + 1]) + 1, "HEC factor"),    # tail pointers out of order
             (perm, 0, n, "level map")]                    # perm out of range
    for arr, i, bad, name in cases:
        old = arr[i].clone()
        arr[i] = bad
        torch.cuda.synchronize()
        expect(name)
        arr[i] = old
        torch.cuda.synchronize()
        hec.sptrsv_plan_check(p)
    # the plan is still the one the library built: a sweep after the checks matches the oracle
    b = synth.uniform_vector(n, 3)
    x = hec.sptrsv_lower(p, dev(b)).cpu().numpy()
    ref = oracle.lower_solve(L, b)
    assert np.max(np.abs(x - ref)) <= 1e-12 * np.max(np.abs(ref))
