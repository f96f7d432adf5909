"""Partitioned sweeps (one thread block per part, SM-local dependencies inside a part, point-to-point
waits across parts) against the oracle: FP64 within 1e-12 for contiguous, box and scattered
partitions, the ILU apply and FGMRES on top of them, and the residency and timeout checks."""
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
    if kind == "5pt":
        A = synth.poisson2d_5pt(64)
        return A, oracle.ilu0(A), None
    if kind == "fv7":
        A = synth.fv7_lognormal(16, seed=1)
        part, _ = synth.box_partition(16, [5, 6, 5])
        return A, oracle.ilu0(A), part
    if kind == "fv7_ilu1":
        A = synth.fv7_lognormal(12, seed=2)
        part, _ = synth.box_partition(12, [6, 6])
        return A, oracle.iluk(A, 1), part
    if kind == "27pt_ilut":
        A = synth.stencil27_jitter(10, seed=2)
        part, _ = synth.box_partition(10, [3, 3, 4])
        return A, oracle.ilut(A, 10, 1e-3), part
    A = synth.random_sparse(900, 0.008, 4)
    return A, oracle.ilut(A, 30, 1e-4), None


def plans(hec, T, uplo, vdt="f64"):
    Td = [dev(a) for a in T]
    lv = hec.sptrsv_analyze(Td[0], Td[1], uplo)
    H = hec.hec_from_csr(*Td, levels=lv, vdt=vdt)
    return hec.sptrsv_plan_create(H, lv, 1)


@pytest.mark.parametrize("kind", ["5pt", "fv7", "fv7_ilu1", "27pt_ilut", "rand"])
@pytest.mark.parametrize("scheme", ["contiguous", "box", "scattered", "single"])
@pytest.mark.parametrize("uplo", [0, 1])
@pytest.mark.parametrize("threads", [256, 1024])
def test_partitioned_sweep_fp64_parity(hec, kind, scheme, uplo, threads):
    A, (L, U), box = factors(kind)
    n = len(A[0]) - 1
    T = L if uplo == 0 else U
    p = plans(hec, T, uplo)
    if scheme == "box" and box is None:
        pytest.skip("no grid partition for this matrix")
    if scheme == "contiguous":
        hec.sptrsv_plan_partition(p, None, 37, threads)
    elif scheme == "box":
        hec.sptrsv_plan_partition(p, dev(box), int(box.max()) + 1, threads)
    elif scheme == "scattered":
        part = np.random.default_rng(7).integers(0, 23, size=n).astype(np.int32)
        hec.sptrsv_plan_partition(p, dev(part), 23, threads)
    else:
        hec.sptrsv_plan_partition(p, None, 1, threads)
    b = synth.uniform_vector(n, 12)
    x = (hec.sptrsv_lower if uplo == 0 else hec.sptrsv_upper)(p, dev(b)).cpu().numpy()
    ref = (oracle.lower_solve if uplo == 0 else oracle.upper_solve)(T, b)
    assert relmax(x, ref) <= 1e-12
    assert hec.hec_sync_status(p) == 0


@pytest.mark.parametrize("vdt", ["f32", "bf16"])
def test_partitioned_reduced_precision_close(hec, vdt):
    A, (L, U), box = factors("fv7")
    n = len(A[0]) - 1
    b = synth.uniform_vector(n, 3)
    for uplo, T in [(0, L), (1, U)]:
        p0 = plans(hec, T, uplo, vdt)
        p1 = plans(hec, T, uplo, vdt)
        hec.sptrsv_plan_partition(p1, dev(box), int(box.max()) + 1)
        f = hec.sptrsv_lower if uplo == 0 else hec.sptrsv_upper
        x0 = f(p0, dev(b)).cpu().numpy()
        x1 = f(p1, dev(b)).cpu().numpy()
        # same rounded values, FP32 sums in another order
        assert relmax(x1, x0) <= 1e-5


def test_partitioned_ilu_fgmres(hec):
    m = 24
    A = synth.fv7_lognormal(m, seed=9)
    n = m ** 3
    L, U = oracle.ilu0(A)
    part, nb = synth.box_partition(m, [6, 6, 6, 6])
    s = hec.IluSolver([dev(a) for a in L], [dev(a) for a in U], A=[dev(a) for a in A], vdt="f64")
    r = synth.uniform_vector(n, 2)
    z0 = s.apply(dev(r)).cpu().numpy()
    s.partition(dev(part), nb)
    z1 = s.apply(dev(r)).cpu().numpy()
    assert relmax(z1, oracle.ilu_apply(L, U, r)) <= 1e-12 and relmax(z1, z0) <= 1e-12
    b = oracle.spmv(A, synth.uniform_vector(n, 4))
    x, info = s.solve(dev(b), rtol=1e-8)
    assert info["converged"]
    assert np.linalg.norm(b - oracle.spmv(A, x.cpu().numpy())) <= 1e-8 * np.linalg.norm(b) * (1 + 1e-6)
    # default: as many contiguous parts as fit
    assert s.partition() >= 1
    z2 = s.apply(dev(r)).cpu().numpy()
    assert relmax(z2, z0) <= 1e-12


def test_partition_residency_limit(hec):
    A, (L, U), _ = factors("5pt")
    p = plans(hec, L, 0)
    cap = hec.sptrsv_partition_capacity(p)
    assert cap >= 1
    with pytest.raises(hec.HecError):
        hec.sptrsv_plan_partition(p, None, cap + 1)
    with pytest.raises(hec.HecError):
        hec.sptrsv_plan_partition(p, dev(np.full(len(L[0]) - 1, 5, np.int32)), 3)  # part id out of range


def test_partitioned_timeout_reports_status(hec):
    A, (L, U), _ = factors("5pt")
    Td = [dev(a) for a in L]
    lv = hec.sptrsv_analyze(Td[0], Td[1], 0)
    H = hec.hec_from_csr(*Td, levels=lv)
    p = hec.sptrsv_plan_create(H, lv, 1, wait_cycles=2_000_000, debug_unpublished_row=500)
    # one grid row per part: the unpublished row's dependents lie in other parts and must wait
    hec.sptrsv_plan_partition(p, None, 64)
    b = dev(synth.uniform_vector(4096, 1))
    hec.sptrsv_lower(p, b)
    assert hec.STATUS_NAMES[hec.hec_sync_status(p)] == "TIMEOUT"


@pytest.mark.parametrize("ras", [False, True])
def test_partitioned_apply_matches_unpartitioned(hec, ras):
    """ILU / RAS apply with both plans partitioned (contiguous parts of the extended numbering for
    RAS, grid boxes for ILU): the same result as the unpartitioned apply, also after the plans are
    partitioned again."""
    m = 12
    A = synth.fv7_lognormal(m, seed=6)
    Ad = [dev(a) for a in A]
    n = m ** 3
    if ras:
        part, ns = synth.box_partition(m, [5, 7])
        s = hec.RasSolver(Ad, dev(part), ns, vdt="f64")
    else:
        L, U = oracle.ilu0(A)
        s = hec.IluSolver([dev(a) for a in L], [dev(a) for a in U], A=Ad, vdt="f64")
    r = dev(synth.uniform_vector(n, 41))
    ref = s.apply(r).cpu().numpy()
    nn = s.lvL.n
    for nb in [(1, 3, 3), (2, 2, 2)]:
        if ras:
            s.partition(None, 7)  # contiguous parts of the extended numbering
        else:
            bx, _ = synth.grid_boxes(m, nb)
            s.partition(dev(bx), nb[0] * nb[1] * nb[2])
        got = s.apply(r).cpu().numpy()
        assert relmax(got, ref) <= 1e-12
        assert s.lvL.n == nn
