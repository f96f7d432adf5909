"""Partitioned sweeps (one thread block per part, SM-local dependencies inside a part, point-to-point
waits across parts) against the oracle: FP64 within 1e-12 for contiguous, box and scattered
partitions, the ILU apply and FGMRES on top of them, and the residency and timeout checks."""
import numpy as np
import pytest
import torch

import _bounds
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
    if scheme == "single":
        hec.sptrsv_plan_partition(p, None, 1, threads)
    else:
        _partition(hec, p, scheme, n, box, threads)
    b = synth.uniform_vector(n, 12)
    x = (hec.sptrsv_lower if uplo == 0 else hec.sptrsv_upper)(p, dev(b)).cpu().numpy()
    ref = (oracle.lower_solve if uplo == 0 else oracle.upper_solve)(T, b)
    assert relmax(x, ref) <= 1e-12
    assert hec.hec_sync_status(p) == 0


def _partition(hec, p, scheme, n, box, threads):
    if scheme == "contiguous":
        hec.sptrsv_plan_partition(p, None, 37, threads)
    elif scheme == "box":
        hec.sptrsv_plan_partition(p, dev(box), int(box.max()) + 1, threads)
    else:
        part = np.random.default_rng(7).integers(0, 23, size=n).astype(np.int32)
        hec.sptrsv_plan_partition(p, dev(part), 23, threads)


@pytest.mark.parametrize("kind", ["fv7", "fv7_ilu1", "27pt_ilut"])
@pytest.mark.parametrize("scheme", ["contiguous", "box", "scattered"])
@pytest.mark.parametrize("threads", [256, 1024])
@pytest.mark.parametrize("vdt", ["f32", "bf16"])
def test_partitioned_reduced_precision_against_oracle(hec, kind, scheme, threads, vdt):
    """The partitioned kernel as the solver runs it with FP32 / BF16 values (the next chunk's row
    prefetched while the current one waits, the right-hand side gathered into plan order in FP32
    before the sweep) against the oracle's FP64 substitution with the same rounded values, under
    the componentwise bound gamma_{q+2}(u32) M(T)^-1 |T| |x| (safety factor 4), for the lower and
    the upper factor; the error against the unrounded FP64 solve is printed."""
    A, (L, U), box = factors(kind)
    n = len(A[0]) - 1
    b = synth.uniform_vector(n, 3)
    for uplo, T in [(0, L), (1, U)]:
        p = plans(hec, T, uplo, vdt)
        _partition(hec, p, scheme, n, box, threads)
        f = hec.sptrsv_lower if uplo == 0 else hec.sptrsv_upper
        x = f(p, dev(b)).cpu().numpy()
        assert hec.hec_sync_status(p) == 0
        Tr = _bounds.rounded(T, vdt)
        xr = (oracle.lower_solve if uplo == 0 else oracle.upper_solve)(Tr, b)
        bound = _bounds.sweep_bound(Tr, uplo, xr)
        assert np.all(np.abs(x - xr) <= 4 * bound + 1e-300), float(np.max(np.abs(x - xr) / (bound + 1e-300)))
        x64 = (oracle.lower_solve if uplo == 0 else oracle.upper_solve)(T, b)
        print(kind, scheme, threads, vdt, uplo, "err/bound %.3f, err vs unrounded fp64 %.3e"
              % (float(np.max(np.abs(x - xr) / (bound + 1e-300))), relmax(x, x64)))


@pytest.mark.parametrize("vdt", ["f32", "bf16"])
def test_partitioned_reduced_precision_ilu_apply_against_oracle(hec, vdt):
    """The ILU apply with both factors partitioned on grid boxes at 1024 threads (the solver's
    single-right-hand-side path) against the oracle's z = U^-1 L^-1 r with the rounded values."""
    A, (L, U), box = factors("fv7")
    n = len(A[0]) - 1
    s = hec.IluSolver([dev(a) for a in L], [dev(a) for a in U], vdt=vdt)
    s.partition(dev(box), int(box.max()) + 1, threads=1024)
    r = synth.uniform_vector(n, 17)
    z = s.apply(dev(r)).cpu().numpy()
    Lr, Ur = _bounds.rounded(L, vdt), _bounds.rounded(U, vdt)
    y = oracle.lower_solve(Lr, r)
    zr = oracle.upper_solve(Ur, y)
    bound = _bounds.apply_bound(Lr, Ur, y, zr)
    assert np.all(np.abs(z - zr) <= 4 * bound + 1e-300)


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


@pytest.mark.parametrize("which", ["both", "lower", "upper"])
@pytest.mark.parametrize("vdt", ["f64", "f32"])
def test_partitioned_repeated_applies_against_oracle(hec, which, vdt):
    """A partitioned sweep polls one of two solution buffers and sets the other to the sentinel for
    the next sweep of the same plan; the ILU apply composes its gather with the lower plan's row
    order and writes y in the upper plan's row order when that plan is partitioned.  Several applies
    in a row with different right-hand sides, with only one factor or both partitioned, and a
    standalone lower sweep on the same plan in between, each against the oracle."""
    A, (L, U), box = factors("fv7")
    n = len(A[0]) - 1
    s = hec.IluSolver([dev(a) for a in L], [dev(a) for a in U], vdt=vdt)
    nb = int(box.max()) + 1
    if which in ("both", "lower"):
        hec.sptrsv_plan_partition(s.pL, dev(box), nb, 1024)
    if which in ("both", "upper"):
        hec.sptrsv_plan_partition(s.pU, dev(box), nb, 1024)
    Lr, Ur = (_bounds.rounded(L, vdt), _bounds.rounded(U, vdt)) if vdt != "f64" else (L, U)
    for k in range(5):
        r = synth.uniform_vector(n, 100 + k)
        z = s.apply(dev(r)).cpu().numpy()
        y = oracle.lower_solve(Lr, r)
        zr = oracle.upper_solve(Ur, y)
        if vdt == "f64":
            assert relmax(z, zr) <= 1e-12
        else:
            assert np.all(np.abs(z - zr) <= 4 * _bounds.apply_bound(Lr, Ur, y, zr) + 1e-300)
        if k == 2:
            yl = hec.sptrsv_lower(s.pL, dev(r)).cpu().numpy()
            if vdt == "f64":
                assert relmax(yl, y) <= 1e-12
            else:
                assert np.all(np.abs(yl - y) <= 4 * _bounds.sweep_bound(Lr, 0, y) + 1e-300)
    assert hec.hec_sync_status(s.pL) == 0 and hec.hec_sync_status(s.pU) == 0
