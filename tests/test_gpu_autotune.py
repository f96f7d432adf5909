"""The sweep autotuner (sptrsv_autotune): residency, lanes per row and, for a partitioned plan, the
partitioned against the global schedule.  Whatever it chooses, sweeps and the ILU apply must still
match the oracle; choices are cached per matrix signature."""
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


def test_autotune_chooses_between_partitioned_and_global(hec):
    m = 24
    A = synth.fv7_lognormal(m, seed=3)
    L, U = oracle.ilu0(A)
    n = m ** 3
    part, nparts = synth.grid_boxes(m, (1, 4, 4))
    s = hec.IluSolver([dev(a) for a in L], [dev(a) for a in U], vdt="f64")
    s.partition(dev(part), nparts, threads=512)
    choices = s.autotune(1)
    for c in choices:
        assert c["block_threads"] in (128, 256) and c["blocks_per_sm"] in (2, 4, 8, 16)
        assert c["lanes_per_row"] in (1, 2, 4, 8) and isinstance(c["partitioned"], bool)
    r = synth.uniform_vector(n, 31)
    assert relmax(s.apply(dev(r)).cpu().numpy(), oracle.ilu_apply(L, U, r)) <= 1e-12
    # the same signature again: the cached choice, without a partition the flag is off
    s2 = hec.IluSolver([dev(a) for a in L], [dev(a) for a in U], vdt="f64")
    c2 = s2.autotune(1)
    assert not any(c["partitioned"] for c in c2)
    s3 = hec.IluSolver([dev(a) for a in L], [dev(a) for a in U], vdt="f64")
    s3.partition(dev(part), nparts, threads=512)
    assert s3.autotune(1) == choices
    assert relmax(s3.apply(dev(r)).cpu().numpy(), oracle.ilu_apply(L, U, r)) <= 1e-12


def test_autotune_global_choice_keeps_partition_for_later(hec):
    """When the tuner keeps the global schedule, the partition stays with the plan unused;
    partitioning the plan again makes single-right-hand-side sweeps take it."""
    A = synth.poisson2d_5pt(64)
    L, U = oracle.ilu0(A)
    Td = [dev(a) for a in L]
    lv = hec.sptrsv_analyze(Td[0], Td[1], 0)
    H = hec.hec_from_csr(*Td, levels=lv, vdt="f64")
    p = hec.sptrsv_plan_create(H, lv, 1)
    hec.sptrsv_plan_partition(p, None, 8, 256)
    c = hec.sptrsv_autotune(p, 1)
    b = synth.uniform_vector(4096, 4)
    assert relmax(hec.sptrsv_lower(p, dev(b)).cpu().numpy(), oracle.lower_solve(L, b)) <= 1e-12
    hec.sptrsv_plan_partition(p, None, 8, 256)
    assert relmax(hec.sptrsv_lower(p, dev(b)).cpu().numpy(), oracle.lower_solve(L, b)) <= 1e-12
    assert isinstance(c["partitioned"], bool)


@pytest.mark.parametrize("vdt", ["f64", "f32"])
def test_autotune_multi_rhs_parity(hec, vdt):
    A = synth.stencil27_jitter(10, seed=2)
    L, U = oracle.ilut(A, 10, 1e-3)
    n = len(A[0]) - 1
    s = hec.IluSolver([dev(a) for a in L], [dev(a) for a in U], vdt=vdt, max_nrhs=16)
    for k in (1, 16):
        s.autotune(k)
        R = synth.uniform_vector(n, 50, nrhs=k)
        Z = s.apply(dev(R)).cpu().numpy().reshape(n, -1)
        R2 = R.reshape(n, -1)
        for q in (0, k - 1):
            ref = oracle.ilu_apply(L, U, R2[:, q])
            assert relmax(Z[:, q], ref) <= (1e-12 if vdt == "f64" else 1e-4)
