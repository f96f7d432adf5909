"""Kernel timing by category: hec_profile_enable records every category, hec_profile_enable_categories
only the ones in its mask; the recorded launch counts follow the solve's structure."""
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


def solve_once(hec):
    A = synth.fv7_lognormal(12, seed=3)
    L, U = oracle.ilu0(A)
    s = hec.IluSolver([dev(a) for a in L], [dev(a) for a in U], A=[dev(a) for a in A], vdt="f32")
    b = oracle.spmv(A, synth.uniform_vector(12 ** 3, 5))
    x, info = s.solve(dev(b), rtol=1e-8)
    torch.cuda.synchronize()
    assert info["converged"]
    return info["iterations"]


def test_profile_all_and_sweeps_only(hec):
    hec.profile_read(reset=True)
    hec.profile_enable(True)
    its = solve_once(hec)
    every = hec.profile_breakdown()
    ms, sweeps = hec.profile_read(reset=True)
    # two sweeps an iteration (L and U), plus SpMV and Gram-Schmidt launches
    assert sweeps >= 2 * its and ms > 0.0
    assert every["spmv"][1] > 0 and every["gram_schmidt"][1] > 0

    hec.profile_enable(True, categories=[0])
    its = solve_once(hec)
    only = hec.profile_breakdown()
    ms, sweeps = hec.profile_read(reset=True)
    assert sweeps >= 2 * its and ms > 0.0
    assert all(n == 0 for name, (_, n) in only.items() if name != "sweep")

    hec.profile_enable(False)
    solve_once(hec)
    assert hec.profile_read(reset=True) == (0.0, 0)
