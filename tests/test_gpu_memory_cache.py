"""The library's cache of released device blocks (hec_release_cached_memory): handles built and
destroyed again reuse the cached blocks (no growth of device memory in use), results do not
change, and the release call hands the blocks back to the CUDA runtime."""
import gc

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


def test_rebuilt_solvers_reuse_cached_blocks(hec):
    A = synth.fv7_lognormal(24, seed=3)
    L, U = oracle.ilu0(A)
    n = len(A[0]) - 1
    b = synth.uniform_vector(n, 5)
    ref = oracle.ilu_apply(L, U, b)
    Ld, Ud, Ad = [dev(a) for a in L], [dev(a) for a in U], [dev(a) for a in A]
    bd = dev(b)
    free_after = []
    for k in range(6):
        s = hec.IluSolver(Ld, Ud, A=Ad, vdt="f64")
        z = s.apply(bd).cpu().numpy()
        assert float(np.max(np.abs(z - ref)) / np.max(np.abs(ref))) <= 1e-12
        del s
        gc.collect()
        torch.cuda.synchronize()
        free_after.append(torch.cuda.mem_get_info()[0])
    # from the second build on, every block comes from the cache: free memory stays put
    assert max(free_after[1:]) - min(free_after[1:]) <= 4 << 20
    released = hec.release_cached_memory()
    assert released > 0
    assert torch.cuda.mem_get_info()[0] >= free_after[-1] + released - (4 << 20)
    assert hec.release_cached_memory() == 0
