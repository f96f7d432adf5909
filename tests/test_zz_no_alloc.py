"""The allocation-free sweep entry point, called through the C ABI.

sptrsv_solve_noalloc serves callers that may not allocate device memory while they solve (their
memory belongs to another allocator, is reserved up front, or a cudaMalloc would stall a
latency-critical loop).  It must give the same answer as the allocating entry points
sptrsv_lower / sptrsv_upper, call after call, although every call reuses one static buffer.
This file is collected last so that a failure here comes after every other test has run."""
import ctypes

import numpy as np
import pytest
import torch

from paper_1606_00541_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hec():
    from paper_1606_00541_gb300 import hec as h
    return h


def _noalloc(hec, plan_matrix, levels, b, x):
    lib = hec._lib
    f = lib.sptrsv_solve_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                  ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_void_p]
    nrhs = 1 if b.dim() == 1 else b.shape[1]
    st_dev = ctypes.c_int(-1)
    st = f(plan_matrix.h, levels.h, nrhs, b.data_ptr(), nrhs, x.data_ptr(), nrhs, ctypes.byref(st_dev),
           torch.cuda.current_stream().cuda_stream)
    return st, st_dev.value


def _setup(hec, uplo, vdt, seed):
    from oracle import ilu0  # test-side input preparation only
    A = synth.fv7_lognormal(14, seed=seed)
    L, U = ilu0(A)
    T = L if uplo == 0 else U
    Td = [torch.as_tensor(a, device="cuda") for a in T]
    lv = hec.sptrsv_analyze(Td[0], Td[1], uplo)
    H = hec.hec_from_csr(*Td, levels=lv, vdt=vdt)
    return len(A[0]) - 1, lv, H


@pytest.mark.parametrize("uplo", [0, 1])
@pytest.mark.parametrize("vdt,nrhs", [("f64", 1), ("f32", 4), ("bf16", 16)])
def test_noalloc_matches_allocating_entry_point_twice(hec, uplo, vdt, nrhs):
    n, lv, H = _setup(hec, uplo, vdt, seed=uplo)
    plan = hec.sptrsv_plan_create(H, lv, max_nrhs=nrhs)
    solve = hec.sptrsv_lower if uplo == 0 else hec.sptrsv_upper
    tol = 1e-12  # the sweep parity tolerance; both entry points run the same kernel
    for call in range(2):  # two calls in a row share the static buffer
        B = torch.as_tensor(synth.uniform_vector(n, 100 + call, nrhs=nrhs), device="cuda")
        ref = solve(plan, B)
        X = torch.full_like(B, float("nan"))
        st, st_dev = _noalloc(hec, H, lv, B, X)
        assert st == 0 and st_dev == 0, hec._lib.hec_last_error()
        torch.cuda.synchronize()
        err = (X - ref).abs().max().item() / ref.abs().max().item()
        assert err <= tol, (call, err)


def test_noalloc_rejects_sizes_beyond_the_static_buffer(hec):
    lib = hec._lib
    lib.sptrsv_noalloc_capacity.restype = ctypes.c_size_t
    cap = lib.sptrsv_noalloc_capacity()
    assert cap == 32 << 20
    m = 700  # 490,000 rows x 16 right-hand sides x 8 bytes = 62.7 MB > 32 MiB
    A = synth.poisson2d_5pt(m)
    n = m * m
    # a diagonal factor is enough to exercise the size check
    T = (np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), np.full(n, 2.0))
    Td = [torch.as_tensor(a, device="cuda") for a in T]
    lv = hec.sptrsv_analyze(Td[0], Td[1], 0)
    H = hec.hec_from_csr(*Td, levels=lv, vdt="f64")
    B = torch.ones(n, 16, dtype=torch.float64, device="cuda")
    X = torch.zeros_like(B)
    st, _ = _noalloc(hec, H, lv, B, X)
    assert hec.STATUS_NAMES[st] == "INVALID_ARG"
    assert b"static buffer" in lib.hec_last_error()
    del A
