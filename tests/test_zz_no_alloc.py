"""The allocation-free sweep entry point, called through the C ABI.

sptrsv_solve_noalloc serves callers that may not allocate device memory while they solve (their
memory belongs to another allocator, is reserved up front, or a cudaMalloc would stall a
latency-critical loop).  It must give the same answer as the allocating entry points
sptrsv_lower / sptrsv_upper and as the oracle's forward / back substitution, call after call,
although every call reuses one static buffer, and after its first call on a device it must leave
the free device memory unchanged.  This file is collected last so that a failure here comes after
every other test has run."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1606_00541_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-12  # the FP64 sweep parity tolerance of the other sweep tests


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


def _factors(kind, seed):
    if kind == "fv7":
        A = synth.fv7_lognormal(14, seed=seed)
        return A, oracle.ilu0(A)
    if kind == "fv7_small":
        A = synth.fv7_lognormal(6, seed=seed)
        return A, oracle.ilu0(A)
    # 27-point ILUT: slab width 10 and long tails, so one right-hand side takes the multi-lane
    # kernel and sixteen take the 8-slot slab batches plus the tail rounds
    A = synth.stencil27_jitter(10, seed=seed)
    return A, oracle.ilut(A, 10, 1e-3)


def _setup(hec, kind, uplo, vdt, seed):
    A, (L, U) = _factors(kind, seed)
    T = L if uplo == 0 else U
    Td = [torch.as_tensor(a, device="cuda") for a in T]
    lv = hec.sptrsv_analyze(Td[0], Td[1], uplo)
    H = hec.hec_from_csr(*Td, levels=lv, vdt=vdt)
    return len(A[0]) - 1, T, lv, H


def _relmax(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _oracle_solve(T, uplo, B):
    f = oracle.lower_solve if uplo == 0 else oracle.upper_solve
    B2 = B.reshape(B.shape[0], -1)
    return np.stack([f(T, B2[:, q]) for q in range(B2.shape[1])], axis=1).reshape(B.shape)


@pytest.mark.parametrize("uplo", [0, 1])
@pytest.mark.parametrize("vdt,nrhs", [("f64", 1), ("f32", 4), ("bf16", 16)])
def test_noalloc_matches_allocating_entry_point_twice(hec, uplo, vdt, nrhs):
    n, T, lv, H = _setup(hec, "fv7", uplo, vdt, seed=uplo)
    plan = hec.sptrsv_plan_create(H, lv, max_nrhs=nrhs)
    solve = hec.sptrsv_lower if uplo == 0 else hec.sptrsv_upper
    for call in range(2):  # two calls in a row share the static buffer
        Bh = synth.uniform_vector(n, 100 + call, nrhs=nrhs)
        B = torch.as_tensor(Bh, device="cuda")
        ref = solve(plan, B)
        X = torch.full_like(B, float("nan"))
        st, st_dev = _noalloc(hec, H, lv, B, X)
        assert st == 0 and st_dev == 0, hec._lib.hec_last_error()
        torch.cuda.synchronize()
        # the same kernel with the same lane layout as a default plan: equal bit for bit
        assert torch.equal(X, ref), call
        if vdt == "f64":
            assert _relmax(X.cpu().numpy(), _oracle_solve(T, uplo, Bh)) <= TOL


@pytest.mark.parametrize("uplo", [0, 1])
@pytest.mark.parametrize("nrhs", [1, 16])
def test_noalloc_long_rows_against_oracle(hec, uplo, nrhs):
    """Wide-slab, tail-heavy ILUT factors (FP64) against the oracle's substitution, twice."""
    n, T, lv, H = _setup(hec, "ilut27", uplo, "f64", seed=2)
    assert H.info().w > 8 or H.info().tail_nnz > 2 * n
    for call in range(2):
        Bh = synth.uniform_vector(n, 300 + call, nrhs=nrhs)
        B = torch.as_tensor(Bh, device="cuda")
        X = torch.full_like(B, float("nan"))
        st, st_dev = _noalloc(hec, H, lv, B, X)
        assert st == 0 and st_dev == 0, hec._lib.hec_last_error()
        assert _relmax(X.cpu().numpy(), _oracle_solve(T, uplo, Bh)) <= TOL, call


def test_noalloc_sizes_back_to_back(hec):
    """A larger problem, then a smaller one, then the larger again: nothing the larger call left in
    the buffer (chunk table entries, published solution words) may leak into the next."""
    big = _setup(hec, "fv7", 0, "f64", seed=5)
    small = _setup(hec, "fv7_small", 1, "f64", seed=6)
    wide = _setup(hec, "ilut27", 0, "f64", seed=7)
    for k, (n, T, lv, H) in enumerate([big, small, wide, small, big]):
        for nrhs in (1, 3):
            Bh = synth.uniform_vector(n, 400 + 10 * k + nrhs, nrhs=nrhs)
            B = torch.as_tensor(Bh, device="cuda")
            X = torch.full_like(B, float("nan"))
            st, st_dev = _noalloc(hec, H, lv, B, X)
            assert st == 0 and st_dev == 0, hec._lib.hec_last_error()
            uplo = lv.uplo
            assert _relmax(X.cpu().numpy(), _oracle_solve(T, uplo, Bh)) <= TOL, (k, nrhs)


def test_noalloc_leaves_free_memory_unchanged(hec):
    """After the first call on the device (which may load the buffer's module), further calls
    allocate nothing: the device's free memory is the same before and after them."""
    n, T, lv, H = _setup(hec, "fv7", 0, "f32", seed=8)
    bufs = [(torch.as_tensor(synth.uniform_vector(n, 500 + i), device="cuda"),
             torch.empty(n, dtype=torch.float64, device="cuda")) for i in range(3)]
    st, _ = _noalloc(hec, H, lv, *bufs[0])  # warm-up: loads the module holding the buffer
    assert st == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for B, X in bufs[1:]:
        st, st_dev = _noalloc(hec, H, lv, B, X)
        assert st == 0 and st_dev == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)


def test_noalloc_rejects_sizes_beyond_the_static_buffer(hec):
    lib = hec._lib
    lib.sptrsv_noalloc_capacity.restype = ctypes.c_size_t
    cap = lib.sptrsv_noalloc_capacity()
    assert cap == 32 << 20
    n = 490_000  # x 16 right-hand sides x 8 bytes = 62.7 MB > 32 MiB
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
