"""Parity of the CUDA path (called through the C ABI) with the CPU oracle, on the same seeded inputs.

Bars: level sets, maps and HEC arrays bit-exact; FP64 sweeps within 1e-12 relative max-norm; FP32 and
BF16 sweeps within an a-priori bound derived from the value rounding (see test docstrings); SpMV within
1e-14; FGMRES to a 1e-8 true relative residual."""
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


def dev(A):
    return tuple(torch.as_tensor(np.ascontiguousarray(a), device="cuda") for a in A)


def relmax(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


# --- inputs -------------------------------------------------------------------------------------

def _factors(kind):
    if kind == "5pt64":
        A = synth.poisson2d_5pt(64)
        return A, oracle.ilu0(A)
    if kind == "fv7_12":
        A = synth.fv7_lognormal(12, seed=1)
        return A, oracle.ilu0(A)
    if kind == "fv7_12_ilu1":
        A = synth.fv7_lognormal(12, seed=1)
        return A, oracle.iluk(A, 1)
    if kind == "27pt_ilut":
        A = synth.stencil27_jitter(10, seed=2)
        return A, oracle.ilut(A, 10, 1e-3)
    if kind == "rand":
        A = synth.random_sparse(700, 0.01, 3)
        return A, oracle.ilut(A, 40, 1e-4)
    raise KeyError(kind)


KINDS = ["5pt64", "fv7_12", "fv7_12_ilu1", "27pt_ilut", "rand"]


# --- level analysis (Eq. 2, Eq. 3) --------------------------------------------------------------

@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("uplo", [0, 1])
def test_levels_and_map_bit_exact(hec, kind, uplo):
    A, (L, U) = _factors(kind)
    T = L if uplo == 0 else U
    lv = hec.sptrsv_analyze(*dev(T[:2]), uplo)
    lev, perm, iperm, lp = [a.cpu().numpy() for a in lv.arrays()]
    ref = oracle.analyze(T, uplo)
    assert lv.nlev == ref["nlev"]
    assert np.array_equal(lev, ref["level"])
    assert np.array_equal(perm, ref["perm"])
    assert np.array_equal(iperm, ref["iperm"])
    assert np.array_equal(lp, ref["level_ptr"])


@pytest.mark.parametrize("n,density,seed", [(1, 0.0, 0), (33, 0.0, 1), (257, 1.0, 2), (5000, 0.0005, 3),
                                            (20000, 0.0002, 4)])
@pytest.mark.parametrize("uplo", [0, 1])
def test_levels_edge_cases(hec, n, density, seed, uplo):
    """n = 1, a diagonal matrix (one level), a dense triangle (n levels, a chain), sparse random
    factors spanning many 32-row chunks with a ragged tail."""
    T = synth.random_lower(n, density, seed, uplo=uplo)
    lv = hec.sptrsv_analyze(*dev(T[:2]), uplo)
    lev, perm, iperm, lp = [a.cpu().numpy() for a in lv.arrays()]
    ref = oracle.analyze(T, uplo)
    assert lv.nlev == ref["nlev"]
    assert np.array_equal(lev, ref["level"]) and np.array_equal(perm, ref["perm"])
    assert np.array_equal(lp, ref["level_ptr"])


def test_analyze_empty(hec):
    rp = torch.zeros(1, dtype=torch.int32, device="cuda")
    ci = torch.zeros(1, dtype=torch.int32, device="cuda")
    lv = hec.sptrsv_analyze(rp, ci[:0], 0)
    assert lv.n == 0 and lv.nlev == 0


@pytest.mark.parametrize("case,status", [("unsorted", "UNSORTED"), ("upper_in_lower", "NOT_TRIANGULAR"),
                                         ("nodiag", "MISSING_DIAG"), ("oob", "UNSORTED")])
def test_analyze_rejects_malformed(hec, case, status):
    rp = np.array([0, 1, 3, 5], np.int32)
    ci = {"unsorted": [0, 1, 0, 0, 2], "upper_in_lower": [0, 0, 2, 0, 2], "nodiag": [0, 0, 1, 0, 1],
          "oob": [0, 0, 7, 0, 2]}[case]
    with pytest.raises(hec.HecError) as e:
        hec.sptrsv_analyze(*dev((rp, np.array(ci, np.int32))), 0)
    assert hec.STATUS_NAMES[e.value.status] == status


# --- HEC packing (Sec. 2.1, Alg. 1) ---------------------------------------------------------------

@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("uplo", [0, 1])
@pytest.mark.parametrize("vdt", ["f64", "f32", "bf16"])
def test_hec_pack_bit_exact(hec, kind, uplo, vdt):
    A, (L, U) = _factors(kind)
    T = L if uplo == 0 else U
    for w in ([-1, 0, 2, 7] if vdt == "f64" else [-1]):
        Td = dev(T)
        lv = hec.sptrsv_analyze(Td[0], Td[1], uplo)
        H = hec.hec_from_csr(*Td, levels=lv, ell_width=w, vdt=vdt).arrays()
        ref = oracle.analyze(T, uplo)
        R = oracle.hec_pack(T, 1, uplo, ref["perm"], ref["iperm"], w=w, vdt=vdt)
        assert H["w"] == R["w"] and H["ld"] == R["ld"]
        for key in ["ell_col", "tptr", "tcol"]:
            assert np.array_equal(H[key].cpu().numpy(), R[key]), key
        for key in ["ell_val", "tval"]:
            got = H[key].cpu().numpy()
            exp = R[key]
            if vdt == "f32":
                got = got.view(np.uint32)
            elif vdt == "bf16":
                got = got.view(np.uint16)
            assert np.array_equal(got, exp), key
        # round trip back to the original CSR
        rp, ci, v = [a.cpu().numpy() for a in hec.hec_to_csr(hec.hec_from_csr(*Td, levels=lv, ell_width=w, vdt=vdt), lv)]
        assert np.array_equal(rp, T[0]) and np.array_equal(ci, T[1])


def test_hec_general_mode_bit_exact(hec):
    A = synth.stencil27_jitter(9, seed=5)
    H = hec.hec_from_csr(*dev(A)).arrays()
    R = oracle.hec_pack(A, 0)
    for key in ["ell_col", "ell_val", "tptr", "tcol", "tval"]:
        assert np.array_equal(H[key].cpu().numpy(), R[key]), key


def test_bf16_rounding_ties_bit_exact(hec):
    """Values at and next to BF16 rounding ties, where rounding FP64 -> FP32 -> BF16 would differ from
    the direct rounding: packed as the diagonal of a diagonal factor."""
    one = 1.0
    vals = np.array([one + 2 ** -8, one + 3 * 2 ** -8, one + 2 ** -8 + 2 ** -40, one + 2 ** -8 - 2 ** -40,
                     -(one + 2 ** -8 + 2 ** -30), 1e-40, -3.3e-39, 3.0e38, 2.5, -7.75e-3])
    n = len(vals)
    T = (np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), vals)
    Td = dev(T)
    lv = hec.sptrsv_analyze(Td[0], Td[1], 0)
    H = hec.hec_from_csr(*Td, levels=lv, vdt="bf16").arrays()
    assert np.array_equal(H["tval"].cpu().numpy().view(np.uint16), oracle.round_bf16_bits(vals))


# --- sweeps (Alg. 2) ------------------------------------------------------------------------------

def _solver(hec, T, uplo, vdt="f64", nrhs=1, **tune):
    Td = dev(T)
    lv = hec.sptrsv_analyze(Td[0], Td[1], uplo)
    H = hec.hec_from_csr(*Td, levels=lv, vdt=vdt)
    return hec.sptrsv_plan_create(H, lv, max_nrhs=nrhs, **tune)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("nrhs", [1, 3, 16])
def test_sweep_fp64_parity(hec, kind, nrhs):
    A, (L, U) = _factors(kind)
    n = len(A[0]) - 1
    B = synth.uniform_vector(n, 11, nrhs=nrhs)
    pL = _solver(hec, L, 0, nrhs=nrhs)
    pU = _solver(hec, U, 1, nrhs=nrhs)
    Bd = torch.as_tensor(B, device="cuda")
    Y = hec.sptrsv_lower(pL, Bd).cpu().numpy()
    X = hec.sptrsv_upper(pU, Bd).cpu().numpy()
    B2 = B.reshape(n, -1)
    for q in range(nrhs):
        y = oracle.lower_solve(L, B2[:, q])
        x = oracle.upper_solve(U, B2[:, q])
        assert relmax(Y.reshape(n, -1)[:, q], y) <= 1e-12
        assert relmax(X.reshape(n, -1)[:, q], x) <= 1e-12
    assert hec.hec_sync_status(pL) == 0 and hec.hec_sync_status(pU) == 0


def _rounded(T, vdt):
    rp, ci, v = T
    if vdt == "f32":
        return rp, ci, v.astype(np.float32).astype(np.float64)
    bits = oracle.round_bf16_bits(v).astype(np.uint32) << 16
    return rp, ci, bits.view(np.float32).astype(np.float64)


@pytest.mark.parametrize("kind", ["5pt64", "fv7_12", "27pt_ilut"])
@pytest.mark.parametrize("vdt", ["f32", "bf16"])
def test_sweep_reduced_precision(hec, kind, vdt):
    """Reduced-precision sweeps store values rounded once (bit-exact, checked above) and accumulate
    in FP32.  Against the FP64 solve with the SAME rounded values the only error is FP32 arithmetic,
    bounded componentwise by gamma_{q+2}(u32) M(T)^-1 |T| |x| (triangular solve backward error, plus
    the rounding of b to FP32); checked here with a safety factor of 4."""
    A, (L, U) = _factors(kind)
    n = len(A[0]) - 1
    b = synth.uniform_vector(n, 3)
    for uplo, T in [(0, L), (1, U)]:
        p = _solver(hec, T, uplo, vdt=vdt)
        x = (hec.sptrsv_lower if uplo == 0 else hec.sptrsv_upper)(p, torch.as_tensor(b, device="cuda")).cpu().numpy()
        Tr = _rounded(T, vdt)
        xr = (oracle.lower_solve if uplo == 0 else oracle.upper_solve)(Tr, b)
        q = int(np.max(np.diff(T[0])))
        u = 2.0 ** -24
        gam = (q + 2) * u / (1 - (q + 2) * u)
        rp, ci, v = Tr
        Mv = np.where(ci == np.repeat(np.arange(n), np.diff(rp)), np.abs(v), -np.abs(v))
        rhs = oracle.spmv((rp, ci, np.abs(v)), np.abs(xr))
        bound = gam * (oracle.lower_solve if uplo == 0 else oracle.upper_solve)((rp, ci, Mv), rhs)
        assert np.all(np.abs(x - xr) <= 4 * bound + 1e-30)
        # and the error against the unrounded FP64 solve is reported (not bounded here)
        x64 = (oracle.lower_solve if uplo == 0 else oracle.upper_solve)(T, b)
        print(kind, vdt, uplo, "err vs fp64 oracle %.3e" % relmax(x, x64))


def test_sweep_unaligned_strides_and_ldb(hec):
    """b and x with a leading dimension larger than nrhs."""
    A, (L, U) = _factors("fv7_12")
    n = len(A[0]) - 1
    B = synth.uniform_vector(n, 5, nrhs=5)
    Bw = np.zeros((n, 8))
    Bw[:, :5] = B
    p = _solver(hec, L, 0, nrhs=5)
    Bd = torch.as_tensor(Bw, device="cuda")
    Xd = torch.full((n, 7), 7.0, dtype=torch.float64, device="cuda")
    hec._check(hec._sptrsv_lower(p.h, 5, Bd.data_ptr(), 8, Xd.data_ptr(), 7, hec._stream(None)), "lower")
    X = Xd.cpu().numpy()
    for q in range(5):
        assert relmax(X[:, q], oracle.lower_solve(L, B[:, q])) <= 1e-12
    assert np.all(X[:, 5:] == 7.0)


def test_sweep_wrong_triangle_rejected(hec):
    A, (L, U) = _factors("5pt64")
    p = _solver(hec, L, 0)
    with pytest.raises(hec.HecError):
        hec.sptrsv_upper(p, torch.zeros(4096, dtype=torch.float64, device="cuda"))


def test_sweep_dependency_timeout_reports_status(hec):
    """Fault injection: one row's solution is never published; its dependents' bounded waits run out
    and the call reports TIMEOUT instead of hanging.  The context stays usable."""
    A, (L, U) = _factors("5pt64")
    p = _solver(hec, L, 0, wait_cycles=2_000_000, debug_unpublished_row=100)
    b = torch.as_tensor(synth.uniform_vector(4096, 1), device="cuda")
    hec.sptrsv_lower(p, b)
    assert hec.STATUS_NAMES[hec.hec_sync_status(p)] == "TIMEOUT"
    assert hec.hec_sync_status(p) == 0  # cleared
    good = _solver(hec, L, 0)
    x = hec.sptrsv_lower(good, b).cpu().numpy()
    assert relmax(x, oracle.lower_solve(L, b.cpu().numpy())) <= 1e-12


# --- preconditioner, SpMV, FGMRES -------------------------------------------------------------------

@pytest.mark.parametrize("kind", KINDS)
def test_ilu_apply_parity(hec, kind):
    A, (L, U) = _factors(kind)
    n = len(A[0]) - 1
    s = hec.IluSolver(dev(L), dev(U), max_nrhs=4)
    R = synth.uniform_vector(n, 9, nrhs=4)
    Z = s.apply(torch.as_tensor(R, device="cuda")).cpu().numpy()
    for q in range(4):
        assert relmax(Z[:, q], oracle.ilu_apply(L, U, R[:, q])) <= 1e-12


@pytest.mark.parametrize("nrhs", [1, 2, 16])
def test_spmv_parity(hec, nrhs):
    A = synth.stencil27_jitter(11, seed=1)
    n = len(A[0]) - 1
    X = synth.uniform_vector(n, 2, nrhs=nrhs)
    Y0 = synth.uniform_vector(n, 3, nrhs=nrhs)
    Ad = hec.hec_from_csr(*dev(A))
    Y = hec.spmv(Ad, torch.as_tensor(X, device="cuda"), torch.as_tensor(Y0, device="cuda"), alpha=-0.5,
                 beta=2.0).cpu().numpy()
    X2, Y02 = X.reshape(n, -1), Y0.reshape(n, -1)
    for q in range(nrhs):
        ref = -0.5 * oracle.spmv(A, X2[:, q]) + 2.0 * Y02[:, q]
        assert relmax(Y.reshape(n, -1)[:, q], ref) <= 1e-14


@pytest.mark.parametrize("vdt", ["f64", "f32", "bf16"])
def test_fgmres_ilu0_converges(hec, vdt):
    A = synth.fv7_lognormal(16, seed=4)
    n = len(A[0]) - 1
    L, U = oracle.ilu0(A)
    xt = synth.uniform_vector(n, 6)
    b = oracle.spmv(A, xt)
    s = hec.IluSolver(dev(L), dev(U), A=dev(A), vdt=vdt)
    x, info = s.solve(torch.as_tensor(b, device="cuda"), rtol=1e-8, max_iters=2000)
    x = x.cpu().numpy()
    assert info["converged"]
    assert np.linalg.norm(b - oracle.spmv(A, x)) <= 1e-8 * np.linalg.norm(b) * (1 + 1e-6)
    ref = oracle.fgmres(A, b, ("ilu", L, U), m=30, rtol=1e-8, max_iters=2000)
    # both solutions satisfy the same residual bound; their difference is bounded by the conditioning
    assert relmax(x, ref["x"]) <= 1e-4
    if vdt == "f64":
        assert abs(info["iterations"] - ref["iters"]) <= 2


def test_fgmres_multi_rhs(hec):
    A = synth.fv7_lognormal(10, seed=2)
    n = len(A[0]) - 1
    L, U = oracle.ilu0(A)
    B = synth.uniform_vector(n, 20, nrhs=4)
    s = hec.IluSolver(dev(L), dev(U), A=dev(A), max_nrhs=4)
    X, info = s.solve(torch.as_tensor(B, device="cuda"), rtol=1e-9)
    X = X.cpu().numpy()
    assert info["converged"]
    for q in range(4):
        assert np.linalg.norm(B[:, q] - oracle.spmv(A, X[:, q])) <= 1e-9 * np.linalg.norm(B[:, q]) * (1 + 1e-6)


# --- GPU factorization ---------------------------------------------------------------------------

@pytest.mark.parametrize("k", [0, 1, 2, 3])
@pytest.mark.parametrize("maker", ["5pt", "fv7", "27pt", "rand"])
def test_ilu_factor_parity(hec, k, maker):
    A = {"5pt": lambda: synth.poisson2d_5pt(40, 23), "fv7": lambda: synth.fv7_lognormal(11, seed=3),
         "27pt": lambda: synth.stencil27_jitter(7, seed=3), "rand": lambda: synth.random_sparse(600, 0.01, 8)}[maker]()
    Lh, Uh = hec.ilu_factor(*dev(A), k=k)
    L, U = [tuple(a.cpu().numpy() for a in h.tensors()) for h in (Lh, Uh)]
    Lo, Uo = oracle.ilu0(A) if k == 0 else oracle.iluk(A, k)
    for got, exp in [(L, Lo), (U, Uo)]:
        assert np.array_equal(got[0], exp[0]) and np.array_equal(got[1], exp[1])
        assert relmax(got[2], exp[2]) <= 1e-12


def test_iluk_large_k_is_exact_lu(hec):
    """With k at least the matrix order every fill entry is kept: the GPU ILU(k) is the exact LU
    (no pivoting) of a diagonally dominant matrix, so L U reproduces A."""
    A = synth.random_sparse(120, 0.05, 5)
    n = len(A[0]) - 1
    Lh, Uh = hec.ilu_factor(*dev(A), k=n)
    L, U = [tuple(a.cpu().numpy() for a in h.tensors()) for h in (Lh, Uh)]
    Ld, Ud, Ad = np.zeros((n, n)), np.zeros((n, n)), np.zeros((n, n))
    for M, (rp, ci, v) in [(Ld, L), (Ud, U), (Ad, A)]:
        for i in range(n):
            M[i, ci[rp[i]:rp[i + 1]]] = v[rp[i]:rp[i + 1]]
    assert np.max(np.abs(Ld @ Ud - Ad)) <= 1e-12 * np.max(np.abs(Ad))


def test_iluk_fgmres_with_gpu_factors(hec):
    """GPU ILU(2) factors in the solver: FGMRES reaches the bound and the oracle's iteration count
    with the oracle's ILU(2)."""
    A = synth.fv7_lognormal(16, seed=7)
    n = len(A[0]) - 1
    Ad = dev(A)
    Lh, Uh = hec.ilu_factor(*Ad, k=2)
    s = hec.IluSolver(Lh.tensors(), Uh.tensors(), A=Ad, vdt="f64")
    b = oracle.spmv(A, synth.uniform_vector(n, 9))
    x, info = s.solve(torch.as_tensor(b, device="cuda"), rtol=1e-8, max_iters=1000)
    assert info["converged"]
    assert np.linalg.norm(b - oracle.spmv(A, x.cpu().numpy())) <= 1e-8 * np.linalg.norm(b) * (1 + 1e-6)
    ref = oracle.fgmres(A, b, ("ilu", *oracle.iluk(A, 2)), m=30, rtol=1e-8)
    assert abs(info["iterations"] - ref["iters"]) <= 2
