"""RAS (Sec. 3, Eq. 4) on the GPU against the oracle: subdomain construction bit-exact, the batched
block-diagonal apply within 1e-12, and RAS-preconditioned FGMRES with 16 right-hand sides."""
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


CASES = [(10, [3, 4, 3]), (12, [5, 7]), (9, [9]), (13, [2, 4, 3, 4])]


@pytest.mark.parametrize("m,cuts", CASES)
def test_ras_setup_bit_exact(hec, m, cuts):
    A = synth.fv7_lognormal(m, seed=m)
    part, ns = synth.box_partition(m, cuts)
    R = hec.ras_setup(*[dev(a) for a in A], dev(part), ns)
    ext_ptr, ext2glob, owned, Aext = [x for x in R.tensors(ns)[:3]] + [R.tensors(ns)[3]]
    ptr, idx = oracle.ras_extend(A, part, ns)
    assert np.array_equal(ext_ptr.cpu().numpy(), ptr)
    assert np.array_equal(ext2glob.cpu().numpy(), idx)
    sub = np.repeat(np.arange(ns), np.diff(ptr))
    assert np.array_equal(owned.cpu().numpy().astype(bool), part[idx] == sub)
    blocks = [oracle.submatrix(A, idx[ptr[s]:ptr[s + 1]]) for s in range(ns)]
    rp, ci, v = oracle.block_diag(blocks)
    got = [t.cpu().numpy() for t in Aext]
    assert np.array_equal(got[0], rp) and np.array_equal(got[1], ci) and np.array_equal(got[2], v)


@pytest.mark.parametrize("m,cuts", CASES[:2])
@pytest.mark.parametrize("nrhs", [1, 16])
def test_ras_apply_with_oracle_factors(hec, m, cuts, nrhs):
    A = synth.fv7_lognormal(m, seed=1)
    part, ns = synth.box_partition(m, cuts)
    Ro = oracle.ras_setup(A, part, ns)
    n = m ** 3
    s = hec.RasSolver([dev(a) for a in A], dev(part), ns, vdt="f64", max_nrhs=nrhs,
                      factors=([dev(a) for a in Ro["L"]], [dev(a) for a in Ro["U"]]))
    R = synth.uniform_vector(n, 7, nrhs=nrhs)
    Z = s.apply(dev(R)).cpu().numpy().reshape(n, -1)
    R2 = R.reshape(n, -1)
    for q in range(nrhs):
        assert relmax(Z[:, q], oracle.ras_apply(Ro, R2[:, q])) <= 1e-12


def test_ras_apply_with_gpu_factors(hec):
    m, cuts = 12, [5, 7]
    A = synth.fv7_lognormal(m, seed=2)
    part, ns = synth.box_partition(m, cuts)
    Ro = oracle.ras_setup(A, part, ns)
    s = hec.RasSolver([dev(a) for a in A], dev(part), ns, vdt="f64")
    for got, exp in [(s.L, Ro["L"]), (s.U, Ro["U"])]:
        g = [t.cpu().numpy() for t in got]
        assert np.array_equal(g[0], exp[0]) and np.array_equal(g[1], exp[1])
        assert relmax(g[2], exp[2]) <= 1e-12
    r = synth.uniform_vector(m ** 3, 3)
    assert relmax(s.apply(dev(r)).cpu().numpy(), oracle.ras_apply(Ro, r)) <= 1e-11


def test_ras_single_subdomain_equals_ilu0(hec):
    m = 9
    A = synth.fv7_lognormal(m, seed=3)
    n = m ** 3
    s = hec.RasSolver([dev(a) for a in A], dev(np.zeros(n, np.int32)), 1, vdt="f64")
    L, U = oracle.ilu0(A)
    r = synth.uniform_vector(n, 4)
    assert relmax(s.apply(dev(r)).cpu().numpy(), oracle.ilu_apply(L, U, r)) <= 1e-12


@pytest.mark.parametrize("vdt", ["f32", "bf16"])
def test_ras_fgmres_16rhs(hec, vdt):
    m, cuts = 16, [6, 10]
    A = synth.fv7_lognormal(m, seed=5)
    part, ns = synth.box_partition(m, cuts)
    n = m ** 3
    s = hec.RasSolver([dev(a) for a in A], dev(part), ns, vdt=vdt, max_nrhs=16)
    shapes = s.autotune(16)
    assert all(sh["block_threads"] in (128, 256) and sh["blocks_per_sm"] in (2, 4, 8, 16) for sh in shapes)
    B = synth.uniform_vector(n, 40, nrhs=16)
    X, info = s.solve(dev(B), rtol=1e-8, max_iters=3000)
    X = X.cpu().numpy()
    assert info["converged"]
    for q in range(16):
        assert np.linalg.norm(B[:, q] - oracle.spmv(A, X[:, q])) <= 1e-8 * np.linalg.norm(B[:, q]) * (1 + 1e-6)
    # the oracle's RAS-FGMRES on the first right-hand side reaches the same tolerance
    Ro = oracle.ras_setup(A, part, ns)
    ref = oracle.fgmres(A, B[:, 0], ("ras", Ro), m=30, rtol=1e-8, max_iters=3000)
    assert ref["converged"]
    assert relmax(X[:, 0], ref["x"]) <= 1e-4


@pytest.mark.parametrize("m,cuts", CASES)
def test_block_ilu_setup_bit_exact_and_apply(hec, m, cuts):
    """Overlap 0 (block ILU): the subdomain system equals the oracle's owned sets and blocks bit for
    bit, and the batched apply with the GPU's own ILU(0) of the blocks matches the oracle's."""
    A = synth.fv7_lognormal(m, seed=m + 1)
    part, ns = synth.box_partition(m, cuts)
    Ad = [dev(a) for a in A]
    R = hec.ras_setup(*Ad, dev(part), ns, overlap=0)
    ext_ptr, ext2glob, owned, Aext = R.tensors(ns)
    ptr, idx = oracle.owned_sets(part, ns)
    assert np.array_equal(ext_ptr.cpu().numpy(), ptr) and np.array_equal(ext2glob.cpu().numpy(), idx)
    assert bool(owned.cpu().numpy().all())
    rp, ci, v = oracle.block_diag([oracle.submatrix(A, idx[ptr[s]:ptr[s + 1]]) for s in range(ns)])
    got = [t.cpu().numpy() for t in Aext]
    assert np.array_equal(got[0], rp) and np.array_equal(got[1], ci) and np.array_equal(got[2], v)
    Ro = oracle.ras_setup(A, part, ns, overlap=0)
    s = hec.RasSolver(Ad, dev(part), ns, vdt="f64", max_nrhs=4, overlap=0)
    Rv = synth.uniform_vector(m ** 3, 3, nrhs=4)
    Z = s.apply(dev(Rv)).cpu().numpy()
    for q in range(4):
        assert relmax(Z[:, q], oracle.ras_apply(Ro, Rv[:, q])) <= 1e-12


def test_block_ilu_fgmres_16_rhs(hec):
    m = 24
    A = synth.fv7_lognormal(m, seed=5)
    part, ns = synth.box_partition(m, [5, 8, 5, 6])
    Ad = [dev(a) for a in A]
    s = hec.RasSolver(Ad, dev(part), ns, vdt="f32", max_nrhs=16, overlap=0)
    Xt = synth.uniform_vector(m ** 3, 11, nrhs=16)
    B = np.column_stack([oracle.spmv(A, Xt[:, q]) for q in range(16)])
    X, info = s.solve(dev(B), rtol=1e-8, max_iters=3000)
    X = X.cpu().numpy()
    assert info["converged"]
    for q in (0, 9, 15):
        r = B[:, q] - oracle.spmv(A, X[:, q])
        assert np.linalg.norm(r) <= 1e-8 * np.linalg.norm(B[:, q]) * (1 + 1e-6)


@pytest.mark.parametrize("overlap", [0, 1])
def test_block_ilut_factors_and_apply(hec, overlap):
    """The paper's BILUT (overlap 0) and RAS with ILUT blocks (overlap 1): the GPU ILUT of the
    block-diagonal subdomain system equals the oracle's per-block ILUT bit for bit, and the
    batched apply matches the oracle's apply with those factors."""
    m, cuts = 12, [5, 7]
    A = synth.fv7_lognormal(m, seed=21)
    part, ns = synth.box_partition(m, cuts)
    Ad = [dev(a) for a in A]
    p, tol = 4, 1e-2
    s = hec.RasSolver(Ad, dev(part), ns, vdt="f64", max_nrhs=2, overlap=overlap, ilut=(p, tol))
    Ro = oracle.ras_setup(A, part, ns, overlap=overlap)
    ptr, idx = Ro["ext_ptr"], Ro["ext_idx"]
    blocks = [oracle.ilut(oracle.submatrix(A, idx[ptr[q]:ptr[q + 1]]), p, tol) for q in range(ns)]
    Ro["L"] = oracle.block_diag([b[0] for b in blocks])
    Ro["U"] = oracle.block_diag([b[1] for b in blocks])
    for got, ref in ((s.L, Ro["L"]), (s.U, Ro["U"])):
        assert all(np.array_equal(g.cpu().numpy(), r) for g, r in zip(got, ref))
    Rv = synth.uniform_vector(m ** 3, 8, nrhs=2)
    Z = s.apply(dev(Rv)).cpu().numpy()
    for q in range(2):
        assert relmax(Z[:, q], oracle.ras_apply(Ro, Rv[:, q])) <= 1e-12
    b = synth.uniform_vector(m ** 3, 9)
    x, info = s.solve(dev(b), rtol=1e-8)
    assert info["converged"]


def test_ras_setup_rejects_other_overlaps(hec):
    A = synth.fv7_lognormal(6, seed=1)
    part, ns = synth.box_partition(6, [3, 3])
    with pytest.raises(Exception):
        hec.ras_setup(*[dev(a) for a in A], dev(part), ns, overlap=2)


@pytest.mark.parametrize("vdt", ["f64", "f32"])
def test_ras_one_part_per_subdomain(hec, vdt):
    """RAS on x-pencil subdomains, every subdomain one part of the partitioned sweeps: the blocks of
    Eq. 4 are independent, so no dependency crosses a part.  The apply equals the unpartitioned
    apply up to summation order, and a second apply (the other of the double-buffered solution
    words) repeats the first bit for bit; with the
    oracle's FP64 factors it matches the oracle's RAS apply to 1e-12 (FP64 values) or, with FP32
    values, the oracle's apply on the same rounded values within the FP32 substitution error; the
    partitioned solve reaches 1e-8 in the oracle's iteration count."""
    m = 16
    A = synth.fv7_lognormal(m, seed=5)
    n = m ** 3
    part, ns = synth.grid_boxes(m, (1, 4, 4))
    Ro = oracle.ras_setup(A, part, ns)
    s = hec.RasSolver([dev(a) for a in A], dev(part), ns, vdt=vdt,
                      factors=([dev(a) for a in Ro["L"]], [dev(a) for a in Ro["U"]]))
    r = synth.uniform_vector(n, 17)
    ref = s.apply(dev(r)).cpu().numpy()
    sizes = np.diff(s.ext_ptr.cpu().numpy())
    sp = np.repeat(np.arange(ns, dtype=np.int32), sizes)
    assert s.partition(dev(sp), ns, threads=512) == ns
    got = s.apply(dev(r)).cpu().numpy()
    assert relmax(got, ref) <= (1e-12 if vdt == "f64" else 1e-5)
    assert np.array_equal(s.apply(dev(r)).cpu().numpy(), got)
    if vdt == "f64":
        assert relmax(got, oracle.ras_apply(Ro, r)) <= 1e-12
    else:
        # the block-diagonal apply on the extended rows with the stored (rounded) values, restricted
        # to the owned rows, under the componentwise FP32 substitution bound
        Lr, Ur = _bounds.rounded(Ro["L"], "f32"), _bounds.rounded(Ro["U"], "f32")
        idx = Ro["ext_idx"]
        y = oracle.lower_solve(Lr, r[idx])
        z = oracle.upper_solve(Ur, y)
        bound = _bounds.apply_bound(Lr, Ur, y, z)
        own = part[idx] == np.repeat(np.arange(ns), np.diff(Ro["ext_ptr"]))
        assert np.count_nonzero(own) == n
        assert np.all(np.abs(got[idx[own]] - z[own]) <= bound[own])
    b = synth.uniform_vector(n, 18)
    x, info = s.solve(dev(b), rtol=1e-8)
    ref_its = oracle.fgmres(A, b, ("ras", Ro), m=30, rtol=1e-8)["iters"]
    assert info["converged"] and info["rel_residual"] <= 1e-8
    assert abs(info["iterations"] - ref_its) <= (1 if vdt == "f64" else 2)
