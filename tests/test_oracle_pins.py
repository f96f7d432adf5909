"""Pins for the CPU oracle: each check ties an oracle function to something other than itself
(a textbook or library routine on a special case, a closed form, brute force on tiny inputs,
or an invariant the mathematics fixes), so that a dropped term, a wrong sign, a wrong index or
a transposed operand in the oracle fails here.  CPU only."""
import fractions
import itertools
import struct

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

from paper_1606_00541_gb300 import synth


def dense(A, n=None):
    rp, ci, v = A
    n = len(rp) - 1 if n is None else n
    return sp.csr_matrix((v, ci, rp), shape=(n, n)).toarray()


def csr_of(D):
    M = sp.csr_matrix(D)
    M.sort_indices()
    return M.indptr.astype(np.int32), M.indices.astype(np.int32), M.data.astype(np.float64)


# --- forward / back substitution (Eq. 1) -----------------------------------------------------

@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("density", [0.05, 0.3, 1.0])
def test_substitution_matches_dense_triangular_solve(orc, seed, density):
    n = 48
    L = synth.random_lower(n, density, seed)
    U = synth.random_lower(n, density, seed + 100, uplo=1)
    b = synth.uniform_vector(n, seed)
    y = orc.lower_solve(L, b)
    x = orc.upper_solve(U, b)
    ry = sla.solve_triangular(dense(L), b, lower=True)
    rx = sla.solve_triangular(dense(U), b, lower=False)
    assert np.max(np.abs(y - ry)) <= 1e-13 * max(1.0, np.max(np.abs(ry)))
    assert np.max(np.abs(x - rx)) <= 1e-13 * max(1.0, np.max(np.abs(rx)))


def _comparison_bound(T, xhat, uplo, orc):
    """Componentwise a-priori bound for triangular substitution: |xhat - x| <= gamma_{q+1}
    M(T)^-1 |T| |xhat| with M(T) the comparison matrix (Higham, Thm. 8.5 and Sec. 8.2)."""
    rp, ci, v = T
    n = len(rp) - 1
    q = int(np.max(np.diff(rp)))
    u = 2.0 ** -53
    gam = (q + 1) * u / (1 - (q + 1) * u)
    absT = (rp, ci, np.abs(v))
    rhs = orc.spmv(absT, np.abs(xhat))
    diag = np.zeros(n)
    for i in range(n):
        for p in range(rp[i], rp[i + 1]):
            if ci[p] == i:
                diag[i] = abs(v[p])
    Mv = np.where(ci == np.repeat(np.arange(n), np.diff(rp)), np.abs(v), -np.abs(v))
    M = (rp, ci, Mv)
    z = orc.lower_solve(M, rhs) if uplo == 0 else orc.upper_solve(M, rhs)
    return gam * z


def test_manufactured_solution_within_a_priori_bound(orc):
    A = synth.fv7_lognormal(12, seed=3)
    L, U = orc.ilu0(A)
    n = len(A[0]) - 1
    xt = synth.uniform_vector(n, 7)
    b = orc.spmv(L, xt)
    y = orc.lower_solve(L, b)
    # the computed solution of the perturbed system is within the backward-error bound of xt
    bound = _comparison_bound(L, y, 0, orc) + 4 * 2.0 ** -53 * np.abs(xt)
    assert np.all(np.abs(y - xt) <= bound * 4 + 1e-300)
    bu = orc.spmv(U, xt)
    x = orc.upper_solve(U, bu)
    bound = _comparison_bound(U, x, 1, orc) + 4 * 2.0 ** -53 * np.abs(xt)
    assert np.all(np.abs(x - xt) <= bound * 4 + 1e-300)


def test_substitution_rejects_malformed(orc):
    L = synth.random_lower(10, 0.3, 1)
    U = synth.random_lower(10, 0.3, 1, uplo=1)
    assert orc.check_triangular(L, 0) == 0 and orc.check_triangular(U, 1) == 0
    assert orc.check_triangular(U, 0) == -1
    rp, ci, v = L
    v0 = v.copy()
    v0[rp[1] - 1] = 0.0  # row 0's diagonal
    assert orc.check_triangular((rp, ci, v0), 0) == -3
    with pytest.raises(orc.OracleError):
        orc.lower_solve((rp, ci, v0), np.ones(10))


# --- levels (Eq. 2) and map (Eq. 3) --------------------------------------------------------

def brute_levels(T, uplo):
    """Longest dependency chain ending at each row, by memoised DFS over the DAG."""
    rp, ci, _ = T
    n = len(rp) - 1
    memo = {}

    def depth(i):
        if i in memo:
            return memo[i]
        deps = [int(j) for j in ci[rp[i]:rp[i + 1]] if (j < i if uplo == 0 else j > i)]
        memo[i] = 0 if not deps else 1 + max(depth(j) for j in deps)
        return memo[i]

    import sys
    sys.setrecursionlimit(10000)
    return np.array([depth(i) for i in range(n)])


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("uplo", [0, 1])
def test_levels_equal_longest_path(orc, seed, uplo):
    n = 200 + 17 * seed
    T = synth.random_lower(n, [0.002, 0.01, 0.05][seed % 3], seed, uplo=uplo)
    lev, nlev = orc.levels(T, uplo)
    ref = brute_levels(T, uplo)
    assert np.array_equal(lev, ref)
    assert nlev == ref.max() + 1
    # invariants: every dependency is on a strictly lower level, every row above level 0 has a
    # dependency exactly one level down
    rp, ci, _ = T
    for i in range(n):
        deps = [j for j in ci[rp[i]:rp[i + 1]] if (j < i if uplo == 0 else j > i)]
        assert all(lev[j] < lev[i] for j in deps)
        if lev[i] > 0:
            assert any(lev[j] == lev[i] - 1 for j in deps)


@pytest.mark.parametrize("a,b", [(64, 64), (7, 13), (1, 9)])
def test_levels_closed_form_5pt(orc, a, b):
    A = synth.poisson2d_5pt(a, b)
    L, U = orc.ilu0(A)
    lev, nlev = orc.levels(L, 0)
    assert nlev == a + b - 1
    g = np.arange(a * b)
    assert np.array_equal(lev, g % a + g // a)  # l = x + y
    levU, nlevU = orc.levels(U, 1)
    assert nlevU == a + b - 1
    assert np.array_equal(levU, (a - 1 - g % a) + (b - 1 - g // a))


@pytest.mark.parametrize("m", [3, 6, 10])
def test_levels_closed_form_7pt_27pt(orc, m):
    A = synth.fv7_lognormal(m, seed=1)
    L, U = orc.ilu0(A)
    g = np.arange(m ** 3)
    x, y, z = g % m, (g // m) % m, g // (m * m)
    lev, nlev = orc.levels(L, 0)
    assert nlev == 3 * m - 2 and np.array_equal(lev, x + y + z)
    A27 = synth.stencil27_jitter(m, seed=2)
    L27, _ = orc.ilu0(A27)
    lev27, nlev27 = orc.levels(L27, 0)
    assert nlev27 == 7 * (m - 1) + 1 and np.array_equal(lev27, x + 2 * y + 4 * z)


def test_level_map_properties(orc):
    T = synth.random_lower(300, 0.01, 5)
    for uplo, TT in [(0, T), (1, synth.random_lower(300, 0.01, 6, uplo=1))]:
        lev, nlev = orc.levels(TT, uplo)
        perm, iperm, lp = orc.level_map(lev, nlev, uplo)
        n = len(lev)
        assert np.array_equal(np.sort(perm), np.arange(n))
        assert np.array_equal(iperm[perm], np.arange(n))
        assert np.array_equal(np.diff(lp), np.bincount(lev, minlength=nlev))
        # rows of level k occupy [lp[k], lp[k+1]) in ascending order of the lower problem's index
        order = np.arange(n) if uplo == 0 else np.arange(n)[::-1]
        expect = np.concatenate([order[lev[order] == k] for k in range(nlev)])
        assert np.array_equal(iperm, expect)
        # L' stays lower triangular: every dependency maps to a smaller new index
        rp, ci, _ = TT
        for i in range(n):
            for j in ci[rp[i]:rp[i + 1]]:
                if j != i:
                    assert perm[j] < perm[i]


def test_level_map_golden(orc):
    """Hand-worked 6x6 example, tests/golden/levels_6x6.txt."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "levels_6x6.txt")
    rows, exp = {}, {}
    for line in open(path):
        line = line.split("#")[0].strip()
        if not line:
            continue
        key, val = line.split(":")
        nums = [int(t) for t in val.split()]
        if key.startswith("row"):
            rows[int(key[3:])] = nums
        else:
            exp[key.strip()] = nums
    n = len(rows)
    rp, ci = [0], []
    for i in range(n):
        ci += rows[i]
        rp.append(len(ci))
    T = (np.array(rp, np.int32), np.array(ci, np.int32), np.ones(len(ci)))
    lev, nlev = orc.levels(T, 0)
    perm, iperm, lp = orc.level_map(lev, nlev, 0)
    assert list(lev) == exp["level"]
    assert nlev == exp["nlev"][0]
    assert list(perm) == exp["perm"]
    assert list(lp) == exp["level_ptr"]


# --- value rounding ------------------------------------------------------------------------

def _bf16_nearest_even(d):
    """Brute force with exact rationals: the bf16 value nearest to d, ties to the even code."""
    f32 = struct.unpack("<I", struct.pack("<f", np.float32(abs(d))))[0]
    base = f32 >> 16
    best = None
    for code in range(max(base - 2, 0), min(base + 3, 0x7F80)):
        val = struct.unpack("<f", struct.pack("<I", code << 16))[0]
        err = abs(fractions.Fraction(val) - fractions.Fraction(abs(d)))
        key = (err, code & 1)
        if best is None or key < best[0]:
            best = (key, code)
    return best[1] | (0x8000 if d < 0 else 0)


def test_bf16_rounding_brute_force(orc):
    rng = np.random.default_rng(0)
    xs = list(rng.normal(0, 1, 400) * 10.0 ** rng.integers(-30, 30, 400))
    # exact ties and near-ties where FP64 -> FP32 -> BF16 double rounding goes wrong
    one = 1.0
    xs += [one + 2 ** -8, one + 3 * 2 ** -8, one + 2 ** -8 + 2 ** -40, one + 2 ** -8 - 2 ** -40,
           -(one + 2 ** -8 + 2 ** -30), 1e-40, -3.3e-39, 3.0e38]
    got = orc.round_bf16_bits(np.array(xs))
    for x, g in zip(xs, got):
        assert int(g) == _bf16_nearest_even(x), x


def test_f32_rounding_matches_numpy(orc):
    xs = np.random.default_rng(1).normal(0, 1, 500) * 10.0 ** np.random.default_rng(2).integers(-30, 30, 500)
    got = orc.round_f32_bits(xs)
    assert np.array_equal(got, xs.astype(np.float32).view(np.uint32))


# --- HEC (Sec. 2.1) ------------------------------------------------------------------------

def test_ell_width_rule_closed_forms(orc):
    A5 = synth.poisson2d_5pt(64)
    L5, _ = orc.ilu0(A5)
    H = orc.hec_pack(L5, 1, 0, *orc.level_map(*orc.levels(L5, 0), 0)[:2])
    assert H["w"] == 2
    A7 = synth.fv7_lognormal(16, seed=0)
    L7, _ = orc.ilu0(A7)
    H7 = orc.hec_pack(L7, 1, 0, *orc.level_map(*orc.levels(L7, 0), 0)[:2])
    assert H7["w"] == 3
    assert orc.ell_width_rule([0] * 10) == 0
    assert orc.ell_width_rule([5] * 7 + [0] * 3) == 5      # 7 of 10 rows >= 5 (7 >= 6.5)
    assert orc.ell_width_rule([5] * 6 + [0] * 4) == 0      # 6 < ceil(6.5)


@pytest.mark.parametrize("vdt", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("uplo", [0, 1])
@pytest.mark.parametrize("w", [-1, 0, 1, 5])
def test_hec_round_trip_and_layout(orc, vdt, uplo, w):
    A = synth.stencil27_jitter(5, seed=4)
    L, U = orc.ilut(A, 10, 1e-3)
    T = L if uplo == 0 else U
    an = orc.analyze(T, uplo)
    H = orc.hec_pack(T, 1, uplo, an["perm"], an["iperm"], w=w, vdt=vdt)
    n, ld, ww = H["n"], H["ld"], H["w"]
    rp, ci, v = orc.hec_unpack(H, 1, an["iperm"])
    assert np.array_equal(rp, T[0]) and np.array_equal(ci, T[1])
    if vdt == "f64":
        assert np.array_equal(v, T[2])
    elif vdt == "f32":
        assert np.array_equal(v, T[2].astype(np.float32).astype(np.float64))
    else:
        bits = orc.round_bf16_bits(T[2]).astype(np.uint32) << 16
        assert np.array_equal(v, bits.view(np.float32).astype(np.float64))
    assert ld % 32 == 0 and ld >= n
    tp = H["tptr"]
    assert np.all(np.diff(tp) >= 1)
    # the last tail entry of every new row r is its diagonal (new column r)
    assert np.array_equal(H["tcol"][tp[1:] - 1], np.arange(n))
    ec = H["ell_col"].reshape(ww, ld) if ww else np.zeros((0, ld), np.int32)
    for r in range(n):
        row = [c for c in ec[:, r] if c >= 0] + list(H["tcol"][tp[r]:tp[r + 1] - 1])
        assert row == sorted(row) and all(c < r for c in row)
        k = len([c for c in ec[:, r] if c >= 0])
        assert np.all(ec[:k, r] >= 0) and np.all(ec[k:, r] == -1)   # padding after the entries
        if tp[r + 1] - tp[r] > 1:
            assert k == ww                                          # tail only when the slab is full
    assert np.all(ec[:, n:] == -1)


def test_hec_general_matrix_round_trip(orc):
    A = synth.fv7_lognormal(6, seed=2)
    H = orc.hec_pack(A, 0)
    assert H["w"] == 7 - 0 or H["w"] <= 7
    rp, ci, v = orc.hec_unpack(H, 0)
    assert np.array_equal(rp, A[0]) and np.array_equal(ci, A[1]) and np.array_equal(v, A[2])


# --- SpMV and factorizations (Sec. 3) ------------------------------------------------------

def test_spmv_matches_scipy(orc):
    A = synth.stencil27_jitter(6, seed=1)
    x = synth.uniform_vector(len(A[0]) - 1, 3)
    ref = sp.csr_matrix((A[2], A[1], A[0])) @ x
    assert np.max(np.abs(orc.spmv(A, x) - ref)) <= 1e-13 * np.max(np.abs(ref))


def _lu_nopivot(D):
    n = D.shape[0]
    P, Lr, Ur = sla.lu(D)
    assert np.array_equal(P, np.eye(n)), "test matrix must not pivot"
    return Lr, Ur


@pytest.mark.parametrize("n", [1, 2, 9, 30])
def test_ilu0_tridiagonal_is_exact_lu(orc, n):
    D = np.diag(np.full(n, 4.0)) + np.diag(np.full(n - 1, -1.3), 1) + np.diag(np.full(n - 1, -0.7), -1)
    L, U = orc.ilu0(csr_of(D))
    Lr, Ur = _lu_nopivot(D)
    assert np.allclose(dense(L), Lr, rtol=0, atol=1e-14)
    assert np.allclose(dense(U), Ur, rtol=0, atol=1e-14)


def test_ilu0_dense_pattern_is_exact_lu(orc):
    rng = np.random.default_rng(3)
    D = rng.uniform(-1, 1, (12, 12))
    D += np.diag(np.abs(D).sum(axis=0) + 1.0)  # column diagonally dominant: no pivoting
    L, U = orc.ilu0(csr_of(D))
    Lr, Ur = _lu_nopivot(D)
    assert np.allclose(dense(L), Lr, atol=1e-13) and np.allclose(dense(U), Ur, atol=1e-13)


@pytest.mark.parametrize("maker", ["fv7", "27pt", "rand"])
def test_ilu0_reproduces_a_on_its_pattern(orc, maker):
    A = {"fv7": lambda: synth.fv7_lognormal(8, seed=5), "27pt": lambda: synth.stencil27_jitter(6, seed=5),
         "rand": lambda: synth.random_sparse(150, 0.03, 5)}[maker]()
    L, U = orc.ilu0(A)
    LU = dense(L) @ dense(U)
    D = dense(A)
    mask = D != 0
    scale = np.abs(D).max()
    assert np.max(np.abs((LU - D)[mask])) <= 1e-13 * scale
    assert np.array_equal(dense(L) != 0, np.tril(mask) | np.eye(len(D), dtype=bool))
    assert np.all(np.diag(dense(L)) == 1.0)


def brute_fill_levels(A):
    """Fill level of (i,j) = (shortest path i -> j in the graph of A whose intermediate
    vertices are all < min(i, j)) - 1 (the path theorem for level of fill)."""
    rp, ci, _ = A
    n = len(rp) - 1
    adj = [set(int(j) for j in ci[rp[i]:rp[i + 1]]) for i in range(n)]
    lev = {}
    for i in range(n):
        for j in range(n):
            lim = min(i, j)
            # BFS from i over vertices < lim, target j
            dist = {i: 0}
            frontier = [i]
            found = None
            while frontier and found is None:
                nxt = []
                for u in frontier:
                    for w in adj[u]:
                        if w == j:
                            found = dist[u] + 1
                            break
                        if w < lim and w not in dist:
                            dist[w] = dist[u] + 1
                            nxt.append(w)
                    if found is not None:
                        break
                frontier = nxt
            if i == j:
                lev[(i, j)] = 0
            elif found is not None:
                lev[(i, j)] = found - 1
    return lev


@pytest.mark.parametrize("k", [0, 1, 2, 3])
def test_iluk_pattern_matches_path_theorem(orc, k):
    A = synth.random_sparse(40, 0.06, 11)
    prp, pci = orc.iluk_pattern(A, k)
    lev = brute_fill_levels(A)
    expect = sorted((i, j) for (i, j), l in lev.items() if l <= k)
    got = sorted((i, int(j)) for i in range(40) for j in pci[prp[i]:prp[i + 1]])
    assert got == expect


def test_iluk_large_k_is_exact_lu(orc):
    A = synth.random_sparse(25, 0.1, 2)
    L, U = orc.iluk(A, 25)
    D = dense(A)
    P, Lr, Ur = sla.lu(D)
    if np.array_equal(P, np.eye(25)):
        assert np.allclose(dense(L), Lr, atol=1e-12) and np.allclose(dense(U), Ur, atol=1e-12)
    assert np.allclose(dense(L) @ dense(U), D, atol=1e-12)


def test_iluk_level1_fill_count_7pt(orc):
    """Interior rows of the ILU(1) factors of a 7-point matrix hold 13 entries of L+U
    (7 original + 6 fill: the (x-1,y+1), (x+1,y-1), (x-1,z+1), (x+1,z-1), (y-1,z+1), (y+1,z-1)
    neighbours)."""
    m = 7
    A = synth.fv7_lognormal(m, seed=0)
    prp, pci = orc.iluk_pattern(A, 1)
    g = np.arange(m ** 3)
    x, y, z = g % m, (g // m) % m, g // (m * m)
    interior = (x > 0) & (x < m - 1) & (y > 0) & (y < m - 1) & (z > 0) & (z < m - 1)
    assert np.all(np.diff(prp)[interior] == 13)


def test_ilut_limits(orc):
    A = synth.random_sparse(30, 0.15, 9)
    D = dense(A)
    L, U = orc.ilut(A, 30, 0.0)         # no dropping: exact LU
    assert np.allclose(dense(L) @ dense(U), D, atol=1e-12)
    L0, U0 = orc.ilut(A, 0, 0.0)        # p = 0: only diagonals survive, U = diag(A)
    assert np.array_equal(dense(L0), np.eye(30))
    assert np.array_equal(dense(U0), np.diag(np.diag(D)))
    A7 = synth.fv7_lognormal(5, seed=1)
    Lt, Ut = orc.ilut(A7, 3, 1e-2)
    rp = A7[0]
    tau = 1e-2 * np.sqrt(np.add.reduceat(A7[2] ** 2, rp[:-1]))
    for T, part in [(Lt, "L"), (Ut, "U")]:
        rpt, cit, vt = T
        for i in range(len(rpt) - 1):
            off = [(c, v) for c, v in zip(cit[rpt[i]:rpt[i + 1]], vt[rpt[i]:rpt[i + 1]]) if c != i]
            assert len(off) <= 3
            assert all(abs(v) >= tau[i] for _, v in off)


def test_ilut_hand_worked_example(orc):
    """ILUT(p = 1, tol = 0.01) (Sec. 3; Saad's dual threshold) on a 4 x 4 matrix, factors worked
    by hand.  tau_i = tol * ||a_i||_2 of the original row; a multiplier below tau is dropped
    before it updates the row; after the row's elimination the p largest of each part survive
    (ties to the smaller column).  Row 0: the tie between columns 1 and 2 keeps column 1.  Row 2:
    the multiplier 0.3 / 4 = 0.075 passes tau_2 = 0.0671 (with a 1-norm tau, 0.093, it would be
    dropped), updates column 1 to 3 - 0.075 = 2.925, and is then dropped by p; (2,1) = 2.925 / 4.5
    = 0.65 and the fill (2,3) = -0.65.  Row 3: the multiplier 0.01 / 6 is below tau_3 = 0.0806 and
    is dropped before updating, so u33 = 8 - 1 / 4.5."""
    A = csr_of(np.array([[4.0, 1.0, 1.0, 0.0],
                         [2.0, 5.0, 0.0, 1.0],
                         [0.3, 3.0, 6.0, 0.0],
                         [0.0, 1.0, 0.01, 8.0]]))
    L, U = orc.ilut(A, 1, 0.01)
    L_hand = np.array([[1.0, 0.0, 0.0, 0.0],
                       [0.5, 1.0, 0.0, 0.0],
                       [0.0, 0.65, 1.0, 0.0],
                       [0.0, 0.2222222222222222, 0.0, 1.0]])
    U_hand = np.array([[4.0, 1.0, 0.0, 0.0],
                       [0.0, 4.5, 0.0, 1.0],
                       [0.0, 0.0, 6.0, -0.65],
                       [0.0, 0.0, 0.0, 7.777777777777778]])
    assert np.abs(dense(L) - L_hand).max() <= 1e-15
    assert np.abs(dense(U) - U_hand).max() <= 1e-15
    # the kept pattern exactly (no explicit zeros where the hand factors are zero)
    assert list(L[1]) == [0, 0, 1, 1, 2, 1, 3] and list(U[1]) == [0, 1, 1, 3, 2, 3, 3]


def test_ilut_tridiagonal_equals_ilu0(orc):
    n = 20
    D = np.diag(np.full(n, 3.0)) + np.diag(np.full(n - 1, -1.0), 1) + np.diag(np.full(n - 1, -1.2), -1)
    A = csr_of(D)
    L0, U0 = orc.ilu0(A)
    Lt, Ut = orc.ilut(A, 5, 1e-12)
    assert np.allclose(dense(L0), dense(Lt), atol=1e-15) and np.allclose(dense(U0), dense(Ut), atol=1e-15)


# --- RAS (Sec. 3, Eq. 4) -------------------------------------------------------------------

def test_ras_single_subdomain_is_ilu0(orc):
    A = synth.fv7_lognormal(6, seed=1)
    n = len(A[0]) - 1
    R = orc.ras_setup(A, np.zeros(n, np.int32), 1)
    L, U = orc.ilu0(A)
    v = synth.uniform_vector(n, 2)
    assert np.array_equal(orc.ras_apply(R, v), orc.ilu_apply(L, U, v))


def test_ras_with_exact_local_solves_matches_dense_definition(orc):
    m = 6
    A = synth.fv7_lognormal(m, seed=2)
    n = m ** 3
    part, ns = synth.box_partition(m, [2, 4])
    ptr, idx = orc.ras_extend(A, part, ns)
    # overlap 1: ext = owned + graph neighbours
    D = dense(A)
    for s in range(ns):
        owned = set(np.nonzero(part == s)[0])
        nb = set(owned)
        for i in owned:
            nb |= set(np.nonzero(D[i])[0])
        assert list(idx[ptr[s]:ptr[s + 1]]) == sorted(nb)
    Ls, Us = [], []
    for s in range(ns):
        As = orc.submatrix(A, idx[ptr[s]:ptr[s + 1]])
        L, U = orc.iluk(As, 10 ** 6)  # exact LU of the subdomain matrix
        Ls.append(L)
        Us.append(U)
    R = dict(ext_ptr=ptr, ext_idx=idx, part=part, ns=ns, L=orc.block_diag(Ls), U=orc.block_diag(Us))
    v = synth.uniform_vector(n, 4)
    z = orc.ras_apply(R, v)
    ref = np.zeros(n)
    for s in range(ns):
        e = idx[ptr[s]:ptr[s + 1]]
        y = np.linalg.solve(D[np.ix_(e, e)], v[e])
        own = part[e] == s
        ref[e[own]] = y[own]
    assert np.max(np.abs(z - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_block_ilu_on_tridiagonal_blocks_is_block_jacobi(orc):
    """Overlap 0 (the paper's block ILU): each subdomain keeps its owned rows; on a tridiagonal
    matrix ILU(0) of every diagonal block is its exact LU, so the apply equals block Jacobi,
    z_s = A[s, s]^-1 v_s, written out densely."""
    n = 40
    D = np.diag(np.full(n, 2.5)) + np.diag(np.full(n - 1, -1.0), 1) + np.diag(np.full(n - 1, -1.1), -1)
    A = csr_of(D)
    part = np.array([0] * 7 + [2] * 13 + [1] * 9 + [0] * 11, dtype=np.int32)  # block 0 not contiguous
    R = orc.ras_setup(A, part, 3, overlap=0)
    ptr, idx = R["ext_ptr"], R["ext_idx"]
    for s in range(3):
        assert list(idx[ptr[s]:ptr[s + 1]]) == list(np.flatnonzero(part == s))
    v = synth.uniform_vector(n, 6)
    z = orc.ras_apply(R, v)
    ref = np.zeros(n)
    for s in range(3):
        e = np.flatnonzero(part == s)
        ref[e] = np.linalg.solve(D[np.ix_(e, e)], v[e])
    assert np.max(np.abs(z - ref)) <= 1e-13 * np.max(np.abs(ref))


# --- symmetric Gauss-Seidel (the smoother use of the sweeps) ----------------------------------

def test_sgs_matches_the_matrix_splitting(orc):
    """The loops against the splitting A = L_s + D + U_s written with dense solves:
    x' = (D + L_s)^-1 (b - U_s x0), x'' = (D + U_s)^-1 (b - L_s x')."""
    A = synth.random_sparse(50, 0.1, 9, dominance=1.5)
    D = dense(A)
    b = synth.uniform_vector(50, 2)
    x0 = synth.uniform_vector(50, 3)
    Ls, Us, Dg = np.tril(D, -1), np.triu(D, 1), np.diag(np.diag(D))
    x1 = np.linalg.solve(Dg + Ls, b - Us @ x0)
    x2 = np.linalg.solve(Dg + Us, b - Ls @ x1)
    assert np.max(np.abs(orc.sgs(A, b, x0, 1) - x2)) <= 1e-12 * np.max(np.abs(x2))


def test_sgs_special_cases(orc):
    # lower triangular: the forward sweep is the exact solve and the backward sweep keeps it
    L = orc.ilu0(synth.fv7_lognormal(4, seed=3))[0]
    b = synth.uniform_vector(64, 4)
    ref = sla.solve_triangular(dense(L), b, lower=True)
    assert np.max(np.abs(orc.sgs(L, b, np.zeros(64), 1) - ref)) <= 1e-13 * np.max(np.abs(ref))
    # diagonal: one sweep divides by the diagonal
    d = np.linspace(1.0, 3.0, 10)
    Dm = csr_of(np.diag(d))
    assert np.array_equal(orc.sgs(Dm, np.ones(10), np.zeros(10), 1), 1.0 / d)


def test_sgs_converges_in_the_energy_norm(orc):
    """For SPD A each symmetric sweep is a contraction in the A-norm of the error."""
    A = synth.poisson2d_5pt(8)
    D = dense(A)
    b = synth.uniform_vector(64, 5)
    xs = np.linalg.solve(D, b)
    x = np.zeros(64)
    prev = np.inf
    for _ in range(100):
        x = orc.sgs(A, b, x, 1)
        e = x - xs
        en = float(e @ D @ e)
        assert en < prev or en < 1e-28
        prev = en
    assert np.max(np.abs(x - xs)) <= 1e-8 * np.max(np.abs(xs))


# --- FGMRES --------------------------------------------------------------------------------

def test_fgmres_unrestarted_matches_dense_solve(orc):
    A = synth.random_sparse(60, 0.08, 4)
    b = synth.uniform_vector(60, 1)
    out = orc.fgmres(A, b, None, m=60, rtol=1e-12, max_iters=60)
    ref = np.linalg.solve(dense(A), b)
    assert out["converged"]
    assert np.max(np.abs(out["x"] - ref)) <= 1e-9 * np.max(np.abs(ref))
    h = out["history"][: out["iters"] + 1]
    assert np.all(np.diff(h) <= 1e-15)  # monotone non-increasing residual estimate


def test_fgmres_exact_preconditioner_one_iteration(orc):
    A = synth.random_sparse(40, 0.1, 6)
    L, U = orc.iluk(A, 40)
    b = synth.uniform_vector(40, 2)
    out = orc.fgmres(A, b, ("ilu", L, U), m=30, rtol=1e-10)
    assert out["converged"] and out["iters"] == 1


def test_fgmres_ilu0_converges_and_true_residual(orc):
    A = synth.fv7_lognormal(10, seed=3)
    n = len(A[0]) - 1
    L, U = orc.ilu0(A)
    xt = synth.uniform_vector(n, 5)
    b = orc.spmv(A, xt)
    out = orc.fgmres(A, b, ("ilu", L, U), m=30, rtol=1e-8, max_iters=2000)
    r = b - orc.spmv(A, out["x"])
    assert out["converged"] and np.linalg.norm(r) <= 1e-8 * np.linalg.norm(b)
    plain = orc.fgmres(A, b, None, m=30, rtol=1e-8, max_iters=5000)
    assert out["iters"] < plain["iters"]
