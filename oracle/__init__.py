"""CPU oracle for the level-scheduled HEC triangular solver (arXiv 1606.00541).

TEST INFRASTRUCTURE ONLY: plain serial FP64 code on CSR matrices (``hec_oracle.c`` plus the
conv3d reference in ``conv_ref.py`` and the learned stage's gated step in ``stage_ref.py``).  Only the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import it.  It shares no code with the CUDA library and does not
import the product package.

Every wrapper below takes and returns numpy arrays; CSR matrices are ``(rowptr, col, val)``
tuples with int32 indices, 0-based, rows sorted by ascending column (Sec. 2).

Parity status of each function (what pins it) is listed in ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hec_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

ERRORS = {-1: "entry on the wrong side of the diagonal", -2: "missing diagonal", -3: "zero pivot",
          -4: "unsorted row or bad column", -5: "bad argument", -6: "out of memory"}


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc -O2 (as the paper's CPU codes were built, Sec. 4)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = ctypes.CDLL(_LIB_PATH)
    return _lib


_i32p = ctypes.POINTER(ctypes.c_int)


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(rc, what):
    if rc < 0:
        raise OracleError("%s: %s (%d)" % (what, ERRORS.get(rc, "error"), rc))
    return rc


def _call(name, *args):
    f = getattr(lib(), name)
    f.restype = ctypes.c_int
    return f(*[_p(a) if isinstance(a, np.ndarray) else a for a in args])


# --- checks and substitution (Eq. 1) --------------------------------------------------------

def check_triangular(A, uplo):
    rp, ci, v = A
    return _call("or_check_triangular", ctypes.c_int(len(rp) - 1), _i32(rp), _i32(ci), _f64(v), ctypes.c_int(uplo))


def lower_solve(L, b):
    rp, ci, v = L
    n = len(rp) - 1
    y = np.zeros(n)
    _check(_call("or_lower_solve", ctypes.c_int(n), _i32(rp), _i32(ci), _f64(v), _f64(b), y), "lower_solve")
    return y


def upper_solve(U, y):
    rp, ci, v = U
    n = len(rp) - 1
    x = np.zeros(n)
    _check(_call("or_upper_solve", ctypes.c_int(n), _i32(rp), _i32(ci), _f64(v), _f64(y), x), "upper_solve")
    return x


# --- levels and map (Eq. 2, Eq. 3; upper factor by reversal) --------------------------------

def levels(T, uplo):
    """Returns (level[n], nlev); level is 0-based (paper level - 1), indexed by original row."""
    rp, ci = T[0], T[1]
    n = len(rp) - 1
    lev = np.zeros(max(n, 1), dtype=np.int32)
    nlev = _check(_call("or_levels", ctypes.c_int(n), _i32(rp), _i32(ci), ctypes.c_int(uplo), lev), "levels")
    return lev[:n], nlev


def level_map(level, nlev, uplo):
    """Returns (perm, iperm, level_ptr): perm[i] = m(i) of Eq. 3 (composite with the reversal
    for the upper factor), iperm its inverse, level_ptr[k] = N_0 + ... + N_{k-1}."""
    n = len(level)
    perm = np.zeros(max(n, 1), dtype=np.int32)
    iperm = np.zeros(max(n, 1), dtype=np.int32)
    lp = np.zeros(nlev + 1, dtype=np.int32)
    _check(_call("or_level_map", ctypes.c_int(n), _i32(level), ctypes.c_int(nlev), ctypes.c_int(uplo), perm, iperm, lp),
           "level_map")
    return perm[:n], iperm[:n], lp


def analyze(T, uplo):
    lev, nlev = levels(T, uplo)
    perm, iperm, lp = level_map(lev, nlev, uplo)
    return dict(level=lev, nlev=nlev, perm=perm, iperm=iperm, level_ptr=lp)


# --- value rounding -------------------------------------------------------------------------

def round_f32_bits(d):
    f = lib().or_round_f32_bits
    f.restype = ctypes.c_uint32
    f.argtypes = [ctypes.c_double]
    return np.array([f(float(x)) for x in np.ravel(d)], dtype=np.uint32)


def round_bf16_bits(d):
    a = np.ascontiguousarray(np.ravel(d), dtype=np.float64)
    out = np.zeros(max(len(a), 1), dtype=np.uint16)
    f = lib().or_round_bf16_array
    f.restype = None
    f(ctypes.c_long(len(a)), _p(a), _p(out))
    return out[:len(a)]


# --- HEC (Sec. 2.1, Alg. 1) -----------------------------------------------------------------

VDT = {"f64": 0, "f32": 1, "bf16": 2}
VDT_NP = {0: np.float64, 1: np.uint32, 2: np.uint16}  # value arrays are returned as raw bits for 32/16


def ell_width_rule(count):
    count = _i32(count)
    return _call("or_ell_width_rule", ctypes.c_int(len(count)), count)


def round_up32(n):
    return (n + 31) // 32 * 32


def hec_pack(T, tri, uplo=0, perm=None, iperm=None, w=-1, vdt="f64"):
    """Alg. 1 steps 3-4 (tri=1) or a plain HEC of a general matrix (tri=0).  Returns a dict with
    n, ld, w, ell_col[w*ld], ell_val[w*ld], tptr[n+1], tcol, tval (values as float64 for f64,
    raw uint32 bits for f32, raw uint16 bits for bf16)."""
    rp, ci, v = _i32(T[0]), _i32(T[1]), _f64(T[2])
    n = len(rp) - 1
    code = VDT[vdt]
    wo = ctypes.c_int(0)
    tn = ctypes.c_long(0)
    f = lib().or_hec_sizes
    f.restype = ctypes.c_int
    _check(f(ctypes.c_int(n), _p(rp), _p(ci), ctypes.c_int(tri), ctypes.c_int(w), ctypes.byref(wo), ctypes.byref(tn)),
           "hec_sizes")
    w = wo.value
    ld = round_up32(n)
    ell_col = np.zeros(max(w * ld, 1), dtype=np.int32)
    ell_val = np.zeros(max(w * ld, 1), dtype=VDT_NP[code])
    tptr = np.zeros(n + 1, dtype=np.int32)
    tcol = np.zeros(max(tn.value, 1), dtype=np.int32)
    tval = np.zeros(max(tn.value, 1), dtype=VDT_NP[code])
    if perm is None:
        perm = np.arange(n, dtype=np.int32)
        iperm = perm
    _check(_call("or_hec_pack", ctypes.c_int(n), rp, ci, v, ctypes.c_int(tri), ctypes.c_int(uplo), _i32(perm),
                 _i32(iperm), ctypes.c_int(w), ctypes.c_int(code), ell_col, ell_val, tptr, tcol, tval), "hec_pack")
    return dict(n=n, ld=ld, w=w, vdt=vdt, ell_col=ell_col[: w * ld], ell_val=ell_val[: w * ld], tptr=tptr,
                tcol=tcol[: tn.value], tval=tval[: tn.value])


def hec_unpack(H, tri, iperm=None):
    n, w = H["n"], H["w"]
    code = VDT[H["vdt"]]
    nnz = int(np.sum(H["ell_col"] >= 0)) + int(H["tptr"][-1])
    rp = np.zeros(n + 1, dtype=np.int32)
    ci = np.zeros(max(nnz, 1), dtype=np.int32)
    v = np.zeros(max(nnz, 1))
    if iperm is None:
        iperm = np.arange(n, dtype=np.int32)
    ev = H["ell_val"] if len(H["ell_val"]) else np.zeros(1, dtype=VDT_NP[code])
    ec = H["ell_col"] if len(H["ell_col"]) else np.zeros(1, dtype=np.int32)
    tc = H["tcol"] if len(H["tcol"]) else np.zeros(1, dtype=np.int32)
    tv = H["tval"] if len(H["tval"]) else np.zeros(1, dtype=VDT_NP[code])
    _check(_call("or_hec_unpack", ctypes.c_int(n), ctypes.c_int(w), _i32(ec), np.ascontiguousarray(ev),
                 _i32(H["tptr"]), _i32(tc), np.ascontiguousarray(tv), ctypes.c_int(tri), _i32(iperm),
                 ctypes.c_int(code), rp, ci, v), "hec_unpack")
    return rp, ci[:nnz], v[:nnz]


# --- SpMV and factorizations (Sec. 3) -------------------------------------------------------

def spmv(A, x):
    rp, ci, v = A
    n = len(rp) - 1
    y = np.zeros(n)
    f = lib().or_spmv
    f.restype = None
    f(ctypes.c_int(n), _p(_i32(rp)), _p(_i32(ci)), _p(_f64(v)), _p(_f64(x)), _p(y))
    return y


def _alloc_lu(n, cap):
    return (np.zeros(n + 1, dtype=np.int32), np.zeros(max(cap, 1), dtype=np.int32), np.zeros(max(cap, 1)),
            np.zeros(n + 1, dtype=np.int32), np.zeros(max(cap, 1), dtype=np.int32), np.zeros(max(cap, 1)))


def _trim(Lrp, Lci, Lv, Urp, Uci, Uv):
    return (Lrp, Lci[: Lrp[-1]], Lv[: Lrp[-1]]), (Urp, Uci[: Urp[-1]], Uv[: Urp[-1]])


def ilu0(A):
    rp, ci, v = _i32(A[0]), _i32(A[1]), _f64(A[2])
    n = len(rp) - 1
    bufs = _alloc_lu(n, int(rp[-1]) + n)
    _check(_call("or_ilu0", ctypes.c_int(n), rp, ci, v, *bufs), "ilu0")
    return _trim(*bufs)


def iluk_pattern(A, k):
    rp, ci = _i32(A[0]), _i32(A[1])
    n = len(rp) - 1
    prp = np.zeros(n + 1, dtype=np.int32)
    f = lib().or_iluk_symbolic
    f.restype = ctypes.c_int
    _check(f(ctypes.c_int(n), _p(rp), _p(ci), ctypes.c_int(k), _p(prp), None), "iluk_symbolic")
    pci = np.zeros(max(int(prp[-1]), 1), dtype=np.int32)
    _check(f(ctypes.c_int(n), _p(rp), _p(ci), ctypes.c_int(k), _p(prp), _p(pci)), "iluk_symbolic")
    return prp, pci[: prp[-1]]


def iluk(A, k):
    rp, ci, v = _i32(A[0]), _i32(A[1]), _f64(A[2])
    n = len(rp) - 1
    prp, pci = iluk_pattern(A, k)
    bufs = _alloc_lu(n, int(prp[-1]) + n)
    _check(_call("or_iluk_numeric", ctypes.c_int(n), rp, ci, v, prp, _i32(pci), *bufs), "iluk_numeric")
    return _trim(*bufs)


def ilut(A, p, tol):
    rp, ci, v = _i32(A[0]), _i32(A[1]), _f64(A[2])
    n = len(rp) - 1
    Lrp = np.zeros(n + 1, dtype=np.int32)
    Urp = np.zeros(n + 1, dtype=np.int32)
    f = lib().or_ilut
    f.restype = ctypes.c_int
    _check(f(ctypes.c_int(n), _p(rp), _p(ci), _p(v), ctypes.c_int(p), ctypes.c_double(tol), _p(Lrp), None, None,
             _p(Urp), None, None), "ilut")
    bufs = (Lrp, np.zeros(max(int(Lrp[-1]), 1), dtype=np.int32), np.zeros(max(int(Lrp[-1]), 1)),
            Urp, np.zeros(max(int(Urp[-1]), 1), dtype=np.int32), np.zeros(max(int(Urp[-1]), 1)))
    _check(f(ctypes.c_int(n), _p(rp), _p(ci), _p(v), ctypes.c_int(p), ctypes.c_double(tol), *[_p(b) for b in bufs]),
           "ilut")
    return _trim(*bufs)


def ilu_apply(L, U, r):
    n = len(L[0]) - 1
    z = np.zeros(n)
    _check(_call("or_ilu_apply", ctypes.c_int(n), _i32(L[0]), _i32(L[1]), _f64(L[2]), _i32(U[0]), _i32(U[1]),
                 _f64(U[2]), _f64(r), z), "ilu_apply")
    return z


# --- RAS (Sec. 3, Eq. 4) --------------------------------------------------------------------

def ras_extend(A, part, ns):
    rp, ci = _i32(A[0]), _i32(A[1])
    n = len(rp) - 1
    ptr = np.zeros(ns + 1, dtype=np.int32)
    f = lib().or_ras_extend
    f.restype = ctypes.c_int
    _check(f(ctypes.c_int(n), _p(rp), _p(ci), _p(_i32(part)), ctypes.c_int(ns), _p(ptr), None), "ras_extend")
    idx = np.zeros(max(int(ptr[-1]), 1), dtype=np.int32)
    _check(f(ctypes.c_int(n), _p(rp), _p(ci), _p(_i32(part)), ctypes.c_int(ns), _p(ptr), _p(idx)), "ras_extend")
    return ptr, idx[: ptr[-1]]


def submatrix(A, idx):
    rp, ci, v = _i32(A[0]), _i32(A[1]), _f64(A[2])
    n = len(rp) - 1
    m = len(idx)
    cap = int(rp[-1])
    srp = np.zeros(m + 1, dtype=np.int32)
    sci = np.zeros(max(cap, 1), dtype=np.int32)
    sv = np.zeros(max(cap, 1))
    _check(_call("or_submatrix", ctypes.c_int(n), rp, ci, v, ctypes.c_int(m), _i32(idx), srp, sci, sv), "submatrix")
    return srp, sci[: srp[-1]], sv[: srp[-1]]


def block_diag(blocks):
    """Eq. 4: diag(B_1, ..., B_s) of CSR blocks as one CSR matrix."""
    rps, cis, vs = [np.zeros(1, dtype=np.int64)], [], []
    off_r, off_nnz = 0, 0
    for rp, ci, v in blocks:
        rps.append(np.asarray(rp[1:], dtype=np.int64) + off_nnz)
        cis.append(np.asarray(ci, dtype=np.int64) + off_r)
        vs.append(np.asarray(v, dtype=np.float64))
        off_r += len(rp) - 1
        off_nnz += int(rp[-1])
    return (np.concatenate(rps).astype(np.int32), np.concatenate(cis).astype(np.int32) if cis else np.zeros(0, np.int32),
            np.concatenate(vs) if vs else np.zeros(0))


def owned_sets(part, ns):
    """Subdomains without overlap: ext(s) = {i : part[i] = s} in ascending order."""
    part = _i32(part)
    idx = np.concatenate([np.flatnonzero(part == s) for s in range(ns)]).astype(np.int32)
    ptr = np.zeros(ns + 1, dtype=np.int32)
    ptr[1:] = np.cumsum(np.bincount(part, minlength=ns))
    return ptr, idx


def ras_setup(A, part, ns, overlap=1):
    """Extended subdomains (overlap 1; overlap 0 keeps the owned rows: block ILU), A_s =
    A[ext, ext], ILU(0) of each, assembled as one block-diagonal pair of factors (Eq. 4)."""
    ptr, idx = ras_extend(A, part, ns) if overlap else owned_sets(part, ns)
    Ls, Us = [], []
    for s in range(ns):
        As = submatrix(A, idx[ptr[s]:ptr[s + 1]])
        L, U = ilu0(As)
        Ls.append(L)
        Us.append(U)
    return dict(ext_ptr=ptr, ext_idx=idx, part=_i32(part), ns=ns, L=block_diag(Ls), U=block_diag(Us))


def ras_apply(R, v):
    n = len(R["part"])
    z = np.zeros(n)
    L, U = R["L"], R["U"]
    _check(_call("or_ras_apply", ctypes.c_int(n), ctypes.c_int(R["ns"]), R["ext_ptr"], R["ext_idx"], R["part"],
                 _i32(L[0]), _i32(L[1]), _f64(L[2]), _i32(U[0]), _i32(U[1]), _f64(U[2]), _f64(v), z), "ras_apply")
    return z


# --- Gauss-Seidel smoother (Sec. 1: the smoother use of triangular solves) -----------------------

def sgs(A, b, x0, sweeps=1):
    """Symmetric Gauss-Seidel, written from its definition: a forward sweep updates x_i, i = 0..n-1,
    to (b_i - sum_{j != i} a_ij x_j) / a_ii with the newest values, then a backward sweep does the
    same for i = n-1..0.  Plain loops (small cases only)."""
    rp, ci, v = _i32(A[0]), _i32(A[1]), _f64(A[2])
    n = len(rp) - 1
    x = _f64(x0).copy()
    b = _f64(b)
    for _ in range(sweeps):
        for order in (range(n), range(n - 1, -1, -1)):
            for i in order:
                s = b[i]
                d = 0.0
                for p in range(rp[i], rp[i + 1]):
                    j = ci[p]
                    if j == i:
                        d = v[p]
                    else:
                        s -= v[p] * x[j]
                x[i] = s / d
    return x


# --- FGMRES ---------------------------------------------------------------------------------

def _fgmres_out(rc, x, info, hist):
    its = int(info[0])
    return dict(x=x, converged=(rc == 0), iters=its, relres=float(info[1]), restarts=int(info[2]),
                history=hist[: its + 1].copy())


def fgmres(A, b, M=None, m=30, rtol=1e-8, max_iters=1000, x0=None):
    """Right-preconditioned FGMRES(m) from x0 (default 0).  M: None (no preconditioner),
    ('ilu', L, U) or ('ras', R)."""
    rp, ci, v = _i32(A[0]), _i32(A[1]), _f64(A[2])
    n = len(rp) - 1
    x = np.zeros(n) if x0 is None else _f64(x0).copy()
    info = np.zeros(3)
    hist = np.zeros(max_iters + 1)
    b = _f64(b)
    ci_ = (ctypes.c_int(m), ctypes.c_double(rtol), ctypes.c_int(max_iters))
    if M is None:
        rc = _call("or_fgmres_identity", ctypes.c_int(n), rp, ci, v, b, x, *ci_, info, hist)
    elif M[0] == "ilu":
        L, U = M[1], M[2]
        rc = _call("or_fgmres_ilu", ctypes.c_int(n), rp, ci, v, _i32(L[0]), _i32(L[1]), _f64(L[2]), _i32(U[0]),
                   _i32(U[1]), _f64(U[2]), b, x, *ci_, info, hist)
    elif M[0] == "ras":
        R = M[1]
        L, U = R["L"], R["U"]
        rc = _call("or_fgmres_ras", ctypes.c_int(n), rp, ci, v, ctypes.c_int(R["ns"]), R["ext_ptr"], R["ext_idx"],
                   R["part"], _i32(L[0]), _i32(L[1]), _f64(L[2]), _i32(U[0]), _i32(U[1]), _f64(U[2]), b, x, *ci_,
                   info, hist)
    else:
        raise ValueError(M[0])
    _check(rc, "fgmres")
    return _fgmres_out(rc, x, info, hist)
