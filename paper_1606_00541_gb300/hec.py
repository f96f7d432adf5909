"""Python binding of libhec (argument marshalling only: every step runs in the CUDA library).

Names follow the C ABI in include/hec.h.  Device arrays are torch CUDA tensors (int32 indices,
float64 values); streams default to torch's current stream.  Importing this module loads
libhec.so and raises ImportError when it is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhec.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("libhec.so is not built (run paper_1606_00541_gb300.build.build() or __graft_entry__.build())")
_lib = ctypes.CDLL(LIB_PATH)

OK, INVALID_ARG, UNSORTED, NOT_TRIANGULAR, MISSING_DIAG, ZERO_PIVOT, OOM, CUDA, TIMEOUT, NOT_CONVERGED, OUT_OF_BOUNDS = range(11)
STATUS_NAMES = ["OK", "INVALID_ARG", "UNSORTED", "NOT_TRIANGULAR", "MISSING_DIAG", "ZERO_PIVOT", "OOM", "CUDA",
                "TIMEOUT", "NOT_CONVERGED", "OUT_OF_BOUNDS"]
DTYPES = {"f64": 0, "f32": 1, "bf16": 2}


class HecError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = _lib.hec_last_error().decode()
        super().__init__("%s: %s (%s)" % (where, STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status, msg))


_vp = ctypes.c_void_p
_i = ctypes.c_int
_d = ctypes.c_double
_ll = ctypes.c_longlong


class HecMatrixInfo(ctypes.Structure):
    _fields_ = [("n", _i), ("ld", _i), ("w", _i), ("tri", _i), ("uplo", _i), ("vdt", _i), ("tail_nnz", _ll),
                ("ell_col", _vp), ("ell_val", _vp), ("tptr", _vp), ("tcol", _vp), ("tval", _vp)]


class HecTune(ctypes.Structure):
    _fields_ = [("block_threads", _i), ("blocks_per_sm", _i), ("wait_cycles", _ll), ("debug_unpublished_row", _i),
                ("backoff_ns", _i), ("lanes_per_row", _i), ("partitioned", _i)]


class HecFgmresInfo(ctypes.Structure):
    _fields_ = [("iterations", _i), ("restarts", _i), ("converged", _i), ("rel_residual", _d), ("seconds", _d),
                ("reorthogonalized", _i)]


def _sig(name, *args):
    f = getattr(_lib, name)
    f.restype = _i
    f.argtypes = list(args)
    return f


_lib.hec_last_error.restype = ctypes.c_char_p
_lib.hec_version.restype = _i
_lib.hec_launch_count.restype = _ll
_sptrsv_analyze = _sig("sptrsv_analyze", _i, _vp, _vp, _i, ctypes.POINTER(_vp), _vp)
_hec_levels_get = _sig("hec_levels_get", _vp, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_i),
                       ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_vp))
_hec_levels_destroy = _sig("hec_levels_destroy", _vp)
_hec_from_csr = _sig("hec_from_csr", _i, _vp, _vp, _vp, _vp, _i, _i, ctypes.POINTER(_vp), _vp)
_hec_matrix_get = _sig("hec_matrix_get", _vp, ctypes.POINTER(HecMatrixInfo))
_hec_to_csr = _sig("hec_to_csr", _vp, _vp, _vp, _vp, _vp, _vp)
_hec_matrix_destroy = _sig("hec_matrix_destroy", _vp)
_sptrsv_plan_create = _sig("sptrsv_plan_create", _vp, _vp, _i, ctypes.POINTER(HecTune), ctypes.POINTER(_vp))
_sptrsv_plan_destroy = _sig("sptrsv_plan_destroy", _vp)
_sptrsv_lower = _sig("sptrsv_lower", _vp, _i, _vp, _i, _vp, _i, _vp)
_sptrsv_upper = _sig("sptrsv_upper", _vp, _i, _vp, _i, _vp, _i, _vp)
_hec_sync_status = _sig("hec_sync_status", _vp, _vp)
_ilu_create = _sig("ilu_create", _vp, _vp, _i, _i, _vp, _vp, ctypes.POINTER(_vp))
_ilu_destroy = _sig("ilu_destroy", _vp)
_ilu_apply = _sig("ilu_apply", _vp, _i, _vp, _i, _vp, _i, _vp)
_spmv = _sig("spmv", _vp, _i, _d, _vp, _i, _d, _vp, _i, _vp)
_fgmres_solve = _sig("fgmres_solve", _vp, _vp, _vp, _i, _vp, _i, _vp, _i, _i, _d, _i, ctypes.POINTER(HecFgmresInfo),
                     _vp)
_hec_csr_get = _sig("hec_csr_get", _vp, ctypes.POINTER(_i), ctypes.POINTER(_ll), ctypes.POINTER(_vp),
                    ctypes.POINTER(_vp), ctypes.POINTER(_vp))
_hec_csr_destroy = _sig("hec_csr_destroy", _vp)
_ilu_factor = _sig("ilu_factor", _i, _vp, _vp, _vp, _i, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _vp)


def _check(st, where):
    if st != OK:
        raise HecError(st, where)


def _stream(stream):
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def _ld(t, nrhs):
    return nrhs if t.dim() == 1 else t.stride(0)


def _nrhs(t):
    return 1 if t.dim() == 1 else t.shape[1]


_hec_profile_enable = _sig("hec_profile_enable", _i)
_hec_profile_enable_categories = _sig("hec_profile_enable_categories", ctypes.c_uint)
_hec_profile_read = _sig("hec_profile_read", ctypes.POINTER(_d), ctypes.POINTER(_ll), _i)


def profile_enable(on=True, categories=None):
    """Kernel timing by category (include/hec.h): all categories, or only those listed
    (0 sweeps, 1 SpMV, 2 Gram-Schmidt, 3 Arnoldi, 4 vector kernels, 5 sentinel fills)."""
    if categories is None or not on:
        _check(_hec_profile_enable(1 if on else 0), "hec_profile_enable")
    else:
        _check(_hec_profile_enable_categories(sum(1 << int(c) for c in categories)), "hec_profile_enable_categories")


_hec_profile_read_category = _sig("hec_profile_read_category", _i, ctypes.POINTER(_d), ctypes.POINTER(_ll))
PROFILE_CATEGORIES = ["sweep", "spmv", "gram_schmidt", "arnoldi", "vector", "fill"]


def profile_read(reset=True):
    """(summed device ms, launches) of the sweep kernels recorded since the last reset."""
    ms, n = _d(), _ll()
    _check(_hec_profile_read(ctypes.byref(ms), ctypes.byref(n), 1 if reset else 0), "hec_profile_read")
    return ms.value, n.value


def profile_breakdown():
    """{category: (device ms, launches)} recorded since the last reset (read before profile_read)."""
    out = {}
    for i, name in enumerate(PROFILE_CATEGORIES):
        ms, n = _d(), _ll()
        _check(_hec_profile_read_category(i, ctypes.byref(ms), ctypes.byref(n)), "hec_profile_read_category")
        out[name] = (ms.value, n.value)
    return out


def version():
    return _lib.hec_version()


def launch_count():
    """Kernel launches the library has issued in this process."""
    return _lib.hec_launch_count()


def library_path():
    return LIB_PATH


_lib.hec_release_cached_memory.restype = ctypes.c_size_t


def release_cached_memory():
    """Returns the device blocks the library keeps for reuse to the CUDA runtime; the number of
    bytes returned (hec_release_cached_memory)."""
    return int(_lib.hec_release_cached_memory())


GS_CLASSICAL, GS_MODIFIED = 0, 1
_hec_set_gram_schmidt = _sig("hec_set_gram_schmidt", _i)


def set_gram_schmidt(mode):
    """Gram-Schmidt variant of fgmres_solve's Arnoldi step, process-wide: "classical" (with
    selective reorthogonalization, the default) or "modified" (hec_set_gram_schmidt)."""
    code = {"classical": GS_CLASSICAL, "modified": GS_MODIFIED}[mode]
    _check(_hec_set_gram_schmidt(code), "hec_set_gram_schmidt")


def get_gram_schmidt():
    return {GS_CLASSICAL: "classical", GS_MODIFIED: "modified"}[_lib.hec_get_gram_schmidt()]


class _DevArray:
    """Borrowed device array exposed through __cuda_array_interface__ (for torch.as_tensor)."""

    def __init__(self, ptr, n, typestr, owner):
        self._owner = owner
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr or 0, False), "version": 3,
                                         "strides": None}


def _view(ptr, n, dtype, owner):
    typestr = {torch.int32: "<i4", torch.float64: "<f8", torch.float32: "<f4", torch.int16: "<i2"}[dtype]
    if n == 0:
        return torch.zeros(0, dtype=dtype, device="cuda")
    return torch.as_tensor(_DevArray(ptr, n, typestr, owner), device="cuda")


class _Handle:
    _destroy = None

    def __init__(self, h, keep=()):
        self.h = h
        self._keep = keep  # objects this handle borrows from

    def close(self):
        if self.h:
            type(self)._destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def _as_parameter_(self):
        return self.h


class Levels(_Handle):
    _destroy = staticmethod(_hec_levels_destroy)

    def _get(self):
        n, nlev, uplo = _i(), _i(), _i()
        p = [_vp() for _ in range(4)]
        _check(_hec_levels_get(self.h, ctypes.byref(n), ctypes.byref(nlev), ctypes.byref(uplo), *[ctypes.byref(x) for x in p]),
               "hec_levels_get")
        return n.value, nlev.value, uplo.value, [x.value for x in p]

    @property
    def n(self):
        return self._get()[0]

    @property
    def nlev(self):
        return self._get()[1]

    @property
    def uplo(self):
        return self._get()[2]

    def arrays(self):
        """Copies of (level, perm, iperm, level_ptr) as torch int32 CUDA tensors."""
        n, nlev, _, (lev, perm, iperm, lp) = self._get()
        return (_view(lev, n, torch.int32, self).clone(), _view(perm, n, torch.int32, self).clone(),
                _view(iperm, n, torch.int32, self).clone(), _view(lp, nlev + 1, torch.int32, self).clone())


class Matrix(_Handle):
    _destroy = staticmethod(_hec_matrix_destroy)

    def info(self):
        inf = HecMatrixInfo()
        _check(_hec_matrix_get(self.h, ctypes.byref(inf)), "hec_matrix_get")
        return inf

    def arrays(self):
        """Copies of the HEC arrays: dict(n, ld, w, ell_col, ell_val, tptr, tcol, tval); f32 and bf16
        values are returned as their raw int32 / int16 bit patterns."""
        inf = self.info()
        vdt = inf.vdt
        vt = {0: torch.float64, 1: torch.int32, 2: torch.int16}[vdt]
        wl = inf.w * inf.ld
        return dict(n=inf.n, ld=inf.ld, w=inf.w, tri=inf.tri, uplo=inf.uplo, vdt=["f64", "f32", "bf16"][vdt],
                    ell_col=_view(inf.ell_col, wl, torch.int32, self).clone(),
                    ell_val=_view(inf.ell_val, wl, vt, self).clone(),
                    tptr=_view(inf.tptr, inf.n + 1, torch.int32, self).clone(),
                    tcol=_view(inf.tcol, inf.tail_nnz, torch.int32, self).clone(),
                    tval=_view(inf.tval, inf.tail_nnz, vt, self).clone())


class Plan(_Handle):
    _destroy = staticmethod(_sptrsv_plan_destroy)


class Precond(_Handle):
    _destroy = staticmethod(_ilu_destroy)


class Csr(_Handle):
    _destroy = staticmethod(_hec_csr_destroy)

    def tensors(self):
        n, nnz = _i(), _ll()
        p = [_vp() for _ in range(3)]
        _check(_hec_csr_get(self.h, ctypes.byref(n), ctypes.byref(nnz), *[ctypes.byref(x) for x in p]), "hec_csr_get")
        return (_view(p[0].value, n.value + 1, torch.int32, self).clone(),
                _view(p[1].value, nnz.value, torch.int32, self).clone(),
                _view(p[2].value, nnz.value, torch.float64, self).clone())


# --- entry points -----------------------------------------------------------------------------

def sptrsv_analyze(rowptr, col, uplo, stream=None):
    n = rowptr.numel() - 1
    out = _vp()
    _check(_sptrsv_analyze(n, _ptr(rowptr), _ptr(col), int(uplo), ctypes.byref(out), _stream(stream)), "sptrsv_analyze")
    return Levels(out.value)


def hec_from_csr(rowptr, col, val, levels=None, ell_width=-1, vdt="f64", stream=None):
    n = rowptr.numel() - 1
    out = _vp()
    _check(_hec_from_csr(n, _ptr(rowptr), _ptr(col), _ptr(val), levels.h if levels is not None else None, int(ell_width),
                         DTYPES[vdt], ctypes.byref(out), _stream(stream)), "hec_from_csr")
    return Matrix(out.value, keep=(levels,))


def hec_to_csr(matrix, levels=None, stream=None):
    inf = matrix.info()
    n = inf.n
    nnz = int((matrix.arrays()["ell_col"] >= 0).sum().item()) + int(inf.tail_nnz)
    rp = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    ci = torch.zeros(max(nnz, 1), dtype=torch.int32, device="cuda")
    v = torch.zeros(max(nnz, 1), dtype=torch.float64, device="cuda")
    _check(_hec_to_csr(matrix.h, levels.h if levels is not None else None, _ptr(rp), _ptr(ci), _ptr(v), _stream(stream)),
           "hec_to_csr")
    return rp, ci[:nnz], v[:nnz]


def sptrsv_plan_create(matrix, levels, max_nrhs=1, block_threads=0, blocks_per_sm=0, wait_cycles=0,
                       debug_unpublished_row=None, backoff_ns=0, lanes_per_row=0):
    t = HecTune(block_threads, blocks_per_sm, wait_cycles,
                0 if debug_unpublished_row is None else int(debug_unpublished_row) + 1, backoff_ns, lanes_per_row, 0)
    out = _vp()
    _check(_sptrsv_plan_create(matrix.h, levels.h, int(max_nrhs), ctypes.byref(t), ctypes.byref(out)), "sptrsv_plan_create")
    return Plan(out.value, keep=(matrix, levels))


def _solve(fn, name, plan, b, x, stream):
    nrhs = _nrhs(b)
    if x is None:
        x = torch.empty_like(b)
    _check(fn(plan.h, nrhs, _ptr(b), _ld(b, nrhs), _ptr(x), _ld(x, nrhs), _stream(stream)), name)
    return x


_sptrsv_plan_partition = _sig("sptrsv_plan_partition", _vp, _vp, _i, _i, _vp)
_lib.sptrsv_partition_capacity.restype = _i
_lib.sptrsv_partition_capacity.argtypes = [_vp, _i]


def sptrsv_plan_partition(plan, part=None, nparts=0, threads=0, stream=None):
    """Partitioned single-RHS sweeps (include/hec.h): part = CUDA int32 tensor [n] of part ids per
    original row, or None for contiguous row ranges; nparts = 0 removes the partition."""
    _check(_sptrsv_plan_partition(plan.h, _ptr(part) if part is not None else None, int(nparts), int(threads),
                                  _stream(stream)), "sptrsv_plan_partition")
    plan._part = part


def sptrsv_partition_capacity(plan, threads=0):
    return _lib.sptrsv_partition_capacity(plan.h, int(threads))


_sptrsv_autotune = _sig("sptrsv_autotune", _vp, _i, ctypes.POINTER(HecTune), _vp)


def sptrsv_autotune(plan, nrhs=1, stream=None):
    """Times the plan's sweep over candidate launch shapes and keeps the fastest; returns it."""
    t = HecTune()
    _check(_sptrsv_autotune(plan.h, int(nrhs), ctypes.byref(t), _stream(stream)), "sptrsv_autotune")
    return dict(block_threads=t.block_threads, blocks_per_sm=t.blocks_per_sm, lanes_per_row=t.lanes_per_row,
                partitioned=bool(t.partitioned))


def sptrsv_lower(plan, b, x=None, stream=None):
    return _solve(_sptrsv_lower, "sptrsv_lower", plan, b, x, stream)


def sptrsv_upper(plan, b, x=None, stream=None):
    return _solve(_sptrsv_upper, "sptrsv_upper", plan, b, x, stream)


_sptrsv_plan_check = _sig("sptrsv_plan_check", _vp, _vp)


def sptrsv_plan_check(plan, stream=None):
    """Device-side check of every index the sweeps follow (include/hec.h); raises HecError
    (OUT_OF_BOUNDS) naming the first failing check."""
    _check(_sptrsv_plan_check(plan.h, _stream(stream)), "sptrsv_plan_check")


def hec_sync_status(plan, stream=None):
    return _hec_sync_status(plan.h, _stream(stream))


def ilu_create(Lplan, Uplan, n_glob=None, ext2glob=None, owned=None):
    n_ext = Lplan and Lplan._keep[0].info().n
    if n_glob is None:
        n_glob = n_ext
    out = _vp()
    _check(_ilu_create(Lplan.h, Uplan.h, int(n_glob), int(n_ext), _ptr(ext2glob), _ptr(owned), ctypes.byref(out)),
           "ilu_create")
    return Precond(out.value, keep=(Lplan, Uplan, ext2glob, owned))


def ilu_apply(M, r, z=None, stream=None):
    nrhs = _nrhs(r)
    if z is None:
        z = torch.empty_like(r)
    _check(_ilu_apply(M.h, nrhs, _ptr(r), _ld(r, nrhs), _ptr(z), _ld(z, nrhs), _stream(stream)), "ilu_apply")
    return z


def spmv(A, x, y=None, alpha=1.0, beta=0.0, stream=None):
    nrhs = _nrhs(x)
    if y is None:
        y = torch.zeros_like(x)
    _check(_spmv(A.h, nrhs, float(alpha), _ptr(x), _ld(x, nrhs), float(beta), _ptr(y), _ld(y, nrhs), _stream(stream)),
           "spmv")
    return y


def fgmres_solve(A, M, b, x=None, restart=30, rtol=1e-8, max_iters=1000, stream=None, raise_on_nonconvergence=True,
                 stage=None):
    nrhs = _nrhs(b)
    if x is None:
        x = torch.zeros_like(b)
    info = HecFgmresInfo()
    st = _fgmres_solve(A.h, M.h if M is not None else None, stage.h if stage is not None else None, nrhs, _ptr(b),
                       _ld(b, nrhs), _ptr(x), _ld(x, nrhs), int(restart), float(rtol), int(max_iters),
                       ctypes.byref(info), _stream(stream))
    if st != OK and not (st == NOT_CONVERGED and not raise_on_nonconvergence):
        raise HecError(st, "fgmres_solve")
    return x, dict(iterations=info.iterations, restarts=info.restarts, converged=bool(info.converged),
                   rel_residual=info.rel_residual, seconds=info.seconds, reorthogonalized=info.reorthogonalized)


def ilu_factor(rowptr, col, val, k=0, stream=None):
    n = rowptr.numel() - 1
    L, U = _vp(), _vp()
    _check(_ilu_factor(n, _ptr(rowptr), _ptr(col), _ptr(val), int(k), ctypes.byref(L), ctypes.byref(U), _stream(stream)),
           "ilu_factor")
    return Csr(L.value), Csr(U.value)


_ilut_factor = _sig("ilut_factor", _i, _vp, _vp, _vp, _i, _d, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _vp)


def ilut_factor(rowptr, col, val, p=10, tol=1e-3, stream=None):
    """ILUT(p, tol) of a device CSR matrix (rows ascending) on the GPU; returns (L, U) handles."""
    n = rowptr.numel() - 1
    L, U = _vp(), _vp()
    _check(_ilut_factor(n, _ptr(rowptr), _ptr(col), _ptr(val), int(p), float(tol), ctypes.byref(L), ctypes.byref(U),
                        _stream(stream)), "ilut_factor")
    return Csr(L.value), Csr(U.value)


_csr_triangle = _sig("csr_triangle", _i, _vp, _vp, _vp, _i, _i, ctypes.POINTER(_vp), _vp)


def csr_triangle(rowptr, col, val, uplo, strict=False, stream=None):
    """Lower (uplo 0) or upper (uplo 1) triangle of a device CSR matrix, without the diagonal
    when strict (csr_triangle)."""
    n = rowptr.numel() - 1
    out = _vp()
    _check(_csr_triangle(n, _ptr(rowptr), _ptr(col), _ptr(val), int(uplo), 1 if strict else 0, ctypes.byref(out),
                         _stream(stream)), "csr_triangle")
    return Csr(out.value)


_sgs_create = _sig("sgs_create", _i, _vp, _vp, _vp, _i, _i, ctypes.POINTER(_vp), _vp)
_sgs_smooth = _sig("sgs_smooth", _vp, _i, _vp, _i, _vp, _i, _i, _vp)
_sgs_sync_status = _sig("sgs_sync_status", _vp, _vp)
_sgs_destroy = _sig("sgs_destroy", _vp)


class SgsSmoother(_Handle):
    """Symmetric Gauss-Seidel on the level-scheduled sweeps (sgs_create / sgs_smooth, include/hec.h):
    a forward sweep solves (D + L) x' = b - U_s x, a backward sweep (D + U) x'' = b - L_s x'."""
    _destroy = staticmethod(_sgs_destroy)

    def __init__(self, A, vdt="f64", max_nrhs=1, stream=None):
        n = A[0].numel() - 1
        out = _vp()
        _check(_sgs_create(n, _ptr(A[0]), _ptr(A[1]), _ptr(A[2]), DTYPES[vdt], int(max_nrhs), ctypes.byref(out),
                           _stream(stream)), "sgs_create")
        super().__init__(out.value)

    def smooth(self, x, b, sweeps=1, stream=None):
        """`sweeps` symmetric Gauss-Seidel sweeps from x (device FP64 [n] or [n, k]); returns the
        new iterate (x is not modified)."""
        y = x.clone()
        nrhs = _nrhs(b)
        _check(_sgs_smooth(self.h, nrhs, _ptr(b), _ld(b, nrhs), _ptr(y), _ld(y, nrhs), int(sweeps), _stream(stream)),
               "sgs_smooth")
        return y

    def sync_status(self, stream=None):
        return _sgs_sync_status(self.h, _stream(stream))


_lib.net_param_count.restype = _i
_net_create = _sig("net_create", _vp, ctypes.POINTER(_vp))
_net_destroy = _sig("net_destroy", _vp)
_net_get_params = _sig("net_get_params", _vp, _vp, _vp)
_net_set_params = _sig("net_set_params", _vp, _vp)
_net_forward = _sig("net_forward", _vp, _i, _i, _i, _i, _vp, _vp, _vp, _vp)
_net_train_step = _sig("net_train_step", _vp, _i, _i, _i, _i, _vp, _vp, ctypes.c_float, _i,
                       ctypes.POINTER(ctypes.c_float), _vp)
_net_backward = _sig("net_backward", _vp, _i, _i, _i, _i, _vp, _vp, ctypes.POINTER(ctypes.c_float), _vp)
_net_adam_step = _sig("net_adam_step", _vp, ctypes.c_float, _vp)
_net_set_engine = _sig("net_set_engine", _vp, _i)
_net_sync_status = _sig("net_sync_status", _vp, _vp)
_stage_create = _sig("stage_create", _vp, _vp, _i, _i, _i, _vp, _d, _d, ctypes.POINTER(_vp))
_stage_stats = _sig("stage_stats", _vp, ctypes.POINTER(_i), ctypes.POINTER(_i), _i)
_stage_apply = _sig("stage_apply", _vp, _vp, _vp, _vp)
_stage_destroy = _sig("stage_destroy", _vp)


def net_param_count():
    return _lib.net_param_count()


class Net(_Handle):
    """The correction network (include/hec.h, learned stage).  params: numpy float32 array."""
    _destroy = staticmethod(_net_destroy)

    def __init__(self, params):
        import numpy as np
        p = np.ascontiguousarray(params, dtype=np.float32)
        assert p.size == net_param_count()
        out = _vp()
        _check(_net_create(p.ctypes.data_as(_vp), ctypes.byref(out)), "net_create")
        super().__init__(out.value)

    def params(self, grads=False):
        import numpy as np
        p = np.zeros(net_param_count(), dtype=np.float32)
        g = np.zeros_like(p)
        _check(_net_get_params(self.h, p.ctypes.data_as(_vp), g.ctypes.data_as(_vp)), "net_get_params")
        return (p, g) if grads else p

    def set_params(self, params):
        import numpy as np
        p = np.ascontiguousarray(params, dtype=np.float32)
        _check(_net_set_params(self.h, p.ctypes.data_as(_vp)), "net_set_params")

    def forward(self, x_in, dims, zs=None, acts=False, stream=None):
        """x_in: CUDA bfloat16 tensor [nvox, 16]; dims = (nx, ny, nz).  Returns the FP32 output
        [nvox] (and the BF16 layer outputs [4, nvox, 16] when acts)."""
        nx, ny, nz = dims
        nvox = nx * ny * nz
        out = torch.empty(nvox, dtype=torch.float32, device="cuda")
        a = torch.empty(4, nvox, 16, dtype=torch.bfloat16, device="cuda") if acts else None
        _check(_net_forward(self.h, nx, ny, nz, zs or nz, _ptr(x_in), _ptr(a) if acts else None, _ptr(out),
                            _stream(stream)), "net_forward")
        return (out, a) if acts else out

    def train_step(self, x_in, target, dims, zs=None, lr=1e-3, update=True, stream=None):
        nx, ny, nz = dims
        loss = ctypes.c_float()
        _check(_net_train_step(self.h, nx, ny, nz, zs or nz, _ptr(x_in), _ptr(target), float(lr), 1 if update else 0,
                               ctypes.byref(loss), _stream(stream)), "net_train_step")
        return loss.value

    def backward(self, x_in, target, dims, zs=None, stream=None):
        """Forward, loss and backward on one minibatch (net_backward); returns the loss."""
        nx, ny, nz = dims
        loss = ctypes.c_float()
        _check(_net_backward(self.h, nx, ny, nz, zs or nz, _ptr(x_in), _ptr(target), ctypes.byref(loss),
                             _stream(stream)), "net_backward")
        return loss.value

    def adam_step(self, lr=1e-3, stream=None):
        """One Adam step from the gradients of the last backward pass (net_adam_step)."""
        _check(_net_adam_step(self.h, float(lr), _stream(stream)), "net_adam_step")

    def set_engine(self, tensor_cores=True):
        """Forward layers 1-3 on tcgen05 (True, the default) or on mma.sync (net_set_engine)."""
        _check(_net_set_engine(self.h, 1 if tensor_cores else 0), "net_set_engine")

    def sync_status(self, stream=None):
        """Raises HecError(TIMEOUT) when a tcgen05 convolution gave up waiting (net_sync_status)."""
        _check(_net_sync_status(self.h, _stream(stream)), "net_sync_status")


class Stage(_Handle):
    """Learned correction stage for fgmres_solve (include/hec.h)."""
    _destroy = staticmethod(_stage_destroy)

    def __init__(self, net, A, dims, aux, aux_scale=0.5, rho=0.99):
        out = _vp()
        nx, ny, nz = dims
        _check(_stage_create(net.h, A.h, nx, ny, nz, _ptr(aux), float(aux_scale), float(rho), ctypes.byref(out)),
               "stage_create")
        super().__init__(out.value, keep=(net, A))

    def stats(self, reset=False):
        a, b = _i(), _i()
        _check(_stage_stats(self.h, ctypes.byref(a), ctypes.byref(b), 1 if reset else 0), "stage_stats")
        return dict(applied=a.value, accepted=b.value)

    def apply(self, v, z1, stream=None):
        """z = z1 + alpha c or z1 (see stage_apply); v, z1 device FP64 [n]; z1 is left unchanged."""
        z = z1.clone()
        _check(_stage_apply(self.h, _ptr(v), _ptr(z), _stream(stream)), "stage_apply")
        return z


_ras_setup = _sig("ras_setup", _i, _vp, _vp, _vp, _vp, _i, ctypes.POINTER(_vp), _vp)
_ras_setup_overlap = _sig("ras_setup_overlap", _i, _vp, _vp, _vp, _vp, _i, _i, ctypes.POINTER(_vp), _vp)
_hec_ras_get = _sig("hec_ras_get", _vp, ctypes.POINTER(_i), ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                    ctypes.POINTER(_vp), ctypes.POINTER(_vp))
_hec_ras_destroy = _sig("hec_ras_destroy", _vp)


class Ras(_Handle):
    """RAS subdomain system built by ras_setup (Sec. 3, Eq. 4)."""
    _destroy = staticmethod(_hec_ras_destroy)

    def _get(self):
        ne = _i()
        p = [_vp() for _ in range(4)]
        _check(_hec_ras_get(self.h, ctypes.byref(ne), *[ctypes.byref(x) for x in p]), "hec_ras_get")
        return ne.value, [x.value for x in p]

    @property
    def n_ext(self):
        return self._get()[0]

    def tensors(self, nsub):
        """(ext_ptr, ext2glob, owned (uint8), A_ext CSR tensors), device copies."""
        ne, (ep, e2g, own, aext) = self._get()
        n, nnz = _i(), _ll()
        q = [_vp() for _ in range(3)]
        _check(_hec_csr_get(aext, ctypes.byref(n), ctypes.byref(nnz), *[ctypes.byref(x) for x in q]), "hec_csr_get")
        owned = torch.as_tensor(_DevArray(own, ne, "|u1", self), device="cuda").clone() if ne else \
            torch.zeros(0, dtype=torch.uint8, device="cuda")
        return (_view(ep, nsub + 1, torch.int32, self).clone(), _view(e2g, ne, torch.int32, self).clone(), owned,
                (_view(q[0].value, n.value + 1, torch.int32, self).clone(),
                 _view(q[1].value, nnz.value, torch.int32, self).clone(),
                 _view(q[2].value, nnz.value, torch.float64, self).clone()))


def ras_setup(rowptr, col, val, part, nsub, stream=None, overlap=1):
    """Subdomain system (ras_setup_overlap): overlap 1 = RAS, overlap 0 = block ILU."""
    n = rowptr.numel() - 1
    out = _vp()
    _check(_ras_setup_overlap(n, _ptr(rowptr), _ptr(col), _ptr(val), _ptr(part), int(nsub), int(overlap),
                              ctypes.byref(out), _stream(stream)), "ras_setup_overlap")
    return Ras(out.value)


# --- convenience: a full ILU solver assembled from the entry points ------------------------------

class IluSolver:
    """A ready-to-use preconditioned solver: levels, HEC factors, plans and the preconditioner for
    given device CSR factors L, U (and optionally the matrix A for FGMRES)."""

    def __init__(self, L, U, A=None, vdt="f64", max_nrhs=1, stream=None, **tune):
        self.lvL = sptrsv_analyze(L[0], L[1], 0, stream)
        self.lvU = sptrsv_analyze(U[0], U[1], 1, stream)
        self.HL = hec_from_csr(*L, levels=self.lvL, vdt=vdt, stream=stream)
        self.HU = hec_from_csr(*U, levels=self.lvU, vdt=vdt, stream=stream)
        self.pL = sptrsv_plan_create(self.HL, self.lvL, max_nrhs, **tune)
        self.pU = sptrsv_plan_create(self.HU, self.lvU, max_nrhs, **tune)
        self.M = ilu_create(self.pL, self.pU)
        self.A = hec_from_csr(*A, vdt="f64", stream=stream) if A is not None else None

    def partition(self, part=None, nparts=None, threads=0, stream=None):
        """Partitioned single-RHS sweeps on both factors (default: as many contiguous parts as fit)."""
        if nparts is None:
            nparts = min(sptrsv_partition_capacity(self.pL, threads), sptrsv_partition_capacity(self.pU, threads))
        sptrsv_plan_partition(self.pL, part, nparts, threads, stream)
        sptrsv_plan_partition(self.pU, part, nparts, threads, stream)
        return nparts

    def autotune(self, nrhs=1, stream=None):
        """Runs the sweep autotuner on both plans; returns the chosen launch shapes."""
        return sptrsv_autotune(self.pL, nrhs, stream), sptrsv_autotune(self.pU, nrhs, stream)

    def apply(self, r, z=None, stream=None):
        return ilu_apply(self.M, r, z, stream)

    def solve(self, b, x=None, restart=30, rtol=1e-8, max_iters=1000, stream=None, **kw):
        return fgmres_solve(self.A, self.M, b, x, restart, rtol, max_iters, stream, **kw)


class RasSolver(IluSolver):
    """RAS preconditioner (Sec. 3, Eq. 4): ras_setup on the GPU, ILU(0) of the block-diagonal
    subdomain system, one pair of batched sweeps for all subdomains, restricted write-back.
    Pass `factors=(L, U)` to use given block-diagonal factors instead of the GPU ILU(0), or
    `ilut=(p, tol)` for the GPU ILUT of every block; overlap=0 gives block ILU / block ILUT (the
    paper's BILU and BILUT: block Jacobi with incomplete-factor blocks)."""

    def __init__(self, A, part, nsub, vdt="f32", max_nrhs=1, stream=None, factors=None, overlap=1, ilut=None,
                 **tune):
        self.R = ras_setup(*A, part, nsub, stream, overlap=overlap)
        self.ext_ptr, self.ext2glob, self.owned, self.A_ext = self.R.tensors(nsub)
        if factors is None and ilut is not None:
            Lh, Uh = ilut_factor(*self.A_ext, p=ilut[0], tol=ilut[1], stream=stream)
            L, U = Lh.tensors(), Uh.tensors()
        elif factors is None:
            Lh, Uh = ilu_factor(*self.A_ext, k=0, stream=stream)
            L, U = Lh.tensors(), Uh.tensors()
        else:
            L, U = factors
        self.L, self.U = L, U
        self.lvL = sptrsv_analyze(L[0], L[1], 0, stream)
        self.lvU = sptrsv_analyze(U[0], U[1], 1, stream)
        self.HL = hec_from_csr(*L, levels=self.lvL, vdt=vdt, stream=stream)
        self.HU = hec_from_csr(*U, levels=self.lvU, vdt=vdt, stream=stream)
        self.pL = sptrsv_plan_create(self.HL, self.lvL, max_nrhs, **tune)
        self.pU = sptrsv_plan_create(self.HU, self.lvU, max_nrhs, **tune)
        n = A[0].numel() - 1
        self.M = ilu_create(self.pL, self.pU, n_glob=n, ext2glob=self.ext2glob, owned=self.owned)
        self.A = hec_from_csr(*A, vdt="f64", stream=stream)
