"""A-priori error bounds for reduced-precision triangular sweeps, evaluated with the oracle.

A sweep with FP32 or BF16 factor values stores each value rounded once (checked bit for bit
elsewhere) and computes in FP32: the right-hand side rounded to FP32, one fused multiply-add per
off-diagonal entry, then a multiply by the FP32-rounded reciprocal of the diagonal.  A row with q
stored entries (diagonal included) therefore sees at most q + 2 roundings, and the standard
componentwise backward-error argument for substitution (Higham, Accuracy and Stability of
Numerical Algorithms, ch. 8) bounds the computed x^ against the exact solution x of the SAME
rounded factor T by

    |x^ - x| <= gamma_{q+2}(u) M(T)^-1 |T| |x|,     gamma_m(u) = m u / (1 - m u),  u = 2^-24,

with M(T) the comparison matrix (|diagonal|, -|off-diagonals|).  The right-hand side is one more
oracle substitution with M(T).  For z = U^-1 L^-1 r the lower sweep's error passes through U^-1,
and |U^-1| <= M(U)^-1 for a triangular matrix, so the bound of the apply is
bound_U(z) + M(U)^-1 bound_L(y).
"""
import numpy as np

import oracle

U32 = 2.0 ** -24


def rounded(T, vdt):
    """The factor with its values rounded as the library stores them (FP64 widening of the FP32
    or BF16 value)."""
    rp, ci, v = T
    if vdt == "f64":
        return T
    if vdt == "f32":
        return rp, ci, v.astype(np.float32).astype(np.float64)
    bits = oracle.round_bf16_bits(v).astype(np.uint32) << 16
    return rp, ci, bits.view(np.float32).astype(np.float64)


def _solve(T, uplo, b):
    return (oracle.lower_solve if uplo == 0 else oracle.upper_solve)(T, b)


def comparison(T):
    rp, ci, v = T
    n = len(rp) - 1
    diag = ci == np.repeat(np.arange(n), np.diff(rp))
    return rp, ci, np.where(diag, np.abs(v), -np.abs(v))


def gamma(T, u=U32):
    q = int(np.max(np.diff(T[0]))) + 2
    return q * u / (1.0 - q * u)


def sweep_bound(Tr, uplo, x, u=U32):
    """gamma_{q+2}(u) M(T)^-1 |T| |x| for the rounded factor Tr and its exact solution x."""
    rp, ci, v = Tr
    rhs = oracle.spmv((rp, ci, np.abs(v)), np.abs(x))
    return gamma(Tr, u) * _solve(comparison(Tr), uplo, rhs)


def apply_bound(Lr, Ur, y, z, u=U32):
    """Bound of z^ - U^-1 L^-1 r for the rounded factors (y = L^-1 r, z = U^-1 y exact)."""
    return sweep_bound(Ur, 1, z, u) + _solve(comparison(Ur), 1, sweep_bound(Lr, 0, y, u))
