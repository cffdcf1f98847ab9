"""Test infrastructure only: the CPU oracle for the methods of Hedtke's
"Methods of Matrix Multiplication" (arXiv:1106.1347).

``oracle.c`` restates each method from the paper as plain, sequential C; this
module compiles it with gcc (``-O2 -ffp-contract=off -fno-fast-math``) and
exposes numpy wrappers.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import it.  It shares no code with the
``paper_1106_1347_gb300`` package, and neither imports the other.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
CFLAGS = ["-O2", "-std=gnu99", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]

_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_build/liboracle.so (idempotent)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, dp, ip = ctypes.c_int64, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32)
            gemm = [i64, i64, i64, dp, i64, dp, i64, dp, i64]
            lib.oracle_norm_inf.argtypes = [i64, i64, dp, i64]
            lib.oracle_norm_inf.restype = ctypes.c_double
            lib.oracle_multiply_with_scalar.argtypes = [i64, i64, ctypes.c_double, dp, i64, dp, i64]
            for name in ("oracle_naiv_standard", "oracle_naiv_kahan", "oracle_winograd_original",
                         "oracle_dot2_product"):
                getattr(lib, name).argtypes = gemm
                getattr(lib, name).restype = None
            lib.oracle_winograd_terms.argtypes = [i64, i64, i64, dp, i64, dp, i64, dp, dp]
            lib.oracle_winograd_scaled.argtypes = gemm
            lib.oracle_winograd_scaled.restype = ctypes.c_int
            lib.oracle_naiv_on_array.argtypes = gemm
            lib.oracle_naiv_on_array.restype = None
            lib.oracle_naiv_unrolled.argtypes = gemm + [ctypes.c_int]
            lib.oracle_naiv_unrolled.restype = ctypes.c_int
            lib.oracle_winograd_rowcol_scaled.argtypes = gemm + [ip, ip]
            lib.oracle_winograd_rowcol_scaled.restype = None
            lib.oracle_brent_lambda.argtypes = [ctypes.c_double, ctypes.c_double]
            lib.oracle_brent_lambda.restype = ctypes.c_int
            lib.oracle_strassen_paper_rule.argtypes = [i64, i64, i64, ctypes.POINTER(ctypes.c_int),
                                                       ctypes.POINTER(ctypes.c_int64)]
            for name in ("oracle_strassen_naiv", "oracle_strassen_winograd"):
                getattr(lib, name).argtypes = gemm + [ctypes.c_int, i64, i64, i64]
                getattr(lib, name).restype = ctypes.c_int
            lib.oracle_split_digits.argtypes = [i64, i64, dp, i64, ctypes.c_int, ctypes.c_int, ctypes.c_int, ip, ip]
            lib.oracle_split_digits.restype = ctypes.c_int
            lib.oracle_split_product.argtypes = gemm + [ctypes.c_int, ctypes.c_int]
            lib.oracle_split_product.restype = ctypes.c_int
            lib.oracle_strassen_emulated.argtypes = [ctypes.c_int] + gemm + [ctypes.c_int, ctypes.c_int, ctypes.c_int]
            lib.oracle_strassen_emulated.restype = ctypes.c_int
            _lib = lib
    return _lib


def _f64(x):
    x = np.asarray(x, dtype=np.float64)
    if x.ndim != 2:
        raise ValueError("expected a 2-D matrix")
    if not x.flags.c_contiguous:
        x = np.ascontiguousarray(x)
    return x


def _ptr(x):
    return x.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ld(x):
    return max(1, x.shape[1])


def _gemm(name, a, b, *extra):
    a, b = _f64(a), _f64(b)
    n, p = a.shape
    p2, m = b.shape
    if p != p2:
        raise ValueError("inner dimensions differ")
    c = np.zeros((n, m), dtype=np.float64)
    rc = getattr(_load(), name)(n, p, m, _ptr(a), _ld(a), _ptr(b), _ld(b), _ptr(c), _ld(c), *extra)
    return c, rc


def norm_inf(a) -> float:
    a = _f64(a)
    return float(_load().oracle_norm_inf(a.shape[0], a.shape[1], _ptr(a), _ld(a)))


def multiply_with_scalar(alpha: float, a):
    a = _f64(a)
    z = np.zeros_like(a)
    _load().oracle_multiply_with_scalar(a.shape[0], a.shape[1], float(alpha), _ptr(a), _ld(a), _ptr(z), _ld(z))
    return z


def naiv_standard(a, b):
    return _gemm("oracle_naiv_standard", a, b)[0]


def naiv_kahan(a, b):
    return _gemm("oracle_naiv_kahan", a, b)[0]


def naiv_on_array(a, b):
    return _gemm("oracle_naiv_on_array", a, b)[0]


def naiv_unrolled(a, b, u: int):
    """NaivLoopUnrollingTwo/Three/Four for u = 2/3/4 (u = 1: NaivStandard)."""
    c, rc = _gemm("oracle_naiv_unrolled", a, b, int(u))
    if rc != 0:
        raise ValueError("unroll factor must be >= 1")
    return c


def naiv_unrolled_2(a, b):
    return naiv_unrolled(a, b, 2)


def naiv_unrolled_3(a, b):
    return naiv_unrolled(a, b, 3)


def naiv_unrolled_4(a, b):
    return naiv_unrolled(a, b, 4)


def winograd_original(a, b):
    return _gemm("oracle_winograd_original", a, b)[0]


def winograd_terms(a, b):
    a, b = _f64(a), _f64(b)
    n, p = a.shape
    m = b.shape[1]
    y = np.zeros(max(n, 1))
    z = np.zeros(max(m, 1))
    _load().oracle_winograd_terms(n, p, m, _ptr(a), _ld(a), _ptr(b), _ld(b),
                                  y.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                  z.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return y[:n], z[:m]


def brent_lambda(norm_a: float, norm_b: float) -> int:
    return int(_load().oracle_brent_lambda(float(norm_a), float(norm_b)))


def winograd_scaled(a, b):
    """Returns (C, lambda)."""
    c, lam = _gemm("oracle_winograd_scaled", a, b)
    return c, int(lam)


def winograd_rowcol_scaled(a, b):
    """Returns (C, e, f): Winograd's form with each row of A scaled by 2^-e_i and
    each column of B by 2^-f_k, the result scaled back by 2^(e_i + f_k)."""
    a, b = _f64(a), _f64(b)
    n, p = a.shape
    m = b.shape[1]
    c = np.zeros((n, m))
    e = np.zeros(max(n, 1), dtype=np.int32)
    f = np.zeros(max(m, 1), dtype=np.int32)
    ipt = ctypes.POINTER(ctypes.c_int32)
    _load().oracle_winograd_rowcol_scaled(n, p, m, _ptr(a), _ld(a), _ptr(b), _ld(b), _ptr(c), _ld(c),
                                          e.ctypes.data_as(ipt), f.ctypes.data_as(ipt))
    return c, e[:n], f[:m]


def strassen_paper_rule(n: int, p: int, m: int):
    k = ctypes.c_int()
    y = ctypes.c_int64()
    _load().oracle_strassen_paper_rule(n, p, m, ctypes.byref(k), ctypes.byref(y))
    return int(k.value), int(y.value)


def _strassen(name, a, b, depth, padded):
    np_, pp, mp = padded if padded is not None else (0, 0, 0)
    c, rc = _gemm(name, a, b, int(depth), int(np_), int(pp), int(mp))
    if rc != 0:
        raise ValueError(f"{name}: bad depth/padding ({depth}, {padded})")
    return c


def strassen_naiv(a, b, depth: int = -1, padded=None):
    """depth=-1: the paper's rule (square embedding); else padded = (Np, Pp, Mp)."""
    return _strassen("oracle_strassen_naiv", a, b, depth, padded)


def strassen_winograd(a, b, depth: int = -1, padded=None):
    return _strassen("oracle_strassen_winograd", a, b, depth, padded)


def strassen_emulated(a, b, variant: int, depth: int, beta: int, s: int):
    """Strassen (variant 0) or Strassen-Winograd (variant 1), `depth` levels, over
    the split product (beta, s); operands zero-padded to multiples of 2^depth."""
    a, b = _f64(a), _f64(b)
    n, p = a.shape
    if b.shape[0] != p:
        raise ValueError("inner dimensions differ")
    m = b.shape[1]
    c = np.zeros((n, m), dtype=np.float64)
    rc = _load().oracle_strassen_emulated(int(variant), n, p, m, _ptr(a), _ld(a), _ptr(b), _ld(b), _ptr(c), _ld(c),
                                          int(depth), int(beta), int(s))
    if rc != 0:
        raise ValueError(f"oracle_strassen_emulated: bad arguments ({variant}, {depth}, {beta}, {s})")
    return c


def dot2_product(a, b):
    return _gemm("oracle_dot2_product", a, b)[0]


def split_digits(x, by_columns: bool, beta: int, s: int):
    """Returns (exponents, digits[s, rows, cols]) of the slice decomposition."""
    x = _f64(x)
    rows, cols = x.shape
    exps = np.zeros(max(cols if by_columns else rows, 1), dtype=np.int32)
    dig = np.zeros((s, rows, cols), dtype=np.int32)
    rc = _load().oracle_split_digits(rows, cols, _ptr(x), _ld(x), int(by_columns), int(beta), int(s),
                                     exps.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                     dig.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    if rc != 0:
        raise ValueError("bad split parameters")
    return exps[: (cols if by_columns else rows)], dig


def split_product(a, b, beta: int, s: int):
    c, rc = _gemm("oracle_split_product", a, b, int(beta), int(s))
    if rc != 0:
        raise ValueError("bad split parameters")
    return c


def rel_inf_error(c, c_ref, a, b) -> float:
    """||C - C_ref||_inf / (||A||_inf ||B||_inf) with the oracle's own NormInf."""
    d = np.asarray(c, dtype=np.float64) - np.asarray(c_ref, dtype=np.float64)
    den = norm_inf(a) * norm_inf(b)
    num = norm_inf(d) if d.size else 0.0
    return num / den if den > 0 else num
