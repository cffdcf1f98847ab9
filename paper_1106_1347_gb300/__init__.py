"""GB300 (sm_103a) library for the methods of Hedtke, "Methods of Matrix
Multiplication" (arXiv:1106.1347), with an FP64-accurate product emulated from
BF16 slices on the tcgen05 tensor cores.

Thin PyTorch binding over the libmm C ABI (include/mm.h): tensors provide
device memory and the current CUDA stream; every step runs in libmm's kernels.
Operands are 2-D float64 CUDA tensors with unit column stride (row-major with
leading dimension = stride(0)); anything else is made contiguous first.
"""
from __future__ import annotations

import ctypes

from ._native import KernelStat, MMError, check, lib

__all__ = ["naive", "naive_unrolled", "kahan", "winograd", "winograd_scaled", "winograd_rowcol_scaled", "strassen", "strassen_winograd", "strassen_emulated", "tune_strassen", "tune_emulated", "emulated_choice", "emulated_auto", "tune_save", "tune_load", "tune_clear", "norm_inf",
           "emulated", "emulated_tiled", "emulated_host", "emulated_group", "emulated_noalloc", "emulated_slices", "probe_fp64_peak", "profile", "device_status", "MMError", "lib", "SLICE_BF16",
           "SLICE_FP8E4M3"]

SLICE_BF16 = 0
SLICE_FP8E4M3 = 1


def _torch():
    import torch

    return torch


def _mat(x, name):
    torch = _torch()
    if not isinstance(x, torch.Tensor) or not x.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if x.dtype != torch.float64 or x.dim() != 2:
        raise TypeError(f"{name} must be a 2-D float64 tensor")
    if x.stride(1) != 1 or (x.shape[0] > 1 and x.stride(0) < max(1, x.shape[1])):
        x = x.contiguous()
    return x


def _ld(x):
    return max(1, x.stride(0) if x.shape[0] > 1 else x.shape[1])


def _stream(device):
    torch = _torch()
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _prep(a, b, out):
    torch = _torch()
    a, b = _mat(a, "A"), _mat(b, "B")
    if a.shape[1] != b.shape[0]:
        raise ValueError(f"inner dimensions differ: {tuple(a.shape)} x {tuple(b.shape)}")
    if a.device != b.device:
        raise ValueError("A and B are on different devices")
    n, p = a.shape
    m = b.shape[1]
    if out is None:
        out = torch.empty((n, m), dtype=torch.float64, device=a.device)
    else:
        if out.shape != (n, m) or out.dtype != torch.float64 or out.device != a.device or out.stride(1) != 1:
            raise ValueError("out must be an N x M float64 tensor with unit column stride on A's device")
    return a, b, out, n, p, m


def _ptr(x):
    return ctypes.c_void_p(x.data_ptr())


def _ws(nbytes, device):
    torch = _torch()
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device)


def _gemm_args(a, b, c, n, p, m):
    return [n, p, m, _ptr(a), _ld(a), _ptr(b), _ld(b), _ptr(c), _ld(c)]


def naive(a, b, out=None):
    """Section "The naive method": C = A B on the FP64 tensor-core MMA."""
    a, b, c, n, p, m = _prep(a, b, out)
    check("mm_naive", lib().mm_naive(*_gemm_args(a, b, c, n, p, m), _stream(a.device)))
    return c


def kahan(a, b, out=None):
    """Section "NaivKahan": naive product with the paper's compensated sum."""
    a, b, c, n, p, m = _prep(a, b, out)
    check("mm_kahan", lib().mm_kahan(*_gemm_args(a, b, c, n, p, m), _stream(a.device)))
    return c


def naive_unrolled(a, b, unroll=1, out=None):
    """Sections "NaivStandard"/"NaivOnArray" (unroll=1) and "Loop unrolling"
    (unroll=2, 3, 4): the naive sum in the paper's order, bit-exact."""
    a, b, c, n, p, m = _prep(a, b, out)
    check("mm_naive_unrolled", lib().mm_naive_unrolled(*_gemm_args(a, b, c, n, p, m), int(unroll), _stream(a.device)))
    return c


def winograd(a, b, out=None):
    """Section "WinogradOriginal"."""
    a, b, c, n, p, m = _prep(a, b, out)
    need = lib().mm_winograd_workspace_bytes(n, p, m)
    ws = _ws(need, a.device)
    check("mm_winograd", lib().mm_winograd(*_gemm_args(a, b, c, n, p, m), _ptr(ws), need, _stream(a.device)))
    return c


def winograd_scaled(a, b, out=None, return_lambda=False):
    """Section "WinogradScaled".  With return_lambda=True returns (C, lambda tensor)."""
    torch = _torch()
    a, b, c, n, p, m = _prep(a, b, out)
    need = lib().mm_winograd_scaled_workspace_bytes(n, p, m)
    ws = _ws(need, a.device)
    lam = torch.zeros(1, dtype=torch.int32, device=a.device)
    check("mm_winograd_scaled", lib().mm_winograd_scaled(*_gemm_args(a, b, c, n, p, m), _ptr(lam), _ptr(ws), need,
                                                         _stream(a.device)))
    return (c, lam) if return_lambda else c


def winograd_rowcol_scaled(a, b, out=None):
    """Winograd's form with each row of A scaled by 2^-e_i and each column of B
    by 2^-f_k (frexp exponents of their maxima), the result by 2^(e_i + f_k):
    the power-of-two scaling of section "WinogradScaled" per row and column."""
    a, b, c, n, p, m = _prep(a, b, out)
    need = lib().mm_winograd_rowcol_scaled_workspace_bytes(n, p, m)
    ws = _ws(need, a.device)
    check("mm_winograd_rowcol_scaled", lib().mm_winograd_rowcol_scaled(*_gemm_args(a, b, c, n, p, m), _ptr(ws), need,
                                                                       _stream(a.device)))
    return c


def _strassen(name, a, b, cutoff, out):
    a, b, c, n, p, m = _prep(a, b, out)
    need = getattr(lib(), name + "_workspace_bytes")(n, p, m, int(cutoff))
    ws = _ws(need, a.device)
    check(name, getattr(lib(), name)(*_gemm_args(a, b, c, n, p, m), int(cutoff), _ptr(ws), need,
                                     _stream(a.device)))
    return c


def strassen(a, b, cutoff=-1, out=None):
    """Section "StrassenNaiv".  cutoff: 0 = the paper's rule, >0 = base size, -1 = tuned."""
    return _strassen("mm_strassen", a, b, cutoff, out)


def strassen_winograd(a, b, cutoff=-1, out=None):
    """Section "StrassenWinograd"."""
    return _strassen("mm_strassen_winograd", a, b, cutoff, out)


def tune_strassen(a, b, variant=0):
    """Times Strassen depths 0..3 on (A, B), records the fastest for this shape
    bucket (used by cutoff=-1) and returns (depth, ms)."""
    a, b, c, n, p, m = _prep(a, b, None)
    need = lib().mm_tune_strassen_workspace_bytes(n, p, m)
    ws = _ws(need, a.device)
    depth, ms = ctypes.c_int32(-1), ctypes.c_double(0.0)
    check("mm_tune_strassen", lib().mm_tune_strassen(int(variant), *_gemm_args(a, b, c, n, p, m), _ptr(ws), need,
                                                     _stream(a.device), ctypes.byref(depth), ctypes.byref(ms)))
    return int(depth.value), float(ms.value)


def tune_emulated(a, b, tier=1e-14):
    """Times the emulated product's candidates (slice format x Strassen-Winograd
    levels, and for the direct product the tile width) for this shape and tier,
    records the fastest for the shape bucket (used by emulated_auto and, for
    format and count, serving method 2) and returns
    (format, slices, levels, ms, tile width)."""
    a, b, c, n, p, m = _prep(a, b, None)
    need = lib().mm_tune_emulated_workspace_bytes(n, p, m, float(tier))
    ws = _ws(need, a.device)
    k, s, lv, ms, tl = ctypes.c_int32(-1), ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_double(0.0), ctypes.c_int32(0)
    check("mm_tune_emulated", lib().mm_tune_emulated(*_gemm_args(a, b, c, n, p, m), float(tier), _ptr(ws), need,
                                                     _stream(a.device), ctypes.byref(k), ctypes.byref(s),
                                                     ctypes.byref(lv), ctypes.byref(ms), ctypes.byref(tl)))
    return int(k.value), int(s.value), int(lv.value), float(ms.value), int(tl.value)


def emulated_choice(n, p, m, tier=1e-14):
    """The (format, slices, levels, tile width) emulated_auto uses for this
    shape and tier, and whether it comes from the tuned table (host only)."""
    k, s, lv, tl = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int32(0)
    rc = lib().mm_tune_emulated_choice(int(n), int(p), int(m), float(tier), ctypes.byref(k), ctypes.byref(s),
                                       ctypes.byref(lv), ctypes.byref(tl))
    if rc < 0:
        check("mm_tune_emulated_choice", rc)
    return (int(k.value), int(s.value), int(lv.value), int(tl.value)), rc == 1


def emulated_auto(a, b, tier=1e-14, out=None, return_choice=False):
    """FP64-accurate product with the autotuned (or modelled) format, slice
    count, Strassen-Winograd levels and tile width for the tier
    (mm_emulated_auto)."""
    a, b, c, n, p, m = _prep(a, b, out)
    need = lib().mm_emulated_auto_workspace_bytes(n, p, m, float(tier))
    ws = _ws(need, a.device)
    used = (ctypes.c_int32 * 4)()
    check("mm_emulated_auto", lib().mm_emulated_auto(*_gemm_args(a, b, c, n, p, m), float(tier), _ptr(ws), need,
                                                     _stream(a.device), used))
    return (c, tuple(int(u) for u in used)) if return_choice else c


def tune_save(path):
    check("mm_tune_save", lib().mm_tune_save(str(path).encode()))


def tune_load(path):
    n = lib().mm_tune_load(str(path).encode())
    if n < 0:
        check("mm_tune_load", n)
    return n


def tune_clear():
    check("mm_tune_clear", lib().mm_tune_clear())


def norm_inf(a):
    """Section "NormInf": returns a 0-d float64 device tensor."""
    torch = _torch()
    a = _mat(a, "A")
    out = torch.empty((), dtype=torch.float64, device=a.device)
    check("mm_norm_inf", lib().mm_norm_inf(a.shape[0], a.shape[1], _ptr(a), _ld(a), _ptr(out), _stream(a.device)))
    return out


def emulated_slices(nslices=0, tier=1e-14, kind=SLICE_BF16):
    return int(lib().mm_emulated_slices(kind, nslices, tier))


def emulated(a, b, nslices=0, tier=1e-14, kind=SLICE_BF16, out=None):
    """FP64-accurate product from BF16 or FP8-E4M3 slices on tcgen05 (see include/mm.h)."""
    a, b, c, n, p, m = _prep(a, b, out)
    need = lib().mm_emulated_workspace_bytes(n, p, m, kind, nslices, tier)
    ws = _ws(need, a.device)
    check("mm_emulated", lib().mm_emulated(*_gemm_args(a, b, c, n, p, m), kind, nslices, float(tier), _ptr(ws), need,
                                           _stream(a.device)))
    return c


def emulated_tiled(a, b, tile_n, nslices=0, tier=1e-14, kind=SLICE_BF16, out=None):
    """mm_emulated with the slice product's tile width chosen (64, 32, or 0 for
    the default); the result is bit-identical to emulated()."""
    a, b, c, n, p, m = _prep(a, b, out)
    need = lib().mm_emulated_workspace_bytes(n, p, m, kind, nslices, tier)
    ws = _ws(need, a.device)
    check("mm_emulated_tiled", lib().mm_emulated_tiled(*_gemm_args(a, b, c, n, p, m), kind, nslices, float(tier),
                                                       int(tile_n), _ptr(ws), need, _stream(a.device)))
    return c


def strassen_emulated(a, b, variant=0, levels=1, nslices=0, tier=1e-14, kind=SLICE_BF16, out=None):
    """Strassen (variant 0) or Strassen-Winograd (1) levels over the emulated
    product: mm_strassen_emulated (see include/mm.h); levels=-1 picks the
    count from the size."""
    a, b, c, n, p, m = _prep(a, b, out)
    need = lib().mm_strassen_emulated_workspace_bytes(n, p, m, int(variant), int(levels), kind, nslices, tier)
    ws = _ws(need, a.device)
    check("mm_strassen_emulated", lib().mm_strassen_emulated(*_gemm_args(a, b, c, n, p, m), int(variant), int(levels),
                                                             kind, nslices, float(tier), _ptr(ws), need,
                                                             _stream(a.device)))
    return c


def emulated_host(a, b, out=None, nslices=0, tier=1e-14, kind=SLICE_BF16, device=None):
    """mm_emulated_host: host (CPU) float64 operands, device workspace; copies
    overlap the products.  Returns the host result after the stream completes."""
    import numpy as np

    torch = _torch()

    def host(x):
        x = x.numpy() if isinstance(x, torch.Tensor) else np.asarray(x)
        if x.dtype != np.float64 or x.ndim != 2 or x.strides[1] != 8:
            raise TypeError("host operands must be 2-D float64 with unit column stride")
        return x

    a, b = host(a), host(b)
    n, p = a.shape
    p2, m = b.shape
    if p != p2:
        raise ValueError("inner dimensions differ")
    c = np.empty((n, m)) if out is None else host(out)
    if c.shape != (n, m):
        raise ValueError("output shape mismatch")
    dev = torch.device("cuda") if device is None else torch.device(device)
    need = lib().mm_emulated_host_workspace_bytes(n, p, m, kind, nslices, tier)
    ws = _ws(need, dev)

    def ld(x):
        return max(1, x.strides[0] // 8 if x.shape[0] > 1 else x.shape[1])

    stream = torch.cuda.current_stream(dev)
    check("mm_emulated_host", lib().mm_emulated_host(n, p, m, a.ctypes.data, ld(a), b.ctypes.data, ld(b),
                                                     c.ctypes.data, ld(c), kind, nslices, float(tier), _ptr(ws), need,
                                                     ctypes.c_void_p(stream.cuda_stream)))
    stream.synchronize()
    return c


def emulated_group(pairs, nslices=0, tier=1e-14, kind=SLICE_BF16, outs=None):
    """Grouped FP64-accurate products: [(A_g, B_g)] -> [C_g] in one launch per kernel."""
    from ._native import Problem

    torch = _torch()
    prepared, results = [], []
    for g, (a, b) in enumerate(pairs):
        a, b, c, n, p, m = _prep(a, b, None if outs is None else outs[g])
        prepared.append((a, b))
        results.append(c)
    if not prepared:
        return []
    arr = (Problem * len(prepared))()
    for g, ((a, b), c) in enumerate(zip(prepared, results)):
        arr[g] = Problem(a.shape[0], a.shape[1], b.shape[1], a.data_ptr(), _ld(a), b.data_ptr(), _ld(b),
                         c.data_ptr(), _ld(c))
    dev = prepared[0][0].device
    need = lib().mm_emulated_group_workspace_bytes(arr, len(prepared), kind, nslices, tier)
    ws = _ws(need, dev)
    check("mm_emulated_group", lib().mm_emulated_group(arr, len(prepared), kind, nslices, float(tier), _ptr(ws), need,
                                                       _stream(dev)))
    return results


def emulated_noalloc(a, b, nslices=0, tier=1e-14, kind=SLICE_BF16, out=None):
    """mm_emulated with its scratch in the library's fixed 64 MiB device array
    instead of a workspace (for callers that cannot allocate device memory).
    Calls sharing a device must not overlap on the GPU; see include/mm.h."""
    a, b, c, n, p, m = _prep(a, b, out)
    check("mm_emulated_noalloc", lib().mm_emulated_noalloc(*_gemm_args(a, b, c, n, p, m), kind, nslices, float(tier),
                                                           _stream(a.device)))
    return c


def probe_fp64_peak(target_ms=100.0, device=None):
    """The FP64 pipe's measured rate on this device (mm_probe_fp64_peak):
    returns (DFMA TFLOP/s, mma.sync f64 TFLOP/s)."""
    torch = _torch()
    dev = torch.device("cuda") if device is None else torch.device(device)
    dfma, dmma = ctypes.c_double(0.0), ctypes.c_double(0.0)
    check("mm_probe_fp64_peak", lib().mm_probe_fp64_peak(float(target_ms), ctypes.byref(dfma), ctypes.byref(dmma),
                                                         _stream(dev)))
    return float(dfma.value), float(dmma.value)


class profile:
    """Context manager recording every libmm kernel launch with CUDA events on
    its own stream.  After exit, ``stats`` maps kernel name -> (launches, ms)."""

    def __enter__(self):
        lib().mm_profile_read(None, 0)
        check("mm_profile_enable", lib().mm_profile_enable(1))
        self.stats = {}
        return self

    def __exit__(self, *exc):
        lib().mm_profile_enable(0)
        buf = (KernelStat * 64)()
        n = lib().mm_profile_read(buf, 64)
        if n < 0:
            check("mm_profile_read", n)
        self.stats = {buf[i].name.decode(): (int(buf[i].launches), float(buf[i].total_ms)) for i in range(min(n, 64))}
        return False


def device_status(device=None):
    """Reads and clears the kernels' timeout status word; returns the raw code."""
    torch = _torch()
    code = ctypes.c_int32(0)
    dev = torch.device("cuda") if device is None else torch.device(device)
    rc = lib().mm_device_status(_stream(dev), ctypes.byref(code))
    if rc not in (0, -5):
        check("mm_device_status", rc)
    return int(code.value)
