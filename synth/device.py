"""Device-side input generation for workloads too large to draw on the host.

Same Philox streams as ``synth`` (host); the integral blocks are then formed
with torch FP64 matrix products.  Equal to the host generator up to FP64
rounding (the host packs symmetric pairs, the device multiplies the blocks
directly; Box-Muller's log/cos/sin may differ by an ulp).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import synth

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "device.cu")
_LIB = os.path.join(_HERE, "libsynth.so")
_lib = None


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        nvcc = "/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else "nvcc"
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.run([nvcc, "-O3", "-shared", "-Xcompiler", "-fPIC", "-gencode", "arch=compute_103a,code=sm_103a",
                        "-o", tmp, _SRC], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _L():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_LIB)
        _lib.synth_factors.argtypes = [ctypes.c_uint, ctypes.c_uint, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                       ctypes.c_void_p, ctypes.c_void_p]
        _lib.synth_factors.restype = ctypes.c_int
    return _lib


def factors(X, Y, nX, nY, naux=synth.NAUX, kappa=synth.KAPPA, seed=synth.SEED, device="cuda"):
    import torch
    n = nX + nY
    B = torch.empty((naux, n, n), dtype=torch.float64, device=device)
    st = torch.cuda.current_stream(B.device).cuda_stream
    rc = _L().synth_factors(seed & 0xFFFFFFFF, synth.dimer_object_id(X, Y), n, naux, kappa, B.data_ptr(), st)
    if rc != 0:
        raise RuntimeError(f"synth_factors launch failed ({rc})")
    return B


def blocks_into(B, nX, s, out):
    """Write [A | K] (contiguous, A = (XX|YY) then K = (XY|YX)) of one dimer into
    the flat FP64 device tensor ``out``."""
    naux, n, _ = B.shape
    nY = n - nX
    Bf = B.reshape(naux, n, n)
    bxx = Bf[:, :nX, :nX].reshape(naux, nX * nX)
    byy = Bf[:, nX:, nX:].reshape(naux, nY * nY)
    bxy = Bf[:, :nX, nX:].reshape(naux, nX * nY)
    byx = Bf[:, nX:, :nX].reshape(naux, nY * nX)
    blk = nX * nX * nY * nY
    out[:blk].view(nX * nX, nY * nY).copy_(bxx.T @ byy).mul_(s)
    out[blk:2 * blk].view(nX * nY, nY * nX).copy_(bxy.T @ byx).mul_(s)
    return out


def workload_blocks(w: synth.Workload, dimers=None, device="cuda"):
    """All (or the listed) dimers' blocks in one flat device buffer.
    Returns (buffer, offsets) with dimer k's [A | K] at buffer[offsets[k]:]."""
    import torch
    dimers = list(range(w.n_dimers)) if dimers is None else list(dimers)
    sizes = [2 * (w.nao[w.pairs[d][0]] ** 2) * (w.nao[w.pairs[d][1]] ** 2) for d in dimers]
    offs, o = [], 0
    for s_ in sizes:
        offs.append(o)
        o += (s_ + 31) // 32 * 32     # 256-byte aligned starts
    buf = torch.empty(o, dtype=torch.float64, device=device)
    for k, d in enumerate(dimers):
        X, Y = w.pairs[d]
        B = factors(X, Y, w.nao[X], w.nao[Y], seed=w.seed, device=device)
        blocks_into(B, w.nao[X], synth.scale_for_distance(w.R[d]), buf[offs[k]:offs[k] + sizes[k]])
    return buf, offs


def fill_views(w: synth.Workload, views, device="cuda"):
    """Producer for streamed runs: write each view's [A | K] blocks (objects
    with ``dimer`` and ``out``) from the dimer's seeded factors."""
    for v in views:
        X, Y = w.pairs[v.dimer]
        B = factors(X, Y, w.nao[X], w.nao[Y], seed=w.seed, device=device)
        blocks_into(B, w.nao[X], synth.scale_for_distance(w.R[v.dimer]), v.out)
        del B
