"""Python binding of libmcpt, the GB300 library for the first-order MCPT(2)
dimer term (C ABI in include/mcpt.h).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of libmcpt.so.  There is no CPU fallback; importing works without a
GPU (so the library can be inspected), but every call that computes needs the
built library and a Blackwell GPU, and fails loudly otherwise.

Host arrays are numpy float64; device arrays may be torch CUDA tensors (their
``data_ptr()`` is passed) or raw integer device addresses.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmcpt.so")

MCPT_OK, MCPT_EINVAL, MCPT_ENOMEM, MCPT_ECUDA, MCPT_ESTATE, MCPT_ETIMEOUT, MCPT_EUNSUPPORTED = range(7)
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ESTATE", 5: "ETIMEOUT", 6: "EUNSUPPORTED"}
MCPT_FP64, MCPT_TF32, MCPT_BF16X3, MCPT_FP32C, MCPT_BF16X2, MCPT_FP64E = range(6)
PRECISIONS = {"fp64": MCPT_FP64, "tf32": MCPT_TF32, "bf16x3": MCPT_BF16X3, "fp32c": MCPT_FP32C,
              "bf16x2": MCPT_BF16X2, "fp64e": MCPT_FP64E}
MCPT_AO_FULL, MCPT_AO_BLOCKS, MCPT_AO_PACKED = 0, 1, 2
MCPT_UPDATE_ASYNC = 1

# every symbol include/mcpt.h declares
EXPORTS = ("mcpt_default_options", "mcpt_create", "mcpt_add_monomer", "mcpt_add_dimer", "mcpt_update_dimer",
           "mcpt_set_precision",
           "mcpt_run", "mcpt_run_range", "mcpt_energies", "mcpt_coupling", "mcpt_singles", "mcpt_set_monomer_doubles", "mcpt_td2",
           "mcpt_add_dimer_df", "mcpt_run_df", "mcpt_df_energies",
           "mcpt_collect_stats", "mcpt_num_monomers",
           "mcpt_num_dimers", "mcpt_last_error", "mcpt_destroy", "mcpt_dimer_fp64_noalloc",
           "mcpt_fp64_fma_rate", "mcpt_update_dimers")


class McptError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"MCPT_{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class mcpt_options(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("stream", ctypes.c_void_p), ("precision", ctypes.c_int),
                ("validate", ctypes.c_int), ("wave_bytes", ctypes.c_size_t), ("tune_cache", ctypes.c_char_p),
                ("timing", ctypes.c_int), ("mem_cap_bytes", ctypes.c_size_t), ("graphs", ctypes.c_int),
                ("coupling", ctypes.c_int), ("wait_limit_ns", ctypes.c_ulonglong), ("withhold_load", ctypes.c_int),
                ("fp64_epilogue", ctypes.c_int)]


class mcpt_run_stats(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_float * 4), ("runs", ctypes.c_int), ("launches", ctypes.c_int),
                ("waves", ctypes.c_int), ("alg_bytes", ctypes.c_double), ("alg_flops", ctypes.c_double),
                ("alg_flops_half", ctypes.c_double)]


_lib = None


def lib():
    """Load libmcpt.so (built in-tree by __graft_entry__.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libmcpt.so is not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        H, I, P, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)
        L.mcpt_default_options.argtypes = [ctypes.POINTER(mcpt_options)]
        L.mcpt_default_options.restype = None
        L.mcpt_create.argtypes = [ctypes.POINTER(H), ctypes.POINTER(mcpt_options)]
        L.mcpt_add_monomer.argtypes = [H, P, P, I, I, ctypes.POINTER(I)]
        L.mcpt_add_dimer.argtypes = [H, I, I, P, I, I, ctypes.POINTER(I)]
        L.mcpt_update_dimer.argtypes = [H, I, P, I, I, I]
        L.mcpt_set_precision.argtypes = [H, I]
        L.mcpt_run.argtypes = [H]
        L.mcpt_run_range.argtypes = [H, I, I]
        L.mcpt_energies.argtypes = [H, P, P, P, P]
        L.mcpt_coupling.argtypes = [H, I, P]
        L.mcpt_singles.argtypes = [H, P, P]
        L.mcpt_set_monomer_doubles.argtypes = [H, I, P, P]
        L.mcpt_td2.argtypes = [H, I, P, P]
        L.mcpt_add_dimer_df.argtypes = [H, I, I, P, I, ctypes.c_double, I, ctypes.POINTER(I)]
        L.mcpt_run_df.argtypes = [H]
        L.mcpt_df_energies.argtypes = [H, P, P, P, P]
        L.mcpt_collect_stats.argtypes = [H, ctypes.POINTER(mcpt_run_stats)]
        for f in ("mcpt_create", "mcpt_add_monomer", "mcpt_add_dimer", "mcpt_update_dimer", "mcpt_set_precision", "mcpt_run",
                  "mcpt_run_range", "mcpt_energies", "mcpt_coupling", "mcpt_singles", "mcpt_set_monomer_doubles",
                  "mcpt_td2", "mcpt_add_dimer_df", "mcpt_run_df", "mcpt_df_energies", "mcpt_collect_stats"):
            getattr(L, f).restype = I
        L.mcpt_num_monomers.argtypes = [H]
        L.mcpt_num_monomers.restype = I
        L.mcpt_num_dimers.argtypes = [H]
        L.mcpt_num_dimers.restype = I
        L.mcpt_last_error.argtypes = [H]
        L.mcpt_last_error.restype = ctypes.c_char_p
        L.mcpt_destroy.argtypes = [H]
        L.mcpt_destroy.restype = None
        L.mcpt_dimer_fp64_noalloc.argtypes = [P, P, P, P, I, I, P, P, I, I, P, P]
        L.mcpt_dimer_fp64_noalloc.restype = I
        L.mcpt_fp64_fma_rate.argtypes = [I, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
        L.mcpt_fp64_fma_rate.restype = I
        L.mcpt_update_dimers.argtypes = [H, I, I, P, P, I, I]
        L.mcpt_update_dimers.restype = I
        _lib = L
    return _lib


def _check(h, st):
    if st != MCPT_OK:
        raise McptError(st, lib().mcpt_last_error(h).decode())


def _ptr(x):
    """Address of a numpy array, a torch tensor, or an int."""
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    raise TypeError(f"cannot take the address of {type(x)}")


# ----------------------------------------------------------- thin wrappers
def mcpt_default_options() -> mcpt_options:
    o = mcpt_options()
    lib().mcpt_default_options(ctypes.byref(o))
    return o


def mcpt_create(opts: mcpt_options | None = None) -> int:
    h = ctypes.c_void_p()
    st = lib().mcpt_create(ctypes.byref(h), ctypes.byref(opts) if opts is not None else None)
    _check(None, st)
    return h.value


def mcpt_add_monomer(h, C, eps, nao: int, nocc: int) -> int:
    C = np.ascontiguousarray(C, dtype=np.float64)
    eps = np.ascontiguousarray(eps, dtype=np.float64)
    out = ctypes.c_int()
    _check(h, lib().mcpt_add_monomer(h, _ptr(C), _ptr(eps), nao, nocc, ctypes.byref(out)))
    return out.value


def mcpt_update_dimer(h, dimer: int, ao_eri, layout: int, on_device: int, flags: int = 0) -> None:
    if isinstance(ao_eri, np.ndarray):
        ao_eri = np.ascontiguousarray(ao_eri, dtype=np.float64)
    _check(h, lib().mcpt_update_dimer(h, dimer, _ptr(ao_eri), layout, on_device, flags))


def mcpt_update_dimers(h, first: int, count: int, ao_eri, offsets, layout: int, flags: int = 0) -> None:
    """Host integrals of dimers first .. first+count-1: dimer first+k's at
    element offsets[k] of ao_eri (a numpy array or a host address)."""
    if isinstance(ao_eri, np.ndarray):
        ao_eri = np.ascontiguousarray(ao_eri, dtype=np.float64)
    off = np.ascontiguousarray(offsets, dtype=np.uint64)
    if off.size != count:
        raise ValueError("offsets must hold count entries")
    _check(h, lib().mcpt_update_dimers(h, first, count, _ptr(ao_eri), off.ctypes.data, layout, flags))


def mcpt_add_dimer(h, X: int, Y: int, ao_eri, layout: int, on_device: int) -> int:
    if isinstance(ao_eri, np.ndarray):
        ao_eri = np.ascontiguousarray(ao_eri, dtype=np.float64)
    out = ctypes.c_int()
    _check(h, lib().mcpt_add_dimer(h, X, Y, _ptr(ao_eri), layout, on_device, ctypes.byref(out)))
    return out.value


def mcpt_set_precision(h, p: int) -> None:
    _check(h, lib().mcpt_set_precision(h, p))


def mcpt_run(h) -> None:
    _check(h, lib().mcpt_run(h))


def mcpt_run_range(h, first: int, count: int) -> None:
    _check(h, lib().mcpt_run_range(h, first, count))


def mcpt_energies(h):
    """(per_monomer_J [N], per_monomer_K [N], per_dimer [D,2], total [2])."""
    N, D = lib().mcpt_num_monomers(h), lib().mcpt_num_dimers(h)
    mj, mk = np.empty(N), np.empty(N)
    pd, tot = np.empty((D, 2)), np.empty(2)
    _check(h, lib().mcpt_energies(h, _ptr(mj), _ptr(mk), _ptr(pd), _ptr(tot)))
    return mj, mk, pd, tot


def mcpt_coupling(h, X: int, dim: int) -> np.ndarray:
    R = np.empty((dim, dim))
    _check(h, lib().mcpt_coupling(h, X, _ptr(R)))
    return R


def mcpt_singles(h, t: np.ndarray) -> np.ndarray:
    """t: every monomer's [o][v] amplitudes concatenated (FP64, 1-D)."""
    t = np.ascontiguousarray(t, dtype=np.float64).ravel()
    s = np.empty_like(t)
    _check(h, lib().mcpt_singles(h, _ptr(t), _ptr(s)))
    return s


def mcpt_set_monomer_doubles(h, X: int, G, U) -> None:
    G = None if G is None else np.ascontiguousarray(G, dtype=np.float64)
    U = None if U is None else np.ascontiguousarray(U, dtype=np.float64)
    _check(h, lib().mcpt_set_monomer_doubles(h, X, None if G is None else _ptr(G), None if U is None else _ptr(U)))


def mcpt_td2(h, n_iter: int):
    """(per_dimer [D, 2] {E_J, E_K}, delta [n_iter])."""
    D = lib().mcpt_num_dimers(h)
    pd, dl = np.empty((D, 2)), np.empty(n_iter)
    _check(h, lib().mcpt_td2(h, n_iter, _ptr(pd), _ptr(dl)))
    return pd, dl


def mcpt_add_dimer_df(h, X: int, Y: int, B, naux: int, s: float, on_device: int) -> int:
    if isinstance(B, np.ndarray):
        B = np.ascontiguousarray(B, dtype=np.float64)
    out = ctypes.c_int()
    _check(h, lib().mcpt_add_dimer_df(h, X, Y, _ptr(B), naux, s, on_device, ctypes.byref(out)))
    return out.value


def mcpt_run_df(h) -> None:
    _check(h, lib().mcpt_run_df(h))


def mcpt_df_energies(h, n_df: int):
    """(per_monomer_J [N], per_monomer_K [N], per_dimer [n_df, 2], total [2])."""
    N = lib().mcpt_num_monomers(h)
    mj, mk = np.empty(N), np.empty(N)
    pd, tot = np.empty((n_df, 2)), np.empty(2)
    _check(h, lib().mcpt_df_energies(h, _ptr(mj), _ptr(mk), _ptr(pd), _ptr(tot)))
    return mj, mk, pd, tot


def mcpt_collect_stats(h) -> mcpt_run_stats:
    s = mcpt_run_stats()
    _check(h, lib().mcpt_collect_stats(h, ctypes.byref(s)))
    return s


def mcpt_last_error(h) -> str:
    return lib().mcpt_last_error(h).decode()


def mcpt_destroy(h) -> None:
    lib().mcpt_destroy(h)


def mcpt_dimer_fp64_noalloc(A, K, C_X, eps_X, nX, nocc_X, C_Y, eps_Y, nY, nocc_Y, E2, stream=None) -> None:
    """One dimer's FP64 {E_J, E_K} into the device buffer E2, allocating
    nothing (fixed 8 MiB scratch inside the library); all arrays are device
    buffers (torch CUDA tensors or addresses).  See include/mcpt.h for the
    limits and the rule that overlapping calls race."""
    st = lib().mcpt_dimer_fp64_noalloc(_ptr(A), _ptr(K), _ptr(C_X), _ptr(eps_X), nX, nocc_X, _ptr(C_Y),
                                       _ptr(eps_Y), nY, nocc_Y, _ptr(E2), stream)
    _check(None, st)


def mcpt_fp64_fma_rate(device: int = 0):
    """(TFLOP/s, ms per launch) of the device's FP64 FMA pipe, measured by the
    library's microbenchmark (the FP64 form's roofline denominator)."""
    t, ms = ctypes.c_double(), ctypes.c_double()
    _check(None, lib().mcpt_fp64_fma_rate(device, ctypes.byref(t), ctypes.byref(ms)))
    return t.value, ms.value


# ----------------------------------------------------------- convenience
class Context:
    """Owns one mcpt handle.  ``stream`` is a cudaStream_t as an int (e.g.
    ``torch.cuda.current_stream().cuda_stream``) or None for a library stream."""

    def __init__(self, precision="fp64", device=0, stream=None, validate=True, wave_bytes=0, timing=False,
                 mem_cap_bytes=0, graphs=True, tune_cache=None, coupling=False, wait_limit_ns=0, withhold_load=0,
                 fp64_epilogue=False):
        o = mcpt_default_options()
        if tune_cache is not None:
            o.tune_cache = os.fsencode(tune_cache)
        o.device = device
        o.stream = stream
        o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        o.validate = int(bool(validate))
        o.wave_bytes = wave_bytes
        o.timing = int(bool(timing))
        o.mem_cap_bytes = mem_cap_bytes
        o.graphs = int(bool(graphs))
        o.coupling = int(bool(coupling))
        o.wait_limit_ns = int(wait_limit_ns)
        o.withhold_load = int(withhold_load)
        o.fp64_epilogue = int(bool(fp64_epilogue))
        self.validate = bool(validate)
        self.stream = stream
        self.h = mcpt_create(o)

    def add_monomer(self, C, eps, nocc):
        C = np.asarray(C)
        return mcpt_add_monomer(self.h, C, eps, C.shape[0], nocc)

    def add_dimer(self, X, Y, ao_eri, layout=MCPT_AO_BLOCKS, on_device=None):
        if on_device is None:
            on_device = 0 if isinstance(ao_eri, np.ndarray) else 1
        return mcpt_add_dimer(self.h, X, Y, ao_eri, layout, on_device)

    def update_dimer(self, dimer, ao_eri, layout=MCPT_AO_BLOCKS, on_device=None, asynchronous=False):
        """New integrals for a registered dimer (stored order X < Y).  With
        asynchronous=True a host buffer is copied on the handle's stream and
        must stay unchanged until the next run completes."""
        if on_device is None:
            on_device = 0 if isinstance(ao_eri, np.ndarray) else 1
        mcpt_update_dimer(self.h, dimer, ao_eri, layout, on_device, MCPT_UPDATE_ASYNC if asynchronous else 0)

    def update_dimers(self, first, count, ao_eri, offsets, layout=MCPT_AO_PACKED, asynchronous=False):
        """New host integrals for dimers first .. first+count-1 in one call
        (dimer first+k's at element offsets[k] of ao_eri): back-to-back
        packed data goes over in large chunks."""
        mcpt_update_dimers(self.h, first, count, ao_eri, offsets, layout, MCPT_UPDATE_ASYNC if asynchronous else 0)

    def set_precision(self, p):
        mcpt_set_precision(self.h, PRECISIONS[p] if isinstance(p, str) else int(p))

    def run(self, first=None, count=None):
        if first is None:
            mcpt_run(self.h)
        else:
            mcpt_run_range(self.h, first, count)

    def energies(self):
        return mcpt_energies(self.h)

    def coupling(self, X, nao, nocc):
        """R_X of Eq. (tm2)'s dimer coupling, (nocc (nao - nocc))^2, after a run
        of a context created with coupling=True."""
        return mcpt_coupling(self.h, X, nocc * (nao - nocc))

    def singles(self, t):
        """Eq. (tm1)'s environment term s_X = sum_{Y,k,c} (ia|kc) t^c_k(Y) of
        every monomer, for amplitudes t = [t_X as (o_X, v_X)] in monomer id
        order, after a run of a context created with coupling=True; returns
        the list of s_X of the same shapes."""
        t = [np.asarray(x, dtype=np.float64) for x in t]
        flat = mcpt_singles(self.h, np.concatenate([x.ravel() for x in t]) if t else np.empty(0))
        out, off = [], 0
        for x in t:
            out.append(flat[off:off + x.size].reshape(x.shape))
            off += x.size
        return out

    def add_dimer_df(self, X, Y, B, naux, s=1.0, on_device=None):
        """Register dimer X-Y (X < Y) of the density-fitted route by its
        factors B[naux][n][n]; returns its id in that route's list."""
        if on_device is None:
            on_device = 0 if isinstance(B, np.ndarray) else 1
        i = mcpt_add_dimer_df(self.h, X, Y, B, naux, s, on_device)
        self.n_df = i + 1
        return i

    def run_df(self):
        mcpt_run_df(self.h)

    def df_energies(self):
        return mcpt_df_energies(self.h, getattr(self, "n_df", 0))

    def set_monomer_doubles(self, X, G=None, U=None):
        """Monomer X's ring matrix G and amplitude matrix U of Eq. (td2)."""
        mcpt_set_monomer_doubles(self.h, X, G, U)

    def td2(self, n_iter):
        """Eq. (td2) by n_iter Jacobi steps for every dimer: (per-dimer
        {E_J, E_K} at the final amplitudes, per-step max |dT|)."""
        return mcpt_td2(self.h, n_iter)

    def stats(self):
        """Timing and launch counts of the runs since the previous call."""
        return mcpt_collect_stats(self.h)

    def close(self):
        if self.h:
            mcpt_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
