"""FP64 CPU oracle for the first-order MCPT(2) dimer term -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline and
reference legs may import this package.  The library never does: it has no CPU
fallback.  The arithmetic lives in ``oracle.c`` (plain C, FP64), which shares
nothing with the CUDA path; this file only compiles it and marshals arrays.

Functions and the passages they follow (Byrd et al., MCPT I):
  transform_J   (i a|j b), Eq. (dp2e), factorised quarter transforms
  transform_K   (i b|j a), the exchange-type form from the (XY|YX) block
  bruteforce_J/K  Eq. (dp2e) summed literally, n^8 (pins the factorisation)
  factor_route  (ia|jb) and (ib|ja) from integral factors B^Q (other arithmetic)
  energy_from_mo  Eq. (ed2) with T = vD and D = 1/eps^{ij}_{ab} (Sec. II.C);
                  E_K = -2 sum (ia|jb)(ib|ja) D (exchange completion)
  dimer         the two transforms plus the energies for one dimer
  accumulate    half-and-half per-monomer split, Neumaier lattice total
  coupling_add  dimer -> monomer doubles coupling of Eq. (tm2) (the c, k sum
                over the neighbour) at the first-order dimer amplitude T = vD

Parity unpinned: the half/half per-monomer split (only its sum is pinned) and
the inclusion and scale of E_K (a reading of the paper, pinned only by the
rank-1 closed form that shares that reading).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, OpenMP over dimers)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11",
                        "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            I, D = ctypes.c_int, ctypes.c_double
            for name in ("oracle_transform_J", "oracle_transform_K"):
                getattr(L, name).argtypes = [_dp, _dp, _dp, I, I, I, I, _dp]
                getattr(L, name).restype = I
            for name in ("oracle_bruteforce_J", "oracle_bruteforce_K"):
                getattr(L, name).argtypes = [_dp, _dp, _dp, I, I, I, I, _dp]
                getattr(L, name).restype = None
            L.oracle_energy_from_mo.argtypes = [_dp, _dp, _dp, _dp, I, I, I, I, _dp, _dp]
            L.oracle_energy_from_mo.restype = None
            L.oracle_dimer.argtypes = [_dp, _dp, _dp, _dp, _dp, _dp, I, I, I, I, _dp]
            L.oracle_dimer.restype = I
            L.oracle_factor_route.argtypes = [_dp, I, D, _dp, _dp, I, I, I, I, _dp, _dp]
            L.oracle_factor_route.restype = I
            L.oracle_accumulate.argtypes = [_dp, ctypes.POINTER(I), ctypes.POINTER(I), I, I, _dp, _dp]
            L.oracle_accumulate.restype = None
            pp = ctypes.POINTER(_dp)
            ip = ctypes.POINTER(I)
            L.oracle_dimers.argtypes = [I, pp, pp, pp, pp, pp, pp, ip, ip, ip, ip, _dp]
            L.oracle_dimers.restype = I
            L.oracle_coupling_add.argtypes = [_dp, _dp, _dp, I, I, I, I, _dp, _dp]
            L.oracle_coupling_add.restype = None
            L.oracle_singles_add.argtypes = [_dp, _dp, _dp, I, I, I, I, _dp, _dp]
            L.oracle_singles_add.restype = None
            L.oracle_td2.argtypes = [_dp, _dp, _dp, _dp, _dp, _dp, I, I, I, I, _dp, _dp, _dp, _dp, I,
                                     _dp, _dp, _dp]
            L.oracle_td2.restype = I
            L.oracle_max_threads.argtypes = []
            L.oracle_max_threads.restype = I
            _lib = L
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a):
    return a.ctypes.data_as(_dp)


def _shape_mo(nX, nY, oX, oY):
    return (oX, nX - oX, oY, nY - oY), (oX, nY - oY, oY, nX - oX)


def transform_J(A, CX, CY, oX, oY):
    A, CX, CY = _f64(A), _f64(CX), _f64(CY)
    nX, nY = CX.shape[0], CY.shape[0]
    V = np.empty(_shape_mo(nX, nY, oX, oY)[0])
    if lib().oracle_transform_J(_p(A), _p(CX), _p(CY), nX, nY, oX, oY, _p(V)):
        raise MemoryError("oracle_transform_J")
    return V


def transform_K(K, CX, CY, oX, oY):
    K, CX, CY = _f64(K), _f64(CX), _f64(CY)
    nX, nY = CX.shape[0], CY.shape[0]
    W = np.empty(_shape_mo(nX, nY, oX, oY)[1])
    if lib().oracle_transform_K(_p(K), _p(CX), _p(CY), nX, nY, oX, oY, _p(W)):
        raise MemoryError("oracle_transform_K")
    return W


def bruteforce_J(A, CX, CY, oX, oY):
    A, CX, CY = _f64(A), _f64(CX), _f64(CY)
    nX, nY = CX.shape[0], CY.shape[0]
    V = np.empty(_shape_mo(nX, nY, oX, oY)[0])
    lib().oracle_bruteforce_J(_p(A), _p(CX), _p(CY), nX, nY, oX, oY, _p(V))
    return V


def bruteforce_K(K, CX, CY, oX, oY):
    K, CX, CY = _f64(K), _f64(CX), _f64(CY)
    nX, nY = CX.shape[0], CY.shape[0]
    W = np.empty(_shape_mo(nX, nY, oX, oY)[1])
    lib().oracle_bruteforce_K(_p(K), _p(CX), _p(CY), nX, nY, oX, oY, _p(W))
    return W


def energy_from_mo(V, W, epsX, epsY, oX, oY):
    V, W, epsX, epsY = _f64(V), _f64(W), _f64(epsX), _f64(epsY)
    nX, nY = epsX.shape[0], epsY.shape[0]
    ej, ek = ctypes.c_double(), ctypes.c_double()
    lib().oracle_energy_from_mo(_p(V), _p(W), _p(epsX), _p(epsY), nX, nY, oX, oY,
                                ctypes.byref(ej), ctypes.byref(ek))
    return ej.value, ek.value


def dimer(A, K, CX, epsX, CY, epsY, oX, oY):
    """(E_J, E_K) of one dimer from its A = (XX|YY) and K = (XY|YX) blocks."""
    A, K, CX, CY, epsX, epsY = (_f64(x) for x in (A, K, CX, CY, epsX, epsY))
    nX, nY = CX.shape[0], CY.shape[0]
    E = np.empty(2)
    if lib().oracle_dimer(_p(A), _p(K), _p(CX), _p(epsX), _p(CY), _p(epsY), nX, nY, oX, oY, _p(E)):
        raise MemoryError("oracle_dimer")
    return float(E[0]), float(E[1])


def factor_route(B, s, CX, CY, oX, oY):
    B, CX, CY = _f64(B), _f64(CX), _f64(CY)
    nX, nY = CX.shape[0], CY.shape[0]
    sV, sW = _shape_mo(nX, nY, oX, oY)
    V, W = np.empty(sV), np.empty(sW)
    if lib().oracle_factor_route(_p(B), B.shape[0], float(s), _p(CX), _p(CY), nX, nY, oX, oY, _p(V), _p(W)):
        raise MemoryError("oracle_factor_route")
    return V, W


def coupling_add(V, epsX, epsY, oX, oY, RX, RY):
    """Add one dimer's coupling to R_X ((oX vX)^2) and R_Y ((oY vY)^2), in place.
    V: (ia|jb) as [oX][vX][oY][vY] (transform_J's layout)."""
    V, epsX, epsY = _f64(V), _f64(epsX), _f64(epsY)
    for R in (RX, RY):
        assert R.dtype == np.float64 and R.flags.c_contiguous
    nX, nY = epsX.shape[0], epsY.shape[0]
    lib().oracle_coupling_add(_p(V), _p(epsX), _p(epsY), nX, nY, oX, oY, _p(RX), _p(RY))


def singles_add(V, tX, tY, sX, sY):
    """Add one dimer's singles environment term of Eq. (tm1) to sX ([oX][vX])
    and sY ([oY][vY]), in place.  V: (ia|kc) as [oX][vX][oY][vY]; tX, tY:
    the monomers' singles amplitudes t^a_i as [o][v]."""
    V, tX, tY = _f64(V), _f64(tX), _f64(tY)
    oX, vX, oY, vY = V.shape
    assert tX.shape == (oX, vX) and tY.shape == (oY, vY)
    for s in (sX, sY):
        assert s.dtype == np.float64 and s.flags.c_contiguous
    assert sX.shape == (oX, vX) and sY.shape == (oY, vY)
    lib().oracle_singles_add(_p(V), _p(tX), _p(tY), oX, vX, oY, vY, _p(sX), _p(sY))


def singles_lattice(w, t, dimers=None, blocks=None):
    """The singles environment term of every monomer of workload w over the
    listed dimers (default all), for amplitudes t = {X: [oX][vX]}: {X: s_X}."""
    ds = range(w.n_dimers) if dimers is None else dimers
    mons, S = {}, {}
    for d in ds:
        X, Y = w.pairs[d]
        for m in (X, Y):
            if m not in mons:
                mons[m] = w.monomer(m)
                S[m] = np.zeros((w.nocc[m], w.nao[m] - w.nocc[m]))
        mX, mY = mons[X], mons[Y]
        A = blocks[d][0] if blocks is not None else w.blocks(d)[0]
        V = transform_J(A, mX.C, mY.C, mX.nocc, mY.nocc)
        singles_add(V, t[X], t[Y], S[X], S[Y])
    return S


def td2(A, K, CX, epsX, CY, epsY, oX, oY, n_iter, GX=None, GY=None, UX=None, UY=None):
    """Eq. (td2) dimer amplitudes after n_iter Jacobi steps from zero and the
    energies at them: (T [oX][vX][oY][vY], (E_J, E_K), per-step max |dT|).
    GX, GY: monomer ring matrices, UX, UY: monomer amplitude matrices
    (2T - T'), each (o v) x (o v) or None (zero)."""
    A, K, CX, CY = _f64(A), _f64(K), _f64(CX), _f64(CY)
    epsX, epsY = _f64(epsX), _f64(epsY)
    nX, nY = CX.shape[0], CY.shape[0]
    T = np.empty(_shape_mo(nX, nY, oX, oY)[0])
    E = np.empty(2)
    delta = np.empty(max(n_iter, 1))
    opt = [None if M is None else _f64(M) for M in (GX, GY, UX, UY)]
    ptrs = [None if M is None else _p(M) for M in opt]
    if lib().oracle_td2(_p(A), _p(K), _p(CX), _p(epsX), _p(CY), _p(epsY), nX, nY, oX, oY,
                        *ptrs, n_iter, _p(T), _p(E), _p(delta)):
        raise MemoryError("oracle_td2")
    return T, (E[0], E[1]), delta[:n_iter]


def coupling_lattice(w, dimers=None, blocks=None):
    """R_X of every monomer of workload w over the listed dimers (default all),
    from host inputs: {X: R_X}.  `blocks` may hold precomputed {d: (A, K)}."""
    ds = range(w.n_dimers) if dimers is None else dimers
    mons, R = {}, {}
    for d in ds:
        X, Y = w.pairs[d]
        for m in (X, Y):
            if m not in mons:
                mons[m] = w.monomer(m)
                n, o = w.nao[m], w.nocc[m]
                R[m] = np.zeros(((o * (n - o)), (o * (n - o))))
        mX, mY = mons[X], mons[Y]
        A = blocks[d][0] if blocks is not None else w.blocks(d)[0]
        V = transform_J(A, mX.C, mY.C, mX.nocc, mY.nocc)
        coupling_add(V, mX.eps, mY.eps, mX.nocc, mY.nocc, R[X], R[Y])
    return R


def accumulate(E2, X, Y, nmon):
    """Per-monomer {J, K} halves and the lattice totals (Neumaier)."""
    E2 = _f64(E2).reshape(-1, 2)
    X = np.ascontiguousarray(X, dtype=np.int32)
    Y = np.ascontiguousarray(Y, dtype=np.int32)
    mon = np.empty((nmon, 2))
    tot = np.empty(2)
    ip = ctypes.POINTER(ctypes.c_int)
    lib().oracle_accumulate(_p(E2), X.ctypes.data_as(ip), Y.ctypes.data_as(ip), E2.shape[0], nmon,
                            _p(mon), _p(tot))
    return mon, tot


def dimers_parallel(items):
    """items: list of (A, K, CX, epsX, CY, epsY, oX, oY); OpenMP over dimers.
    Returns an (nd, 2) array of {E_J, E_K}."""
    nd = len(items)
    keep = []
    arrs = [[] for _ in range(6)]
    for it in items:
        for k in range(6):
            a = _f64(it[k])
            keep.append(a)
            arrs[k].append(_p(a))
    P = [(_dp * nd)(*a) for a in arrs]
    I = ctypes.c_int * nd
    nX = I(*[int(np.asarray(it[2]).shape[0]) for it in items])
    nY = I(*[int(np.asarray(it[4]).shape[0]) for it in items])
    oX = I(*[int(it[6]) for it in items])
    oY = I(*[int(it[7]) for it in items])
    E = np.empty((nd, 2))
    if lib().oracle_dimers(nd, *P, nX, nY, oX, oY, _p(E)):
        raise MemoryError("oracle_dimers")
    return E


def max_threads() -> int:
    return int(lib().oracle_max_threads())
