"""Shared helpers for the GPU tests: build a library context from a workload
and compute oracle references on the same host inputs."""
from __future__ import annotations

import functools

import numpy as np

import oracle
import synth


@functools.lru_cache(maxsize=None)
def host_workload(name: str, dimers: tuple | None = None):
    """(workload, monomers, {d: (A, K)}, oracle E [len(dimers), 2]) on host inputs."""
    w = synth.workload(name)
    ds = tuple(range(w.n_dimers)) if dimers is None else dimers
    mons = {}
    blocks = {}
    items = []
    for d in ds:
        X, Y = w.pairs[d]
        for m in (X, Y):
            if m not in mons:
                mons[m] = w.monomer(m)
        blocks[d] = w.blocks(d)
        mX, mY = mons[X], mons[Y]
        items.append((*blocks[d], mX.C, mX.eps, mY.C, mY.eps, mX.nocc, mY.nocc))
    E = oracle.dimers_parallel(items)
    return w, mons, blocks, E


def load_context(ctx, w, mons, blocks, dimers):
    """Register every monomer of w (ids = workload ids) and the listed dimers
    (host BLOCKS layout).  Returns the library dimer ids."""
    for X in range(w.n_monomers):
        m = mons.get(X)
        if m is None:
            m = w.monomer(X)
        ctx.add_monomer(m.C, m.eps, m.nocc)
    ids = []
    import paper_1409_2700_gb300 as M
    for d in dimers:
        X, Y = w.pairs[d]
        A, K = blocks[d]
        ids.append(ctx.add_dimer(X, Y, np.concatenate([A.ravel(), K.ravel()]), M.MCPT_AO_BLOCKS))
    return ids


def rand_dimer(rng, nX, nY, oX, oY):
    """Non-symmetric random blocks and orthonormal C (so any axis mix-up shows)."""
    A = rng.standard_normal((nX, nX, nY, nY)) * 1e-3
    K = rng.standard_normal((nX, nY, nY, nX)) * 1e-3
    CX = np.linalg.qr(rng.standard_normal((nX, nX)))[0]
    CY = np.linalg.qr(rng.standard_normal((nY, nY)))[0]
    eX = np.concatenate([np.sort(rng.uniform(-1.5, -0.5, oX)), np.sort(rng.uniform(0.2, 3.0, nX - oX))])
    eY = np.concatenate([np.sort(rng.uniform(-1.5, -0.5, oY)), np.sort(rng.uniform(0.2, 3.0, nY - oY))])
    return A, K, CX, eX, CY, eY
