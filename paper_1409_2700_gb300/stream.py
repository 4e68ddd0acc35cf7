"""Dimer lists larger than device memory, run in waves through one context.

A lattice whose AO blocks do not fit on the device at once (42,092 dimers of
16.8 MB each, or 3,258 dimers of 4.3 GB each) runs wave by wave.  Every dimer
is registered once, in list order, with a device address inside one reusable
wave buffer; before each wave runs (``mcpt_run_range`` over its dimers) the
caller's producer writes that wave's integral blocks [A | K] (BLOCKS layout)
at those addresses.  Per-dimer terms and per-monomer sums accumulate in the
context as for any other run and are complete once every wave has run.

The context must be created with ``validate=False``: with validation the
library checks device integrals when they are registered, before any
producer has written them.
"""
from __future__ import annotations

from dataclasses import dataclass

MCPT_AO_BLOCKS = 1
_ALIGN = 32          # elements (256 bytes) between consecutive dimers' blocks


def block_elems(nX: int, nY: int) -> int:
    """FP64 elements of one dimer's [A | K] blocks."""
    return 2 * nX * nX * nY * nY


def plan_waves(elems, budget_elems: int):
    """Split the list (in order) into waves whose blocks fit `budget_elems`.
    Returns (waves, offsets): waves = [(first, count)], offsets[d] = element
    offset of dimer d inside the wave buffer (256-byte aligned)."""
    waves, offs = [], [0] * len(elems)
    first, used = 0, 0
    for d, n in enumerate(elems):
        step = (n + _ALIGN - 1) // _ALIGN * _ALIGN
        if step > budget_elems:
            raise ValueError(f"dimer {d} needs {n * 8} bytes, more than the wave budget {budget_elems * 8}")
        if used + step > budget_elems and d > first:
            waves.append((first, d - first))
            first, used = d, 0
        offs[d] = used
        used += step
    if elems:
        waves.append((first, len(elems) - first))
    return waves, offs


@dataclass
class WaveView:
    dimer: int       # index in the list (= library dimer id)
    X: int
    Y: int
    out: object      # 1-D FP64 device tensor of block_elems(nX, nY) elements


class Streamed:
    """Registers `pairs` (X < Y; monomers already added with sizes `nao`) in
    every context of `ctxs`, all pointing into one wave buffer of at most
    `budget_bytes` on `device`.  Give the contexts the stream the producer
    writes on (``stream=torch.cuda.current_stream().cuda_stream``) so that
    filling and running a wave stay ordered without host waits."""

    def __init__(self, ctxs, pairs, nao, budget_bytes: int, device="cuda"):
        import torch
        self.ctxs = list(ctxs) if isinstance(ctxs, (list, tuple)) else [ctxs]
        for c in self.ctxs:
            if getattr(c, "validate", False):
                raise ValueError("streamed runs need contexts created with validate=False")
        self.pairs = list(pairs)
        self.elems = [block_elems(nao[X], nao[Y]) for X, Y in self.pairs]
        self.waves, self.offs = plan_waves(self.elems, budget_bytes // 8)
        need = 0
        for first, count in self.waves:
            last = first + count - 1
            need = max(need, self.offs[last] + self.elems[last])
        self.buf = torch.empty(need, dtype=torch.float64, device=device)
        base = self.buf.data_ptr()
        for c in self.ctxs:
            for d, (X, Y) in enumerate(self.pairs):
                if c.add_dimer(X, Y, base + 8 * self.offs[d], MCPT_AO_BLOCKS, on_device=1) != d:
                    raise ValueError("streamed runs need contexts with no dimers registered before")

    def __len__(self):
        return len(self.waves)

    def views(self, k: int):
        """The wave's dimers with the buffer slices their producer fills."""
        first, count = self.waves[k]
        out = []
        for d in range(first, first + count):
            X, Y = self.pairs[d]
            out.append(WaveView(d, X, Y, self.buf[self.offs[d]:self.offs[d] + self.elems[d]]))
        return out

    def run(self, k: int, ctxs=None):
        """Enqueue wave k's dimers in each context (asynchronous, on its
        stream).  The buffer must not be refilled until those runs complete."""
        first, count = self.waves[k]
        for c in (self.ctxs if ctxs is None else ctxs):
            c.run(first, count)
