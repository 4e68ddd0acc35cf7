"""Failure detection on the GPU without a device fault (marked gpu).

Every wait of the tensor-core kernels is bounded.  Here a context is made
with a 2 ms wait limit and the test aid withhold_load: the first CTA's TMA
producer stops issuing integral loads, so its converter warps wait for a
load that never comes.  They give up at the limit, the CTA drains its own
copies and MMAs, frees its tensor memory and returns, and mcpt_energies
reports MCPT_ETIMEOUT.  No kernel traps or hangs.  A fresh context on the
same GPU afterwards runs the same dimers to the oracle's values, which shows
that nothing was left waiting and the tensor memory was released.
"""
import numpy as np
import pytest

from helpers import host_workload, load_context

pytestmark = pytest.mark.gpu

M = pytest.importorskip("paper_1409_2700_gb300")


@pytest.mark.parametrize("prec,withhold", [("tf32", 1), ("bf16x2", 40), ("bf16x3", 7)])
def test_wait_limit_gives_up_and_gpu_stays_usable(prec, withhold):
    w, mons, blocks, E = host_workload("lattice-2x2x2")
    ds = list(range(w.n_dimers))
    for graphs in (False, True):
        with M.Context(precision=prec, wait_limit_ns=2_000_000, withhold_load=withhold, graphs=graphs) as ctx:
            load_context(ctx, w, mons, blocks, ds)
            ctx.run()
            with pytest.raises(M.McptError) as ei:
                ctx.energies()
            assert ei.value.status == M.MCPT_ETIMEOUT
            assert "gave up" in M.mcpt_last_error(ctx.h)
    # a fresh context on the same GPU: the oracle's values
    with M.Context(precision=prec) as ctx:
        load_context(ctx, w, mons, blocks, ds)
        ctx.run()
        _, _, pd, _ = ctx.energies()
    assert np.all(np.abs(pd[:, 0] - E[:, 0]) <= 5e-5 * np.abs(E[:, 0]))


def test_wait_limit_alone_changes_nothing():
    """A short limit without the test aid: every wait completes in time and
    the energies are those of the default limit, bit for bit."""
    w, mons, blocks, E = host_workload("lattice-2x2x2")
    ds = list(range(w.n_dimers))
    out = []
    for lim in (0, 500_000_000):
        with M.Context(precision="bf16x2", wait_limit_ns=lim) as ctx:
            load_context(ctx, w, mons, blocks, ds)
            ctx.run()
            out.append(ctx.energies()[2])
    assert np.array_equal(out[0], out[1])


def test_negative_withhold_is_rejected():
    with pytest.raises(M.McptError) as ei:
        M.Context(precision="tf32", withhold_load=-1)
    assert ei.value.status == M.MCPT_EINVAL
