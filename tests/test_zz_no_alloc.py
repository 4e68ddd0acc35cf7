"""The allocation-free entry point (mcpt_dimer_fp64_noalloc) against the CPU
oracle and the handle-based path.  It is for callers that may not allocate
device memory; its scratch is a fixed array inside the library, shared by
every call, so this test makes several calls in a row with different dimers
and checks each result -- a call that read leftovers of the previous one
would show.  This file is collected last on purpose."""
import numpy as np
import pytest

import oracle
import synth
from helpers import rand_dimer

pytestmark = pytest.mark.gpu

M = pytest.importorskip("paper_1409_2700_gb300")

TOL = 1e-12   # the FP64 form's per-dimer tolerance used by the parity tests


def _existing(A, K, CX, eX, CY, eY, oX, oY):
    with M.Context(precision="fp64") as ctx:
        ctx.add_monomer(CX, eX, oX)
        ctx.add_monomer(CY, eY, oY)
        ctx.add_dimer(0, 1, np.concatenate([A.ravel(), K.ravel()]), M.MCPT_AO_BLOCKS)
        ctx.run()
        return ctx.energies()[2][0]


def _noalloc(torch, A, K, CX, eX, CY, eY, oX, oY):
    dev = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in (A, K, CX, eX, CY, eY)]
    E2 = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    M.mcpt_dimer_fp64_noalloc(dev[0], dev[1], dev[2], dev[3], CX.shape[0], oX, dev[4], dev[5], CY.shape[0], oY,
                              E2, stream)
    torch.cuda.current_stream().synchronize()
    return E2.cpu().numpy()


def test_noalloc_matches_oracle_on_consecutive_calls():
    torch = pytest.importorskip("torch")
    w = synth.workload("lattice-2x2x2")
    cases = []
    for d in (0, 20):
        X, Y = w.pairs[d]
        mX, mY = w.monomer(X), w.monomer(Y)
        A, K = w.blocks(d)
        cases.append((A, K, mX.C, mX.eps, mY.C, mY.eps, mX.nocc, mY.nocc))
    rng = np.random.default_rng(21)
    cases.append((*rand_dimer(rng, 7, 12, 3, 2), 3, 2))     # small, odd, non-symmetric
    cases.append((*rand_dimer(rng, 96, 20, 7, 3), 7, 3))    # 96 AO: the second half's shared-memory limit
    refs = [oracle.dimer(*c) for c in cases]
    # two rounds over all cases: every call follows one with other sizes
    for _ in range(2):
        for c, ref in zip(cases, refs):
            got = _noalloc(torch, *c)
            assert abs(got[0] - ref[0]) <= TOL * abs(ref[0]), (got, ref)
            assert abs(got[1] - ref[1]) <= TOL * abs(ref[0]), (got, ref)
    # and the handle-based FP64 path agrees on the same inputs
    for c, ref in zip(cases[:3], refs):
        got = _existing(*c)
        assert abs(got[0] - ref[0]) <= TOL * abs(ref[0]), (got, ref)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    # 2 * 96 * 96 * 16 * 16 doubles > the fixed 1048576
    with pytest.raises(M.McptError) as ei:
        M.mcpt_dimer_fp64_noalloc(buf, buf, buf, buf, 96, 16, buf, buf, 96, 16, buf)
    assert ei.value.status == M.MCPT_EINVAL
    assert "scratch" in M.mcpt_last_error(None)
    with pytest.raises(M.McptError) as ei:
        M.mcpt_dimer_fp64_noalloc(buf, buf, buf, buf, 128, 5, buf, buf, 32, 5, buf)
    assert ei.value.status == M.MCPT_EINVAL
    # a following valid call clears the message
    rng = np.random.default_rng(22)
    A, K, CX, eX, CY, eY = rand_dimer(rng, 6, 5, 2, 2)
    got = _noalloc(torch, A, K, CX, eX, CY, eY, 2, 2)
    assert np.all(np.isfinite(got))
    assert M.mcpt_last_error(None) == ""
