"""The mixed forms' energy epilogue on FP32 pairs against the same epilogue on
the FP64 pipe (mcpt_options.fp64_epilogue), through the C ABI.

Both runs share the first half and the virtual quarter transformations bit
for bit, so the per-dimer terms differ only by the epilogue's own rounding:
D = 1/(e_i + e_j - e_a - e_b) to ~2^-45 relative in either (an FP32-pair
Newton step, or one FP64 Newton step from an FP32 seed), exact or FP64
products with D, and sums that keep ~2^-45 per pair of the (pair, a) partials.
Per dimer the two agree to a few times 1e-13 relative; the bound below is
2e-12 |E_J|, three orders under the closest parity bound of any mixed form
(1e-7 on lattice dimers), so a wrong denominator, a dropped low part or a
lost compensation term in either epilogue fails it.  Both monomer-size paths
(<= 32 AO, one warp per pair; larger, register-tiled) and the coupling store
are covered.
"""
import numpy as np
import pytest

import synth
from helpers import host_workload, load_context

pytestmark = pytest.mark.gpu

M = pytest.importorskip("paper_1409_2700_gb300")

MIXED = ["fp32c", "bf16x3", "bf16x2", "tf32"]
TOL = 2e-12


@pytest.fixture(scope="module")
def lat8():
    return host_workload("lattice-2x2x2")


def _energies(prec, fp64_epilogue, load, coupling=False, monomers=()):
    with M.Context(precision=prec, fp64_epilogue=fp64_epilogue, coupling=coupling) as ctx:
        load(ctx)
        ctx.run()
        out = ctx.energies()
        R = [ctx.coupling(*m) for m in monomers] if coupling else []
    return out, R


def _check_pd(pd_ff, pd_64, what):
    scale = np.abs(pd_64[:, 0])
    dJ = np.abs(pd_ff[:, 0] - pd_64[:, 0]) / scale
    dK = np.abs(pd_ff[:, 1] - pd_64[:, 1]) / scale
    print(f"{what}: FP32-pair vs FP64-pipe epilogue, max rel diff J {dJ.max():.2e} K {dK.max():.2e}")
    assert np.all(dJ <= TOL), what
    assert np.all(dK <= TOL), what
    # not the same computation: the two must not coincide everywhere by accident
    assert np.any(pd_ff != pd_64), what


@pytest.mark.parametrize("prec", MIXED)
def test_pairs_epilogue_matches_fp64_pipe_lattice(lat8, prec):
    w, mons, blocks, _ = lat8
    load = lambda ctx: load_context(ctx, w, mons, blocks, range(w.n_dimers))
    (mj_a, mk_a, pd_a, tot_a), _ = _energies(prec, False, load)
    (mj_b, mk_b, pd_b, tot_b), _ = _energies(prec, True, load)
    _check_pd(pd_a, pd_b, f"{prec} lattice-2x2x2")
    assert abs(tot_a[0] - tot_b[0]) <= TOL * abs(tot_b[0])
    assert abs(tot_a[1] - tot_b[1]) <= TOL * abs(tot_b[0])
    assert np.all(np.abs(mj_a - mj_b) <= TOL * np.abs(mj_b))


@pytest.mark.parametrize("prec", MIXED)
def test_pairs_epilogue_matches_fp64_pipe_tiled(prec):
    """Monomers of 16..56 AO: waves with monomers above 32 AO take the
    register-tiled second half, whose per-thread 8 x 4 blocks carry the
    pair sums."""
    w = synth.workload("uneven-4096")
    ds = [k for k in range(200) if w.nao[2 * k] <= 56 and w.nao[2 * k + 1] <= 56][:10]
    assert max(max(w.nao[2 * k], w.nao[2 * k + 1]) for k in ds) > 32

    def load(ctx):
        for k, d in enumerate(ds):
            X, Y = w.pairs[d]
            mX, mY = w.monomer(X), w.monomer(Y)
            ctx.add_monomer(mX.C, mX.eps, mX.nocc)
            ctx.add_monomer(mY.C, mY.eps, mY.nocc)
            A, K = w.blocks(d)
            ctx.add_dimer(2 * k, 2 * k + 1, np.concatenate([A.ravel(), K.ravel()]))

    (_, _, pd_a, _), _ = _energies(prec, False, load)
    (_, _, pd_b, _), _ = _energies(prec, True, load)
    _check_pd(pd_a, pd_b, f"{prec} uneven 16..56 AO")


@pytest.mark.parametrize("prec", ["bf16x2", "fp32c"])
def test_pairs_epilogue_with_coupling_store(lat8, prec):
    """With the coupling on, the second half also stores T = vD (FP32) per
    term: both epilogues round the same v D to FP32 once, so the coupling
    matrices agree to a few FP32 ulps, and the energies as above."""
    w, mons, blocks, _ = lat8
    load = lambda ctx: load_context(ctx, w, mons, blocks, range(w.n_dimers))
    ms = [(X, w.nao[X], w.nocc[X]) for X in range(w.n_monomers)]
    (_, _, pd_a, _), Ra = _energies(prec, False, load, coupling=True, monomers=ms)
    (_, _, pd_b, _), Rb = _energies(prec, True, load, coupling=True, monomers=ms)
    _check_pd(pd_a, pd_b, f"{prec} lattice-2x2x2 with coupling")
    for X, (a, b) in enumerate(zip(Ra, Rb)):
        scale = np.abs(b).max()
        assert np.abs(a - b).max() <= 1e-6 * scale, X
