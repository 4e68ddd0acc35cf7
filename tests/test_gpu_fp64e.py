"""The FP64-emulating tensor-core form (MCPT_FP64E) against the FP64 oracle
and the FP64 form, through the C ABI (all marked gpu).

Tolerance, from the arithmetic.  Each integral row chunk (32 p2 values of one
p0) and each C_Y column is held in 48-bit fixed point relative to its largest
power of two (floor: at most 2^-47 of it dropped per element), cut into six
byte digits; the tensor cores sum the digit products exactly and the seven
levels kept (0-6) leave out products below 2^-48 of the vectors' scale.  A
unit's T = sum_p2 x c is then within ~2^-45 of max|x| max|c| (the host model
of the digit scheme measures 2^-45.2 at worst over 500 random chunks of wide
dynamic range), and the FP32-pair steps after it (level combination, the p0
quarter transformation, H) each add ~2^-45 relative.  Per dimer that is
~1e-13 of |E_J| for lattice dimers (many terms, errors that average); the
bound below is the FP64 form's 1e-12 |E_J|, and 5e-12 for the few-term
random cases whose energies are sums of a handful of terms.  The lattice
target is the FP64 form's 1e-8 Eh; at these sizes it is held to 1e-10 Eh.
"""
import numpy as np
import pytest

import oracle
from helpers import host_workload, load_context, rand_dimer

pytestmark = pytest.mark.gpu

M = pytest.importorskip("paper_1409_2700_gb300")

PER_DIMER_LATTICE = 1e-12
PER_DIMER_RANDOM = 5e-12


@pytest.fixture(scope="module")
def lat8():
    return host_workload("lattice-2x2x2")


def _one(A, K, CX, eX, CY, eY, oX, oY, prec="fp64e"):
    with M.Context(precision=prec) as ctx:
        ctx.add_monomer(CX, eX, oX)
        ctx.add_monomer(CY, eY, oY)
        ctx.add_dimer(0, 1, np.concatenate([A.ravel(), K.ravel()]), M.MCPT_AO_BLOCKS)
        ctx.run()
        return ctx.energies()[2][0]


def test_fp64e_lattice_2x2x2(lat8):
    w, mons, blocks, E = lat8
    with M.Context(precision="fp64e") as ctx:
        load_context(ctx, w, mons, blocks, range(w.n_dimers))
        ctx.run()
        mj, mk, pd, tot = ctx.energies()
    scale = np.abs(E[:, 0])
    rJ = np.abs(pd[:, 0] - E[:, 0]) / scale
    rK = np.abs(pd[:, 1] - E[:, 1]) / scale
    print(f"fp64e lattice-2x2x2: max rel err J {rJ.max():.2e} K {rK.max():.2e}")
    assert np.all(rJ <= PER_DIMER_LATTICE) and np.all(rK <= PER_DIMER_LATTICE)
    omon, otot = oracle.accumulate(E, [p[0] for p in w.pairs], [p[1] for p in w.pairs], w.n_monomers)
    print(f"fp64e lattice E_J {tot[0]:.15e} oracle {otot[0]:.15e} diff {tot[0] - otot[0]:.2e} Eh")
    assert abs(tot[0] - otot[0]) <= 1e-10 and abs(tot[1] - otot[1]) <= 1e-10
    assert np.all(np.abs(mj - omon[:, 0]) <= 1e-10) and np.all(np.abs(mk - omon[:, 1]) <= 1e-10)


def test_fp64e_random_blocks():
    """Non-symmetric random integrals (only the literal index mapping of
    Eq. (dp2e) matches the oracle) over the form's size range: one and two
    p2 chunks, ragged last chunks, occupations 1-5 on either side."""
    rng = np.random.default_rng(23)
    cases = [(6, 10, 2, 3), (14, 8, 3, 1), (32, 32, 5, 5), (40, 24, 5, 4), (16, 64, 3, 5), (64, 16, 5, 3),
             (24, 50, 4, 5), (64, 64, 5, 5), (4, 6, 1, 5), (6, 4, 5, 1), (2, 2, 1, 1)]
    worst = 0.0
    for nX, nY, oX, oY in cases:
        A, K, CX, eX, CY, eY = rand_dimer(rng, nX, nY, oX, oY)
        ref = oracle.dimer(A, K, CX, eX, CY, eY, oX, oY)
        got = _one(A, K, CX, eX, CY, eY, oX, oY)
        s = abs(ref[0])
        err = max(abs(got[0] - ref[0]), abs(got[1] - ref[1])) / s
        worst = max(worst, err)
        assert err <= PER_DIMER_RANDOM, (nX, nY, oX, oY, got, ref, err)
    print(f"fp64e random blocks: max rel err {worst:.2e}")


def test_fp64e_wide_dynamic_range():
    """Integrals spanning 12 decades inside every row chunk: the fixed point
    of a chunk follows its largest element, the small ones keep what lies
    above 2^-47 of it -- their contribution to the energy stays within the
    bound because it scales with the chunk's largest."""
    rng = np.random.default_rng(29)
    nX, nY, oX, oY = 32, 40, 5, 4
    A, K, CX, eX, CY, eY = rand_dimer(rng, nX, nY, oX, oY)
    A = A * 10.0 ** rng.uniform(-12, 0, A.shape)
    K = K * 10.0 ** rng.uniform(-12, 0, K.shape)
    ref = oracle.dimer(A, K, CX, eX, CY, eY, oX, oY)
    got = _one(A, K, CX, eX, CY, eY, oX, oY)
    err = max(abs(got[0] - ref[0]), abs(got[1] - ref[1])) / abs(ref[0])
    print(f"fp64e wide dynamic range: rel err {err:.2e}")
    assert err <= PER_DIMER_RANDOM


def test_fp64e_zero_integrals_give_zero():
    rng = np.random.default_rng(31)
    A, K, CX, eX, CY, eY = rand_dimer(rng, 8, 6, 2, 2)
    got = _one(np.zeros_like(A), np.zeros_like(K), CX, eX, CY, eY, 2, 2)
    assert got[0] == 0.0 and got[1] == 0.0


def test_fp64e_matches_fp64_form_and_replays(lat8):
    """Against the GPU FP64 form on the same inputs (no oracle rounding in
    between), and bit for bit across graph replays and an eager run."""
    w, mons, blocks, E = lat8
    outs = {}
    for prec, graphs in (("fp64e", True), ("fp64e", False), ("fp64", True)):
        with M.Context(precision=prec, graphs=graphs) as ctx:
            load_context(ctx, w, mons, blocks, range(w.n_dimers))
            ctx.run()
            first = ctx.energies()[2].copy()
            ctx.run()
            second = ctx.energies()[2].copy()
        assert np.array_equal(first, second), (prec, graphs)
        outs[(prec, graphs)] = first
    assert np.array_equal(outs[("fp64e", True)], outs[("fp64e", False)])
    a, b = outs[("fp64e", True)], outs[("fp64", True)]
    rel = np.abs(a - b).max(axis=1) / np.abs(b[:, 0])
    print(f"fp64e vs the FP64 form: max rel diff {rel.max():.2e}")
    assert np.all(rel <= PER_DIMER_LATTICE)


def test_fp64e_rejects_sizes_beyond_its_kernel():
    """Six occupied orbitals, or a Y monomer above 64 AO: MCPT_EUNSUPPORTED
    from the run, with a message."""
    rng = np.random.default_rng(37)
    for nX, nY, oX, oY in [(16, 16, 6, 2), (16, 72, 2, 2)]:
        A, K, CX, eX, CY, eY = rand_dimer(rng, nX, nY, oX, oY)
        with M.Context(precision="fp64e") as ctx:
            ctx.add_monomer(CX, eX, oX)
            ctx.add_monomer(CY, eY, oY)
            ctx.add_dimer(0, 1, np.concatenate([A.ravel(), K.ravel()]), M.MCPT_AO_BLOCKS)
            with pytest.raises(M.McptError) as ei:
                ctx.run()
            assert ei.value.status == M.MCPT_EUNSUPPORTED
            assert "64 AO" in str(ei.value)


def test_fp64e_coupling_matches_fp64_form(lat8):
    """With the coupling on, the pair second half also stores (ia|jb) and
    T = vD in FP64: every monomer's R_X of Eq. (tm2) against the FP64
    form's, and the energies unchanged by the store."""
    w, mons, blocks, E = lat8
    R, pd = {}, {}
    for prec in ("fp64e", "fp64"):
        with M.Context(precision=prec, coupling=True) as ctx:
            load_context(ctx, w, mons, blocks, range(w.n_dimers))
            ctx.run()
            pd[prec] = ctx.energies()[2].copy()
            R[prec] = [ctx.coupling(X, w.nao[X], w.nocc[X]) for X in range(w.n_monomers)]
    rel = np.abs(pd["fp64e"] - pd["fp64"]).max(axis=1) / np.abs(pd["fp64"][:, 0])
    assert np.all(rel <= PER_DIMER_LATTICE)
    worst = 0.0
    for a, b in zip(R["fp64e"], R["fp64"]):
        worst = max(worst, np.abs(a - b).max() / np.abs(b).max())
    print(f"fp64e coupling vs the FP64 form: max rel diff {worst:.2e}")
    assert worst <= 1e-12
