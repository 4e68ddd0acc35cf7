"""Dimer -> monomer doubles coupling of Eq. (tm2) at first order and the
singles environment term of Eq. (tm1), GPU vs the FP64 oracle, through the
C ABI (marked gpu).

Tolerances, relative to the largest |R_X| element, from each form's first
half: fp64 1e-11; fp32c and bf16x3 (FP32-accurate (ia|jb), FP32 sums over
~1e3 terms) 1e-5; tf32 (10-bit integrals) 2e-3.  The singles term takes
the same tolerances relative to the largest |s_X| element.
"""
import numpy as np
import pytest

import oracle
from helpers import load_context

pytestmark = pytest.mark.gpu

M = pytest.importorskip("paper_1409_2700_gb300")

TOL = {"fp64": 1e-11, "fp32c": 1e-5, "bf16x3": 1e-5, "tf32": 2e-3}
FORMS = ["fp64", "fp32c", "bf16x3", "tf32"]


@pytest.fixture(scope="module")
def lat8_coupling(lat8):
    w, mons, blocks, E = lat8
    return oracle.coupling_lattice(w, blocks=blocks)


@pytest.fixture(scope="module")
def lat8():
    from helpers import host_workload
    return host_workload("lattice-2x2x2")


@pytest.mark.parametrize("prec", FORMS)
def test_coupling_lattice_2x2x2(lat8, lat8_coupling, prec):
    """Every monomer's R_X over its 7 neighbours; its trace equals the
    monomer's half-share of E_J computed by the same run."""
    w, mons, blocks, E = lat8
    with M.Context(precision=prec, coupling=True) as ctx:
        load_context(ctx, w, mons, blocks, range(w.n_dimers))
        ctx.run()
        mj, mk, pd, tot = ctx.energies()
        worst = 0.0
        for X in range(w.n_monomers):
            R = ctx.coupling(X, w.nao[X], w.nocc[X])
            ref = lat8_coupling[X]
            scale = np.abs(ref).max()
            err = np.abs(R - ref).max() / scale
            worst = max(worst, err)
            assert err <= TOL[prec], (prec, X, err)
            assert np.array_equal(R, R.T)
            assert abs(np.trace(R) - mj[X]) <= max(TOL[prec], 1e-12) * abs(mj[X]) * 10
        print(f"{prec}: coupling max rel err {worst:.2e}")
        # again: deterministic
        ctx.run()
        R2 = ctx.coupling(0, w.nao[0], w.nocc[0])
        ctx.run()
        assert np.array_equal(R2, ctx.coupling(0, w.nao[0], w.nocc[0]))


def _amplitudes(seed, sizes):
    rng = np.random.default_rng(seed)
    return [rng.standard_normal((o, n - o)) * 0.01 for n, o in sizes]


@pytest.mark.parametrize("prec", FORMS)
def test_singles_lattice_2x2x2(lat8, prec):
    """Every monomer's Eq. (tm1) environment term over its 7 neighbours for
    seeded amplitudes; two calls agree bit for bit."""
    w, mons, blocks, E = lat8
    t = _amplitudes(41, [(w.nao[X], w.nocc[X]) for X in range(w.n_monomers)])
    ref = oracle.singles_lattice(w, {X: t[X] for X in range(w.n_monomers)}, blocks=blocks)
    with M.Context(precision=prec, coupling=True) as ctx:
        load_context(ctx, w, mons, blocks, range(w.n_dimers))
        ctx.run()
        s = ctx.singles(t)
        worst = 0.0
        for X in range(w.n_monomers):
            err = np.abs(s[X] - ref[X]).max() / np.abs(ref[X]).max()
            worst = max(worst, err)
            assert err <= TOL[prec], (prec, X, err)
        print(f"{prec}: singles max rel err {worst:.2e}")
        s2 = ctx.singles(t)
        assert all(np.array_equal(a, b) for a, b in zip(s, s2))


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_coupling_uneven_and_occupation_blocks(prec):
    """Monomers of different sizes in a chain X0 - X1 - X2 - X3 (X1 and X2
    couple to both sides); X1 has 20 occupied orbitals, so the tensor-core
    forms run its dimers as occupation blocks that write into the same stored
    (ia|jb).  The o v sizes 21, 400, 95, 128 take output tiles of edge 32,
    48 (ragged), 48 and 64; a fifth monomer has no dimers and R = 0."""
    rng = np.random.default_rng(31)
    sizes = [(10, 3), (40, 20), (24, 5), (36, 4), (12, 2)]
    mons = []
    for n, o in sizes:
        C = np.linalg.qr(rng.standard_normal((n, n)))[0]
        e = np.concatenate([np.sort(rng.uniform(-1.5, -0.5, o)), np.sort(rng.uniform(0.2, 3.0, n - o))])
        mons.append((C, e, o))
    pairs = [(0, 1), (1, 2), (2, 3)]
    blks = {}
    for X, Y in pairs:
        nX, nY = sizes[X][0], sizes[Y][0]
        blks[(X, Y)] = (rng.standard_normal((nX, nX, nY, nY)) * 1e-3, rng.standard_normal((nX, nY, nY, nX)) * 1e-3)
    R = {m: np.zeros(((sizes[m][1] * (sizes[m][0] - sizes[m][1])),) * 2) for m in range(len(sizes))}
    t = _amplitudes(42, sizes)
    S = [np.zeros_like(x) for x in t]
    for X, Y in pairs:
        (CX, eX, oX), (CY, eY, oY) = mons[X], mons[Y]
        V = oracle.transform_J(blks[(X, Y)][0], CX, CY, oX, oY)
        oracle.coupling_add(V, eX, eY, oX, oY, R[X], R[Y])
        oracle.singles_add(V, t[X], t[Y], S[X], S[Y])
    with M.Context(precision=prec, coupling=True) as ctx:
        for C, e, o in mons:
            ctx.add_monomer(C, e, o)
        for X, Y in pairs:
            A, K = blks[(X, Y)]
            ctx.add_dimer(X, Y, np.concatenate([A.ravel(), K.ravel()]), M.MCPT_AO_BLOCKS)
        ctx.run()
        for m in range(len(sizes)):
            G = ctx.coupling(m, *sizes[m])
            assert np.array_equal(G, G.T)
            if m == 4:
                assert not G.any()
                continue
            err = np.abs(G - R[m]).max() / np.abs(R[m]).max()
            print(f"{prec} monomer {m} ({sizes[m][0]} AO, {sizes[m][1]} occ): rel err {err:.2e}")
            assert err <= TOL[prec]
        s = ctx.singles(t)
        assert not s[4].any()
        for m in range(4):
            err = np.abs(s[m] - S[m]).max() / np.abs(S[m]).max()
            print(f"{prec} monomer {m}: singles rel err {err:.2e}")
            assert err <= TOL[prec]
        # new integrals: the coupling is stale until the next run
        A, K = blks[(0, 1)]
        ctx.update_dimer(0, 2.0 * np.concatenate([A.ravel(), K.ravel()]))
        with pytest.raises(M.McptError) as ei:
            ctx.coupling(0, *sizes[0])
        assert ei.value.status == M.MCPT_ESTATE
        with pytest.raises(M.McptError) as ei:
            ctx.singles(t)
        assert ei.value.status == M.MCPT_ESTATE
        ctx.run()
        G = ctx.coupling(0, *sizes[0])
        assert np.allclose(G, 4.0 * R[0], rtol=0, atol=TOL[prec] * 4 * np.abs(R[0]).max())
    with M.Context(precision=prec) as ctx:          # coupling not requested
        ctx.add_monomer(*mons[0][:2], mons[0][2])
        with pytest.raises(M.McptError) as ei:
            ctx.coupling(0, *sizes[0])
        assert ei.value.status == M.MCPT_ESTATE
        with pytest.raises(M.McptError) as ei:
            ctx.singles(t[:1])
        assert ei.value.status == M.MCPT_ESTATE
