"""The density-fitted route (three-index factors) through the C ABI vs the
oracle's factor route (marked gpu).  The factor route is pinned to the
four-index oracle (exact in exact arithmetic for factorised integrals), so
the GPU terms are also checked against the four-index oracle values.

Tolerances per dimer, relative to |E_J|: fp64 1e-12; the FP32 forms 5e-7
(FP32 sums over naux = 192 products; measured 3.4e-8).
"""
import numpy as np
import pytest

import oracle
import synth
from helpers import host_workload

pytestmark = pytest.mark.gpu

M = pytest.importorskip("paper_1409_2700_gb300")
torch = pytest.importorskip("torch")

TOL = {"fp64": 1e-12, "fp32c": 5e-7, "bf16x3": 5e-7, "tf32": 5e-7}


@pytest.fixture(scope="module")
def lat8():
    w, mons, blocks, E = host_workload("lattice-2x2x2")
    ref = []
    for d in range(w.n_dimers):
        X, Y = w.pairs[d]
        V, W = oracle.factor_route(w.factors(d), synth.scale_for_distance(w.R[d]), mons[X].C, mons[Y].C,
                                   mons[X].nocc, mons[Y].nocc)
        ref.append(oracle.energy_from_mo(V, W, mons[X].eps, mons[Y].eps, mons[X].nocc, mons[Y].nocc))
    return w, mons, E, np.array(ref)


@pytest.mark.parametrize("prec", ["fp64", "fp32c", "tf32"])
def test_df_lattice_2x2x2(lat8, prec):
    w, mons, E4, ref = lat8
    assert np.max(np.abs(ref - E4) / np.abs(E4[:, :1])) <= 1e-12      # factor route = four-index oracle
    keep = []
    with M.Context(precision=prec) as ctx:
        for X in range(w.n_monomers):
            ctx.add_monomer(mons[X].C, mons[X].eps, mons[X].nocc)
        for d in range(w.n_dimers):
            X, Y = w.pairs[d]
            B = w.factors(d)
            s = synth.scale_for_distance(w.R[d])
            if d % 2:                             # half of them borrowed from device memory
                t = torch.from_numpy(np.ascontiguousarray(B)).cuda()
                keep.append(t)
                assert ctx.add_dimer_df(X, Y, t.data_ptr(), B.shape[0], s, on_device=1) == d
            else:
                assert ctx.add_dimer_df(X, Y, B, B.shape[0], s) == d
        with pytest.raises(M.McptError) as ei:
            ctx.df_energies()
        assert ei.value.status == M.MCPT_ESTATE
        ctx.run_df()
        mj, mk, pd, tot = ctx.df_energies()
        err = np.max(np.abs(pd - ref) / np.abs(ref[:, :1]))
        print(f"{prec}: density-fitted route max rel err {err:.2e}")
        assert err <= TOL[prec]
        X = np.array([p[0] for p in w.pairs])
        Y = np.array([p[1] for p in w.pairs])
        omon, otot = oracle.accumulate(pd, X, Y, w.n_monomers)
        assert np.allclose(mj, omon[:, 0], rtol=1e-12, atol=0)
        assert np.allclose(mk, omon[:, 1], rtol=1e-12, atol=1e-300)
        assert abs(tot[0] - otot[0]) <= 1e-13 * abs(otot[0])
        ctx.run_df()
        assert np.array_equal(ctx.df_energies()[2], pd)               # deterministic
        with pytest.raises(M.McptError) as ei:
            ctx.add_dimer_df(1, 0, w.factors(0), 192, 1.0)
        assert ei.value.status == M.MCPT_EINVAL


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_df_unequal_sizes(prec):
    rng = np.random.default_rng(81)
    sizes = [(16, 3), (24, 4), (40, 7)]
    mons = []
    for n, o in sizes:
        C = np.linalg.qr(rng.standard_normal((n, n)))[0]
        e = np.concatenate([np.sort(rng.uniform(-1.5, -0.5, o)), np.sort(rng.uniform(0.2, 3.0, n - o))])
        mons.append((C, e, o))
    pairs = [(0, 1), (1, 2), (0, 2)]
    with M.Context(precision=prec) as ctx:
        for C, e, o in mons:
            ctx.add_monomer(C, e, o)
        ref = []
        for k, (X, Y) in enumerate(pairs):
            n = sizes[X][0] + sizes[Y][0]
            naux = 40 + 7 * k
            B = rng.standard_normal((naux, n, n)) * 0.01     # not symmetric: the route uses B as given
            V, W = oracle.factor_route(B, 0.5, mons[X][0], mons[Y][0], mons[X][2], mons[Y][2])
            ref.append(oracle.energy_from_mo(V, W, mons[X][1], mons[Y][1], mons[X][2], mons[Y][2]))
            ctx.add_dimer_df(X, Y, B, naux, 0.5)
        ctx.run_df()
        pd = ctx.df_energies()[2]
        ref = np.array(ref)
        err = np.max(np.abs(pd - ref) / np.abs(ref[:, :1]))
        print(f"{prec}: unequal sizes max rel err {err:.2e}")
        assert err <= TOL[prec]
