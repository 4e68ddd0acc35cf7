"""The dimer doubles iteration of Eq. (td2) on the GPU vs the FP64 oracle,
through the C ABI (marked gpu).

Tolerances per dimer, relative to |E_J|: fp64 1e-11; the other forms run the
iteration in FP32 (integral transformation, contractions and amplitudes;
energy sums FP64): 5e-7 (measured 2.6e-8).  One step is the first-order term.
"""
import numpy as np
import pytest

import oracle
import synth
from helpers import host_workload, load_context

pytestmark = pytest.mark.gpu

M = pytest.importorskip("paper_1409_2700_gb300")
torch = pytest.importorskip("torch")

TOL = {"fp64": 1e-11, "fp32c": 5e-7, "bf16x3": 5e-7, "tf32": 5e-7}
FORMS = ["fp64", "fp32c", "bf16x3", "tf32"]
NIT = 6


@pytest.fixture(scope="module")
def lat8():
    return host_workload("lattice-2x2x2")


@pytest.fixture(scope="module")
def lat8_td2(lat8):
    w, mons, blocks, E = lat8
    md = {X: synth.monomer_doubles(X, w.nao[X], w.nocc[X]) for X in range(w.n_monomers)}
    ref, ref1, dl = [], [], None
    for d in range(w.n_dimers):
        X, Y = w.pairs[d]
        A, K = blocks[d]
        _, e, dd = oracle.td2(A, K, mons[X].C, mons[X].eps, mons[Y].C, mons[Y].eps, mons[X].nocc, mons[Y].nocc,
                              NIT, md[X][0], md[Y][0], md[X][1], md[Y][1])
        ref.append(e)
        _, e1, _ = oracle.td2(A, K, mons[X].C, mons[X].eps, mons[Y].C, mons[Y].eps, mons[X].nocc, mons[Y].nocc, 1)
        ref1.append(e1)
        dl = dd if dl is None else np.maximum(dl, dd)
    return md, np.array(ref), np.array(ref1), dl


@pytest.mark.parametrize("prec", FORMS)
def test_td2_lattice_2x2x2(lat8, lat8_td2, prec):
    w, mons, blocks, E = lat8
    md, ref, ref1, dl = lat8_td2
    with M.Context(precision=prec) as ctx:
        load_context(ctx, w, mons, blocks, range(w.n_dimers))
        one, d1 = ctx.td2(1)                    # no monomer matrices yet: first order
        err1 = np.max(np.abs(one[:, 0] - ref1[:, 0]) / np.abs(ref1[:, 0]))
        assert err1 <= TOL[prec], err1
        assert np.allclose(one[:, 1], ref1[:, 1], rtol=0, atol=TOL[prec] * np.abs(ref1[:, 0]).max())
        for X in range(w.n_monomers):
            ctx.set_monomer_doubles(X, *md[X])
        got, delta = ctx.td2(NIT)
        errJ = np.max(np.abs(got[:, 0] - ref[:, 0]) / np.abs(ref[:, 0]))
        errK = np.max(np.abs(got[:, 1] - ref[:, 1]) / np.abs(ref[:, 0]))
        print(f"{prec}: td2 {NIT} steps max rel err J {errJ:.2e} K {errK:.2e}; delta {delta}")
        assert errJ <= TOL[prec] and errK <= TOL[prec]
        # the step sizes follow the oracle's until they reach the form's rounding level
        if prec == "fp64":
            assert np.all(np.abs(delta - dl) <= 1e-2 * dl + 1e-17)
            assert np.all(np.diff(delta) < 0)
        else:
            assert abs(delta[0] - dl[0]) <= 1e-5 * dl[0]
            assert np.all(np.diff(delta[:3]) < 0)
        again, _ = ctx.td2(NIT)
        assert np.array_equal(again, got)


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_td2_uneven_sizes_full_layout_and_missing_matrices(prec):
    """Monomers of 16, 24 and 12 AO; dimer (0, 1) given as the full tensor
    on the device (strided blocks); monomer 2 has no matrices (zero)."""
    rng = np.random.default_rng(71)
    sizes = [(16, 3), (24, 4), (12, 2)]
    mons = []
    for n, o in sizes:
        C = np.linalg.qr(rng.standard_normal((n, n)))[0]
        e = np.concatenate([np.sort(rng.uniform(-1.5, -0.5, o)), np.sort(rng.uniform(0.2, 3.0, n - o))])
        mons.append((C, e, o))
    md = [synth.monomer_doubles(X, n, o) for X, (n, o) in enumerate(sizes[:2])] + [(None, None)]
    pairs = [(0, 1), (1, 2), (0, 2)]
    Bs = {}
    for X, Y in pairs:
        nX, nY = sizes[X][0], sizes[Y][0]
        B = rng.standard_normal((6, nX + nY, nX + nY)) * 0.02
        Bs[(X, Y)] = B + np.transpose(B, (0, 2, 1))
    ref = []
    for X, Y in pairs:
        A, K = synth.eri_blocks(Bs[(X, Y)], sizes[X][0], 0.6)
        _, e, _ = oracle.td2(A, K, mons[X][0], mons[X][1], mons[Y][0], mons[Y][1], mons[X][2], mons[Y][2], NIT,
                             md[X][0], md[Y][0], md[X][1], md[Y][1])
        ref.append(e)
    ref = np.array(ref)
    with M.Context(precision=prec) as ctx:
        for C, e, o in mons:
            ctx.add_monomer(C, e, o)
        full = torch.from_numpy(synth.eri_full(Bs[(0, 1)], sizes[0][0], 0.6)).cuda()
        ctx.add_dimer(0, 1, full.data_ptr(), M.MCPT_AO_FULL, on_device=1)
        for X, Y in pairs[1:]:
            A, K = synth.eri_blocks(Bs[(X, Y)], sizes[X][0], 0.6)
            ctx.add_dimer(X, Y, np.concatenate([A.ravel(), K.ravel()]), M.MCPT_AO_BLOCKS)
        for X in range(2):
            ctx.set_monomer_doubles(X, *md[X])
        got, delta = ctx.td2(NIT)
        err = np.max(np.abs(got - ref) / np.abs(ref[:, :1]))
        print(f"{prec}: uneven td2 max rel err {err:.2e}")
        assert err <= TOL[prec]
        with pytest.raises(M.McptError) as ei:
            ctx.td2(0)
        assert ei.value.status == M.MCPT_EINVAL
