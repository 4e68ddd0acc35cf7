"""Symmetry-packed integral input (MCPT_AO_PACKED) through the C ABI (marked
gpu).  Expanding the packed elements on the device reproduces the symmetric
blocks exactly, so every form gives per-dimer terms bit for bit equal to the
same run from BLOCKS input, and within the form's tolerance of the oracle."""
import numpy as np
import pytest

import oracle
import synth
from helpers import host_workload

pytestmark = pytest.mark.gpu

M = pytest.importorskip("paper_1409_2700_gb300")
torch = pytest.importorskip("torch")

PER_DIMER = {"fp64": 1e-12, "fp32c": 2e-6, "bf16x3": 2e-6, "tf32": 2e-3}


@pytest.fixture(scope="module")
def lat8():
    return host_workload("lattice-2x2x2")


def _run(w, mons, blocks, prec, packed, device=False):
    with M.Context(precision=prec) as ctx:
        for X in range(w.n_monomers):
            m = mons[X]
            ctx.add_monomer(m.C, m.eps, m.nocc)
        keep = []
        for d in range(w.n_dimers):
            X, Y = w.pairs[d]
            A, K = blocks[d]
            if packed:
                p = synth.pack_blocks(A, K)
                if device:
                    t = torch.from_numpy(p).cuda()
                    keep.append(t)
                    ctx.add_dimer(X, Y, t.data_ptr(), M.MCPT_AO_PACKED, on_device=1)
                else:
                    ctx.add_dimer(X, Y, p, M.MCPT_AO_PACKED)
            else:
                ctx.add_dimer(X, Y, np.concatenate([A.ravel(), K.ravel()]), M.MCPT_AO_BLOCKS)
        del keep                                  # packed data is expanded before add_dimer returns
        ctx.run()
        return ctx.energies()


@pytest.mark.parametrize("prec", ["fp64", "fp32c", "bf16x3", "tf32"])
def test_packed_equals_blocks_lattice_2x2x2(lat8, prec):
    w, mons, blocks, E = lat8
    ref = _run(w, mons, blocks, prec, packed=False)
    for device in (False, True):
        got = _run(w, mons, blocks, prec, packed=True, device=device)
        assert np.array_equal(got[2], ref[2]), (prec, device)
        assert np.array_equal(got[3], ref[3])
    err = np.max(np.abs(ref[2] - E) / np.abs(E[:, :1]))
    assert err <= PER_DIMER[prec]


def test_packed_unequal_sizes_and_update():
    """Monomers of 16 and 24 AO in both orders of size; an asynchronous packed
    update from pinned host memory scaled by 4 gives terms scaled by 16
    exactly; packed input with X > Y is rejected."""
    rng = np.random.default_rng(52)
    sizes = [(16, 3), (24, 4), (12, 2)]
    mons = []
    for n, o in sizes:
        C = np.linalg.qr(rng.standard_normal((n, n)))[0]
        e = np.concatenate([np.sort(rng.uniform(-1.5, -0.5, o)), np.sort(rng.uniform(0.2, 3.0, n - o))])
        mons.append((C, e, o))
    pairs = [(0, 1), (1, 2), (0, 2)]
    blks = {}
    for X, Y in pairs:
        nX, nY = sizes[X][0], sizes[Y][0]
        B = rng.standard_normal((6, nX + nY, nX + nY)) * 0.01
        blks[(X, Y)] = synth.eri_blocks(B + np.transpose(B, (0, 2, 1)), nX, 0.5)
    for prec in ("fp64", "bf16x3"):
        out = {}
        for packed in (False, True):
            with M.Context(precision=prec) as ctx:
                for C, e, o in mons:
                    ctx.add_monomer(C, e, o)
                for X, Y in pairs:
                    A, K = blks[(X, Y)]
                    if packed:
                        ctx.add_dimer(X, Y, synth.pack_blocks(A, K), M.MCPT_AO_PACKED)
                    else:
                        ctx.add_dimer(X, Y, np.concatenate([A.ravel(), K.ravel()]), M.MCPT_AO_BLOCKS)
                ctx.run()
                out[packed] = ctx.energies()[2]
                if packed:
                    ref = [oracle.dimer(*blks[(X, Y)], mons[X][0], mons[X][1], mons[Y][0], mons[Y][1],
                                        mons[X][2], mons[Y][2]) for X, Y in pairs]
                    err = np.max(np.abs(out[packed] - np.array(ref)) / np.abs(np.array(ref)[:, :1]))
                    assert err <= PER_DIMER[prec]
                    A, K = blks[(0, 1)]
                    host = torch.from_numpy(4.0 * synth.pack_blocks(A, K)).pin_memory()
                    ctx.update_dimer(0, host.data_ptr(), M.MCPT_AO_PACKED, on_device=0, asynchronous=True)
                    ctx.run()
                    e2 = ctx.energies()[2]
                    assert np.array_equal(e2[0], 16.0 * out[packed][0])
                    assert np.array_equal(e2[1:], out[packed][1:])
                    with pytest.raises(M.McptError) as ei:
                        ctx.add_dimer(2, 1, synth.pack_blocks(*blks[(1, 2)]), M.MCPT_AO_PACKED)
                    assert ei.value.status == M.MCPT_EINVAL
        assert np.array_equal(out[True], out[False]), prec


@pytest.mark.parametrize("prec", ["fp64", "bf16x2"])
def test_update_dimers_batched_equals_one_by_one(lat8, prec):
    """mcpt_update_dimers (one call for many dimers: back-to-back packed data
    copied in chunks, one expansion launch per chunk) gives the terms of the
    same integrals registered one by one, bit for bit: first the lattice's
    own integrals after a doubling (terms x 4), then back, from one pinned
    buffer asynchronously; BLOCKS data too; a dimer whose data were borrowed
    device memory gets storage of its own; and a sub-range."""
    w, mons, blocks, E = lat8
    ref = _run(w, mons, blocks, prec, packed=False)
    packed = [synth.pack_blocks(*blocks[d]) for d in range(w.n_dimers)]
    offs = np.cumsum([0] + [p.size for p in packed[:-1]]).astype(np.uint64)
    flat = np.concatenate(packed)
    pinned = torch.from_numpy(flat).pin_memory()
    with M.Context(precision=prec) as ctx:
        for X in range(w.n_monomers):
            m = mons[X]
            ctx.add_monomer(m.C, m.eps, m.nocc)
        dev0 = torch.from_numpy(np.concatenate([blocks[0][0].ravel(), blocks[0][1].ravel()])).cuda()
        X0, Y0 = w.pairs[0]
        ctx.add_dimer(X0, Y0, dev0.data_ptr(), M.MCPT_AO_BLOCKS, on_device=1)   # borrowed
        for d in range(1, w.n_dimers):
            X, Y = w.pairs[d]
            ctx.add_dimer(X, Y, packed[d], M.MCPT_AO_PACKED)
        ctx.run()
        assert np.array_equal(ctx.energies()[2], ref[2])
        ctx.update_dimers(0, w.n_dimers, 2.0 * flat, offs, M.MCPT_AO_PACKED)
        with pytest.raises(M.McptError):
            ctx.energies()                                   # not computed since the update
        ctx.run()
        assert np.array_equal(ctx.energies()[2], 4.0 * ref[2])
        ctx.update_dimers(0, w.n_dimers, pinned.data_ptr(), offs, M.MCPT_AO_PACKED, asynchronous=True)
        ctx.run()
        got = ctx.energies()
        assert np.array_equal(got[2], ref[2]) and np.array_equal(got[3], ref[3])
        bl = [np.concatenate([blocks[d][0].ravel(), blocks[d][1].ravel()]) for d in range(w.n_dimers)]
        boffs = np.cumsum([0] + [b.size for b in bl[:-1]]).astype(np.uint64)
        ctx.update_dimers(0, w.n_dimers, 0.5 * np.concatenate(bl), boffs, M.MCPT_AO_BLOCKS)
        ctx.run()
        assert np.array_equal(ctx.energies()[2], 0.25 * ref[2])
        ctx.update_dimers(5, 10, flat, offs[5:15], M.MCPT_AO_PACKED)   # a sub-range: the rest stays halved
        ctx.run()
        got = ctx.energies()[2]
        assert np.array_equal(got[5:15], ref[2][5:15])
        assert np.array_equal(got[:5], 0.25 * ref[2][:5]) and np.array_equal(got[15:], 0.25 * ref[2][15:])
        with pytest.raises(M.McptError) as ei:
            ctx.update_dimers(20, 10, flat, offs[:10], M.MCPT_AO_PACKED)
        assert ei.value.status == M.MCPT_EINVAL
