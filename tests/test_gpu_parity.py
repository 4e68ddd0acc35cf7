"""GPU path vs the FP64 oracle, through the C ABI (all marked gpu).

Tolerances (per form, from the arithmetic):
  fp64    same sums in another order: |dE| <= 1e-12 |E_J| per dimer; the
          lattice target is 1e-8 Eh, checked with margin.
  fp32c   FP32 inputs (u = 2^-24) with Dot2 sums and an FP32 second half:
          per dimer |dE| <= 2e-6 |E_J|; lattice <= 1e-6 Eh.
  bf16x3  32-bit fixed-point digits per vector with exact tensor-core sums,
          an FP32 second half: FP32-level like fp32c, per dimer <= 2e-6 |E_J|
          (kernel variants that keep the hi/lo floating split, <= 2e-4);
          lattice <= 1e-6 Eh.
  bf16x2  integrals in 16-bit fixed point per 32-value row chunk (error
          <= 2^-17 of the chunk's largest power of two), C_Y as in bf16x3,
          exact tensor-core sums: per dimer <= 5e-5 |E_J| (4 x 2^-17 x the
          few-term growth of the random cases); lattice <= 1e-6 Eh.
  tf32    integrals with 10-bit mantissas (u = 2^-11, round to nearest),
          C_Y as two TF32 planes, truncating FP32 accumulation in the tensor
          core: per dimer <= 2e-3 |E_J| (= 4u, the bound without any averaging:
          reached only by dimers of a handful of terms); lattice <= 1e-6 Eh at
          the sizes tested here.
Lattice dimers (thousands of terms per (ia|jb), errors that average) are held
to the tighter PER_DIMER_LATTICE bounds, set a few times above what the forms
measure on lattice-2x2x2.
E_K is checked against the same scale (|E_J|): it is three orders smaller
and its relative error is not meaningful on its own.
"""
import numpy as np
import pytest

import oracle
import synth
from helpers import host_workload, load_context, rand_dimer

pytestmark = pytest.mark.gpu

M = pytest.importorskip("paper_1409_2700_gb300")

PER_DIMER = {"fp64": 1e-12, "fp32c": 2e-6, "bf16x3": 2e-6, "bf16x2": 5e-5, "tf32": 2e-3}
PER_DIMER_LATTICE = {"fp64": 1e-12, "fp32c": 1e-7, "bf16x3": 1e-7, "bf16x2": 2e-6, "tf32": 5e-5}
PER_DIMER_KRON = {"bf16x3": 2e-4, "tf32": 2e-3}   # Kronecker kernel: whole (p0, p2) sums in the tensor core
LATTICE = {"fp64": 1e-10, "fp32c": 1e-6, "bf16x3": 1e-6, "bf16x2": 1e-6, "tf32": 1e-6}
FORMS = ["fp64", "fp32c", "bf16x3", "bf16x2", "tf32"]


@pytest.fixture(scope="module")
def lat8():
    return host_workload("lattice-2x2x2")


def _run(prec, w, mons, blocks, dimers, **kw):
    with M.Context(precision=prec, **kw) as ctx:
        load_context(ctx, w, mons, blocks, dimers)
        ctx.run()
        return ctx.energies()


@pytest.mark.parametrize("prec", FORMS)
def test_lattice_2x2x2_all_forms(lat8, prec):
    w, mons, blocks, E = lat8
    mj, mk, pd, tot = _run(prec, w, mons, blocks, range(w.n_dimers))
    scale = np.abs(E[:, 0])
    errJ = np.abs(pd[:, 0] - E[:, 0])
    errK = np.abs(pd[:, 1] - E[:, 1])
    print(f"{prec}: max rel err J {np.max(errJ / scale):.3e} K {np.max(errK / scale):.3e}")
    assert np.all(errJ <= PER_DIMER_LATTICE[prec] * scale)
    assert np.all(errK <= PER_DIMER_LATTICE[prec] * scale)
    omon, otot = oracle.accumulate(E, [p[0] for p in w.pairs], [p[1] for p in w.pairs], w.n_monomers)
    print(f"{prec}: lattice E_J {tot[0]:.12e} oracle {otot[0]:.12e} diff {tot[0] - otot[0]:.3e} Eh")
    assert abs(tot[0] - otot[0]) <= LATTICE[prec]
    assert abs(tot[1] - otot[1]) <= LATTICE[prec]
    assert np.all(np.abs(mj - omon[:, 0]) <= LATTICE[prec])
    assert np.all(np.abs(mk - omon[:, 1]) <= LATTICE[prec])
    # the split conserves the total
    assert abs(mj.sum() - tot[0]) <= 1e-14 * abs(tot[0]) * w.n_monomers


@pytest.mark.parametrize("prec", FORMS)
def test_nonsymmetric_random_blocks(prec):
    """Random non-symmetric integrals: only the literal index mapping of
    Eq. (dp2e) gives the oracle's numbers; sizes span several tiles with
    ragged edges (tensor-core forms need even AO counts)."""
    rng = np.random.default_rng(3)
    cases = [(6, 10, 2, 3), (14, 8, 3, 1), (32, 32, 5, 5), (40, 24, 7, 4)]
    if prec in ("fp64", "fp32c"):
        cases += [(5, 7, 2, 3), (9, 3, 1, 2)]
    if prec != "fp64":
        # up to four 32-p2 chunks per p0 (ragged last chunk), 128-AO rows
        cases += [(16, 128, 3, 16), (24, 100, 4, 12), (128, 16, 16, 3)]
    for nX, nY, oX, oY in cases:
        A, K, CX, eX, CY, eY = rand_dimer(rng, nX, nY, oX, oY)
        ref = oracle.dimer(A, K, CX, eX, CY, eY, oX, oY)
        with M.Context(precision=prec) as ctx:
            ctx.add_monomer(CX, eX, oX)
            ctx.add_monomer(CY, eY, oY)
            ctx.add_dimer(0, 1, np.concatenate([A.ravel(), K.ravel()]), M.MCPT_AO_BLOCKS)
            ctx.run()
            _, _, pd, _ = ctx.energies()
        s = abs(ref[0])
        assert abs(pd[0, 0] - ref[0]) <= PER_DIMER[prec] * s, (nX, nY, oX, oY, pd[0], ref)
        assert abs(pd[0, 1] - ref[1]) <= PER_DIMER[prec] * s, (nX, nY, oX, oY, pd[0], ref)


def test_full_layout_host_and_device_match_blocks(lat8):
    torch = pytest.importorskip("torch")
    w, mons, blocks, E = lat8
    d = 3
    X, Y = w.pairs[d]
    G = w.full(d)
    A, K = blocks[d]
    out = []
    for how in ("blocks", "full-host", "full-device", "blocks-device"):
        with M.Context(precision="fp64") as ctx:
            for m in range(w.n_monomers):
                mm = w.monomer(m)
                ctx.add_monomer(mm.C, mm.eps, mm.nocc)
            if how == "blocks":
                ctx.add_dimer(X, Y, np.concatenate([A.ravel(), K.ravel()]), M.MCPT_AO_BLOCKS)
            elif how == "full-host":
                ctx.add_dimer(X, Y, G, M.MCPT_AO_FULL)
            elif how == "full-device":
                t = torch.from_numpy(G).cuda()
                ctx.add_dimer(X, Y, t, M.MCPT_AO_FULL, on_device=1)
            else:
                t = torch.from_numpy(np.concatenate([A.ravel(), K.ravel()])).cuda()
                ctx.add_dimer(X, Y, t, M.MCPT_AO_BLOCKS, on_device=1)
            ctx.run()
            out.append(ctx.energies()[2][0].copy())
    for o in out[1:]:
        assert np.array_equal(o, out[0])   # same values, same arithmetic
    assert abs(out[0][0] - E[d, 0]) <= 1e-12 * abs(E[d, 0])


@pytest.mark.parametrize("prec", ["fp64", "tf32"])
def test_full_layout_device_tensor_core_path(lat8, prec):
    """Device-resident full tensors are read in place through strided views
    (tensor maps for the tensor-core forms)."""
    torch = pytest.importorskip("torch")
    w, mons, blocks, E = lat8
    ds = [0, 7, 19]
    with M.Context(precision=prec) as ctx:
        for m in range(w.n_monomers):
            mm = w.monomer(m)
            ctx.add_monomer(mm.C, mm.eps, mm.nocc)
        keep = []
        for d in ds:
            X, Y = w.pairs[d]
            t = torch.from_numpy(w.full(d)).cuda()
            keep.append(t)
            ctx.add_dimer(X, Y, t, M.MCPT_AO_FULL, on_device=1)
        ctx.run()
        pd = ctx.energies()[2]
    for k, d in enumerate(ds):
        assert abs(pd[k, 0] - E[d, 0]) <= PER_DIMER[prec] * abs(E[d, 0])


def test_swapped_order_relabels(lat8):
    """(Y, X) with the caller's integrals in Y-first order gives the same term."""
    w, mons, blocks, E = lat8
    d = 11
    X, Y = w.pairs[d]
    nX = w.nao[X]
    G = w.full(d)
    perm = np.concatenate([np.arange(nX, 2 * nX), np.arange(nX)])
    Gs = np.ascontiguousarray(G[np.ix_(perm, perm, perm, perm)])
    As, Ks = synth.extract_blocks(Gs, w.nao[Y])
    for layout, arr in ((M.MCPT_AO_FULL, Gs), (M.MCPT_AO_BLOCKS, np.concatenate([As.ravel(), Ks.ravel()]))):
        with M.Context(precision="fp64") as ctx:
            for m in range(w.n_monomers):
                mm = w.monomer(m)
                ctx.add_monomer(mm.C, mm.eps, mm.nocc)
            ctx.add_dimer(Y, X, arr, layout)
            ctx.run()
            pd = ctx.energies()[2]
        assert abs(pd[0, 0] - E[d, 0]) <= 1e-12 * abs(E[d, 0])
        assert abs(pd[0, 1] - E[d, 1]) <= 1e-12 * abs(E[d, 0])


@pytest.mark.parametrize("prec", FORMS)
def test_edge_sizes_and_zero(prec):
    rng = np.random.default_rng(11)
    # nocc = 1 and nvirt = 1 on either side
    for nX, nY, oX, oY in [(4, 6, 1, 5), (6, 4, 5, 1), (2, 2, 1, 1), (8, 16, 7, 1)]:
        A, K, CX, eX, CY, eY = rand_dimer(rng, nX, nY, oX, oY)
        ref = oracle.dimer(A, K, CX, eX, CY, eY, oX, oY)
        with M.Context(precision=prec) as ctx:
            ctx.add_monomer(CX, eX, oX)
            ctx.add_monomer(CY, eY, oY)
            ctx.add_dimer(0, 1, np.concatenate([A.ravel(), K.ravel()]), M.MCPT_AO_BLOCKS)
            ctx.run()
            _, _, pd, _ = ctx.energies()
        assert abs(pd[0, 0] - ref[0]) <= PER_DIMER[prec] * abs(ref[0])
    # zero integrals give exactly zero
    A, K, CX, eX, CY, eY = rand_dimer(rng, 8, 6, 2, 2)
    with M.Context(precision=prec) as ctx:
        ctx.add_monomer(CX, eX, 2)
        ctx.add_monomer(CY, eY, 2)
        ctx.add_dimer(0, 1, np.zeros(2 * A.size), M.MCPT_AO_BLOCKS)
        ctx.run()
        mj, mk, pd, tot = ctx.energies()
    assert pd[0, 0] == 0.0 and pd[0, 1] == 0.0 and tot[0] == 0.0


def test_determinism_and_range(lat8):
    w, mons, blocks, E = lat8
    ds = list(range(w.n_dimers))
    for prec in ("fp64", "tf32"):
        with M.Context(precision=prec) as ctx:
            load_context(ctx, w, mons, blocks, ds)
            ctx.run()
            a = ctx.energies()
            ctx.run()
            b = ctx.energies()
            for x, y in zip(a, b):
                assert np.array_equal(x, y)
        with M.Context(precision=prec) as ctx:
            load_context(ctx, w, mons, blocks, ds)
            ctx.run(0, 10)
            with pytest.raises(M.McptError) as ei:
                ctx.energies()
            assert ei.value.status == M.MCPT_ESTATE
            ctx.run(10, 18)
            c = ctx.energies()
            for x, y in zip(a, c):
                assert np.array_equal(x, y)


@pytest.mark.parametrize("prec", ["tf32", "bf16x2"])
def test_alternating_ranges_keep_their_plans(lat8, prec):
    """Runs that alternate between dimer ranges (the waves of a streamed
    lattice) each keep their own plan and CUDA graph: replayed graphs equal
    eager runs bit for bit, and the lattice equals the one-range run."""
    w, mons, blocks, E = lat8
    ds = list(range(w.n_dimers))
    out = {}
    for graphs in (False, True):
        with M.Context(precision=prec, graphs=graphs) as ctx:
            load_context(ctx, w, mons, blocks, ds)
            for _ in range(3):
                for first, count in ((0, 10), (10, 9), (19, 9)):
                    ctx.run(first, count)
            out[graphs] = ctx.energies()
    whole = _run(prec, w, mons, blocks, ds)
    for x, y, z in zip(out[False], out[True], whole):
        assert np.array_equal(x, y)
        assert np.array_equal(x, z)
    assert np.all(np.abs(out[True][2][:, 0] - E[:, 0]) <= PER_DIMER_LATTICE[prec] * np.abs(E[:, 0]))


def test_waves_match_single_wave(lat8):
    w, mons, blocks, E = lat8
    ds = list(range(w.n_dimers))
    res = []
    for wave_bytes in (0, 1):   # 1 byte: one dimer per wave
        with M.Context(precision="tf32", wave_bytes=wave_bytes, timing=True) as ctx:
            load_context(ctx, w, mons, blocks, ds)
            ctx.run()
            res.append(ctx.energies())
            st = ctx.stats()
            assert st.waves == (1 if wave_bytes == 0 else w.n_dimers)
            assert st.ms[3] > 0
    for x, y in zip(*res):
        assert np.array_equal(x, y)


def test_error_codes():
    rng = np.random.default_rng(5)
    A, K, CX, eX, CY, eY = rand_dimer(rng, 6, 6, 2, 2)
    blk = np.concatenate([A.ravel(), K.ravel()])
    with M.Context(precision="fp64") as ctx:
        with pytest.raises(M.McptError) as ei:
            ctx.run()
        assert ei.value.status == M.MCPT_ESTATE
        with pytest.raises(M.McptError) as ei:
            ctx.add_monomer(CX, eX, 0)
        assert ei.value.status == M.MCPT_EINVAL
        with pytest.raises(M.McptError) as ei:
            ctx.add_monomer(CX, eX, 6)
        assert ei.value.status == M.MCPT_EINVAL
        bad = eX.copy()
        bad[3] = np.nan
        with pytest.raises(M.McptError) as ei:
            ctx.add_monomer(CX, bad, 2)
        assert ei.value.status == M.MCPT_EINVAL
        ctx.add_monomer(CX, eX, 2)
        ctx.add_monomer(CY, eY, 2)
        for X, Y in ((0, 0), (0, 5), (-1, 1)):
            with pytest.raises(M.McptError) as ei:
                ctx.add_dimer(X, Y, blk)
            assert ei.value.status == M.MCPT_EINVAL
        nanblk = blk.copy()
        nanblk[17] = np.inf
        with pytest.raises(M.McptError) as ei:
            ctx.add_dimer(0, 1, nanblk)
        assert ei.value.status == M.MCPT_EINVAL
        with pytest.raises(M.McptError) as ei:
            ctx.energies()
        assert ei.value.status == M.MCPT_ESTATE
        ctx.add_dimer(0, 1, blk)
        with pytest.raises(M.McptError) as ei:
            ctx.add_dimer(1, 0, blk)
        assert ei.value.status == M.MCPT_EINVAL       # duplicate pair
    # odd AO counts are outside the tensor-core forms
    A, K, CX, eX, CY, eY = rand_dimer(rng, 5, 6, 2, 2)
    with M.Context(precision="tf32") as ctx:
        ctx.add_monomer(CX, eX, 2)
        ctx.add_monomer(CY, eY, 2)
        ctx.add_dimer(0, 1, np.concatenate([A.ravel(), K.ravel()]))
        with pytest.raises(M.McptError) as ei:
            ctx.run()
        assert ei.value.status == M.MCPT_EUNSUPPORTED
    # device memory cap
    with M.Context(precision="fp64", mem_cap_bytes=1024) as ctx:
        ctx.add_monomer(CX, eX, 2)
        ctx.add_monomer(CY, eY, 2)
        with pytest.raises(M.McptError) as ei:
            ctx.add_dimer(0, 1, np.concatenate([A.ravel(), K.ravel()]))
        assert ei.value.status == M.MCPT_ENOMEM


@pytest.mark.parametrize("prec", FORMS)
def test_uneven_sizes_batch(prec):
    """A batch mixing 16..56-AO monomers (the uneven workload's smaller size
    classes) in one run: one persistent launch covers every size pair."""
    w = synth.workload("uneven-4096")
    ds = [k for k in range(200) if w.nao[2 * k] <= 56 and w.nao[2 * k + 1] <= 56][:10]
    items, blocks = [], {}
    for d in ds:
        X, Y = w.pairs[d]
        mX, mY = w.monomer(X), w.monomer(Y)
        blocks[d] = w.blocks(d)
        items.append((*blocks[d], mX.C, mX.eps, mY.C, mY.eps, mX.nocc, mY.nocc))
    E = oracle.dimers_parallel(items)
    with M.Context(precision=prec) as ctx:
        for k, d in enumerate(ds):
            X, Y = w.pairs[d]
            mX, mY = w.monomer(X), w.monomer(Y)
            ctx.add_monomer(mX.C, mX.eps, mX.nocc)
            ctx.add_monomer(mY.C, mY.eps, mY.nocc)
            A, K = blocks[d]
            ctx.add_dimer(2 * k, 2 * k + 1, np.concatenate([A.ravel(), K.ravel()]))
        ctx.run()
        pd = ctx.energies()[2]
    for k in range(len(ds)):
        assert abs(pd[k, 0] - E[k, 0]) <= PER_DIMER[prec] * abs(E[k, 0]), (prec, ds[k])
        assert abs(pd[k, 1] - E[k, 1]) <= PER_DIMER[prec] * abs(E[k, 0]), (prec, ds[k])


@pytest.mark.parametrize("prec,variant", [(p, v) for p in ("tf32", "bf16x3")
                                          for v in ("rank", "rank8", "rankbig", "rankwide", "kron")]
                         + [("bf16x2", v) for v in ("rank", "rank8", "rankbig", "rankwide")])
def test_tensor_core_kernel_variants(lat8, prec, variant, monkeypatch):
    """Both tcgen05 kernels (forced through MCPT_TC_KERNEL) against the oracle.
    The rank-1 variant keeps each tensor-core sum to n2/8 steps; its mean
    signed error over the lattice must stay well below the per-dimer bound."""
    monkeypatch.setenv("MCPT_TC_KERNEL", variant)
    w, mons, blocks, E = lat8
    mj, mk, pd, tot = _run(prec, w, mons, blocks, range(w.n_dimers))
    rel = (pd[:, 0] - E[:, 0]) / np.abs(E[:, 0])
    print(f"{prec}/{variant}: mean signed rel err {rel.mean():.3e}, max |rel| {np.abs(rel).max():.3e}, "
          f"lattice diff {tot[0] - E[:, 0].sum():.3e} Eh")
    assert np.all(np.abs(rel) <= (PER_DIMER_KRON if variant == "kron" else PER_DIMER)[prec])
    assert abs(tot[0] - E[:, 0].sum()) <= LATTICE[prec]
    pos = float(np.mean(rel > 0))
    print(f"{prec}/{variant}: fraction of dimers with positive error {pos:.2f}")


@pytest.mark.parametrize("prec", FORMS)
def test_uneven_large_occupations(prec):
    """Dimers of 56-96 AO (occupations 9-16) from the uneven workload: the
    tensor-core forms take the rank kernel with TMEM accumulators, the second
    half the general (n > 32) path; one launch covers the mixed sizes."""
    w = synth.workload("uneven-4096")
    ds = [k for k in range(400) if 56 <= w.nao[2 * k] <= 80 and 56 <= w.nao[2 * k + 1] <= 80][:3]
    assert len(ds) == 3
    items, blocks = [], {}
    for d in ds:
        X, Y = w.pairs[d]
        mX, mY = w.monomer(X), w.monomer(Y)
        B = w.factors(d)
        blocks[d] = synth.eri_blocks_direct(B, w.nao[X], synth.scale_for_distance(w.R[d]))
        items.append((*blocks[d], mX.C, mX.eps, mY.C, mY.eps, mX.nocc, mY.nocc))
    E = oracle.dimers_parallel(items)
    with M.Context(precision=prec) as ctx:
        for k, d in enumerate(ds):
            X, Y = w.pairs[d]
            mX, mY = w.monomer(X), w.monomer(Y)
            ctx.add_monomer(mX.C, mX.eps, mX.nocc)
            ctx.add_monomer(mY.C, mY.eps, mY.nocc)
            A, K = blocks[d]
            ctx.add_dimer(2 * k, 2 * k + 1, np.concatenate([A.ravel(), K.ravel()]))
        ctx.run()
        pd = ctx.energies()[2]
    for k in range(len(ds)):
        print(prec, ds[k], w.nao[2 * ds[k]], w.nao[2 * ds[k] + 1], pd[k], E[k])
        assert abs(pd[k, 0] - E[k, 0]) <= PER_DIMER[prec] * abs(E[k, 0]), (prec, ds[k])
        assert abs(pd[k, 1] - E[k, 1]) <= PER_DIMER[prec] * abs(E[k, 0]), (prec, ds[k])


@pytest.mark.parametrize("prec", ["fp64", "tf32", "bf16x2"])
def test_graph_replay_matches_eager(lat8, prec):
    """Runs replayed as a captured CUDA graph give bitwise the eager results,
    replay after replay."""
    w, mons, blocks, E = lat8
    out = {}
    for graphs in (False, True):
        with M.Context(precision=prec, graphs=graphs) as ctx:
            load_context(ctx, w, mons, blocks, range(w.n_dimers))
            res = []
            for _ in range(3):
                ctx.run()
                res.append(ctx.energies())
            for r in res[1:]:
                for x, y in zip(res[0], r):
                    assert np.array_equal(x, y)
            out[graphs] = res[0]
    for x, y in zip(out[False], out[True]):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("prec", ["tf32", "bf16x3", "bf16x2"])
def test_autotuner_cache(lat8, prec, tmp_path):
    """With a tune cache the first plan times every candidate launch of its
    wave and writes one line for the wave's shape signature; a second context
    reuses the line without timing; energies stay within the form's
    tolerance whatever launch won."""
    w, mons, blocks, E = lat8
    cache = tmp_path / "tune.txt"
    res = []
    for _ in range(2):
        with M.Context(precision=prec, tune_cache=str(cache)) as ctx:
            load_context(ctx, w, mons, blocks, range(w.n_dimers))
            ctx.run()
            res.append(ctx.energies())
        lines = cache.read_text().splitlines()
        assert len(lines) == 1, lines
    key, variant1, sf, grid, ms = lines[0].split()
    assert key.startswith(prec + ":") and int(variant1) in (1, 2, 3, 4, 5) and int(sf) >= 2 and int(grid) >= 1
    print(f"{prec}: tuned {lines[0]}")
    for mj, mk, pd, tot in res:
        assert np.all(np.abs(pd[:, 0] - E[:, 0]) <= PER_DIMER[prec] * np.abs(E[:, 0]))
        assert abs(tot[0] - E[:, 0].sum()) <= LATTICE[prec]
    assert np.array_equal(res[0][2], res[1][2])


@pytest.mark.parametrize("prec", ["tf32", "bf16x3", "bf16x2"])
def test_occupations_above_16_run_as_blocks(prec):
    """More than 16 occupied orbitals on a monomer: the tensor-core forms run
    the dimer as blocks of at most 20 x 16 occupied pairs (i of X, j of Y;
    each over all virtual orbitals) and add the blocks' terms -- (20, 18) as
    two 20 x 9 blocks and (17, 3) as one block in the wide TMEM-accumulator
    kernel, (2, 33) as three blocks -- and the result is the whole dimer's,
    on non-symmetric random integrals."""
    rng = np.random.default_rng(17)
    for nX, nY, oX, oY in [(40, 36, 20, 18), (24, 34, 17, 3), (18, 40, 2, 33)]:
        A, K, CX, eX, CY, eY = rand_dimer(rng, nX, nY, oX, oY)
        ref = oracle.dimer(A, K, CX, eX, CY, eY, oX, oY)
        with M.Context(precision=prec) as ctx:
            ctx.add_monomer(CX, eX, oX)
            ctx.add_monomer(CY, eY, oY)
            ctx.add_dimer(0, 1, np.concatenate([A.ravel(), K.ravel()]), M.MCPT_AO_BLOCKS)
            ctx.run()
            _, _, pd, tot = ctx.energies()
        s = abs(ref[0])
        print(f"{prec} {nX}x{nY} occ {oX}x{oY}: rel err J {abs(pd[0, 0] - ref[0]) / s:.2e} K {abs(pd[0, 1] - ref[1]) / s:.2e}")
        assert abs(pd[0, 0] - ref[0]) <= PER_DIMER[prec] * s
        assert abs(pd[0, 1] - ref[1]) <= PER_DIMER[prec] * s
        assert tot[0] == pd[0, 0]



@pytest.mark.parametrize("prec", ["fp64", "tf32", "bf16x3", "bf16x2"])
def test_update_dimer(lat8, prec):
    """New integrals for registered dimers: doubling every integral scales
    both terms by exactly 4 (v and v' double; D is unchanged; a power-of-two
    scale is exact in every form).  Host updates (synchronous, and
    asynchronous from pinned memory) reuse the dimers' storage; a device
    update re-points the dimer; each is followed by the right energies,
    bit for bit."""
    torch = pytest.importorskip("torch")
    w, mons, blocks, E = lat8
    with M.Context(precision=prec) as ctx:
        load_context(ctx, w, mons, blocks, range(w.n_dimers))
        ctx.run()
        base = ctx.energies()[2].copy()
        # synchronous host update, one dimer at a time
        for d in range(w.n_dimers):
            A, K = blocks[d]
            ctx.update_dimer(d, 2.0 * np.concatenate([A.ravel(), K.ravel()]))
        with pytest.raises(M.McptError):
            ctx.energies()                    # not computed since the update
        ctx.run()
        pd2 = ctx.energies()[2].copy()
        assert np.array_equal(pd2, 4.0 * base), np.abs(pd2 / base - 4).max()
        # asynchronous host update from one pinned buffer, back to the original
        n = sum(blocks[d][0].size + blocks[d][1].size for d in range(w.n_dimers))
        pinned = torch.empty(n, dtype=torch.float64, pin_memory=True)
        o = 0
        for d in range(w.n_dimers):
            A, K = blocks[d]
            blk = np.concatenate([A.ravel(), K.ravel()])
            pinned[o:o + blk.size] = torch.from_numpy(blk)
            ctx.update_dimer(d, pinned.data_ptr() + 8 * o, on_device=0, asynchronous=True)
            o += blk.size
        ctx.run()
        assert np.array_equal(ctx.energies()[2], base)
        # device update of dimer 0: integrals x4, terms x16
        A, K = blocks[0]
        dev = torch.from_numpy(4.0 * np.concatenate([A.ravel(), K.ravel()])).cuda()
        ctx.update_dimer(0, dev.data_ptr(), on_device=1)
        ctx.run()
        pd3 = ctx.energies()[2]
        assert np.array_equal(pd3[0], 16.0 * base[0]) and np.array_equal(pd3[1:], base[1:])
        # errors
        with pytest.raises(M.McptError) as ei:
            ctx.update_dimer(w.n_dimers, dev.data_ptr(), on_device=1)
        assert ei.value.status == M.MCPT_EINVAL
