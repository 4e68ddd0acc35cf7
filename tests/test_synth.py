"""The seeded input generator: Philox known answers, distributions, shapes."""
import math

import numpy as np

import synth


def test_philox_known_answers():
    """Known-answer vectors of Philox4x32-10 (Random123 distribution)."""
    cases = [
        ((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
        ((0xFFFFFFFF,) * 4, (0xFFFFFFFF,) * 2, (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
        ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
         (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
    ]
    for ctr, key, want in cases:
        got = synth.philox4x32_10(*ctr, *key)
        assert tuple(int(x) for x in got) == want


def test_normals_and_uniforms_statistics():
    z = synth.normals(synth.SEED, 1, 2, synth.TAG_B, 200001)
    assert z.size == 200001
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1.0) < 0.01
    u = synth.uniforms(synth.SEED, 1, 2, synth.TAG_R, 100000)
    assert u.min() >= 0.0 and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.01
    # counter-based: a prefix of a longer draw equals a shorter draw
    assert np.array_equal(synth.normals(synth.SEED, 1, 2, synth.TAG_B, 11), z[:11])


def test_monomer_orthonormal_and_sorted():
    m = synth.monomer(17, 32, 5)
    assert np.abs(m.C.T @ m.C - np.eye(32)).max() < 1e-13
    eo, ev = m.eps[:5], m.eps[5:]
    assert np.all(np.diff(eo) > 0) and np.all(np.diff(ev) > 0)
    assert eo.min() >= -1.5 and eo.max() < -0.5 and ev.min() >= 0.2 and ev.max() < 3.0
    assert np.array_equal(m.C, synth.monomer(17, 32, 5).C)


def test_workload_sizes():
    assert synth.workload("lattice-2x2x2").n_dimers == 28
    w = synth.workload("lattice-5x5x5-cheb1")
    assert w.n_monomers == 125 and w.n_dimers == 1036
    R = np.round(w.R, 3)
    assert (R == 3.0).sum() == 300 and (R == 4.243).sum() == 480 and (R == 5.196).sum() == 256
    u = synth.workload("uneven-4096")
    assert u.n_dimers == 4096 and set(u.nao) == set(synth.SIZE_CLASSES)
    assert all(o == synth.nocc_for(n) for n, o in zip(u.nao, u.nocc))
    assert synth.nocc_for(32) == 5 and synth.nocc_for(16) == 3 and synth.nocc_for(40) == 7


def test_blocks_scale():
    w = synth.workload("lattice-2x2x2")
    A, K = w.blocks(0)
    assert A.shape == (32, 32, 32, 32) and K.shape == (32, 32, 32, 32)
    s = synth.scale_for_distance(w.R[0])
    assert abs(s - math.exp(-1.5)) < 1e-15
    # |ERI| ~ s kappa^2 sqrt(naux) scale
    assert 1e-4 < np.abs(A).mean() / s < 1e-2
