"""The symmetry-packed integral layout (MCPT_AO_PACKED) on the host: the
packer follows the layout's definition, and expanding the packed elements by
that definition gives back symmetric blocks exactly (CPU only)."""
import numpy as np

import synth


def _unpack(packed, nX, nY):
    """Expansion written from the layout's definition, element by element."""
    tY = nY * (nY + 1) // 2
    kOff = (nX * (nX + 1) // 2) * tY

    def t(a, b):
        a, b = max(a, b), min(a, b)
        return a * (a + 1) // 2 + b

    A = np.empty((nX, nX, nY, nY))
    K = np.empty((nX, nY, nY, nX))
    for mu in range(nX):
        for nu in range(nX):
            for la in range(nY):
                for sg in range(nY):
                    A[mu, nu, la, sg] = packed[t(mu, nu) * tY + t(la, sg)]
                    K[mu, la, sg, nu] = packed[kOff + t(mu * nY + la, nu * nY + sg)]
    return A, K


def test_pack_round_trip_on_symmetric_blocks():
    rng = np.random.default_rng(51)
    for nX, nY in [(3, 5), (6, 4), (5, 5)]:
        B = rng.standard_normal((4, nX + nY, nX + nY))
        B = B + np.transpose(B, (0, 2, 1))
        A, K = synth.eri_blocks(B, nX, 0.7)
        p = synth.pack_blocks(A, K)
        assert p.shape == (synth.packed_elems(nX, nY),)
        A2, K2 = _unpack(p, nX, nY)
        assert np.array_equal(A2, A) and np.array_equal(K2, K)


def test_packed_size_at_32_ao():
    # 528 x 528 Coulomb pairs and 1024 x 1025 / 2 exchange pairs
    assert synth.packed_elems(32, 32) == 278784 + 524800
    assert 2 * 32 ** 4 / synth.packed_elems(32, 32) > 2.6


def test_gather_index_matches_packer():
    rng = np.random.default_rng(53)
    for nX, nY in [(4, 6), (5, 3)]:
        B = rng.standard_normal((3, nX + nY, nX + nY))
        A, K = synth.eri_blocks(B + np.transpose(B, (0, 2, 1)), nX, 0.3)
        flat = np.concatenate([A.ravel(), K.ravel()])
        assert np.array_equal(flat[synth.packed_gather_index(nX, nY)], synth.pack_blocks(A, K))


def test_monomer_doubles_are_seeded_symmetric_and_scaled():
    G, U = synth.monomer_doubles(7, 32, 5)
    G2, U2 = synth.monomer_doubles(7, 32, 5)
    assert G.shape == U.shape == (135, 135)
    assert np.array_equal(G, G2) and np.array_equal(U, U2)                  # seeded
    assert np.array_equal(G, G.T) and np.array_equal(U, U.T)                # symmetric
    assert not np.array_equal(G, synth.monomer_doubles(8, 32, 5)[0])        # per monomer
    assert 0.5 * synth.RING_SCALE < G.std() < 2 * synth.RING_SCALE
    assert 0.5 * synth.UAMP_SCALE < U.std() < 2 * synth.UAMP_SCALE
