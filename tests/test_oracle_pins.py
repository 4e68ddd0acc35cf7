"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics,
not by the oracle itself (CPU only).

Each test names the mistake class it guards against: a transposed operand, a
wrong index, a dropped term, a wrong sign or factor.
"""

import numpy as np
import pytest

import oracle
import synth
from conftest import read_golden
from helpers import rand_dimer

RNG_SEED = 1409


def _rand_dimer(rng, nX, nY, sym=False):
    A = rng.standard_normal((nX, nX, nY, nY))
    K = rng.standard_normal((nX, nY, nY, nX))
    CX = rng.standard_normal((nX, nX))
    CY = rng.standard_normal((nY, nY))
    return A, K, CX, CY


# ---------------------------------------------------------------- P1
@pytest.mark.parametrize("nX,nY,oX,oY", [(3, 3, 1, 1), (4, 3, 1, 2), (3, 5, 2, 1),
                                         (5, 4, 2, 1), (6, 6, 2, 2), (4, 6, 1, 2)])
def test_factorised_equals_bruteforce(nX, nY, oX, oY):
    """Eq. (dp2e) summed literally (n^8) vs the factorised quarter transforms,
    on NON-symmetric random blocks so that any index/axis mix-up shows."""
    rng = np.random.default_rng(RNG_SEED + nX * 7 + nY)
    A, K, CX, CY = _rand_dimer(rng, nX, nY)
    V, Vb = oracle.transform_J(A, CX, CY, oX, oY), oracle.bruteforce_J(A, CX, CY, oX, oY)
    W, Wb = oracle.transform_K(K, CX, CY, oX, oY), oracle.bruteforce_K(K, CX, CY, oX, oY)
    assert np.abs(V - Vb).max() <= 1e-13 * np.abs(Vb).max()
    assert np.abs(W - Wb).max() <= 1e-13 * np.abs(Wb).max()


def test_transform_matches_einsum_definition():
    """Independent library statement of Eq. (dp2e): numpy einsum over the full
    four-fold AO sum, same non-symmetric inputs."""
    rng = np.random.default_rng(RNG_SEED)
    nX, nY, oX, oY = 5, 6, 2, 3
    A, K, CX, CY = _rand_dimer(rng, nX, nY)
    Ve = np.einsum("mnls,mi,na,lj,sb->iajb", A, CX[:, :oX], CX[:, oX:], CY[:, :oY], CY[:, oY:])
    We = np.einsum("mlsn,mi,lb,sj,na->ibja", K, CX[:, :oX], CY[:, oY:], CY[:, :oY], CX[:, oX:])
    assert np.allclose(oracle.transform_J(A, CX, CY, oX, oY), Ve, rtol=0, atol=1e-12 * np.abs(Ve).max())
    assert np.allclose(oracle.transform_K(K, CX, CY, oX, oY), We, rtol=0, atol=1e-12 * np.abs(We).max())


# ---------------------------------------------------------------- golden
def test_hand_derived_dimer():
    """2+2 AO dimer worked by hand (tests/golden/hand_dimer_2x2.txt)."""
    g = read_golden("hand_dimer_2x2.txt")
    CX = np.array([[0.6, -0.8], [0.8, 0.6]])
    CY = np.eye(2)
    A = np.full((2, 2, 2, 2), 100.0)
    A[:, :, 0, 1] = [[1, 2], [3, 4]]
    K = np.full((2, 2, 2, 2), -50.0)
    K[:, 1, 0, :] = [[2, 0], [1, -1]]
    eX, eY = np.array([-1.0, 2.0]), np.array([-0.5, 1.5])
    V = oracle.transform_J(A, CX, CY, 1, 1)
    W = oracle.transform_K(K, CX, CY, 1, 1)
    assert V.shape == (1, 1, 1, 1) and W.shape == (1, 1, 1, 1)
    assert abs(V.item() - g["V"]) < 1e-14
    assert abs(W.item() - g["W"]) < 1e-14
    EJ, EK = oracle.dimer(A, K, CX, eX, CY, eY, 1, 1)
    assert abs(EJ - g["EJ"]) < 1e-15 and abs(EK - g["EK"]) < 1e-15


# ---------------------------------------------------------------- P2
def test_generator_eightfold_symmetry_and_blocks():
    """(mn|ls) = (nm|ls) = (mn|sl) = (ls|mn): bitwise, and the A/K blocks are
    bitwise the corresponding elements of the full tensor."""
    B = synth.factors(3, 5, 4, 3, naux=7)
    s = synth.scale_for_distance(4.2)
    G = synth.eri_full(B, 4, s)
    for perm in [(1, 0, 2, 3), (0, 1, 3, 2), (2, 3, 0, 1), (3, 2, 1, 0), (1, 0, 3, 2)]:
        assert np.array_equal(G, G.transpose(perm))
    A, K = synth.eri_blocks(B, 4, s)
    A2, K2 = synth.extract_blocks(G, 4)
    assert np.array_equal(A, A2) and np.array_equal(K, K2)
    # the distance scale touches exactly the cross-monomer elements
    G1 = synth.eri_full(B, 4, 1.0)
    assert np.array_equal(G[:4, :4, :4, :4], G1[:4, :4, :4, :4])
    assert np.array_equal(G[4:, 4:, 4:, 4:], G1[4:, 4:, 4:, 4:])
    assert np.array_equal(A, s * G1[:4, :4, 4:, 4:])


# ---------------------------------------------------------------- P3
def _dimer_from_full(G, nX, CX, eX, CY, eY, oX, oY):
    A, K = synth.extract_blocks(G, nX)
    return oracle.dimer(A, K, CX, eX, CY, eY, oX, oY)


def test_swap_invariance():
    """Adding the dimer as (Y, X) -- Y's functions first -- gives the same
    E_J and E_K (relabel i<->j, a<->b)."""
    nX, nY, oX, oY = 6, 5, 2, 1
    mX, mY = synth.monomer(0, nX, oX), synth.monomer(1, nY, oY)
    B = synth.factors(0, 1, nX, nY, naux=11)
    G = synth.eri_full(B, nX, synth.scale_for_distance(3.0))
    e = _dimer_from_full(G, nX, mX.C, mX.eps, mY.C, mY.eps, oX, oY)
    perm = np.concatenate([np.arange(nX, nX + nY), np.arange(nX)])
    Gs = G[np.ix_(perm, perm, perm, perm)]
    es = _dimer_from_full(Gs, nY, mY.C, mY.eps, mX.C, mX.eps, oY, oX)
    assert abs(e[0] - es[0]) <= 1e-14 * abs(e[0])
    assert abs(e[1] - es[1]) <= 1e-13 * abs(e[1])


# ---------------------------------------------------------------- P4
def _rank1_inputs(nX, nY, oX, oY, degenerate):
    rng = np.random.default_rng(77)
    z = rng.standard_normal(nX + nY)
    B = np.outer(z, z)[None]
    mX, mY = synth.monomer(10, nX, oX), synth.monomer(11, nY, oY)
    eX, eY = mX.eps.copy(), mY.eps.copy()
    if degenerate:
        eX[:oX], eX[oX:] = -0.9, 1.1
        eY[:oY], eY[oY:] = -0.9, 1.1
    return z, B, mX.C, eX, mY.C, eY


@pytest.mark.parametrize("degenerate", [True, False])
def test_rank1_closed_form(degenerate):
    """Separable integrals (pq|rs) = s z_p z_q z_r z_s give (ia|jb) = (ib|ja)
    = s xi_i xi_a yj_j yj_b with xi = C_X^T x, yj = C_Y^T y, hence
    E_J = 4 s^2 sum xi_i^2 xi_a^2 yj_j^2 yj_b^2 D, and E_K = -E_J/2; for
    degenerate eps: E_J = 4 s^2 aXo aXv aYo aYv / (2 e_o - 2 e_v)."""
    nX, nY, oX, oY = 7, 6, 2, 2
    z, B, CX, eX, CY, eY = _rank1_inputs(nX, nY, oX, oY, degenerate)
    s = synth.scale_for_distance(4.24)
    A, K = synth.eri_blocks(B, nX, s)
    EJ, EK = oracle.dimer(A, K, CX, eX, CY, eY, oX, oY)
    xi, yj = CX.T @ z[:nX], CY.T @ z[nX:]
    if degenerate:
        aXo, aXv = np.sum(xi[:oX] ** 2), np.sum(xi[oX:] ** 2)
        aYo, aYv = np.sum(yj[:oY] ** 2), np.sum(yj[oY:] ** 2)
        ref = 4 * s * s * aXo * aXv * aYo * aYv / (2 * -0.9 - 2 * 1.1)
    else:
        ref = 0.0
        for i in range(oX):
            for a in range(oX, nX):
                for j in range(oY):
                    for b in range(oY, nY):
                        ref += 4 * s * s * xi[i] ** 2 * xi[a] ** 2 * yj[j] ** 2 * yj[b] ** 2 / (
                            eX[i] + eY[j] - eX[a] - eY[b])
    assert abs(EJ - ref) <= 1e-13 * abs(ref)
    assert abs(EK + 0.5 * EJ) <= 1e-13 * abs(EJ)


# ---------------------------------------------------------------- P5
def _numpy_factor_route(B, s, CX, CY, oX, oY):
    nX = CX.shape[0]
    Xo, Xv, Yo, Yv = CX[:, :oX], CX[:, oX:], CY[:, :oY], CY[:, oY:]
    xx = np.einsum("mi,qmn,na->qia", Xo, B[:, :nX, :nX], Xv)
    yy = np.einsum("lj,qls,sb->qjb", Yo, B[:, nX:, nX:], Yv)
    xy = np.einsum("mi,qml,lb->qib", Xo, B[:, :nX, nX:], Yv)
    yx = np.einsum("sj,qsn,na->qja", Yo, B[:, nX:, :nX], Xv)
    V = s * np.einsum("qia,qjb->iajb", xx, yy)
    W = s * np.einsum("qib,qja->ibja", xy, yx)
    return V, W


def test_factor_route_three_ways():
    """Four-index route (oracle) == factor route (oracle C) == factor route
    (numpy einsum, written independently here) on a 32-AO lattice dimer."""
    w = synth.workload("lattice-2x2x2")
    d = 5
    X, Y = w.pairs[d]
    mX, mY = w.monomer(X), w.monomer(Y)
    B = w.factors(d)
    s = synth.scale_for_distance(w.R[d])
    A, K = synth.eri_blocks(B, 32, s)
    V4, W4 = oracle.transform_J(A, mX.C, mY.C, 5, 5), oracle.transform_K(K, mX.C, mY.C, 5, 5)
    Vf, Wf = oracle.factor_route(B, s, mX.C, mY.C, 5, 5)
    Vn, Wn = _numpy_factor_route(B, s, mX.C, mY.C, 5, 5)
    for a, b in [(V4, Vf), (Vf, Vn), (W4, Wf), (Wf, Wn)]:
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()
    e4 = oracle.energy_from_mo(V4, W4, mX.eps, mY.eps, 5, 5)
    ef = oracle.energy_from_mo(Vf, Wf, mX.eps, mY.eps, 5, 5)
    assert abs(e4[0] - ef[0]) <= 1e-12 * abs(ef[0])
    assert abs(e4[1] - ef[1]) <= 1e-12 * abs(ef[0])


# ---------------------------------------------------------------- P6
def _orth(rng, n):
    q, r = np.linalg.qr(rng.standard_normal((n, n)))
    return q


def test_ao_rotation_invariance():
    """C_X' = U C_X with the X axes of the integrals rotated by U: same energies."""
    rng = np.random.default_rng(5)
    nX, nY, oX, oY = 6, 5, 2, 2
    mX, mY = synth.monomer(2, nX, oX), synth.monomer(3, nY, oY)
    A, K = synth.eri_blocks(synth.factors(2, 3, nX, nY, naux=9), nX, 0.3)
    U = _orth(rng, nX)
    A2 = np.einsum("pm,qn,mnls->pqls", U, U, A)
    K2 = np.einsum("pm,qn,mlsn->plsq", U, U, K)
    e1 = oracle.dimer(A, K, mX.C, mX.eps, mY.C, mY.eps, oX, oY)
    e2 = oracle.dimer(A2, K2, U @ mX.C, mX.eps, mY.C, mY.eps, oX, oY)
    assert abs(e1[0] - e2[0]) <= 1e-12 * abs(e1[0])
    assert abs(e1[1] - e2[1]) <= 1e-12 * abs(e1[0])


# ---------------------------------------------------------------- P7
def test_eps_shift_and_kappa_scaling():
    nX, nY, oX, oY = 6, 6, 2, 1
    mX, mY = synth.monomer(4, nX, oX), synth.monomer(5, nY, oY)
    B = synth.factors(4, 5, nX, nY, naux=8)
    A, K = synth.eri_blocks(B, nX, 0.4)
    e = oracle.dimer(A, K, mX.C, mX.eps, mY.C, mY.eps, oX, oY)
    # a common shift of every orbital energy leaves every denominator unchanged
    es = oracle.dimer(A, K, mX.C, mX.eps + 0.375, mY.C, mY.eps + 0.375, oX, oY)
    assert abs(e[0] - es[0]) <= 1e-14 * abs(e[0]) and abs(e[1] - es[1]) <= 1e-13 * abs(e[0])
    # B -> 2B: integrals x4 exactly, energies x16 exactly
    A2, K2 = synth.eri_blocks(2.0 * B, nX, 0.4)
    e2 = oracle.dimer(A2, K2, mX.C, mX.eps, mY.C, mY.eps, oX, oY)
    assert e2[0] == 16.0 * e[0] and e2[1] == 16.0 * e[1]
    A3, K3 = synth.eri_blocks(3.0 * B, nX, 0.4)
    e3 = oracle.dimer(A3, K3, mX.C, mX.eps, mY.C, mY.eps, oX, oY)
    assert abs(e3[0] - 81.0 * e[0]) <= 1e-14 * abs(e3[0])


# ---------------------------------------------------------------- P8
def test_signs_zeros_and_distance():
    w = synth.workload("lattice-2x2x2")
    for d in (0, 13, 27):
        X, Y = w.pairs[d]
        mX, mY = w.monomer(X), w.monomer(Y)
        A, K = w.blocks(d)
        EJ, _ = oracle.dimer(A, K, mX.C, mX.eps, mY.C, mY.eps, 5, 5)
        assert EJ < 0.0
    # zero cross blocks give exactly zero
    z = np.zeros((6, 6, 5, 5)), np.zeros((6, 5, 5, 6))
    mX, mY = synth.monomer(0, 6, 2), synth.monomer(1, 5, 2)
    assert oracle.dimer(z[0], z[1], mX.C, mX.eps, mY.C, mY.eps, 2, 2) == (0.0, 0.0)
    # E scales as s^2 with the distance factor
    B = synth.factors(0, 1, 6, 5, naux=5)
    eR = [oracle.dimer(*synth.eri_blocks(B, 6, synth.scale_for_distance(R)), mX.C, mX.eps, mY.C, mY.eps, 2, 2)
          for R in (3.0, 9.0, 60.0)]
    r = (synth.scale_for_distance(9.0) / synth.scale_for_distance(3.0)) ** 2
    assert abs(eR[1][0] - r * eR[0][0]) <= 1e-13 * abs(eR[0][0])
    assert abs(eR[2][0]) < 1e-14 * abs(eR[0][0])


# ---------------------------------------------------------------- P9
def test_occupied_rotation_invariance_degenerate():
    """With degenerate occupied energies, rotating the occupied columns of C_X
    leaves the dimer energy unchanged (same for the virtuals)."""
    rng = np.random.default_rng(9)
    nX, nY, oX, oY = 7, 6, 3, 2
    mX, mY = synth.monomer(6, nX, oX), synth.monomer(7, nY, oY)
    eX = mX.eps.copy()
    eX[:oX] = -1.0
    eX[oX:] = 0.7
    A, K = synth.eri_blocks(synth.factors(6, 7, nX, nY, naux=6), nX, 0.5)
    e = oracle.dimer(A, K, mX.C, eX, mY.C, mY.eps, oX, oY)
    C2 = mX.C.copy()
    C2[:, :oX] = C2[:, :oX] @ _orth(rng, oX)
    C2[:, oX:] = C2[:, oX:] @ _orth(rng, nX - oX)
    e2 = oracle.dimer(A, K, C2, eX, mY.C, mY.eps, oX, oY)
    assert abs(e[0] - e2[0]) <= 1e-13 * abs(e[0])
    assert abs(e[1] - e2[1]) <= 1e-12 * abs(e[0])


# ---------------------------------------------------------------- accumulation
def test_accumulate_split_and_neumaier():
    E2 = np.array([[1e16, 1.0], [1.0, 2.0], [-1e16, 3.0], [1.0, 4.0]])
    X = np.array([0, 0, 1, 2])
    Y = np.array([1, 2, 2, 3])
    mon, tot = oracle.accumulate(E2, X, Y, 4)
    assert tot[0] == 2.0            # a naive left-to-right sum gives 0 or 1
    assert tot[1] == 10.0
    # half of each dimer term to each partner
    assert np.allclose(mon[:, 1], [0.5 * 1 + 0.5 * 2, 0.5 * 1 + 0.5 * 3, 0.5 * 2 + 0.5 * 3 + 0.5 * 4, 0.5 * 4])
    assert mon[:, 1].sum() == tot[1]


def test_lattice_monomer_sum_equals_total():
    w = synth.workload("lattice-2x2x2")
    items = []
    for d in range(0, 28, 4):
        X, Y = w.pairs[d]
        mX, mY = w.monomer(X), w.monomer(Y)
        A, K = w.blocks(d)
        items.append((A, K, mX.C, mX.eps, mY.C, mY.eps, 5, 5))
    E = oracle.dimers_parallel(items)
    sel = [w.pairs[d] for d in range(0, 28, 4)]
    mon, tot = oracle.accumulate(E, [p[0] for p in sel], [p[1] for p in sel], 8)
    assert abs(mon[:, 0].sum() - tot[0]) <= 1e-15 * abs(tot[0]) * 8
    assert abs(mon[:, 1].sum() - tot[1]) <= 1e-15 * abs(tot[0]) * 8
    for k, it in enumerate(items):
        assert tuple(E[k]) == oracle.dimer(*it)


# ---------------------------------------------------------------- coupling (Eq. tm2)
def _rand_mo(rng, nX, nY, oX, oY):
    vX, vY = nX - oX, nY - oY
    V = rng.standard_normal((oX, vX, oY, vY))
    eX = np.concatenate([np.sort(rng.uniform(-1.5, -0.5, oX)), np.sort(rng.uniform(0.2, 3.0, vX))])
    eY = np.concatenate([np.sort(rng.uniform(-1.5, -0.5, oY)), np.sort(rng.uniform(0.2, 3.0, vY))])
    return V, eX, eY


def test_coupling_literal_sum_and_symmetry():
    """The coupling summed literally over (i, a, i1, a1, k, c) as Eq. (tm2)
    writes it (v^{a1 k}_{i1 c} T^{ac}_{ik} + v^{ak}_{ic} T^{a1 c}_{i1 k}), for
    both monomers of a dimer; R is symmetric."""
    rng = np.random.default_rng(21)
    nX, nY, oX, oY = 5, 4, 2, 1
    V, eX, eY = _rand_mo(rng, nX, nY, oX, oY)
    vX, vY = nX - oX, nY - oY
    RX = np.zeros((oX * vX, oX * vX))
    RY = np.zeros((oY * vY, oY * vY))
    oracle.coupling_add(V, eX, eY, oX, oY, RX, RY)

    def T(i, a, k, c):
        return V[i, a, k, c] / (eX[i] + eY[k] - eX[oX + a] - eY[oY + c])

    for i in range(oX):
        for a in range(vX):
            for i1 in range(oX):
                for a1 in range(vX):
                    s = sum(V[i1, a1, k, c] * T(i, a, k, c) + V[i, a, k, c] * T(i1, a1, k, c)
                            for k in range(oY) for c in range(vY))
                    assert abs(RX[i * vX + a, i1 * vX + a1] - s) <= 1e-13 * (1 + abs(s))
    for j in range(oY):
        for b in range(vY):
            for j1 in range(oY):
                for b1 in range(vY):
                    s = sum(V[i, a, j1, b1] * T(i, a, j, b) + V[i, a, j, b] * T(i, a, j1, b1)
                            for i in range(oX) for a in range(vX))
                    assert abs(RY[j * vY + b, j1 * vY + b1] - s) <= 1e-13 * (1 + abs(s))
    assert np.array_equal(RX, RX.T) and np.array_equal(RY, RY.T)


def test_coupling_trace_is_half_the_dimer_energy():
    """tr R_X = 2 sum v^2 D = E_J / 2, and the same for R_Y: ties the coupling
    to the energy of Eq. (ed2) computed by the independent energy routine."""
    rng = np.random.default_rng(22)
    for nX, nY, oX, oY in [(7, 6, 2, 3), (9, 5, 4, 1)]:
        A, K, CX, eX, CY, eY = rand_dimer(rng, nX, nY, oX, oY)
        V = oracle.transform_J(A, CX, CY, oX, oY)
        W = oracle.transform_K(K, CX, CY, oX, oY)
        EJ, _ = oracle.energy_from_mo(V, W, eX, eY, oX, oY)
        RX = np.zeros((oX * (nX - oX),) * 2)
        RY = np.zeros((oY * (nY - oY),) * 2)
        oracle.coupling_add(V, eX, eY, oX, oY, RX, RY)
        assert abs(np.trace(RX) - EJ / 2) <= 1e-13 * abs(EJ)
        assert abs(np.trace(RY) - EJ / 2) <= 1e-13 * abs(EJ)


def test_coupling_rank1_closed_form():
    """Rank-1 separable integrals (naux = 1, B = z z^T) with degenerate
    orbital energies: (ia|jb) = s x_i x_a y_j y_b and D is one constant, so
    R_X = 2 D s^2 (sum_j y_j^2)(sum_b y_b^2) (x_i x_a)(x_i1 x_a1)."""
    nX, nY, oX, oY = 7, 6, 2, 2
    rng = np.random.default_rng(23)
    z = rng.standard_normal(nX + nY)
    s = 0.3
    A, K = synth.eri_blocks(np.outer(z, z)[None], nX, s)
    CX = np.linalg.qr(rng.standard_normal((nX, nX)))[0]
    CY = np.linalg.qr(rng.standard_normal((nY, nY)))[0]
    eo, ev = -0.8, 1.1
    eX = np.array([eo] * oX + [ev] * (nX - oX))
    eY = np.array([eo] * oY + [ev] * (nY - oY))
    V = oracle.transform_J(A, CX, CY, oX, oY)
    RX = np.zeros((oX * (nX - oX),) * 2)
    RY = np.zeros((oY * (nY - oY),) * 2)
    oracle.coupling_add(V, eX, eY, oX, oY, RX, RY)
    x, y = CX.T @ z[:nX], CY.T @ z[nX:]
    D = 1.0 / (2 * eo - 2 * ev)
    u = np.outer(x[:oX], x[oX:]).ravel()
    ref = 2 * D * s * s * np.sum(y[:oY] ** 2) * np.sum(y[oY:] ** 2) * np.outer(u, u)
    assert np.max(np.abs(RX - ref)) <= 1e-13 * np.max(np.abs(ref))
    w_ = np.outer(y[:oY], y[oY:]).ravel()
    refY = 2 * D * s * s * np.sum(x[:oX] ** 2) * np.sum(x[oX:] ** 2) * np.outer(w_, w_)
    assert np.max(np.abs(RY - refY)) <= 1e-13 * np.max(np.abs(refY))


# ---------------------------------------------------------------- singles environment term (Eq. tm1)
def _ao_route_singles(A, CX, CY, oX, oY, tX, tY):
    """sum_{kc} (ia|kc) t_kc through the AO integrals: the amplitudes become
    an AO matrix P = C_occ t C_virt^T of the neighbour, contracted with the
    Coulomb block over the neighbour's two AO indices and projected onto
    (i, a) -- no four-index MO tensor is formed."""
    PY = CY[:, :oY] @ tY @ CY[:, oY:].T
    PX = CX[:, :oX] @ tX @ CX[:, oX:].T
    FX = np.einsum("mnls,ls->mn", A, PY)
    FY = np.einsum("mnls,mn->ls", A, PX)
    return CX[:, :oX].T @ FX @ CX[:, oX:], CY[:, :oY].T @ FY @ CY[:, oY:]


def test_singles_against_ao_route():
    """The environment term of Eq. (tm1), v^{ak}_{ic} t^c_k summed over the
    neighbour's (k, c), agrees with the AO-density route for both monomers,
    on non-symmetric integrals and unequal sizes."""
    rng = np.random.default_rng(24)
    for nX, nY, oX, oY in [(7, 6, 2, 3), (9, 5, 4, 1), (6, 8, 1, 5)]:
        A, K, CX, eX, CY, eY = rand_dimer(rng, nX, nY, oX, oY)
        tX = rng.standard_normal((oX, nX - oX))
        tY = rng.standard_normal((oY, nY - oY))
        V = oracle.transform_J(A, CX, CY, oX, oY)
        sX, sY = np.zeros_like(tX), np.zeros_like(tY)
        oracle.singles_add(V, tX, tY, sX, sY)
        rX, rY = _ao_route_singles(A, CX, CY, oX, oY, tX, tY)
        assert np.max(np.abs(sX - rX)) <= 1e-13 * np.max(np.abs(rX))
        assert np.max(np.abs(sY - rY)) <= 1e-13 * np.max(np.abs(rY))
        # the pairing t_X . s_X = t_Y . s_Y = t_X^T V t_Y is symmetric
        assert abs(np.sum(tX * sX) - np.sum(tY * sY)) <= 1e-13 * np.sum(np.abs(tX * sX))


def test_singles_accumulates_and_is_linear():
    """Calls add into s; zero amplitudes give exactly zero; the term is
    linear in t."""
    rng = np.random.default_rng(25)
    oX, vX, oY, vY = 3, 4, 2, 5
    V = rng.standard_normal((oX, vX, oY, vY))
    tX, tY = rng.standard_normal((oX, vX)), rng.standard_normal((oY, vY))
    s1X, s1Y = np.zeros((oX, vX)), np.zeros((oY, vY))
    oracle.singles_add(V, tX, tY, s1X, s1Y)
    s2X, s2Y = s1X.copy(), s1Y.copy()
    oracle.singles_add(V, tX, tY, s2X, s2Y)
    assert np.array_equal(s2X, 2 * s1X) and np.array_equal(s2Y, 2 * s1Y)
    zX, zY = np.zeros((oX, vX)), np.zeros((oY, vY))
    oracle.singles_add(V, np.zeros_like(tX), np.zeros_like(tY), zX, zY)
    assert not zX.any() and not zY.any()
    s3X, s3Y = np.zeros((oX, vX)), np.zeros((oY, vY))
    oracle.singles_add(V, 4.0 * tX, 4.0 * tY, s3X, s3Y)
    assert np.array_equal(s3X, 4 * s1X) and np.array_equal(s3Y, 4 * s1Y)
