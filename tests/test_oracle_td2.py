"""Pins of the oracle's dimer doubles iteration, Eq. (td2) (CPU only).

* One Jacobi step from zero is the first-order amplitude T = v D, so its
  energies equal the independent first-order routine.
* The converged amplitudes satisfy the equation as printed: its residual is
  evaluated here term by term with einsum straight from the AO block (each
  transformed block formed by its own contraction, no shared code), on
  non-symmetric integrals and non-symmetric monomer matrices, so that a
  wrong index placement, a transposed matrix or a dropped or sign-flipped
  term leaves a residual.
* Exchanging the roles of X and Y (relabelled symmetric integrals, swapped
  monomer matrices) leaves both energies unchanged.
"""
import numpy as np

import oracle
import synth
from helpers import rand_dimer


def _mo(A, CX, CY, sl):
    """(p q|r s) over the four column ranges sl = (X p, X q, Y r, Y s)."""
    return np.einsum("mnls,mp,nq,lr,st->pqrt", A, CX[:, sl[0]], CX[:, sl[1]], CY[:, sl[2]], CY[:, sl[3]],
                     optimize=True)


def _residual(A, CX, eX, CY, eY, oX, oY, T, GX, GY, UX, UY):
    """(e_i + e_j - e_a - e_b) T - (v + S + L(T)) with every term as printed."""
    nX, nY = CX.shape[0], CY.shape[0]
    vX, vY = nX - oX, nY - oY
    o_x, v_x, o_y, v_y = slice(0, oX), slice(oX, nX), slice(0, oY), slice(oY, nY)
    v = _mo(A, CX, CY, (o_x, v_x, o_y, v_y))                 # (ia|jb)
    lad = _mo(A, CX, CY, (v_x, v_x, v_y, v_y))               # (a a1|b b1)
    hol = _mo(A, CX, CY, (o_x, o_x, o_y, o_y))               # (i1 i|j1 j)
    m3 = _mo(A, CX, CY, (o_x, o_x, v_y, v_y))                # (i1 i|b b1)
    m4 = _mo(A, CX, CY, (v_x, v_x, o_y, o_y))                # (a a1|j1 j)
    mX, mY = oX * vX, oY * vY
    S = (UX @ v.reshape(mX, mY) + v.reshape(mX, mY) @ UY.T).reshape(v.shape)
    L = (np.einsum("aAbB,iAjB->iajb", lad, T)
         + np.einsum("IiJj,IaJb->iajb", hol, T)
         - np.einsum("IibB,IajB->iajb", m3, T)
         - np.einsum("aAJj,iAJb->iajb", m4, T)
         + (GX @ T.reshape(mX, mY)).reshape(T.shape)
         + (T.reshape(mX, mY) @ GY.T).reshape(T.shape))
    e = eX[:oX, None, None, None] + eY[None, None, :oY, None] - eX[None, oX:, None, None] - eY[None, None, None, oY:]
    return e * T - (v + S + L), v


def _monomer_mats(rng, m, scale):
    R = rng.standard_normal((m, m)) * scale
    return R                                       # non-symmetric on purpose


def test_one_step_is_first_order():
    rng = np.random.default_rng(61)
    for nX, nY, oX, oY in [(7, 6, 2, 3), (9, 5, 4, 1)]:
        A, K, CX, eX, CY, eY = rand_dimer(rng, nX, nY, oX, oY)
        _, E, _ = oracle.td2(A, K, CX, eX, CY, eY, oX, oY, 1)
        E1 = oracle.dimer(A, K, CX, eX, CY, eY, oX, oY)
        assert abs(E[0] - E1[0]) <= 1e-14 * abs(E1[0])
        assert abs(E[1] - E1[1]) <= 1e-13 * abs(E1[0])


def test_converged_amplitudes_satisfy_the_printed_equation():
    rng = np.random.default_rng(62)
    for nX, nY, oX, oY in [(7, 6, 2, 3), (6, 8, 3, 2)]:
        A, K, CX, eX, CY, eY = rand_dimer(rng, nX, nY, oX, oY)
        A = A * 30.0                                # couplings large enough to matter
        mX, mY = oX * (nX - oX), oY * (nY - oY)
        GX, GY = _monomer_mats(rng, mX, 0.02), _monomer_mats(rng, mY, 0.02)
        UX, UY = _monomer_mats(rng, mX, 0.02), _monomer_mats(rng, mY, 0.02)
        T, E, dl = oracle.td2(A, K, CX, eX, CY, eY, oX, oY, 80, GX, GY, UX, UY)
        assert dl[-1] <= 1e-15 * np.abs(T).max()
        r, v = _residual(A, CX, eX, CY, eY, oX, oY, T, GX, GY, UX, UY)
        assert np.abs(r).max() <= 1e-12 * np.abs(v).max()
        # the iteration moved away from first order (the terms are not negligible)
        T1, _, _ = oracle.td2(A, K, CX, eX, CY, eY, oX, oY, 1, GX, GY, UX, UY)
        assert np.abs(T - T1).max() > 1e-3 * np.abs(T).max()
        assert abs(E[0] - 4 * np.sum(v * T)) <= 1e-13 * abs(E[0])


def test_exchange_of_monomers():
    rng = np.random.default_rng(63)
    nX, nY, oX, oY = 7, 5, 2, 2
    B = rng.standard_normal((5, nX + nY, nX + nY)) * 0.05
    A, K = synth.eri_blocks(B + np.transpose(B, (0, 2, 1)), nX, 0.8)
    _, _, CX, eX, CY, eY = rand_dimer(rng, nX, nY, oX, oY)
    mX, mY = oX * (nX - oX), oY * (nY - oY)
    GX, GY = _monomer_mats(rng, mX, 0.02), _monomer_mats(rng, mY, 0.02)
    UX, UY = _monomer_mats(rng, mX, 0.02), _monomer_mats(rng, mY, 0.02)
    _, E, _ = oracle.td2(A, K, CX, eX, CY, eY, oX, oY, 40, GX, GY, UX, UY)
    # (Y, X): A' = (YY|XX), K'[lam][mu][nu][sig] = K[mu][lam][sig][nu]
    A2 = np.ascontiguousarray(A.transpose(2, 3, 0, 1))
    K2 = np.ascontiguousarray(K.transpose(1, 0, 3, 2))
    _, E2, _ = oracle.td2(A2, K2, CY, eY, CX, eX, oY, oX, 40, GY, GX, UY, UX)
    assert abs(E2[0] - E[0]) <= 1e-13 * abs(E[0])
    assert abs(E2[1] - E[1]) <= 1e-12 * abs(E[0])
