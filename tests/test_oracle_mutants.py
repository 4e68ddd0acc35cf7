"""Planted mistakes in the oracle must be caught by its pins (CPU only).

Each mutant is a copy of oracle/oracle.c with one plausible mistake -- a
wrong index or axis, a transposed operand, a dropped term, a wrong factor or
sign -- compiled in a temporary directory and loaded in a subprocess, where
a compact set of the pins runs against it.  The unmodified source passes all
of them.
"""
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

MUTANTS = {
    "virtual index starts at 0": (
        "CX, nX, oX, nX - oX,    /* nu  -> a */\n                      CY, nY, 0, oY,          /* lam -> j */",
        "CX, nX, 0, nX - oX,     /* nu  -> a */\n                      CY, nY, 0, oY,          /* lam -> j */"),
    "exchange axes swapped": (
        "CY, nY, oY, nY - oY,    /* lam -> b */\n                      CY, nY, 0, oY,          /* sig -> j */",
        "CY, nY, 0, oY,          /* lam -> b */\n                      CY, nY, oY, nY - oY,    /* sig -> j */"),
    "factor 4 -> 2": ("ej += 4.0 * v * v * D;", "ej += 2.0 * v * v * D;"),
    "denominator sign": ("1.0 / (epsX[i] + epsY[j] - epsX[oX + a] - epsY[oY + b])",
                         "1.0 / (epsX[i] - epsY[j] - epsX[oX + a] - epsY[oY + b])"),
    "exchange integral dropped": ("ek += -2.0 * v * w * D;", "ek += -2.0 * v * v * D;"),
    "brute force lam/sig swapped": ("CY[la * nY + j] * CY[si * nY + oY + b]", "CY[si * nY + j] * CY[la * nY + oY + b]"),
    "compensation dropped": ("    return s + c;\n}", "    return s;\n}"),
    "whole term to each monomer": ("double v = 0.5 * E2[2 * d + f];", "double v = E2[2 * d + f];"),
    "coupling pairs T with the wrong row": ("s += V[q * mY + r] * T[p * mY + r] + V[p * mY + r] * T[q * mY + r];",
                                            "s += V[q * mY + r] * T[p * mY + r] + V[p * mY + r] * T[p * mY + r];"),
    "coupling without the denominator": ("T[e] = V[e] / (epsX[i] + epsY[k] - epsX[oX + a] - epsY[oY + c]);",
                                         "T[e] = V[e];"),
    "singles reads the amplitudes transposed": ("s += V[(((size_t)i * vX + a) * oY + k) * vY + c] * tY[k * vY + c];",
                                                "s += V[(((size_t)i * vX + a) * oY + k) * vY + c] * tY[c * oY + k];"),
    "singles Y side takes its own amplitudes": ("s += V[(((size_t)i * vX + a) * oY + k) * vY + c] * tX[i * vX + a];",
                                                "s += V[(((size_t)i * vX + a) * oY + k) * vY + c] * tY[k * vY + c];"),
    "td2 particle ladder dropped": ("r += G4(oX + a, oX + a1, oY + b, oY + b1) * T[IDX(i, a1, j, b1)];",
                                    "r += 0.0 * T[IDX(i, a1, j, b1)];"),
    "td2 hole ladder indices swapped": ("r += G4(i1, i, j1, j) * T[IDX(i1, a, j1, b)];",
                                        "r += G4(i, i1, j1, j) * T[IDX(i1, a, j1, b)];"),
    "td2 mixed term sign": ("r -= G4(i1, i, oY + b, oY + b1) * T[IDX(i1, a, j, b1)];",
                            "r += G4(i1, i, oY + b, oY + b1) * T[IDX(i1, a, j, b1)];"),
    "td2 ring matrix transposed": ("r += GX[((size_t)i * vX + a) * mX + (size_t)i1 * vX + a1] * T[IDX(i1, a1, j, b)];",
                                   "r += GX[((size_t)i1 * vX + a1) * mX + (size_t)i * vX + a] * T[IDX(i1, a1, j, b)];"),
    "td2 energy-tensor sign": ("const double t = r / (epsX[i] + epsY[j] - epsX[oX + a] - epsY[oY + b]);",
                               "const double t = -r / (epsX[i] + epsY[j] - epsX[oX + a] - epsY[oY + b]);"),
    "factor route exchange factors swapped": (
        "W[(((size_t)i * vY + b) * oY + j) * vX + a] += s * xy[i * vY + b] * yx[j * vX + a];",
        "W[(((size_t)i * vY + b) * oY + j) * vX + a] += s * xy[i * vY + b] * xx[i * vX + a];"),
    "factor route scale dropped": (
        "V[(((size_t)i * vX + a) * oY + j) * vY + b] += s * xx[i * vX + a] * yy[j * vY + b];",
        "V[(((size_t)i * vX + a) * oY + j) * vY + b] += xx[i * vX + a] * yy[j * vY + b];"),
}

CHECKS = r'''
import sys, numpy as np
sys.path.insert(0, ROOT)
import oracle, synth
oracle._SRC, oracle._LIB, oracle._lib = SRCFILE, LIBFILE, None
fails = []
def check(name, ok):
    if not ok: fails.append(name)
rng = np.random.default_rng(2)
nX, nY, oX, oY = 5, 4, 2, 1
A = rng.standard_normal((nX, nX, nY, nY)); K = rng.standard_normal((nX, nY, nY, nX))
CX = rng.standard_normal((nX, nX)); CY = rng.standard_normal((nY, nY))
V, Vb = oracle.transform_J(A, CX, CY, oX, oY), oracle.bruteforce_J(A, CX, CY, oX, oY)
W, Wb = oracle.transform_K(K, CX, CY, oX, oY), oracle.bruteforce_K(K, CX, CY, oX, oY)
Ve = np.einsum("mnls,mi,na,lj,sb->iajb", A, CX[:, :oX], CX[:, oX:], CY[:, :oY], CY[:, oY:])
check("bruteforce J", np.abs(V - Vb).max() <= 1e-13 * np.abs(Vb).max())
check("bruteforce K", np.abs(W - Wb).max() <= 1e-13 * np.abs(Wb).max())
check("einsum J", np.abs(Vb - Ve).max() <= 1e-12 * np.abs(Ve).max())
# hand-derived 2+2 dimer
CXh = np.array([[0.6, -0.8], [0.8, 0.6]]); CYh = np.eye(2)
Ah = np.full((2, 2, 2, 2), 100.0); Ah[:, :, 0, 1] = [[1, 2], [3, 4]]
Kh = np.full((2, 2, 2, 2), -50.0); Kh[:, 1, 0, :] = [[2, 0], [1, -1]]
EJ, EK = oracle.dimer(Ah, Kh, CXh, np.array([-1.0, 2.0]), CYh, np.array([-0.5, 1.5]), 1, 1)
check("hand E_J", abs(EJ + 0.04608) < 1e-14)
check("hand E_K", abs(EK + 0.19968) < 1e-14)
# rank-1 closed form
z = rng.standard_normal(13); B = np.outer(z, z)[None]
mX, mY = synth.monomer(10, 7, 2), synth.monomer(11, 6, 2)
s = 0.3
Ar, Kr = synth.eri_blocks(B, 7, s)
EJ, EK = oracle.dimer(Ar, Kr, mX.C, mX.eps, mY.C, mY.eps, 2, 2)
xi, yj = mX.C.T @ z[:7], mY.C.T @ z[7:]
ref = sum(4 * s * s * xi[i] ** 2 * xi[a] ** 2 * yj[j] ** 2 * yj[b] ** 2 /
          (mX.eps[i] + mY.eps[j] - mX.eps[a] - mY.eps[b])
          for i in range(2) for a in range(2, 7) for j in range(2) for b in range(2, 6))
check("rank-1 E_J", abs(EJ - ref) <= 1e-13 * abs(ref))
check("rank-1 E_K", abs(EK + 0.5 * EJ) <= 1e-13 * abs(EJ))
# accumulation
E2 = np.array([[1e16, 1.0], [1.0, 2.0], [-1e16, 3.0], [1.0, 4.0]])
mon, tot = oracle.accumulate(E2, np.array([0, 0, 1, 2]), np.array([1, 2, 2, 3]), 4)
check("Neumaier total", tot[0] == 2.0)
check("split conserves total", mon[:, 1].sum() == tot[1])
# coupling of Eq. (tm2): rank-1 closed form with degenerate energies, and symmetry
eo, ev = -0.8, 1.1
eXd = np.array([eo] * 2 + [ev] * 5); eYd = np.array([eo] * 2 + [ev] * 4)
Vr = oracle.transform_J(Ar, mX.C, mY.C, 2, 2)
RX = np.zeros((10, 10)); RY = np.zeros((8, 8))
oracle.coupling_add(Vr, eXd, eYd, 2, 2, RX, RY)
Dd = 1.0 / (2 * eo - 2 * ev)
u = np.outer(xi[:2], xi[2:]).ravel()
refR = 2 * Dd * s * s * np.sum(yj[:2] ** 2) * np.sum(yj[2:] ** 2) * np.outer(u, u)
check("coupling rank-1", np.max(np.abs(RX - refR)) <= 1e-13 * np.max(np.abs(refR)))
V2 = rng.standard_normal((2, 3, 1, 3)); e2X = np.array([-1.0, -0.7, 0.4, 0.9, 2.0]); e2Y = np.array([-0.6, 0.5, 1.2, 2.5])
R2X = np.zeros((6, 6)); R2Y = np.zeros((3, 3))
oracle.coupling_add(V2, e2X, e2Y, 2, 1, R2X, R2Y)
check("coupling symmetric", np.array_equal(R2X, R2X.T) and np.array_equal(R2Y, R2Y.T))
# singles of Eq. (tm1) against the AO-density route
for (n1, n2, o1, o2) in [(6, 8, 1, 5), (7, 6, 2, 3)]:
    A1 = rng.standard_normal((n1, n1, n2, n2))
    C1 = rng.standard_normal((n1, n1)); C2 = rng.standard_normal((n2, n2))
    t1 = rng.standard_normal((o1, n1 - o1)); t2 = rng.standard_normal((o2, n2 - o2))
    V1 = oracle.transform_J(A1, C1, C2, o1, o2)
    s1 = np.zeros_like(t1); s2 = np.zeros_like(t2)
    oracle.singles_add(V1, t1, t2, s1, s2)
    P2 = C2[:, :o2] @ t2 @ C2[:, o2:].T; P1 = C1[:, :o1] @ t1 @ C1[:, o1:].T
    r1 = C1[:, :o1].T @ np.einsum("mnls,ls->mn", A1, P2) @ C1[:, o1:]
    r2 = C2[:, :o2].T @ np.einsum("mnls,mn->ls", A1, P1) @ C2[:, o2:]
    check("singles X", np.abs(s1 - r1).max() <= 1e-12 * np.abs(r1).max())
    check("singles Y", np.abs(s2 - r2).max() <= 1e-12 * np.abs(r2).max())
# Eq. (td2): one step is first order; the converged amplitudes satisfy the printed equation
n1, n2, o1, o2 = 6, 7, 2, 3
v1, v2 = n1 - o1, n2 - o2
A3 = rng.standard_normal((n1, n1, n2, n2)) * 0.03; K3 = rng.standard_normal((n1, n2, n2, n1)) * 0.03
C1 = np.linalg.qr(rng.standard_normal((n1, n1)))[0]; C2 = np.linalg.qr(rng.standard_normal((n2, n2)))[0]
e1 = np.concatenate([np.sort(rng.uniform(-1.5, -0.5, o1)), np.sort(rng.uniform(0.2, 3.0, v1))])
e2 = np.concatenate([np.sort(rng.uniform(-1.5, -0.5, o2)), np.sort(rng.uniform(0.2, 3.0, v2))])
m1, m2 = o1 * v1, o2 * v2
GX = rng.standard_normal((m1, m1)) * 0.02; GY = rng.standard_normal((m2, m2)) * 0.02
UX = rng.standard_normal((m1, m1)) * 0.02; UY = rng.standard_normal((m2, m2)) * 0.02
_, Ea, _ = oracle.td2(A3, K3, C1, e1, C2, e2, o1, o2, 1)
Eb = oracle.dimer(A3, K3, C1, e1, C2, e2, o1, o2)
check("td2 one step", abs(Ea[0] - Eb[0]) <= 1e-13 * abs(Eb[0]))
T3, E3, _ = oracle.td2(A3, K3, C1, e1, C2, e2, o1, o2, 80, GX, GY, UX, UY)
def mo(sl):
    return np.einsum("mnls,mp,nq,lr,st->pqrt", A3, C1[:, sl[0]], C1[:, sl[1]], C2[:, sl[2]], C2[:, sl[3]])
ox, vx, oy, vy = slice(0, o1), slice(o1, n1), slice(0, o2), slice(o2, n2)
v3 = mo((ox, vx, oy, vy))
L3 = (np.einsum("aAbB,iAjB->iajb", mo((vx, vx, vy, vy)), T3) + np.einsum("IiJj,IaJb->iajb", mo((ox, ox, oy, oy)), T3)
      - np.einsum("IibB,IajB->iajb", mo((ox, ox, vy, vy)), T3) - np.einsum("aAJj,iAJb->iajb", mo((vx, vx, oy, oy)), T3)
      + (GX @ T3.reshape(m1, m2)).reshape(T3.shape) + (T3.reshape(m1, m2) @ GY.T).reshape(T3.shape)
      + (UX @ v3.reshape(m1, m2) + v3.reshape(m1, m2) @ UY.T).reshape(T3.shape))
ee = e1[:o1, None, None, None] + e2[None, None, :o2, None] - e1[None, o1:, None, None] - e2[None, None, None, o2:]
check("td2 residual", np.abs(ee * T3 - v3 - L3).max() <= 1e-11 * np.abs(v3).max())
# density-fitted factor route against the four-index transformation of the blocks it defines
n5, n6, o5, o6 = 6, 5, 2, 2
B5 = rng.standard_normal((4, n5 + n6, n5 + n6))
B5 = B5 + np.transpose(B5, (0, 2, 1))
A5, K5 = synth.eri_blocks(B5, n5, 0.7)
C5 = np.linalg.qr(rng.standard_normal((n5, n5)))[0]; C6 = np.linalg.qr(rng.standard_normal((n6, n6)))[0]
V5, W5 = oracle.factor_route(B5, 0.7, C5, C6, o5, o6)
V5r = oracle.transform_J(A5, C5, C6, o5, o6); W5r = oracle.transform_K(K5, C5, C6, o5, o6)
check("factor route J", np.abs(V5 - V5r).max() <= 1e-12 * np.abs(V5r).max())
check("factor route K", np.abs(W5 - W5r).max() <= 1e-12 * np.abs(W5r).max())
print("FAILS:" + ",".join(fails))
'''


def _run_checks(src_text):
    with tempfile.TemporaryDirectory() as tmp:
        src = os.path.join(tmp, "oracle.c")
        lib = os.path.join(tmp, "liboracle.so")
        with open(src, "w") as f:
            f.write(src_text)
        code = f"ROOT = {ROOT!r}\nSRCFILE = {src!r}\nLIBFILE = {lib!r}\n" + CHECKS
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
        if r.returncode != 0:
            return None, r.stderr[-500:]   # a crash also counts as caught
        line = [l for l in r.stdout.splitlines() if l.startswith("FAILS:")][0]
        fails = [x for x in line[len("FAILS:"):].split(",") if x]
        return fails, ""


def test_unmodified_oracle_passes_every_check():
    fails, err = _run_checks(open(SRC).read())
    assert fails == [], (fails, err)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name):
    old, new = MUTANTS[name]
    text = open(SRC).read()
    assert text.count(old) == 1, f"mutation site for '{name}' not found exactly once"
    fails, err = _run_checks(text.replace(old, new))
    assert fails is None or len(fails) > 0, f"mutant '{name}' passed every pin"
