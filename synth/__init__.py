"""Seeded synthetic inputs for the MCPT(2) dimer second-order term.

This module is the one input generator that both the FP64 CPU oracle and the
CUDA library are fed from.  It holds none of the method's arithmetic (no
four-index transformation, no denominators, no energies): it only draws

* monomer orbital coefficients C (Householder-QR orthonormal, columns = MOs,
  the first ``nocc`` occupied) and orbital energies eps,
* per-dimer symmetric Gaussian factors B^Q (a density-fitting-like stand-in
  for real integrals, which need basis sets and an integral code), and
* the AO two-electron integral blocks built from them,
  (mu nu|lam sig) = s^[cross] * sum_Q B^Q_{mu nu} B^Q_{lam sig},
  with s = exp(-R_XY / 2 Angstrom) applied to every element whose four AO
  indices are not all on one monomer,
* lattices of monomer sites and their dimer lists.

Every random number comes from Philox4x32-10 (Salmon, Moraes, Dror, Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC'11), keyed by the global seed
and counted by (object, index), so any object can be regenerated alone, on the
host here or on the device by ``synth.device``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED = 20141409
KAPPA = 0.01
NAUX = 192
SPACING = 3.0  # Angstrom, cubic lattice
KEY1 = 0x4D435054  # second key word: ASCII "MCPT"

# counter word 3 ("purpose tag") of every Philox draw
TAG_C = 1
TAG_EPS_OCC = 2
TAG_EPS_VIRT = 3
TAG_B = 4
TAG_SIZES = 5
TAG_R = 6
TAG_RING = 7
TAG_UAMP = 8
# scales of the synthetic monomer doubles matrices of Eq. (td2): the ring
# matrix 2 v^{i1 a}_{a1 i} - v^{a i1}_{a1 i} (monomer integrals, ~1e-3 at
# kappa = 0.01) and 2 T^{a a1}_{i i1} - T^{a a1}_{i1 i} (first-order monomer
# amplitudes, ~v D)
RING_SCALE = 2e-3
UAMP_SCALE = 1e-3

_M0, _M1 = np.uint64(0xD2511F53), np.uint64(0xCD9E8D57)
_W0, _W1 = np.uint64(0x9E3779B9), np.uint64(0xBB67AE85)
_MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox4x32 with 10 rounds on uint32 words held in uint64 arrays.

    One round: (hi0, lo0) = M0*c0, (hi1, lo1) = M1*c2 (full 64-bit products);
    c <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0); the key is then bumped by
    the Weyl constants (W0, W1).
    """
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) & _MASK for c in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint64) & _MASK
    k1 = np.asarray(k1, dtype=np.uint64) & _MASK
    for _ in range(10):
        p0 = _M0 * c0
        p1 = _M1 * c2
        c0, c1, c2, c3 = ((p1 >> np.uint64(32)) ^ c1 ^ k0, p1 & _MASK,
                          (p0 >> np.uint64(32)) ^ c3 ^ k1, p0 & _MASK)
        k0 = (k0 + _W0) & _MASK
        k1 = (k1 + _W1) & _MASK
    return c0, c1, c2, c3


def _u53(hi, lo):
    """Two uint32 words -> double uniform in [0, 1) with 53 random bits."""
    return ((hi >> np.uint64(5)).astype(np.float64) * 67108864.0
            + (lo >> np.uint64(6)).astype(np.float64)) / 9007199254740992.0


def uniforms(seed, obj, sub, tag, count):
    """``count`` uniforms in [0,1); draw k uses counter (k//2, obj, sub, tag)."""
    k = np.arange((count + 1) // 2, dtype=np.uint64)
    r0, r1, r2, r3 = philox4x32_10(k, obj, sub, tag, seed, KEY1)
    u = np.empty(2 * k.size)
    u[0::2] = _u53(r0, r1)
    u[1::2] = _u53(r2, r3)
    return u[:count]


def normals(seed, obj, sub, tag, count):
    """``count`` N(0,1) draws; pair k = Box-Muller of the k-th Philox block.

    z0 = sqrt(-2 ln(1-u0)) cos(2 pi u1), z1 = sqrt(-2 ln(1-u0)) sin(2 pi u1).
    """
    k = np.arange((count + 1) // 2, dtype=np.uint64)
    r0, r1, r2, r3 = philox4x32_10(k, obj, sub, tag, seed, KEY1)
    u0 = _u53(r0, r1)
    u1 = _u53(r2, r3)
    rad = np.sqrt(-2.0 * np.log1p(-u0))
    z = np.empty(2 * k.size)
    z[0::2] = rad * np.cos(2.0 * math.pi * u1)
    z[1::2] = rad * np.sin(2.0 * math.pi * u1)
    return z[:count]


# ----------------------------------------------------------------- monomers
@dataclass
class Monomer:
    C: np.ndarray     # [nao][nao] row-major: C[mu][p], columns are MOs
    eps: np.ndarray   # [nao]: occupied ascending, then virtual ascending
    nocc: int

    @property
    def nao(self) -> int:
        return self.C.shape[0]


def monomer(X: int, nao: int, nocc: int, seed: int = SEED) -> Monomer:
    """Orthonormal C = Q of a Householder QR of an nao x nao N(0,1) matrix,
    column signs fixed so that diag(R) > 0; eps_occ ~ U[-1.5,-0.5),
    eps_virt ~ U[0.2, 3.0), each sorted ascending."""
    g = normals(seed, X, 0, TAG_C, nao * nao).reshape(nao, nao)
    q, r = np.linalg.qr(g)
    q = q * np.where(np.diag(r) < 0, -1.0, 1.0)[None, :]
    eo = np.sort(-1.5 + uniforms(seed, X, 0, TAG_EPS_OCC, nocc))
    ev = np.sort(0.2 + 2.8 * uniforms(seed, X, 0, TAG_EPS_VIRT, nao - nocc))
    return Monomer(np.ascontiguousarray(q), np.concatenate([eo, ev]), nocc)


def monomer_doubles(X: int, nao: int, nocc: int, seed: int = SEED):
    """Synthetic stand-ins for monomer X's quantities in Eq. (td2): the ring
    matrix G and the amplitude matrix U, each (o v) x (o v) (index i v + a),
    symmetric like the quantities they stand for: scale (R + R^T) / sqrt(2),
    R of N(0,1) draws of stream (X, 0, tag)."""
    m = nocc * (nao - nocc)
    out = []
    for tag, scale in ((TAG_RING, RING_SCALE), (TAG_UAMP, UAMP_SCALE)):
        r = normals(seed, X, 0, tag, m * m).reshape(m, m)
        out.append(scale * (r + r.T) / math.sqrt(2.0))
    return out[0], out[1]


# ------------------------------------------------------------------ dimers
def dimer_object_id(X: int, Y: int) -> int:
    return (X << 16) | Y


def factors(X: int, Y: int, nX: int, nY: int, naux: int = NAUX,
            kappa: float = KAPPA, seed: int = SEED) -> np.ndarray:
    """B[Q][p][q] = kappa (G^Q_pq + G^Q_qp)/sqrt(2) over the dimer AO space
    (n = nX + nY, X's functions first); G^Q_pq is draw (p*n + q) of stream
    (dimer, Q).  Exactly symmetric."""
    n = nX + nY
    obj = dimer_object_id(X, Y)
    B = np.empty((naux, n, n))
    for q in range(naux):
        g = normals(seed, obj, q, TAG_B, n * n).reshape(n, n)
        B[q] = kappa * (g + g.T) / math.sqrt(2.0)
    return B


def _pair_index(n):
    """Packed index of the unordered pair (p, q), symmetric in p, q."""
    p = np.arange(n)[:, None]
    q = np.arange(n)[None, :]
    hi = np.maximum(p, q)
    lo = np.minimum(p, q)
    return hi * (hi + 1) // 2 + lo


def _pair_products(B):
    """M[P][Q] = sum_aux B[aux][P] B[aux][Q] over packed pairs, made exactly
    symmetric, so that every tensor built from it has exact 8-fold symmetry."""
    naux, n, _ = B.shape
    il = np.tril_indices(n)
    Bp = B[:, il[0], il[1]]                     # [naux][npairs], pair order = _pair_index
    M = Bp.T @ Bp
    return 0.5 * (M + M.T)


def scale_for_distance(R: float) -> float:
    return math.exp(-R / 2.0)


def eri_full(B, nX: int, s: float) -> np.ndarray:
    """Full dimer tensor G[mu][nu][lam][sig] over n = nX+nY functions."""
    n = B.shape[1]
    M = _pair_products(B)
    P = _pair_index(n)
    G = M[P.reshape(-1)][:, P.reshape(-1)].reshape(n, n, n, n)
    onX = np.arange(n) < nX
    allX = onX[:, None, None, None] & onX[None, :, None, None] & onX[None, None, :, None] & onX[None, None, None, :]
    allY = ~onX[:, None, None, None] & ~onX[None, :, None, None] & ~onX[None, None, :, None] & ~onX[None, None, None, :]
    return np.where(allX | allY, G, s * G)


def eri_blocks(B, nX: int, s: float):
    """The two blocks the dimer term reads, as contiguous arrays:
    A[mu][nu][lam][sig] = G[mu][nu][nX+lam][nX+sig]  (Coulomb-type (XX|YY))
    K[mu][lam][sig][nu] = G[mu][nX+lam][nX+sig][nu]  (exchange-type (XY|YX)).
    Bitwise equal to the same elements of ``eri_full``."""
    n = B.shape[1]
    nY = n - nX
    M = _pair_products(B)
    P = _pair_index(n)
    x = np.arange(nX)
    y = nX + np.arange(nY)
    A = M[P[np.ix_(x, x)].reshape(-1)][:, P[np.ix_(y, y)].reshape(-1)].reshape(nX, nX, nY, nY)
    K = M[P[np.ix_(x, y)].reshape(-1)][:, P[np.ix_(y, x)].reshape(-1)].reshape(nX, nY, nY, nX)
    return np.ascontiguousarray(s * A), np.ascontiguousarray(s * K)


def eri_blocks_direct(B, nX: int, s: float):
    """The same two blocks straight from factor products, for dimers too large
    for the packed-pair route (equal to ``eri_blocks`` up to FP64 rounding;
    not bitwise 8-fold symmetric)."""
    naux, n, _ = B.shape
    nY = n - nX
    bxx = B[:, :nX, :nX].reshape(naux, -1)
    byy = B[:, nX:, nX:].reshape(naux, -1)
    bxy = B[:, :nX, nX:].reshape(naux, -1)
    byx = B[:, nX:, :nX].reshape(naux, -1)
    A = (s * (bxx.T @ byy)).reshape(nX, nX, nY, nY)
    K = (s * (bxy.T @ byx)).reshape(nX, nY, nY, nX)
    return np.ascontiguousarray(A), np.ascontiguousarray(K)


def extract_blocks(G, nX: int):
    """A and K blocks cut out of a full tensor (layout conversion only)."""
    A = G[:nX, :nX, nX:, nX:]
    K = G[:nX, nX:, nX:, :nX]
    return np.ascontiguousarray(A), np.ascontiguousarray(K)


def packed_elems(nX: int, nY: int) -> int:
    """Length of the symmetry-packed [A_p | K_p] of an nX + nY dimer."""
    tX, tY, pq = nX * (nX + 1) // 2, nY * (nY + 1) // 2, nX * nY
    return tX * tY + pq * (pq + 1) // 2


def packed_gather_index(nX: int, nY: int):
    """Flat indices into [A | K] (BLOCKS layout, 2 nX^2 nY^2) whose elements,
    in order, form the packed layout: packed = blocks[index]."""
    ix, iy = np.tril_indices(nX), np.tril_indices(nY)
    ia = ((ix[0][:, None] * nX + ix[1][:, None]) * nY + iy[0][None, :]) * nY + iy[1][None, :]
    ip = np.tril_indices(nX * nY)
    mu, la = np.divmod(ip[0], nY)
    nu, sg = np.divmod(ip[1], nY)
    ik = nX * nX * nY * nY + ((mu * nY + la) * nY + sg) * nX + nu
    return np.concatenate([ia.ravel(), ik]).astype(np.int64)


def pack_blocks(A, K):
    """The unique elements of symmetric A[mu][nu][lam][sig] and
    K[mu][lam][sig][nu] in the packed order of the library's MCPT_AO_PACKED
    layout (layout conversion only): A_p[t(mu,nu)][t(lam,sig)] over
    mu >= nu, lam >= sig, then the lower triangle of M[P][Q] =
    K[mu][lam][sig][nu], P = mu nY + lam, Q = nu nY + sig; t(a,b) =
    a(a+1)/2 + b.  Elements above the triangles are not read."""
    nX, nY = A.shape[0], A.shape[2]
    ix, iy = np.tril_indices(nX), np.tril_indices(nY)
    Ap = A[ix[0], ix[1]][:, iy[0], iy[1]]
    M = np.transpose(K, (0, 1, 3, 2)).reshape(nX * nY, nX * nY)
    ip = np.tril_indices(nX * nY)
    return np.concatenate([Ap.ravel(), M[ip]])


# ----------------------------------------------------------------- lattices
@dataclass
class Workload:
    """A set of monomers and the dimer list (X < Y) with distances R_XY."""
    name: str
    nao: list = field(default_factory=list)
    nocc: list = field(default_factory=list)
    pairs: list = field(default_factory=list)   # (X, Y), X < Y
    R: list = field(default_factory=list)       # Angstrom
    seed: int = SEED

    @property
    def n_monomers(self) -> int:
        return len(self.nao)

    @property
    def n_dimers(self) -> int:
        return len(self.pairs)

    def monomer(self, X: int) -> Monomer:
        return monomer(X, self.nao[X], self.nocc[X], self.seed)

    def factors(self, d: int) -> np.ndarray:
        X, Y = self.pairs[d]
        return factors(X, Y, self.nao[X], self.nao[Y], seed=self.seed)

    def blocks(self, d: int):
        X, Y = self.pairs[d]
        return eri_blocks(self.factors(d), self.nao[X], scale_for_distance(self.R[d]))

    def full(self, d: int):
        X, Y = self.pairs[d]
        return eri_full(self.factors(d), self.nao[X], scale_for_distance(self.R[d]))


def cubic_lattice(L: int, cheb: int, nao: int, nocc: int, name: str = "",
                  seed: int = SEED, spacing: float = SPACING) -> Workload:
    """L^3 sites at spacing 3.0 A, id = ix + L(iy + L iz); all unordered pairs
    with Chebyshev lattice distance in [1, cheb]; R = Euclidean site distance."""
    ids = np.arange(L ** 3)
    ix, iy, iz = ids % L, (ids // L) % L, ids // (L * L)
    w = Workload(name or f"cubic{L}x{L}x{L}-cheb{cheb}", [nao] * L ** 3, [nocc] * L ** 3, seed=seed)
    for X in range(L ** 3):
        for Y in range(X + 1, L ** 3):
            dx, dy, dz = abs(ix[X] - ix[Y]), abs(iy[X] - iy[Y]), abs(iz[X] - iz[Y])
            if max(dx, dy, dz) <= cheb:
                w.pairs.append((X, Y))
                w.R.append(spacing * math.sqrt(dx * dx + dy * dy + dz * dz))
    return w


SIZE_CLASSES = (16, 24, 32, 40, 48, 56, 64, 72, 80, 88, 96)


def nocc_for(nao: int) -> int:
    """nocc = nao/6 rounded to nearest (n/6 has fractional part 0, 1/3 or 2/3)."""
    return int(math.floor(nao / 6.0 + 0.5))


def batched_uneven(n_dimers: int = 4096, seed: int = SEED) -> Workload:
    """2*n_dimers monomers, nao uniform over 16,24,...,96, dimer k = (2k, 2k+1),
    R drawn uniformly from the first-shell distances {3.0, 3*sqrt2, 3*sqrt3}."""
    nmon = 2 * n_dimers
    u = uniforms(seed, 0, 0, TAG_SIZES, nmon)
    nao = [SIZE_CLASSES[min(int(x * len(SIZE_CLASSES)), len(SIZE_CLASSES) - 1)] for x in u]
    shells = (SPACING, SPACING * math.sqrt(2.0), SPACING * math.sqrt(3.0))
    ur = uniforms(seed, 0, 0, TAG_R, n_dimers)
    w = Workload(f"batched-uneven-{n_dimers}", nao, [nocc_for(n) for n in nao], seed=seed)
    for k in range(n_dimers):
        w.pairs.append((2 * k, 2 * k + 1))
        w.R.append(shells[min(int(ur[k] * 3), 2)])
    return w


WORKLOADS = {
    "lattice-2x2x2": lambda: cubic_lattice(2, 1, 32, 5, "lattice-2x2x2"),
    "lattice-5x5x5-cheb1": lambda: cubic_lattice(5, 1, 32, 5, "lattice-5x5x5-cheb1"),
    "uneven-4096": lambda: batched_uneven(4096),
    "lattice-10x10x10-cheb2": lambda: cubic_lattice(10, 2, 32, 5, "lattice-10x10x10-cheb2"),
    "lattice-7x7x7-cheb1-ao128": lambda: cubic_lattice(7, 1, 128, 20, "lattice-7x7x7-cheb1-ao128"),
}


def workload(name: str) -> Workload:
    """Named synthetic workloads.  The 32-AO / 5-occupied monomer matches the
    size of HF in aug-cc-pCVDZ used for the paper's HF crystal (Sec. IV), and
    the lattices span 2^3 to 10^3 sites as that study does.
      lattice-2x2x2             8 monomers, all 28 dimers
      lattice-5x5x5-cheb1       125 monomers, 1036 dimers (Chebyshev <= 1)
      uneven-4096               8192 monomers of 16..96 AO, 4096 dimers
      lattice-10x10x10-cheb2    1000 monomers, 42092 dimers (Chebyshev <= 2)
      lattice-7x7x7-cheb1-ao128 343 monomers of 128 AO / 20 occ, 3258 dimers
    """
    return WORKLOADS[name]()
