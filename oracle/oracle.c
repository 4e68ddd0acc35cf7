/*
 * oracle.c -- plain, slow FP64 CPU reference for the first-order MCPT(2)
 * dimer term.  TEST INFRASTRUCTURE ONLY: it is called by the tests, by
 * __graft_entry__.smoke() and by bench.py's CPU-baseline / reference legs,
 * never by the library.  It shares no code, header, table or helper with the
 * CUDA path.
 *
 * What it computes (Byrd et al., "Molecular Cluster Perturbation Theory. I",
 * Sec. II.B-II.C):
 *
 *  (1) Eq. (dp2e): the dimer MO integral
 *        (p r|q s) = sum_{mu nu in X, lam sig in Y} C_{mu p} C_{nu r} C_{lam q} C_{sig s} (mu nu|lam sig)
 *      with monomer-centred, mutually non-orthogonal orbitals (block-diagonal
 *      C, no orthogonalisation between monomers).  With p=i, r=a in X and
 *      q=j, s=b in Y this is v^{ij}_{ab} = (i a|j b) (real orbitals).
 *  (2) the exchange-type form (i b|j a) = sum C^X_{mu i} C^Y_{lam b} C^Y_{sig j} C^X_{nu a} (mu lam|sig nu)
 *      taken from the same dimer integrals (XY|YX).
 *  (3) energy tensor and denominator, Sec. II.C: eps^{ij}_{ab} = e_i + e_j - e_a - e_b,
 *      D = 1 / eps^{ij}_{ab}.
 *  (4) first-order dimer amplitude T^{ab}_{ij} = v^{ab}_{ij} D^{ij}_{ab}: Eq. (td2)
 *      with every amplitude-dependent term dropped (one Jacobi step from T=0),
 *      sign taken so that the energy below is <= 0.
 *  (5) Eq. (ed2): E_D2(XY) = 4 v^{ij}_{ab} T^{ab}_{ij} = 4 sum (ia|jb)^2 D      -> "E_J"
 *      and the exchange completion E_K(XY) = -2 sum (ia|jb)(ib|ja) D, reported
 *      separately (the 2J-K pattern of Eq. (em2)).
 *  (6) per-monomer accumulation: half of each dimer term to X and half to Y;
 *      lattice total = sum over the dimer list with Neumaier's compensated sum
 *      (the cluster Hamiltonian of Eq. (clusterH) is a sum over dimers).
 *
 * Storage conventions (all row-major, FP64):
 *   C[mu][p]            nao x nao, columns are MOs, the first nocc occupied
 *   eps[p]              nao
 *   A[mu][nu][lam][sig] nX*nX*nY*nY   (mu,nu in X; lam,sig in Y)
 *   K[mu][lam][sig][nu] nX*nY*nY*nX   (mu,nu in X; lam,sig in Y)
 *   V[i][a][j][b]       oX*vX*oY*vY   = (i a|j b)
 *   W[i][b][j][a]       oX*vY*oY*vX   = (i b|j a)
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------------- */
/* One quarter transformation: contract axis `ax` (0..3) of the 4-index     */
/* tensor T[d0][d1][d2][d3] with the columns c0..c0+m-1 of U[p][*] (U has    */
/* `ldu` columns): out[..t..] = sum_p U[p][c0+t] T[..p..].                  */
static void quarter(const double *T, const int d[4], int ax,
                    const double *U, int ldu, int c0, int m,
                    double *out)
{
    int od[4] = {d[0], d[1], d[2], d[3]};
    od[ax] = m;
    size_t n_out = (size_t)od[0] * od[1] * od[2] * od[3];
    memset(out, 0, n_out * sizeof(double));
    for (int i0 = 0; i0 < d[0]; i0++)
    for (int i1 = 0; i1 < d[1]; i1++)
    for (int i2 = 0; i2 < d[2]; i2++)
    for (int i3 = 0; i3 < d[3]; i3++) {
        int idx[4] = {i0, i1, i2, i3};
        double x = T[(((size_t)i0 * d[1] + i1) * d[2] + i2) * d[3] + i3];
        int p = idx[ax];
        for (int t = 0; t < m; t++) {
            idx[ax] = t;
            size_t o = (((size_t)idx[0] * od[1] + idx[1]) * od[2] + idx[2]) * od[3] + idx[3];
            out[o] += U[(size_t)p * ldu + c0 + t] * x;
        }
    }
}

/* Factorised O(n^5) transformation of a generic block E[p0][p1][p2][p3]:
 *   out[t0][t1][t2][t3] = sum E[p0 p1 p2 p3] U0[p0][c0+t0] U1[p1][c1+t1] U2[p2][c2+t2] U3[p3][c3+t3]
 * contracting the two occupied axes (0 and 2) first, then 3, then 1.  */
static int transform4(const double *E, const int n[4],
                      const double *U0, int ld0, int c0, int m0,
                      const double *U1, int ld1, int c1, int m1,
                      const double *U2, int ld2, int c2, int m2,
                      const double *U3, int ld3, int c3, int m3,
                      double *out)
{
    int d[4] = {n[0], n[1], n[2], n[3]};
    size_t s1 = (size_t)n[0] * n[1] * m2 * n[3];
    size_t s2 = (size_t)m0 * n[1] * m2 * n[3];
    size_t s3 = (size_t)m0 * n[1] * m2 * m3;
    double *t1 = malloc(s1 * sizeof(double));
    double *t2 = malloc(s2 * sizeof(double));
    double *t3 = malloc(s3 * sizeof(double));
    if (!t1 || !t2 || !t3) { free(t1); free(t2); free(t3); return -1; }
    quarter(E, d, 2, U2, ld2, c2, m2, t1);  d[2] = m2;
    quarter(t1, d, 0, U0, ld0, c0, m0, t2); d[0] = m0;
    quarter(t2, d, 3, U3, ld3, c3, m3, t3); d[3] = m3;
    quarter(t3, d, 1, U1, ld1, c1, m1, out);
    free(t1); free(t2); free(t3);
    return 0;
}

/* (i a|j b) from the Coulomb-type block A (Eq. dp2e with p=i, r=a, q=j, s=b). */
int oracle_transform_J(const double *A, const double *CX, const double *CY,
                       int nX, int nY, int oX, int oY, double *V)
{
    int n[4] = {nX, nX, nY, nY};
    return transform4(A, n,
                      CX, nX, 0, oX,          /* mu  -> i */
                      CX, nX, oX, nX - oX,    /* nu  -> a */
                      CY, nY, 0, oY,          /* lam -> j */
                      CY, nY, oY, nY - oY,    /* sig -> b */
                      V);
}

/* (i b|j a) from the exchange-type block K[mu][lam][sig][nu]. */
int oracle_transform_K(const double *K, const double *CX, const double *CY,
                       int nX, int nY, int oX, int oY, double *W)
{
    int n[4] = {nX, nY, nY, nX};
    return transform4(K, n,
                      CX, nX, 0, oX,          /* mu  -> i */
                      CY, nY, oY, nY - oY,    /* lam -> b */
                      CY, nY, 0, oY,          /* sig -> j */
                      CX, nX, oX, nX - oX,    /* nu  -> a */
                      W);
}

/* Energies from the transformed integrals: Eq. (ed2) with T = v D, and the
 * exchange completion.  Plain FP64 sums in (i, a, j, b) order. */
void oracle_energy_from_mo(const double *V, const double *W,
                           const double *epsX, const double *epsY,
                           int nX, int nY, int oX, int oY,
                           double *EJ, double *EK)
{
    int vX = nX - oX, vY = nY - oY;
    double ej = 0.0, ek = 0.0;
    for (int i = 0; i < oX; i++)
    for (int a = 0; a < vX; a++)
    for (int j = 0; j < oY; j++)
    for (int b = 0; b < vY; b++) {
        double D = 1.0 / (epsX[i] + epsY[j] - epsX[oX + a] - epsY[oY + b]);
        double v = V[(((size_t)i * vX + a) * oY + j) * vY + b];
        double w = W[(((size_t)i * vY + b) * oY + j) * vX + a];
        ej += 4.0 * v * v * D;
        ek += -2.0 * v * w * D;
    }
    *EJ = ej;
    *EK = ek;
}

/* Dimer -> monomer doubles coupling of Eq. (tm2) (the sum over c, k of the
 * neighbour Y) for this dimer, at the first-order dimer amplitude
 * T^{ac}_{ik} = v^{ac}_{ik} D^{ik}_{ac} (the same T as the energy above):
 *   R_X[(i,a)][(i1,a1)] += sum_{k,c} ( v^{a1 k}_{i1 c} T^{ac}_{ik} + v^{ak}_{ic} T^{a1 c}_{i1 k} )
 * with v^{ak}_{ic} = (i a|k c) = V[i][a][k][c] (i, a of X; k, c of Y), and the
 * same with the roles of X and Y exchanged for R_Y[(j,b)][(j1,b1)].  R_X is
 * (oX vX) x (oX vX) row-major, R_Y (oY vY) x (oY vY). */
void oracle_coupling_add(const double *V, const double *epsX, const double *epsY,
                         int nX, int nY, int oX, int oY, double *RX, double *RY)
{
    int vX = nX - oX, vY = nY - oY;
    size_t mX = (size_t)oX * vX, mY = (size_t)oY * vY;
    double *T = malloc(mX * mY * sizeof(double));
    if (!T) return;
    for (int i = 0; i < oX; i++)
    for (int a = 0; a < vX; a++)
    for (int k = 0; k < oY; k++)
    for (int c = 0; c < vY; c++) {
        size_t e = ((size_t)i * vX + a) * mY + (size_t)k * vY + c;
        T[e] = V[e] / (epsX[i] + epsY[k] - epsX[oX + a] - epsY[oY + c]);
    }
    /* X's matrix: (i,a) x (i1,a1), summed over the pairs (k,c) of Y */
    for (size_t p = 0; p < mX; p++)
    for (size_t q = 0; q < mX; q++) {
        double s = 0.0;
        for (size_t r = 0; r < mY; r++)
            s += V[q * mY + r] * T[p * mY + r] + V[p * mY + r] * T[q * mY + r];
        RX[p * mX + q] += s;
    }
    /* Y's matrix: (j,b) x (j1,b1), summed over the pairs (i,a) of X */
    for (size_t p = 0; p < mY; p++)
    for (size_t q = 0; q < mY; q++) {
        double s = 0.0;
        for (size_t r = 0; r < mX; r++)
            s += V[r * mY + q] * T[r * mY + p] + V[r * mY + p] * T[r * mY + q];
        RY[p * mY + q] += s;
    }
    free(T);
}

/* The environment term of the monomer singles equation, Eq. (tm1): monomer
 * X receives from each neighbour Y the sum over Y's occupied k and virtual c
 * of v^{ak}_{ic} t^c_k, with v^{ak}_{ic} = (i a|k c) = V[i][a][k][c] and Y's
 * singles amplitudes tY[k][c] (oY x vY row-major):
 *   sX[(i,a)] += sum_{k,c} V[i][a][k][c] tY[k][c]
 * and Y receives the same from X:
 *   sY[(k,c)] += sum_{i,a} V[i][a][k][c] tX[i][a]. */
void oracle_singles_add(const double *V, const double *tX, const double *tY,
                        int oX, int vX, int oY, int vY, double *sX, double *sY)
{
    for (int i = 0; i < oX; i++)
    for (int a = 0; a < vX; a++) {
        double s = 0.0;
        for (int k = 0; k < oY; k++)
        for (int c = 0; c < vY; c++)
            s += V[(((size_t)i * vX + a) * oY + k) * vY + c] * tY[k * vY + c];
        sX[i * vX + a] += s;
    }
    for (int k = 0; k < oY; k++)
    for (int c = 0; c < vY; c++) {
        double s = 0.0;
        for (int i = 0; i < oX; i++)
        for (int a = 0; a < vX; a++)
            s += V[(((size_t)i * vX + a) * oY + k) * vY + c] * tX[i * vX + a];
        sY[k * vY + c] += s;
    }
}

/* Dimer doubles amplitudes of Eq. (td2) by Jacobi steps from T = 0, and the
 * dimer energy of Eq. (ed2) at the final amplitudes.
 *
 * i, i1 (a, a1) run over X's occupied (virtual) orbitals, j, j1 (b, b1) over
 * Y's.  With g[p][q][r][s] = (p q|r s) the full MO transformation of the
 * Coulomb block (p, q MOs of X; r, s MOs of Y) and physicist integrals
 * <pq|rs> = (pr|qs), the equation's terms are
 *   v^{ab}_{ij}       = (ia|jb)                     = v[i][a][j][b]
 *   v^{ab}_{a1 b1}    = (a a1|b b1)                 (particle ladder)
 *   v^{i1 j1}_{ij}    = (i1 i|j1 j)                 (hole ladder)
 *   v^{b i1}_{b1 i}   = (b b1|i1 i) = (i1 i|b b1)   (enters with -)
 *   v^{a j1}_{a1 j}   = (a a1|j1 j)                 (enters with -)
 *   (2 v^{i1 a}_{a1 i} - v^{a i1}_{a1 i})           monomer X ring matrix GX[(i,a)][(i1,a1)]
 *   (2 v^{j1 b}_{b1 j} - v^{b j1}_{b1 j})           monomer Y ring matrix GY[(j,b)][(j1,b1)]
 *   v^{i1 b}_{a1 j} (2 T^{a a1}_{i i1} - T^{a a1}_{i1 i}) = sum UX[(i,a)][(i1,a1)] v[i1][a1][j][b]
 *   v^{j1 a}_{b1 i} (2 T^{b b1}_{j j1} - T^{b b1}_{j1 j}) = sum UY[(j,b)][(j1,b1)] v[i][a][j1][b1]
 * GX, GY, UX, UY are the monomers' own quantities (row-major (o v)^2,
 * index i*v + a), given by the caller; NULL means zero.  Each step sets
 *   T <- D (v + S + L(T)),  D = 1/(e_i + e_j - e_a - e_b),
 * S the two monomer-amplitude terms and L the six amplitude-dependent terms
 * with their signs as printed; the sign of the energy-tensor term is taken
 * as for the first-order amplitude (so that one step gives T = v D).
 * Energies: E_J = 4 sum v T (Eq. ed2), E_K = -2 sum (ib|ja) T.
 * T: out, [oX][vX][oY][vY]; E: out {E_J, E_K}; delta: out (n_iter values,
 * or NULL), max |T_new - T_old| of each step.  Returns 0 on success. */
int oracle_td2(const double *A, const double *K,
               const double *CX, const double *epsX, const double *CY, const double *epsY,
               int nX, int nY, int oX, int oY,
               const double *GX, const double *GY, const double *UX, const double *UY,
               int n_iter, double *T, double *E, double *delta)
{
    const int vX = nX - oX, vY = nY - oY;
    const size_t mX = (size_t)oX * vX, mY = (size_t)oY * vY, nt = mX * mY;
    const size_t ng = (size_t)nX * nX * nY * nY;
    int n[4] = {nX, nX, nY, nY};
    double *g = malloc(ng * sizeof(double));
    double *v = malloc(nt * sizeof(double));
    double *W = malloc(nt * sizeof(double));
    double *S = malloc(nt * sizeof(double));
    double *Tn = malloc(nt * sizeof(double));
    int rc = -1;
    if (!g || !v || !W || !S || !Tn) goto out;
    if (transform4(A, n, CX, nX, 0, nX, CX, nX, 0, nX, CY, nY, 0, nY, CY, nY, 0, nY, g)) goto out;
    if (oracle_transform_K(K, CX, CY, nX, nY, oX, oY, W)) goto out;
#define G4(p, q, r, s) g[(((size_t)(p) * nX + (q)) * nY + (r)) * nY + (s)]
#define IDX(i, a, j, b) ((((size_t)(i) * vX + (a)) * oY + (j)) * vY + (b))
    for (int i = 0; i < oX; i++)
    for (int a = 0; a < vX; a++)
    for (int j = 0; j < oY; j++)
    for (int b = 0; b < vY; b++)
        v[IDX(i, a, j, b)] = G4(i, oX + a, j, oY + b);
    for (int i = 0; i < oX; i++)
    for (int a = 0; a < vX; a++)
    for (int j = 0; j < oY; j++)
    for (int b = 0; b < vY; b++) {
        double s = 0.0;
        if (UX)
            for (int i1 = 0; i1 < oX; i1++)
            for (int a1 = 0; a1 < vX; a1++)
                s += UX[((size_t)i * vX + a) * mX + (size_t)i1 * vX + a1] * v[IDX(i1, a1, j, b)];
        if (UY)
            for (int j1 = 0; j1 < oY; j1++)
            for (int b1 = 0; b1 < vY; b1++)
                s += UY[((size_t)j * vY + b) * mY + (size_t)j1 * vY + b1] * v[IDX(i, a, j1, b1)];
        S[IDX(i, a, j, b)] = s;
    }
    memset(T, 0, nt * sizeof(double));
    for (int it = 0; it < n_iter; it++) {
        double dmax = 0.0;
        for (int i = 0; i < oX; i++)
        for (int a = 0; a < vX; a++)
        for (int j = 0; j < oY; j++)
        for (int b = 0; b < vY; b++) {
            double r = v[IDX(i, a, j, b)] + S[IDX(i, a, j, b)];
            for (int a1 = 0; a1 < vX; a1++)                 /* particle ladder */
            for (int b1 = 0; b1 < vY; b1++)
                r += G4(oX + a, oX + a1, oY + b, oY + b1) * T[IDX(i, a1, j, b1)];
            for (int i1 = 0; i1 < oX; i1++)                 /* hole ladder */
            for (int j1 = 0; j1 < oY; j1++)
                r += G4(i1, i, j1, j) * T[IDX(i1, a, j1, b)];
            for (int i1 = 0; i1 < oX; i1++)                 /* - v^{b i1}_{b1 i} T^{a b1}_{i1 j} */
            for (int b1 = 0; b1 < vY; b1++)
                r -= G4(i1, i, oY + b, oY + b1) * T[IDX(i1, a, j, b1)];
            for (int a1 = 0; a1 < vX; a1++)                 /* - v^{a j1}_{a1 j} T^{a1 b}_{i j1} */
            for (int j1 = 0; j1 < oY; j1++)
                r -= G4(oX + a, oX + a1, j1, j) * T[IDX(i, a1, j1, b)];
            if (GX)
                for (int i1 = 0; i1 < oX; i1++)
                for (int a1 = 0; a1 < vX; a1++)
                    r += GX[((size_t)i * vX + a) * mX + (size_t)i1 * vX + a1] * T[IDX(i1, a1, j, b)];
            if (GY)
                for (int j1 = 0; j1 < oY; j1++)
                for (int b1 = 0; b1 < vY; b1++)
                    r += GY[((size_t)j * vY + b) * mY + (size_t)j1 * vY + b1] * T[IDX(i, a, j1, b1)];
            const double t = r / (epsX[i] + epsY[j] - epsX[oX + a] - epsY[oY + b]);
            const double dt = fabs(t - T[IDX(i, a, j, b)]);
            if (dt > dmax) dmax = dt;
            Tn[IDX(i, a, j, b)] = t;
        }
        memcpy(T, Tn, nt * sizeof(double));
        if (delta) delta[it] = dmax;
    }
    {
        double ej = 0.0, ek = 0.0;
        for (int i = 0; i < oX; i++)
        for (int a = 0; a < vX; a++)
        for (int j = 0; j < oY; j++)
        for (int b = 0; b < vY; b++) {
            const double t = T[IDX(i, a, j, b)];
            ej += 4.0 * v[IDX(i, a, j, b)] * t;
            ek += -2.0 * W[(((size_t)i * vY + b) * oY + j) * vX + a] * t;
        }
        E[0] = ej;
        E[1] = ek;
    }
#undef G4
#undef IDX
    rc = 0;
out:
    free(g); free(v); free(W); free(S); free(Tn);
    return rc;
}

/* One dimer term {E_J, E_K} from the two AO blocks.  Returns 0 on success. */
int oracle_dimer(const double *A, const double *K,
                 const double *CX, const double *epsX,
                 const double *CY, const double *epsY,
                 int nX, int nY, int oX, int oY, double *E2)
{
    size_t nv = (size_t)oX * (nX - oX) * oY * (nY - oY);
    double *V = malloc(nv * sizeof(double));
    double *W = malloc(nv * sizeof(double));
    int rc = (!V || !W) ? -1 : 0;
    if (!rc) rc = oracle_transform_J(A, CX, CY, nX, nY, oX, oY, V);
    if (!rc) rc = oracle_transform_K(K, CX, CY, nX, nY, oX, oY, W);
    if (!rc) oracle_energy_from_mo(V, W, epsX, epsY, nX, nY, oX, oY, &E2[0], &E2[1]);
    free(V); free(W);
    return rc;
}

/* Eq. (dp2e) written out literally: every output element is the full
 * four-fold AO sum (cost n^4 per element, n^8 overall).  Used only to pin
 * the factorised path on tiny inputs. */
void oracle_bruteforce_J(const double *A, const double *CX, const double *CY,
                         int nX, int nY, int oX, int oY, double *V)
{
    int vX = nX - oX, vY = nY - oY;
    for (int i = 0; i < oX; i++)
    for (int a = 0; a < vX; a++)
    for (int j = 0; j < oY; j++)
    for (int b = 0; b < vY; b++) {
        double s = 0.0;
        for (int mu = 0; mu < nX; mu++)
        for (int nu = 0; nu < nX; nu++)
        for (int la = 0; la < nY; la++)
        for (int si = 0; si < nY; si++)
            s += CX[mu * nX + i] * CX[nu * nX + oX + a] * CY[la * nY + j] * CY[si * nY + oY + b]
               * A[(((size_t)mu * nX + nu) * nY + la) * nY + si];
        V[(((size_t)i * vX + a) * oY + j) * vY + b] = s;
    }
}

void oracle_bruteforce_K(const double *K, const double *CX, const double *CY,
                         int nX, int nY, int oX, int oY, double *W)
{
    int vX = nX - oX, vY = nY - oY;
    for (int i = 0; i < oX; i++)
    for (int b = 0; b < vY; b++)
    for (int j = 0; j < oY; j++)
    for (int a = 0; a < vX; a++) {
        double s = 0.0;
        for (int mu = 0; mu < nX; mu++)
        for (int la = 0; la < nY; la++)
        for (int si = 0; si < nY; si++)
        for (int nu = 0; nu < nX; nu++)
            s += CX[mu * nX + i] * CY[la * nY + oY + b] * CY[si * nY + j] * CX[nu * nX + oX + a]
               * K[(((size_t)mu * nY + la) * nY + si) * nX + nu];
        W[(((size_t)i * vY + b) * oY + j) * vX + a] = s;
    }
}

/* Factor route for integrals of the form (pq|rs) = s_XY sum_Q B^Q_pq B^Q_rs
 * (B[Q][p][q] over the n = nX+nY dimer functions, X first):
 *   (i a|j b) = s sum_Q (C_X^T B^Q_XX C_X)_{ia} (C_Y^T B^Q_YY C_Y)_{jb}
 *   (i b|j a) = s sum_Q (C_X^T B^Q_XY C_Y)_{ib} (C_Y^T B^Q_YX C_X)_{ja}
 * Exact in exact arithmetic, O(n^3 naux); a different arithmetic path from
 * the four-index route.  Fills V and W in the same layouts as above. */
int oracle_factor_route(const double *B, int naux, double s,
                        const double *CX, const double *CY,
                        int nX, int nY, int oX, int oY, double *V, double *W)
{
    int n = nX + nY, vX = nX - oX, vY = nY - oY;
    /* half-transformed factors: F[p][q] = sum_{mu,nu} C[mu][p] B[mu][nu] C[nu][q] */
    double *xx = malloc((size_t)oX * vX * sizeof(double));
    double *yy = malloc((size_t)oY * vY * sizeof(double));
    double *xy = malloc((size_t)oX * vY * sizeof(double));
    double *yx = malloc((size_t)oY * vX * sizeof(double));
    if (!xx || !yy || !xy || !yx) { free(xx); free(yy); free(xy); free(yx); return -1; }
    size_t nV = (size_t)oX * vX * oY * vY;
    memset(V, 0, nV * sizeof(double));
    memset(W, 0, nV * sizeof(double));
    for (int q = 0; q < naux; q++) {
        const double *Bq = B + (size_t)q * n * n;
        for (int i = 0; i < oX; i++) for (int a = 0; a < vX; a++) {
            double t = 0.0;
            for (int mu = 0; mu < nX; mu++) for (int nu = 0; nu < nX; nu++)
                t += CX[mu * nX + i] * Bq[mu * n + nu] * CX[nu * nX + oX + a];
            xx[i * vX + a] = t;
        }
        for (int j = 0; j < oY; j++) for (int b = 0; b < vY; b++) {
            double t = 0.0;
            for (int la = 0; la < nY; la++) for (int si = 0; si < nY; si++)
                t += CY[la * nY + j] * Bq[(nX + la) * n + nX + si] * CY[si * nY + oY + b];
            yy[j * vY + b] = t;
        }
        for (int i = 0; i < oX; i++) for (int b = 0; b < vY; b++) {
            double t = 0.0;
            for (int mu = 0; mu < nX; mu++) for (int la = 0; la < nY; la++)
                t += CX[mu * nX + i] * Bq[mu * n + nX + la] * CY[la * nY + oY + b];
            xy[i * vY + b] = t;
        }
        for (int j = 0; j < oY; j++) for (int a = 0; a < vX; a++) {
            double t = 0.0;
            for (int si = 0; si < nY; si++) for (int nu = 0; nu < nX; nu++)
                t += CY[si * nY + j] * Bq[(nX + si) * n + nu] * CX[nu * nX + oX + a];
            yx[j * vX + a] = t;
        }
        for (int i = 0; i < oX; i++) for (int a = 0; a < vX; a++)
        for (int j = 0; j < oY; j++) for (int b = 0; b < vY; b++) {
            V[(((size_t)i * vX + a) * oY + j) * vY + b] += s * xx[i * vX + a] * yy[j * vY + b];
            W[(((size_t)i * vY + b) * oY + j) * vX + a] += s * xy[i * vY + b] * yx[j * vX + a];
        }
    }
    free(xx); free(yy); free(xy); free(yx);
    return 0;
}

/* Neumaier's compensated summation of x[0..n-1] in index order. */
static double neumaier(const double *x, size_t n, size_t stride)
{
    double s = 0.0, c = 0.0;
    for (size_t k = 0; k < n; k++) {
        double v = x[k * stride];
        double t = s + v;
        if (fabs(s) >= fabs(v)) c += (s - t) + v;
        else                    c += (v - t) + s;
        s = t;
    }
    return s + c;
}

/* Lattice accumulation from per-dimer terms E2[d] = {E_J, E_K}:
 *   mon[2X] += E_J/2, mon[2Y] += E_J/2, mon[2X+1] += E_K/2, mon[2Y+1] += E_K/2
 * summed per monomer in dimer order (Neumaier), and the lattice totals. */
void oracle_accumulate(const double *E2, const int *X, const int *Y, int nd,
                       int nmon, double *mon /* 2*nmon */, double *total /* 2 */)
{
    double *sum = calloc((size_t)2 * nmon, sizeof(double));
    double *cmp = calloc((size_t)2 * nmon, sizeof(double));
    for (int d = 0; d < nd; d++) {
        for (int f = 0; f < 2; f++) {
            int who[2] = {X[d], Y[d]};
            for (int w = 0; w < 2; w++) {
                size_t k = (size_t)2 * who[w] + f;
                double v = 0.5 * E2[2 * d + f];
                double t = sum[k] + v;
                if (fabs(sum[k]) >= fabs(v)) cmp[k] += (sum[k] - t) + v;
                else                         cmp[k] += (v - t) + sum[k];
                sum[k] = t;
            }
        }
    }
    for (int k = 0; k < 2 * nmon; k++) mon[k] = sum[k] + cmp[k];
    total[0] = neumaier(E2, nd, 2);
    total[1] = neumaier(E2 + 1, nd, 2);
    free(sum); free(cmp);
}

/* Many independent dimers, OpenMP over dimers (used to time the oracle on
 * the host cores).  Pointers are per dimer.  Returns 0 if all succeeded. */
int oracle_dimers(int nd, const double *const *A, const double *const *K,
                  const double *const *CX, const double *const *epsX,
                  const double *const *CY, const double *const *epsY,
                  const int *nX, const int *nY, const int *oX, const int *oY,
                  double *E2)
{
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(|:bad)
    for (int d = 0; d < nd; d++)
        bad |= (oracle_dimer(A[d], K[d], CX[d], epsX[d], CY[d], epsY[d],
                             nX[d], nY[d], oX[d], oY[d], E2 + 2 * d) != 0);
    return bad;
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
