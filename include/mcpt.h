/*
 * mcpt.h -- C ABI of the GB300 (sm_103a) library for the first-order MCPT(2)
 * dimer term (Byrd, Jindal, Molt, Bartlett, Sanders, Lotrich, "Molecular
 * Cluster Perturbation Theory. I. Formalism").
 *
 * For every dimer X-Y of a lattice of monomers the library computes
 *
 *   (i a|j b) = sum_{mu nu in X, lam sig in Y} C_{mu i} C_{nu a} C_{lam j} C_{sig b} (mu nu|lam sig)
 *                                                             Eq. (dp2e), p=i r=a q=j s=b
 *   (i b|j a) = sum C_{mu i} C_{lam b} C_{sig j} C_{nu a} (mu lam|sig nu)   exchange-type form
 *   D^{ij}_{ab} = 1 / (e_i + e_j - e_a - e_b)                 energy tensor, Sec. II.C
 *   E_J(XY) = 4 sum (ia|jb)^2 D                                Eq. (ed2) with T = vD (first
 *                                                              Jacobi step of Eq. (td2))
 *   E_K(XY) = -2 sum (ia|jb)(ib|ja) D                          exchange completion (2J-K)
 *
 * and accumulates half of each dimer term onto each of its two monomers (the
 * dimer sum of the cluster Hamiltonian, Eq. (clusterH)), with a compensated
 * lattice total.  Orbitals are monomer-centred and not orthogonalised between
 * monomers (remark after Eq. (dp2e)), so C is block diagonal and each
 * monomer's C and eps are given once.
 *
 * Conventions
 *   - All matrices are row-major FP64.  C[mu][p] is nao x nao: row = AO,
 *     column = MO, the first nocc columns occupied, eps[p] the matching
 *     orbital energies.
 *   - A dimer's AO basis is X's functions first, then Y's (n = nX + nY).
 *     MCPT_AO_FULL: the full tensor G[n][n][n][n] (mu nu|lam sig).
 *     MCPT_AO_BLOCKS: the two blocks the term reads, back to back:
 *        A[nX][nX][nY][nY] = G[mu][nu][nX+lam][nX+sig]  (XX|YY)
 *        K[nX][nY][nY][nX] = G[mu][nX+lam][nX+sig][nu]  (XY|YX)
 *     MCPT_AO_PACKED: only the elements that the real-orbital pair symmetry
 *       (pq|rs) = (qp|rs) = (pq|sr) = (rs|pq) leaves unique, back to back
 *       (t(a, b) = a (a + 1) / 2 + b for a >= b):
 *        A_p[t(mu,nu)][t(lam,sig)]  mu >= nu, lam >= sig
 *                                   (nX(nX+1)/2 x nY(nY+1)/2, row-major)
 *        K_p[t(P,Q)]                P = mu nY + lam >= Q = nu nY + sig
 *                                   ((nX nY)(nX nY + 1)/2 elements), where
 *                                   K[mu][lam][sig][nu] = K_p[t(max(P,Q), min(P,Q))]
 *       2.6x fewer bytes than BLOCKS at 32 AO; the library expands them on
 *       the device into BLOCKS storage of its own.  The term computed is
 *       that of the symmetric blocks these elements define.
 *   - Monomer ids are 0..N-1 in add order; dimer ids 0..D-1 in add order.
 *
 * Errors: every call returns a status and never aborts or exits;
 * mcpt_last_error(h) returns the handle's last message.  A handle is not
 * thread-safe: one host thread at a time.
 */
#ifndef MCPT_H
#define MCPT_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mcpt_ctx *mcpt_handle;

typedef enum {
    MCPT_OK = 0,
    MCPT_EINVAL = 1,        /* bad argument: size, id, pointer, non-finite value */
    MCPT_ENOMEM = 2,        /* device or host allocation failed, or the memory cap was hit */
    MCPT_ECUDA = 3,         /* a CUDA runtime/driver call failed (message has the CUDA error) */
    MCPT_ESTATE = 4,        /* call out of order (e.g. energies before any run) */
    MCPT_ETIMEOUT = 5,      /* a bounded device-side wait gave up */
    MCPT_EUNSUPPORTED = 6   /* valid request this build/precision does not handle */
} mcpt_status;

/* Arithmetic of the four-index transformation.  Denominators, the energy
 * products and every energy sum are at FP64 accuracy in all forms (FP64 in the
 * FP64 form; in the mixed forms see mcpt_options.fp64_epilogue). */
typedef enum {
    MCPT_FP64 = 0,    /* FP64 everywhere (CUDA-core DFMA) */
    MCPT_TF32 = 1,    /* AO integrals rounded to TF32 (to nearest, ties away from zero), C_Y as two TF32
                         planes (hi + lo), tcgen05 MMA, FP32 accumulate */
    MCPT_BF16X3 = 2,  /* both operands as 32-bit fixed-point values relative to the largest power of
                         two of each integral row chunk (32 values) and each C_Y column (the integrals
                         through an FP32 value: their leading 24 significant bits), cut into four
                         BF16 digits; the tcgen05 MMAs add only integer digit products whose FP32 partial
                         sums stay below 2^24, so every tensor-core accumulation is exact (the Kronecker
                         kernel, selected only by MCPT_TC_KERNEL=kron, keeps a hi/lo BF16 split) */
    MCPT_FP32C = 3,   /* FP32 FMA with error-free TwoProduct/TwoSum compensation (Ogita-Rump-Oishi) */
    MCPT_BF16X2 = 4,  /* as MCPT_BF16X3 for C_Y (32-bit fixed point, four digits), but each integral
                         row chunk in 16-bit fixed point (two BF16 digits, rounded half up in magnitude,
                         read from the high word of each double): exact tensor-core sums with half the
                         digit work and half the MMAs; integrals carry 2^-17 of their chunk's largest
                         power of two as rounding error */
    MCPT_FP64E = 5    /* the FP64 form's accuracy from the tensor cores (Ozaki-style slicing, Ozaki
                         et al., Numer. Algorithms 59 (2012) 95): each integral row chunk and each C_Y
                         column in 48-bit fixed point, six unsigned byte digits carrying the element's
                         sign, every digit product summed exactly in FP32 by tcgen05 FP16 MMAs (21
                         products in six levels); the levels, the p0 quarter transformation and the
                         first-half result on FP32 pairs (48-bit).  Monomers of up to 32 AO: the
                         result written as FP32 pairs, and the second half (virtual quarter
                         transformations, denominators, energy terms) on FP32 pairs with FP64 sums;
                         larger ones: the result written as FP64 and the second half as in
                         MCPT_FP64.  n_Y of up to 64 AO and 5 occupied orbitals per monomer
                         (MCPT_EUNSUPPORTED beyond) */
} mcpt_precision;

typedef enum {
    MCPT_AO_FULL = 0,
    MCPT_AO_BLOCKS = 1,
    MCPT_AO_PACKED = 2
} mcpt_ao_layout;

typedef struct {
    int device;               /* CUDA device ordinal */
    void *stream;             /* cudaStream_t to run on, or NULL for a library-owned stream */
    mcpt_precision precision; /* see above */
    int validate;             /* 1: reject non-finite C / eps / integrals (adds a pass over inputs) */
    size_t wave_bytes;        /* cap on per-run device scratch; dimers run in waves under it (0 = 1 GiB) */
    const char *tune_cache;   /* path of the autotuner's cache, or NULL: with a path, each tensor-core
                                 wave's launch choices (kernel variant, staging depth, grid) are timed on
                                 the first plan of its shape signature and kept in that text file */
    int timing;               /* 1: record CUDA events per phase of mcpt_run (see mcpt_run_stats) */
    size_t mem_cap_bytes;     /* cap on library-owned device memory (0 = no cap) */
    int graphs;               /* 1: with timing = 0, replay each run as a CUDA graph captured on the
                                 first run of a plan (the plan = dimer set, range and precision);
                                 runs on a stream that is itself being captured are launched directly */
    int coupling;             /* 1: mcpt_run also forms each monomer's dimer -> monomer doubles
                                 coupling R_X of Eq. (tm2) at first order (see mcpt_coupling); the
                                 dimers' (ia|jb) and T = vD stay on the device (2 o_X v_X o_Y v_Y
                                 elements each) */
    unsigned long long wait_limit_ns; /* limit of each device-side wait of the tensor-core kernels
                                 (0 = 4 s); when one runs out the kernel gives up, drains its own
                                 copies and MMAs, frees its tensor memory and returns, and the next
                                 mcpt_energies reports MCPT_ETIMEOUT */
    int withhold_load;        /* test aid, 0 = off: N > 0 makes the first CTA of each tensor-core
                                 launch stop issuing integral loads after N - 1 of them, so that its
                                 consumers wait for a load that never comes and give up at
                                 wait_limit_ns (failure detection without a device fault) */
    int fp64_epilogue;        /* mixed forms only.  0 (default): each term's last denominator
                                 subtraction, D = 1/x, the products with D and the sums over b run on
                                 FP32 pairs (48-bit double-length arithmetic, D to ~2^-45 relative),
                                 added to the FP64 sums once per occupied pair; e_i + e_j - e_a is
                                 FP64.  1: the same on the FP64 pipe, five FP64 operations per term
                                 (same accuracy class, slower on GB300) */
} mcpt_options;

/* Defaults: device 0, own stream, MCPT_FP64, validate 1, 1 GiB waves, no cache, no timing,
 * graphs 1, no memory cap. */
void mcpt_default_options(mcpt_options *opt);

/* Create a handle.  opt may be NULL (defaults).  *out is NULL on failure.
 * Errors: EINVAL (out NULL, bad precision), ECUDA (device/stream). */
mcpt_status mcpt_create(mcpt_handle *out, const mcpt_options *opt);

/* Register monomer `*id_out` (ids are assigned 0, 1, ... in call order).
 * C: host pointer to nao*nao FP64, row-major C[mu][p] (MO coefficients, the
 *    monomer Hartree-Fock solution of Sec. III's program flow, step 1);
 * eps: host pointer to nao FP64 orbital energies (occupied first).
 * Both are copied before the call returns.
 * Errors: EINVAL if nao < 2 or nao > 128, nocc not in [1, nao-1], a pointer
 * is NULL, or (validate) a value is not finite; ESTATE after mcpt_destroy. */
mcpt_status mcpt_add_monomer(mcpt_handle h, const double *C, const double *eps,
                             int nao, int nocc, int *id_out);

/* Register dimer X-Y with its AO integrals (Eq. (dp2e) input).
 * ao_eri: FP64 in `layout` for the (X, Y) order given.  If X > Y the library
 *   stores the dimer as (Y, X) with the integrals relabelled (Y's functions
 *   first); the term is symmetric in X and Y.
 * on_device = 0: host pointer, copied (blocks only) before the call returns.
 * on_device = 1: device pointer on the handle's device, BORROWED: it must
 *   stay valid and unmodified until the last mcpt_run that uses it has
 *   completed (mcpt_energies returns).  Requires X < Y.
 * MCPT_AO_PACKED (requires X < Y): host or device data is expanded into
 *   library storage by work on the handle's stream before the call returns,
 *   after which the caller's buffer is no longer read.
 * Errors: EINVAL (unknown or equal ids, duplicate pair, NULL, bad layout,
 *   non-finite with validate=1, X > Y with on_device=1), ENOMEM, ECUDA. */
mcpt_status mcpt_add_dimer(mcpt_handle h, int X, int Y, const double *ao_eri,
                           mcpt_ao_layout layout, int on_device, int *id_out);

/* Flags of mcpt_update_dimer. */
enum { MCPT_UPDATE_ASYNC = 1 };

/* Replace the AO integrals of registered dimer `id` for later runs (same
 * monomers, same sizes), e.g. the next geometry of a sequence of lattices.
 * ao_eri: FP64 in `layout` for the dimer's stored order (X < Y as registered;
 *   no relabelling).
 * on_device = 0: host pointer.  The integrals go into the dimer's library
 *   storage (allocated on its first host update if it had been given on the
 *   device), copied before the call returns; with MCPT_UPDATE_ASYNC and the
 *   BLOCKS or PACKED layout the copy (and the expansion of packed data) is
 *   only enqueued on the handle's stream, and the host buffer must stay
 *   valid and unmodified until the next mcpt_run has completed
 *   (mcpt_energies returns) -- with pinned host memory the copies of many
 *   dimers then run back to back at the link's bandwidth.
 * on_device = 1: device pointer, BORROWED as in mcpt_add_dimer (PACKED:
 *   expanded into the dimer's library storage, with MCPT_UPDATE_ASYNC only
 *   enqueued, so the buffer must then stay unmodified until that work ends).
 * The dimer counts as not computed until the next run that covers it.  The
 * run plan (and its CUDA graph) is kept when the integrals' device addresses
 * do not change (host updates into existing storage).
 * Errors: EINVAL (unknown id, NULL, bad layout, unknown flags, non-finite with
 *   validate=1, on_device=1 with host memory), ENOMEM, ECUDA. */
mcpt_status mcpt_update_dimer(mcpt_handle h, int id, const double *ao_eri, mcpt_ao_layout layout,
                              int on_device, int flags);

/* mcpt_update_dimer for dimers first .. first+count-1 in one call, host
 * memory only: dimer first+k's integrals at ao_eri + offsets[k] (elements),
 * in `layout` (MCPT_AO_BLOCKS or MCPT_AO_PACKED) for its stored order, with
 * the same flags and ownership rules.  For MCPT_AO_PACKED the dimers whose
 * data lie back to back in the buffer are copied together, in chunks of up
 * to 256 MB and 64 dimers through two device staging buffers (one copy
 * stream each), and each chunk is expanded by one launch: with pinned memory and MCPT_UPDATE_ASYNC the
 * copies run at the link's bandwidth instead of being paced by one call per
 * dimer.  A dimer whose integrals were borrowed device memory gets storage
 * of its own (its run plan is rebuilt).  Not a step of the paper's method: the
 * ingest of a sequence of lattices.
 * Errors: EINVAL (range, NULL, layout, flags, non-finite with validate=1),
 *   ENOMEM, ECUDA. */
mcpt_status mcpt_update_dimers(mcpt_handle h, int first, int count, const double *ao_eri, const size_t *offsets,
                               mcpt_ao_layout layout, int flags);

/* Switch the transformation arithmetic for later runs (no re-upload). */
mcpt_status mcpt_set_precision(mcpt_handle h, mcpt_precision p);

/* Compute every registered dimer term and the per-monomer accumulation
 * (Sec. III program flow, steps 2 and 6 at first order) on the handle's
 * stream.  Asynchronous: returns once the work is enqueued.  Re-running
 * recomputes everything.
 * Errors: ESTATE (no dimers), EUNSUPPORTED (precision cannot handle a dimer's
 * sizes: tensor-core forms need even nX, nY <= 128, the FP64 form nX, nY <= 96;
 * tensor-core dimers with more than 20 occupied orbitals on X or 16 on Y run
 * as near-equal blocks of at most 20 x 16 occupied pairs, each reading the
 * integrals; MCPT_FP64E needs nY <= 64 and at most 5 occupied orbitals per
 * monomer),
 * ENOMEM, ECUDA, ETIMEOUT. */
mcpt_status mcpt_run(mcpt_handle h);

/* Compute only dimers [first, first+count) (resume / partial runs).  Their
 * terms replace earlier ones; the per-monomer sums cover all dimers and are
 * valid once every dimer has been computed at least once. */
mcpt_status mcpt_run_range(mcpt_handle h, int first, int count);

/* Wait for the handle's stream and copy results to host buffers (each may be
 * NULL): per_monomer_J, per_monomer_K: N each; per_dimer: 2*D as {E_J, E_K};
 * total: 2 as {sum E_J, sum E_K} (Neumaier-compensated, fixed order).
 * Errors: ESTATE if a dimer has not been computed since it was added;
 * ETIMEOUT if a device-side wait gave up during the run; ECUDA. */
mcpt_status mcpt_energies(mcpt_handle h, double *per_monomer_J, double *per_monomer_K,
                          double *per_dimer, double *total);

/* Dimer -> monomer doubles coupling of Eq. (tm2) (the sum over the
 * neighbours' occupied k and virtual c), evaluated at the first-order dimer
 * amplitudes T^{ab}_{ij} = (ia|jb) D^{ij}_{ab} of the last mcpt_run:
 *   R_X[(i,a)][(i1,a1)] = sum_{Y, k, c} (i1 a1|k c) T^{ac}_{ik} + (i a|k c) T^{a1 c}_{i1 k}
 * over every registered dimer containing X (i, i1 occupied and a, a1 virtual
 * orbitals of X).  R: caller's buffer of (o_X v_X)^2 doubles, row-major,
 * index i * v_X + a; symmetric.  Waits for the handle's stream.
 * Arithmetic: the form's (FP32 for the mixed forms, FP64 for the FP64 form),
 * summed over dimers in ascending order.
 * Errors: EINVAL (unknown X, NULL), ESTATE (options.coupling = 0, or no
 *   mcpt_run of every dimer since the integrals last changed), ECUDA. */
mcpt_status mcpt_coupling(mcpt_handle h, int X, double *R);

/* Environment term of the monomer singles equation, Eq. (tm1) (the sum over
 * the neighbours' occupied k and virtual c), from the integrals of the last
 * mcpt_run of every dimer in a context created with options.coupling = 1:
 *   s_X[(i,a)] = sum_{Y, k, c} (i a|k c) t^c_k(Y)
 * over every registered dimer containing X.  t: host array of every
 * monomer's singles amplitudes t^a_i, monomer by monomer in id order, each
 * o_X x v_X row-major (index i * v_X + a), sum_X o_X v_X doubles in all; it
 * is copied before the call returns.  s: host output of the same layout.
 * Waits for the handle's stream.  Arithmetic: the form's storage type per
 * dimer (FP32 for the mixed forms, in partial sums of 32 terms added in
 * FP64), FP64 over dimers in ascending order; deterministic.
 * Errors: EINVAL (NULL, or a non-finite t with validate = 1), ESTATE
 *   (options.coupling = 0, or no mcpt_run of every dimer since the
 *   integrals last changed), ETIMEOUT, ECUDA. */
mcpt_status mcpt_singles(mcpt_handle h, const double *t, double *s);

/* Monomer X's own quantities in the dimer doubles equation, Eq. (td2),
 * each (o_X v_X) x (o_X v_X) row-major with index i * v_X + a (host
 * pointers, copied; NULL = zero, the default):
 *   G[(i,a)][(i1,a1)] = 2 v^{i1 a}_{a1 i} - v^{a i1}_{a1 i}   (ring matrix)
 *   U[(i,a)][(i1,a1)] = 2 T^{a a1}_{i i1} - T^{a a1}_{i1 i}   (monomer doubles)
 * Errors: EINVAL (unknown X, non-finite with validate = 1). */
mcpt_status mcpt_set_monomer_doubles(mcpt_handle h, int X, const double *G, const double *U);

/* The dimer doubles amplitudes of Eq. (td2) for every registered dimer by
 * n_iter Jacobi steps from zero,
 *   T <- D (v + S + L(T)),  D = 1 / (e_i + e_j - e_a - e_b),
 * with v = (ia|jb), S = sum U_X v + v U_Y^T (the monomer-amplitude terms)
 * and L(T) the particle ladder (a a1|b b1), the hole ladder (i1 i|j1 j),
 * -(i1 i|b b1) and -(a a1|j1 j) contractions and the two ring-matrix
 * terms, all with their printed signs; the energy-tensor term's sign is
 * read as for the first-order amplitude, so one step gives T = v D and the
 * first-order terms of mcpt_run.  The integrals come from the dimers'
 * registered AO blocks (the full MO transformation of the Coulomb block,
 * the (ib|ja) part of the exchange block), formed on the device.
 * per_dimer: 2 D doubles {E_J, E_K} at the final amplitudes (E_J = 4 sum v T,
 *   Eq. (ed2); E_K = -2 sum (ib|ja) T), or NULL.
 * delta: n_iter doubles, the largest |T_new - T_old| over all dimers at each
 *   step, or NULL.
 * Arithmetic: FP64 in the FP64 form, FP32 otherwise (energy sums FP64).
 * Dimers run in batches under max(options.wave_bytes, 4 GiB) of scratch.
 * Synchronous.  Errors: EINVAL (n_iter outside [1, 10000]), ESTATE (no
 * dimers), ENOMEM, ECUDA. */
mcpt_status mcpt_td2(mcpt_handle h, int n_iter, double *per_dimer, double *delta);

/* Density-fitted route (not the paper's four-index transformation): dimer
 * terms from three-index factors, with
 *   (ia|jb) = s sum_Q (C_X^T B^Q_XX C_X)_{ia} (C_Y^T B^Q_YY C_Y)_{jb}
 *   (ib|ja) = s sum_Q (C_X^T B^Q_XY C_Y)_{ib} (C_Y^T B^Q_YX C_X)_{ja}
 * and the same D, E_J, E_K and per-monomer accumulation as mcpt_run.  Exact
 * whenever the integrals are (mu nu|lam sig) = s sum_Q B^Q_{mu nu} B^Q_{lam sig}
 * on the dimer blocks.
 * mcpt_add_dimer_df registers dimer X-Y (X < Y) in a list of its own (ids
 * 0, 1, ... in call order): B is naux x n x n FP64 row-major over the dimer's
 * n = nX + nY AO functions, X's first; on_device = 0: host, copied before the
 * call returns; 1: device memory of the handle's device, BORROWED until the
 * last mcpt_run_df that uses it has completed.  s scales the dimer's
 * integrals (1 for plain factors).
 * Errors: EINVAL (unknown ids, X >= Y, duplicate, NULL, naux < 1, non-finite
 *   s, non-finite factors with validate = 1), ENOMEM, ECUDA. */
mcpt_status mcpt_add_dimer_df(mcpt_handle h, int X, int Y, const double *B, int naux, double s,
                              int on_device, int *id_out);
/* Compute every density-fitted dimer's terms and their per-monomer sums on
 * the handle's stream; FP64 in the FP64 form, FP32 otherwise (the
 * denominators and energy sums FP64).  Waits for the work.
 * Errors: ESTATE (no such dimers), EUNSUPPORTED (a dimer whose factor slice
 *   B^Q, C_X, C_Y and occupied rows, n^2 + n_X^2 + n_Y^2 + (o_X + o_Y) n
 *   values, exceed 200 KB of shared memory: above about 56 + 56 AO in FP64,
 *   80 + 80 in FP32), ENOMEM, ECUDA. */
mcpt_status mcpt_run_df(mcpt_handle h);
/* Results of the last mcpt_run_df, as mcpt_energies (per-monomer halves of
 * the density-fitted dimers, per-dimer {E_J, E_K} in their id order, the
 * Neumaier totals); each pointer may be NULL.  Errors: ESTATE (no run since
 * the last dimer was added), ECUDA. */
mcpt_status mcpt_df_energies(mcpt_handle h, double *per_monomer_J, double *per_monomer_K,
                             double *per_dimer, double *total);

/* Per-phase timing and launch counts of every run since the previous call
 * (timing requires options.timing = 1; CUDA events are recorded on the
 * handle's stream around each phase, and this call waits for the stream).
 * ms[0] = first half (the AO-reading transform kernel), ms[1] = finish
 * (second half + denominators + energies), ms[2] = per-monomer reduction
 * (and the coupling, when enabled),
 * ms[3] = whole run: each summed over the `runs` collected runs;
 * launches = kernels those runs launched; waves = waves per run;
 * alg_bytes = algorithmic AO bytes read per run (2 nX^2 nY^2 x 8 B per dimer);
 * alg_flops = algorithmic flops per run of both halves (occupied-first
 * factorised count, both forms); alg_flops_half = those of the first half. */
typedef struct {
    float ms[4];
    int runs;
    int launches;
    int waves;
    double alg_bytes;
    double alg_flops;
    double alg_flops_half;
} mcpt_run_stats;
mcpt_status mcpt_collect_stats(mcpt_handle h, mcpt_run_stats *out);

/* Counts registered so far. */
int mcpt_num_monomers(mcpt_handle h);
int mcpt_num_dimers(mcpt_handle h);

/* Last error message of the handle ("" if none); with h == NULL, the last
 * error of a failed mcpt_create on this thread. */
const char *mcpt_last_error(mcpt_handle h);

/* One dimer's FP64 {E_J, E_K} without allocating any memory.  The paper has
 * no counterpart: this exists for callers that must not allocate device
 * memory -- code living inside another framework's memory pool or budget,
 * hooks that are handed their buffers, paths that may not call cudaMalloc or
 * cudaFree (which synchronise the device and can fail midway).  All
 * arguments are DEVICE pointers owned by the caller, on the current device:
 * A (nX,nX,nY,nY) then K (nX,nY,nY,nX) blocks as in MCPT_AO_BLOCKS (separate
 * pointers), C_X (nX x nX), eps_X (nX), C_Y, eps_Y, and E2 (2 doubles,
 * written {E_J, E_K}).  Work is enqueued on `stream` (cudaStream_t, NULL =
 * legacy default stream); read E2 after synchronising it.
 * Scratch: a fixed 8 MiB device array inside the library (every GPU that
 * loads the library holds it until the process exits), so 2*nX*nY*nocc_X*
 * nocc_Y must not exceed 1048576 doubles; nX, nY <= 96.  The first call on a
 * device looks the array's device address up (cudaGetSymbolAddress) and sets
 * a kernel attribute; make that first call before any stream capture.  All
 * calls share the array: calls whose work overlaps on the GPU (different
 * streams, or different host threads) race and give wrong results; calls on
 * one stream are ordered.  Nothing in the array needs to start at zero --
 * every call overwrites all of the scratch it reads.
 * Errors (message via mcpt_last_error(NULL)): EINVAL for NULL pointers, sizes
 * outside the limits above; ECUDA if set-up or a launch fails.  A successful
 * call clears that message. */
mcpt_status mcpt_dimer_fp64_noalloc(const double *A, const double *K,
                                    const double *C_X, const double *eps_X, int nX, int nocc_X,
                                    const double *C_Y, const double *eps_Y, int nY, int nocc_Y,
                                    double *E2, void *stream);

/* Measured FP64 FMA rate of `device` (a microbenchmark: independent FMA
 * chains on every SM, timed with CUDA events after a warm-up launch).  Not a
 * step of the path and without counterpart in the paper: the FP64 form is
 * bound by this pipe, and its roofline needs the rate.  *tflops receives
 * TFLOP/s (2 flops per FMA), *ms_per_launch (may be NULL) the time of one
 * of the five timed launches (about 33 ms on a GB300).  Errors (mcpt_last_error(NULL)):
 * EINVAL for tflops NULL, ECUDA. */
mcpt_status mcpt_fp64_fma_rate(int device, double *tflops, double *ms_per_launch);

/* Release the handle and every library-owned device buffer.  Borrowed
 * pointers are not touched.  NULL is a no-op. */
void mcpt_destroy(mcpt_handle h);

#ifdef __cplusplus
}
#endif

#endif /* MCPT_H */
