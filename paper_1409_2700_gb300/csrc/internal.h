// internal.h -- device-side descriptors and kernel launchers of libmcpt.
//
// Geometry of one dimer "form" (f = 0: the Coulomb-type block A, giving
// (i a|j b); f = 1: the exchange-type block K, giving (i b|j a)).  Both are
// a 4-index block E[p0][p1][p2][p3] whose axes 0 and 2 carry occupied
// outputs (i from X, j from Y):
//   f = 0: E = A[mu][nu][lam][sig]   p0=mu->i  p1=nu->a   p2=lam->j  p3=sig->b
//   f = 1: E = K[mu][lam][sig][nu]   p0=mu->i  p1=lam->b  p2=sig->j  p3=nu->a
// (Eq. dp2e with (p r|q s) = (i a|j b), resp. its exchange-type form.)
//
// The path has two halves:
//   first half  ("transform", reads every AO byte once):
//       H_f[(i,j)][(p1,p3)] = sum_{p0,p2} C_X[p0][i] C_Y[p2][j] E[p0][p1][p2][p3]
//       (stored pair-major: one contiguous nX*nY slice per occupied pair)
//   second half ("finish"):  (i a|j b) = sum_{nu,sig} C_X[nu][a] C_Y[sig][b] H_0[(nu,sig)][(i,j)]
//                            (i b|j a) = sum_{lam,nu} C_Y[lam][b] C_X[nu][a] H_1[(lam,nu)][(i,j)]
//       then D = 1/(e_i+e_j-e_a-e_b) and the two energy sums in FP64.
#pragma once
#include <cuda_runtime.h>

#include <vector>
#include <stdint.h>

namespace mcpt {

constexpr int kMaxAO = 256;          // any form (FP64 / FP32C)
constexpr int kMaxAOTensor = 128;    // tensor-core forms
constexpr int kMaxOccTensor = 16;    // occupied orbitals per monomer in one tensor-core work item
constexpr int kMaxOccTensorX = 20;   // ... of the first monomer (X), with kMaxOccTensor of Y (the wide
                                     //   TMEM-accumulator kernel)

struct DimerDesc {
    const double* E[2];   // block base of form 0 (A) and form 1 (K)
    long long st[2][3];   // element strides of axes p0, p1, p2 (axis p3 is contiguous)
    int nX, nY, oX, oY;   // AO counts; occupied orbitals of this descriptor's block
    int cX, cY;           // pool offsets of the block's first occupied column of C_X, C_Y
    int eX, eY;           // pool offsets of the block's first occupied eps_X, eps_Y
    int cXv, cYv;         // pool offsets of the first virtual column of C_X, C_Y
    int eXv, eYv;         // pool offsets of the first virtual eps_X, eps_Y
    int vX, vY;           // virtual orbital counts
    int iX0, jY0;         // first occupied orbital of this block within the monomer
    int oXt, oYt;         // the monomers' occupied counts
    long long vt_off;     // coupling storage of the dimer (-1: none): (ia|jb) then T = vD, each
                          //   [(j,b)][(i,a)] of (oYt vY) x (oXt vX) elements
    // A dimer whose occupations exceed what one tensor-core work item holds
    // runs as several descriptors, one per block of occupied orbitals (i, j);
    // each covers all virtual orbitals, and their terms are added per dimer.
    int X, Y;             // monomer ids
    long long h_off;      // first-half result H: element (form f, pair i*oY+j, row) at
                          //   h_off + (f*oX*oY + i*oY + j) * nX*nY + row   (pair-major)
    int npad;             // oX*oY padded to 16: N of the Kronecker tensor-core GEMM
    int slot;             // index of this descriptor's {E_J, E_K} in the per-dimer output
                          // (blocks of a split dimer: entries past the dimers, folded)
};

// Per-monomer accumulation lists: dimers touching monomer m are
// list[start[m] .. start[m+1]) (ascending dimer slot).
struct MonomerLists {
    const int* start;
    const int* list;
    int n_mon;
};

// ---- launchers (each returns the launch error; work is asynchronous) ----

// FP64 first half on CUDA cores, one thread per output row.
cudaError_t launch_half_fp64(const DimerDesc* d_desc, int nd, int max_rows, int max_occ,
                             const double* Cpool, double* H, cudaStream_t s);

// FP32 first half with compensated (TwoProduct/TwoSum) accumulation.
cudaError_t launch_half_fp32c(const DimerDesc* d_desc, int nd, int max_rows, int max_occ,
                              const float* Cf, float* H, cudaStream_t s);

// Second half of monomers above 32 AO: one CTA per task = a range of one
// dimer's occupied pairs; the tasks of a dimer are consecutive.
struct FinTask {
    int dimer;            // descriptor index within the wave
    int pr0, pr1;         // pairs [pr0, pr1) (pair = i*oY + j)
    int first;            // index of the dimer's first task
    int ntasks;           // tasks of the dimer
};
// Split each dimer's pairs into tasks of about `pairs_per_task`.
void finish_tasks(const DimerDesc* h_desc, int nd, int pairs_per_task, std::vector<FinTask>* out);

// Second half + denominators + energies.  H is double (FP64 form) or float.
// Waves whose monomers all have <= 32 AO run one CTA of w32_warps (4 or 5)
// warps per dimer; larger ones run the tasks (`tasks`, device array of
// `ntasks`) and sum each dimer's task partials (`part`, 2 doubles per task)
// in task order.
// With VT non-null, descriptors with vt_off >= 0 also store their (ia|jb)
// and T = vD for the coupling.  FP32 (mixed forms): the energy epilogue on
// FP32 pairs, or with fp64_epilogue on the FP64 pipe term by term.
cudaError_t launch_finish_fp64(const DimerDesc* d_desc, int nd, int max_ao,
                               const double* Cpool, const double* Epool, const double* H,
                               double* E2, const FinTask* tasks, int ntasks, double* part, double* VT,
                               int w32_warps, cudaStream_t s);
cudaError_t launch_finish_fp32(const DimerDesc* d_desc, int nd, int max_ao,
                               const float* Cf, const double* Epool, const float* H,
                               double* E2, const FinTask* tasks, int ntasks, double* part, float* VT,
                               bool fp64_epilogue, int w32_warps, cudaStream_t s);

// FP64E second half (monomers of at most 32 AO): H as FP32 pairs (written so
// by the FP64E first half), every step on FP32 pairs, FP64 sums; VT (may be
// null) gets FP64 (ia|jb) and T = vD as launch_finish_fp64 stores them.
cudaError_t launch_finish_ff(const DimerDesc* d_desc, int nd, int max_ao, const double* Cpool, const double* Epool,
                             const void* H, double* E2, double* VT, int w32_warps, cudaStream_t s);

// The 32-AO second half's forms, and its warps per CTA for the host
// descriptors h[0, nd) of a wave: 4 or 5, whichever takes fewer rounds of
// one occupied pair per warp over the CTAs an SM holds at once.
enum FinForm { FIN_F64 = 0, FIN_F32_PAIRS = 1, FIN_F32_F64EPI = 2, FIN_FF = 3 };
int finish_w32_warps(const DimerDesc* h, int nd, int form);

// Dimer -> monomer doubles coupling of Eq. (tm2) at first order.
struct CoupDim {
    int X, Y;             // monomer ids
    int mX, mY;           // oX vX and oY vY
    long long vt_off;     // (ia|jb) at vt_off, T at vt_off + mX*mY, both [(j,b)][(i,a)]
};
struct CoupTile {
    int mon;              // monomer
    int p0, q0;           // output tile origin in R_mon
};
// R_mon = sum over the monomer's dimers (ascending) of T V^T + V T^T (X side)
// or the transposed contractions (Y side); one CTA per output tile with
// q0 >= p0, writing both mirror halves.  tiles: ntile[0] tiles of edge 64,
// then ntile[1] of edge 48, then ntile[2] of edge 32 (host array of three
// counts).  dims: every dimer; lists: the per-monomer dimer lists; R: per
// monomer at r_off[mon], (o v)^2 doubles row-major.  T = float or double.
cudaError_t launch_coupling_fp32(const CoupTile* tiles, const int* ntile, const CoupDim* dims, MonomerLists lists,
                                 const int* mdim, const long long* r_off, const float* VT, double* R,
                                 cudaStream_t s);
cudaError_t launch_coupling_fp64(const CoupTile* tiles, const int* ntile, const CoupDim* dims, MonomerLists lists,
                                 const int* mdim, const long long* r_off, const double* VT, double* R,
                                 cudaStream_t s);

// Singles environment term of Eq. (tm1) from the same stored (ia|kc):
// s_mon[(i,a)] = sum over the monomer's dimers (ascending) of
// sum_{(k,c)} (ia|kc) t_other[(k,c)].  Two launches: each (dimer, side)
// writes its contribution to part (dimer d's X part at part_off[d], its Y
// part right after, m_X + m_Y doubles in all), then one thread per output
// (tiles of 256 per monomer) adds the monomer's parts in ascending order.
// t and s: FP64, monomer blocks of o v (at most 64 x 64 at 128 AO) at
// s_off[mon].
struct SingTile {
    int mon;              // monomer
    int p0;               // first output (i,a) index of the tile
};
cudaError_t launch_singles_fp32(const SingTile* tiles, int ntiles, const CoupDim* dims, int ndims, MonomerLists lists,
                                const int* mdim, const long long* s_off, const long long* part_off, const float* VT,
                                const double* t, double* part, double* s, cudaStream_t st);
cudaError_t launch_singles_fp64(const SingTile* tiles, int ntiles, const CoupDim* dims, int ndims, MonomerLists lists,
                                const int* mdim, const long long* s_off, const long long* part_off, const double* VT,
                                const double* t, double* part, double* s, cudaStream_t st);

// ---- dimer doubles iteration of Eq. (td2) ----
// One quarter step of a four-index transformation, per dimer of a batch:
//   Out[n][m] = sum_k C[k][c0 + n] In(m, k),  n < N, m < M, k < K,
// In(m, k) = in[(m / (d1 d2)) st0 + ((m / d2) % d1) st1 + (m % d2) st2 + k]
// (the contracted index is the innermost, stride 1); Out is [N][M]
// contiguous, so the new index comes first and four steps return the
// original index order.  ldc: row length of C.
template <typename TI, typename TO>
struct QStep {
    const TI* in;
    long long st0, st1, st2;
    int d1, d2;
    const double* C;
    int ldc, c0;
    int M, N, K;
    TO* out;
};
// A pair-indexed contraction, per dimer of a batch:
//   Out(r, c) += alpha sum_k W(r, k) Z(k, c),  r < R, c < C, k < K,
// each operand addressed by separable two-index axes: an index x of an axis
// {n1, s0, s1} sits at (x / n1) s0 + (x % n1) s1.
struct PAxis {
    int n1;
    long long s0, s1;
};
template <typename T>
struct PGemm {
    const T* W;
    PAxis wr, wk;
    const T* Z;
    PAxis zk, zc;
    T* out;
    PAxis orow, ocol;
    int R, C, K;
    T alpha;
};
// Per-dimer state of the iteration (element offsets into the batch arena of
// type T; [i][a][j][b] order for V, R0, R and the amplitudes Tc; [i][b][j][a] for W).
struct Td2Dim {
    int nX, nY, oX, oY;
    int eX, eY;                       // offsets of the monomers' orbital energies
    long long V, W, R0, R, Tc;
};
template <typename TI, typename TO>
cudaError_t launch_qstep(const QStep<TI, TO>* steps, int nd, int max_m, int max_n, cudaStream_t s);
template <typename T>
cudaError_t launch_pgemm(const PGemm<T>* tabs, int nd, int max_r, int max_c, cudaStream_t s);
// The same contraction with W given k-major as a dense matrix Wt[k][r] at
// W + k * ld + r, ld = wr.s1 a multiple of 4 and the padding zero (wk unused).
template <typename T>
cudaError_t launch_pgemm_dw(const PGemm<T>* tabs, int nd, int max_r, int max_c, cudaStream_t s);
// Wt[(a1,b1)][(a,b)] = g[oX+a][oX+a1][oY+b][oY+b1] per dimer at wd_off[d],
// rows of ld = round4(vX vY) with zero padding.
template <typename T>
cudaError_t launch_pack_ladder(const Td2Dim* dims, const long long* g_off, const long long* wd_off, int nd,
                               int max_rows, T* arena, cudaStream_t s);
// V, R0 <- (ia|jb) gathered from the full MO block g (per dimer at g_off[d]:
// [p][q][r][s] over all MOs); Tc <- 0.
template <typename T>
cudaError_t launch_td2_init(const Td2Dim* dims, const long long* g_off, int nd, int max_m, T* arena, cudaStream_t s);
// Tc <- R / (e_i + e_j - e_a - e_b); delta_bits <- max |Tc_new - Tc_old|
// (the bits of a non-negative T, compared as unsigned integers).
template <typename T>
cudaError_t launch_td2_update(const Td2Dim* dims, int nd, int max_m, const double* eps, T* arena,
                              void* delta_bits, cudaStream_t s);
// E[2d] = 4 sum V Tc, E[2d+1] = -2 sum W Tc, FP64, fixed order (one CTA per dimer).
template <typename T>
cudaError_t launch_td2_energy(const Td2Dim* dims, int nd, const T* arena, double* E, cudaStream_t s);

// ---- density-fitted route ----
// One dimer given by its three-index factors B[naux][n][n] (n = nX + nY, X's
// functions first, FP64 device memory): (ia|jb) = s sum_Q (C_X^T B^Q_XX C_X)_{ia}
// (C_Y^T B^Q_YY C_Y)_{jb}, (ib|ja) = s sum_Q (C_X^T B^Q_XY C_Y)_{ib} (C_Y^T B^Q_YX C_X)_{ja}.
struct DfDim {
    const double* B;
    int naux, nX, nY, oX, oY;
    int cX, cY, eX, eY;       // offsets of C and eps in the monomer pools
    double s;
    long long h_off;          // half-transformed blocks: naux x (oX vX + oY vY + oX vY + oY vX) elements
    int p_off;                // first pair partial (pairs of doubles)
    int id;                   // row of E2
};
// Terms of nd dimers into E2 (2 doubles each): FP64 arithmetic if fp64,
// else FP32 (energy epilogue FP64).  max_on = max over dimers of the
// half-transformation's shared elements n^2 + nX^2 + nY^2 + (oX + oY) n;
// max_v = max(vX, vY); half: scratch of the half-transformed blocks;
// part: 2 doubles per occupied pair.
cudaError_t launch_df(bool fp64, const DfDim* dims, int nd, int max_naux, int max_pairs, int max_on, int max_v,
                      const double* C, const double* eps, void* half, double* part, double* E2, cudaStream_t s);

// Split dimers: E2[dimer] = sum, in block order, of E2[first .. first+n) for
// each (dimer, first, n) triple of `fold` (device, 3 ints each).
cudaError_t launch_fold(const int* fold, int nfold, double* E2, cudaStream_t s);

// Per-monomer halves and the compensated lattice total (two launches: the
// per-monomer sums with the total's block partials, then their merge).
// scratch: 4 * kReduceBlocks doubles.
constexpr int kReduceBlocks = 128;
cudaError_t launch_reduce(const double* E2, int nd, MonomerLists lists,
                          double* mon /* 2*n_mon */, double* total /* 2 */, double* scratch, cudaStream_t s);

// Finiteness check of n doubles; sets *flag to 1 if any is NaN/Inf.
// Symmetry-packed dimer integrals (MCPT_AO_PACKED): packed_elems(nX, nY)
// doubles expanded into blocks = [A | K] (BLOCKS layout, 2 nX^2 nY^2).
size_t packed_elems(int nX, int nY);
cudaError_t launch_unpack(const double* packed, double* blocks, int nX, int nY, cudaStream_t s);
// Several dimers' packed integrals staged back to back, expanded by one
// launch: dimer k's packed data at staging + e[k].src, its blocks to e[k].dst.
struct UnpackEntry {
    long long src;
    double* dst;
    int nX, nY;
};
constexpr int kUnpackBatch = 64;
struct UnpackBatch {
    const double* staging;
    int n;
    UnpackEntry e[kUnpackBatch];
};
cudaError_t launch_unpack_batch(const UnpackBatch& B, cudaStream_t s);
cudaError_t launch_check_finite(const double* x, long long n, int* flag, cudaStream_t s);
// Same for a strided 4-index block.
cudaError_t launch_check_finite4(const double* x, const int dims[4], const long long st[3],
                                 int* flag, cudaStream_t s);

// Record the calling thread's last error (read by mcpt_last_error(NULL)) for
// entry points that have no handle.
void set_thread_error(const char* msg);

// ---- tensor-core first half (tcgen05) ----
enum TcKind { TC_TF32 = 0, TC_BF16X3 = 1, TC_BF16X2 = 2, TC_FP64E = 3 };

// Everything one launch of the tensor-core kernel needs; filled by
// tc_prepare (host work: tensor maps, work items, their upload), replayed by
// tc_launch (kernel launch only).
struct TcLaunch {
    const void* items;          // device TcItem array
    int n_items;
    const void* maps;           // device CUtensorMap array, [dimer][form]
    const DimerDesc* desc;      // device descriptors of the launch's dimers
    const float* Cf;            // FP32 coefficient pool
    const double* Cd;           // FP64 coefficient pool (TC_FP64E)
    void* H;                    // first-half result: float, or double for TC_FP64E
    int h_pairs;                // TC_FP64E: H as FP32 pairs (waves of monomers of <= 32 AO)
    int* status;
    int sf;                     // FP64 staging stages
    unsigned f_stage_bytes, w_stage_bytes, tmem_cols;
    int kind;
    int variant;                // 0: Kronecker (p0,p2) GEMM; 1, 3: p2 GEMM + FP32 rank-1 epilogue in registers
                                // (occupations <= 8, <= 5); 2: the same with TMEM accumulators (<= 16);
                                // 4: TMEM accumulators for o_X <= 20, o_Y <= 16
    int kcs_max;                // p2 chunks of 32 (largest n_Y of the launch)
    int grid;
    size_t smem;
    unsigned long long wait_ns; // limit of each device-side wait (0 = 4 s)
    int withhold;               // test aid: CTA 0 issues only withhold - 1 integral loads (0 = off)
};

// Launch choices of one tensor-core launch (0 in a field = the default):
// kernel variant + 1 (1 Kronecker, 2 rank with register accumulators, 3 rank
// with TMEM accumulators, 4 rank with register accumulators for occupations
// <= 5, 5 rank with TMEM accumulators for o_X <= 20), FP64 staging depth, CTAs.
struct TcTune {
    int variant1;
    int sf;
    int grid;
};

// Bytes of device work space (tensor maps + items) the dimers need.
size_t tc_work_bytes(TcKind kind, const DimerDesc* h_desc, int nd);
// The launch choices worth timing for these dimers (at most `max`): the
// exact kernels that accept them (the Kronecker kernel only where no rank
// kernel does), a few staging depths, and two grid sizes.
int tc_candidates(TcKind kind, const DimerDesc* h_desc, int nd, TcTune* out, int max);
// Encode tensor maps, order work items (longest first), upload them to
// d_work, and fill *out.  Synchronous w.r.t. the host buffers.  `tune`
// (may be NULL) overrides the default launch choices.
cudaError_t tc_prepare(TcKind kind, const DimerDesc* h_desc, const DimerDesc* d_desc, int nd, const float* Cf,
                       const double* Cd, void* H, void* d_work, size_t work_bytes, int* d_status, cudaStream_t s,
                       const TcTune* tune, TcLaunch* out, char* err, size_t errlen);
cudaError_t tc_launch(const TcLaunch& L, cudaStream_t s);

}  // namespace mcpt
