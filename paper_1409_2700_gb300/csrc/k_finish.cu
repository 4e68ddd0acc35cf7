// k_finish.cu -- second half of the dimer transformation, the FP64 energy
// epilogue, and the per-monomer accumulation.
//
// For each occupied pair (i, j) the first half left two nX x nY matrices
//   H_0[(nu,sig)][(i,j)]   (nu in X, sig in Y)   from the (XX|YY) block
//   H_1[(lam,nu)][(i,j)]   (lam in Y, nu in X)   from the (XY|YX) block
// and the virtual quarter transformations of Eq. (dp2e) finish them:
//   (i a|j b) = sum_nu C_X[nu][a] sum_sig H_0[nu][sig] C_Y[sig][b]
//   (i b|j a) = sum_lam C_Y[lam][b] sum_nu H_1[lam][nu] C_X[nu][a]
// Then, at FP64 accuracy (Sec. II.C energy tensor, Eq. (ed2) with T = vD):
//   D = 1/(e_i + e_j - e_a - e_b),  E_J += 4 (ia|jb)^2 D,  E_K += -2 (ia|jb)(ib|ja) D.
// GB300's FP64 unit runs at 1/64 of its FP32 rate.  The FP64 form keeps every
// step on it at the fewest operations per term: v D from an FP32 reciprocal
// seed and two Newton steps in FP64, the last folded into the product
// (convert.h), then one FMA each for E_J and E_K.  The mixed forms take
// e_i + e_j - e_a in FP64 once per (pair, a) and the rest on FP32 pairs
// (48-bit double-length arithmetic, below): the last subtraction, D to ~2^-45
// relative (the accuracy of one FP64 Newton step from an FP32 seed), the
// products with D and the sums over b, added to the FP64 sums once per pair --
// no FP64 operation per term.  The FP64-pipe variant of that epilogue (five
// FP64 operations per term) stays selectable for comparison.
// Monomers of at most 32 AO: one CTA per dimer, one warp per occupied pair.
// Larger ones: register-tiled GEMMs, one CTA per range of a dimer's pairs,
// the ranges' partial sums added per dimer in range order.  Every sum has a
// fixed order: the energies are deterministic run to run, with no atomics.
#include "internal.h"
#include "convert.h"
#include "ff.h"

#include <algorithm>

namespace mcpt {
namespace {

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// FP64 to the storage type (FP32 through the integer pipes)
template <typename T> __device__ __forceinline__ T narrow(double x);
template <> __device__ __forceinline__ double narrow<double>(double x) { return x; }
template <> __device__ __forceinline__ float narrow<float>(double x) { return f32_from_f64(x); }

// The mixed forms' terms of one (i, a, j, b) on FP32 pairs: x = e_ija - e_b,
// D = 1/x, E_J += v^2 D, E_K += v vk D into the pair accumulators sj, sk;
// returns v D (FP32) for the coupling store.  v^2 and v vk are FP32 products
// as in the FP64 variant; D, the products with D and the sums keep ~2^-45.
__device__ __forceinline__ float energy_terms_ff(float v, float vk, FF eija, FF eb, FF& sj, FF& sk)
{
    const FF D = ff_rcp(ff_sub(eija, eb));
    ff_acc(sj, __fmul_rn(v, v), D);
    ff_acc(sk, __fmul_rn(v, vk), D);
    return fmaf(v, D.l, __fmul_rn(v, D.h));
}

// The energy terms of one (i, a, j, b) with v = (ia|jb), vk = (ib|ja) and the
// FP64 denominator x = e_i + e_j - e_a - e_b: D = 1/x in FP64, then
// E_J += v^2 D and E_K += v vk D as FP64 sums; *vd (may be null) gets v D.
// FP64 form: v D by two Newton steps from an FP32 seed, the last folded into
// the product (full FP64 accuracy).  Mixed forms: D = r + r (1 - x r) from
// the FP32 seed r (relative error ~2^-46), v^2 and v vk as FP32 products (one
// rounding of 2^-24, far below the error these forms carry into v): five
// FP64 operations per term, the fewest that keep D and the sums in FP64.
template <typename T>
__device__ __forceinline__ void energy_terms(T v, T vk, double x, double& ej, double& ek, double* vd)
{
    if constexpr (sizeof(T) == 8) {
        const double t = div_newton<2>(v, x);
        ej = fma(t, v, ej);
        ek = fma(t, vk, ek);
        if (vd) *vd = t;
    } else {
        const double r = rcp_seed_f64(x);
        const double D = fma(r, fma(-x, r, 1.0), r);
        ej = fma(f64_from_f32(v * v), D, ej);
        ek = fma(f64_from_f32(v * vk), D, ek);
        if (vd) *vd = f64_from_f32(v) * D;
    }
}

// ---------------------------------------------------------------------------
// Monomers of at most 32 AO: one warp per occupied pair (i, j).
//   lane b:  tm[nu] = sum_sig H0[nu][sig] C_Y[sig][b]         (C_Y column b in registers)
//            VA[a][b] = sum_nu C_X[nu][a] tm[nu]              (C_X rows broadcast from smem)
//   lane a:  tk[lam] = sum_nu H1[lam][nu] C_X[nu][a]
//            VK[b][a] = sum_lam C_Y[lam][b] tk[lam]           (FP32: all b, into a third slab;
//                                                              FP64: b by b in the energy loop)
//            for each b, with VA[a][b], VK and the FP64 denominator, the two
//            energy terms of (a, b)
// Two slice buffers per warp swap roles every pair and are filled by cp.async
// one step ahead: H1 of this pair streams in during the H0 work, H0 of the
// next pair during the H1 work, so the warp rarely waits on memory.  VA
// takes the place of H0 in its buffer.  Per-lane sums reduce in a fixed order.
// W warps per CTA (4 or 5, chosen per wave by finish_w32_warps from the
// occupancy of each and the rounds of one pair per warp a dimer takes: o_X o_Y
// = 25 pairs fill five warps evenly, but at 166 registers five warps fit two
// CTAs per SM against four warps' three, and four measured faster).
constexpr int kW32Slab = 32 * 33;      // one padded 32 x 32 tile (row stride 33)
constexpr int kCS = 36;                // row stride of the staged C columns: 16-byte rows for vector
                                       // loads, lane rows 4 banks apart (4-way instead of 32-way)

// FP32 (the mixed forms) adds a third slab per warp: the pair's (ib|ja),
// formed for all b before the energy loop, which then runs no multiply-add
// chain of its own (the FP64 form keeps two slabs, for its occupancy).
template <typename T>
__host__ __device__ constexpr int w32_slabs() { return sizeof(T) == 4 ? 3 : 2; }

template <typename T>
constexpr size_t w32_smem_bytes(int W)
{
    return 32 * sizeof(double) + 32 * sizeof(FF) + 2 * 32 * kCS * sizeof(T) +
           W * w32_slabs<T>() * kW32Slab * sizeof(T);
}

// sum_{m < 32} a[m] x[m], a a 16-byte aligned row in shared memory (read as
// broadcasts), x in registers.  FP64 (the FP64 form): one chain in m order.
__device__ __forceinline__ double dot32(const double* a, const double (&x)[32])
{
    double acc = 0;
#pragma unroll
    for (int m = 0; m < 32; m++) acc = fma(a[m], x[m], acc);
    return acc;
}

// FP32: the sums of R rows at once, rows a + r * stride (16-byte aligned),
// each as two chains (even and odd m) advanced together by the packed FP32
// multiply-add (one instruction per two products) and added at the end; the
// R rows' chains interleave in issue order, so that a warp has R
// multiply-adds in flight instead of one dependent chain.
template <int R>
__device__ __forceinline__ void dots32(const float* a, int stride, const float (&x)[32], float (&out)[R])
{
    float2 acc[R];
#pragma unroll
    for (int r = 0; r < R; r++) acc[r] = make_float2(0.f, 0.f);
#pragma unroll
    for (int q = 0; q < 8; q++) {
        float4 v[R];
#pragma unroll
        for (int r = 0; r < R; r++) v[r] = reinterpret_cast<const float4*>(a + r * stride)[q];
#pragma unroll
        for (int r = 0; r < R; r++)
            acc[r] = __ffma2_rn(make_float2(v[r].x, v[r].y), make_float2(x[4 * q], x[4 * q + 1]), acc[r]);
#pragma unroll
        for (int r = 0; r < R; r++)
            acc[r] = __ffma2_rn(make_float2(v[r].z, v[r].w), make_float2(x[4 * q + 2], x[4 * q + 3]), acc[r]);
    }
#pragma unroll
    for (int r = 0; r < R; r++) out[r] = __fadd_rn(acc[r].x, acc[r].y);
}

// The same sum as two chains (even and odd m), for the FP64 form.
__device__ __forceinline__ double dot32_2(const double* a, const double (&x)[32])
{
    double v0 = 0, v1 = 0;
#pragma unroll
    for (int m = 0; m < 32; m += 2) {
        v0 = fma(a[m], x[m], v0);
        v1 = fma(a[m + 1], x[m + 1], v1);
    }
    return v0 + v1;
}

// One warp starts the asynchronous copy of an nr x nc (<= 32 x 32) row-major
// slice into a zero-padded 32 x 32 tile (lane c copies column c of every
// row; padding is written as zeros by the copy itself) and commits it as one
// group of this lane's cp.async operations.
template <typename T>
__device__ __forceinline__ void prefetch_slice(T* S, const T* __restrict__ h, int nr, int nc, int lane)
{
    const T* p = h + lane;
    const bool col = lane < nc;
    const unsigned dst0 = (unsigned)__cvta_generic_to_shared(S + lane);
#pragma unroll 4
    for (int r = 0; r < 32; r++) {
        const bool ok = r < nr && col;
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(dst0 + (unsigned)(r * 32 * sizeof(T))),
                     "l"(ok ? p : h), "n"(sizeof(T)), "r"(ok ? (int)sizeof(T) : 0)
                     : "memory");
        p += nc;
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// Wait until at most N of this lane's copy groups are in flight, then make
// the whole warp's copies visible to the warp.
template <int N>
__device__ __forceinline__ void slice_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
    __syncwarp();
}

// STORE: also write the dimer's (ia|jb) and T for the coupling (a separate
// instantiation keeps the plain path's registers).  PAIRS (mixed forms only):
// the energy terms on FP32 pairs, summed per (pair, a) and added to the FP64
// sums once per pair; otherwise on the FP64 pipe term by term.
template <typename T, bool STORE, bool PAIRS, int W>
__global__ void __launch_bounds__(W * 32, W == 4 ? 3 : 2)
k_finish_w32(const DimerDesc* __restrict__ dd, const T* __restrict__ C, const double* __restrict__ Epool,
             const T* __restrict__ H, double* __restrict__ E2, T* __restrict__ VT)
{
    const DimerDesc& d = dd[blockIdx.x];
    const int nX = d.nX, nY = d.nY, oX = d.oX, oY = d.oY;
    const int vX = d.vX, vY = d.vY;
    const int rows = nX * nY, pairs = oX * oY;
    const T* CXv = C + d.cXv;                 // virtual columns
    const T* CYv = C + d.cYv;
    const double* eX = Epool + d.eX;          // occupied energies of this block
    const double* eY = Epool + d.eY;
    const T* H0 = H + d.h_off;
    const T* H1 = H + d.h_off + (long long)pairs * rows;

    extern __shared__ __align__(16) unsigned char smraw[];
    static_assert(!PAIRS || sizeof(T) == 4, "FP32 pairs serve the mixed forms");
    double* eYv = reinterpret_cast<double*>(smraw);          // [b]: e_b (read as a broadcast)
    FF* eYs = reinterpret_cast<FF*>(eYv + 32);                // [b]: e_b as an FP32 pair
    T* CXT = reinterpret_cast<T*>(eYs + 32);                  // [a][nu], zero padded, row stride kCS
    T* CYT = CXT + 32 * kCS;                                  // [b][sig]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T* const buf = CYT + 32 * kCS + warp * (w32_slabs<T>() * kW32Slab);   // two slice buffers of kW32Slab
    [[maybe_unused]] T* const SV = buf + 2 * kW32Slab;        // FP32: (ib|ja) as [b][a] (stride 33)

    // the warp's first pair streams in while the block stages C and the energies
    if (warp < pairs) {
        prefetch_slice(buf, H0 + (long long)warp * rows, nX, nY, lane);
        prefetch_slice(buf + kW32Slab, H1 + (long long)warp * rows, nY, nX, lane);
    }
    {
        // all loads first (independent, in flight together), then the stores;
        // lanes run along a, the contiguous index of the coefficient rows
        constexpr int kPer = (32 * 32 + W * 32 - 1) / (W * 32);
        T cxv[kPer], cyv[kPer];
#pragma unroll
        for (int t = 0; t < kPer; t++) {
            const int k = threadIdx.x + t * W * 32;
            const int m = k >> 5, a = k & 31;
            cxv[t] = (a < vX && m < nX) ? CXv[m * nX + a] : T(0);   // k >= 1024 gives m >= 32 > nX
            cyv[t] = (a < vY && m < nY) ? CYv[m * nY + a] : T(0);
        }
#pragma unroll
        for (int t = 0; t < kPer; t++) {
            const int k = threadIdx.x + t * W * 32;
            if (k < 32 * 32) {
                CXT[(k & 31) * kCS + (k >> 5)] = cxv[t];
                CYT[(k & 31) * kCS + (k >> 5)] = cyv[t];
            }
        }
        if (threadIdx.x < 32) {
            const double e = threadIdx.x < vY ? Epool[d.eYv + threadIdx.x] : 0.0;
            eYv[threadIdx.x] = e;
            eYs[threadIdx.x] = ff_split(e);
        }
    }
    __syncthreads();

    const bool live = lane < vX;
    const double ea = live ? Epool[d.eXv + lane] : 0.0;   // this lane's virtual orbital a
    // coupling storage: (ia|jb) and T = vD as [(j,b)][(i,a)] over the whole dimer
    const bool store = STORE && d.vt_off >= 0;
    const long long mXc = (long long)d.oXt * vX, mYc = (long long)d.oYt * vY;
    T* const Vst = store ? VT + d.vt_off : nullptr;
    double ej = 0.0, ek = 0.0;
    int x = 0;                                   // buffer holding this pair's H0
    for (int pr = warp; pr < pairs; pr += W, x ^= 1) {
        const int i = pr / oY, j = pr % oY;
        const double eija = (eX[i] + eY[j]) - ea;  // e_i + e_j - e_a of this lane
        [[maybe_unused]] const FF eijas = PAIRS ? ff_split(eija) : FF{0.f, 0.f};
        [[maybe_unused]] FF sj{0.f, 0.f}, sk{0.f, 0.f};   // this pair's sums over even b (PAIRS)
        [[maybe_unused]] FF sj1{0.f, 0.f}, sk1{0.f, 0.f}; // and over odd b
        const int nx = pr + W;                   // next pair of this warp
        T* SX = x ? buf + kW32Slab : buf;        // H0, then VA [a][b] (stride 33)
        T* SY = x ? buf : buf + kW32Slab;        // H1, then the next pair's H0
        // ---- (i a|j b): SX[nu][sig] = H0 slice; lane b
        slice_wait<1>();
        {
            T cy[32], tm[32];
#pragma unroll
            for (int m = 0; m < 32; m++) cy[m] = CYT[lane * kCS + m];
            if constexpr (sizeof(T) == 4) {
#pragma unroll
                for (int nu = 0; nu < 32; nu += 2) {
                    float o[2];
                    dots32<2>(SX + nu * 32, 32, cy, o);
                    tm[nu] = o[0];
                    tm[nu + 1] = o[1];
                }
            } else {
#pragma unroll
                for (int nu = 0; nu < 32; nu++) tm[nu] = dot32(SX + nu * 32, cy);
            }
            __syncwarp();                        // H0 consumed: VA takes its place
            // rows a >= vX of VA are never read (only lanes a < vX form terms)
            if constexpr (sizeof(T) == 4) {
#pragma unroll 1
                for (int a = 0; a < vX; a += 4) {   // CXT rows up to 32 are zero padded
                    float o[4];
                    dots32<4>(CXT + a * kCS, kCS, tm, o);
#pragma unroll
                    for (int r = 0; r < 4; r++) SX[(a + r) * 33 + lane] = o[r];
                }
            } else {
#pragma unroll 4
                for (int a = 0; a < vX; a++) SX[a * 33 + lane] = dot32(CXT + a * kCS, tm);
            }
        }
        // ---- (i b|j a): SY[lam][nu] = H1 slice; lane a
        slice_wait<0>();
        {
            T cx[32], tk[32];
#pragma unroll
            for (int m = 0; m < 32; m++) cx[m] = CXT[lane * kCS + m];
            if constexpr (sizeof(T) == 4) {
#pragma unroll
                for (int lam = 0; lam < 32; lam += 2) {
                    float o[2];
                    dots32<2>(SY + lam * 32, 32, cx, o);
                    tk[lam] = o[0];
                    tk[lam + 1] = o[1];
                }
            } else {
#pragma unroll
                for (int lam = 0; lam < 32; lam++) tk[lam] = dot32(SY + lam * 32, cx);
            }
            __syncwarp();                        // H1 consumed: the next pair's H0 streams into SY
            if (nx < pairs) prefetch_slice(SY, H0 + (long long)nx * rows, nX, nY, lane);
            // ---- FP32: (ib|ja) of every b into this lane's column of SV, four
            // independent multiply-add chains at a time (each lane reads back
            // only its own column)
            if constexpr (sizeof(T) == 4) {
#pragma unroll 1
                for (int b = 0; b < vY; b += 4) {   // CYT rows up to 32 are zero padded
                    float o[4];
                    dots32<4>(CYT + b * kCS, kCS, tk, o);
#pragma unroll
                    for (int r = 0; r < 4; r++) SV[(b + r) * 33 + lane] = o[r];
                }
            }
            // ---- denominators and energy sums, lane a over b
            if constexpr (PAIRS) {
                // two b at a time, even b into (sj, sk) and odd b into (sj1, sk1):
                // independent chains for the FP32 pipes; an odd vY's last odd b
                // adds exact zeros
#pragma unroll 1
                for (int b = 0; b < vY; b += 2) {
                    const bool has1 = b + 1 < vY;
                    if (live) {
                        const T v0 = SX[lane * 33 + b], vk0 = SV[b * 33 + lane];
                        const T v1 = has1 ? SX[lane * 33 + b + 1] : T(0);
                        const T vk1 = has1 ? SV[(b + 1) * 33 + lane] : T(0);
                        const T tv0 = energy_terms_ff(v0, vk0, eijas, eYs[b], sj, sk);
                        const T tv1 = energy_terms_ff(v1, vk1, eijas, eYs[b + 1], sj1, sk1);
                        if (store) {
                            const long long e = ((long long)(d.jY0 + j) * vY + b) * mXc + (long long)(d.iX0 + i) * vX + lane;
                            Vst[e] = v0;
                            Vst[mXc * mYc + e] = tv0;
                            if (has1) {
                                Vst[e + mXc] = v1;
                                Vst[mXc * mYc + e + mXc] = tv1;
                            }
                        }
                    }
                }
            } else {
#pragma unroll 1
                for (int b = 0; b < vY; b++) {
                    T vk;
                    if constexpr (sizeof(T) == 4) vk = SV[b * 33 + lane];
                    else vk = dot32_2(CYT + b * kCS, tk);   // two chains of 16
                    if (live) {
                        const T vab = SX[lane * 33 + b];
                        double t;
                        energy_terms<T>(vab, vk, eija - eYv[b], ej, ek, store ? &t : nullptr);
                        if (store) {
                            const long long e = ((long long)(d.jY0 + j) * vY + b) * mXc + (long long)(d.iX0 + i) * vX + lane;
                            Vst[e] = vab;
                            Vst[mXc * mYc + e] = narrow<T>(t);
                        }
                    }
                }
            }
        }
        if constexpr (PAIRS) {
            ej += ff_f64(sj);
            ek += ff_f64(sk);
            ej += ff_f64(sj1);
            ek += ff_f64(sk1);
        }
        __syncwarp();                            // VA consumed: the next pair's H1 streams into SX
        if (nx < pairs) prefetch_slice(SX, H1 + (long long)nx * rows, nY, nX, lane);
    }
    __shared__ double red[2][W];
    ej = warp_sum(ej);
    ek = warp_sum(ek);
    if (lane == 0) { red[0][warp] = ej; red[1][warp] = ek; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sj = 0.0, sk = 0.0;
        for (int w = 0; w < W; w++) { sj += red[0][w]; sk += red[1][w]; }
        E2[2 * d.slot + 0] = 4.0 * sj;
        E2[2 * d.slot + 1] = -2.0 * sk;
    }
}

// ---------------------------------------------------------------------------
// FP64E second half, monomers of at most 32 AO: the structure of
// k_finish_w32 with every value an FP32 pair (ff.h) -- the H slices written
// as pairs by the first half, C, the virtual quarter transformations as pair
// multiply-adds, and the energy terms with v^2 and v vk as pair products and
// D = 1/x on pairs -- so that the FP64 form's accuracy (~2^-45 per step) is
// kept off the FP64 pipe, whose rate a multiply-add per (row, pair) term
// would otherwise set.  The C columns stay in shared memory (a lane's column
// as pairs would take 64 registers); four outputs accumulate at once so that
// each lane runs independent chains.  Per-lane sums over b go into FP64 sums
// once per occupied pair; with STORE the dimer's (ia|jb) and T = vD are
// written as FP64 for the coupling.
constexpr int kFFSlab = 32 * 33;   // one padded 32 x 32 tile of pairs (row stride 33)
constexpr int kFFChains = 4;       // independent pair multiply-add chains per lane (eight measured slower)

size_t w32_ff_smem_bytes(int W) { return (32 + 2 * (size_t)kFFSlab + 2 * (size_t)W * kFFSlab) * sizeof(FF); }

template <bool STORE, int W>
__global__ void __launch_bounds__(W * 32, 2)
k_finish_w32_ff(const DimerDesc* __restrict__ dd, const double* __restrict__ C, const double* __restrict__ Epool,
                const FF* __restrict__ H, double* __restrict__ E2, double* __restrict__ VT)
{
    const DimerDesc& d = dd[blockIdx.x];
    const int nX = d.nX, nY = d.nY, oX = d.oX, oY = d.oY;
    const int vX = d.vX, vY = d.vY;
    const int rows = nX * nY, pairs = oX * oY;
    const double* CXv = C + d.cXv;            // virtual columns
    const double* CYv = C + d.cYv;
    const double* eX = Epool + d.eX;          // occupied energies of this block
    const double* eY = Epool + d.eY;
    const FF* H0 = H + d.h_off;
    const FF* H1 = H + d.h_off + (long long)pairs * rows;

    extern __shared__ __align__(16) unsigned char smraw[];
    FF* eYs = reinterpret_cast<FF*>(smraw);   // [b]: e_b
    FF* CXT = eYs + 32;                       // [a][nu], row stride 33, zero padded
    FF* CYT = CXT + kFFSlab;                  // [b][sig]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    FF* const buf = CYT + kFFSlab + warp * (2 * kFFSlab);   // two slice buffers

    if (warp < pairs) {
        prefetch_slice(buf, H0 + (long long)warp * rows, nX, nY, lane);
        prefetch_slice(buf + kFFSlab, H1 + (long long)warp * rows, nY, nX, lane);
    }
    for (int k = threadIdx.x; k < 32 * 32; k += W * 32) {
        const int m = k >> 5, a = k & 31;       // lanes along the contiguous index a
        CXT[a * 33 + m] = (a < vX && m < nX) ? ff_split(CXv[m * nX + a]) : FF{0.f, 0.f};
        CYT[a * 33 + m] = (a < vY && m < nY) ? ff_split(CYv[m * nY + a]) : FF{0.f, 0.f};
    }
    if (threadIdx.x < 32) eYs[threadIdx.x] = threadIdx.x < vY ? ff_split(Epool[d.eYv + threadIdx.x]) : FF{0.f, 0.f};
    __syncthreads();

    const bool live = lane < vX;
    const double ea = live ? Epool[d.eXv + lane] : 0.0;   // this lane's virtual orbital a
    const bool store = STORE && d.vt_off >= 0;
    const long long mXc = (long long)d.oXt * vX, mYc = (long long)d.oYt * vY;
    double* const Vst = store ? VT + d.vt_off : nullptr;
    double ej = 0.0, ek = 0.0;
    int x = 0;                                   // buffer holding this pair's H0
    for (int pr = warp; pr < pairs; pr += W, x ^= 1) {
        const int i = pr / oY, j = pr % oY;
        const FF eija = ff_split((eX[i] + eY[j]) - ea);   // e_i + e_j - e_a of this lane
        FF sj{0.f, 0.f}, sk{0.f, 0.f};
        const int nx = pr + W;
        FF* SX = x ? buf + kFFSlab : buf;        // H0 (row stride 32), then VA [a][b] (stride 33)
        FF* SY = x ? buf : buf + kFFSlab;        // H1, then the next pair's H0
        // ---- (i a|j b): lane b, tm[nu] = sum_sig H0[nu][sig] C_Y[sig][b]
        slice_wait<1>();
        {
            FF tm[32];
            const FF* cy = CYT + lane * 33;
#pragma unroll
            for (int nu = 0; nu < 32; nu += kFFChains) {
                FF acc[kFFChains];
#pragma unroll
                for (int q = 0; q < kFFChains; q++) acc[q] = FF{0.f, 0.f};
#pragma unroll 4
                for (int m = 0; m < 32; m++) {
                    const FF c = cy[m];
#pragma unroll
                    for (int q = 0; q < kFFChains; q++) ff_mac(acc[q], SX[(nu + q) * 32 + m], c);
                }
#pragma unroll
                for (int q = 0; q < kFFChains; q++) tm[nu + q] = acc[q];
            }
            __syncwarp();                        // H0 consumed: VA takes its place
#pragma unroll 1
            for (int a = 0; a < 32; a += kFFChains) {
                FF acc[kFFChains];
#pragma unroll
                for (int q = 0; q < kFFChains; q++) acc[q] = FF{0.f, 0.f};
#pragma unroll
                for (int nu = 0; nu < 32; nu++)
#pragma unroll
                    for (int q = 0; q < kFFChains; q++) ff_mac(acc[q], CXT[(a + q) * 33 + nu], tm[nu]);
#pragma unroll
                for (int q = 0; q < kFFChains; q++) SX[(a + q) * 33 + lane] = acc[q];
            }
        }
        // ---- (i b|j a): lane a, tk[lam] = sum_nu H1[lam][nu] C_X[nu][a]
        slice_wait<0>();
        {
            FF tk[32];
            const FF* cx = CXT + lane * 33;
#pragma unroll
            for (int lam = 0; lam < 32; lam += kFFChains) {
                FF acc[kFFChains];
#pragma unroll
                for (int q = 0; q < kFFChains; q++) acc[q] = FF{0.f, 0.f};
#pragma unroll 4
                for (int m = 0; m < 32; m++) {
                    const FF c = cx[m];
#pragma unroll
                    for (int q = 0; q < kFFChains; q++) ff_mac(acc[q], SY[(lam + q) * 32 + m], c);
                }
#pragma unroll
                for (int q = 0; q < kFFChains; q++) tk[lam + q] = acc[q];
            }
            __syncwarp();                        // H1 consumed: the next pair's H0 streams into SY
            if (nx < pairs) prefetch_slice(SY, H0 + (long long)nx * rows, nX, nY, lane);
            // ---- denominators and energy sums, lane a over b
#pragma unroll 1
            for (int b = 0; b < vY; b++) {
                FF v0{0.f, 0.f}, v1{0.f, 0.f};   // two chains of 16
#pragma unroll
                for (int lam = 0; lam < 32; lam += 2) {
                    ff_mac(v0, CYT[b * 33 + lam], tk[lam]);
                    ff_mac(v1, CYT[b * 33 + lam + 1], tk[lam + 1]);
                }
                if (live) {
                    const FF v = SX[lane * 33 + b];
                    const FF vk = ff_add(v0, v1);
                    const FF D = ff_rcp(ff_sub(eija, eYs[b]));
                    ff_mac(sj, ff_mul(v, v), D);
                    ff_mac(sk, ff_mul(v, vk), D);
                    if (store) {
                        const long long e = ((long long)(d.jY0 + j) * vY + b) * mXc + (long long)(d.iX0 + i) * vX + lane;
                        Vst[e] = ff_f64(v);
                        Vst[mXc * mYc + e] = ff_f64(ff_mul(v, D));
                    }
                }
            }
        }
        ej += ff_f64(sj);
        ek += ff_f64(sk);
        __syncwarp();                            // VA consumed: the next pair's H1 streams into SX
        if (nx < pairs) prefetch_slice(SX, H1 + (long long)nx * rows, nY, nX, lane);
    }
    __shared__ double red[2][W];
    ej = warp_sum(ej);
    ek = warp_sum(ek);
    if (lane == 0) { red[0][warp] = ej; red[1][warp] = ek; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sjt = 0.0, skt = 0.0;
        for (int w = 0; w < W; w++) { sjt += red[0][w]; skt += red[1][w]; }
        E2[2 * d.slot + 0] = 4.0 * sjt;
        E2[2 * d.slot + 1] = -2.0 * skt;
    }
}

// ---------------------------------------------------------------------------
// Monomers above 32 AO: the virtual quarter transformations of one occupied
// pair are four small GEMMs,
//   Tm  [nu][b]  = sum_sig H0[nu][sig]  C_Y[sig][oY+b]      (nX x vY, K = nY)
//   TmK [lam][a] = sum_nu  H1[lam][nu]  C_X[nu][oX+a]       (nY x vX, K = nX)
//   VA  [a][b]   = sum_nu  C_X[nu][oX+a] Tm[nu][b]          (vX x vY, K = nX)
//   VKT [a][b]   = sum_lam TmK[lam][a]  C_Y[lam][oY+b]      (vX x vY, K = nY)
// Each GEMM's M x N outputs are cut into 8 x 4 blocks dealt round-robin to the
// 256 threads, so small and ragged shapes keep the threads on useful work;
// a thread accumulates its block in registers (per K step 12 loads feed 32
// FMAs).  H slices and Tm/TmK live in shared memory, the C columns are read
// through L1.  VA and VKT use the same blocks, so each thread meets its own
// (a, b) terms for the FP64 epilogue (VA goes through shared memory to free
// its registers).  One CTA runs a range of pairs of one dimer; its FP64
// partial sums are written per task and added in task order by k_finish_sum.
constexpr int kTThreads = 256;
constexpr int kTM = 8, kTN = 4;

template <typename T>
size_t tiled_smem_bytes(int max_ao)
{
    const size_t n = (size_t)max_ao;
    return (n * n + 2 * n * n) * sizeof(T) + 2 * n * (sizeof(double) + sizeof(FF)) + 64;
}

// acc[i][j] = sum_k A(m0 + i, k) B(k, n0 + j) over rows < M, columns < N.
template <typename T, typename FA, typename FB>
__device__ __forceinline__ void mm_block(T (&acc)[kTM][kTN], int m0, int n0, int M, int N, int K, FA A, FB B)
{
#pragma unroll
    for (int i = 0; i < kTM; i++)
#pragma unroll
        for (int j = 0; j < kTN; j++) acc[i][j] = T(0);
    bool mok[kTM], nok[kTN];
#pragma unroll
    for (int i = 0; i < kTM; i++) mok[i] = m0 + i < M;
#pragma unroll
    for (int j = 0; j < kTN; j++) nok[j] = n0 + j < N;
#pragma unroll 2
    for (int k = 0; k < K; k++) {
        T a[kTM], b[kTN];
#pragma unroll
        for (int i = 0; i < kTM; i++) a[i] = mok[i] ? A(m0 + i, k) : T(0);
#pragma unroll
        for (int j = 0; j < kTN; j++) b[j] = nok[j] ? B(k, n0 + j) : T(0);
#pragma unroll
        for (int i = 0; i < kTM; i++)
#pragma unroll
            for (int j = 0; j < kTN; j++) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
}

template <typename T>
__device__ __forceinline__ void copy_slice(T* S, const T* __restrict__ src, int n, int tid)
{
    for (int k0 = 0; k0 < n; k0 += 4 * kTThreads) {
        T v[4];
#pragma unroll
        for (int t = 0; t < 4; t++) {
            const int k = k0 + t * kTThreads + tid;
            v[t] = k < n ? src[k] : T(0);
        }
#pragma unroll
        for (int t = 0; t < 4; t++) {
            const int k = k0 + t * kTThreads + tid;
            if (k < n) S[k] = v[t];
        }
    }
}

template <typename T, bool PAIRS>
__global__ void __launch_bounds__(kTThreads, 2)
k_finish_tiled(const DimerDesc* __restrict__ dd, const FinTask* __restrict__ tasks, const T* __restrict__ C,
               const double* __restrict__ Epool, const T* __restrict__ H, double* __restrict__ part,
               int smem_elems, T* __restrict__ VT)
{
    const FinTask tk = tasks[blockIdx.x];
    const DimerDesc& d = dd[tk.dimer];
    const int nX = d.nX, nY = d.nY, oY = d.oY;
    const int vX = d.vX, vY = d.vY;
    const int rows = nX * nY, pairs = d.oX * oY;
    const T* __restrict__ CXv = C + d.cXv;    // virtual columns
    const T* __restrict__ CYv = C + d.cYv;
    const double* eX = Epool + d.eX;          // occupied energies of this block
    const double* eY = Epool + d.eY;
    const T* H0 = H + d.h_off;
    const T* H1 = H + d.h_off + (long long)pairs * rows;

    extern __shared__ __align__(16) unsigned char smraw[];
    double* eXv = reinterpret_cast<double*>(smraw);           // [vX]
    double* eYv = eXv + nX;                                   // [vY]
    FF* eXs = reinterpret_cast<FF*>(eYv + nY);                // [vX]: e_a as FP32 pairs
    FF* eYs = eXs + nX;                                       // [vY]
    T* base = reinterpret_cast<T*>(eYs + nY);
    // a group of np pairs runs each phase together (one barrier per phase for
    // the group): as many as the launch's shared memory holds
    const int per_pair = rows + nX * vY + nY * vX;
    const int gmax = max(1, min(tk.pr1 - tk.pr0, smem_elems / per_pair));
    T* S = base;                                              // H slices [np][rows], then VA [np][vX][vY]
    T* Tm = S + gmax * rows;                                  // [np][nX][vY]
    T* TmK = Tm + gmax * nX * vY;                             // [np][nY][vX]
    const int tid = threadIdx.x;
    for (int k = tid; k < vX; k += kTThreads) { eXv[k] = Epool[d.eXv + k]; eXs[k] = ff_split(eXv[k]); }
    for (int k = tid; k < vY; k += kTThreads) { eYv[k] = Epool[d.eYv + k]; eYs[k] = ff_split(eYv[k]); }
    // 8 x 4 output blocks of each GEMM shape, per pair
    const int bn_vY = (vY + kTN - 1) / kTN, bn_vX = (vX + kTN - 1) / kTN;
    const int nb1 = ((nX + kTM - 1) / kTM) * bn_vY;          // Tm
    const int nb3 = ((nY + kTM - 1) / kTM) * bn_vX;          // TmK
    const int nb2 = ((vX + kTM - 1) / kTM) * bn_vY;          // VA, VKT

    const bool store = VT != nullptr && d.vt_off >= 0;
    const long long mXc = (long long)d.oXt * vX, mYc = (long long)d.oYt * vY;
    T* const Vst = store ? VT + d.vt_off : nullptr;
    double ej = 0.0, ek = 0.0;
    for (int g0 = tk.pr0; g0 < tk.pr1; g0 += gmax) {
        const int np = min(gmax, tk.pr1 - g0);
        T acc[kTM][kTN];
        // ---- Tm = H0 C_Y(virtual), every pair of the group
        copy_slice(S, H0 + (long long)g0 * rows, np * rows, tid);
        __syncthreads();
        for (int blk = tid; blk < np * nb1; blk += kTThreads) {
            const int p = blk / nb1, q = blk - p * nb1;
            const int m0 = (q / bn_vY) * kTM, n0 = (q % bn_vY) * kTN;
            const T* Sp = S + p * rows;
            T* Tp = Tm + p * nX * vY;
            mm_block<T>(acc, m0, n0, nX, vY, nY, [&](int m, int k) { return Sp[m * nY + k]; },
                        [&](int k, int n) { return __ldg(CYv + k * nY + n); });
#pragma unroll
            for (int a = 0; a < kTM; a++)
#pragma unroll
                for (int b = 0; b < kTN; b++)
                    if (m0 + a < nX && n0 + b < vY) Tp[(m0 + a) * vY + n0 + b] = acc[a][b];
        }
        __syncthreads();
        // ---- TmK = H1 C_X(virtual)
        copy_slice(S, H1 + (long long)g0 * rows, np * rows, tid);
        __syncthreads();
        for (int blk = tid; blk < np * nb3; blk += kTThreads) {
            const int p = blk / nb3, q = blk - p * nb3;
            const int m0 = (q / bn_vX) * kTM, n0 = (q % bn_vX) * kTN;
            const T* Sp = S + p * rows;
            T* Kp = TmK + p * nY * vX;
            mm_block<T>(acc, m0, n0, nY, vX, nX, [&](int m, int k) { return Sp[m * nX + k]; },
                        [&](int k, int n) { return __ldg(CXv + k * nX + n); });
#pragma unroll
            for (int a = 0; a < kTM; a++)
#pragma unroll
                for (int b = 0; b < kTN; b++)
                    if (m0 + a < nY && n0 + b < vX) Kp[(m0 + a) * vX + n0 + b] = acc[a][b];
        }
        __syncthreads();
        // ---- VA, VKT and the FP64 epilogue, block by block
        for (int blk = tid; blk < np * nb2; blk += kTThreads) {
            const int p = blk / nb2, q = blk - p * nb2;
            const int m0 = (q / bn_vY) * kTM, n0 = (q % bn_vY) * kTN;
            const int pr = g0 + p, i = pr / oY, j = pr - i * oY;
            const double eij = eX[i] + eY[j];
            const T* Tp = Tm + p * nX * vY;
            const T* Kp = TmK + p * nY * vX;
            T* Vp = S + p * rows;                                 // VA of pair p (own elements)
            mm_block<T>(acc, m0, n0, vX, vY, nX, [&](int m, int k) { return __ldg(CXv + k * nX + m); },
                        [&](int k, int n) { return Tp[k * vY + n]; });
#pragma unroll
            for (int a = 0; a < kTM; a++)
#pragma unroll
                for (int b = 0; b < kTN; b++)
                    if (m0 + a < vX && n0 + b < vY) Vp[(m0 + a) * vY + n0 + b] = acc[a][b];
            mm_block<T>(acc, m0, n0, vX, vY, nY, [&](int m, int k) { return Kp[k * vX + m]; },
                        [&](int k, int n) { return __ldg(CYv + k * nY + n); });
            [[maybe_unused]] const FF eijs = PAIRS ? ff_split(eij) : FF{0.f, 0.f};
            [[maybe_unused]] FF sj{0.f, 0.f}, sk{0.f, 0.f};   // this block's sums (PAIRS)
#pragma unroll
            for (int a = 0; a < kTM; a++) {
                const int m = m0 + a;
                [[maybe_unused]] FF eijas{0.f, 0.f};
                if constexpr (PAIRS)
                    if (m < vX) eijas = ff_sub(eijs, eXs[m]);
#pragma unroll
                for (int b = 0; b < kTN; b++) {
                    const int n = n0 + b;
                    if (m < vX && n < vY) {
                        const T vab = Vp[m * vY + n];
                        T tv;
                        if constexpr (PAIRS) {
                            tv = energy_terms_ff(vab, acc[a][b], eijas, eYs[n], sj, sk);
                        } else {
                            double t;
                            energy_terms<T>(vab, acc[a][b], eij - (eXv[m] + eYv[n]), ej, ek, store ? &t : nullptr);
                            tv = store ? narrow<T>(t) : T(0);
                        }
                        if (store) {
                            const long long e =
                                ((long long)(d.jY0 + j) * vY + n) * mXc + (long long)(d.iX0 + i) * vX + m;
                            Vst[e] = vab;
                            Vst[mXc * mYc + e] = tv;
                        }
                    }
                }
            }
            if constexpr (PAIRS) {
                ej += ff_f64(sj);
                ek += ff_f64(sk);
            }
        }
        __syncthreads();
    }
    // fixed-order block reduction
    __shared__ double red[2][kTThreads / 32];
    ej = warp_sum(ej);
    ek = warp_sum(ek);
    if ((tid & 31) == 0) { red[0][tid >> 5] = ej; red[1][tid >> 5] = ek; }
    __syncthreads();
    if (tid == 0) {
        double sj = 0.0, sk = 0.0;
        for (int w = 0; w < kTThreads / 32; w++) { sj += red[0][w]; sk += red[1][w]; }
        part[2 * blockIdx.x + 0] = sj;
        part[2 * blockIdx.x + 1] = sk;
    }
}

// Per dimer: its task partials in task order -> {4 sum, -2 sum}.
__global__ void k_finish_sum(const DimerDesc* __restrict__ dd, int nd, const FinTask* __restrict__ tasks,
                             const int* __restrict__ first_task, const double* __restrict__ part,
                             double* __restrict__ E2)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nd) return;
    const FinTask t0 = tasks[first_task[k]];
    double sj = 0.0, sk = 0.0;
    for (int t = t0.first; t < t0.first + t0.ntasks; t++) {
        sj += part[2 * t];
        sk += part[2 * t + 1];
    }
    E2[2 * dd[k].slot + 0] = 4.0 * sj;
    E2[2 * dd[k].slot + 1] = -2.0 * sk;
}

template <typename T, bool PAIRS, int W>
cudaError_t launch_w32(const DimerDesc* d_desc, int nd, const T* C, const double* Epool, const T* H, double* E2,
                       T* VT, cudaStream_t s)
{
    const size_t smem = w32_smem_bytes<T>(W);
    auto fn = VT ? k_finish_w32<T, true, PAIRS, W> : k_finish_w32<T, false, PAIRS, W>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    // all of the unified L1 as shared memory, so that the CTAs the registers
    // allow are also resident by shared memory
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    fn<<<nd, W * 32, smem, s>>>(d_desc, C, Epool, H, E2, VT);
    return cudaGetLastError();
}

template <typename T, bool PAIRS>
cudaError_t launch_finish(const DimerDesc* d_desc, int nd, int max_ao, const T* C, const double* Epool,
                          const T* H, double* E2, const FinTask* tasks, int ntasks, double* part, T* VT,
                          int w32_warps, cudaStream_t s)
{
    if (nd <= 0) return cudaSuccess;
    if (max_ao <= 32)
        return w32_warps == 5 ? launch_w32<T, PAIRS, 5>(d_desc, nd, C, Epool, H, E2, VT, s)
                              : launch_w32<T, PAIRS, 4>(d_desc, nd, C, Epool, H, E2, VT, s);
    if (!tasks || ntasks <= 0 || !part) return cudaErrorInvalidValue;
    const size_t smem = tiled_smem_bytes<T>(max_ao);
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k_finish_tiled<T, PAIRS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int smem_elems = (int)((smem - 2 * max_ao * (sizeof(double) + sizeof(FF)) - 64) / sizeof(T));
    k_finish_tiled<T, PAIRS><<<ntasks, kTThreads, smem, s>>>(d_desc, tasks, C, Epool, H, part, smem_elems, VT);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // the dimers' first-task indices follow the task array
    const int* first = reinterpret_cast<const int*>(tasks + ntasks);
    k_finish_sum<<<(nd + 127) / 128, 128, 0, s>>>(d_desc, nd, tasks, first, part, E2);
    return cudaGetLastError();
}

template <int W>
cudaError_t launch_finish_ff_t(const DimerDesc* d_desc, int nd, const double* C, const double* Epool, const FF* H,
                               double* E2, double* VT, cudaStream_t s)
{
    if (nd <= 0) return cudaSuccess;
    const size_t smem = w32_ff_smem_bytes(W);
    auto fn = VT ? k_finish_w32_ff<true, W> : k_finish_w32_ff<false, W>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    fn<<<nd, W * 32, smem, s>>>(d_desc, C, Epool, H, E2, VT);
    return cudaGetLastError();
}

// CTAs of the 32-AO second half resident per SM with W warps (the plain
// instantiation of the form; 0 if the query fails).
template <int W>
int w32_ctas_per_sm(int form)
{
    int n = 0, dev = 0, max_smem = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaError_t e = cudaErrorInvalidValue;
    auto occ = [&](auto fn, size_t smem) {
        if ((int)smem > max_smem) return cudaErrorInvalidValue;
        cudaError_t r = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (r == cudaSuccess && form != FIN_FF)
            r = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
        return r != cudaSuccess ? r : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, W * 32, smem);
    };
    switch (form) {
    case FIN_F64: e = occ(k_finish_w32<double, false, false, W>, w32_smem_bytes<double>(W)); break;
    case FIN_F32_PAIRS: e = occ(k_finish_w32<float, false, true, W>, w32_smem_bytes<float>(W)); break;
    case FIN_F32_F64EPI: e = occ(k_finish_w32<float, false, false, W>, w32_smem_bytes<float>(W)); break;
    case FIN_FF: e = occ(k_finish_w32_ff<false, W>, w32_ff_smem_bytes(W)); break;
    }
    return e == cudaSuccess ? n : 0;
}

// Split dimers: the blocks' terms added in block order.
__global__ void k_fold(const int* __restrict__ fold, int nfold, double* __restrict__ E2)
{
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nfold) return;
    const int d = fold[3 * f], first = fold[3 * f + 1], n = fold[3 * f + 2];
    double sj = 0.0, sk = 0.0;
    for (int b = 0; b < n; b++) {
        sj += E2[2 * (first + b)];
        sk += E2[2 * (first + b) + 1];
    }
    E2[2 * d] = sj;
    E2[2 * d + 1] = sk;
}

// ------------------------------------------------------------ reduction
__device__ __forceinline__ void neumaier_add(double& s, double& c, double v)
{
    const double t = s + v;
    if (fabs(s) >= fabs(v)) c += (s - t) + v;
    else                    c += (v - t) + s;
    s = t;
}

constexpr int kRedThreads = 256;
constexpr int kMonWarps = kRedThreads / 32;   // per-monomer sums: one warp per monomer

// Knuth's TwoSum of two compensated sums (s, c) and (s2, c2) into (s, c).
__device__ __forceinline__ void twosum_pair(double& s, double& c, double s2, double c2)
{
    const double t = s + s2;
    const double bp = t - s;
    const double err = (s - (t - bp)) + (s2 - bp);
    c = c + c2 + err;
    s = t;
}

// Blocks [0, nbm): one warp per monomer.  Lane l sums half of the terms of
// the monomer's dimers l, l + 32, ... of its list (Neumaier), and a fixed
// shuffle tree merges the 32 lane sums (TwoSum per merge): the list's loads
// are in flight together instead of one dependent load pair per dimer.
// Blocks [nbm, nbm + nbt): lattice-total partials, block b over a fixed
// contiguous range of the dimer list, its threads over fixed sub-chunks
// (Neumaier), merged by a fixed pairwise tree (TwoSum keeps each merge's
// rounding); k_total_merge then adds the block partials by the same tree.
// Long dependent FP64 chains are slow on GB300 and one SM's FP64 pipe is
// small, so the work is spread over many blocks; the partition depends only
// on the dimer and monomer counts, so every run gives the same bits.
__device__ __forceinline__ void twosum_merge(double* part, int t, int w)
{
#pragma unroll
    for (int f = 0; f < 4; f += 2) {
        const double a = part[f * kRedThreads + t], b = part[f * kRedThreads + t + w];
        const double s = a + b;
        const double bp = s - a;
        const double err = (a - (s - bp)) + (b - bp);
        part[f * kRedThreads + t] = s;
        part[(f + 1) * kRedThreads + t] = part[(f + 1) * kRedThreads + t] + part[(f + 1) * kRedThreads + t + w] + err;
    }
}

__global__ void __launch_bounds__(kRedThreads)
k_reduce(const double* __restrict__ E2, int nd, MonomerLists L, double* __restrict__ mon, int nbm, int nbt,
         double* __restrict__ partials)
{
    if ((int)blockIdx.x < nbm) {
        const int m = blockIdx.x * kMonWarps + (int)(threadIdx.x >> 5), lane = threadIdx.x & 31;
        if (m >= L.n_mon) return;                 // whole warps
        double sj = 0, cj = 0, sk = 0, ck = 0;
        for (int k = L.start[m] + lane; k < L.start[m + 1]; k += 32) {
            const int dslot = L.list[k];
            neumaier_add(sj, cj, 0.5 * E2[2 * dslot]);
            neumaier_add(sk, ck, 0.5 * E2[2 * dslot + 1]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double sj2 = __shfl_down_sync(0xffffffffu, sj, o), cj2 = __shfl_down_sync(0xffffffffu, cj, o);
            const double sk2 = __shfl_down_sync(0xffffffffu, sk, o), ck2 = __shfl_down_sync(0xffffffffu, ck, o);
            twosum_pair(sj, cj, sj2, cj2);
            twosum_pair(sk, ck, sk2, ck2);
        }
        if (lane == 0) {
            mon[m] = sj + cj;
            mon[L.n_mon + m] = sk + ck;
        }
        return;
    }
    __shared__ double part[4 * kRedThreads];
    const int b = blockIdx.x - nbm, t = threadIdx.x;
    const int per = (nd + nbt - 1) / nbt;
    const int b0 = b * per, b1 = min(nd, b0 + per);
    const int chunk = (per + kRedThreads - 1) / kRedThreads;
    const int lo = b0 + t * chunk, hi = min(b1, lo + chunk);
    double sj = 0, cj = 0, sk = 0, ck = 0;
    for (int k = lo; k < hi; k++) {
        neumaier_add(sj, cj, E2[2 * k]);
        neumaier_add(sk, ck, E2[2 * k + 1]);
    }
    part[t] = sj; part[kRedThreads + t] = cj; part[2 * kRedThreads + t] = sk; part[3 * kRedThreads + t] = ck;
    __syncthreads();
    for (int w = kRedThreads / 2; w > 0; w >>= 1) {
        if (t < w) twosum_merge(part, t, w);
        __syncthreads();
    }
    if (t < 4) partials[4 * b + t] = part[t * kRedThreads];
}

__global__ void __launch_bounds__(kRedThreads)
k_total_merge(const double* __restrict__ partials, int nbt, double* __restrict__ total)
{
    __shared__ double part[4 * kRedThreads];
    const int t = threadIdx.x;
#pragma unroll
    for (int f = 0; f < 4; f++) part[f * kRedThreads + t] = t < nbt ? partials[4 * t + f] : 0.0;
    __syncthreads();
    for (int w = kRedThreads / 2; w > 0; w >>= 1) {
        if (t < w) twosum_merge(part, t, w);
        __syncthreads();
    }
    if (t == 0) {
        total[0] = part[0] + part[kRedThreads];
        total[1] = part[2 * kRedThreads] + part[3 * kRedThreads];
    }
}

__global__ void k_check_finite(const double* __restrict__ x, long long n, int* flag)
{
    bool bad = false;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x)
        bad |= !isfinite(x[k]);
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
}

__global__ void k_check_finite4(const double* __restrict__ x, int d0, int d1, int d2, int d3,
                                long long s0, long long s1, long long s2, int* flag)
{
    const long long n = (long long)d0 * d1 * d2 * d3;
    bool bad = false;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        long long r = k;
        const int i3 = r % d3; r /= d3;
        const int i2 = r % d2; r /= d2;
        const int i1 = r % d1; r /= d1;
        const int i0 = (int)r;
        bad |= !isfinite(x[i0 * s0 + i1 * s1 + i2 * s2 + i3]);
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
}

}  // namespace

cudaError_t launch_finish_fp64(const DimerDesc* d_desc, int nd, int max_ao, const double* Cpool,
                               const double* Epool, const double* H, double* E2, const FinTask* tasks,
                               int ntasks, double* part, double* VT, int w32_warps, cudaStream_t s)
{
    return launch_finish<double, false>(d_desc, nd, max_ao, Cpool, Epool, H, E2, tasks, ntasks, part, VT,
                                        w32_warps, s);
}

cudaError_t launch_finish_fp32(const DimerDesc* d_desc, int nd, int max_ao, const float* Cf,
                               const double* Epool, const float* H, double* E2, const FinTask* tasks,
                               int ntasks, double* part, float* VT, bool fp64_epilogue, int w32_warps,
                               cudaStream_t s)
{
    return fp64_epilogue
               ? launch_finish<float, false>(d_desc, nd, max_ao, Cf, Epool, H, E2, tasks, ntasks, part, VT,
                                             w32_warps, s)
               : launch_finish<float, true>(d_desc, nd, max_ao, Cf, Epool, H, E2, tasks, ntasks, part, VT,
                                            w32_warps, s);
}

cudaError_t launch_finish_ff(const DimerDesc* d_desc, int nd, int max_ao, const double* Cpool, const double* Epool,
                             const void* H, double* E2, double* VT, int w32_warps, cudaStream_t s)
{
    if (max_ao > 32) return cudaErrorInvalidValue;
    const FF* Hf = static_cast<const FF*>(H);
    return w32_warps == 5 ? launch_finish_ff_t<5>(d_desc, nd, Cpool, Epool, Hf, E2, VT, s)
                          : launch_finish_ff_t<4>(d_desc, nd, Cpool, Epool, Hf, E2, VT, s);
}

int finish_w32_warps(const DimerDesc* h, int nd, int form)
{
    // a dimer's CTA takes ceil(pairs / W) rounds of one pair per warp; the
    // wave's time goes as the rounds over the CTAs an SM holds at once
    double t[2] = {0.0, 0.0};
    const int ctas[2] = {w32_ctas_per_sm<4>(form), w32_ctas_per_sm<5>(form)};
    if (form == FIN_FF) return 4;   // five warps per CTA measured slower for the FP32-pair form
    for (int w = 0; w < 2; w++) {
        if (ctas[w] <= 0) return 4;
        for (int k = 0; k < nd; k++) t[w] += (double)((h[k].oX * h[k].oY + 3 + w) / (4 + w)) / ctas[w];
    }
    return t[1] < t[0] ? 5 : 4;
}

void finish_tasks(const DimerDesc* h, int nd, int fma_per_task, std::vector<FinTask>* out)
{
    out->clear();
    for (int k = 0; k < nd; k++) {
        const long long nX = h[k].nX, nY = h[k].nY, vX = h[k].vX, vY = h[k].vY;
        const int pairs = h[k].oX * h[k].oY;
        const long long per_pair = 2 * (nX * nY * vY + vX * vY * nX);   // FMAs of one pair, both forms
        const int ppt = (int)std::max<long long>(1, std::min<long long>(pairs, fma_per_task / std::max(1LL, per_pair)));
        const int ntasks = (pairs + ppt - 1) / ppt;
        const int first = (int)out->size();
        for (int t = 0; t < ntasks; t++)
            out->push_back(FinTask{k, t * ppt, std::min(pairs, (t + 1) * ppt), first, ntasks});
    }
}

cudaError_t launch_fold(const int* fold, int nfold, double* E2, cudaStream_t s)
{
    if (nfold <= 0) return cudaSuccess;
    k_fold<<<(nfold + 127) / 128, 128, 0, s>>>(fold, nfold, E2);
    return cudaGetLastError();
}

cudaError_t launch_reduce(const double* E2, int nd, MonomerLists lists, double* mon, double* total,
                          double* scratch, cudaStream_t s)
{
    const int nbm = (lists.n_mon + kMonWarps - 1) / kMonWarps;
    // about 512 dimers per total block, at most kReduceBlocks blocks
    const int nbt = std::max(1, std::min(kReduceBlocks, (nd + 511) / 512));
    k_reduce<<<nbm + nbt, kRedThreads, 0, s>>>(E2, nd, lists, mon, nbm, nbt, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_total_merge<<<1, kRedThreads, 0, s>>>(scratch, nbt, total);
    return cudaGetLastError();
}

cudaError_t launch_check_finite(const double* x, long long n, int* flag, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    long long blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    k_check_finite<<<(int)blocks, 256, 0, s>>>(x, n, flag);
    return cudaGetLastError();
}

cudaError_t launch_check_finite4(const double* x, const int dims[4], const long long st[3], int* flag,
                                 cudaStream_t s)
{
    const long long n = (long long)dims[0] * dims[1] * dims[2] * dims[3];
    if (n <= 0) return cudaSuccess;
    long long blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    k_check_finite4<<<(int)blocks, 256, 0, s>>>(x, dims[0], dims[1], dims[2], dims[3], st[0], st[1], st[2], flag);
    return cudaGetLastError();
}

}  // namespace mcpt
