// k_finish.cu -- second half of the dimer transformation, the FP64 energy
// epilogue, and the per-monomer accumulation.
//
// For each occupied pair (i, j) the first half left two nX x nY matrices
//   H_0[(nu,sig)][(i,j)]   (nu in X, sig in Y)   from the (XX|YY) block
//   H_1[(lam,nu)][(i,j)]   (lam in Y, nu in X)   from the (XY|YX) block
// and the virtual quarter transformations of Eq. (dp2e) finish them:
//   (i a|j b) = sum_nu C_X[nu][a] sum_sig H_0[nu][sig] C_Y[sig][b]
//   (i b|j a) = sum_lam C_Y[lam][b] sum_nu H_1[lam][nu] C_X[nu][a]
// Then, in FP64 (Sec. II.C energy tensor, Eq. (ed2) with T = vD):
//   D = 1/(e_i + e_j - e_a - e_b),  E_J += 4 (ia|jb)^2 D,  E_K += -2 (ia|jb)(ib|ja) D.
// GB300's FP64 unit is small, so D is an FP32 reciprocal refined by Newton
// steps in FP64 (convert.h) rather than a full FP64 division -- two for the
// FP64 form (full FP64 accuracy), one for the mixed forms (relative error
// ~1.4e-14, far below their transform error) -- and the FP32 -> FP64 widening
// of the mixed forms' integrals runs on integer pipes.
// One CTA owns one dimer, so the per-dimer energies come out of a fixed-order
// block reduction: deterministic run to run, no atomics.
#include "internal.h"
#include "convert.h"

namespace mcpt {
namespace {

constexpr int kFinThreads = 256;

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double to_f64(double x) { return x; }
__device__ __forceinline__ double to_f64(float x) { return f64_from_f32(x); }   // integer pipes

// T: arithmetic type of the second half (double for the FP64 form, float for
// the mixed forms) -- also the type of the coefficient pool C and of H.
// Per occupied pair (i, j):
//   TmA[nu][b] = sum_sig H0[nu][sig] C_Y[sig][b];   VA[a][b] = sum_nu C_X[nu][a] TmA[nu][b]
//   TmK[lam][a] = sum_nu H1[lam][nu] C_X[nu][a];    VK[b][a] = sum_lam C_Y[lam][b] TmK[lam][a]
// then one FP64 denominator per (a, b) feeds both energy sums.
template <typename T>
__global__ void __launch_bounds__(kFinThreads)
k_finish(const DimerDesc* __restrict__ dd, const T* __restrict__ C, const double* __restrict__ Epool,
         const T* __restrict__ H, double* __restrict__ E2)
{
    const DimerDesc& d = dd[blockIdx.x];
    const int nX = d.nX, nY = d.nY, oX = d.oX, oY = d.oY;
    const int vX = nX - oX, vY = nY - oY;
    const int rows = nX * nY, pairs = oX * oY;
    const T* CX = C + d.cX;
    const T* CY = C + d.cY;
    const double* eX = Epool + d.eX;
    const double* eY = Epool + d.eY;
    const T* H0 = H + d.h_off;
    const T* H1 = H + d.h_off + (long long)pairs * rows;

    extern __shared__ __align__(16) unsigned char smraw[];
    T* S = reinterpret_cast<T*>(smraw);                 // [rows]
    T* Tm = S + rows;                                   // [max(nX*vY, nY*vX)]
    T* VA = Tm + (nX * vY > nY * vX ? nX * vY : nY * vX);  // [vX][vY]

    double ej = 0.0, ek = 0.0;
    const int tid = threadIdx.x;
    for (int i = 0; i < oX; i++) {
        for (int j = 0; j < oY; j++) {
            const int col = i * oY + j;
            const double eij = eX[i] + eY[j];
            // ---- (i a|j b) from H_0
            for (int k = tid; k < rows; k += kFinThreads) S[k] = H0[(long long)col * rows + k];
            __syncthreads();
            for (int k = tid; k < nX * vY; k += kFinThreads) {
                const int nu = k / vY, b = k % vY;
                const T* s = S + nu * nY;
                T acc = 0;
                for (int sg = 0; sg < nY; sg++) acc = fma(s[sg], __ldg(CY + sg * nY + oY + b), acc);
                Tm[k] = acc;
            }
            __syncthreads();
            for (int k = tid; k < vX * vY; k += kFinThreads) {
                const int a = k / vY, b = k % vY;
                T acc = 0;
                for (int nu = 0; nu < nX; nu++) acc = fma(__ldg(CX + nu * nX + oX + a), Tm[nu * vY + b], acc);
                VA[k] = acc;
            }
            __syncthreads();
            // ---- (i b|j a) from H_1
            for (int k = tid; k < rows; k += kFinThreads) S[k] = H1[(long long)col * rows + k];
            __syncthreads();
            for (int k = tid; k < nY * vX; k += kFinThreads) {
                const int lam = k / vX, a = k % vX;
                const T* s = S + lam * nX;
                T acc = 0;
                for (int nu = 0; nu < nX; nu++) acc = fma(s[nu], __ldg(CX + nu * nX + oX + a), acc);
                Tm[k] = acc;
            }
            __syncthreads();
            // ---- energies: one denominator per (a, b)
            for (int k = tid; k < vX * vY; k += kFinThreads) {
                const int a = k / vY, b = k % vY;
                T acc = 0;
                for (int lam = 0; lam < nY; lam++) acc = fma(__ldg(CY + lam * nY + oY + b), Tm[lam * vX + a], acc);
                const double va = to_f64(VA[k]);
                const double vk = to_f64(acc);
                const double D = rcp_f64<sizeof(T) == 8 ? 2 : 1>(eij - (eX[oX + a] + eY[oY + b]));
                ej = fma(va * va, D, ej);
                ek = fma(va * vk, D, ek);
            }
            __syncthreads();
        }
    }
    // fixed-order block reduction
    __shared__ double red[2][kFinThreads / 32];
    ej = warp_sum(ej);
    ek = warp_sum(ek);
    if ((tid & 31) == 0) { red[0][tid >> 5] = ej; red[1][tid >> 5] = ek; }
    __syncthreads();
    if (tid == 0) {
        double sj = 0.0, sk = 0.0;
        for (int w = 0; w < kFinThreads / 32; w++) { sj += red[0][w]; sk += red[1][w]; }
        E2[2 * d.slot + 0] = 4.0 * sj;
        E2[2 * d.slot + 1] = -2.0 * sk;
    }
}

// ---------------------------------------------------------------------------
// Monomers of at most 32 AO: one warp per occupied pair (i, j), one lane per
// virtual orbital.  For pair (i, j):
//   lane b:  tm[nu] = sum_sig H0[nu][sig] C_Y[sig][b]        (C_Y column b in registers)
//            VA[a][b] = sum_nu C_X[nu][a] tm[nu]             (C_X rows broadcast from smem)
//   lane a:  tk[lam] = sum_nu H1[lam][nu] C_X[nu][a]
//            VK[b][a] = sum_lam C_Y[lam][b] tk[lam], and with VA[a][b] (transposed
//            through smem) and D from the precomputed e_a + e_b the two FP64 sums.
// The H slices are contiguous (pair-major), read with coalesced loads into a
// zero-padded 32 x 32 tile.  Per-lane sums reduce in a fixed order.
constexpr int kW32Warps = 4;

template <typename T>
__global__ void __launch_bounds__(kW32Warps * 32)
k_finish_w32(const DimerDesc* __restrict__ dd, const T* __restrict__ C, const double* __restrict__ Epool,
             const T* __restrict__ H, double* __restrict__ E2)
{
    const DimerDesc& d = dd[blockIdx.x];
    const int nX = d.nX, nY = d.nY, oX = d.oX, oY = d.oY;
    const int vX = nX - oX, vY = nY - oY;
    const int rows = nX * nY, pairs = oX * oY;
    const T* CX = C + d.cX;
    const T* CY = C + d.cY;
    const double* eX = Epool + d.eX;
    const double* eY = Epool + d.eY;
    const T* H0 = H + d.h_off;
    const T* H1 = H + d.h_off + (long long)pairs * rows;

    extern __shared__ __align__(16) unsigned char smraw[];
    double* eab = reinterpret_cast<double*>(smraw);          // [32][32]: e_a + e_b
    T* CXT = reinterpret_cast<T*>(eab + 32 * 32);             // [a][nu], zero padded
    T* CYT = CXT + 32 * 32;                                   // [b][sig]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T* S = CYT + 32 * 32 + warp * (32 * 32 + 32 * 33);        // [32][32] integral slice
    T* VAs = S + 32 * 32;                                     // [a][b], stride 33

    for (int k = threadIdx.x; k < 32 * 32; k += kW32Warps * 32) {
        const int a = k >> 5, m = k & 31;
        CXT[k] = (a < vX && m < nX) ? CX[m * nX + oX + a] : T(0);
        CYT[k] = (a < vY && m < nY) ? CY[m * nY + oY + a] : T(0);
        eab[k] = (a < vX && m < vY) ? eX[oX + a] + eY[oY + m] : 0.0;
    }
    __syncthreads();

    double ej = 0.0, ek = 0.0;
    for (int pr = warp; pr < pairs; pr += kW32Warps) {
        const int i = pr / oY, j = pr % oY;
        const double eij = eX[i] + eY[j];
        // ---- (i a|j b): S[nu][sig] = H0 slice
        const T* h0 = H0 + (long long)pr * rows;
        for (int k = lane; k < 32 * 32; k += 32) {
            const int r = k >> 5, c = k & 31;
            S[k] = (r < nX && c < nY) ? h0[r * nY + c] : T(0);
        }
        __syncwarp();
        {
            T cy[32], tm[32];
#pragma unroll
            for (int m = 0; m < 32; m++) cy[m] = CYT[lane * 32 + m];
#pragma unroll
            for (int nu = 0; nu < 32; nu++) {
                T acc = 0;
#pragma unroll
                for (int m = 0; m < 32; m++) acc = fma(S[nu * 32 + m], cy[m], acc);
                tm[nu] = acc;
            }
#pragma unroll 4
            for (int a = 0; a < 32; a++) {
                T acc = 0;
#pragma unroll
                for (int nu = 0; nu < 32; nu++) acc = fma(CXT[a * 32 + nu], tm[nu], acc);
                VAs[a * 33 + lane] = acc;
            }
        }
        __syncwarp();
        // ---- (i b|j a): S[lam][nu] = H1 slice
        const T* h1 = H1 + (long long)pr * rows;
        for (int k = lane; k < 32 * 32; k += 32) {
            const int r = k >> 5, c = k & 31;
            S[k] = (r < nY && c < nX) ? h1[r * nX + c] : T(0);
        }
        __syncwarp();
        {
            T cx[32], tk[32];
#pragma unroll
            for (int m = 0; m < 32; m++) cx[m] = CXT[lane * 32 + m];
#pragma unroll
            for (int lam = 0; lam < 32; lam++) {
                T acc = 0;
#pragma unroll
                for (int m = 0; m < 32; m++) acc = fma(S[lam * 32 + m], cx[m], acc);
                tk[lam] = acc;
            }
            const bool live = lane < vX;
#pragma unroll 2
            for (int b = 0; b < 32; b++) {
                T vk = 0;
#pragma unroll
                for (int lam = 0; lam < 32; lam++) vk = fma(CYT[b * 32 + lam], tk[lam], vk);
                if (live && b < vY) {
                    const double va = to_f64(VAs[lane * 33 + b]);
                    const double D = rcp_f64<sizeof(T) == 8 ? 2 : 1>(eij - eab[lane * 32 + b]);
                    ej = fma(va * va, D, ej);
                    ek = fma(va * to_f64(vk), D, ek);
                }
            }
        }
        __syncwarp();
    }
    __shared__ double red[2][kW32Warps];
    ej = warp_sum(ej);
    ek = warp_sum(ek);
    if (lane == 0) { red[0][warp] = ej; red[1][warp] = ek; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sj = 0.0, sk = 0.0;
        for (int w = 0; w < kW32Warps; w++) { sj += red[0][w]; sk += red[1][w]; }
        E2[2 * d.slot + 0] = 4.0 * sj;
        E2[2 * d.slot + 1] = -2.0 * sk;
    }
}

template <typename T>
cudaError_t launch_finish(const DimerDesc* d_desc, int nd, int max_ao, const T* C, const double* Epool,
                          const T* H, double* E2, cudaStream_t s)
{
    if (nd <= 0) return cudaSuccess;
    if (max_ao <= 32) {
        const size_t smem = 32 * 32 * sizeof(double) + 2 * 32 * 32 * sizeof(T) +
                            kW32Warps * (32 * 32 + 32 * 33) * sizeof(T);
        cudaError_t e = cudaFuncSetAttribute(k_finish_w32<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_finish_w32<T><<<nd, kW32Warps * 32, smem, s>>>(d_desc, C, Epool, H, E2);
        return cudaGetLastError();
    }
    const size_t smem = (size_t)3 * max_ao * max_ao * sizeof(T);
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k_finish<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_finish<T><<<nd, kFinThreads, smem, s>>>(d_desc, C, Epool, H, E2);
    return cudaGetLastError();
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

// Blocks [0, nbm): one thread per monomer sums half of each of its dimers'
// terms in ascending dimer order.  Last block: lattice totals from a fixed
// partition of the dimer list into kRedThreads contiguous chunks (Neumaier
// within a chunk), merged by a fixed pairwise tree.  Long dependent FP64
// chains are slow on GB300, so no thread walks more than a chunk.
__global__ void __launch_bounds__(kRedThreads)
k_reduce(const double* __restrict__ E2, int nd, MonomerLists L, double* __restrict__ mon,
         double* __restrict__ total)
{
    const int nbm = (L.n_mon + kRedThreads - 1) / kRedThreads;
    if ((int)blockIdx.x < nbm) {
        const int m = blockIdx.x * kRedThreads + threadIdx.x;
        if (m >= L.n_mon) return;
        double sj = 0, cj = 0, sk = 0, ck = 0;
        for (int k = L.start[m]; k < L.start[m + 1]; k++) {
            const int dslot = L.list[k];
            neumaier_add(sj, cj, 0.5 * E2[2 * dslot]);
            neumaier_add(sk, ck, 0.5 * E2[2 * dslot + 1]);
        }
        mon[m] = sj + cj;
        mon[L.n_mon + m] = sk + ck;
        return;
    }
    __shared__ double part[4][kRedThreads];
    const int t = threadIdx.x;
    const int chunk = (nd + kRedThreads - 1) / kRedThreads;
    const int lo = t * chunk, hi = min(nd, lo + chunk);
    double sj = 0, cj = 0, sk = 0, ck = 0;
    for (int k = lo; k < hi; k++) {
        neumaier_add(sj, cj, E2[2 * k]);
        neumaier_add(sk, ck, E2[2 * k + 1]);
    }
    part[0][t] = sj; part[1][t] = cj; part[2][t] = sk; part[3][t] = ck;
    __syncthreads();
    // pairwise tree over the chunk partials, fixed pairing: (sum, compensation)
    // pairs are merged with Knuth's TwoSum so the rounding of each merge is kept
    for (int w = kRedThreads / 2; w > 0; w >>= 1) {
        if (t < w) {
#pragma unroll
            for (int f = 0; f < 4; f += 2) {
                const double a = part[f][t], b = part[f][t + w];
                const double s = a + b;
                const double bp = s - a;
                const double err = (a - (s - bp)) + (b - bp);
                part[f][t] = s;
                part[f + 1][t] = part[f + 1][t] + part[f + 1][t + w] + err;
            }
        }
        __syncthreads();
    }
    if (t == 0) {
        total[0] = part[0][0] + part[1][0];
        total[1] = part[2][0] + part[3][0];
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
                               const double* Epool, const double* H, double* E2, cudaStream_t s)
{
    return launch_finish<double>(d_desc, nd, max_ao, Cpool, Epool, H, E2, s);
}

cudaError_t launch_finish_fp32(const DimerDesc* d_desc, int nd, int max_ao, const float* Cf,
                               const double* Epool, const float* H, double* E2, cudaStream_t s)
{
    return launch_finish<float>(d_desc, nd, max_ao, Cf, Epool, H, E2, s);
}

cudaError_t launch_reduce(const double* E2, int nd, MonomerLists lists, double* mon, double* total,
                          cudaStream_t s)
{
    const int nbm = (lists.n_mon + kRedThreads - 1) / kRedThreads;
    k_reduce<<<nbm + 1, kRedThreads, 0, s>>>(E2, nd, lists, mon, total);
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
