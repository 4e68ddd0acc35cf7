// noalloc.cu -- the FP64 dimer term for callers that must not allocate.
//
// The handle-based API allocates device memory (the dimer descriptors, the
// first-half scratch, result buffers).  Some callers cannot allow that: code
// that runs inside another framework's memory pool or budget, plug-in hooks
// that are handed their buffers and may not grow the process's footprint,
// and code paths that must not call cudaMalloc/cudaFree at all (those calls
// synchronise the device and can fail or stall at arbitrary points).  For
// them this file provides one entry point that computes a single dimer's
// {E_J, E_K} in FP64 from caller-owned device buffers, using a fixed
// file-scope device array for its only scratch -- the half-transformed
// integrals H.  That array is part of the library image: every GPU that
// loads the library holds it (8 MiB) until the process exits.
//
// The arithmetic is the FP64 form of the library's path: the occupied
// quarter transformations of Eq. (dp2e) (thread per output row, DFMA), then
// the virtual ones, the denominators of the energy tensor (Sec. II.C) and the
// energy sums of Eq. (ed2) (first Jacobi step, T = vD) and the exchange
// completion, reduced in a fixed order.
#include "mcpt.h"
#include "internal.h"

#include <cstdio>
#include <mutex>

namespace mcpt {
namespace {

// Scratch for H: 2 forms x (nX*nY rows) x (oX*oY) doubles.
constexpr long long kNoAllocScratchDoubles = 1ll << 20;   // 8 MiB
constexpr int kNoAllocMaxAO = 96;                          // shared-memory bound of the second half

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

constexpr int kHalfThreads = 128;
constexpr int kOB = 4;
constexpr int kFinThreads = 256;

// H[f][row = p1*n3 + p3][i*oY + j] = sum_{p0,p2} C_X[p0][i] C_Y[p2][j] E_f[p0][p1][p2][p3]
// with E_0 = A[mu][nu][lam][sig] (nX,nX,nY,nY) and E_1 = K[mu][lam][sig][nu] (nX,nY,nY,nX).
__global__ void __launch_bounds__(kHalfThreads)
k_noalloc_half(const double* __restrict__ A, const double* __restrict__ K, const double* __restrict__ CX,
               const double* __restrict__ CY, int nX, int nY, int oX, int oY, double* __restrict__ H)
{
    const int f = blockIdx.y;
    const int n0 = nX, n1 = f ? nY : nX, n2 = nY, n3 = f ? nX : nY;
    const int rows = n1 * n3;
    const int r = blockIdx.x * kHalfThreads + threadIdx.x;
    if (r >= rows) return;
    const int p1 = r / n3, p3 = r % n3;
    const long long s2 = n3, s1 = (long long)n2 * n3, s0 = (long long)n1 * n2 * n3;
    const double* __restrict__ E = (f ? K : A) + p1 * s1 + p3;
    const int ld = oX * oY;
    double* out = H + (long long)f * rows * ld + (long long)r * ld;
    for (int t0b = 0; t0b < oX; t0b += kOB) {
        for (int t2b = 0; t2b < oY; t2b += kOB) {
            double acc[kOB][kOB] = {};
            for (int p0 = 0; p0 < n0; p0++) {
                double F[kOB] = {};
                for (int p2 = 0; p2 < n2; p2++) {
                    const double e = __ldg(E + p0 * s0 + p2 * s2);
#pragma unroll
                    for (int t = 0; t < kOB; t++)
                        if (t2b + t < oY) F[t] = fma(__ldg(CY + p2 * nY + t2b + t), e, F[t]);
                }
#pragma unroll
                for (int a = 0; a < kOB; a++) {
                    const double w = t0b + a < oX ? __ldg(CX + p0 * nX + t0b + a) : 0.0;
#pragma unroll
                    for (int t = 0; t < kOB; t++) acc[a][t] = fma(w, F[t], acc[a][t]);
                }
            }
#pragma unroll
            for (int a = 0; a < kOB; a++)
#pragma unroll
                for (int t = 0; t < kOB; t++)
                    if (t0b + a < oX && t2b + t < oY) out[(t0b + a) * oY + t2b + t] = acc[a][t];
        }
    }
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// One block: virtual quarter transformations per occupied pair, FP64
// denominators, E_J = 4 sum v^2 D, E_K = -2 sum v v' D.
__global__ void __launch_bounds__(kFinThreads)
k_noalloc_finish(const double* __restrict__ H, const double* __restrict__ CX, const double* __restrict__ eX,
                 const double* __restrict__ CY, const double* __restrict__ eY, int nX, int nY, int oX, int oY,
                 double* __restrict__ E2)
{
    const int vX = nX - oX, vY = nY - oY, rows = nX * nY, ld = oX * oY;
    const double* H0 = H;
    const double* H1 = H + (long long)rows * ld;
    extern __shared__ double sm[];
    double* S = sm;                                          // [rows]
    double* Tm = S + rows;                                   // [max(nX*vY, nY*vX)]
    double* VA = Tm + (nX * vY > nY * vX ? nX * vY : nY * vX);
    const int tid = threadIdx.x;
    double ej = 0.0, ek = 0.0;
    for (int i = 0; i < oX; i++) {
        for (int j = 0; j < oY; j++) {
            const int col = i * oY + j;
            const double eij = eX[i] + eY[j];
            for (int k = tid; k < rows; k += kFinThreads) S[k] = H0[(long long)k * ld + col];
            __syncthreads();
            for (int k = tid; k < nX * vY; k += kFinThreads) {
                const int nu = k / vY, b = k % vY;
                double acc = 0.0;
                for (int sg = 0; sg < nY; sg++) acc = fma(S[nu * nY + sg], CY[sg * nY + oY + b], acc);
                Tm[k] = acc;
            }
            __syncthreads();
            for (int k = tid; k < vX * vY; k += kFinThreads) {
                const int a = k / vY, b = k % vY;
                double acc = 0.0;
                for (int nu = 0; nu < nX; nu++) acc = fma(CX[nu * nX + oX + a], Tm[nu * vY + b], acc);
                VA[k] = acc;
            }
            __syncthreads();
            for (int k = tid; k < rows; k += kFinThreads) S[k] = H1[(long long)k * ld + col];
            __syncthreads();
            for (int k = tid; k < nY * vX; k += kFinThreads) {
                const int lam = k / vX, a = k % vX;
                double acc = 0.0;
                for (int nu = 0; nu < nX; nu++) acc = fma(S[lam * nX + nu], CX[nu * nX + oX + a], acc);
                Tm[k] = acc;
            }
            __syncthreads();
            for (int k = tid; k < vX * vY; k += kFinThreads) {
                const int a = k / vY, b = k % vY;
                double vk = 0.0;
                for (int lam = 0; lam < nY; lam++) vk = fma(CY[lam * nY + oY + b], Tm[lam * vX + a], vk);
                const double D = 1.0 / (eij - (eX[oX + a] + eY[oY + b]));
                ej = fma(VA[k] * VA[k], D, ej);
                ek = fma(VA[k] * vk, D, ek);
            }
            __syncthreads();
        }
    }
    __shared__ double red[2][kFinThreads / 32];
    ej = warp_sum(ej);
    ek = warp_sum(ek);
    if ((tid & 31) == 0) { red[0][tid >> 5] = ej; red[1][tid >> 5] = ek; }
    __syncthreads();
    if (tid == 0) {
        double sj = 0.0, sk = 0.0;
        for (int w = 0; w < kFinThreads / 32; w++) { sj += red[0][w]; sk += red[1][w]; }
        E2[0] = 4.0 * sj;
        E2[1] = -2.0 * sk;
    }
}

// Device address of the scratch array, looked up once per device with that
// device current (a host-side reference to the symbol is not a device address).
constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_scratch_ptr[kMaxDevices] = {};

cudaError_t scratch_for_current_device(double** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(k_noalloc_finish, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(3 * kNoAllocMaxAO * kNoAllocMaxAO * sizeof(double)));
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

mcpt_status noalloc_fail(mcpt_status st, const char* fmt, long long a = 0, long long b = 0)
{
    char buf[256];
    snprintf(buf, sizeof buf, fmt, a, b);
    set_thread_error(buf);
    return st;
}

}  // namespace
}  // namespace mcpt

using namespace mcpt;

extern "C" mcpt_status mcpt_dimer_fp64_noalloc(const double* A, const double* K, const double* CX,
                                               const double* epsX, int nX, int oX, const double* CY,
                                               const double* epsY, int nY, int oY, double* E2, void* stream)
{
    if (!A || !K || !CX || !epsX || !CY || !epsY || !E2)
        return noalloc_fail(MCPT_EINVAL, "mcpt_dimer_fp64_noalloc: NULL pointer argument");
    if (nX < 2 || nY < 2 || nX > kNoAllocMaxAO || nY > kNoAllocMaxAO)
        return noalloc_fail(MCPT_EINVAL, "mcpt_dimer_fp64_noalloc: AO counts (%lld, %lld) outside [2, 96]", nX, nY);
    if (oX < 1 || oX > nX - 1 || oY < 1 || oY > nY - 1)
        return noalloc_fail(MCPT_EINVAL, "mcpt_dimer_fp64_noalloc: nocc (%lld, %lld) outside [1, nao-1]", oX, oY);
    const long long need = 2ll * nX * nY * oX * oY;
    if (need > kNoAllocScratchDoubles)
        return noalloc_fail(MCPT_EINVAL,
                            "mcpt_dimer_fp64_noalloc: needs %lld doubles of scratch, the fixed maximum is %lld "
                            "(2*nX*nY*nocc_X*nocc_Y <= 1048576)",
                            need, kNoAllocScratchDoubles);
    double* H = nullptr;
    cudaError_t e = scratch_for_current_device(&H);
    if (e != cudaSuccess)
        return noalloc_fail(MCPT_ECUDA, "mcpt_dimer_fp64_noalloc: scratch set-up failed (CUDA error %lld)", (long long)e);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int rows = nX * nY;
    dim3 grid((rows + kHalfThreads - 1) / kHalfThreads, 2);
    k_noalloc_half<<<grid, kHalfThreads, 0, s>>>(A, K, CX, CY, nX, nY, oX, oY, H);
    const int nmax = nX > nY ? nX : nY;
    const size_t smem = 3 * (size_t)nmax * nmax * sizeof(double);
    k_noalloc_finish<<<1, kFinThreads, smem, s>>>(H, CX, epsX, CY, epsY, nX, nY, oX, oY, E2);
    e = cudaGetLastError();
    if (e != cudaSuccess)
        return noalloc_fail(MCPT_ECUDA, "mcpt_dimer_fp64_noalloc: launch failed (CUDA error %lld)", (long long)e);
    set_thread_error("");   // a successful call leaves no stale message for mcpt_last_error(NULL)
    return MCPT_OK;
}
