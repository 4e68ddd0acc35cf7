// k_td2.cu -- the dimer doubles iteration of Eq. (td2) on CUDA cores.
//
// Per dimer X-Y the iteration needs, besides (ia|jb), the Coulomb-block
// integrals (a a1|b b1), (i1 i|j1 j), (i1 i|b b1) and (a a1|j1 j): together
// most of the full MO transformation g[p][q][r][s] = (pq|rs) of the
// (XX|YY) block, which is formed whole by four quarter steps (k_qstep).  The
// exchange-type (ib|ja), needed only for E_K, takes four quarter steps of the
// (XY|YX) block over the needed MO ranges.  Every amplitude-dependent term of
// the equation is a contraction over a pair of indices, Out(r, c) +=
// alpha sum_k W(r, k) Z(k, c), with each operand a strided view of g, of the
// amplitudes or of a monomer matrix (k_pgemm); a Jacobi step then divides by
// the energy tensor (k_td2_update).  Each output tile is written by one CTA
// and every sum has a fixed order, so the results are deterministic.
#include "internal.h"

namespace mcpt {
namespace {

// ---------------------------------------------------------------- quarter steps
constexpr int kQM = 64, kQN = 32, kQK = 32, kQThreads = 256;

template <typename TI, typename TO>
__global__ void __launch_bounds__(kQThreads)
k_qstep(const QStep<TI, TO>* __restrict__ steps)
{
    const QStep<TI, TO> q = steps[blockIdx.z];
    const int m0 = blockIdx.x * kQM, n0 = blockIdx.y * kQN;
    if (m0 >= q.M || n0 >= q.N) return;
    __shared__ TO sIn[kQK][kQM + 1];           // [k][m]
    __shared__ TO sC[kQK][kQN];                // [k][n]
    const int tid = threadIdx.x, tm = tid & 31, tn = tid >> 5;   // outputs m = tm + 32 u, n = 4 tn + w
    TO acc[2][4];
#pragma unroll
    for (int u = 0; u < 2; u++)
#pragma unroll
        for (int w = 0; w < 4; w++) acc[u][w] = TO(0);
    for (int k0 = 0; k0 < q.K; k0 += kQK) {
        const int kn = min(kQK, q.K - k0);
        for (int e = tid; e < kQM * kQK; e += kQThreads) {
            const int mm = e / kQK, kk = e % kQK, m = m0 + mm, k = k0 + kk;
            TO x = TO(0);
            if (m < q.M && k < q.K) {
                const long long o = (long long)(m / (q.d1 * q.d2)) * q.st0 + (long long)((m / q.d2) % q.d1) * q.st1 +
                                    (long long)(m % q.d2) * q.st2 + k;
                x = (TO)q.in[o];
            }
            sIn[kk][mm] = x;
        }
        for (int e = tid; e < kQK * kQN; e += kQThreads) {
            const int kk = e / kQN, nn = e % kQN, k = k0 + kk, n = n0 + nn;
            sC[kk][nn] = (k < q.K && n < q.N) ? (TO)q.C[(long long)k * q.ldc + q.c0 + n] : TO(0);
        }
        __syncthreads();
        for (int k = 0; k < kn; k++) {
            const TO a0 = sIn[k][tm], a1 = sIn[k][tm + 32];
#pragma unroll
            for (int w = 0; w < 4; w++) {
                const TO c = sC[k][4 * tn + w];
                acc[0][w] = fma(a0, c, acc[0][w]);
                acc[1][w] = fma(a1, c, acc[1][w]);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 2; u++)
#pragma unroll
        for (int w = 0; w < 4; w++) {
            const int m = m0 + tm + 32 * u, n = n0 + 4 * tn + w;
            if (m < q.M && n < q.N) q.out[(long long)n * q.M + m] = acc[u][w];
        }
}

// ---------------------------------------------------------------- pair contractions
constexpr int kPT = 32, kPThreads = 256;

__device__ __forceinline__ long long ax_off(const PAxis& a, int x)
{
    return (long long)(x / a.n1) * a.s0 + (long long)(x % a.n1) * a.s1;
}

template <typename T>
__global__ void __launch_bounds__(kPThreads)
k_pgemm(const PGemm<T>* __restrict__ tabs)
{
    const PGemm<T> g = tabs[blockIdx.z];
    const int r0 = blockIdx.x * kPT, c0 = blockIdx.y * kPT;
    if (r0 >= g.R || c0 >= g.C) return;
    __shared__ T sW[kPT][kPT + 1];             // [k][r]
    __shared__ T sZ[kPT][kPT + 1];             // [k][c]
    __shared__ long long oWr[kPT], oZc[kPT], oOr[kPT], oOc[kPT], oWk[kPT], oZk[kPT];
    const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;  // outputs r = ty + 8 u, c = tx
    if (tid < kPT) {
        oWr[tid] = r0 + tid < g.R ? ax_off(g.wr, r0 + tid) : 0;
        oOr[tid] = r0 + tid < g.R ? ax_off(g.orow, r0 + tid) : 0;
    } else if (tid < 2 * kPT) {
        const int c = c0 + tid - kPT;
        oZc[tid - kPT] = c < g.C ? ax_off(g.zc, c) : 0;
        oOc[tid - kPT] = c < g.C ? ax_off(g.ocol, c) : 0;
    }
    T acc[4] = {T(0), T(0), T(0), T(0)};
    for (int k0 = 0; k0 < g.K; k0 += kPT) {
        const int kn = min(kPT, g.K - k0);
        __syncthreads();                       // offsets ready; previous chunk consumed
        if (tid < kPT) oWk[tid] = k0 + tid < g.K ? ax_off(g.wk, k0 + tid) : 0;
        else if (tid < 2 * kPT) oZk[tid - kPT] = k0 + tid - kPT < g.K ? ax_off(g.zk, k0 + tid - kPT) : 0;
        __syncthreads();
        for (int e = tid; e < kPT * kPT; e += kPThreads) {
            const int a = e / kPT, kk = e % kPT;                   // a: row (W) or column (Z) in the tile
            const bool okk = kk < kn;
            sW[kk][a] = (okk && r0 + a < g.R) ? g.W[oWr[a] + oWk[kk]] : T(0);
            sZ[kk][a] = (okk && c0 + a < g.C) ? g.Z[oZk[kk] + oZc[a]] : T(0);
        }
        __syncthreads();
        for (int k = 0; k < kn; k++) {
            const T z = sZ[k][tx];
#pragma unroll
            for (int u = 0; u < 4; u++) acc[u] = fma(sW[k][ty + 8 * u], z, acc[u]);
        }
    }
#pragma unroll
    for (int u = 0; u < 4; u++) {
        const int r = ty + 8 * u, c = tx;
        if (r0 + r < g.R && c0 + c < g.C) {
            T* o = g.out + oOr[r] + oOc[c];
            *o = fma(g.alpha, acc[u], *o);
        }
    }
}

// ---------------------------------------------------------------- elementwise parts
template <typename T>
__global__ void __launch_bounds__(256)
k_td2_init(const Td2Dim* __restrict__ dims, const long long* __restrict__ g_off, T* __restrict__ arena)
{
    const Td2Dim d = dims[blockIdx.y];
    const int vX = d.nX - d.oX, vY = d.nY - d.oY, mY = d.oY * vY, n = d.oX * vX * mY;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const int ia = e / mY, jb = e % mY;
    const int i = ia / vX, a = ia % vX, j = jb / vY, b = jb % vY;
    const T v = arena[g_off[blockIdx.y] + (((long long)i * d.nX + d.oX + a) * d.nY + j) * d.nY + d.oY + b];
    arena[d.V + e] = v;
    arena[d.R0 + e] = v;
    arena[d.Tc + e] = T(0);
}

__device__ __forceinline__ void max_bits(void* p, float x)
{
    atomicMax(static_cast<unsigned int*>(p), __float_as_uint(x));
}
__device__ __forceinline__ void max_bits(void* p, double x)
{
    atomicMax(static_cast<unsigned long long*>(p), (unsigned long long)__double_as_longlong(x));
}

template <typename T>
__global__ void __launch_bounds__(256)
k_td2_update(const Td2Dim* __restrict__ dims, const double* __restrict__ eps, T* __restrict__ arena,
             void* delta_bits)
{
    const Td2Dim d = dims[blockIdx.y];
    const int vX = d.nX - d.oX, vY = d.nY - d.oY, mY = d.oY * vY, n = d.oX * vX * mY;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    T dt = T(0);
    if (e < n) {
        const int ia = e / mY, jb = e % mY;
        const int i = ia / vX, a = ia % vX, j = jb / vY, b = jb % vY;
        const double den = eps[d.eX + i] + eps[d.eY + j] - eps[d.eX + d.oX + a] - eps[d.eY + d.oY + b];
        const T t = arena[d.R + e] / (T)den;
        dt = fabs(t - arena[d.Tc + e]);
        arena[d.Tc + e] = t;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) dt = fmax(dt, __shfl_xor_sync(0xffffffffu, dt, o));
    if ((threadIdx.x & 31) == 0 && dt > T(0)) max_bits(delta_bits, dt);
}

template <typename T>
__global__ void __launch_bounds__(256)
k_td2_energy(const Td2Dim* __restrict__ dims, const T* __restrict__ arena, double* __restrict__ E)
{
    const Td2Dim d = dims[blockIdx.x];
    const int vX = d.nX - d.oX, vY = d.nY - d.oY, mY = d.oY * vY, n = d.oX * vX * mY;
    double ej = 0.0, ek = 0.0;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const int ia = e / mY, jb = e % mY;
        const int i = ia / vX, a = ia % vX, j = jb / vY, b = jb % vY;
        const double t = (double)arena[d.Tc + e];
        ej += (double)arena[d.V + e] * t;
        ek += (double)arena[d.W + (((long long)i * vY + b) * d.oY + j) * vX + a] * t;
    }
    __shared__ double sj[256], sk[256];
    sj[threadIdx.x] = ej;
    sk[threadIdx.x] = ek;
    __syncthreads();
    for (int w = 128; w; w >>= 1) {
        if (threadIdx.x < w) {
            sj[threadIdx.x] += sj[threadIdx.x + w];
            sk[threadIdx.x] += sk[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        E[2 * blockIdx.x] = 4.0 * sj[0];
        E[2 * blockIdx.x + 1] = -2.0 * sk[0];
    }
}

}  // namespace

template <typename TI, typename TO>
cudaError_t launch_qstep(const QStep<TI, TO>* steps, int nd, int max_m, int max_n, cudaStream_t s)
{
    if (nd <= 0) return cudaSuccess;
    const dim3 grid((max_m + kQM - 1) / kQM, (max_n + kQN - 1) / kQN, nd);
    k_qstep<TI, TO><<<grid, kQThreads, 0, s>>>(steps);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_pgemm(const PGemm<T>* tabs, int nd, int max_r, int max_c, cudaStream_t s)
{
    if (nd <= 0 || max_r <= 0 || max_c <= 0) return cudaSuccess;     // no dimer has this term
    const dim3 grid((max_r + kPT - 1) / kPT, (max_c + kPT - 1) / kPT, nd);
    k_pgemm<T><<<grid, kPThreads, 0, s>>>(tabs);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_td2_init(const Td2Dim* dims, const long long* g_off, int nd, int max_m, T* arena, cudaStream_t s)
{
    if (nd <= 0) return cudaSuccess;
    k_td2_init<T><<<dim3((max_m + 255) / 256, nd), 256, 0, s>>>(dims, g_off, arena);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_td2_update(const Td2Dim* dims, int nd, int max_m, const double* eps, T* arena,
                              void* delta_bits, cudaStream_t s)
{
    if (nd <= 0) return cudaSuccess;
    k_td2_update<T><<<dim3((max_m + 255) / 256, nd), 256, 0, s>>>(dims, eps, arena, delta_bits);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_td2_energy(const Td2Dim* dims, int nd, const T* arena, double* E, cudaStream_t s)
{
    if (nd <= 0) return cudaSuccess;
    k_td2_energy<T><<<nd, 256, 0, s>>>(dims, arena, E);
    return cudaGetLastError();
}

template cudaError_t launch_qstep<double, float>(const QStep<double, float>*, int, int, int, cudaStream_t);
template cudaError_t launch_qstep<float, float>(const QStep<float, float>*, int, int, int, cudaStream_t);
template cudaError_t launch_qstep<double, double>(const QStep<double, double>*, int, int, int, cudaStream_t);
template cudaError_t launch_pgemm<float>(const PGemm<float>*, int, int, int, cudaStream_t);
template cudaError_t launch_pgemm<double>(const PGemm<double>*, int, int, int, cudaStream_t);
template cudaError_t launch_td2_init<float>(const Td2Dim*, const long long*, int, int, float*, cudaStream_t);
template cudaError_t launch_td2_init<double>(const Td2Dim*, const long long*, int, int, double*, cudaStream_t);
template cudaError_t launch_td2_update<float>(const Td2Dim*, int, int, const double*, float*, void*, cudaStream_t);
template cudaError_t launch_td2_update<double>(const Td2Dim*, int, int, const double*, double*, void*, cudaStream_t);
template cudaError_t launch_td2_energy<float>(const Td2Dim*, int, const float*, double*, cudaStream_t);
template cudaError_t launch_td2_energy<double>(const Td2Dim*, int, const double*, double*, cudaStream_t);

}  // namespace mcpt
