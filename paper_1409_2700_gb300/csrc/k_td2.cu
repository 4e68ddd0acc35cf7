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
#include "convert.h"

namespace mcpt {
namespace {

// FP64 -> T; to FP32 on the integer pipes (a cvt.f32.f64 would issue on the
// small FP64 unit for every element read).
template <typename T>
__device__ __forceinline__ T from_f64(double x);
template <>
__device__ __forceinline__ float from_f64<float>(double x) { return f32_from_f64(x); }
template <>
__device__ __forceinline__ double from_f64<double>(double x) { return x; }
// An element of a quarter step's input (FP64 AO block or the previous step's T) as TO.
template <typename TO>
__device__ __forceinline__ TO to_out(double x) { return from_f64<TO>(x); }
template <typename TO>
__device__ __forceinline__ TO to_out(float x) { return (TO)x; }

template <typename T>
__device__ __forceinline__ void ld4(const T* p, T (&x)[4])
{
    if constexpr (sizeof(T) == 4) {
        const float4 v = *reinterpret_cast<const float4*>(p);
        x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
    } else {
        const double2 a = *reinterpret_cast<const double2*>(p), b = *reinterpret_cast<const double2*>(p + 2);
        x[0] = a.x; x[1] = a.y; x[2] = b.x; x[3] = b.y;
    }
}

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
    __shared__ __align__(16) TO sC[kQK][kQN];  // [k][n]
    __shared__ long long rowOff[kQM];          // In(m0 + mm, 0)
    const int tid = threadIdx.x, tm = tid & 31, tn = tid >> 5;   // outputs m = tm + 32 u, n = 4 tn + w
    if (tid < kQM) {
        const int m = m0 + tid;
        rowOff[tid] = m < q.M ? (long long)(m / (q.d1 * q.d2)) * q.st0 + (long long)((m / q.d2) % q.d1) * q.st1 +
                                    (long long)(m % q.d2) * q.st2
                              : 0;
    }
    TO acc[2][4];
#pragma unroll
    for (int u = 0; u < 2; u++)
#pragma unroll
        for (int w = 0; w < 4; w++) acc[u][w] = TO(0);
    for (int k0 = 0; k0 < q.K; k0 += kQK) {
        const int kn = min(kQK, q.K - k0);
        __syncthreads();                       // row offsets ready; previous chunk consumed
        {
            // every load of the chunk first (independent, in flight together),
            // then the conversions and the shared-memory stores
            constexpr int kPerIn = kQM * kQK / kQThreads, kPerC = kQK * kQN / kQThreads;
            static_assert(kPerIn * kQThreads == kQM * kQK && kPerC * kQThreads == kQK * kQN, "whole passes");
            TI vin[kPerIn];
            double vc[kPerC];
#pragma unroll
            for (int t = 0; t < kPerIn; t++) {
                const int e = tid + t * kQThreads, mm = e / kQK, k = k0 + e % kQK;
                vin[t] = (m0 + mm < q.M && k < q.K) ? q.in[rowOff[mm] + k] : TI(0);
            }
#pragma unroll
            for (int t = 0; t < kPerC; t++) {
                const int e = tid + t * kQThreads, k = k0 + e / kQN, n = n0 + e % kQN;
                vc[t] = (k < q.K && n < q.N) ? q.C[(long long)k * q.ldc + q.c0 + n] : 0.0;
            }
#pragma unroll
            for (int t = 0; t < kPerIn; t++) {
                const int e = tid + t * kQThreads;
                sIn[e % kQK][e / kQK] = to_out<TO>(vin[t]);
            }
#pragma unroll
            for (int t = 0; t < kPerC; t++) {
                const int e = tid + t * kQThreads;
                sC[e / kQN][e % kQN] = from_f64<TO>(vc[t]);
            }
        }
        __syncthreads();
        for (int k = 0; k < kn; k++) {
            const TO a0 = sIn[k][tm], a1 = sIn[k][tm + 32];
            TO c[4];
            ld4(&sC[k][4 * tn], c);
#pragma unroll
            for (int w = 0; w < 4; w++) {
                acc[0][w] = fma(a0, c[w], acc[0][w]);
                acc[1][w] = fma(a1, c[w], acc[1][w]);
            }
        }
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
constexpr int kPR = 64, kPC = 32, kPK = 32, kPThreads = 256;

__device__ __forceinline__ long long ax_off(const PAxis& a, int x)
{
    return (long long)(x / a.n1) * a.s0 + (long long)(x % a.n1) * a.s1;
}

// 64 x 32 output tile; thread (tr, tc) holds rows 4 tr .. 4 tr + 3 and
// columns 2 tc, 2 tc + 1: per k six shared loads (the four row values are
// broadcast within half-warps) feed 8 FMAs.  The staged operands are kept
// [row][k] with an odd stride, so that the gathers (consecutive threads
// along k, usually the operand's contiguous index) store without bank
// conflicts.  Operand offsets are tabulated per tile (rows, columns) and
// per chunk (k), so the gathers do no division.
template <typename T>
__global__ void __launch_bounds__(kPThreads)
k_pgemm(const PGemm<T>* __restrict__ tabs)
{
    const PGemm<T> g = tabs[blockIdx.z];
    const int r0 = blockIdx.x * kPR, c0 = blockIdx.y * kPC;
    if (r0 >= g.R || c0 >= g.C) return;
    __shared__ T sW[kPR][kPK + 1];             // [r][k]
    __shared__ T sZ[kPC][kPK + 1];             // [c][k]
    __shared__ long long oWr[kPR], oOr[kPR], oZc[kPC], oOc[kPC], oWk[kPK], oZk[kPK];
    const int tid = threadIdx.x, tr = tid >> 4, tc = tid & 15;
    if (tid < kPR) {
        oWr[tid] = r0 + tid < g.R ? ax_off(g.wr, r0 + tid) : 0;
        oOr[tid] = r0 + tid < g.R ? ax_off(g.orow, r0 + tid) : 0;
    } else if (tid < kPR + kPC) {
        const int c = c0 + tid - kPR;
        oZc[tid - kPR] = c < g.C ? ax_off(g.zc, c) : 0;
        oOc[tid - kPR] = c < g.C ? ax_off(g.ocol, c) : 0;
    }
    T acc[4][2];
#pragma unroll
    for (int u = 0; u < 4; u++) acc[u][0] = acc[u][1] = T(0);
    for (int k0 = 0; k0 < g.K; k0 += kPK) {
        const int kn = min(kPK, g.K - k0);
        __syncthreads();                       // offsets ready; previous chunk consumed
        if (tid < kPK) oWk[tid] = k0 + tid < g.K ? ax_off(g.wk, k0 + tid) : 0;
        else if (tid < 2 * kPK) oZk[tid - kPK] = k0 + tid - kPK < g.K ? ax_off(g.zk, k0 + tid - kPK) : 0;
        __syncthreads();
        {
            // every gather of the chunk first (independent, in flight together), then the stores
            constexpr int kPerW = kPR * kPK / kPThreads, kPerZ = kPC * kPK / kPThreads;
            static_assert(kPerW * kPThreads == kPR * kPK && kPerZ * kPThreads == kPC * kPK, "whole passes");
            T vw[kPerW], vz[kPerZ];
#pragma unroll
            for (int t = 0; t < kPerW; t++) {
                const int e = tid + t * kPThreads, a = e / kPK, kk = e % kPK;   // W row a of the tile
                vw[t] = (kk < kn && r0 + a < g.R) ? g.W[oWr[a] + oWk[kk]] : T(0);
            }
#pragma unroll
            for (int t = 0; t < kPerZ; t++) {
                const int e = tid + t * kPThreads, a = e / kPK, kk = e % kPK;   // Z column a of the tile
                vz[t] = (kk < kn && c0 + a < g.C) ? g.Z[oZk[kk] + oZc[a]] : T(0);
            }
#pragma unroll
            for (int t = 0; t < kPerW; t++) {
                const int e = tid + t * kPThreads;
                sW[e / kPK][e % kPK] = vw[t];
            }
#pragma unroll
            for (int t = 0; t < kPerZ; t++) {
                const int e = tid + t * kPThreads;
                sZ[e / kPK][e % kPK] = vz[t];
            }
        }
        __syncthreads();
        for (int k = 0; k < kn; k++) {
            T w[4];
#pragma unroll
            for (int u = 0; u < 4; u++) w[u] = sW[4 * tr + u][k];
            const T z0 = sZ[2 * tc][k], z1 = sZ[2 * tc + 1][k];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                acc[u][0] = fma(w[u], z0, acc[u][0]);
                acc[u][1] = fma(w[u], z1, acc[u][1]);
            }
        }
    }
#pragma unroll
    for (int u = 0; u < 4; u++)
#pragma unroll
        for (int v = 0; v < 2; v++) {
            const int r = 4 * tr + u, c = 2 * tc + v;
            if (r0 + r < g.R && c0 + c < g.C) {
                T* o = g.out + oOr[r] + oOc[c];
                *o = fma(g.alpha, acc[u][v], *o);
            }
        }
}

// The particle ladder with its integrals packed once per dimer, k-major, into
// a dense matrix Wt[(a1,b1)][(a,b)] = (a a1|b b1) (row length ld, a multiple
// of 4, the padding zero), constant over the steps: 64 x 32 output tiles, the
// W chunk (32 k-rows x 64 output rows) streamed by 16-byte cp.async straight
// into a [k][r] layout (two buffers: the next chunk in flight while the
// current one is summed), the amplitudes gathered into [k][c] through their
// offset tables; per k one 4-wide and one 2-wide shared load feed 8 FMAs.
template <typename T>
__global__ void __launch_bounds__(256)
k_pack_ladder(const Td2Dim* __restrict__ dims, const long long* __restrict__ g_off,
              const long long* __restrict__ wd_off, T* __restrict__ arena)
{
    const Td2Dim d = dims[blockIdx.y];
    const int vX = d.nX - d.oX, vY = d.nY - d.oY, n = vX * vY, ld = (n + 3) / 4 * 4;
    const int row = blockIdx.x;                // (a, b)
    if (row >= n) return;
    const int a1 = row / vY, b1 = row % vY;    // row of Wt: (a1, b1); column (a, b)
    const T* g = arena + g_off[blockIdx.y];
    T* w = arena + wd_off[blockIdx.y] + (long long)row * ld;
    for (int c = threadIdx.x; c < ld; c += blockDim.x) {
        T x = T(0);
        if (c < n) {
            const int a = c / vY, b = c % vY;
            x = g[(((long long)(d.oX + a) * d.nX + d.oX + a1) * d.nY + d.oY + b) * d.nY + d.oY + b1];
        }
        w[c] = x;
    }
}

constexpr int kLS = kPR + 4;                   // staged W row stride [k][r] (16-byte aligned rows)
constexpr int kZS = kPC + 2;                   // staged Z row stride [k][c] (8-byte aligned pairs)

// Rows k0 .. k0 + kPK of Wt, columns r0 .. r0 + kPR, into sW[k][r]; rows
// beyond K and columns beyond ld are zero-filled without reading.
template <typename T>
__device__ __forceinline__ void stage_w(T (*sW)[kLS], const T* __restrict__ W, int ld, int K, int r0, int k0,
                                        int tid)
{
    constexpr int kV = 16 / sizeof(T);         // elements per 16-byte copy
    constexpr int kG = kPR / kV;               // copies per k-row
    for (int e = tid; e < kPK * kG; e += kPThreads) {
        const int kk = e / kG, c = (e % kG) * kV, k = k0 + kk, r = r0 + c;
        const bool ok = k < K && r < ld;
        const T* src = ok ? W + (long long)k * ld + r : W;
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"((unsigned)__cvta_generic_to_shared(&sW[kk][c])),
                     "l"(src), "r"(ok ? 16 : 0)
                     : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

template <typename T>
__device__ __forceinline__ void ld2(const T* p, T& x0, T& x1)
{
    if constexpr (sizeof(T) == 4) {
        const float2 v = *reinterpret_cast<const float2*>(p);
        x0 = v.x; x1 = v.y;
    } else {
        const double2 v = *reinterpret_cast<const double2*>(p);
        x0 = v.x; x1 = v.y;
    }
}

template <typename T>
__global__ void __launch_bounds__(kPThreads)
k_pgemm_dw(const PGemm<T>* __restrict__ tabs)
{
    const PGemm<T> g = tabs[blockIdx.z];
    const int r0 = blockIdx.x * kPR, c0 = blockIdx.y * kPC;
    if (r0 >= g.R || c0 >= g.C) return;
    const int ld = (int)g.wr.s1;               // dense Wt: row k at k * ld
    __shared__ __align__(16) T sW[2][kPK][kLS];
    __shared__ __align__(16) T sZ[kPK][kZS];
    __shared__ long long oOr[kPR], oZc[kPC], oOc[kPC], oZk[kPK];
    const int tid = threadIdx.x, tr = tid >> 4, tc = tid & 15;
    if (tid < kPR) {
        oOr[tid] = r0 + tid < g.R ? ax_off(g.orow, r0 + tid) : 0;
    } else if (tid < kPR + kPC) {
        const int c = c0 + tid - kPR;
        oZc[tid - kPR] = c < g.C ? ax_off(g.zc, c) : 0;
        oOc[tid - kPR] = c < g.C ? ax_off(g.ocol, c) : 0;
    }
    T acc[4][2];
#pragma unroll
    for (int u = 0; u < 4; u++) acc[u][0] = acc[u][1] = T(0);
    stage_w(sW[0], g.W, ld, g.K, r0, 0, tid);
    int b = 0;
    for (int k0 = 0; k0 < g.K; k0 += kPK, b ^= 1) {
        const int kn = min(kPK, g.K - k0);
        __syncthreads();                       // offsets ready; buffers of the previous chunk consumed
        if (k0 + kPK < g.K) {
            stage_w(sW[b ^ 1], g.W, ld, g.K, r0, k0 + kPK, tid);
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        if (tid < kPK) oZk[tid] = k0 + tid < g.K ? ax_off(g.zk, k0 + tid) : 0;
        __syncthreads();
        for (int e = tid; e < kPC * kPK; e += kPThreads) {
            const int kk = e / kPC, c = e % kPC;
            sZ[kk][c] = (kk < kn && c0 + c < g.C) ? g.Z[oZk[kk] + oZc[c]] : T(0);
        }
        __syncthreads();
        for (int k = 0; k < kn; k++) {
            T w[4], z0, z1;
            ld4(&sW[b][k][4 * tr], w);
            ld2(&sZ[k][2 * tc], z0, z1);
#pragma unroll
            for (int u = 0; u < 4; u++) {
                acc[u][0] = fma(w[u], z0, acc[u][0]);
                acc[u][1] = fma(w[u], z1, acc[u][1]);
            }
        }
    }
#pragma unroll
    for (int u = 0; u < 4; u++)
#pragma unroll
        for (int v = 0; v < 2; v++) {
            const int r = 4 * tr + u, c = 2 * tc + v;
            if (r0 + r < g.R && c0 + c < g.C) {
                T* o = g.out + oOr[r] + oOc[c];
                *o = fma(g.alpha, acc[u][v], *o);
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

// Raise the running maximum at p (bits of a non-negative value) to x; the
// plain read first skips the atomic when x cannot raise it (most CTAs once
// a large value is in), so the updates do not serialise on one address.
__device__ __forceinline__ void max_bits(void* p, float x)
{
    unsigned int* q = static_cast<unsigned int*>(p);
    const unsigned int u = __float_as_uint(x);
    if (u > *(volatile unsigned int*)q) atomicMax(q, u);
}
__device__ __forceinline__ void max_bits(void* p, double x)
{
    unsigned long long* q = static_cast<unsigned long long*>(p);
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    if (u > *(volatile unsigned long long*)q) atomicMax(q, u);
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
        const T t = arena[d.R + e] / from_f64<T>(den);
        dt = fabs(t - arena[d.Tc + e]);
        arena[d.Tc + e] = t;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) dt = fmax(dt, __shfl_xor_sync(0xffffffffu, dt, o));
    __shared__ T wmax[8];                      // one atomic per CTA, not per warp
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = dt;
    __syncthreads();
    if (threadIdx.x == 0) {
        T m = wmax[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); w++) m = fmax(m, wmax[w]);
        if (m > T(0)) max_bits(delta_bits, m);
    }
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
    const dim3 grid((max_r + kPR - 1) / kPR, (max_c + kPC - 1) / kPC, nd);
    k_pgemm<T><<<grid, kPThreads, 0, s>>>(tabs);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_pgemm_dw(const PGemm<T>* tabs, int nd, int max_r, int max_c, cudaStream_t s)
{
    if (nd <= 0 || max_r <= 0 || max_c <= 0) return cudaSuccess;
    const dim3 grid((max_r + kPR - 1) / kPR, (max_c + kPC - 1) / kPC, nd);
    k_pgemm_dw<T><<<grid, kPThreads, 0, s>>>(tabs);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_pack_ladder(const Td2Dim* dims, const long long* g_off, const long long* wd_off, int nd,
                               int max_rows, T* arena, cudaStream_t s)
{
    if (nd <= 0 || max_rows <= 0) return cudaSuccess;
    k_pack_ladder<T><<<dim3(max_rows, nd), 256, 0, s>>>(dims, g_off, wd_off, arena);
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
template cudaError_t launch_pgemm_dw<float>(const PGemm<float>*, int, int, int, cudaStream_t);
template cudaError_t launch_pgemm_dw<double>(const PGemm<double>*, int, int, int, cudaStream_t);
template cudaError_t launch_pack_ladder<float>(const Td2Dim*, const long long*, const long long*, int, int, float*,
                                               cudaStream_t);
template cudaError_t launch_pack_ladder<double>(const Td2Dim*, const long long*, const long long*, int, int, double*,
                                                cudaStream_t);
template cudaError_t launch_td2_init<float>(const Td2Dim*, const long long*, int, int, float*, cudaStream_t);
template cudaError_t launch_td2_init<double>(const Td2Dim*, const long long*, int, int, double*, cudaStream_t);
template cudaError_t launch_td2_update<float>(const Td2Dim*, int, int, const double*, float*, void*, cudaStream_t);
template cudaError_t launch_td2_update<double>(const Td2Dim*, int, int, const double*, double*, void*, cudaStream_t);
template cudaError_t launch_td2_energy<float>(const Td2Dim*, int, const float*, double*, cudaStream_t);
template cudaError_t launch_td2_energy<double>(const Td2Dim*, int, const double*, double*, cudaStream_t);

}  // namespace mcpt
