// k_df.cu -- the density-fitted route to the dimer terms: (ia|jb) and
// (ib|ja) from three-index factors B^Q over the dimer's AO space instead of
// the four-index blocks,
//   (ia|jb) = s sum_Q (C_X^T B^Q_XX C_X)_{ia} (C_Y^T B^Q_YY C_Y)_{jb}
//   (ib|ja) = s sum_Q (C_X^T B^Q_XY C_Y)_{ib} (C_Y^T B^Q_YX C_X)_{ja},
// then the same denominators and energies as the four-index path.
//
// k_df_half: one CTA per (dimer, Q) forms the occupied rows of the factor
// first, u_X = C_X,occ^T B^Q[X rows] and u_Y = C_Y,occ^T B^Q[Y rows] (over
// all n columns), then the four o x v half-transformed blocks.
// k_df_pair: one CTA per (dimer, occupied pair i, j) sums the two vX x vY
// tiles over Q, staged in chunks, and applies the FP64 epilogue; the pairs'
// partial energies are added per dimer in fixed order (k_df_sum).
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

template <typename T>
__global__ void __launch_bounds__(256)
k_df_half(const DfDim* __restrict__ dims, const double* __restrict__ C, T* __restrict__ half)
{
    const DfDim d = dims[blockIdx.y];
    const int q = blockIdx.x;
    if (q >= d.naux) return;
    const int nX = d.nX, nY = d.nY, n = nX + nY, oX = d.oX, oY = d.oY, vX = nX - oX, vY = nY - oY;
    const double* B = d.B + (long long)q * n * n;
    // shared: B^Q [n][n], C_X [nX][nX], C_Y [nY][nY], then u_X [oX][n], u_Y [oY][n]
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sB = reinterpret_cast<T*>(smem_raw);
    T* sCX = sB + n * n;
    T* sCY = sCX + nX * nX;
    T* uX = sCY + nY * nY;
    T* uY = uX + oX * n;
    // eight loads in flight per thread
    for (int e0 = threadIdx.x; e0 < n * n; e0 += 8 * blockDim.x) {
        double x[8];
#pragma unroll
        for (int u = 0; u < 8; u++) {
            const int e = e0 + u * blockDim.x;
            x[u] = e < n * n ? B[e] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 8; u++) {
            const int e = e0 + u * blockDim.x;
            if (e < n * n) sB[e] = from_f64<T>(x[u]);
        }
    }
    for (int e = threadIdx.x; e < nX * nX; e += blockDim.x) sCX[e] = from_f64<T>(C[d.cX + e]);
    for (int e = threadIdx.x; e < nY * nY; e += blockDim.x) sCY[e] = from_f64<T>(C[d.cY + e]);
    __syncthreads();
    for (int e = threadIdx.x; e < (oX + oY) * n; e += blockDim.x) {
        const int r = e / n, c = e % n;
        T a0 = T(0), a1 = T(0);                // two chains for latency
        if (r < oX) {
            int mu = 0;
            for (; mu + 1 < nX; mu += 2) {
                a0 = fma(sCX[mu * nX + r], sB[mu * n + c], a0);
                a1 = fma(sCX[(mu + 1) * nX + r], sB[(mu + 1) * n + c], a1);
            }
            if (mu < nX) a0 = fma(sCX[mu * nX + r], sB[mu * n + c], a0);
        } else {
            const int j = r - oX;
            int la = 0;
            for (; la + 1 < nY; la += 2) {
                a0 = fma(sCY[la * nY + j], sB[(nX + la) * n + c], a0);
                a1 = fma(sCY[(la + 1) * nY + j], sB[(nX + la + 1) * n + c], a1);
            }
            if (la < nY) a0 = fma(sCY[la * nY + j], sB[(nX + la) * n + c], a0);
        }
        uX[e] = a0 + a1;                       // uY follows uX contiguously
    }
    __syncthreads();
    const long long mX = (long long)oX * vX, mY = (long long)oY * vY, xb = (long long)oX * vY, yb = (long long)oY * vX;
    T* xx = half + d.h_off + (long long)q * mX;
    T* yy = half + d.h_off + (long long)d.naux * mX + (long long)q * mY;
    T* xy = half + d.h_off + (long long)d.naux * (mX + mY) + (long long)q * xb;
    T* yx = half + d.h_off + (long long)d.naux * (mX + mY + xb) + (long long)q * yb;
    // the four o x v blocks: out[r][c] = sum_k u[r][k0 + k] C[k][o + c]
    const int tot = (int)(mX + mY + xb + yb);
    for (int e = threadIdx.x; e < tot; e += blockDim.x) {
        const T* u;
        const T* Cm;
        int len, ldc, co, r, c;
        T* out;
        if (e < mX) {
            r = e / vX; c = e % vX; u = uX + r * n; Cm = sCX; len = nX; ldc = nX; co = oX; out = xx + e;
        } else if (e < mX + mY) {
            const int f = e - (int)mX;
            r = f / vY; c = f % vY; u = uY + r * n + nX; Cm = sCY; len = nY; ldc = nY; co = oY; out = yy + f;
        } else if (e < mX + mY + xb) {
            const int f = e - (int)(mX + mY);
            r = f / vY; c = f % vY; u = uX + r * n + nX; Cm = sCY; len = nY; ldc = nY; co = oY; out = xy + f;
        } else {
            const int f = e - (int)(mX + mY + xb);
            r = f / vX; c = f % vX; u = uY + r * n; Cm = sCX; len = nX; ldc = nX; co = oX; out = yx + f;
        }
        T a0 = T(0), a1 = T(0);
        int k = 0;
        for (; k + 1 < len; k += 2) {
            a0 = fma(u[k], Cm[k * ldc + co + c], a0);
            a1 = fma(u[k + 1], Cm[(k + 1) * ldc + co + c], a1);
        }
        if (k < len) a0 = fma(u[k], Cm[k * ldc + co + c], a0);
        *out = a0 + a1;
    }
}

constexpr int kDQ = 32;                        // Q values per staged chunk

template <typename T>
__global__ void __launch_bounds__(256)
k_df_pair(const DfDim* __restrict__ dims, const double* __restrict__ eps, const T* __restrict__ half,
          double* __restrict__ part)
{
    const DfDim d = dims[blockIdx.y];
    const int nX = d.nX, nY = d.nY, oX = d.oX, oY = d.oY, vX = nX - oX, vY = nY - oY;
    const int pr = blockIdx.x;                 // occupied pair i * oY + j
    if (pr >= oX * oY) return;
    const int i = pr / oY, j = pr % oY;
    const long long mX = (long long)oX * vX, mY = (long long)oY * vY, xb = (long long)oX * vY, yb = (long long)oY * vX;
    const T* xx = half + d.h_off;
    const T* yy = xx + (long long)d.naux * mX;
    const T* xy = yy + (long long)d.naux * mY;
    const T* yx = xy + (long long)d.naux * xb;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sxx = reinterpret_cast<T*>(smem_raw);   // [kDQ][vX]: xx[Q][i][.]
    T* syy = sxx + kDQ * vX;                   // [kDQ][vY]: yy[Q][j][.]
    T* sxy = syy + kDQ * vY;                   // [kDQ][vY]: xy[Q][i][.]
    T* syx = sxy + kDQ * vY;                   // [kDQ][vX]: yx[Q][j][.]
    double* red = reinterpret_cast<double*>(syx + kDQ * vX + (kDQ * vX) % 2);
    const int nab = vX * vY;
    double ej = 0.0, ek = 0.0;
    // the thread owns the (a, b) elements e0 + tid + 256 u of each block of 1024
    for (int e0 = 0; e0 < nab; e0 += 256 * 4) {
        T v[4] = {T(0), T(0), T(0), T(0)}, w[4] = {T(0), T(0), T(0), T(0)};
        for (int q0 = 0; q0 < d.naux; q0 += kDQ) {
            const int qn = min(kDQ, d.naux - q0);
            __syncthreads();
            for (int e = threadIdx.x; e < qn * vX; e += blockDim.x) {
                const int qq = e / vX, a = e % vX;
                sxx[qq * vX + a] = xx[(long long)(q0 + qq) * mX + i * vX + a];
                syx[qq * vX + a] = yx[(long long)(q0 + qq) * yb + j * vX + a];
            }
            for (int e = threadIdx.x; e < qn * vY; e += blockDim.x) {
                const int qq = e / vY, b = e % vY;
                syy[qq * vY + b] = yy[(long long)(q0 + qq) * mY + j * vY + b];
                sxy[qq * vY + b] = xy[(long long)(q0 + qq) * xb + i * vY + b];
            }
            __syncthreads();
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const int e = e0 + threadIdx.x + 256 * u;
                if (e < nab) {
                    const int a = e / vY, b = e % vY;
                    T vv = v[u], ww = w[u];
                    for (int qq = 0; qq < qn; qq++) {
                        vv = fma(sxx[qq * vX + a], syy[qq * vY + b], vv);
                        ww = fma(sxy[qq * vY + b], syx[qq * vX + a], ww);
                    }
                    v[u] = vv;
                    w[u] = ww;
                }
            }
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int e = e0 + threadIdx.x + 256 * u;
            if (e < nab) {
                const int a = e / vY, b = e % vY;
                const double D = 1.0 / (eps[d.eX + i] + eps[d.eY + j] - eps[d.eX + oX + a] - eps[d.eY + oY + b]);
                const double vs = d.s * (double)v[u], ws = d.s * (double)w[u];
                ej += 4.0 * vs * vs * D;
                ek += -2.0 * vs * ws * D;
            }
        }
    }
    red[threadIdx.x] = ej;
    red[256 + threadIdx.x] = ek;
    __syncthreads();
    for (int h = 128; h; h >>= 1) {
        if (threadIdx.x < h) {
            red[threadIdx.x] += red[threadIdx.x + h];
            red[256 + threadIdx.x] += red[256 + threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * (d.p_off + pr)] = red[0];
        part[2 * (d.p_off + pr) + 1] = red[256];
    }
}

__global__ void k_df_sum(const DfDim* __restrict__ dims, int nd, const double* __restrict__ part,
                         double* __restrict__ E2)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nd) return;
    const DfDim d = dims[k];
    double ej = 0.0, ek = 0.0;
    for (int p = 0; p < d.oX * d.oY; p++) {
        ej += part[2 * (d.p_off + p)];
        ek += part[2 * (d.p_off + p) + 1];
    }
    E2[2 * d.id] = ej;
    E2[2 * d.id + 1] = ek;
}

template <typename T>
size_t pair_smem(int max_v)
{
    return (size_t)4 * kDQ * max_v * sizeof(T) + 16 + 512 * sizeof(double);
}

template <typename T>
cudaError_t launch_df_t(const DfDim* dims, int nd, int max_naux, int max_pairs, int max_on, int max_v,
                        const double* C, const double* eps, T* half, double* part, double* E2, cudaStream_t s)
{
    if (nd <= 0) return cudaSuccess;
    const size_t sh = (size_t)max_on * sizeof(T);    // B^Q, C_X, C_Y, u_X, u_Y
    cudaError_t e = cudaFuncSetAttribute(k_df_half<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
    if (e != cudaSuccess) return e;
    k_df_half<T><<<dim3(max_naux, nd), 256, sh, s>>>(dims, C, half);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const size_t sp = pair_smem<T>(max_v);
    e = cudaFuncSetAttribute(k_df_pair<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sp);
    if (e != cudaSuccess) return e;
    k_df_pair<T><<<dim3(max_pairs, nd), 256, sp, s>>>(dims, eps, half, part);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_df_sum<<<(nd + 127) / 128, 128, 0, s>>>(dims, nd, part, E2);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_df(bool fp64, const DfDim* dims, int nd, int max_naux, int max_pairs, int max_on, int max_v,
                      const double* C, const double* eps, void* half, double* part, double* E2, cudaStream_t s)
{
    return fp64 ? launch_df_t<double>(dims, nd, max_naux, max_pairs, max_on, max_v, C, eps,
                                      static_cast<double*>(half), part, E2, s)
                : launch_df_t<float>(dims, nd, max_naux, max_pairs, max_on, max_v, C, eps,
                                     static_cast<float*>(half), part, E2, s);
}

}  // namespace mcpt
