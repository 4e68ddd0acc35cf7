// k_fp64.cu -- FP64 first half of the dimer transformation on CUDA cores.
//
// H_f[(p1,p3)][(i,j)] = sum_{p0} C_X[p0][i] sum_{p2} C_Y[p2][j] E[p0][p1][p2][p3]
// (the two occupied quarter transformations of Eq. (dp2e), done first because
// they shrink the data most).  One thread owns one output row (p1, p3): a warp
// reads 32 consecutive p3 of one (p0, p1, p2) line, so every load is
// coalesced, and each loaded integral feeds OB DFMAs from registers.  The
// occupied pairs (i, j) are covered in OB x OB blocks; each block re-reads
// the thread's integrals (from L2 for the sizes that need several blocks).
#include "internal.h"

namespace mcpt {
namespace {

constexpr int kThreads = 128;

template <int OB>
__global__ void __launch_bounds__(kThreads)
k_half_fp64(const DimerDesc* __restrict__ dd, const double* __restrict__ Cpool,
            double* __restrict__ H)
{
    const DimerDesc& d = dd[blockIdx.z];
    const int f = blockIdx.y;
    const int n0 = d.nX, n1 = f ? d.nY : d.nX, n2 = d.nY, n3 = f ? d.nX : d.nY;
    const int rows = n1 * n3;
    if (blockIdx.x * kThreads >= rows) return;   // uniform per block

    const int o0 = d.oX, o2 = d.oY;
    extern __shared__ double sm[];
    double* U0 = sm;               // [n0][OB]  one block of C_X occupied columns
    double* U2 = sm + n0 * OB;     // [n2][OB]  one block of C_Y occupied columns
    const double* CX = Cpool + d.cX;
    const double* CY = Cpool + d.cY;

    const int r = blockIdx.x * kThreads + threadIdx.x;
    const bool active = r < rows;
    const int p1 = active ? r / n3 : 0, p3 = active ? r % n3 : 0;
    const long long s0 = d.st[f][0], s1 = d.st[f][1], s2 = d.st[f][2];
    const double* __restrict__ Erow = d.E[f] + p1 * s1 + p3;
    double* out = H + d.h_off + (long long)f * d.oX * d.oY * rows + r;   // pair-major

    for (int t0b = 0; t0b < o0; t0b += OB) {
        for (int t2b = 0; t2b < o2; t2b += OB) {
            __syncthreads();   // previous block's tables are no longer read
            for (int k = threadIdx.x; k < n0 * OB; k += kThreads) {
                int p = k / OB, t = t0b + k % OB;
                U0[k] = t < o0 ? CX[p * d.nX + t] : 0.0;
            }
            for (int k = threadIdx.x; k < n2 * OB; k += kThreads) {
                int p = k / OB, t = t2b + k % OB;
                U2[k] = t < o2 ? CY[p * d.nY + t] : 0.0;
            }
            __syncthreads();
            if (!active) continue;
            double acc[OB][OB];
#pragma unroll
            for (int a = 0; a < OB; a++)
#pragma unroll
                for (int t = 0; t < OB; t++) acc[a][t] = 0.0;
            for (int p0 = 0; p0 < n0; p0++) {
                const double* __restrict__ Ep = Erow + p0 * s0;
                double F[OB];
#pragma unroll
                for (int t = 0; t < OB; t++) F[t] = 0.0;
#pragma unroll 4
                for (int p2 = 0; p2 < n2; p2++) {
                    const double e = __ldg(Ep + p2 * s2);
                    const double* u = U2 + p2 * OB;
#pragma unroll
                    for (int t = 0; t < OB; t++) F[t] = fma(u[t], e, F[t]);
                }
                const double* u0 = U0 + p0 * OB;
#pragma unroll
                for (int a = 0; a < OB; a++) {
                    const double w = u0[a];
#pragma unroll
                    for (int t = 0; t < OB; t++) acc[a][t] = fma(w, F[t], acc[a][t]);
                }
            }
#pragma unroll
            for (int a = 0; a < OB; a++)
#pragma unroll
                for (int t = 0; t < OB; t++)
                    if (t0b + a < o0 && t2b + t < o2) out[(long long)((t0b + a) * o2 + t2b + t) * rows] = acc[a][t];
        }
    }
}

template <int OB>
cudaError_t launch(const DimerDesc* d_desc, int nd, int max_rows, const double* Cpool,
                   double* H, cudaStream_t s)
{
    const size_t smem = (size_t)2 * kMaxAO * OB * sizeof(double);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_half_fp64<OB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    dim3 grid((max_rows + kThreads - 1) / kThreads, 2, nd);
    k_half_fp64<OB><<<grid, kThreads, smem, s>>>(d_desc, Cpool, H);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_half_fp64(const DimerDesc* d_desc, int nd, int max_rows, int max_occ,
                             const double* Cpool, double* H, cudaStream_t s)
{
    if (nd <= 0) return cudaSuccess;
    if (max_occ <= 4) return launch<4>(d_desc, nd, max_rows, Cpool, H, s);
    if (max_occ <= 5) return launch<5>(d_desc, nd, max_rows, Cpool, H, s);
    if (max_occ <= 6) return launch<6>(d_desc, nd, max_rows, Cpool, H, s);
    return launch<8>(d_desc, nd, max_rows, Cpool, H, s);
}

}  // namespace mcpt
