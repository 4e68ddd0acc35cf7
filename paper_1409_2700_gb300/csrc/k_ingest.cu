// k_ingest.cu -- expansion of symmetry-packed dimer integrals into the two
// blocks the term reads (the a0 ingest step for MCPT_AO_PACKED input).
//
// Real-orbital integrals satisfy (pq|rs) = (qp|rs) = (pq|sr) = (rs|pq).  So
// A[mu][nu][lam][sig] = (mu nu|lam sig) is fixed by its elements with
// mu >= nu, lam >= sig, and K[mu][lam][sig][nu] = (mu lam|sig nu) =
// (nu sig|lam mu) is a symmetric matrix M[P][Q] over the pairs
// P = (mu, lam), Q = (nu, sig), fixed by its lower triangle.  Packed order:
// A_p[t(mu,nu)][t(lam,sig)] then K_p[t(P,Q)], t(a,b) = a(a+1)/2 + b, a >= b.
//
// One CTA per output row (and, batched, per dimer of a staged chunk): A rows
// (mu, nu) of nY^2 elements, then K rows
// P = (mu, lam) of nY nX elements, written coalesced; the gathers read one
// row of A_p, or row / column P of the K_p triangle (6.4 MB at 32 AO, L2
// resident).  All indices fit 32 bits for n <= 128.
#include "internal.h"

namespace mcpt {
namespace {

__device__ __forceinline__ int tri(int a, int b)
{
    return a >= b ? a * (a + 1) / 2 + b : b * (b + 1) / 2 + a;
}

// One output row of one dimer: the body of both expansion kernels.
__device__ __forceinline__ void unpack_row(const double* __restrict__ packed, double* __restrict__ blocks, int nX,
                                           int nY, int row)
{
    const int tY = nY * (nY + 1) / 2;
    if (row < nX * nX) {                        // A[mu][nu][.][.]
        const int mu = row / nX, nu = row - mu * nX;
        const double* src = packed + (size_t)tri(mu, nu) * tY;
        double* dst = blocks + (size_t)row * nY * nY;
        for (int j = threadIdx.x; j < nY * nY; j += blockDim.x) {
            const int la = j / nY, sg = j - la * nY;
            dst[j] = src[tri(la, sg)];
        }
    } else {                                    // K[mu][lam][.][.], P = mu nY + lam
        const int P = row - nX * nX;
        const double* src = packed + (size_t)(nX * (nX + 1) / 2) * tY;
        double* dst = blocks + (size_t)nX * nX * nY * nY + (size_t)P * nY * nX;
        for (int j = threadIdx.x; j < nY * nX; j += blockDim.x) {
            const int sg = j / nX, nu = j - sg * nX;
            dst[j] = src[tri(P, nu * nY + sg)];
        }
    }
}

__global__ void __launch_bounds__(256)
k_unpack(const double* __restrict__ packed, double* __restrict__ blocks, int nX, int nY)
{
    unpack_row(packed, blocks, nX, nY, blockIdx.x);
}

// Several dimers of one staged chunk: CTA (row, dimer of the batch).
__global__ void __launch_bounds__(256) k_unpack_batch(const __grid_constant__ UnpackBatch B)
{
    const UnpackEntry& e = B.e[blockIdx.y];
    if ((int)blockIdx.x >= e.nX * e.nX + e.nX * e.nY) return;
    unpack_row(B.staging + e.src, e.dst, e.nX, e.nY, blockIdx.x);
}

}  // namespace

size_t packed_elems(int nX, int nY)
{
    const size_t tX = (size_t)nX * (nX + 1) / 2, tY = (size_t)nY * (nY + 1) / 2, pq = (size_t)nX * nY;
    return tX * tY + pq * (pq + 1) / 2;
}

cudaError_t launch_unpack(const double* packed, double* blocks, int nX, int nY, cudaStream_t s)
{
    k_unpack<<<nX * nX + nX * nY, 256, 0, s>>>(packed, blocks, nX, nY);
    return cudaGetLastError();
}

cudaError_t launch_unpack_batch(const UnpackBatch& B, cudaStream_t s)
{
    if (B.n <= 0) return cudaSuccess;
    int rows = 0;
    for (int k = 0; k < B.n; k++) rows = max(rows, B.e[k].nX * B.e[k].nX + B.e[k].nX * B.e[k].nY);
    k_unpack_batch<<<dim3(rows, B.n), 256, 0, s>>>(B);
    return cudaGetLastError();
}

}  // namespace mcpt
