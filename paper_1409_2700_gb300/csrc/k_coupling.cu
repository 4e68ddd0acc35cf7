// k_coupling.cu -- the dimer -> monomer doubles coupling of Eq. (tm2), the
// sum over the neighbour's (k, c) pairs, at the first-order dimer amplitude
// T = v D of the energy path:
//   R_X[(i,a)][(i1,a1)] = sum_{Y, k, c} v^{a1 k}_{i1 c} T^{ac}_{ik} + v^{ak}_{ic} T^{a1 c}_{i1 k}
// For a dimer (X, Y) the second half stored V = (ia|jb) and T = V D as
// [(j,b)][(i,a)] matrices S_V, S_T (m_Y x m_X, m = o v).  Then
//   X side: R_X[p][q] += sum_{r=(j,b)} S_T[r][p] S_V[r][q] + S_V[r][p] S_T[r][q]
//   Y side: R_Y[p][q] += sum_{r=(i,a)} S_T[p][r] S_V[q][r] + S_V[p][r] S_T[q][r]
// (the Y side reads the stored rows as columns).
// One CTA per 64 x 64 tile of one monomer's R; it walks the monomer's
// dimers in ascending order and their rows in chunks of 32 staged in shared
// memory, each thread accumulating a 4 x 4 block (rows ty + 16 u, columns
// tx + 16 w) in registers: per row 16 loads feed 32 FMAs.  Every sum has a
// fixed order, so R is deterministic run to run.
#include "internal.h"

namespace mcpt {
namespace {

constexpr int kCT = 64;          // output tile edge
constexpr int kCThreads = 256;
template <typename T>
__host__ __device__ constexpr int ck() { return sizeof(T) == 8 ? 16 : 32; }   // rows per staged chunk (32 KB of operands)

template <typename T>
__global__ void __launch_bounds__(kCThreads)
k_coupling(const CoupTile* __restrict__ tiles, const CoupDim* __restrict__ dims, MonomerLists L,
           const int* __restrict__ mdim, const long long* __restrict__ r_off, const T* __restrict__ VT,
           double* __restrict__ R)
{
    constexpr int kCK = ck<T>();
    const CoupTile tile = tiles[blockIdx.x];
    const int mon = tile.mon, m = mdim[mon];
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    __shared__ T sTp[kCK][kCT], sVp[kCK][kCT], sTq[kCK][kCT], sVq[kCK][kCT];
    T acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; u++)
#pragma unroll
        for (int w = 0; w < 4; w++) acc[u][w] = T(0);

    for (int li = L.start[mon]; li < L.start[mon + 1]; li++) {
        const CoupDim cd = dims[L.list[li]];
        const T* V = VT + cd.vt_off;
        const T* Tm = V + (long long)cd.mX * cd.mY;
        const bool xside = cd.X == mon;
        const int K = xside ? cd.mY : cd.mX;        // rows summed over
        const int ld = cd.mX;                       // row length of the stored [(j,b)][(i,a)]
        for (int k0 = 0; k0 < K; k0 += kCK) {
            __syncthreads();
            // stage rows k0.. of the four operand columns blocks (p and q tiles)
            for (int e = tid; e < kCK * kCT; e += kCThreads) {
                int r, c;
                if (xside) { r = e / kCT; c = e % kCT; }      // contiguous along the (i,a) columns
                else       { c = e / kCK; r = e % kCK; }      // contiguous along the (i,a) rows read
                const int k = k0 + r, p = tile.p0 + c, q = tile.q0 + c;
                T tp = T(0), vp = T(0), tq = T(0), vq = T(0);
                if (k < K) {
                    if (xside) {
                        const long long rowk = (long long)k * ld;
                        if (p < m) { tp = Tm[rowk + p]; vp = V[rowk + p]; }
                        if (q < m) { tq = Tm[rowk + q]; vq = V[rowk + q]; }
                    } else {
                        if (p < m) { tp = Tm[(long long)p * ld + k]; vp = V[(long long)p * ld + k]; }
                        if (q < m) { tq = Tm[(long long)q * ld + k]; vq = V[(long long)q * ld + k]; }
                    }
                }
                sTp[r][c] = tp; sVp[r][c] = vp; sTq[r][c] = tq; sVq[r][c] = vq;
            }
            __syncthreads();
            const int kn = min(kCK, K - k0);
            for (int r = 0; r < kn; r++) {
                T at[4], av[4], bt[4], bv[4];
#pragma unroll
                for (int u = 0; u < 4; u++) { at[u] = sTp[r][ty + 16 * u]; av[u] = sVp[r][ty + 16 * u]; }
#pragma unroll
                for (int w = 0; w < 4; w++) { bt[w] = sTq[r][tx + 16 * w]; bv[w] = sVq[r][tx + 16 * w]; }
#pragma unroll
                for (int u = 0; u < 4; u++)
#pragma unroll
                    for (int w = 0; w < 4; w++) acc[u][w] = fma(at[u], bv[w], fma(av[u], bt[w], acc[u][w]));
            }
        }
    }
    double* Rm = R + r_off[mon];
#pragma unroll
    for (int u = 0; u < 4; u++)
#pragma unroll
        for (int w = 0; w < 4; w++) {
            const int p = tile.p0 + ty + 16 * u, q = tile.q0 + tx + 16 * w;
            if (p < m && q < m) Rm[(long long)p * m + q] = (double)acc[u][w];
        }
}

template <typename T>
cudaError_t launch(const CoupTile* tiles, int ntiles, const CoupDim* dims, MonomerLists lists, const int* mdim,
                   const long long* r_off, const T* VT, double* R, cudaStream_t s)
{
    if (ntiles <= 0) return cudaSuccess;
    k_coupling<T><<<ntiles, kCThreads, 0, s>>>(tiles, dims, lists, mdim, r_off, VT, R);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_coupling_fp32(const CoupTile* tiles, int ntiles, const CoupDim* dims, MonomerLists lists,
                                 const int* mdim, const long long* r_off, const float* VT, double* R,
                                 cudaStream_t s)
{
    return launch<float>(tiles, ntiles, dims, lists, mdim, r_off, VT, R, s);
}

cudaError_t launch_coupling_fp64(const CoupTile* tiles, int ntiles, const CoupDim* dims, MonomerLists lists,
                                 const int* mdim, const long long* r_off, const double* VT, double* R,
                                 cudaStream_t s)
{
    return launch<double>(tiles, ntiles, dims, lists, mdim, r_off, VT, R, s);
}

}  // namespace mcpt
