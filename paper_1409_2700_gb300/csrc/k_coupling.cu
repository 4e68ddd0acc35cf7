// k_coupling.cu -- the dimer -> monomer doubles coupling of Eq. (tm2), the
// sum over the neighbour's (k, c) pairs, at the first-order dimer amplitude
// T = v D of the energy path:
//   R_X[(i,a)][(i1,a1)] = sum_{Y, k, c} v^{a1 k}_{i1 c} T^{ac}_{ik} + v^{ak}_{ic} T^{a1 c}_{i1 k}
// For a dimer (X, Y) the second half stored V = (ia|jb) and T = V D as
// [(j,b)][(i,a)] matrices S_V, S_T (m_Y x m_X, m = o v).  Then
//   X side: R_X[p][q] += sum_{r=(j,b)} S_T[r][p] S_V[r][q] + S_V[r][p] S_T[r][q]
//   Y side: R_Y[p][q] += sum_{r=(i,a)} S_T[p][r] S_V[q][r] + S_V[p][r] S_T[q][r]
// (the Y side reads the stored rows as columns).
// R is symmetric, so only tiles with q0 >= p0 run, each writing R[p][q] and
// its mirror R[q][p] for p <= q (R is exactly symmetric).  A monomer's tiles
// have edge 64, 48 or 32, whichever covers its o v rows with the least padded
// work, one launch per edge.  A CTA walks the monomer's dimers in ascending
// order and their rows in chunks of 32 (16 in FP64), staged in shared memory
// by cp.async into two buffers: the next chunk is in flight while the
// current one is summed.  (Chunks of 16 or 24 rows, which fit five CTAs of
// edge 48 per SM, measured slower: the barriers cost more than the wave.)  Rows are padded by 4 so the transposed Y side
// stages without bank conflicts (eight rows by four columns per warp); each
// thread accumulates a contiguous 4 x 4 block in registers: per row four
// 4-wide shared loads feed 32 FMAs.  Every sum has a fixed order, so R is
// deterministic run to run.
#include "internal.h"

namespace mcpt {
namespace {

template <typename T>
__host__ __device__ constexpr int ck() { return sizeof(T) == 8 ? 16 : 32; }   // rows per staged chunk
template <int CT>
__host__ __device__ constexpr int cthreads() { return ((CT / 4) * (CT / 4) + 31) / 32 * 32; }
template <typename T, int CT>
__host__ __device__ constexpr size_t coupling_smem() { return 2 * 4 * ck<T>() * (CT + 4) * sizeof(T); }

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

// One element copy global -> shared; an invalid source writes zero (no read).
template <typename T>
__device__ __forceinline__ void cp_elem(T* dst, const T* src, bool ok, const T* any)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(ok ? src : any), "n"(sizeof(T)), "r"(ok ? (int)sizeof(T) : 0)
                 : "memory");
}

// Start the copies of rows k0 .. k0 + kCK of one dimer's operands into
// buffer B (4 planes: T and V of the p columns, T and V of the q columns),
// committed as one group per thread.
template <typename T, int CT>
__device__ __forceinline__ void stage_chunk(T* B, const CoupDim& cd, bool xside, int k0, const T* VT, int m,
                                            const CoupTile& tile, bool diag, int tid)
{
    constexpr int kCK = ck<T>(), kLD = CT + 4, kNT = cthreads<CT>(), kPL = kCK * kLD;
    const T* V = VT + cd.vt_off;
    const T* Tm = V + (long long)cd.mX * cd.mY;
    const int K = xside ? cd.mY : cd.mX;
    const long long ld = cd.mX;
    if (xside) {                                // rows k of the stored matrices, contiguous along c
        for (int e = tid; e < kCK * CT; e += kNT) {
            const int r = e / CT, c = e % CT, k = k0 + r, p = tile.p0 + c, q = tile.q0 + c;
            const bool okk = k < K;
            const long long rowk = (long long)k * ld;
            T* d = B + r * kLD + c;
            cp_elem(d, Tm + rowk + p, okk && p < m, VT);
            cp_elem(d + kPL, V + rowk + p, okk && p < m, VT);
            if (!diag) {
                cp_elem(d + 2 * kPL, Tm + rowk + q, okk && q < m, VT);
                cp_elem(d + 3 * kPL, V + rowk + q, okk && q < m, VT);
            }
        }
    } else {                                    // columns k of the stored rows p, q: 8 rows x 4 columns a warp
        constexpr int kRG = kCK / 8;
        const int lane = tid & 31, warp = tid >> 5;
        for (int g = warp; g < kRG * (CT / 4); g += kNT / 32) {
            const int r = (g % kRG) * 8 + (lane & 7), c = (g / kRG) * 4 + (lane >> 3);
            const int k = k0 + r, p = tile.p0 + c, q = tile.q0 + c;
            const bool okk = k < K;
            T* d = B + r * kLD + c;
            cp_elem(d, Tm + p * ld + k, okk && p < m, VT);
            cp_elem(d + kPL, V + p * ld + k, okk && p < m, VT);
            if (!diag) {
                cp_elem(d + 2 * kPL, Tm + q * ld + k, okk && q < m, VT);
                cp_elem(d + 3 * kPL, V + q * ld + k, okk && q < m, VT);
            }
        }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

template <typename T, int CT>
__global__ void __launch_bounds__(cthreads<CT>())
k_coupling(const CoupTile* __restrict__ tiles, const CoupDim* __restrict__ dims, MonomerLists L,
           const int* __restrict__ mdim, const long long* __restrict__ r_off, const T* __restrict__ VT,
           double* __restrict__ R)
{
    constexpr int kCK = ck<T>(), kLD = CT + 4, kTW = CT / 4, kPL = kCK * kLD;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* buf = reinterpret_cast<T*>(smem_raw);   // 2 buffers x 4 planes x kCK x kLD
    const CoupTile tile = tiles[blockIdx.x];
    const int mon = tile.mon, m = mdim[mon];
    const bool diag = tile.p0 == tile.q0;
    const int tid = threadIdx.x;
    const bool active = tid < kTW * kTW;
    const int ty = tid / kTW, tx = tid % kTW;
    const int qs = diag ? 0 : 2;      // a diagonal tile reads its p operands twice
    T acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; u++)
#pragma unroll
        for (int w = 0; w < 4; w++) acc[u][w] = T(0);

    // the chunk sequence: (dimer li, rows k0) in order; `next` is staged one ahead
    int li = L.start[mon];
    const int lend = L.start[mon + 1];
    if (li >= lend) goto write;
    {
        CoupDim cd = dims[L.list[li]];
        int k0 = 0, b = 0;
        stage_chunk<T, CT>(buf, cd, cd.X == mon, 0, VT, m, tile, diag, tid);
        for (;;) {
            const int K = cd.X == mon ? cd.mY : cd.mX;
            const int kn = min(kCK, K - k0);
            // the chunk after this one
            int nli = li, nk0 = k0 + kCK;
            if (nk0 >= K) { nli = li + 1; nk0 = 0; }
            const bool more = nli < lend;
            CoupDim ncd = cd;
            if (more) {
                if (nli != li) ncd = dims[L.list[nli]];
                stage_chunk<T, CT>(buf + (b ^ 1) * 4 * kPL, ncd, ncd.X == mon, nk0, VT, m, tile, diag, tid);
                asm volatile("cp.async.wait_group 1;" ::: "memory");
            } else {
                asm volatile("cp.async.wait_group 0;" ::: "memory");
            }
            __syncthreads();
            if (active) {
                const T* S = buf + b * 4 * kPL;
#pragma unroll 2
                for (int r = 0; r < kn; r++) {
                    T at[4], av[4], bt[4], bv[4];
                    ld4(S + r * kLD + 4 * ty, at);
                    ld4(S + kPL + r * kLD + 4 * ty, av);
                    ld4(S + qs * kPL + r * kLD + 4 * tx, bt);
                    ld4(S + (qs + 1) * kPL + r * kLD + 4 * tx, bv);
#pragma unroll
                    for (int u = 0; u < 4; u++)
#pragma unroll
                        for (int w = 0; w < 4; w++) acc[u][w] = fma(at[u], bv[w], fma(av[u], bt[w], acc[u][w]));
                }
            }
            __syncthreads();            // buffer b is refilled two chunks on
            if (!more) break;
            li = nli; k0 = nk0; cd = ncd; b ^= 1;
        }
    }
write:
    if (!active) return;
    double* Rm = R + r_off[mon];
#pragma unroll
    for (int u = 0; u < 4; u++)
#pragma unroll
        for (int w = 0; w < 4; w++) {
            const int p = tile.p0 + 4 * ty + u, q = tile.q0 + 4 * tx + w;
            if (p < m && q < m && p <= q) {
                Rm[(long long)p * m + q] = (double)acc[u][w];
                Rm[(long long)q * m + p] = (double)acc[u][w];
            }
        }
}

template <typename T, int CT>
cudaError_t launch_edge(const CoupTile* tiles, int n, const CoupDim* dims, MonomerLists lists, const int* mdim,
                        const long long* r_off, const T* VT, double* R, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    constexpr size_t smem = coupling_smem<T, CT>();
    cudaError_t e = cudaFuncSetAttribute(k_coupling<T, CT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_coupling<T, CT><<<n, cthreads<CT>(), smem, s>>>(tiles, dims, lists, mdim, r_off, VT, R);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch(const CoupTile* tiles, const int* ntile, const CoupDim* dims, MonomerLists lists, const int* mdim,
                   const long long* r_off, const T* VT, double* R, cudaStream_t s)
{
    // tiles: the edge-64 tiles, then the edge-48, then the edge-32 ones
    cudaError_t e = launch_edge<T, 64>(tiles, ntile[0], dims, lists, mdim, r_off, VT, R, s);
    if (e == cudaSuccess) e = launch_edge<T, 48>(tiles + ntile[0], ntile[1], dims, lists, mdim, r_off, VT, R, s);
    if (e == cudaSuccess)
        e = launch_edge<T, 32>(tiles + ntile[0] + ntile[1], ntile[2], dims, lists, mdim, r_off, VT, R, s);
    return e;
}

// Singles environment term of Eq. (tm1): s_X[(i,a)] = sum over X's dimers
// (ascending) of sum_{(k,c)} (ia|kc) t_Y[(k,c)], in two launches.  First one
// CTA of 256 threads per (dimer, side) forms that dimer's contribution to one
// of its monomers, with the neighbour's amplitudes converted to the storage
// type in shared memory: X side, a thread per output column p walks the
// stored rows in order (partial sums of 32 rows added in FP64); Y side, a warp
// per output row, a dot product of the stored row with t_X (lanes strided
// over the row, then a butterfly).  Then one thread per output adds the
// contributions of the monomer's dimers in ascending order.  Fixed orders
// throughout, so s is deterministic run to run.
constexpr int kSThreads = 256;
constexpr int kSMaxM = 4096;     // o v <= 64 x 64 for any monomer of at most 128 AO

template <typename T>
__global__ void __launch_bounds__(kSThreads)
k_singles_part(const CoupDim* __restrict__ dims, const long long* __restrict__ s_off,
               const long long* __restrict__ part_off, const T* __restrict__ VT, const double* __restrict__ t,
               double* __restrict__ part)
{
    __shared__ T st[kSMaxM];
    const int d = blockIdx.x >> 1, side = blockIdx.x & 1;
    const CoupDim cd = dims[d];
    const T* V = VT + cd.vt_off;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int mo = side == 0 ? cd.mY : cd.mX;                 // length of the neighbour's amplitudes
    const double* to = t + s_off[side == 0 ? cd.Y : cd.X];
    for (int e = tid; e < mo; e += kSThreads) st[e] = (T)to[e];
    __syncthreads();
    double* out = part + part_off[d] + (side == 0 ? 0 : cd.mX);
    if (side == 0) {
        for (int p = tid; p < cd.mX; p += kSThreads) {
            double acc = 0.0;
            for (int r0 = 0; r0 < cd.mY; r0 += 32) {
                const int r1 = min(r0 + 32, cd.mY);
                T x = T(0);
#pragma unroll 8
                for (int r = r0; r < r1; r++) x = fma(V[(long long)r * cd.mX + p], st[r], x);
                acc += (double)x;
            }
            out[p] = acc;
        }
    } else {
        for (int r = warp; r < cd.mY; r += kSThreads / 32) {
            const T* row = V + (long long)r * cd.mX;
            T x = T(0);
            for (int q = lane; q < cd.mX; q += 32) x = fma(row[q], st[q], x);
#pragma unroll
            for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            if (lane == 0) out[r] = (double)x;
        }
    }
}

__global__ void __launch_bounds__(kSThreads)
k_singles_sum(const SingTile* __restrict__ tiles, const CoupDim* __restrict__ dims, MonomerLists L,
              const int* __restrict__ mdim, const long long* __restrict__ s_off,
              const long long* __restrict__ part_off, const double* __restrict__ part, double* __restrict__ s)
{
    const SingTile tile = tiles[blockIdx.x];
    const int mon = tile.mon, p = tile.p0 + threadIdx.x;
    if (p >= mdim[mon]) return;
    double acc = 0.0;
    for (int li = L.start[mon]; li < L.start[mon + 1]; li++) {
        const int d = L.list[li];
        const CoupDim cd = dims[d];
        acc += part[part_off[d] + (cd.X == mon ? 0 : cd.mX) + p];
    }
    s[s_off[mon] + p] = acc;
}

template <typename T>
cudaError_t launch_s(const SingTile* tiles, int ntiles, const CoupDim* dims, int ndims, MonomerLists lists,
                     const int* mdim, const long long* s_off, const long long* part_off, const T* VT,
                     const double* t, double* part, double* s, cudaStream_t st)
{
    if (ndims > 0) k_singles_part<T><<<2 * ndims, kSThreads, 0, st>>>(dims, s_off, part_off, VT, t, part);
    if (ntiles > 0) k_singles_sum<<<ntiles, kSThreads, 0, st>>>(tiles, dims, lists, mdim, s_off, part_off, part, s);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_coupling_fp32(const CoupTile* tiles, const int* ntile, const CoupDim* dims, MonomerLists lists,
                                 const int* mdim, const long long* r_off, const float* VT, double* R,
                                 cudaStream_t s)
{
    return launch<float>(tiles, ntile, dims, lists, mdim, r_off, VT, R, s);
}

cudaError_t launch_coupling_fp64(const CoupTile* tiles, const int* ntile, const CoupDim* dims, MonomerLists lists,
                                 const int* mdim, const long long* r_off, const double* VT, double* R,
                                 cudaStream_t s)
{
    return launch<double>(tiles, ntile, dims, lists, mdim, r_off, VT, R, s);
}

cudaError_t launch_singles_fp32(const SingTile* tiles, int ntiles, const CoupDim* dims, int ndims, MonomerLists lists,
                                const int* mdim, const long long* s_off, const long long* part_off, const float* VT,
                                const double* t, double* part, double* s, cudaStream_t st)
{
    return launch_s<float>(tiles, ntiles, dims, ndims, lists, mdim, s_off, part_off, VT, t, part, s, st);
}

cudaError_t launch_singles_fp64(const SingTile* tiles, int ntiles, const CoupDim* dims, int ndims, MonomerLists lists,
                                const int* mdim, const long long* s_off, const long long* part_off, const double* VT,
                                const double* t, double* part, double* s, cudaStream_t st)
{
    return launch_s<double>(tiles, ntiles, dims, ndims, lists, mdim, s_off, part_off, VT, t, part, s, st);
}

}  // namespace mcpt
