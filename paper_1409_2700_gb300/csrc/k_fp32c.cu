// k_fp32c.cu -- compensated-FP32 first half of the dimer transformation.
//
// Same contraction as the FP64 form,
//   H_f[(p1,p3)][(i,j)] = sum_{p0} C_X[p0][i] sum_{p2} C_Y[p2][j] E[p0][p1][p2][p3],
// but on the FP32 pipes: integrals and coefficients are rounded once to FP32,
// and every dot product is accumulated with the error-free transformations of
// Ogita, Rump and Oishi ("Accurate sum and dot product", SIAM J. Sci.
// Comput. 26, 2005): TwoProduct by FMA (h = x*y, r = fma(x, y, -h)) and
// Knuth's TwoSum, so each sum is as accurate as if computed in twice the
// working precision and then rounded (their Dot2).  The FP64 -> FP32
// rounding of each integral runs on the integer pipes (convert.h).  The inner sum over p2 is
// kept as an unevaluated pair (hi, lo) and multiplied into the outer sum over
// p0 the same way.
#include "internal.h"
#include "convert.h"

namespace mcpt {
namespace {

constexpr int kThreads = 128;

struct ff { float hi, lo; };   // value hi + lo, |lo| <= ulp(hi)/2 after renormalising

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = a + b;
    const float z = s - a;
    e = (a - (s - z)) + (b - z);
}

// acc += x * y with the product's and the sum's rounding errors kept in acc.lo
__device__ __forceinline__ void dot2_step(ff& acc, float x, float y)
{
    const float h = x * y;
    const float r = fmaf(x, y, -h);
    float s, q;
    two_sum(acc.hi, h, s, q);
    acc.hi = s;
    acc.lo += q + r;
}

// acc += w * (v.hi + v.lo)
__device__ __forceinline__ void dot2_step_ff(ff& acc, float w, ff v)
{
    dot2_step(acc, w, v.hi);
    acc.lo = fmaf(w, v.lo, acc.lo);
}

template <int OB>
__global__ void __launch_bounds__(kThreads)
k_half_fp32c(const DimerDesc* __restrict__ dd, const float* __restrict__ Cf, float* __restrict__ H)
{
    const DimerDesc& d = dd[blockIdx.z];
    const int f = blockIdx.y;
    const int n0 = d.nX, n1 = f ? d.nY : d.nX, n2 = d.nY, n3 = f ? d.nX : d.nY;
    const int rows = n1 * n3;
    if (blockIdx.x * kThreads >= rows) return;

    const int o0 = d.oX, o2 = d.oY;
    extern __shared__ float smf[];
    float* U0 = smf;               // [n0][OB]
    float* U2 = smf + n0 * OB;     // [n2][OB]
    const float* CX = Cf + d.cX;
    const float* CY = Cf + d.cY;

    const int r = blockIdx.x * kThreads + threadIdx.x;
    const bool active = r < rows;
    const int p1 = active ? r / n3 : 0, p3 = active ? r % n3 : 0;
    const long long s0 = d.st[f][0], s1 = d.st[f][1], s2 = d.st[f][2];
    const double* __restrict__ Erow = d.E[f] + p1 * s1 + p3;
    float* out = H + d.h_off + (long long)f * d.oX * d.oY * rows + r;   // pair-major

    for (int t0b = 0; t0b < o0; t0b += OB) {
        for (int t2b = 0; t2b < o2; t2b += OB) {
            __syncthreads();
            for (int k = threadIdx.x; k < n0 * OB; k += kThreads) {
                int p = k / OB, t = t0b + k % OB;
                U0[k] = t < o0 ? CX[p * d.nX + t] : 0.f;
            }
            for (int k = threadIdx.x; k < n2 * OB; k += kThreads) {
                int p = k / OB, t = t2b + k % OB;
                U2[k] = t < o2 ? CY[p * d.nY + t] : 0.f;
            }
            __syncthreads();
            if (!active) continue;
            ff acc[OB][OB];
#pragma unroll
            for (int a = 0; a < OB; a++)
#pragma unroll
                for (int t = 0; t < OB; t++) acc[a][t] = ff{0.f, 0.f};
            for (int p0 = 0; p0 < n0; p0++) {
                const double* __restrict__ Ep = Erow + p0 * s0;
                ff F[OB];
#pragma unroll
                for (int t = 0; t < OB; t++) F[t] = ff{0.f, 0.f};
#pragma unroll 4
                for (int p2 = 0; p2 < n2; p2++) {
                    const float e = f32_from_f64(__ldg(Ep + p2 * s2));   // integer-pipe conversion
                    const float* u = U2 + p2 * OB;
#pragma unroll
                    for (int t = 0; t < OB; t++) dot2_step(F[t], u[t], e);
                }
                const float* u0 = U0 + p0 * OB;
#pragma unroll
                for (int a = 0; a < OB; a++) {
                    const float w = u0[a];
#pragma unroll
                    for (int t = 0; t < OB; t++) dot2_step_ff(acc[a][t], w, F[t]);
                }
            }
#pragma unroll
            for (int a = 0; a < OB; a++)
#pragma unroll
                for (int t = 0; t < OB; t++)
                    if (t0b + a < o0 && t2b + t < o2) out[(long long)((t0b + a) * o2 + t2b + t) * rows] = acc[a][t].hi + acc[a][t].lo;
        }
    }
}

template <int OB>
cudaError_t launch(const DimerDesc* d_desc, int nd, int max_rows, const float* Cf, float* H, cudaStream_t s)
{
    const size_t smem = (size_t)2 * kMaxAOTensor * OB * sizeof(float);
    dim3 grid((max_rows + kThreads - 1) / kThreads, 2, nd);
    k_half_fp32c<OB><<<grid, kThreads, smem, s>>>(d_desc, Cf, H);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_half_fp32c(const DimerDesc* d_desc, int nd, int max_rows, int max_occ, const float* Cf,
                              float* H, cudaStream_t s)
{
    if (nd <= 0) return cudaSuccess;
    if (max_occ <= 4) return launch<4>(d_desc, nd, max_rows, Cf, H, s);
    if (max_occ <= 5) return launch<5>(d_desc, nd, max_rows, Cf, H, s);
    return launch<8>(d_desc, nd, max_rows, Cf, H, s);
}

}  // namespace mcpt
