// device.cu -- device twin of the synthetic input generator (synth/__init__.py).
// Draws the same Philox4x32-10 streams as the host code (Salmon et al., SC'11):
// counter (k, object, Q, tag), key (seed, "MCPT"); Box-Muller in FP64.  Holds
// none of the MCPT arithmetic; it only makes the factors the integrals are
// built from.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

__device__ __forceinline__ void philox(uint32_t c[4], uint32_t k0, uint32_t k1)
{
    for (int r = 0; r < 10; r++) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
        const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c[1] ^ k0;
        const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = (uint32_t)p1;
        c[2] = n2;
        c[3] = (uint32_t)p0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

__device__ __forceinline__ double u53(uint32_t hi, uint32_t lo)
{
    return ((double)(hi >> 5) * 67108864.0 + (double)(lo >> 6)) / 9007199254740992.0;
}

// draw f of stream (obj, sub, tag): pair f/2, component f%2
__device__ double normal(uint32_t seed, uint32_t obj, uint32_t sub, uint32_t tag, uint32_t f)
{
    uint32_t c[4] = {f >> 1, obj, sub, tag};
    philox(c, seed, 0x4D435054u);
    const double u0 = u53(c[0], c[1]);
    const double u1 = u53(c[2], c[3]);
    const double rad = sqrt(-2.0 * log1p(-u0));
    const double ang = 2.0 * 3.141592653589793 * u1;
    return (f & 1) ? rad * sin(ang) : rad * cos(ang);
}

__global__ void k_factors(uint32_t seed, uint32_t obj, int n, int naux, double kappa, double* B)
{
    const long long total = (long long)naux * n * n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int q = (int)(e / ((long long)n * n));
        const int pq = (int)(e % ((long long)n * n));
        const int p = pq / n, r = pq % n;
        const double a = normal(seed, obj, q, 4u, (uint32_t)(p * n + r));
        const double b = normal(seed, obj, q, 4u, (uint32_t)(r * n + p));
        B[e] = kappa * (a + b) / 1.4142135623730951;
    }
}

}  // namespace

extern "C" int synth_factors(unsigned seed, unsigned obj, int n, int naux, double kappa, double* B, void* stream)
{
    const long long total = (long long)naux * n * n;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 8192) blocks = 8192;
    k_factors<<<blocks, 256, 0, (cudaStream_t)stream>>>(seed, obj, n, naux, kappa, B);
    return (int)cudaGetLastError();
}
