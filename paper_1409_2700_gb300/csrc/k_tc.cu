// k_tc.cu -- first half of the dimer transformation on the 5th-generation
// tensor cores (tcgen05, sm_103a), TF32 or BF16x3 operands, FP32 accumulate.
//
// Two kernels.  The "rank" kernel (further down; the one every supported
// size runs) contracts p2 on the tensor cores and applies p0 as a rank-1
// update in the epilogue.  The Kronecker kernel described here, selected
// only by MCPT_TC_KERNEL=kron, fuses both occupied quarter transformations
// of Eq. (dp2e) into one GEMM per dimer form (see internal.h for the axis
// naming):
//   H[(p1,p3)][(i,j)] = sum_{(p0,p2)} E[p0][p1][p2][p3] * W[(p0,p2)][(i,j)],
//   W[(p0,p2)][(i,j)] = C_X[p0][i] C_Y[p2][j]            (Kronecker product)
// M = rows (p1,p3) in tiles of 128, N = nocc_X*nocc_Y padded to 16, K = (p0,p2).
// It reads every AO integral exactly once and is bound by HBM: the padded
// tensor-core work (o_X o_Y / o_Y times the factorised flops) stays far below
// the time the integrals take to stream in.
//
// Per CTA (persistent, one per SM), warp roles:
//   warp 0     TMA producer: 4-D tensor-map loads of FP64 integral boxes
//              E[p0][p1 range][p2 chunk of 32][all p3] into a staging ring
//   warp 1     MMA issuer (one thread) and TMEM owner
//   warps 2-5  converters: FP64 -> TF32 (round to nearest) or BF16 hi/lo,
//              written as 128-row K-major SWIZZLE_128B operand tiles; they
//              also build the W tile of each K-block
//   warps 6-9  epilogue: tcgen05.ld of the FP32 accumulators -> global H
// Accumulators are double-buffered in TMEM so one work item drains while the
// next one accumulates.  Every wait is bounded by wall-clock time: on expiry
// the CTA records an error code, drains its own copies and MMAs, frees TMEM
// and returns.
#include "internal.h"
#include "convert.h"
#include "ff.h"

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <type_traits>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

namespace mcpt {

struct TcItem {
    int dimer;   // index within the launch's descriptor array
    int form;    // 0: A block, 1: K block
    int mt0;     // first M-tile
    int mts;     // number of M-tiles (accumulators) in this item
};

namespace {

constexpr int kWarps = 10;
constexpr int kThreadsTc = kWarps * 32;
constexpr int kKC = 32;              // p2 values per K-block (128 B of TF32 per operand row)
constexpr int kAccCols = 256;        // TMEM columns per accumulator set (x2 sets)
constexpr int kABytes = 128 * 128;   // one 128-row operand tile
constexpr unsigned long long kWaitNs = 4000000000ull;   // 4 s per wait

// error codes written to the status word
constexpr int kErrTimeoutBase = 0x100;

struct __align__(8) TcShared {
    unsigned long long full_f[8], empty_f[8];
    unsigned long long full_a[2], empty_a[2];
    unsigned long long full_w[2], empty_w[2];
    unsigned long long tmem_full[2], tmem_empty[2];
    unsigned long long drain;
    unsigned int tmem_base;
    volatile int abort;
};

struct TcParams {
    const TcItem* items;
    int n_items;
    const CUtensorMap* maps;       // [dimer][form]
    const DimerDesc* desc;
    const float* Cf;
    const double* Cd;              // FP64 coefficients (TC_FP64E)
    void* H;                       // float, or double for TC_FP64E (FP32 pairs with h_pairs)
    int h_pairs;                   // TC_FP64E: H written as FP32 pairs (the pair second half reads them)
    int* status;
    int sf;                        // FP64 staging stages
    unsigned int f_stage_bytes;    // bytes per staging slot
    unsigned int w_stage_bytes;    // bytes per W slot
    unsigned int tmem_cols;
    int kind;                      // TC_TF32 / TC_BF16X3 / TC_BF16X2 / TC_FP64E
    int kcs_max;                   // largest p2 chunk count of the launch (rank variant)
    unsigned long long wait_ns;    // limit of each wait (kWaitNs if 0)
    int withhold;                  // test aid: CTA 0 issues only withhold - 1 integral loads (0 = off)
};

// ------------------------------------------------------------------ PTX
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long now_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(unsigned long long* b, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned long long* b)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_tx(unsigned long long* b, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_test(unsigned long long* b, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase of parity `parity` to complete; false on timeout/abort.
__device__ __forceinline__ bool mbar_wait(unsigned long long* b, unsigned parity, volatile int* abort, int* status,
                                          int where, unsigned long long limit = kWaitNs)
{
    if (mbar_test(b, parity)) return true;
    const unsigned long long t0 = now_ns();
    while (true) {
        if (mbar_test(b, parity)) return true;
        if (*abort) return false;
        if (now_ns() - t0 > limit) {
            *abort = 1;
            atomicCAS(status, 0, kErrTimeoutBase + where);
            return false;
        }
    }
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Every AO integral is read exactly once, so the loads carry an L2
// evict-first policy: the stream then does not push out the first-half
// results (written a few rows at a time by many CTAs) before they are complete.
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, unsigned long long* bar, int c0,
                                            int c1, int c2, int c3)
{
    unsigned long long pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1, "
        "{%2, %3, %4, %5}], [%6], %7;" ::"r"(smem_u32(dst)),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar)), "l"(pol)
        : "memory");
}

__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_commit(unsigned long long* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

template <int KIND>
__device__ __forceinline__ void tc_mma(unsigned dtmem, unsigned long long adesc, unsigned long long bdesc,
                                       unsigned idesc, unsigned accum)
{
    if (KIND == TC_TF32)
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(
                dtmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
            : "memory");
    else
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
                dtmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
            : "memory");
}

// TMEM loads whose destination registers are produced only once the data
// has landed: the loads and tcgen05.wait::ld sit in one asm statement, so the
// compiler can neither read nor spill a destination while its load is pending.
// tmem_ld_l<L>x<J>: L loads of J columns, 16 columns apart, from taddr.
__device__ __forceinline__ void tmem_ld_l1x8(unsigned taddr, unsigned (&r)[8])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
        : "r"(taddr + 0u)
        : "memory");
}
__device__ __forceinline__ void tmem_ld_l1x16(unsigned taddr, unsigned (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr + 0u)
        : "memory");
}
__device__ __forceinline__ void tmem_ld_l2x8(unsigned taddr, unsigned (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%16];\n"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8, %9, %10, %11, %12, %13, %14, %15}, [%17];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr + 0u), "r"(taddr + 16u)
        : "memory");
}
__device__ __forceinline__ void tmem_ld_l3x8(unsigned taddr, unsigned (&r)[24])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%24];\n"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8, %9, %10, %11, %12, %13, %14, %15}, [%25];\n"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%16, %17, %18, %19, %20, %21, %22, %23}, [%26];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23])
        : "r"(taddr + 0u), "r"(taddr + 16u), "r"(taddr + 32u)
        : "memory");
}
__device__ __forceinline__ void tmem_ld_l3x16(unsigned taddr, unsigned (&r)[48])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%48];\n"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%49];\n"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47}, [%50];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47])
        : "r"(taddr + 0u), "r"(taddr + 16u), "r"(taddr + 32u)
        : "memory");
}
__device__ __forceinline__ void tmem_ld_l4x8(unsigned taddr, unsigned (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%32];\n"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8, %9, %10, %11, %12, %13, %14, %15}, [%33];\n"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%16, %17, %18, %19, %20, %21, %22, %23}, [%34];\n"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%24, %25, %26, %27, %28, %29, %30, %31}, [%35];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr + 0u), "r"(taddr + 16u), "r"(taddr + 32u), "r"(taddr + 48u)
        : "memory");
}
__device__ __forceinline__ void tmem_ld_l4x16(unsigned taddr, unsigned (&r)[64])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%64];\n"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%65];\n"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47}, [%66];\n"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%48, %49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, %61, %62, %63}, [%67];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]), "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
        : "r"(taddr + 0u), "r"(taddr + 16u), "r"(taddr + 32u), "r"(taddr + 48u)
        : "memory");
}
__device__ __forceinline__ void tmem_ld_l2x16(unsigned taddr, unsigned (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%32];\n"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%33];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr + 0u), "r"(taddr + 16u)
        : "memory");
}

// 32 lanes x 16 consecutive 32-bit columns per warp, as floats
__device__ __forceinline__ void tmem_ld16(unsigned taddr, float* v)
{
    unsigned r[16];
    tmem_ld_l1x16(taddr, r);
#pragma unroll
    for (int k = 0; k < 16; k++) v[k] = __uint_as_float(r[k]);
}

// TMEM stores of the accumulators that live in TMEM (tcgen05.wait::st before
// the columns are read again).
__device__ __forceinline__ void tmem_st16(unsigned taddr, const unsigned (&r)[16])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16};" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
        "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
        : "memory");
}
__device__ __forceinline__ void tmem_st8(unsigned taddr, const unsigned (&r)[8])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
                 "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
                 : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// K-major operand with SWIZZLE_128B: 8-row x 128-byte atoms stacked along the
// row dimension (stride 1024 B); the 16-byte chunk c of row r sits at chunk
// position c ^ (r % 8).  Matrix-descriptor fields: start address >> 4,
// leading-dimension offset (unused for this layout, 16 B), stride offset
// 1024 B >> 4, descriptor version 1, swizzle mode 2 (128 B).
__device__ __forceinline__ unsigned long long sw128_desc(const void* tile)
{
    const unsigned long long a = (smem_u32(tile) & 0x3FFFFu) >> 4;
    return a | (1ull << 16) | (64ull << 32) | (1ull << 46) | (2ull << 61);
}

__device__ __forceinline__ unsigned sw128_off(int row, int chunk)
{
    return (unsigned)((row >> 3) * 1024 + (row & 7) * 128 + ((chunk ^ (row & 7)) << 4));
}

// Instruction descriptor: D = F32, A/B = TF32 (2), BF16 (1) or FP16 (0, the
// FP64E digits), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__device__ __forceinline__ unsigned make_idesc(int kind, int N)
{
    const unsigned fmt = kind == TC_TF32 ? 2u : kind == TC_FP64E ? 0u : 1u;
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((unsigned)(N >> 3) << 17) | ((unsigned)(128 >> 4) << 24);
}

__device__ __forceinline__ unsigned to_tf32(float x)
{
    unsigned r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ unsigned short to_bf16_bits(float x)
{
    return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}

// Geometry of the current item, derived from its descriptor.
struct ItemGeo {
    int n0, n1, n2, n3;
    int o0, o2;
    int p1t;          // p1 values per M-tile
    int kcs;          // p2 chunks
    int kblocks;      // n0 * kcs
    int N;            // padded pair count (npad)
    int rows;         // n1 * n3
};

__device__ __forceinline__ ItemGeo geo_of(const DimerDesc& d, int f)
{
    ItemGeo g;
    g.n0 = d.nX;
    g.n1 = f ? d.nY : d.nX;
    g.n2 = d.nY;
    g.n3 = f ? d.nX : d.nY;
    g.o0 = d.oX;
    g.o2 = d.oY;
    g.p1t = 128 / g.n3;
    g.kcs = (g.n2 + kKC - 1) / kKC;
    g.kblocks = g.n0 * g.kcs;
    g.N = d.npad;
    g.rows = g.n1 * g.n3;
    return g;
}

// FP64 staging box [p1l][32 p2][n3] -> one 128-row K-major SW128 operand tile.
// TF32: 8 chunks of 4 p2 per row; BF16x3: hi in chunks 0-3, lo in chunks 4-7.
template <int KIND>
__device__ __forceinline__ void convert_a_tile(const double* F, unsigned char* A, int tile_rows_full, int n3, int ct)
{
    if (KIND == TC_TF32) {
        for (int task = ct; task < 128 * 8; task += 128) {
            const int c = task >> 7, r = task & 127;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (r < tile_rows_full) {
                const int p1l = r / n3, p3 = r % n3;
                const double* src = F + ((size_t)(p1l * kKC + c * 4) * n3 + p3);
                const unsigned* s32 = reinterpret_cast<const unsigned*>(src) + 1;   // high words
                v.x = tf32_from_f64_hi(s32[0]);
                v.y = tf32_from_f64_hi(s32[2 * n3]);
                v.z = tf32_from_f64_hi(s32[4 * n3]);
                v.w = tf32_from_f64_hi(s32[6 * n3]);
            }
            *reinterpret_cast<uint4*>(A + sw128_off(r, c)) = v;
        }
    } else {
        for (int task = ct; task < 128 * 4; task += 128) {
            const int c = task >> 7, r = task & 127;
            uint4 vh = make_uint4(0, 0, 0, 0), vl = make_uint4(0, 0, 0, 0);
            if (r < tile_rows_full) {
                const int p1l = r / n3, p3 = r % n3;
                const double* src = F + ((size_t)(p1l * kKC + c * 8) * n3 + p3);
                unsigned short hb[8], lb[8];
#pragma unroll
                for (int e = 0; e < 8; e++) {
                    const uint2 b = reinterpret_cast<const uint2*>(src)[e * n3];
                    const float x = f32_from_f64_bits(b.x, b.y);
                    hb[e] = to_bf16_bits(x);
                    lb[e] = to_bf16_bits(x - __bfloat162float(__ushort_as_bfloat16(hb[e])));
                }
                vh = make_uint4(hb[0] | (hb[1] << 16), hb[2] | (hb[3] << 16), hb[4] | (hb[5] << 16),
                                hb[6] | (hb[7] << 16));
                vl = make_uint4(lb[0] | (lb[1] << 16), lb[2] | (lb[3] << 16), lb[4] | (lb[5] << 16),
                                lb[6] | (lb[7] << 16));
            }
            *reinterpret_cast<uint4*>(A + sw128_off(r, c)) = vh;
            *reinterpret_cast<uint4*>(A + sw128_off(r, 4 + c)) = vl;
        }
    }
}

template <int KIND>
__global__ void __launch_bounds__(kThreadsTc, 1) k_half_tc(const TcParams P)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte aligned carve-out: [F ring][A ring][W ring][TcShared]
    unsigned char* base = (unsigned char*)(((size_t)smem_raw + 1023) & ~(size_t)1023);
    unsigned char* Fr = base;
    unsigned char* Ar = Fr + (size_t)P.sf * P.f_stage_bytes;
    unsigned char* Wr = Ar + 2 * kABytes;
    TcShared* sh = reinterpret_cast<TcShared*>(Wr + 2 * P.w_stage_bytes);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < P.sf; s++) { mbar_init(&sh->full_f[s], 1); mbar_init(&sh->empty_f[s], 4); }
        for (int s = 0; s < 2; s++) {
            mbar_init(&sh->full_a[s], 4); mbar_init(&sh->empty_a[s], 1);
            mbar_init(&sh->full_w[s], 4); mbar_init(&sh->empty_w[s], 1);
            mbar_init(&sh->tmem_full[s], 1); mbar_init(&sh->tmem_empty[s], 4);
        }
        mbar_init(&sh->drain, 1);
        sh->abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sh->tmem_base)),
                     "r"(P.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = sh->tmem_base;

    if (warp == 0) {
        // ------------------------------------------------ TMA producer
        if (lane == 0) {
            unsigned gF = 0;
            unsigned issued_phase[8];
            bool issued[8];
            for (int s = 0; s < 8; s++) issued[s] = false;
            for (int it = blockIdx.x; it < P.n_items && !sh->abort; it += gridDim.x) {
                const TcItem item = P.items[it];
                const DimerDesc& d = P.desc[item.dimer];
                const ItemGeo g = geo_of(d, item.form);
                const CUtensorMap* map = P.maps + 2 * item.dimer + item.form;
                const unsigned box = (unsigned)g.n3 * kKC * g.p1t * 8u;
                for (int kb = 0; kb < g.kblocks && !sh->abort; kb++) {
                    const int p0 = kb / g.kcs, kc = kb % g.kcs;
                    for (int mt = 0; mt < item.mts; mt++, gF++) {
                        const int s = gF % P.sf;
                        const unsigned ph = (gF / P.sf) & 1;
                        if (!mbar_wait(&sh->empty_f[s], ph ^ 1, &sh->abort, P.status, 1, P.wait_ns)) break;
                        mbar_arrive_tx(&sh->full_f[s], box);
                        tma_load_4d(Fr + (size_t)s * P.f_stage_bytes, map, &sh->full_f[s], 0, kc * kKC,
                                    (item.mt0 + mt) * g.p1t, p0);
                        issued[s] = true;
                        issued_phase[s] = ph;
                    }
                }
            }
            // copies in flight must land before the CTA may exit
            for (int s = 0; s < P.sf; s++)
                if (issued[s]) {
                    const unsigned long long t0 = now_ns();
                    while (!mbar_test(&sh->full_f[s], issued_phase[s]) && now_ns() - t0 < kWaitNs) {}
                }
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            unsigned gA = 0, gW = 0, li = 0;
            bool any = false;
            for (int it = blockIdx.x; it < P.n_items && !sh->abort; it += gridDim.x, li++) {
                const TcItem item = P.items[it];
                const ItemGeo g = geo_of(P.desc[item.dimer], item.form);
                const unsigned idesc = make_idesc(KIND, g.N);
                const int b = li & 1;
                if (!mbar_wait(&sh->tmem_empty[b], ((li >> 1) & 1) ^ 1, &sh->abort, P.status, 2, P.wait_ns)) break;
                tc_fence_after();
                bool ok = true;
                for (int kb = 0; kb < g.kblocks && ok; kb++, gW++) {
                    const int ws = gW & 1;
                    if (!(ok = mbar_wait(&sh->full_w[ws], (gW >> 1) & 1, &sh->abort, P.status, 3, P.wait_ns))) break;
                    const unsigned long long bdesc = sw128_desc(Wr + (size_t)ws * P.w_stage_bytes);
                    for (int mt = 0; mt < item.mts; mt++, gA++) {
                        const int as = gA & 1;
                        if (!(ok = mbar_wait(&sh->full_a[as], (gA >> 1) & 1, &sh->abort, P.status, 4, P.wait_ns))) break;
                        tc_fence_after();
                        const unsigned long long adesc = sw128_desc(Ar + (size_t)as * kABytes);
                        const unsigned dt = tmem + (unsigned)(b * kAccCols + mt * g.N);
                        if (KIND == TC_TF32) {
#pragma unroll
                            for (int k = 0; k < 4; k++)   // K = 8 per MMA: 32 bytes
                                tc_mma<KIND>(dt, adesc + 2 * k, bdesc + 2 * k, idesc, (kb > 0 || k > 0) ? 1u : 0u);
                        } else {
#pragma unroll
                            for (int k = 0; k < 2; k++) {   // K = 16 per MMA; hi at +0, lo at +64 bytes
                                const unsigned long long ah = adesc + 2 * k, al = adesc + 4 + 2 * k;
                                const unsigned long long bh = bdesc + 2 * k, bl = bdesc + 4 + 2 * k;
                                tc_mma<KIND>(dt, ah, bh, idesc, (kb > 0 || k > 0) ? 1u : 0u);
                                tc_mma<KIND>(dt, ah, bl, idesc, 1u);
                                tc_mma<KIND>(dt, al, bh, idesc, 1u);
                            }
                        }
                        tc_commit(&sh->empty_a[as]);
                        any = true;
                    }
                    if (ok) tc_commit(&sh->empty_w[ws]);
                }
                if (!ok) break;
                tc_commit(&sh->tmem_full[b]);
            }
            if (any) {
                // every issued MMA has retired before TMEM is released
                tc_commit(&sh->drain);
                const unsigned long long t0 = now_ns();
                while (!mbar_test(&sh->drain, 0) && now_ns() - t0 < kWaitNs) {}
            }
        }
    } else if (warp < 6) {
        // ------------------------------------------------ converters
        const int ct = threadIdx.x - 64;   // 0..127
        unsigned gF = 0, gA = 0, gW = 0;
        for (int it = blockIdx.x; it < P.n_items && !sh->abort; it += gridDim.x) {
            const TcItem item = P.items[it];
            const DimerDesc& d = P.desc[item.dimer];
            const ItemGeo g = geo_of(d, item.form);
            const float* CX = P.Cf + d.cX;
            const float* CY = P.Cf + d.cY;
            const int npairs = g.o0 * g.o2;
            const int tile_rows_full = g.p1t * g.n3;
            bool ok = true;
            for (int kb = 0; kb < g.kblocks && ok; kb++, gW++) {
                const int p0 = kb / g.kcs, kc = kb % g.kcs;
                // ---- W tile of this K-block: row n = (i, j), K = p2 in the chunk
                const int ws = gW & 1;
                if (!(ok = mbar_wait(&sh->empty_w[ws], ((gW >> 1) & 1) ^ 1, &sh->abort, P.status, 5, P.wait_ns))) break;
                unsigned char* W = Wr + (size_t)ws * P.w_stage_bytes;
                if (KIND == TC_TF32) {
                    for (int task = ct; task < g.N * 8; task += 128) {
                        const int n = task >> 3, c = task & 7;
                        uint4 v = make_uint4(0, 0, 0, 0);
                        if (n < npairs) {
                            const int i = n / g.o2, j = n % g.o2;
                            const float u0 = __ldg(CX + p0 * d.nX + i);
                            unsigned w4[4];
#pragma unroll
                            for (int e = 0; e < 4; e++) {
                                const int p2 = kc * kKC + c * 4 + e;
                                const float u2 = p2 < g.n2 ? __ldg(CY + p2 * d.nY + j) : 0.f;
                                w4[e] = to_tf32(u0 * u2);
                            }
                            v = make_uint4(w4[0], w4[1], w4[2], w4[3]);
                        }
                        *reinterpret_cast<uint4*>(W + sw128_off(n, c)) = v;
                    }
                } else {
                    for (int task = ct; task < g.N * 4; task += 128) {
                        const int n = task >> 2, c = task & 3;
                        uint4 vh = make_uint4(0, 0, 0, 0), vl = make_uint4(0, 0, 0, 0);
                        if (n < npairs) {
                            const int i = n / g.o2, j = n % g.o2;
                            const float u0 = __ldg(CX + p0 * d.nX + i);
                            unsigned short hb[8], lb[8];
#pragma unroll
                            for (int e = 0; e < 8; e++) {
                                const int p2 = kc * kKC + c * 8 + e;
                                const float w = p2 < g.n2 ? u0 * __ldg(CY + p2 * d.nY + j) : 0.f;
                                hb[e] = to_bf16_bits(w);
                                lb[e] = to_bf16_bits(w - __bfloat162float(__ushort_as_bfloat16(hb[e])));
                            }
                            vh = make_uint4(hb[0] | (hb[1] << 16), hb[2] | (hb[3] << 16), hb[4] | (hb[5] << 16),
                                            hb[6] | (hb[7] << 16));
                            vl = make_uint4(lb[0] | (lb[1] << 16), lb[2] | (lb[3] << 16), lb[4] | (lb[5] << 16),
                                            lb[6] | (lb[7] << 16));
                        }
                        *reinterpret_cast<uint4*>(W + sw128_off(n, c)) = vh;
                        *reinterpret_cast<uint4*>(W + sw128_off(n, 4 + c)) = vl;
                    }
                }
                fence_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(&sh->full_w[ws]);

                // ---- A tiles of this K-block, one per M-tile of the item
                for (int mt = 0; mt < item.mts; mt++, gF++, gA++) {
                    const int s = gF % P.sf;
                    if (!(ok = mbar_wait(&sh->full_f[s], (gF / P.sf) & 1, &sh->abort, P.status, 6, P.wait_ns))) break;
                    const int as = gA & 1;
                    if (!(ok = mbar_wait(&sh->empty_a[as], ((gA >> 1) & 1) ^ 1, &sh->abort, P.status, 7, P.wait_ns))) break;
                    const double* F = reinterpret_cast<const double*>(Fr + (size_t)s * P.f_stage_bytes);
                    unsigned char* A = Ar + (size_t)as * kABytes;
                    if (KIND == TC_TF32) {
                        // task = (row r, chunk c): 4 consecutive p2 of row r
                        for (int task = ct; task < 128 * 8; task += 128) {
                            const int c = task >> 7, r = task & 127;
                            uint4 v = make_uint4(0, 0, 0, 0);
                            if (r < tile_rows_full) {
                                const int p1l = r / g.n3, p3 = r % g.n3;
                                const double* src = F + ((size_t)(p1l * kKC + c * 4) * g.n3 + p3);
                                const unsigned* s32 = reinterpret_cast<const unsigned*>(src) + 1;   // high words
                                v.x = tf32_from_f64_hi(s32[0]);
                                v.y = tf32_from_f64_hi(s32[2 * g.n3]);
                                v.z = tf32_from_f64_hi(s32[4 * g.n3]);
                                v.w = tf32_from_f64_hi(s32[6 * g.n3]);
                            }
                            *reinterpret_cast<uint4*>(A + sw128_off(r, c)) = v;
                        }
                    } else {
                        for (int task = ct; task < 128 * 4; task += 128) {
                            const int c = task >> 7, r = task & 127;
                            uint4 vh = make_uint4(0, 0, 0, 0), vl = make_uint4(0, 0, 0, 0);
                            if (r < tile_rows_full) {
                                const int p1l = r / g.n3, p3 = r % g.n3;
                                const double* src = F + ((size_t)(p1l * kKC + c * 8) * g.n3 + p3);
                                unsigned short hb[8], lb[8];
#pragma unroll
                                for (int e = 0; e < 8; e++) {
                                    const uint2 b = reinterpret_cast<const uint2*>(src)[e * g.n3];
                                    const float x = f32_from_f64_bits(b.x, b.y);
                                    hb[e] = to_bf16_bits(x);
                                    lb[e] = to_bf16_bits(x - __bfloat162float(__ushort_as_bfloat16(hb[e])));
                                }
                                vh = make_uint4(hb[0] | (hb[1] << 16), hb[2] | (hb[3] << 16), hb[4] | (hb[5] << 16),
                                                hb[6] | (hb[7] << 16));
                                vl = make_uint4(lb[0] | (lb[1] << 16), lb[2] | (lb[3] << 16), lb[4] | (lb[5] << 16),
                                                lb[6] | (lb[7] << 16));
                            }
                            *reinterpret_cast<uint4*>(A + sw128_off(r, c)) = vh;
                            *reinterpret_cast<uint4*>(A + sw128_off(r, 4 + c)) = vl;
                        }
                    }
                    fence_async_smem();
                    __syncwarp();
                    if (lane == 0) {
                        mbar_arrive(&sh->full_a[as]);
                        mbar_arrive(&sh->empty_f[s]);
                    }
                }
            }
        }
    } else {
        // ------------------------------------------------ epilogue
        const int q = warp & 3;          // TMEM lane quarter this warp may access
        const int r = q * 32 + lane;     // accumulator row = TMEM lane
        unsigned li = 0;
        for (int it = blockIdx.x; it < P.n_items && !sh->abort; it += gridDim.x, li++) {
            const TcItem item = P.items[it];
            const DimerDesc& d = P.desc[item.dimer];
            const ItemGeo g = geo_of(d, item.form);
            const int b = li & 1;
            if (!mbar_wait(&sh->tmem_full[b], (li >> 1) & 1, &sh->abort, P.status, 8, P.wait_ns)) break;
            tc_fence_after();
            const int npairs = g.o0 * g.o2;
            float* Hf = static_cast<float*>(P.H) + d.h_off + (long long)item.form * npairs * g.rows;
            for (int mt = 0; mt < item.mts; mt++) {
                const int tile = item.mt0 + mt;
                const int p1_lo = tile * g.p1t;
                const int p1_hi = min(g.n1, p1_lo + g.p1t);
                const int valid = (p1_hi - p1_lo) * g.n3;
                float* out = Hf + p1_lo * g.n3 + r;
                for (int c = 0; c < g.N; c += 16) {
                    float v[16];
                    tmem_ld16(tmem + ((unsigned)(q * 32) << 16) + (unsigned)(b * kAccCols + mt * g.N + c), v);
                    if (r < valid) {
#pragma unroll
                        for (int k = 0; k < 16; k++)
                            if (c + k < npairs) out[(long long)(c + k) * g.rows] = v[k];
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&sh->tmem_empty[b]);
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(P.tmem_cols)
                     : "memory");
    }
}

// ==========================================================================
// "Rank" variant: the tensor core contracts only p2 for one (M-tile, p0) at a
// time,
//     T[(p1,p3)][j] = sum_{p2} E[p0][p1][p2][p3] C_Y[p2][j]      (N = 16 >= o2)
// accumulating over at most n2/8 MMA steps, into a ring of 16-column TMEM
// slots; the epilogue warps then apply the p0 quarter transformation as a
// rank-1 update in registers,
//     H[(p1,p3)][(i,j)] += C_X[p0][i] T[(p1,p3)][j],
// with round-to-nearest FP32 FMAs.  Long accumulations inside the tensor
// core do not round to nearest and drift toward zero over many steps; this
// split keeps each tensor-core sum short.  The B operand (C_Y's occupied
// columns) is constant per work item and reused for every p0 and row, so its
// rounding error would act as a slightly wrong orbital and bias the energy:
// it is split into two TF32 planes (hi + lo, two MMAs per step), which
// represents it to about FP32 accuracy; the integrals keep TF32's rounding,
// independent from element to element.
// BF16x3 goes further and makes every tensor-core sum exact.  Each operand
// vector is held in 32-bit fixed point relative to its largest power of two:
// an integral row (p1,p3) of one p0 over one chunk of 32 p2 values (each
// (p0, chunk) is a unit of its own), x ~ 2^(e-31) N_x, and a C_Y column j,
// c ~ 2^(f-31) N_c, |N| <= 2^32, cut into four balanced base-256
// digits N = d0 2^24 + d1 2^16 + d2 2^8 + d3 (|d0| <= 256, the others <= 128,
// each exact in BF16).  The digits come from the FP32 value by round-to-
// nearest-even FMAs (FP32 pipe), so every integral keeps its 24 FP32 bits
// unless it lies more than 2^8 below its row's largest.  The four levels
//     L0 = A0.B0, L1 = A0.B1 + A1.B0, L2 = A0.B2 + A1.B1 + A2.B0,
//     L3 = A0.B3 + A1.B2 + A2.B1 + A3.B0
// (four MMAs per K step: A_u times the stacked digit planes B_0..B_(3-u) of
// C_Y, N = 64, 48, 32, 16, landing in the four 16-column TMEM slots of levels
// u..3) are sums of at most
// 4 x 32 integer products per unit, each at most 2^16, so every partial sum
// is an integer below 2^24 and the tensor core adds them without rounding.
// The epilogue forms each unit's T = 2^(e+f-14) (L0 + 2^-8 L1 + 2^-16 L2 +
// 2^-24 L3) in FP32 with round-to-nearest and adds it into H through the
// rank-1 update (the chunks of a row are summed there, in FP32 with
// round-to-nearest); the dropped digit products lie below 2^-31 of the
// vectors' largest terms.
// BIG = false: the rank-1 accumulators live in registers (o_X, o_Y <= 8),
// T slots use all 512 TMEM columns.  BIG = true (o_X, o_Y <= 16): the
// accumulators live in TMEM columns 256-511 (row r = lane r, column
// 256 + 16 i + j) and the epilogue updates them four occupied i at a time
// (tcgen05.ld, FFMA, tcgen05.st); the T ring shrinks to 16 slots.
constexpr int kNT = 16;           // TMEM slot width = MMA N
constexpr int kSlots = 32;        // 32 x 16 = 512 TMEM columns (16 slots when BIG)
constexpr int kFxUnits = 8;       // BF16x3: 4-slot p0 units in 512 columns (4 when BIG)
constexpr int kOB = 8;            // register accumulator block: o_X, o_Y <= 8
constexpr int kOB5 = 5;           // the same sized for o_X, o_Y <= 5 (fewer rank-1 FMAs)
constexpr int kFp64eMaxAO = 64;   // FP64E: p2 chunks <= 2, so that its three-tile A ring fits
constexpr int kKCMax = 4;         // p2 chunks: n2 <= 128
constexpr int kConvWarps = 8;     // converter warps per group: one unit (128 rows) per group
// Groups of converter warps take alternate units.  The variants with
// occupations <= 5 and with TMEM accumulators run two (four converter warps
// per SM sub-partition: the converters are latency bound) within the register
// budget that 22 warps leave; the 8 x 8 register variant keeps one group and
// the larger per-thread budget.
// The TMEM-accumulator variant runs two as well (its epilogue keeps T and a
// two-row block of accumulators in registers).  FP64E keeps one group: its
// epilogue's FP32-pair accumulators need the larger per-thread budget.  Its
// epilogue, latency bound on dependent pair arithmetic, runs as eight warps:
// two per TMEM lane quarter, each with part of the occupied columns j.
template <bool BIG, int OB, int KIND = TC_TF32>
__host__ __device__ constexpr int conv_groups() { return ((BIG || OB == 5) && KIND != TC_FP64E) ? 2 : 1; }
template <int KIND>
__host__ __device__ constexpr int epi_warps() { return KIND == TC_FP64E ? 8 : 4; }
template <bool BIG, int OB, int KIND = TC_TF32>
__host__ __device__ constexpr int rank_threads()
{
    return (2 + kConvWarps * conv_groups<BIG, OB, KIND>() + epi_warps<KIND>()) * 32;
}
constexpr int kFFCols = 3;        // FP64E: occupied columns j per epilogue warp (two warps cover o_Y <= 5)
constexpr int kOBig = 16;         // TMEM accumulators: o_X, o_Y <= 16
constexpr int kOBigI = 20;        // wide TMEM accumulators (OB = kOBigI): o_X <= 20, o_Y <= 16, at
                                  // columns 192-511 (three T units below instead of four)
// C_X occupied rows of one item (n0 <= 128), per parity: the register
// accumulator kernel stages kOB columns (FP64E: each as an FP32 pair), the
// TMEM one kOBig (24 for the wide form: o_X <= 20, float2-aligned rows).
__host__ __device__ constexpr int cx_floats(bool big, int kind = TC_TF32, bool wide = false)
{
    return 128 * (big ? (wide ? 24 : kOBig) : kOB) * (kind == TC_FP64E ? 2 : 1);
}

struct __align__(8) RankShared {
    unsigned long long full_f[8], empty_f[8];
    unsigned long long full_a[2], empty_a[2];
    unsigned long long full_w[2], empty_w[2];
    unsigned long long cx_full[2], cx_empty[2];
    unsigned long long slot_full[kSlots], slot_empty[kSlots];
    unsigned long long exp_full[kFxUnits];   // BF16x3: unit scales written
    unsigned long long colx_full[2];         // BF16x3: column exponent partials written
    unsigned long long drain;
    unsigned int tmem_base;
    volatile int abort;
};

// TMEM columns of one p0 unit and units in the ring (FP64E: seven levels).
template <int KIND, bool BIG>
__host__ __device__ constexpr int unit_cols() { return KIND == TC_FP64E ? 7 * kNT : KIND != TC_TF32 ? 4 * kNT : kNT; }
template <int KIND, bool BIG, int OB = kOB>
__host__ __device__ constexpr int n_units() { return (BIG ? (OB > kOBig ? 192 : 256) : 512) / unit_cols<KIND, BIG>(); }
// Shared bytes of the A ring (two slots; BF16x3 uses two tiles per slot,
// FP64E three) and of the fixed-point unit scales (row scales 128 + column
// scales 16 per unit).
__host__ __device__ constexpr size_t a_ring_bytes(int kind)
{
    return 2 * (size_t)kABytes * (kind == TC_FP64E ? 3 : kind == TC_BF16X3 ? 2 : 1);
}
// Bytes of one parity of the B operand (C_Y's occupied columns) for an item
// of kcs_max p2 chunks.  TF32: per chunk two 16-row planes (hi, lo).  BF16x3:
// per pair of chunks one 64-row tile, row 16 v + j = digit v of column j,
// chunk kc in bytes 64 (kc % 2) .. +63 of the row.  FP64E: the same with six
// digits and a seventh all-zero plane, 112 rows per pair of chunks.
__host__ __device__ constexpr int w_rows(int kind) { return kind == TC_FP64E ? 112 : 64; }
__host__ __device__ constexpr size_t w_stride_bytes(int kind, int kcs_max)
{
    return kind != TC_TF32 ? (size_t)((kcs_max + 1) / 2) * w_rows(kind) * 128 : (size_t)kcs_max * 2 * kNT * 128;
}
__host__ __device__ constexpr size_t fx_scale_bytes(int kind)
{
    return kind != TC_TF32 ? kFxUnits * (128 + kNT) * 4 + 2 * 16 * kNT * 4 : 0;
}

// ---- BF16x3 fixed-point digits
// Round-to-nearest-even integer of |v| < 2^22 by the FP32 magic constant
// 1.5 * 2^23 (one FMA with the scale, one subtraction).
__device__ __forceinline__ float rint_scaled(float v, float scale)
{
    return fmaf(v, scale, 12582912.0f) - 12582912.0f;
}
// Balanced base-256 digits of y (|y| <= 2^32, an FP32 value scaled to the
// vector's fixed point): y ~ d0 2^24 + d1 2^16 + d2 2^8 + d3, the last digit
// rounded to nearest; every remainder is exact (FMA of a digit multiple).
__device__ __forceinline__ void digits4(float y, float (&d)[4])
{
    d[0] = rint_scaled(y, 0x1p-24f);
    y = fmaf(-d[0], 16777216.0f, y);
    d[1] = rint_scaled(y, 0x1p-16f);
    y = fmaf(-d[1], 65536.0f, y);
    d[2] = rint_scaled(y, 0x1p-8f);
    y = fmaf(-d[2], 256.0f, y);
    d[3] = rint_scaled(y, 1.0f);
}
// digits4 for two values at once with the packed FP32 instructions of sm_100+
// (one issue per pair of lanes' values): the same operations, elementwise.
__device__ __forceinline__ float2 rint_scaled2(float2 v, float scale)
{
    const float2 m = make_float2(12582912.0f, 12582912.0f);
    return __fadd2_rn(__ffma2_rn(v, make_float2(scale, scale), m), make_float2(-12582912.0f, -12582912.0f));
}
__device__ __forceinline__ void digits4x2(float2 y, float2 (&d)[4])
{
    d[0] = rint_scaled2(y, 0x1p-24f);
    y = __ffma2_rn(d[0], make_float2(-16777216.0f, -16777216.0f), y);
    d[1] = rint_scaled2(y, 0x1p-16f);
    y = __ffma2_rn(d[1], make_float2(-65536.0f, -65536.0f), y);
    d[2] = rint_scaled2(y, 0x1p-8f);
    y = __ffma2_rn(d[2], make_float2(-256.0f, -256.0f), y);
    d[3] = rint_scaled2(y, 1.0f);
}

// Two BF16 digits (exact: integers of at most 9 bits) packed low | high.
__device__ __forceinline__ unsigned pack_bf16(float lo, float hi)
{
    return __byte_perm(__float_as_uint(lo), __float_as_uint(hi), 0x7632);
}
// An FP64 row element scaled to the row's 32-bit fixed point, y = x 2^(31-e)
// with e = emax - 1023, as FP32 (mantissa rounded half away from zero),
// built from the bit fields on the integer pipes: the double's exponent and
// leading 23 mantissa bits shifted into FP32 position, the exponent offset
// 158 - emax added modulo 2^9 (exact, the result lies in [1, 158]), the sign
// put back.  Elements below 2^-157 of the row's largest (and every element of
// a row marked invalid) become 0.
struct FxRow {
    unsigned add;   // (158 - emax) << 23, modulo 2^32
    unsigned thr;   // |hi| below this flushes to 0
};
__device__ __forceinline__ FxRow fx_row(int emax, bool valid)
{
    FxRow f;
    f.add = (unsigned)((158 - emax) & 511) << 23;
    f.thr = valid ? (unsigned)max(1, emax - 157) << 20 : 0xFFFFFFFFu;
    return f;
}
__device__ __forceinline__ float fx_y(unsigned lo, unsigned hi, FxRow f)
{
    unsigned w = __funnelshift_l(lo, hi, 3) + f.add + ((lo >> 28) & 1u);
    w = (w & 0x7FFFFFFFu) | (hi & 0x80000000u);
    return (hi & 0x7FFFFFFFu) < f.thr ? 0.f : __uint_as_float(w);
}
// The same for an FP32 vector (f = fmax - 127).
__device__ __forceinline__ float fx_scale_f32(int fmax)
{
    return (fmax >= 31 && fmax <= 254) ? __uint_as_float((unsigned)(285 - fmax) << 23) : 0.f;
}
// 2^(e - 7) with e = emax - 1023, the row's share of the product scale
// (0 where the row's digits are zero).
__device__ __forceinline__ float row_scale(int emax)
{
    return emax >= 927 ? __uint_as_float((unsigned)(emax - 903) << 23) : 0.f;
}
// 2^(f - 7) with f = fmax - 127.
__device__ __forceinline__ float col_scale(int fmax)
{
    return fmax >= 31 ? __uint_as_float((unsigned)(fmax - 7) << 23) : 0.f;
}

// A converter thread's fixed share of every A tile of an item: row r of the
// 128-row tile and where that row's integrals sit in the FP64 staging box.
struct ConvRow {
    int src;        // element offset of (p1l, p2 = 0, p3) in the box
    unsigned dst;   // byte offset of row r's 128-byte line in the tile
    int r7;         // swizzle phase of the row
    bool valid;
};

__device__ __forceinline__ ConvRow conv_row(int r, int tile_rows_full, int n3)
{
    ConvRow c;
    c.valid = r < tile_rows_full;
    const int p1l = c.valid ? r / n3 : 0, p3 = c.valid ? r % n3 : 0;
    c.src = p1l * kKC * n3 + p3;
    c.dst = (unsigned)((r >> 3) * 1024 + (r & 7) * 128);
    c.r7 = r & 7;
    return c;
}

// Row r of one A tile, chunks c0, c0+2, ... (the two converter threads of a
// row split the 128-byte line).  TF32: 4 chunks of 4 p2 from the high words
// of the doubles; BF16x3: 2 chunks of 8 p2, hi in chunk c and lo in 4 + c.
template <int KIND>
__device__ __forceinline__ void convert_row(const double* __restrict__ F, unsigned char* __restrict__ A,
                                            const ConvRow& cr, int n3, int c0)
{
    if (KIND == TC_TF32) {
        const unsigned* __restrict__ hw = reinterpret_cast<const unsigned*>(F + cr.src) + 1;
        unsigned v[4][4];
#pragma unroll
        for (int q = 0; q < 4; q++)
#pragma unroll
            for (int e = 0; e < 4; e++) {
                const unsigned w = hw[2 * ((c0 + 2 * q) * 4 + e) * n3];
                v[q][e] = cr.valid ? tf32_from_f64_hi(w) : 0u;
            }
#pragma unroll
        for (int q = 0; q < 4; q++)
            *reinterpret_cast<uint4*>(A + cr.dst + (((c0 + 2 * q) ^ cr.r7) << 4)) =
                make_uint4(v[q][0], v[q][1], v[q][2], v[q][3]);
    } else {
        const uint2* __restrict__ dw = reinterpret_cast<const uint2*>(F + cr.src);
        unsigned hv[2][4], lv[2][4];
#pragma unroll
        for (int q = 0; q < 2; q++) {
            const int c = c0 + 2 * q;
#pragma unroll
            for (int e = 0; e < 8; e += 2) {
                unsigned short hb[2], lb[2];
#pragma unroll
                for (int u = 0; u < 2; u++) {
                    const uint2 b = dw[(c * 8 + e + u) * n3];
                    const float x = cr.valid ? f32_from_f64_bits(b.x, b.y) : 0.f;
                    hb[u] = to_bf16_bits(x);
                    lb[u] = to_bf16_bits(x - __bfloat162float(__ushort_as_bfloat16(hb[u])));
                }
                hv[q][e / 2] = hb[0] | ((unsigned)hb[1] << 16);
                lv[q][e / 2] = lb[0] | ((unsigned)lb[1] << 16);
            }
        }
#pragma unroll
        for (int q = 0; q < 2; q++) {
            const int c = c0 + 2 * q;
            *reinterpret_cast<uint4*>(A + cr.dst + ((c ^ cr.r7) << 4)) = make_uint4(hv[q][0], hv[q][1], hv[q][2], hv[q][3]);
            *reinterpret_cast<uint4*>(A + cr.dst + (((4 + c) ^ cr.r7) << 4)) =
                make_uint4(lv[q][0], lv[q][1], lv[q][2], lv[q][3]);
        }
    }
}

// Digit levels the epilogue combines: BF16x3 four, BF16x2 three (its fourth,
// A0 B3 + A1 B2, lies 2^-24 below the first and is not formed).
template <int KIND>
__host__ __device__ constexpr int n_levels()
{
    return KIND == TC_FP64E ? 7 : KIND == TC_BF16X3 ? 4 : KIND == TC_BF16X2 ? 3 : 1;
}

// T[(p1,p3) = this lane's row][j < NJ] of one unit, written to T (add =
// false) or added to it.  TF32: the slot itself.  Fixed-point forms: the
// digit levels, loaded together, combined in FP32 (round to nearest) as
// ((L3/256 + L2)/256 + L1)/256 + L0, times the unit's row scale and, with
// COLS, the item's column scales (without, the caller applies those once
// per output).
template <int KIND, int NJ, bool COLS>
__device__ __forceinline__ void unit_T(unsigned taddr, float (&T)[NJ], const float* srow, const float* scol, bool add)
{
    constexpr int NL = n_levels<KIND>();
    if constexpr (NJ == 16 && NL > 1) {
        // TMEM-accumulator kernel: the levels one at a time (16 registers each),
        // combined in the same order as below
        float v[NJ];
        {
            unsigned raw[NJ];
            tmem_ld_l1x16(taddr + 16u * (NL - 1), raw);
#pragma unroll
            for (int j = 0; j < NJ; j++) v[j] = __uint_as_float(raw[j]);
        }
#pragma unroll
        for (int l = NL - 2; l >= 0; l--) {
            unsigned raw[NJ];
            tmem_ld_l1x16(taddr + 16u * l, raw);
#pragma unroll
            for (int j = 0; j < NJ; j++) v[j] = fmaf(v[j], 0x1p-8f, __uint_as_float(raw[j]));
        }
        const float sr = *srow;
#pragma unroll
        for (int j = 0; j < NJ; j++) {
            const float f = COLS ? sr * scol[j] : sr;
            T[j] = add ? fmaf(v[j], f, T[j]) : v[j] * f;
        }
        return;
    }
    unsigned raw[NL][NJ];
    unsigned(&flat)[NL * NJ] = *reinterpret_cast<unsigned(*)[NL * NJ]>(&raw[0][0]);
    if constexpr (NL == 1 && NJ == 8) tmem_ld_l1x8(taddr, flat);
    else if constexpr (NL == 1 && NJ == 16) tmem_ld_l1x16(taddr, flat);
    else if constexpr (NL == 3 && NJ == 8) tmem_ld_l3x8(taddr, flat);
    else if constexpr (NL == 3 && NJ == 16) tmem_ld_l3x16(taddr, flat);
    else if constexpr (NL == 4 && NJ == 8) tmem_ld_l4x8(taddr, flat);
    else tmem_ld_l4x16(taddr, flat);
    if constexpr (KIND == TC_TF32) {
#pragma unroll
        for (int j = 0; j < NJ; j++) T[j] = add ? T[j] + __uint_as_float(raw[0][j]) : __uint_as_float(raw[0][j]);
    } else {
        float v[NJ];
#pragma unroll
        for (int j = 0; j < NJ; j++) v[j] = __uint_as_float(raw[NL - 1][j]);
#pragma unroll
        for (int l = NL - 2; l >= 0; l--)
#pragma unroll
            for (int j = 0; j < NJ; j++) v[j] = fmaf(v[j], 0x1p-8f, __uint_as_float(raw[l][j]));
        const float sr = *srow;
#pragma unroll
        for (int j = 0; j < NJ; j++) {
            const float f = COLS ? sr * scol[j] : sr;
            T[j] = add ? fmaf(v[j], f, T[j]) : v[j] * f;
        }
    }
}

// BF16x3: row r of one staged box (one p2 chunk of one p0) as four digit
// planes, chunks c0 and c0 + 2 of 8 p2 each: tile 1 holds [d0 | d1] (bytes
// 0-63 / 64-127), tile 2 [d2 | d3].  The thread's 16 values are loaded once;
// the row's largest magnitude over the chunk is their bitwise maximum (|x|
// orders like its bit pattern) combined with the partner lane (l ^ 16), which
// fixes the chunk's fixed point.  Returns the row's exponent field.
__device__ __forceinline__ int convert_row_fx1(const double* __restrict__ F, unsigned char* __restrict__ A1,
                                               unsigned char* __restrict__ A2, const ConvRow& cr, int n3, int c0)
{
    const uint2* __restrict__ dw = reinterpret_cast<const uint2*>(F + cr.src);
    uint2 v[2][8];
    unsigned m = 0;
#pragma unroll
    for (int q = 0; q < 2; q++)
#pragma unroll
        for (int e = 0; e < 8; e++) {
            v[q][e] = dw[((c0 + 2 * q) * 8 + e) * n3];
            m = max(m, v[q][e].y & 0x7FFFFFFFu);
        }
    m = max(m, __shfl_xor_sync(0xffffffffu, m, 16));
    const int emax = cr.valid ? (int)(m >> 20) : 0;
    const FxRow fr = fx_row(emax, cr.valid);
#pragma unroll
    for (int q = 0; q < 2; q++) {
        const int c = c0 + 2 * q;
        unsigned w[4][4];
#pragma unroll
        for (int e = 0; e < 8; e += 2) {
            float2 d[4];
            digits4x2(make_float2(fx_y(v[q][e].x, v[q][e].y, fr), fx_y(v[q][e + 1].x, v[q][e + 1].y, fr)), d);
#pragma unroll
            for (int k = 0; k < 4; k++) w[k][e / 2] = pack_bf16(d[k].x, d[k].y);
        }
        *reinterpret_cast<uint4*>(A1 + cr.dst + ((c ^ cr.r7) << 4)) = make_uint4(w[0][0], w[0][1], w[0][2], w[0][3]);
        *reinterpret_cast<uint4*>(A1 + cr.dst + (((4 + c) ^ cr.r7) << 4)) =
            make_uint4(w[1][0], w[1][1], w[1][2], w[1][3]);
        *reinterpret_cast<uint4*>(A2 + cr.dst + ((c ^ cr.r7) << 4)) = make_uint4(w[2][0], w[2][1], w[2][2], w[2][3]);
        *reinterpret_cast<uint4*>(A2 + cr.dst + (((4 + c) ^ cr.r7) << 4)) =
            make_uint4(w[3][0], w[3][1], w[3][2], w[3][3]);
    }
    return emax;
}

// BF16x2: row r of one staged box as the two digit planes of a 16-bit fixed
// point, tile [d0 | d1] (bytes 0-63 / 64-127), chunks c0 and c0 + 2 of 8 p2.
// Only the high word of each double is read: its 20 mantissa bits hold every
// bit above the rounding position.  The row chunk's largest exponent field
// emax (bitwise maximum of |hi|, combined with the partner lane l ^ 16) fixes
// y = x 2^(15 - e), e = emax - 1023, built on the integer pipes: the
// exponent field lowered by emax - 142 while still 11 bits wide (elements
// below 2^-142 of the row's largest, zeros and invalid rows go negative and
// are clamped to 0), then moved into FP32 position.  The lowest FP32
// mantissa bit of y is set: it stands in for the dropped low word, so a
// truncated value never sits exactly on a rounding tie and round-to-nearest
// gives the correctly rounded digits of the full double, for either sign.
// Balanced digits 2^8 d0 + d1 = rn(y): d0 = rn(y / 2^8) in [-256, 256],
// d1 = rn(y - 2^8 d0) in [-128, 128], both exact in BF16.
__device__ __forceinline__ int convert_row_fx2(const double* __restrict__ F, unsigned char* __restrict__ A,
                                               const ConvRow& cr, int n3, int c0)
{
    const unsigned* __restrict__ hw = reinterpret_cast<const unsigned*>(F + cr.src) + 1;
    unsigned h[2][8];
    unsigned m = 0;
#pragma unroll
    for (int q = 0; q < 2; q++)
#pragma unroll
        for (int e = 0; e < 8; e++) {
            h[q][e] = hw[2 * ((c0 + 2 * q) * 8 + e) * n3];
            m = max(m, h[q][e] & 0x7FFFFFFFu);
        }
    m = max(m, __shfl_xor_sync(0xffffffffu, m, 16));
    const int emax = cr.valid ? (int)(m >> 20) : 0;
    // |hi| - K keeps the FP32 exponent field e_d - emax + 142 in bits 20-30 (negative
    // below zero); an invalid row subtracts more than any |hi| so that all of it clamps to 0
    const int K = cr.valid ? (emax - 142) * (1 << 20) : 0x7FFFFFFF;
    const float2 magic = make_float2(12582912.0f, 12582912.0f);      // 1.5 * 2^23
    const float2 nmagic = make_float2(-12582912.0f, -12582912.0f);
#pragma unroll
    for (int q = 0; q < 2; q++) {
        const int c = c0 + 2 * q;
        unsigned w0[4], w1[4];
#pragma unroll
        for (int e = 0; e < 8; e += 2) {
            float2 y;
            {
                const unsigned ha = h[q][e], hb = h[q][e + 1];
                const int ta = max((int)(ha & 0x7FFFFFFFu) - K, 0), tb = max((int)(hb & 0x7FFFFFFFu) - K, 0);
                y.x = __uint_as_float(((unsigned)ta << 3) | 1u | (ha & 0x80000000u));
                y.y = __uint_as_float(((unsigned)tb << 3) | 1u | (hb & 0x80000000u));
            }
            const float2 d0 = __fadd2_rn(__ffma2_rn(y, make_float2(0x1p-8f, 0x1p-8f), magic), nmagic);
            const float2 r = __ffma2_rn(d0, make_float2(-256.0f, -256.0f), y);        // exact
            const float2 d1 = __fadd2_rn(__fadd2_rn(r, magic), nmagic);
            w0[e / 2] = pack_bf16(d0.x, d0.y);
            w1[e / 2] = pack_bf16(d1.x, d1.y);
        }
        *reinterpret_cast<uint4*>(A + cr.dst + ((c ^ cr.r7) << 4)) = make_uint4(w0[0], w0[1], w0[2], w0[3]);
        *reinterpret_cast<uint4*>(A + cr.dst + (((4 + c) ^ cr.r7) << 4)) = make_uint4(w1[0], w1[1], w1[2], w1[3]);
    }
    return emax;
}

// ---- FP64E: six unsigned byte digits of a 48-bit fixed point
// |x| of an FP64 vector element relative to the vector's largest exponent
// field emax: N = floor(|x| 2^(47 - e)), e = emax - 1023, so |x| = N 2^(e-47)
// less at most one unit (2^-47 of the vector's largest power of two), and
// N < 2^48, returned as nh (16 bits) : nl.  Integer pipes only: the 53-bit
// significand shifted right by emax - ex + 5 >= 5 (two clamped funnel shifts
// cover every distance up to 64).  Zeros and FP64 denormals give N = 0, and
// so does every element when emax is 0 (an invalid or all-zero vector).
__device__ __forceinline__ void fx48(unsigned lo, unsigned hi, int emax, unsigned& nh, unsigned& nl)
{
    const int ex = (int)((hi >> 20) & 0x7FFu);
    const unsigned mh = (hi & 0xFFFFFu) | 0x100000u;
    const unsigned sh = ex ? (unsigned)(emax - ex + 5) : 64u;   // ex > emax only for emax = 0: huge
    const unsigned s1 = min(sh, 32u);
    nh = __funnelshift_rc(mh, 0u, s1);
    nl = __funnelshift_rc(__funnelshift_rc(lo, mh, s1), 0u, sh - s1);
}

// Byte k of wa and of wb as two exact FP16 values packed low | high, each
// with its element's sign: a byte permute puts the bytes in the low byte of
// each half, one three-input logic operation keeps them and sets the FP16
// bits of +-(1024 + b) (0x6400 | b, sign from `magic`), one packed FP16
// addition of -+1024 (`off`) leaves +-b, exact (every value involved is an
// FP16 integer below 2048).
__device__ __forceinline__ unsigned f16_digit_pair(unsigned wa, unsigned wb, unsigned k, unsigned magic, unsigned off)
{
    const unsigned t = (__byte_perm(wa, wb, k | ((4u + k) << 8)) & 0x00FF00FFu) | magic;
    const __half2 r = __hadd2(*reinterpret_cast<const __half2*>(&t), *reinterpret_cast<const __half2*>(&off));
    return *reinterpret_cast<const unsigned*>(&r);
}

// The six digit planes of two consecutive elements (a, b) of one vector:
// N = d0 2^40 + d1 2^32 + d2 2^24 + d3 2^16 + d4 2^8 + d5, each digit an
// FP16 integer carrying its element's sign; w[v] = digit v of (a | b << 16).
__device__ __forceinline__ void digits6_pair(uint2 a, uint2 b, int emax, unsigned (&w)[6])
{
    unsigned ha, la, hb, lb;
    fx48(a.x, a.y, emax, ha, la);
    fx48(b.x, b.y, emax, hb, lb);
    const unsigned sg = ((a.y >> 16) & 0x8000u) | (b.y & 0x80000000u);
    const unsigned magic = 0x64006400u | sg;        // +-(1024 + b) once the bytes are in
    const unsigned off = 0xE400E400u ^ sg;          // -1024 where positive, +1024 where negative
    w[0] = f16_digit_pair(ha, hb, 1u, magic, off);
    w[1] = f16_digit_pair(ha, hb, 0u, magic, off);
    w[2] = f16_digit_pair(la, lb, 3u, magic, off);
    w[3] = f16_digit_pair(la, lb, 2u, magic, off);
    w[4] = f16_digit_pair(la, lb, 1u, magic, off);
    w[5] = f16_digit_pair(la, lb, 0u, magic, off);
}

// FP64E: row r of one staged box as the six digit planes of its 48-bit fixed
// point, tiles [d0 | d1], [d2 | d3], [d4 | d5] (bytes 0-63 / 64-127 of each
// 128-byte row), chunks c0 and c0 + 2 of 8 p2.  Both words of each double are
// read; the row chunk's largest exponent field (bitwise maximum of |hi|,
// combined with the partner lane l ^ 16) fixes the fixed point.  Returns it.
__device__ __forceinline__ int convert_row_fx6(const double* __restrict__ F, unsigned char* __restrict__ A,
                                               const ConvRow& cr, int n3, int c0)
{
    // two passes over the thread's 16 elements (shared memory, cheap to read
    // again): the high words for the row maximum, then each chunk of 8
    // converted from both words -- half the live registers of one pass
    const uint2* __restrict__ dw = reinterpret_cast<const uint2*>(F + cr.src);
    const unsigned* __restrict__ hw = reinterpret_cast<const unsigned*>(F + cr.src) + 1;
    unsigned m = 0;
#pragma unroll
    for (int q = 0; q < 2; q++)
#pragma unroll
        for (int e = 0; e < 8; e++) m = max(m, hw[2 * ((c0 + 2 * q) * 8 + e) * n3] & 0x7FFFFFFFu);
    m = max(m, __shfl_xor_sync(0xffffffffu, m, 16));
    const int emax = cr.valid ? (int)(m >> 20) : 0;
#pragma unroll
    for (int q = 0; q < 2; q++) {
        const int c = c0 + 2 * q;
        unsigned w[6][4];
#pragma unroll
        for (int e = 0; e < 8; e += 2) {
            unsigned d[6];
            digits6_pair(dw[(c * 8 + e) * n3], dw[(c * 8 + e + 1) * n3], emax, d);
#pragma unroll
            for (int k = 0; k < 6; k++) w[k][e / 2] = d[k];
        }
#pragma unroll
        for (int t = 0; t < 3; t++) {
            unsigned char* At = A + (size_t)t * kABytes + cr.dst;
            *reinterpret_cast<uint4*>(At + ((c ^ cr.r7) << 4)) =
                make_uint4(w[2 * t][0], w[2 * t][1], w[2 * t][2], w[2 * t][3]);
            *reinterpret_cast<uint4*>(At + (((4 + c) ^ cr.r7) << 4)) =
                make_uint4(w[2 * t + 1][0], w[2 * t + 1][1], w[2 * t + 1][2], w[2 * t + 1][3]);
        }
    }
    return emax;
}

// FP64E: the seven digit levels of one unit for this lane's row, columns
// J0 .. J0 + NJ - 1, combined into FP32 pairs: S = L6, then S = S 2^-8 + L_k
// for k = 5 .. 0 (each L_k an exact integer below 2^24, the scaling exact,
// the addition a TwoSum), times the unit's row scale (a power of two).  The
// column scales are applied once per output.
template <int NJ, int J0 = 0>
__device__ __forceinline__ void unit_T_ff(unsigned taddr, FF (&T)[8], float srow, bool add)
{
    // Levels 6-3 in plain FP32 (three FMAs: their sum carries weight 2^-24,
    // so its rounding lies near 2^-48 of the fixed point's full scale 2^24 --
    // an absolute error the size of the digits' own truncation), then
    // the Horner steps of levels 2-0 on pairs.  S.l shrinks by 2^8 per step
    // while each new TwoSum error is below ulp(S.h) / 2, so it stays within
    // ulp(S.h) without renormalising (once, at the end).  Levels are loaded
    // three, one and three at a time.
    FF S[NJ];
    {
        unsigned hi[3][8];   // L4, L5, L6
        tmem_ld_l3x8(taddr + 64u, *reinterpret_cast<unsigned(*)[24]>(&hi[0][0]));
#pragma unroll
        for (int j = 0; j < NJ; j++)
            S[j].h = fmaf(fmaf(__uint_as_float(hi[2][J0 + j]), 0x1p-8f, __uint_as_float(hi[1][J0 + j])), 0x1p-8f,
                          __uint_as_float(hi[0][J0 + j]));
    }
    {
        unsigned l3[8];
        tmem_ld_l1x8(taddr + 48u, l3);
#pragma unroll
        for (int j = 0; j < NJ; j++) S[j] = FF{fmaf(S[j].h, 0x1p-8f, __uint_as_float(l3[J0 + j])), 0.f};
    }
    {
        unsigned lv[3][8];   // L0, L1, L2
        tmem_ld_l3x8(taddr, *reinterpret_cast<unsigned(*)[24]>(&lv[0][0]));
#pragma unroll
        for (int k = 2; k >= 0; k--)
#pragma unroll
            for (int j = 0; j < NJ; j++) {
                float e;
                S[j].h = two_sum(__uint_as_float(lv[k][J0 + j]), __fmul_rn(S[j].h, 0x1p-8f), e);
                S[j].l = fmaf(S[j].l, 0x1p-8f, e);
            }
    }
#pragma unroll
    for (int j = 0; j < NJ; j++) {
        FF v = ff_norm(S[j]);
        v.h = __fmul_rn(v.h, srow);
        v.l = __fmul_rn(v.l, srow);
        T[j] = add ? ff_add(T[j], v) : v;
    }
}

// FP64E: T of one p0 (the units of its p2 chunks added in chunk order, as
// pairs), with the first unit's column scales copied to sc (if non-null).
// Frees each unit's slot after reading it.  False on timeout/abort.
template <int NS, int UC, int NJ, int J0>
__device__ __forceinline__ bool load_p0_T_ff(FF (&T)[8], RankShared* sh, unsigned& gS, int kcs, unsigned lanebase,
                                             const float* exps, const float* scu, int r, int lane, float* sc,
                                             volatile int* abort, int* status, unsigned long long lim)
{
    for (int u = 0; u < kcs; u++, gS++) {
        const int s = gS % NS;
        if (!mbar_wait(&sh->slot_full[s], (gS / NS) & 1, abort, status, 18, lim)) return false;
        if (!mbar_wait(&sh->exp_full[s], (gS / NS) & 1, abort, status, 23, lim)) return false;
        tc_fence_after();
        if (sc && u == 0) {
#pragma unroll
            for (int j = 0; j < NJ; j++) sc[j] = scu[s * kNT + J0 + j];
        }
        unit_T_ff<NJ, J0>(lanebase + (unsigned)(s * UC), T, exps[s * 128 + r], u > 0);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&sh->slot_empty[s]);
    }
    return true;
}

// T[row][j < NJ] of one p0 for this lane's row: TF32 reads the p0's unit;
// the fixed-point forms add the units of the p2 chunks in chunk order (FP32,
// round to nearest).  With sc (non-null) the first unit's column scales are
// copied there (COLS = false: the caller applies them).  Frees each unit's
// slot after reading it.  False on timeout/abort.
template <int KIND, int NS, int UC, int NJ, bool COLS>
__device__ __forceinline__ bool load_p0_T(float (&T)[NJ], RankShared* sh, unsigned& gS, int kcs, unsigned lanebase,
                                          const float* exps, const float* scu, int r, int lane, float* sc,
                                          volatile int* abort, int* status, unsigned long long lim)
{
    const int nunits = KIND != TC_TF32 ? kcs : 1;
    for (int u = 0; u < nunits; u++, gS++) {
        const int s = gS % NS;
        if (!mbar_wait(&sh->slot_full[s], (gS / NS) & 1, abort, status, 18, lim)) return false;
        if (KIND != TC_TF32 && !mbar_wait(&sh->exp_full[s], (gS / NS) & 1, abort, status, 23, lim)) return false;
        tc_fence_after();
        if (KIND != TC_TF32 && sc && u == 0) {
#pragma unroll
            for (int j = 0; j < NJ; j++) sc[j] = scu[s * kNT + j];
        }
        unit_T<KIND, NJ, COLS>(lanebase + (unsigned)(s * UC), T, exps + s * 128 + r, scu + s * kNT, u > 0);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&sh->slot_empty[s]);
    }
    return true;
}

template <int KIND, bool BIG, int OB = kOB>
__global__ void __launch_bounds__(rank_threads<BIG, OB, KIND>(), 1) k_half_tc_rank(const TcParams P)
{
    constexpr int NG = conv_groups<BIG, OB, KIND>();   // converter groups
    constexpr int CT = kConvWarps * NG;             // converter warps
    constexpr int EW0 = 2 + CT;                     // first epilogue warp
    constexpr int EPW = epi_warps<KIND>();          // epilogue warps
    constexpr bool FX = KIND != TC_TF32;            // fixed-point digit planes (BF16x3, BF16x2)
    constexpr int UC = unit_cols<KIND, BIG>();      // TMEM columns per p0 unit
    constexpr int NS = n_units<KIND, BIG, OB>();    // p0 units in the ring
    constexpr bool WIDE = BIG && OB > kOBig;        // o_X <= 20: accumulators from column 192
    constexpr int CXW = BIG ? (WIDE ? 24 : kOBig) : kOB;   // staged C_X occupied columns per row
    constexpr size_t ASLOT = a_ring_bytes(KIND) / 2;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = (unsigned char*)(((size_t)smem_raw + 1023) & ~(size_t)1023);
    // [F ring][A ring x2][W: 2 parities x kcs_max x 2 planes x 2 KB][C_X rows x2][barriers]
    unsigned char* Fr = base;
    unsigned char* Ar = Fr + (size_t)P.sf * P.f_stage_bytes;
    unsigned char* Wr = Ar + a_ring_bytes(KIND);
    const int wstride = (int)w_stride_bytes(KIND, P.kcs_max);   // bytes per parity
    float* cxs = reinterpret_cast<float*>(Wr + 2 * wstride);
    constexpr int CXF = cx_floats(BIG, KIND, WIDE);
    float* exps = cxs + 2 * CXF;                        // BF16x3: [unit][128 rows] row scales
    float* scu = exps + kFxUnits * 128;                 //          [unit][16 columns] column scales
    int* colx = reinterpret_cast<int*>(scu + kFxUnits * kNT);   // [parity][16 parts][16 columns] exponents
    RankShared* sh = reinterpret_cast<RankShared*>(reinterpret_cast<unsigned char*>(cxs + 2 * CXF) +
                                                   fx_scale_bytes(KIND));

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < P.sf; s++) { mbar_init(&sh->full_f[s], 1); mbar_init(&sh->empty_f[s], kConvWarps); }
        for (int s = 0; s < 2; s++) {
            mbar_init(&sh->full_a[s], kConvWarps); mbar_init(&sh->empty_a[s], 1);
            mbar_init(&sh->full_w[s], CT); mbar_init(&sh->empty_w[s], 1);
            mbar_init(&sh->cx_full[s], 32 * EPW); mbar_init(&sh->cx_empty[s], 32 * EPW);
        }
        for (int s = 0; s < kSlots; s++) { mbar_init(&sh->slot_full[s], 1); mbar_init(&sh->slot_empty[s], EPW); }
        for (int s = 0; s < kFxUnits; s++) mbar_init(&sh->exp_full[s], kConvWarps);
        for (int s = 0; s < 2; s++) mbar_init(&sh->colx_full[s], kConvWarps);
        mbar_init(&sh->drain, 1);
        sh->abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sh->tmem_base)),
                     "r"(P.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = sh->tmem_base;
    volatile int* abort = &sh->abort;

    if (warp == 0) {
        // ------------------------------------------------ TMA producer
        if (lane == 0) {
            unsigned gF = 0;
            unsigned issued_phase[8];
            bool issued[8];
            for (int s = 0; s < 8; s++) issued[s] = false;
            bool ok = true;
            for (int it = blockIdx.x; it < P.n_items && ok && !*abort; it += gridDim.x) {
                const TcItem item = P.items[it];
                const ItemGeo g = geo_of(P.desc[item.dimer], item.form);
                const CUtensorMap* map = P.maps + 2 * item.dimer + item.form;
                const unsigned box = (unsigned)g.n3 * kKC * g.p1t * 8u;
                for (int mt = 0; mt < item.mts && ok; mt++)
                    for (int p0 = 0; p0 < g.n0 && ok; p0++)
                        for (int kc = 0; kc < g.kcs; kc++, gF++) {
                            const int s = gF % P.sf;
                            const unsigned ph = (gF / P.sf) & 1;
                            // test aid: stop issuing; the consumers' waits then run out
                            if (P.withhold && blockIdx.x == 0 && gF + 1 >= (unsigned)P.withhold) {
                                ok = false;
                                break;
                            }
                            if (!(ok = mbar_wait(&sh->empty_f[s], ph ^ 1, abort, P.status, 11, P.wait_ns))) break;
                            mbar_arrive_tx(&sh->full_f[s], box);
                            tma_load_4d(Fr + (size_t)s * P.f_stage_bytes, map, &sh->full_f[s], 0, kc * kKC,
                                        (item.mt0 + mt) * g.p1t, p0);
                            issued[s] = true;
                            issued_phase[s] = ph;
                        }
            }
            for (int s = 0; s < P.sf; s++)
                if (issued[s]) {
                    const unsigned long long t0 = now_ns();
                    while (!mbar_test(&sh->full_f[s], issued_phase[s]) && now_ns() - t0 < kWaitNs) {}
                }
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            unsigned gA = 0, gS = 0, li = 0;
            bool any = false, ok = true;
            const unsigned idesc = make_idesc(KIND, kNT);
            const unsigned idesc_fx[4] = {make_idesc(KIND, 4 * kNT), make_idesc(KIND, 3 * kNT),
                                          make_idesc(KIND, 2 * kNT), make_idesc(KIND, kNT)};
            [[maybe_unused]] unsigned idesc_f6[6];   // FP64E: A_u x [B0..B(6-u)], N = 16 (7 - u)
#pragma unroll
            for (int u = 0; u < 6; u++) idesc_f6[u] = make_idesc(KIND, (7 - u) * kNT);
            for (int it = blockIdx.x; it < P.n_items && ok && !*abort; it += gridDim.x, li++) {
                const TcItem item = P.items[it];
                const ItemGeo g = geo_of(P.desc[item.dimer], item.form);
                const int wp = li & 1;
                if (!(ok = mbar_wait(&sh->full_w[wp], (li >> 1) & 1, abort, P.status, 12, P.wait_ns))) break;
                for (int mt = 0; mt < item.mts && ok; mt++)
                    for (int p0 = 0; p0 < g.n0 && ok; p0++) {
                        if constexpr (!FX) {
                            // one unit per p0: the tensor core accumulates over the p2 chunks
                            const int s = gS % NS;
                            if (!(ok = mbar_wait(&sh->slot_empty[s], ((gS / NS) & 1) ^ 1, abort, P.status, 13, P.wait_ns)))
                                break;
                            tc_fence_after();
                            const unsigned dt = tmem + (unsigned)(s * UC);
                            for (int kc = 0; kc < g.kcs && ok; kc++, gA++) {
                                const int as = gA & 1;
                                if (!(ok = mbar_wait(&sh->full_a[as], (gA >> 1) & 1, abort, P.status, 14, P.wait_ns))) break;
                                tc_fence_after();
                                const unsigned long long adesc = sw128_desc(Ar + (size_t)as * ASLOT);
                                unsigned char* wk = Wr + (size_t)wp * wstride + (size_t)kc * 2 * kNT * 128;
                                const unsigned long long b0 = sw128_desc(wk);
                                const unsigned long long b1 = sw128_desc(wk + kNT * 128);
                                // C_Y = hi + lo (two TF32 planes): A (hi + lo)
#pragma unroll
                                for (int k = 0; k < 4; k++) {
                                    tc_mma<KIND>(dt, adesc + 2 * k, b0 + 2 * k, idesc, (kc > 0 || k > 0) ? 1u : 0u);
                                    tc_mma<KIND>(dt, adesc + 2 * k, b1 + 2 * k, idesc, 1u);
                                }
                                tc_commit(&sh->empty_a[as]);
                                any = true;
                            }
                            if (ok) tc_commit(&sh->slot_full[s]);
                            gS++;
                        } else {
                            // one unit per (p0, p2 chunk): each chunk has its own fixed point
                            for (int kc = 0; kc < g.kcs && ok; kc++, gA++, gS++) {
                                const int s = gS % NS;
                                if (!(ok = mbar_wait(&sh->slot_empty[s], ((gS / NS) & 1) ^ 1, abort, P.status, 13, P.wait_ns)))
                                    break;
                                const int as = gA & 1;
                                if (!(ok = mbar_wait(&sh->full_a[as], (gA >> 1) & 1, abort, P.status, 14, P.wait_ns))) break;
                                tc_fence_after();
                                const unsigned dt = tmem + (unsigned)(s * UC);
                                // digit planes: A tile 1 = [d0 | d1], tile 2 = [d2 | d3] (BF16x3
                                // only); the B tile stacks C_Y's digits B0..B3 as rows 0-63.
                                // A_u x [B0..B(3-u)] lands A_u B_v in the slot of level u + v;
                                // A0's MMA opens all four slots.
                                const unsigned long long adesc = sw128_desc(Ar + (size_t)as * ASLOT);
                                const unsigned long long bk =
                                    sw128_desc(Wr + (size_t)wp * wstride + (size_t)(kc >> 1) * w_rows(KIND) * 128) +
                                    (unsigned long long)((kc & 1) * 4);
                                // FP64E: tiles [d0|d1], [d2|d3], [d4|d5]; A_u x [B0..B(6-u)] lands
                                // A_u B_v in the slot of level u + v (levels 0-6 kept; B6 = 0, so
                                // A0's MMA opens all seven slots)
                                if constexpr (KIND == TC_FP64E) {
#pragma unroll
                                    for (int k = 0; k < 2; k++)
#pragma unroll
                                        for (int u = 0; u < 6; u++) {
                                            const unsigned long long au =
                                                sw128_desc(Ar + (size_t)as * ASLOT + (size_t)(u >> 1) * kABytes) +
                                                (unsigned long long)((u & 1) * 4);
                                            tc_mma<KIND>(dt + u * kNT, au + 2 * k, bk + 2 * k, idesc_f6[u],
                                                         (u > 0 || k > 0) ? 1u : 0u);
                                        }
                                } else {
#pragma unroll
                                    for (int k = 0; k < 2; k++) {
                                        const unsigned acc = k > 0 ? 1u : 0u;
                                        // BF16x2 forms levels 0-2 only: A0 x [B0..B2], A1 x [B0, B1]
                                        constexpr int lv = KIND == TC_BF16X2 ? 1 : 0;
                                        tc_mma<KIND>(dt, adesc + 2 * k, bk + 2 * k, idesc_fx[lv], acc);
                                        tc_mma<KIND>(dt + kNT, adesc + 4 + 2 * k, bk + 2 * k, idesc_fx[lv + 1], 1u);
                                        if constexpr (KIND == TC_BF16X3) {
                                            const unsigned long long a2 = sw128_desc(Ar + (size_t)as * ASLOT + kABytes);
                                            tc_mma<KIND>(dt + 2 * kNT, a2 + 2 * k, bk + 2 * k, idesc_fx[2], 1u);
                                            tc_mma<KIND>(dt + 3 * kNT, a2 + 4 + 2 * k, bk + 2 * k, idesc_fx[3], 1u);
                                        }
                                    }
                                }
                                tc_commit(&sh->empty_a[as]);
                                any = true;
                                tc_commit(&sh->slot_full[s]);
                            }
                        }
                    }
                if (ok) tc_commit(&sh->empty_w[wp]);
            }
            if (any) {
                tc_commit(&sh->drain);
                const unsigned long long t0 = now_ns();
                while (!mbar_test(&sh->drain, 0) && now_ns() - t0 < kWaitNs) {}
            }
        }
    } else if (warp < EW0) {
        // ------------------------------------------------ converters
        const int cta = threadIdx.x - 64;                // 0 .. 32*CT-1
        const int grp = cta / (32 * kConvWarps);         // this warp's group: units with gA % NG == grp
        const int ct = cta % (32 * kConvWarps);          // position within the group
        // tile row and first chunk; the fixed-point forms keep both threads of a row in one warp
        const int r = FX ? (((ct >> 5) << 4) | (lane & 15)) : (ct & 127);
        const int c0 = FX ? (lane >> 4) : (ct >> 7);
        unsigned gF = 0, gA = 0, gU = 0, li = 0;
        bool ok = true;
        for (int it = blockIdx.x; it < P.n_items && ok && !*abort; it += gridDim.x, li++) {
            const TcItem item = P.items[it];
            const DimerDesc& d = P.desc[item.dimer];
            const ItemGeo g = geo_of(d, item.form);
            const float* CY = P.Cf + d.cY;
            [[maybe_unused]] const double* CYd = P.Cd + d.cY;   // FP64E: C_Y in FP64
            const int wp = li & 1;
            const ConvRow cr = conv_row(r, g.p1t * g.n3, g.n3);
            // a warp whose rows all lie past the tile's valid rows (n3 > 64 leaves
            // up to 56 of the 128 rows empty) converts nothing: those rows' MMA
            // results are never stored, whatever the tile holds there
            const bool live = __any_sync(0xffffffffu, cr.valid);
            // ---- B operand of this item: row j < 16, K = p2: C_Y[p2][j] (zero past o2 / n2)
            if (!(ok = mbar_wait(&sh->empty_w[wp], ((li >> 1) & 1) ^ 1, abort, P.status, 15, P.wait_ns))) break;
            float sc_mine = 0.f;                 // BF16x3: column scale of column ct (< 16)
            int* cx_part = colx + wp * 16 * kNT;
            if constexpr (FX) {
                // largest exponent field of each occupied C_Y column: 16 parts x 16
                // columns, each part a strided eighth of the rows, then combined
                // (the first group forms the parts, every converter reads them)
                if (grp == 0) {
                    const int j = ct & 15, part = ct >> 4;
                    int fm = 0;
#pragma unroll
                    for (int t = 0; t < 8; t++) {
                        const int p2 = part + 16 * t;
                        if (j < g.o2 && p2 < g.n2) {
                            if constexpr (KIND == TC_FP64E)
                                fm = max(fm, (int)((__double2hiint(__ldg(CYd + p2 * d.nY + j)) >> 20) & 0x7FF));
                            else
                                fm = max(fm, (int)((__float_as_uint(__ldg(CY + p2 * d.nY + j)) >> 23) & 0xFFu));
                        }
                    }
                    cx_part[part * kNT + j] = fm;
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&sh->colx_full[wp]);
                }
                if (!(ok = mbar_wait(&sh->colx_full[wp], (li >> 1) & 1, abort, P.status, 24, P.wait_ns))) break;
                if (ct < kNT) {
                    int m = 0;
                    for (int q = 0; q < 16; q++) m = max(m, cx_part[q * kNT + ct]);
                    sc_mine = KIND == TC_FP64E ? row_scale(m) : col_scale(m);   // 2^(f - 7)
                }
            }
            for (int kc = 0; kc < g.kcs; kc++) {
                unsigned char* W0 = FX ? Wr + (size_t)wp * wstride + (size_t)(kc >> 1) * w_rows(KIND) * 128
                                       : Wr + (size_t)wp * wstride + (size_t)kc * 2 * kNT * 128;
                unsigned char* W1 = W0 + kNT * 128;
                if (KIND == TC_TF32) {
                    for (int task = cta; task < kNT * 8; task += 32 * CT) {
                        const int j = task >> 3, c = task & 7;
                        unsigned h4[4], l4[4];
#pragma unroll
                        for (int e = 0; e < 4; e++) {
                            const int p2 = kc * kKC + c * 4 + e;
                            const float x = (j < g.o2 && p2 < g.n2) ? __ldg(CY + p2 * d.nY + j) : 0.f;
                            h4[e] = to_tf32(x);
                            l4[e] = to_tf32(x - __uint_as_float(h4[e]));
                        }
                        *reinterpret_cast<uint4*>(W0 + sw128_off(j, c)) = make_uint4(h4[0], h4[1], h4[2], h4[3]);
                        *reinterpret_cast<uint4*>(W1 + sw128_off(j, c)) = make_uint4(l4[0], l4[1], l4[2], l4[3]);
                    }
                } else if constexpr (KIND == TC_FP64E) {
                    // C_Y column j in 48-bit fixed point relative to its largest exponent, six digits
                    for (int task = cta; task < kNT * 4; task += 32 * CT) {
                        const int j = task >> 2, c = task & 3;
                        int fmax = 0;
                        for (int q = 0; q < 16; q++) fmax = max(fmax, cx_part[q * kNT + j]);
                        unsigned w[6][4];
#pragma unroll
                        for (int e = 0; e < 8; e += 2) {
                            uint2 xb[2];
#pragma unroll
                            for (int u = 0; u < 2; u++) {
                                const int p2 = kc * kKC + c * 8 + e + u;
                                const double x = (j < g.o2 && p2 < g.n2) ? __ldg(CYd + p2 * d.nY + j) : 0.0;
                                xb[u] = make_uint2((unsigned)__double2loint(x), (unsigned)__double2hiint(x));
                            }
                            unsigned dg[6];
                            digits6_pair(xb[0], xb[1], fmax, dg);
#pragma unroll
                            for (int k = 0; k < 6; k++) w[k][e / 2] = dg[k];
                        }
#pragma unroll
                        for (int v = 0; v < 6; v++)
                            *reinterpret_cast<uint4*>(W0 + sw128_off(v * kNT + j, (kc & 1) * 4 + c)) =
                                make_uint4(w[v][0], w[v][1], w[v][2], w[v][3]);
                        // plane 6 is zero: A0's MMA spans all seven level slots and opens them
                        *reinterpret_cast<uint4*>(W0 + sw128_off(6 * kNT + j, (kc & 1) * 4 + c)) = make_uint4(0, 0, 0, 0);
                    }
                } else {
                    // C_Y column j in fixed point relative to its largest exponent, four digits
                    for (int task = cta; task < kNT * 4; task += 32 * CT) {
                        const int j = task >> 2, c = task & 3;
                        int fmax = 0;
                        for (int q = 0; q < 16; q++) fmax = max(fmax, cx_part[q * kNT + j]);
                        const float scale = fx_scale_f32(fmax);
                        unsigned w[4][4];
#pragma unroll
                        for (int e = 0; e < 8; e += 2) {
                            float dg[2][4];
#pragma unroll
                            for (int u = 0; u < 2; u++) {
                                const int p2 = kc * kKC + c * 8 + e + u;
                                const float x = (j < g.o2 && p2 < g.n2) ? __ldg(CY + p2 * d.nY + j) : 0.f;
                                digits4(x * scale, dg[u]);
                            }
#pragma unroll
                            for (int k = 0; k < 4; k++) w[k][e / 2] = pack_bf16(dg[0][k], dg[1][k]);
                        }
#pragma unroll
                        for (int v = 0; v < 4; v++)
                            *reinterpret_cast<uint4*>(W0 + sw128_off(v * kNT + j, (kc & 1) * 4 + c)) =
                                make_uint4(w[v][0], w[v][1], w[v][2], w[v][3]);
                    }
                }
            }
            fence_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(&sh->full_w[wp]);

            for (int mt = 0; mt < item.mts && ok; mt++)
                for (int p0 = 0; p0 < g.n0 && ok; p0++) {
                    if constexpr (!FX) {
                        for (int kc = 0; kc < g.kcs; kc++, gF++, gA++) {
                            if ((int)(gA % NG) != grp) continue;   // the other group's unit
                            const int s = gF % P.sf;
                            if (!(ok = mbar_wait(&sh->full_f[s], (gF / P.sf) & 1, abort, P.status, 16, P.wait_ns))) break;
                            const int as = gA & 1;
                            if (!(ok = mbar_wait(&sh->empty_a[as], ((gA >> 1) & 1) ^ 1, abort, P.status, 17, P.wait_ns)))
                                break;
                            if (live)
                                convert_row<KIND>(reinterpret_cast<const double*>(Fr + (size_t)s * P.f_stage_bytes),
                                                  Ar + (size_t)as * ASLOT, cr, g.n3, c0);
                            fence_async_smem();
                            __syncwarp();
                            if (lane == 0) {
                                mbar_arrive(&sh->full_a[as]);
                                mbar_arrive(&sh->empty_f[s]);
                            }
                        }
                    } else {
                        // one unit per p2 chunk: fused load, row maximum and digit planes,
                        // then the unit's row and column scales for the epilogue
                        for (int kc = 0; kc < g.kcs && ok; kc++, gF++, gA++, gU++) {
                            if ((int)(gA % NG) != grp) continue;   // the other group's unit
                            const int s = gF % P.sf;
                            if (!(ok = mbar_wait(&sh->full_f[s], (gF / P.sf) & 1, abort, P.status, 16, P.wait_ns))) break;
                            const int as = gA & 1;
                            if (!(ok = mbar_wait(&sh->empty_a[as], ((gA >> 1) & 1) ^ 1, abort, P.status, 17, P.wait_ns)))
                                break;
                            unsigned char* At = Ar + (size_t)as * ASLOT;
                            const double* Fs = reinterpret_cast<const double*>(Fr + (size_t)s * P.f_stage_bytes);
                            int emax = 0;                   // row scale 0 for rows not converted
                            if (live) {
                                if constexpr (KIND == TC_BF16X3)
                                    emax = convert_row_fx1(Fs, At, At + kABytes, cr, g.n3, c0);
                                else if constexpr (KIND == TC_FP64E)
                                    emax = convert_row_fx6(Fs, At, cr, g.n3, c0);
                                else
                                    emax = convert_row_fx2(Fs, At, cr, g.n3, c0);
                            }
                            fence_async_smem();
                            __syncwarp();
                            if (lane == 0) {
                                mbar_arrive(&sh->full_a[as]);
                                mbar_arrive(&sh->empty_f[s]);
                            }
                            const int su = gU % NS;
                            if (!(ok = mbar_wait(&sh->slot_empty[su], ((gU / NS) & 1) ^ 1, abort, P.status, 22, P.wait_ns)))
                                break;
                            if (c0 == 0) exps[su * 128 + r] = row_scale(emax);
                            if (ct < kNT) scu[su * kNT + ct] = sc_mine;
                            __syncwarp();
                            if (lane == 0) mbar_arrive(&sh->exp_full[su]);
                        }
                    }
                }
        }
    } else {
        // ------------------------------------------------ epilogue
        const int q = warp & 3;
        const int r = q * 32 + lane;                    // accumulator row = TMEM lane
        const int e = (warp - EW0) * 32 + lane;   // C_X row this thread stages (rows past n0: none)
        unsigned gS = 0, li = 0;
        bool ok = true;
        for (int it = blockIdx.x; it < P.n_items && ok && !*abort; it += gridDim.x, li++) {
            const TcItem item = P.items[it];
            const DimerDesc& d = P.desc[item.dimer];
            const ItemGeo g = geo_of(d, item.form);
            const int par = li & 1;
            float* cx = cxs + par * CXF;
            // stage C_X's occupied columns, row p0 = e, for this item
            if (!(ok = mbar_wait(&sh->cx_empty[par], ((li >> 1) & 1) ^ 1, abort, P.status, 19, P.wait_ns))) break;
            if (e < g.n0) {
                if constexpr (KIND == TC_FP64E) {
                    // C_X from the FP64 pool as FP32 pairs
                    const double* CX = P.Cd + d.cX + e * d.nX;
                    FF* cx2 = reinterpret_cast<FF*>(cx);
#pragma unroll
                    for (int i = 0; i < CXW; i++) cx2[e * CXW + i] = i < g.o0 ? ff_split(__ldg(CX + i)) : FF{0.f, 0.f};
                } else {
                    const float* CX = P.Cf + d.cX + e * d.nX;
#pragma unroll
                    for (int i = 0; i < CXW; i++) cx[e * CXW + i] = i < g.o0 ? __ldg(CX + i) : 0.f;
                }
            }
            mbar_arrive(&sh->cx_full[par]);
            if (!(ok = mbar_wait(&sh->cx_full[par], (li >> 1) & 1, abort, P.status, 20, P.wait_ns))) break;
            float* Hf = static_cast<float*>(P.H) + d.h_off + (long long)item.form * g.o0 * g.o2 * g.rows;
            [[maybe_unused]] double* Hd = static_cast<double*>(P.H) + d.h_off + (long long)item.form * g.o0 * g.o2 * g.rows;
            const unsigned lanebase = tmem + ((unsigned)(q * 32) << 16);
            for (int mt = 0; mt < item.mts && ok; mt++) {
                const int p1_lo = (item.mt0 + mt) * g.p1t;
                if constexpr (KIND == TC_FP64E) {
                    // H[(p1,p3)][(i,j)] = sum_p0 C_X[p0][i] T_p0[(p1,p3)][j] on FP32 pairs, for this
                    // warp's columns j = j0 .. j0 + 2 (the two warps of a lane quarter split o_Y <= 5)
                    const int half = (warp - EW0) >> 2;
                    const int j0 = half * kFFCols;
                    FF acc[OB][kFFCols];
#pragma unroll
                    for (int i = 0; i < OB; i++)
#pragma unroll
                        for (int j = 0; j < kFFCols; j++) acc[i][j] = FF{0.f, 0.f};
                    float sc[kFFCols];   // the item's column scales 2^(f - 7), applied once per output
#pragma unroll
                    for (int j = 0; j < kFFCols; j++) sc[j] = 1.f;
                    const FF* cx2 = reinterpret_cast<const FF*>(cx);
                    for (int p0 = 0; p0 < g.n0; p0++) {
                        FF T[8];
                        ok = half ? load_p0_T_ff<NS, UC, kFFCols, kFFCols>(T, sh, gS, g.kcs, lanebase, exps, scu, r, lane,
                                                                       p0 == 0 ? sc : nullptr, abort, P.status,
                                                                       P.wait_ns)
                                  : load_p0_T_ff<NS, UC, kFFCols, 0>(T, sh, gS, g.kcs, lanebase, exps, scu, r, lane,
                                                                     p0 == 0 ? sc : nullptr, abort, P.status, P.wait_ns);
                        if (!ok) break;
#pragma unroll
                        for (int i = 0; i < OB; i++) {
                            const FF c = cx2[p0 * kOB + i];
#pragma unroll
                            for (int j = 0; j < kFFCols; j++) ff_mac_nr(acc[i][j], c, T[j]);
                        }
                        if ((p0 & 7) == 7) {   // the low parts gather at most eight products' errors
#pragma unroll
                            for (int i = 0; i < OB; i++)
#pragma unroll
                                for (int j = 0; j < kFFCols; j++) acc[i][j] = ff_norm(acc[i][j]);
                        }
                    }
                    if (!ok) break;
                    const int valid = (min(g.n1, p1_lo + g.p1t) - p1_lo) * g.n3;
                    if (r < valid) {
                        // pair (i, j) of this row at element (i*o2 + j) * rows; the column
                        // scale is a power of two, so scaling a pair keeps it exact
                        const size_t row0 = (size_t)(p1_lo * g.n3 + r);
#pragma unroll
                        for (int i = 0; i < OB; i++)
#pragma unroll
                            for (int jj = 0; jj < kFFCols; jj++) {
                                const int j = j0 + jj;
                                if (i < g.o0 && j < g.o2) {
                                    const size_t q = row0 + (size_t)(i * g.o2 + j) * g.rows;
                                    const FF v = ff_norm(FF{__fmul_rn(acc[i][jj].h, sc[jj]), __fmul_rn(acc[i][jj].l, sc[jj])});
                                    if (P.h_pairs) reinterpret_cast<FF*>(Hd)[q] = v;
                                    else Hd[q] = ff_f64(v);
                                }
                            }
                    }
                } else if constexpr (!BIG) {
                    float acc[OB][OB];
#pragma unroll
                    for (int i = 0; i < OB; i++)
#pragma unroll
                        for (int j = 0; j < OB; j++) acc[i][j] = 0.f;
                    float sc[8];   // the item's column scales (fixed-point forms), applied once per output
#pragma unroll
                    for (int j = 0; j < 8; j++) sc[j] = 1.f;
                    for (int p0 = 0; p0 < g.n0; p0++) {
                        float T[8];
                        if (!(ok = load_p0_T<KIND, NS, UC, 8, false>(T, sh, gS, g.kcs, lanebase, exps, scu, r, lane,
                                                                      p0 == 0 ? sc : nullptr, abort, P.status,
                                                                      P.wait_ns)))
                            break;
                        const float4 ca = *reinterpret_cast<const float4*>(cx + p0 * kOB);
                        const float4 cb = *reinterpret_cast<const float4*>(cx + p0 * kOB + 4);
                        const float cv[kOB] = {ca.x, ca.y, ca.z, ca.w, cb.x, cb.y, cb.z, cb.w};
#pragma unroll
                        for (int i = 0; i < OB; i++)
#pragma unroll
                            for (int j = 0; j < OB; j++) acc[i][j] = fmaf(cv[i], T[j], acc[i][j]);
                    }
                    if (!ok) break;
                    const int valid = (min(g.n1, p1_lo + g.p1t) - p1_lo) * g.n3;
                    float* out = Hf + p1_lo * g.n3 + r;   // pair-major: coalesced over rows
                    if (r < valid) {
                        // pair (i, j) of this row lives at out + (i*o2 + j) * rows
                        const size_t step = (size_t)g.rows;
                        float* q = out;
#pragma unroll
                        for (int i = 0; i < OB; i++) {
                            if (i < g.o0) {
#pragma unroll
                                for (int j = 0; j < OB; j++)
                                    if (j < g.o2) { *q = acc[i][j] * sc[j]; q += step; }
                            }
                        }
                    }
                } else {
                    const unsigned accbase = lanebase + (WIDE ? 192u : 256u);
                    const int nchunk = (g.o0 + 1) >> 1;   // two occupied i per TMEM round trip
                    // NJ columns j per accumulator row: 8 when o_Y <= 8 (the rest of each
                    // 16-column row is never read), else 16 -- half the T combination, FMAs and
                    // TMEM traffic for the smaller occupations; same results either way
                    auto rank1_over_p0 = [&](auto njc) {
                        constexpr int NJ = decltype(njc)::value;
                        for (int p0 = 0; p0 < g.n0; p0++) {
                            float T[NJ];
                            if (!(ok = load_p0_T<KIND, NS, UC, NJ, true>(T, sh, gS, g.kcs, lanebase, exps, scu, r,
                                                                          lane, nullptr, abort, P.status, P.wait_ns)))
                                break;
                            const float* cp = cx + p0 * CXW;
#pragma unroll 1
                            for (int ic = 0; ic < nchunk; ic++) {
                                unsigned a[2][NJ];
                                if (p0 > 0) {
                                    if constexpr (NJ == 16)
                                        tmem_ld_l2x16(accbase + (unsigned)(ic * 32),
                                                      *reinterpret_cast<unsigned(*)[32]>(&a[0][0]));
                                    else
                                        tmem_ld_l2x8(accbase + (unsigned)(ic * 32),
                                                     *reinterpret_cast<unsigned(*)[16]>(&a[0][0]));
                                } else {
#pragma unroll
                                    for (int u = 0; u < 2; u++)
#pragma unroll
                                        for (int j = 0; j < NJ; j++) a[u][j] = 0u;
                                }
                                const float2 c2 = *reinterpret_cast<const float2*>(cp + ic * 2);
                                const float cv[2] = {c2.x, c2.y};
#pragma unroll
                                for (int u = 0; u < 2; u++)
#pragma unroll
                                    for (int j = 0; j < NJ; j++)
                                        a[u][j] = __float_as_uint(fmaf(cv[u], T[j], __uint_as_float(a[u][j])));
#pragma unroll
                                for (int u = 0; u < 2; u++) {
                                    if constexpr (NJ == 16) tmem_st16(accbase + (unsigned)((ic * 2 + u) * 16), a[u]);
                                    else tmem_st8(accbase + (unsigned)((ic * 2 + u) * 16), a[u]);
                                }
                            }
                            tmem_wait_st();   // this p0's updates land before the next one reads them
                        }
                    };
                    if (g.o2 <= 8) rank1_over_p0(std::integral_constant<int, 8>{});
                    else rank1_over_p0(std::integral_constant<int, 16>{});
                    if (!ok) break;
                    const int valid = (min(g.n1, p1_lo + g.p1t) - p1_lo) * g.n3;
                    float* out = Hf + p1_lo * g.n3 + r;
                    const size_t step = (size_t)g.rows;
                    float* q = out;
                    for (int i = 0; i < g.o0; i++) {
                        float v[16];
                        tmem_ld16(accbase + (unsigned)(i * 16), v);
#pragma unroll
                        for (int j = 0; j < 16; j++)
                            if (j < g.o2) {
                                if (r < valid) *q = v[j];
                                q += step;
                            }
                    }
                }
            }
            mbar_arrive(&sh->cx_empty[par]);
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(P.tmem_cols)
                     : "memory");
    }
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// The rank variants (1-3) run one M-tile per item; variant 0 groups as many
// M-tiles as one TMEM accumulator set holds.
int items_per_form(const DimerDesc& d, int f, int variant, int* mts_max)
{
    const int n1 = f ? d.nY : d.nX, n3 = f ? d.nX : d.nY;
    const int p1t = 128 / n3;
    const int tiles = (n1 + p1t - 1) / p1t;
    const int mmax = variant >= 1 ? 1 : std::max(1, std::min(8, kAccCols / d.npad));
    *mts_max = mmax;
    return (tiles + mmax - 1) / mmax;
}

// 3: rank kernel, register accumulators sized for occupations <= 5; 1: the
// same for <= 8; 2: rank kernel, TMEM accumulators (<= 16); 4: the same with
// o_X <= 20, o_Y <= 16 (a 20-occupied dimer as two blocks of Y's occupied
// orbitals instead of 2 x 2); 0: Kronecker kernel (anything else TF32/BF16x3
// accept).  MCPT_TC_KERNEL=kron|rank8|rankbig|rankwide forces a kernel where
// the sizes allow it.
int choose_variant(TcKind kind, const DimerDesc* h, int nd)
{
    int omax = 0, nymax = 0, oxmax = 0, oymax = 0;
    for (int k = 0; k < nd; k++) {
        omax = std::max(omax, std::max(h[k].oX, h[k].oY));
        oxmax = std::max(oxmax, h[k].oX);
        oymax = std::max(oymax, h[k].oY);
        nymax = std::max(nymax, h[k].nY);
    }
    const bool fits_rank = nymax <= kKCMax * kKC && omax <= kOBig;
    const bool fits_wide = nymax <= kKCMax * kKC && oxmax <= kOBigI && oymax <= kOBig;
    if (kind == TC_FP64E) return 3;   // the one kernel it has (limits checked by tc_prepare)
    const char* env = getenv("MCPT_TC_KERNEL");
    // BF16x2 runs the rank kernels only (the tensor-core size limits always fit them)
    if (env && !strcmp(env, "kron") && kind != TC_BF16X2) return 0;
    if (env && !strcmp(env, "rankbig") && fits_rank) return 2;
    if (env && !strcmp(env, "rank8") && omax <= kOB) return 1;
    if (env && !strcmp(env, "rankwide") && fits_wide) return 4;
    if (!fits_rank) return fits_wide ? 4 : kind == TC_BF16X2 ? 2 : 0;
    return omax <= kOB5 ? 3 : omax <= kOB ? 1 : 2;
}

}  // namespace

size_t tc_work_bytes(TcKind kind, const DimerDesc* h, int nd)
{
    size_t items = 0;
    const int variant = choose_variant(kind, h, nd);
    for (int k = 0; k < nd; k++)
        for (int f = 0; f < 2; f++) {
            int m;
            items += items_per_form(h[k], f, variant, &m);
        }
    return (size_t)nd * 2 * sizeof(CUtensorMap) + items * sizeof(TcItem) + 256;
}

// Shared-memory bytes of a launch apart from its staging ring, and the
// deepest ring that fits.
static size_t fixed_smem(TcKind kind, int variant, int kcs_max, unsigned w_stage_bytes)
{
    return variant >= 1 ? 1024 + a_ring_bytes(kind) + 2 * w_stride_bytes(kind, kcs_max) +
                              2 * (size_t)cx_floats(variant == 2 || variant == 4, kind, variant == 4) * 4 +
                              fx_scale_bytes(kind) + sizeof(RankShared)
                        : 1024 /*align*/ + 2 * (size_t)kABytes + 2 * (size_t)w_stage_bytes + sizeof(TcShared);
}

static void launch_shape(const DimerDesc* h, int nd, int* kcs_max, unsigned* f_stage, unsigned* w_stage)
{
    int maxN = 16, kc = 1;
    unsigned box = 0;
    for (int k = 0; k < nd; k++) {
        maxN = std::max(maxN, h[k].npad);
        kc = std::max(kc, (h[k].nY + kKC - 1) / kKC);
        for (int f = 0; f < 2; f++) {
            const int n3 = f ? h[k].nX : h[k].nY;
            box = std::max(box, (unsigned)(n3 * kKC * (128 / n3) * 8));
        }
    }
    *kcs_max = kc;
    *f_stage = (box + 1023) & ~1023u;
    *w_stage = (unsigned)(((size_t)maxN * 128 + 1023) & ~(size_t)1023);
}

int tc_candidates(TcKind kind, const DimerDesc* h, int nd, TcTune* out, int max)
{
    int omax = 0, nymax = 0;
    for (int k = 0; k < nd; k++) {
        omax = std::max(omax, std::max(h[k].oX, h[k].oY));
        nymax = std::max(nymax, h[k].nY);
    }
    std::vector<int> vars;
    if (kind == TC_FP64E) {
        vars.push_back(3);
    } else if (nymax <= kKCMax * kKC && omax <= kOBig) {
        // the accumulator tiles: 5 x 5 and 8 x 8 in registers, 16 x 16 in TMEM
        // with four T units, 20 x 16 in TMEM with three
        if (omax <= kOB5) vars.push_back(3);
        if (omax <= kOB) vars.push_back(1);
        vars.push_back(2);
        vars.push_back(4);
    } else if (choose_variant(kind, h, nd) == 4) {
        vars.push_back(4);
    } else {
        vars.push_back(0);
    }
    int dev = 0, nsm = 0, max_smem = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    int kcs_max;
    unsigned fs, ws;
    launch_shape(h, nd, &kcs_max, &fs, &ws);
    int n = 0;
    for (int v : vars) {
        const int sf_max = std::min(8, (int)(((size_t)max_smem - fixed_smem(kind, v, kcs_max, ws)) / fs));
        const int sf_min = 2;
        if (sf_max < sf_min) continue;
        int sfs[3] = {sf_min, (sf_min + sf_max) / 2, sf_max};
        for (int a = 0; a < 3; a++) {
            if (a > 0 && sfs[a] == sfs[a - 1]) continue;
            for (int gdiv = 0; gdiv < 2; gdiv++)
                if (n < max) out[n++] = TcTune{v + 1, sfs[a], gdiv ? nsm - nsm / 4 : nsm};
        }
    }
    return n;
}

cudaError_t tc_prepare(TcKind kind, const DimerDesc* h_desc, const DimerDesc* d_desc, int nd, const float* Cf,
                       const double* Cd, void* H, void* d_work, size_t work_bytes, int* d_status, cudaStream_t s,
                       const TcTune* tune, TcLaunch* out, char* err, size_t errlen)
{
    if (nd <= 0) return cudaSuccess;
    auto encode = get_encode();
    if (!encode) {
        snprintf(err, errlen, "cuTensorMapEncodeTiled unavailable");
        return cudaErrorNotSupported;
    }
    std::vector<CUtensorMap> maps((size_t)nd * 2);
    std::vector<TcItem> items;
    const int variant = (tune && tune->variant1) ? tune->variant1 - 1 : choose_variant(kind, h_desc, nd);
    if (kind == TC_FP64E) {
        for (int k = 0; k < nd; k++)
            if (std::max(h_desc[k].oX, h_desc[k].oY) > kOB5 || h_desc[k].nY > kFp64eMaxAO || variant != 3) {
                snprintf(err, errlen, "the FP64-emulating form handles monomers of up to %d AO and %d occupied",
                         kFp64eMaxAO, kOB5);
                return cudaErrorNotSupported;
            }
    }
    int maxN = 16;
    unsigned max_box = 0;
    for (int k = 0; k < nd; k++) {
        const DimerDesc& d = h_desc[k];
        maxN = std::max(maxN, d.npad);
        for (int f = 0; f < 2; f++) {
            const int n0 = d.nX, n1 = f ? d.nY : d.nX, n2 = d.nY, n3 = f ? d.nX : d.nY;
            const int p1t = 128 / n3;
            cuuint64_t dims[4] = {(cuuint64_t)n3, (cuuint64_t)n2, (cuuint64_t)n1, (cuuint64_t)n0};
            cuuint64_t strides[3] = {(cuuint64_t)d.st[f][2] * 8, (cuuint64_t)d.st[f][1] * 8, (cuuint64_t)d.st[f][0] * 8};
            cuuint32_t box[4] = {(cuuint32_t)n3, (cuuint32_t)kKC, (cuuint32_t)p1t, 1};
            cuuint32_t estr[4] = {1, 1, 1, 1};
            CUresult r = encode(&maps[2 * k + f], CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4, (void*)d.E[f], dims, strides,
                                box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) {
                snprintf(err, errlen, "cuTensorMapEncodeTiled failed (%d) for dimer %d form %d", (int)r, k, f);
                return cudaErrorInvalidValue;
            }
            max_box = std::max(max_box, (unsigned)(n3 * kKC * p1t * 8));
            int mmax;
            const int nit = items_per_form(d, f, variant, &mmax);
            const int tiles = (n1 + p1t - 1) / p1t;
            for (int q = 0; q < nit; q++) {
                TcItem it;
                it.dimer = k;
                it.form = f;
                it.mt0 = q * mmax;
                it.mts = std::min(mmax, tiles - it.mt0);
                items.push_back(it);
            }
        }
    }
    // longest items first (cost ~ AO bytes read), stable so equal items keep dimer order
    std::stable_sort(items.begin(), items.end(), [&](const TcItem& a, const TcItem& b) {
        auto cost = [&](const TcItem& t) {
            const DimerDesc& d = h_desc[t.dimer];
            return (long long)t.mts * d.nX * d.nY * 128;
        };
        return cost(a) > cost(b);
    });
    const size_t need = maps.size() * sizeof(CUtensorMap) + items.size() * sizeof(TcItem);
    if (need > work_bytes) {
        snprintf(err, errlen, "work buffer too small (%zu < %zu)", work_bytes, need);
        return cudaErrorInvalidValue;
    }
    unsigned char* w = static_cast<unsigned char*>(d_work);
    cudaError_t e = cudaMemcpyAsync(w, maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    const size_t items_off = maps.size() * sizeof(CUtensorMap);
    e = cudaMemcpyAsync(w + items_off, items.data(), items.size() * sizeof(TcItem), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;

    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int max_smem = 0;
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);

    TcLaunch& P = *out;
    P.items = w + items_off;
    P.n_items = (int)items.size();
    P.maps = w;
    P.desc = d_desc;
    P.Cf = Cf;
    P.Cd = Cd;
    P.H = H;
    P.h_pairs = 0;
    if (kind == TC_FP64E) {
        int ao = 0;
        for (int k = 0; k < nd; k++) ao = std::max(ao, std::max(h_desc[k].nX, h_desc[k].nY));
        P.h_pairs = ao <= 32;
    }
    P.status = d_status;
    P.kind = kind;
    P.f_stage_bytes = (max_box + 1023) & ~1023u;
    P.w_stage_bytes = (unsigned)(((size_t)maxN * 128 + 1023) & ~(size_t)1023);
    P.tmem_cols = 2 * kAccCols;   // both accumulator sets / all 32 slots
    P.variant = variant;
    int kcs_max = 1;
    for (int k = 0; k < nd; k++) kcs_max = std::max(kcs_max, (h_desc[k].nY + kKC - 1) / kKC);
    P.kcs_max = kcs_max;
    const size_t fixed = fixed_smem(kind, variant, kcs_max, P.w_stage_bytes);
    int sf = (int)(((size_t)max_smem - fixed) / P.f_stage_bytes);
    sf = std::min(sf, 8);
    if (tune && tune->sf) sf = std::min(sf, tune->sf);
    const int sf_min = 2;
    if (sf < sf_min) {
        snprintf(err, errlen, "not enough shared memory for the staging ring (%d < %d stages)", sf, sf_min);
        return cudaErrorInvalidConfiguration;
    }
    P.sf = sf;
    P.smem = fixed + (size_t)sf * P.f_stage_bytes;
    P.grid = std::min<int>((int)items.size(), (tune && tune->grid) ? std::min(tune->grid, nsm) : nsm);
    return cudaSuccess;
}

cudaError_t tc_launch(const TcLaunch& L, cudaStream_t s)
{
    TcParams P;
    P.items = static_cast<const TcItem*>(L.items);
    P.n_items = L.n_items;
    P.maps = static_cast<const CUtensorMap*>(L.maps);
    P.desc = L.desc;
    P.Cf = L.Cf;
    P.Cd = L.Cd;
    P.H = L.H;
    P.h_pairs = L.h_pairs;
    P.status = L.status;
    P.sf = L.sf;
    P.f_stage_bytes = L.f_stage_bytes;
    P.w_stage_bytes = L.w_stage_bytes;
    P.tmem_cols = L.tmem_cols;
    P.kind = L.kind;
    P.kcs_max = L.kcs_max;
    P.wait_ns = L.wait_ns ? L.wait_ns : kWaitNs;
    P.withhold = L.withhold;
    void (*fn)(const TcParams);
    if (L.kind == TC_FP64E) {
        if (L.variant != 3) return cudaErrorNotSupported;
        fn = k_half_tc_rank<TC_FP64E, false, kOB5>;
    } else if (L.variant == 1)
        fn = L.kind == TC_TF32     ? k_half_tc_rank<TC_TF32, false>
             : L.kind == TC_BF16X2 ? k_half_tc_rank<TC_BF16X2, false>
                                   : k_half_tc_rank<TC_BF16X3, false>;
    else if (L.variant == 3)
        fn = L.kind == TC_TF32     ? k_half_tc_rank<TC_TF32, false, kOB5>
             : L.kind == TC_BF16X2 ? k_half_tc_rank<TC_BF16X2, false, kOB5>
                                   : k_half_tc_rank<TC_BF16X3, false, kOB5>;
    else if (L.variant == 2)
        fn = L.kind == TC_TF32     ? k_half_tc_rank<TC_TF32, true>
             : L.kind == TC_BF16X2 ? k_half_tc_rank<TC_BF16X2, true>
                                   : k_half_tc_rank<TC_BF16X3, true>;
    else if (L.variant == 4)
        fn = L.kind == TC_TF32     ? k_half_tc_rank<TC_TF32, true, kOBigI>
             : L.kind == TC_BF16X2 ? k_half_tc_rank<TC_BF16X2, true, kOBigI>
                                   : k_half_tc_rank<TC_BF16X3, true, kOBigI>;
    else if (L.kind == TC_BF16X2)
        return cudaErrorNotSupported;   // the Kronecker kernel has no 16-bit fixed-point form
    else fn = L.kind == TC_TF32 ? k_half_tc<TC_TF32> : k_half_tc<TC_BF16X3>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem);
    if (e != cudaSuccess) return e;
    const int threads = L.kind == TC_FP64E ? rank_threads<false, kOB5, TC_FP64E>()
                        : L.variant == 3   ? rank_threads<false, kOB5>()
                        : L.variant == 2 ? rank_threads<true, kOB>()
                        : L.variant == 4 ? rank_threads<true, kOBigI>()
                        : L.variant == 1 ? rank_threads<false, kOB>()
                                         : kThreadsTc;
    fn<<<L.grid, threads, L.smem, s>>>(P);
    return cudaGetLastError();
}

}  // namespace mcpt
