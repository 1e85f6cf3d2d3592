// tcgen05 building blocks shared by the Gram and orbital-update GEMMs:
// PTX wrappers (mbarriers, bulk copies, tensor-memory allocation, MMA issue
// and readback), shared-memory and instruction descriptors, the canonical
// no-swizzle K-major tile layout, and the split of an FP32 value into 16-bit
// parts (Sec. V.B.7; Henry, Tang and Heinecke, ARITH 2019).
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdint>

#include "mlmd.h"

namespace mlmd {
namespace tc {

constexpr int BM = 128, BN = 128, BK = 64;          // output tile and K-step of one pipeline stage
constexpr int KSTEPS_PER_MMA = BK / 16;             // MMAs of K = 16 per K-step
constexpr long long kWaitCycles = 4000000000LL;

// ---- PTX wrappers -----------------------------------------------------------
static __device__ __forceinline__ uint32_t smem_u32(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

static __device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

static __device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

static __device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

static __device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > kWaitCycles) return false;
    return true;
}

// Shared-memory matrix descriptor, no swizzle, K-major canonical layout:
// start address, leading-dimension byte offset (between the two core
// matrices adjacent along K), stride byte offset (between 8-row groups),
// descriptor version 1 (bits 46-47), layout type 0 (no swizzle).
static __device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of tcgen05.mma kind::f16: FP32 accumulator, A and B
// both BF16 (fmt 1) or both FP16 (fmt 0), K-major A and B, N = 128, M = 128.
__host__ __device__ constexpr uint32_t instr_desc(uint32_t ab_fmt) {
    return (1u << 4)                    // D format: FP32
           | (ab_fmt << 7)              // A format
           | (ab_fmt << 10)             // B format
           | ((uint32_t)(BN >> 3) << 17)
           | ((uint32_t)(BM >> 4) << 24);
}

static __device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                        uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
        ::"r"(d_tmem), "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

static __device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

static __device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
static __device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
static __device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 consecutive FP32 columns of this warp's 32 TMEM lanes.
static __device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// ---- operand splitting ------------------------------------------------------
template <int MODE> struct Split;
// parts of x and the products (i, j) summed
template <> struct Split<MLMD_GEMM_BF16> { static constexpr int NPART = 1, NPROD = 1; };
template <> struct Split<MLMD_GEMM_BF16X2> { static constexpr int NPART = 2, NPROD = 3; };
template <> struct Split<MLMD_GEMM_BF16X3> { static constexpr int NPART = 3, NPROD = 6; };
template <> struct Split<MLMD_GEMM_FP16> { static constexpr int NPART = 1, NPROD = 1; };

// Split products (i, j) by size, largest first: (0,0), (0,1), (1,0), (0,2),
// (1,1), (2,0); a mode with NPROD products uses the first NPROD.
__host__ __device__ constexpr int size_rank_a(int q) { return q == 0 ? 0 : q == 1 ? 0 : q == 2 ? 1 : q == 3 ? 0 : q == 4 ? 1 : 2; }
__host__ __device__ constexpr int size_rank_b(int q) { return q == 0 ? 0 : q == 1 ? 1 : q == 2 ? 0 : q == 3 ? 2 : q == 4 ? 1 : 0; }
// The p-th product issued into an accumulator, smallest first: the FP32
// accumulation in tensor memory rounds towards zero, so adding the small
// correction products to a still-small accumulator and the leading product
// x0 y0 last keeps the truncation relative to the final sum to a few ulps.
__host__ __device__ constexpr int prod_a(int p, int nprod) { return size_rank_a(nprod - 1 - p); }
__host__ __device__ constexpr int prod_b(int p, int nprod) { return size_rank_b(nprod - 1 - p); }

template <int MODE>
static __device__ __forceinline__ void split_value(float x, float fscale, uint16_t (&part)[3]) {
    if (MODE == MLMD_GEMM_FP16) {
        part[0] = __half_as_ushort(__float2half_rn(x * fscale));
        part[1] = part[2] = 0;
        return;
    }
    float r = x;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        if (i < Split<MODE>::NPART) {
            const __nv_bfloat16 b = __float2bfloat16_rn(r);
            part[i] = __bfloat16_as_ushort(b);
            r -= __bfloat162float(b);
        } else {
            part[i] = 0;
        }
    }
}

// Byte offset of element (row, k) in a K-major canonical tile of BM rows x BK
// 16-bit elements: core matrix (row/8, k/8) of 8 rows x 16 bytes; the eight
// K-cores of a row group are adjacent (LBO = 128 B), row groups SBO = 1024 B.
static __device__ __forceinline__ uint32_t tile_offset(int row, int k) {
    return (uint32_t)((row >> 3) * 1024 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

constexpr uint32_t kTileBytes = BM * BK * 2;        // 16 KiB per 16-bit operand tile

static __device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

static __device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// pipeline stages of A and B tiles (all parts) that fit beside each other
// in 192 KiB of shared memory
template <int MODE> struct Stages { static constexpr int value = Split<MODE>::NPART == 1 ? 6 : (Split<MODE>::NPART == 2 ? 3 : 2); };

}  // namespace tc
}  // namespace mlmd
