// Gram / overlap matrix on the tcgen05 tensor cores with split-precision
// operands (Sec. V.B.7, Sec. VI.C).
//
// For complex64 orbitals X, Y ([N_g][ld] interleaved) the overlap
// S = scale * X^H Y comes from one real product G = Xr^T Yr of the real views
// Xr, Yr ([N_g][2 ld]): S[n][m] = G[2n][2m] + G[2n+1][2m+1]
//                                  + i (G[2n][2m+1] - G[2n+1][2m]).
// Each FP32 operand x is split into 16-bit parts: BF16 (x ~ x0), BF16X2
// (x ~ x0 + x1, products 00, 01, 10), BF16X3 (x ~ x0 + x1 + x2, products with
// i + j <= 2: 00, 01, 10, 02, 11, 20 -- the split-product scheme of Henry, Tang
// and Heinecke, ARITH 2019) or FP16 after a power-of-two scale.  All products
// of a tile accumulate in FP32 in tensor memory; K-slices of the grid go to
// different CTAs and their FP32 tiles are summed in FP64.
//
// Kernel structure: one CTA computes a 128 x 128 tile of G over a K range of
// grid points.  Per K-step of 64 points, all 256 threads read the FP32 rows
// of both operands (8 consecutive points of one column per item), split them
// and store the 16-bit parts in shared memory in the canonical no-swizzle
// K-major core-matrix layout (8 rows x 16 bytes per core matrix, one 16-byte
// store per part); thread 0 then issues the tcgen05.mma instructions (M = 128,
// N = 128, K = 16 each) and commits them to an mbarrier; two buffers let the
// conversion of the next step overlap the MMAs of this one.  The epilogue
// reads the accumulator with tcgen05.ld, pairs rows 2a / 2a+1 with a lane
// shuffle and writes the complex FP64 partial tile.  Every mbarrier wait is
// bounded; tensor memory is always freed.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>

#include "mlmd_internal.cuh"

namespace mlmd {
namespace {

constexpr int BM = 128, BN = 128, BK = 64;          // tile and K-step (grid points)
constexpr int KSTEPS_PER_MMA = BK / 16;             // MMAs of K = 16 per K-step
constexpr long long kWaitCycles = 4000000000LL;

// ---- PTX wrappers -----------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > kWaitCycles) return false;
    return true;
}

// Shared-memory matrix descriptor, no swizzle, K-major canonical layout:
// start address, leading-dimension byte offset (between the two core
// matrices adjacent along K), stride byte offset (between 8-row groups),
// descriptor version 1 (bits 46-47), layout type 0 (no swizzle).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
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

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                        uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
        ::"r"(d_tmem), "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 consecutive FP32 columns of this warp's 32 TMEM lanes.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
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

__host__ __device__ constexpr int prod_a(int p) { return p == 0 ? 0 : p == 1 ? 0 : p == 2 ? 1 : p == 3 ? 0 : p == 4 ? 1 : 2; }
__host__ __device__ constexpr int prod_b(int p) { return p == 0 ? 0 : p == 1 ? 1 : p == 2 ? 0 : p == 3 ? 2 : p == 4 ? 1 : 0; }

template <int MODE>
__device__ __forceinline__ void split_value(float x, float fscale, uint16_t (&part)[3]) {
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
__device__ __forceinline__ uint32_t tile_offset(int row, int k) {
    return (uint32_t)((row >> 3) * 1024 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

constexpr uint32_t kTileBytes = BM * BK * 2;        // 16 KiB per 16-bit operand tile

// part[z][n][m] (complex FP64) for output tile (tn, tm) of G over K-slice z.
// Rows of G: real columns [r0, r0 + 128) of X; columns: [c0, c0 + 128) of Y.
template <int MODE>
__global__ void __launch_bounds__(256, 1)
    k_gram_tc(const float* __restrict__ X, const float* __restrict__ Y, int64_t ng, int ld, int n_orb,
              int64_t kchunk, float fscale, double unscale, double* __restrict__ part, int* __restrict__ err) {
    constexpr int NPART = Split<MODE>::NPART, NPROD = Split<MODE>::NPROD;
    constexpr uint32_t STAGE_BYTES = 2 * NPART * kTileBytes;   // A parts + B parts
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    __shared__ __align__(8) uint64_t mma_bar[2];
    __shared__ uint32_t tmem_base;
    __shared__ int abort_sh;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int r0 = blockIdx.y * BM, c0 = blockIdx.x * BN;   // real columns of X (rows of G), of Y
    const int64_t g0 = (int64_t)blockIdx.z * kchunk;
    const int64_t g1 = min(ng, g0 + kchunk);
    const int nsteps = (int)((g1 - g0 + BK - 1) / BK);
    const int ncols_real = 2 * ld;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(128u)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(&mma_bar[0], 1);
        mbar_init(&mma_bar[1], 1);
        abort_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    constexpr uint32_t IDESC = instr_desc(MODE == MLMD_GEMM_FP16 ? 0u : 1u);

    int uses[2] = {0, 0};     // commits issued per buffer (thread 0)
    for (int s = 0; s < nsteps; ++s) {
        const int b = s & 1;
        unsigned char* As = smem + b * STAGE_BYTES;
        unsigned char* Bs = As + NPART * kTileBytes;
        // the MMAs that last read this buffer (step s-2) must be complete
        if (s >= 2) {
            bool ok = mbar_wait_bounded(&mma_bar[b], (uint32_t)(((s - 2) >> 1) & 1));
            if (!ok) abort_sh = 1;
        }
        __syncthreads();
        if (abort_sh) break;
        // stage: item (operand, k-group, column) = 8 consecutive grid points of
        // one real column, split into 16-bit parts and stored as one 16-byte
        // core-matrix row per part
        const int64_t gk = g0 + (int64_t)s * BK;
        for (int item = tid; item < 2 * (BK / 8) * BM; item += 256) {
            const int c = item % BM, kg = (item / BM) % (BK / 8), op = item / (BM * (BK / 8));
            const float* src = op == 0 ? X : Y;
            const int col = (op == 0 ? r0 : c0) + c;
            uint16_t pk[3][8];
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) {
                const int64_t g = gk + kg * 8 + kk;
                const float x = (g < g1 && col < ncols_real) ? __ldg(src + g * ncols_real + col) : 0.f;
                uint16_t pp[3];
                split_value<MODE>(x, fscale, pp);
#pragma unroll
                for (int i = 0; i < 3; ++i) pk[i][kk] = pp[i];
            }
            unsigned char* dst = (op == 0 ? As : Bs) + tile_offset(c, kg * 8);
#pragma unroll
            for (int i = 0; i < NPART; ++i) {
                uint4 w;
                w.x = pk[i][0] | ((uint32_t)pk[i][1] << 16);
                w.y = pk[i][2] | ((uint32_t)pk[i][3] << 16);
                w.z = pk[i][4] | ((uint32_t)pk[i][5] << 16);
                w.w = pk[i][6] | ((uint32_t)pk[i][7] << 16);
                *reinterpret_cast<uint4*>(dst + i * kTileBytes) = w;
            }
        }
        fence_async_smem();       // generic-proxy stores -> visible to the tensor cores
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
#pragma unroll
            for (int p = 0; p < NPROD; ++p) {
                const uint32_t a_base = smem_u32(As + prod_a(p) * kTileBytes);
                const uint32_t b_base = smem_u32(Bs + prod_b(p) * kTileBytes);
#pragma unroll
                for (int kk = 0; kk < KSTEPS_PER_MMA; ++kk) {
                    // K = 16 elements = two K-adjacent core matrices = 256 bytes
                    const uint64_t ad = smem_desc(a_base + kk * 256, 128, 1024);
                    const uint64_t bd = smem_desc(b_base + kk * 256, 128, 1024);
                    mma_f16(tmem, ad, bd, IDESC, (s > 0 || p > 0 || kk > 0) ? 1u : 0u);
                }
            }
            mma_commit(&mma_bar[b]);
            uses[b]++;
        }
    }
    // wait for the last commits of both buffers
    if (tid == 0) {
        for (int b = 0; b < 2; ++b)
            if (uses[b] > 0 && !abort_sh) {
                if (!mbar_wait_bounded(&mma_bar[b], (uint32_t)((uses[b] - 1) & 1))) abort_sh = 1;
            }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (abort_sh) {
        if (tid == 0) atomicExch(err, 1);
    } else if (nsteps > 0) {
        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31 (rows of the
        // tile) and columns 64 (w / 4) .. +63
        const int quarter = warp & 3, half = warp >> 2;
        const int row = r0 + quarter * 32 + lane;                     // real row of G
        for (int cb = half * 64; cb < half * 64 + 64; cb += 32) {
            float v[32];
            tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)cb, v);
            // pair rows 2a (even lane) and 2a+1 (odd lane)
#pragma unroll
            for (int cc = 0; cc < 32; cc += 2) {
                const float ee = v[cc], eo = v[cc + 1];                 // G[row][2b], G[row][2b+1]
                const float oe = __shfl_xor_sync(0xffffffffu, ee, 1);  // from the partner row
                const float oo = __shfl_xor_sync(0xffffffffu, eo, 1);
                if ((lane & 1) == 0) {
                    const int n = row >> 1, m = (c0 + cb + cc) >> 1;
                    if (n < n_orb && m < n_orb) {
                        // even row: G[2n][2m] = ee, G[2n][2m+1] = eo; odd row (partner): oe, oo
                        double* dst = part + (((int64_t)blockIdx.z * n_orb + n) * n_orb + m) * 2;
                        dst[0] = unscale * ((double)ee + (double)oo);
                        dst[1] = unscale * ((double)eo - (double)oe);
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128u) : "memory");
    }
}

__global__ void k_gram_reduce(const double* __restrict__ part, int nsplit, int64_t n, double scale,
                              double* __restrict__ S) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int k = 0; k < nsplit; ++k) s += part[(int64_t)k * n + e];
        S[e] = scale * s;
    }
}

template <int MODE>
void launch_mode(Domain& d, const float* X, const float* Y, int64_t kchunk, int nsplit, float fscale, double unscale,
                 double* part) {
    constexpr uint32_t smem = 2 * 2 * Split<MODE>::NPART * kTileBytes + 1024;
    static bool attr = false;
    if (!attr) {
        MLMD_CUDA(cudaFuncSetAttribute(k_gram_tc<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr = true;
    }
    const int tiles = (2 * d.ld + BM - 1) / BM;
    dim3 grid(tiles, tiles, (unsigned)nsplit);
    k_gram_tc<MODE><<<grid, 256, smem, d.stream>>>(X, Y, d.ng, d.ld, d.desc.n_orb, kchunk, fscale, unscale, part,
                                                   d.err_flag);
}

}  // namespace

bool launch_overlap_tc(Domain& d, const void* X, const void* Y, double scale, double* S) {
    const int mode = d.desc.gemm_mode;
    if (!d.c64() || mode == MLMD_GEMM_FP32) return false;
    const int no = d.desc.n_orb;
    const int tiles = (2 * d.ld + BM - 1) / BM;
    // about four CTAs per SM over all tiles and K-slices
    int64_t nsplit = std::max<int64_t>(1, std::min<int64_t>((4 * 152 + tiles * tiles / 2) / (tiles * tiles),
                                                            (d.ng + BK - 1) / BK));
    const int64_t kchunk = ((d.ng + nsplit - 1) / nsplit + BK - 1) / BK * BK;
    nsplit = (d.ng + kchunk - 1) / kchunk;
    double* part = (double*)d.mem.get((size_t)nsplit * no * no * 2 * sizeof(double));
    // FP16: a power-of-two scale so that a normalised orbital's entries are O(1)
    float fscale = 1.f;
    double unscale = 1.0;
    if (mode == MLMD_GEMM_FP16) {
        const double typical = 1.0 / std::sqrt((double)d.ng * d.desc.h * d.desc.h * d.desc.h);
        const int e = (int)std::lround(-std::log2(typical));
        fscale = std::ldexp(1.f, e);
        unscale = std::ldexp(1.0, -2 * e);
    }
    const float* Xf = static_cast<const float*>(X);
    const float* Yf = static_cast<const float*>(Y);
    switch (mode) {
        case MLMD_GEMM_BF16: launch_mode<MLMD_GEMM_BF16>(d, Xf, Yf, kchunk, (int)nsplit, fscale, unscale, part); break;
        case MLMD_GEMM_BF16X2: launch_mode<MLMD_GEMM_BF16X2>(d, Xf, Yf, kchunk, (int)nsplit, fscale, unscale, part); break;
        case MLMD_GEMM_BF16X3: launch_mode<MLMD_GEMM_BF16X3>(d, Xf, Yf, kchunk, (int)nsplit, fscale, unscale, part); break;
        default: launch_mode<MLMD_GEMM_FP16>(d, Xf, Yf, kchunk, (int)nsplit, fscale, unscale, part); break;
    }
    const int64_t n = (int64_t)no * no * 2;
    k_gram_reduce<<<(int)std::min<int64_t>((n + 255) / 256, 2048), 256, 0, d.stream>>>(part, (int)nsplit, n, scale, S);
    d.launches += 2;
    MLMD_CUDA(cudaGetLastError());
    d.mem.put(part);
    return true;
}

}  // namespace mlmd
