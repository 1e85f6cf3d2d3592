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
// and Heinecke, ARITH 2019) or FP16 after a power-of-two scale.  The products
// accumulate in FP32 in tensor memory in short runs (about 24 MMAs): the
// tensor core's FP32 accumulation rounds towards zero, so one run over a
// whole K-slice of 10^5 grid points biased the diagonal of S by about 5e-4;
// drain warps add each run into FP32 running sums in registers (rounded to
// nearest), and K-slices of the grid go to different CTAs whose tiles are
// summed in FP64.
//
// Structure: a split pass converts each FP32 operand once into its 16-bit
// parts, stored pre-tiled in device memory: every 128-column x 64-point tile
// is a 16 KiB image of the canonical no-swizzle K-major core-matrix layout
// (core matrix = 8 rows x 16 bytes; K-adjacent cores 128 B apart, 8-row
// groups 1024 B apart).  The GEMM kernel computes one 128 x 128 tile of G
// over a K range: thread 0 streams the tiles with one bulk copy each into a
// ring of shared-memory stages (full / empty mbarriers), thread 32 issues
// the tcgen05.mma instructions (M = N = 128, K = 16, FP32 accumulator in
// tensor memory, two accumulator buffers used in turn, one per run) and frees
// each stage with tcgen05.commit, and warps 2-5 read each finished run with
// tcgen05.ld into their running sums (filled / drained mbarriers), then pair
// rows 2a / 2a+1 with a lane shuffle and write the complex FP64 partial tile.  For a Gram of one array
// with itself only the upper-triangular tiles are computed.  Every mbarrier
// wait is bounded; tensor memory is always freed.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>

#include "mlmd_internal.cuh"
#include "tc_ptx.cuh"

namespace mlmd {
namespace {

using namespace tc;

// Split pass: X (FP32, [N_g][ncols] real) -> parts[p][mt][ks] 16 KiB tile
// images (128 real columns x 64 grid points, canonical K-major core-matrix
// layout), zero-padded beyond N_g and ncols.  Block (mt, ks), 256 threads,
// item = (column c, k-group kg): 8 consecutive points of one column.
template <int MODE>
__global__ void __launch_bounds__(256) k_split_tiles(const float* __restrict__ X, int64_t ng, int ncols, int nmt,
                                                     int nks, float fscale, unsigned char* __restrict__ parts) {
    constexpr int NPART = Split<MODE>::NPART;
    const int mt = blockIdx.x;
    const int64_t ks = blockIdx.y;
    for (int item = threadIdx.x; item < (BK / 8) * BM; item += 256) {
        const int c = item % BM, kg = item / BM;
        const int col = mt * BM + c;
        uint16_t pk[3][8];
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
            const int64_t g = ks * BK + kg * 8 + kk;
            const float x = (g < ng && col < ncols) ? __ldg(X + g * ncols + col) : 0.f;
            uint16_t pp[3];
            split_value<MODE>(x, fscale, pp);
#pragma unroll
            for (int i = 0; i < 3; ++i) pk[i][kk] = pp[i];
        }
#pragma unroll
        for (int i = 0; i < NPART; ++i) {
            uint4 w;
            w.x = pk[i][0] | ((uint32_t)pk[i][1] << 16);
            w.y = pk[i][2] | ((uint32_t)pk[i][3] << 16);
            w.z = pk[i][4] | ((uint32_t)pk[i][5] << 16);
            w.w = pk[i][6] | ((uint32_t)pk[i][7] << 16);
            unsigned char* tile = parts + (((int64_t)i * nmt + mt) * nks + ks) * kTileBytes;
            *reinterpret_cast<uint4*>(tile + tile_offset(c, kg * 8)) = w;
        }
    }
}

// K-steps (BK grid points each) per accumulation run: about 24 MMAs
template <int MODE> struct RunSteps {
    static constexpr int value = (24 / (Split<MODE>::NPROD * KSTEPS_PER_MMA)) > 0
                                     ? 24 / (Split<MODE>::NPROD * KSTEPS_PER_MMA) : 1;
};

// part[z][n][m] (complex FP64) for the real output tile (ta, tb) of G = Xr^T Yr
// over K-slice z.  Thread 0 feeds a ring of STAGES buffers with bulk copies
// of the pre-split tiles; thread 32 issues the MMAs, frees each buffer with
// a commit and closes each run of RunSteps K-steps with a commit to
// filled[b] (runs alternate between the two accumulators b = 0, 1); warps
// 2-5 add each finished run to their FP32 running sums and arrive on
// drained[b] so the accumulator can take the run after next.  tri != 0:
// blockIdx.x enumerates the upper-triangular tile pairs (ta <= tb).
template <int MODE>
__global__ void __launch_bounds__(192, 1)
    k_gram_tc(const unsigned char* __restrict__ pa, const unsigned char* __restrict__ pb, int nmt, int nks,
              int ks_per_split, int n_orb, int tri, double unscale, double* __restrict__ part, int* __restrict__ err) {
    constexpr int NPART = Split<MODE>::NPART, NPROD = Split<MODE>::NPROD, STAGES = Stages<MODE>::value;
    constexpr int RUN = RunSteps<MODE>::value;
    constexpr uint32_t STAGE_BYTES = 2 * NPART * kTileBytes;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES], filled[2], drained[2], done;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_sh;
    __shared__ int consumed_sh;          // steps whose copies the MMA thread has seen land

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int ta, tb;
    if (tri) {          // blockIdx.x -> (ta, tb), ta <= tb, row-major over the upper triangle
        int r = blockIdx.x, a = 0;
        while (r >= nmt - a) { r -= nmt - a; ++a; }
        ta = a;
        tb = a + r;
    } else {
        ta = blockIdx.x / nmt;
        tb = blockIdx.x % nmt;
    }
    const int ks0 = blockIdx.y * ks_per_split;
    const int nsteps = min(ks_per_split, nks - ks0);
    const int nruns = (nsteps + RUN - 1) / RUN;

    if (warp == 0) {     // two 128-column FP32 accumulators
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(256u)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int st = 0; st < STAGES; ++st) {
            mbar_init(&full[st], 1);
            mbar_init(&empty[st], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&filled[b], 1);
            mbar_init(&drained[b], 4);       // one arrival per drain warp
        }
        mbar_init(&done, 1);
        abort_sh = 0;
        consumed_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    constexpr uint32_t IDESC = instr_desc(MODE == MLMD_GEMM_FP16 ? 0u : 1u);
    bool drained_all = false;            // drain warps: every run is in the sums
    float sum[BN];                       // drain warps: running sums of one tile row

    int issued = 0;                      // producer: steps whose copies were issued
    if (tid == 0) {                     // producer
        for (int i = 0; i < nsteps && !abort_sh; ++i) {
            const int st = i % STAGES;
            if (i >= STAGES && !mbar_wait_bounded(&empty[st], (uint32_t)((i / STAGES - 1) & 1))) {
                abort_sh = 1;
                break;
            }
            unsigned char* As = smem + st * STAGE_BYTES;
            unsigned char* Bs = As + NPART * kTileBytes;
            mbar_expect_tx(&full[st], STAGE_BYTES);
            const int64_t ks = ks0 + i;
#pragma unroll
            for (int p = 0; p < NPART; ++p) {
                bulk_load(As + p * kTileBytes, pa + (((int64_t)p * nmt + ta) * nks + ks) * kTileBytes, kTileBytes,
                          &full[st]);
                bulk_load(Bs + p * kTileBytes, pb + (((int64_t)p * nmt + tb) * nks + ks) * kTileBytes, kTileBytes,
                          &full[st]);
            }
            issued = i + 1;
        }
    } else if (tid == 32) {             // MMA issuer
        for (int i = 0; i < nsteps; ++i) {
            const int run = i / RUN, b = run & 1;
            const bool first = (i % RUN) == 0;
            // the run before last in this accumulator must have been drained
            if (first && run >= 2 && !mbar_wait_bounded(&drained[b], (uint32_t)((run / 2 - 1) & 1))) {
                abort_sh = 1;
                break;
            }
            const int st = i % STAGES;
            if (!mbar_wait_bounded(&full[st], (uint32_t)((i / STAGES) & 1))) {
                abort_sh = 1;
                break;
            }
            consumed_sh = i + 1;
            tc_fence_after();
            const uint32_t As = smem_u32(smem + st * STAGE_BYTES);
            const uint32_t Bs = As + NPART * kTileBytes;
            const uint32_t acc = tmem + (uint32_t)(b * BN);
#pragma unroll
            for (int p = 0; p < NPROD; ++p)
#pragma unroll
                for (int kk = 0; kk < KSTEPS_PER_MMA; ++kk) {
                    const uint64_t ad = smem_desc(As + prod_a(p, NPROD) * kTileBytes + kk * 256, 128, 1024);
                    const uint64_t bd = smem_desc(Bs + prod_b(p, NPROD) * kTileBytes + kk * 256, 128, 1024);
                    mma_f16(acc, ad, bd, IDESC, (first && p == 0 && kk == 0) ? 0u : 1u);
                }
            mma_commit(&empty[st]);
            if ((i % RUN) == RUN - 1 || i == nsteps - 1) mma_commit(&filled[b]);
        }
        mma_commit(&done);              // all MMAs issued above have completed when this fires
    } else if (warp >= 2) {             // drain warps: TMEM lanes 32 (warp % 4) .. +31
        const uint32_t lanes = (uint32_t)((warp & 3) * 32) << 16;
#pragma unroll
        for (int c = 0; c < BN; ++c) sum[c] = 0.f;
        int r = 0;
        for (; r < nruns; ++r) {
            const int b = r & 1;
            if (!mbar_wait_bounded(&filled[b], (uint32_t)((r / 2) & 1))) {
                abort_sh = 1;
                break;
            }
            tc_fence_after();
#pragma unroll
            for (int cb = 0; cb < BN; cb += 32) {
                float v[32];
                tmem_ld32(tmem + lanes + (uint32_t)(b * BN + cb), v);
#pragma unroll
                for (int cc = 0; cc < 32; ++cc) sum[cb + cc] += v[cc];
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&drained[b]);
        }
        drained_all = r == nruns;
    }
    __syncthreads();
    if (nsteps > 0 && !mbar_wait_bounded(&done, 0)) abort_sh = 1;
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (abort_sh) {
        if (tid == 0) {
            atomicExch(err, 1);
            // let the bulk copies still in flight land (bounded): every step
            // issued but not seen by the MMA thread, on its own phase
            for (int i = consumed_sh; i < issued; ++i)
                (void)mbar_wait_bounded(&full[i % STAGES], (uint32_t)((i / STAGES) & 1));
        }
    } else if (warp >= 2 && drained_all && nsteps > 0) {
        // row of G held by this lane; rows 2a and 2a+1 sit in neighbouring lanes
        const int row = ta * BM + (warp & 3) * 32 + lane;
#pragma unroll
        for (int cc = 0; cc < BN; cc += 2) {
            const float ee = sum[cc], eo = sum[cc + 1];                 // G[row][2b], G[row][2b+1]
            const float oe = __shfl_xor_sync(0xffffffffu, ee, 1);      // the partner row's
            const float oo = __shfl_xor_sync(0xffffffffu, eo, 1);
            if ((lane & 1) == 0) {
                const int n = row >> 1, m = (tb * BN + cc) >> 1;
                if (n < n_orb && m < n_orb) {
                    double* dst = part + (((int64_t)blockIdx.y * n_orb + n) * n_orb + m) * 2;
                    dst[0] = unscale * ((double)ee + (double)oo);
                    dst[1] = unscale * ((double)eo - (double)oe);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256u) : "memory");
    }
}

// S[n][m] = scale * sum_z part[z][n][m]; with tri, entries below the computed
// tile triangle are conj(S[m][n]).
__global__ void k_gram_reduce(const double* __restrict__ part, int nsplit, int n_orb, int tri, double scale,
                              double* __restrict__ S) {
    const int64_t nn = (int64_t)n_orb * n_orb;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nn; e += (int64_t)gridDim.x * blockDim.x) {
        const int n = (int)(e / n_orb), m = (int)(e % n_orb);
        const bool mirror = tri && (n / (BM / 2)) > (m / (BN / 2));
        const int64_t src = mirror ? (int64_t)m * n_orb + n : e;
        double re = 0.0, im = 0.0;
        for (int k = 0; k < nsplit; ++k) {
            re += part[((int64_t)k * nn + src) * 2];
            im += part[((int64_t)k * nn + src) * 2 + 1];
        }
        S[e * 2] = scale * re;
        S[e * 2 + 1] = scale * (mirror ? -im : im);
    }
}

template <int MODE>
void gram_mode(Domain& d, const float* X, const float* Y, double scale, double* S, float fscale, double unscale) {
    constexpr int NPART = Split<MODE>::NPART, STAGES = Stages<MODE>::value;
    const int ncols = 2 * d.ld, no = d.desc.n_orb;
    const int nmt = (ncols + BM - 1) / BM;
    const int nks = (int)((d.ng + BK - 1) / BK);
    const bool same = X == Y;
    const size_t part_bytes = (size_t)NPART * nmt * nks * kTileBytes;
    unsigned char* pa = (unsigned char*)d.mem.get(part_bytes);
    unsigned char* pb = same ? pa : (unsigned char*)d.mem.get(part_bytes);
    k_split_tiles<MODE><<<dim3(nmt, nks), 256, 0, d.stream>>>(X, d.ng, ncols, nmt, nks, fscale, pa);
    d.launches++;
    if (!same) {
        k_split_tiles<MODE><<<dim3(nmt, nks), 256, 0, d.stream>>>(Y, d.ng, ncols, nmt, nks, fscale, pb);
        d.launches++;
    }
    const int tiles = same ? nmt * (nmt + 1) / 2 : nmt * nmt;
    // about three CTAs per SM (one resident at a time) over tile pairs and K-slices
    int nsplit = std::max(1, std::min((3 * 152 + tiles / 2) / tiles, nks));
    const int ks_per_split = (nks + nsplit - 1) / nsplit;
    nsplit = (nks + ks_per_split - 1) / ks_per_split;
    double* part = (double*)d.mem.get((size_t)nsplit * no * no * 2 * sizeof(double));
    constexpr uint32_t smem = STAGES * 2 * NPART * kTileBytes + 1024;
    ensure_dynamic_smem(reinterpret_cast<const void*>(k_gram_tc<MODE>), smem);
    k_gram_tc<MODE><<<dim3(tiles, nsplit), 192, smem, d.stream>>>(pa, pb, nmt, nks, ks_per_split, no, same ? 1 : 0,
                                                                  unscale, part, d.err_flag);
    const int64_t nn = (int64_t)no * no;
    k_gram_reduce<<<(int)std::min<int64_t>((nn + 255) / 256, 2048), 256, 0, d.stream>>>(part, nsplit, no, same ? 1 : 0,
                                                                                      scale, S);
    d.launches += 2;
    MLMD_CUDA(cudaGetLastError());
    d.mem.put(part);
    if (!same) d.mem.put(pb);
    d.mem.put(pa);
}

}  // namespace

bool launch_overlap_tc(Domain& d, const void* X, const void* Y, double scale, double* S) {
    const int mode = d.desc.gemm_mode;
    if (!d.c64() || mode == MLMD_GEMM_FP32) return false;
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
        case MLMD_GEMM_BF16: gram_mode<MLMD_GEMM_BF16>(d, Xf, Yf, scale, S, fscale, unscale); break;
        case MLMD_GEMM_BF16X2: gram_mode<MLMD_GEMM_BF16X2>(d, Xf, Yf, scale, S, fscale, unscale); break;
        case MLMD_GEMM_BF16X3: gram_mode<MLMD_GEMM_BF16X3>(d, Xf, Yf, scale, S, fscale, unscale); break;
        default: gram_mode<MLMD_GEMM_FP16>(d, Xf, Yf, scale, S, fscale, unscale); break;
    }
    return true;
}

}  // namespace mlmd
