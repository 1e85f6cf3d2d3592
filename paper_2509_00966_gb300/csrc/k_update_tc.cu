// Orbital updates Y = Z + X Mc on the tcgen05 tensor cores (Sec. V.B.7):
// the re-orthonormalisation Psi <- Psi L^{-H} of Sec. VI.C, written as
// Y = X + X (M - I) so that the split-precision error scales with |M - I|,
// which is small when the orbitals were nearly orthonormal already; and the
// KS-space nonlocal correction of Eq. 5, Psi(t) + Psi(0) (-delta C).
//
// For complex64 X ([N_g][ld] interleaved) the complex product is one real
// GEMM on the real view Xr ([N_g][2 ld]):  Yr = Xr + Xr R  with the real
// 2ld x 2ld embedding R of M - I:
//     R[2a][2b] = R[2a+1][2b+1] = Re(M - I)[a][b],
//     R[2a][2b+1] = Im M[a][b],   R[2a+1][2b] = -Im M[a][b].
// (R embeds Mc the same way.)  The MMA's M dimension is the grid point (128
// points per tile), N the output real column (128 per tile) and K the input
// real column.  A = Xr is K-major as stored; B is R^T, built K-major from M.  Both are split once into 16-bit
// parts and stored as 16 KiB canonical tile images (the layout of the Gram
// kernel); the GEMM kernel streams them with bulk copies through a ring of
// shared-memory stages, accumulates all split products in FP32 in tensor
// memory and adds X in the epilogue.  FP16 operands carry power-of-two
// scales: X by the typical orbital magnitude, R by its largest entry (found
// on the device).
#include <algorithm>
#include <cmath>

#include "mlmd_internal.cuh"
#include "tc_ptx.cuh"

namespace mlmd {
namespace {

using namespace tc;

// Split pass for A: Xr [N_g][ncols] FP32 -> parts[p][gt][kt], tile image of
// 128 grid points (rows) x 64 real columns (K), zero beyond N_g and ncols.
// Block (kt, gt), 256 threads; item = (row r, K-group kg of 8 columns).
template <int MODE>
__global__ void __launch_bounds__(256) k_split_rows(const float* __restrict__ X, int64_t ng, int ncols, int ngt,
                                                    int nkt, float fscale, unsigned char* __restrict__ parts) {
    constexpr int NPART = Split<MODE>::NPART;
    const int kt = blockIdx.x, gt = blockIdx.y;
    for (int item = threadIdx.x; item < BM * (BK / 8); item += 256) {
        const int kg = item & 7, r = item >> 3;
        const int64_t g = (int64_t)gt * BM + r;
        const int c0 = kt * BK + kg * 8;
        float x[8];
        if (g < ng && c0 < ncols) {             // ncols is a multiple of 16: all 8 columns valid
            const float4 a = __ldg(reinterpret_cast<const float4*>(X + g * ncols + c0));
            const float4 b = __ldg(reinterpret_cast<const float4*>(X + g * ncols + c0 + 4));
            x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
            x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
        } else {
#pragma unroll
            for (int i = 0; i < 8; ++i) x[i] = 0.f;
        }
        uint16_t pk[3][8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            uint16_t pp[3];
            split_value<MODE>(x[i], fscale, pp);
#pragma unroll
            for (int q = 0; q < 3; ++q) pk[q][i] = pp[q];
        }
#pragma unroll
        for (int q = 0; q < NPART; ++q) {
            uint4 w;
            w.x = pk[q][0] | ((uint32_t)pk[q][1] << 16);
            w.y = pk[q][2] | ((uint32_t)pk[q][3] << 16);
            w.z = pk[q][4] | ((uint32_t)pk[q][5] << 16);
            w.w = pk[q][6] | ((uint32_t)pk[q][7] << 16);
            unsigned char* tile = parts + (((int64_t)q * ngt + gt) * nkt + kt) * kTileBytes;
            *reinterpret_cast<uint4*>(tile + tile_offset(r, kg * 8)) = w;
        }
    }
}

// Largest |entry| of M - I (sub_id) or M (as FP32 bits; non-negative floats
// order like their bit patterns), for the FP16 scale of R.
__global__ void k_update_maxabs(const double* __restrict__ M, int n, int sub_id, unsigned int* __restrict__ out) {
    float m = 0.f;
    const int64_t nn = (int64_t)n * n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nn; e += (int64_t)gridDim.x * blockDim.x) {
        const int a = (int)(e / n), b = (int)(e % n);
        const double re = M[e * 2] - (sub_id && a == b ? 1.0 : 0.0), im = M[e * 2 + 1];
        m = fmaxf(m, (float)fmax(fabs(re), fabs(im)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

// 2^-e with 2^e the power of two just above the largest entry of R (1 if R = 0)
__device__ __forceinline__ float r_scale(const unsigned int* maxbits) {
    const float m = __uint_as_float(*maxbits);
    if (!(m > 0.f) || !isfinite(m)) return 1.f;
    int e;
    frexpf(m, &e);          // m = f 2^e, f in [0.5, 1)
    return ldexpf(1.f, -e);
}

// Split pass for B: tile images of R^T, parts[p][jt][kt], 128 output real
// columns j (rows of the tile) x 64 input real columns k (K).  Block (kt, jt).
template <int MODE>
__global__ void __launch_bounds__(256) k_split_embed(const double* __restrict__ M, int n, int sub_id, int njt, int nkt,
                                                     const unsigned int* __restrict__ maxbits,
                                                     unsigned char* __restrict__ parts) {
    constexpr int NPART = Split<MODE>::NPART;
    const int kt = blockIdx.x, jt = blockIdx.y;
    const float fscale = (MODE == MLMD_GEMM_FP16) ? r_scale(maxbits) : 1.f;
    for (int item = threadIdx.x; item < BN * (BK / 8); item += 256) {
        const int kg = item & 7, r = item >> 3;
        const int j = jt * BN + r, b = j >> 1, t = j & 1;
        uint16_t pk[3][8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int k = kt * BK + kg * 8 + i, a = k >> 1, s = k & 1;
            float v = 0.f;
            if (a < n && b < n) {
                const double re = M[((int64_t)a * n + b) * 2] - (sub_id && a == b ? 1.0 : 0.0);
                const double im = M[((int64_t)a * n + b) * 2 + 1];
                v = (float)(s == t ? re : (s == 0 ? im : -im));
            }
            uint16_t pp[3];
            split_value<MODE>(v, fscale, pp);
#pragma unroll
            for (int q = 0; q < 3; ++q) pk[q][i] = pp[q];
        }
#pragma unroll
        for (int q = 0; q < NPART; ++q) {
            uint4 w;
            w.x = pk[q][0] | ((uint32_t)pk[q][1] << 16);
            w.y = pk[q][2] | ((uint32_t)pk[q][3] << 16);
            w.z = pk[q][4] | ((uint32_t)pk[q][5] << 16);
            w.w = pk[q][6] | ((uint32_t)pk[q][7] << 16);
            unsigned char* tile = parts + (((int64_t)q * njt + jt) * nkt + kt) * kTileBytes;
            *reinterpret_cast<uint4*>(tile + tile_offset(r, kg * 8)) = w;
        }
    }
}

// One 128-point x 128-column tile of Y: thread 0 streams A and B tiles into a
// ring of STAGES shared-memory buffers, thread 32 issues the MMAs (all split
// products of each K-step into one FP32 accumulator) and frees each buffer
// with a commit; then the four warps read their 32 rows of the accumulator
// and write Y = Z + unscale * acc.  Every wait is bounded; on a timeout the
// kernel raises *err, lets copies in flight land and frees tensor memory.
template <int MODE>
__global__ void __launch_bounds__(128, 1)
    k_update_tc(const unsigned char* __restrict__ pa, const unsigned char* __restrict__ pb, int ngt, int njt, int nkt,
                const float* __restrict__ Z, float* __restrict__ Y, int64_t ng, int ncols, float xunscale,
                const unsigned int* __restrict__ maxbits, int upper, int* __restrict__ err) {
    constexpr int NPART = Split<MODE>::NPART, NPROD = Split<MODE>::NPROD, STAGES = Stages<MODE>::value;
    constexpr uint32_t STAGE_BYTES = 2 * NPART * kTileBytes;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES], done;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_sh;
    __shared__ int consumed_sh;          // steps whose copies the MMA thread has seen land

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int jt = blockIdx.x, gt = blockIdx.y;
    // upper-triangular M: output columns of tile jt (orbitals jt*64 .. +63)
    // take inputs only from orbitals <= jt*64 + 63, i.e. K-tiles <= 2 jt + 1
    const int nk = upper ? min(nkt, 2 * jt + 2) : nkt;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(128u)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int st = 0; st < STAGES; ++st) {
            mbar_init(&full[st], 1);
            mbar_init(&empty[st], 1);
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

    int issued = 0;                      // producer: steps whose copies were issued
    if (tid == 0) {                     // producer
        for (int i = 0; i < nk && !abort_sh; ++i) {
            const int st = i % STAGES;
            if (i >= STAGES && !mbar_wait_bounded(&empty[st], (uint32_t)((i / STAGES - 1) & 1))) {
                abort_sh = 1;
                break;
            }
            unsigned char* As = smem + st * STAGE_BYTES;
            unsigned char* Bs = As + NPART * kTileBytes;
            mbar_expect_tx(&full[st], STAGE_BYTES);
#pragma unroll
            for (int p = 0; p < NPART; ++p) {
                bulk_load(As + p * kTileBytes, pa + (((int64_t)p * ngt + gt) * nkt + i) * kTileBytes, kTileBytes,
                          &full[st]);
                bulk_load(Bs + p * kTileBytes, pb + (((int64_t)p * njt + jt) * nkt + i) * kTileBytes, kTileBytes,
                          &full[st]);
            }
            issued = i + 1;
        }
    } else if (tid == 32) {             // MMA issuer
        for (int i = 0; i < nk; ++i) {
            const int st = i % STAGES;
            if (!mbar_wait_bounded(&full[st], (uint32_t)((i / STAGES) & 1))) {
                abort_sh = 1;
                break;
            }
            consumed_sh = i + 1;
            tc_fence_after();
            const uint32_t As = smem_u32(smem + st * STAGE_BYTES);
            const uint32_t Bs = As + NPART * kTileBytes;
#pragma unroll
            for (int p = 0; p < NPROD; ++p)
#pragma unroll
                for (int kk = 0; kk < KSTEPS_PER_MMA; ++kk) {
                    const uint64_t ad = smem_desc(As + prod_a(p, NPROD) * kTileBytes + kk * 256, 128, 1024);
                    const uint64_t bd = smem_desc(Bs + prod_b(p, NPROD) * kTileBytes + kk * 256, 128, 1024);
                    mma_f16(tmem, ad, bd, IDESC, (i > 0 || p > 0 || kk > 0) ? 1u : 0u);
                }
            mma_commit(&empty[st]);
        }
        mma_commit(&done);
    }
    __syncthreads();
    // the MMA thread commits `done` after its loop in every case, so the MMAs
    // it issued have finished reading shared memory and writing TMEM once it fires
    if (nk > 0 && !mbar_wait_bounded(&done, 0)) abort_sh = 1;
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
    } else {
        const float unscale = (MODE == MLMD_GEMM_FP16) ? xunscale / r_scale(maxbits) : 1.f;
        const int64_t g = (int64_t)gt * BM + warp * 32 + lane;
        for (int cb = 0; cb < BN; cb += 32) {
            float v[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cb, v);
            const int j0 = jt * BN + cb;
            if (g < ng) {
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int j = j0 + 4 * q;
                    if (j < ncols) {
                        const float4 x = *reinterpret_cast<const float4*>(Z + g * ncols + j);
                        float4 y;
                        y.x = x.x + unscale * v[4 * q];
                        y.y = x.y + unscale * v[4 * q + 1];
                        y.z = x.z + unscale * v[4 * q + 2];
                        y.w = x.w + unscale * v[4 * q + 3];
                        *reinterpret_cast<float4*>(Y + g * ncols + j) = y;
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

template <int MODE>
void update_mode(Domain& d, const float* X, const double* M, int sub_id, const float* Z, float* Y, bool upper) {
    constexpr int NPART = Split<MODE>::NPART, STAGES = Stages<MODE>::value;
    const int n = d.desc.n_orb, ncols = 2 * d.ld;
    const int ngt = (int)((d.ng + BM - 1) / BM);
    const int nkt = (ncols + BK - 1) / BK;
    const int njt = (ncols + BN - 1) / BN;
    // X scale for FP16: a power of two that makes a normalised orbital's entries O(1)
    float fx = 1.f, xunscale = 1.f;
    if (MODE == MLMD_GEMM_FP16) {
        const double typical = 1.0 / std::sqrt((double)d.ng * d.desc.h * d.desc.h * d.desc.h);
        const int e = (int)std::lround(-std::log2(typical));
        fx = std::ldexp(1.f, e);
        xunscale = std::ldexp(1.f, -e);
    }
    unsigned char* pa = (unsigned char*)d.mem.get((size_t)NPART * ngt * nkt * kTileBytes);
    unsigned char* pb = (unsigned char*)d.mem.get((size_t)NPART * njt * nkt * kTileBytes);
    unsigned int* maxbits = (unsigned int*)d.mem.get(256);
    MLMD_CUDA(cudaMemsetAsync(maxbits, 0, sizeof(unsigned int), d.stream));
    if (MODE == MLMD_GEMM_FP16) {
        const int64_t nn = (int64_t)n * n;
        k_update_maxabs<<<(int)std::min<int64_t>((nn + 255) / 256, 1024), 256, 0, d.stream>>>(M, n, sub_id, maxbits);
        d.launches++;
    }
    k_split_rows<MODE><<<dim3(nkt, ngt), 256, 0, d.stream>>>(X, d.ng, ncols, ngt, nkt, fx, pa);
    k_split_embed<MODE><<<dim3(nkt, njt), 256, 0, d.stream>>>(M, n, sub_id, njt, nkt, maxbits, pb);
    d.launches += 2;
    constexpr uint32_t smem = STAGES * 2 * NPART * kTileBytes + 1024;
    ensure_dynamic_smem(reinterpret_cast<const void*>(k_update_tc<MODE>), smem);
    k_update_tc<MODE><<<dim3(njt, ngt), 128, smem, d.stream>>>(pa, pb, ngt, njt, nkt, Z, Y, d.ng, ncols, xunscale,
                                                               maxbits, upper ? 1 : 0, d.err_flag);
    d.launches++;
    MLMD_CUDA(cudaGetLastError());
    d.mem.put(maxbits);
    d.mem.put(pb);
    d.mem.put(pa);
}

}  // namespace

namespace {

bool gemm_tc(Domain& d, const void* X, const double* M, int sub_id, const void* Z, void* Y, bool upper) {
    const int mode = d.desc.gemm_mode;
    if (!d.c64() || mode == MLMD_GEMM_FP32) return false;
    const float* Xf = static_cast<const float*>(X);
    const float* Zf = static_cast<const float*>(Z);
    float* Yf = static_cast<float*>(Y);
    switch (mode) {
        case MLMD_GEMM_BF16: update_mode<MLMD_GEMM_BF16>(d, Xf, M, sub_id, Zf, Yf, upper); break;
        case MLMD_GEMM_BF16X2: update_mode<MLMD_GEMM_BF16X2>(d, Xf, M, sub_id, Zf, Yf, upper); break;
        case MLMD_GEMM_BF16X3: update_mode<MLMD_GEMM_BF16X3>(d, Xf, M, sub_id, Zf, Yf, upper); break;
        default: update_mode<MLMD_GEMM_FP16>(d, Xf, M, sub_id, Zf, Yf, upper); break;
    }
    return true;
}

}  // namespace

bool launch_update_tc(Domain& d, const void* X, const double* M, void* Y, bool upper) {
    return gemm_tc(d, X, M, 1, X, Y, upper);
}

bool launch_gemm_add_tc(Domain& d, const void* X, const double* Mc, const void* Z, void* Y) {
    return gemm_tc(d, X, Mc, 0, Z, Y, false);
}

}  // namespace mlmd
