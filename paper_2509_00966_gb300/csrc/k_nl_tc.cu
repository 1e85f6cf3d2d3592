// Nonlocal term of Eq. 3 on the tcgen05 tensor cores, for domains where
// many projector spheres overlap every grid point (Sec. V.B.5: projection
// and scatter-back as GEMMs; Sec. V.B.7: BF16 split products).
//
// The grid is cut into bricks of 8 x 4 x 4 = 128 points.  For one brick the
// atoms whose spheres touch it give R = NP x (atoms) projector rows, and the
// two halves of the nonlocal term are dense GEMMs over the brick:
//
//   scatter     out[p][n] += gamma sum_r B[p][r] (D o P)[r][n]     (M = points, K = rows,   N = orbital reals)
//   projection  P[r][n]   += dV    sum_p B[p][r] w[p][n]           (M = rows,   K = points, N = orbital reals)
//
// with B[p][r] = beta_r(p) if p lies in the sphere of r's atom, else 0.
// Complex orbitals enter as interleaved (re, im) real columns (B is real).
// B is not stored: the producer warps evaluate the projector values of the
// brick's atoms in FP32 (min-image displacement, Gaussian, normalisation
// from the FP64 lists) and mask them with a per-(brick, atom) 128-bit
// membership set taken from the exact FP64 neighbour lists, so sphere
// membership is the lists' own.  Every FP32 operand is split into three
// bf16 parts (x ~ x0 + x1 + x2) and the six products with i + j <= 2 are
// accumulated in FP32 in tensor memory, smallest first.
//
// Pipeline of one CTA (256 threads): every thread produces its share of a
// K-chunk (32 rows or 32 points) into a ring stage in shared memory, fences
// the writes into the async proxy and arrives on the stage's `full`
// barrier; thread 0 waits for `full`, issues the MMAs of the chunk and
// commits them to the stage's `empty` barrier, which the producers wait on
// before they refill the stage.  Every wait is bounded (~2 s); on expiry
// the CTA raises the domain's error word, waits (bounded) for its MMAs and
// frees its tensor memory.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <vector>

#include "mlmd_internal.cuh"
#include "tc_ptx.cuh"

namespace mlmd {

struct NlTc {
    int nbx = 0, nby = 0, nbz = 0, nbricks = 0;
    int max_atoms = 0;            // most atoms touching one brick
    int32_t* bstart = nullptr;    // [nbricks + 1] ranges of batom / bmask
    int32_t* batom = nullptr;     // global atom ids, ascending per brick
    uint4* bmask = nullptr;       // membership of the brick's 128 points in the atom's sphere
    float4* apos = nullptr;       // [n_atoms] positions (x, y, z, 0), bohr
    float* anrm = nullptr;        // [n_atoms][NP] normalisation of each projector (dV sum b^2 = 1)
    float* aD = nullptr;          // [n_atoms][NP] strengths D
};

namespace {

using namespace tc;

constexpr int BX = 8, BY = 4, BZ = 4, BP = BX * BY * BZ;   // brick of 128 points
constexpr int KC = 32;                                      // K elements per ring stage
constexpr uint32_t A_PART = 128 * KC * 2;                   // one 16-bit part of a 128-row A tile
constexpr int NT = 256;                                     // threads per CTA

struct TcGeo {
    int nx, ny, nz, nbx, nby;
    int ld2;                      // real columns of an orbital row (2 ld)
    float h, L[3], invL[3];
    float cexp[2];                // -log2(e) / (2 rc^2) of the two projector widths
    float invrc[2];
    const int32_t* bstart;
    const int32_t* batom;
    const uint4* bmask;
    const float4* apos;
    const float* anrm;
    const float* aD;
};

// Byte offset of the 16-byte unit (row, K-octet j) of a K-major canonical
// tile with K = 32: core matrices of 8 rows x 16 bytes, the four K-cores of
// a row group adjacent (LBO = 128 B), row groups 512 B apart (SBO).
__device__ __forceinline__ uint32_t unit_off(int row, int j) { return (uint32_t)((row >> 3) * 512 + j * 128 + (row & 7) * 16); }

// tcgen05.mma kind::f16 instruction descriptor: FP32 accumulator, BF16 A and
// B, K-major, M = 128, N given (a multiple of 16, at most 256).
__device__ __forceinline__ uint32_t idesc_n(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void bf16x3(float x, uint16_t (&p)[3]) { split_value<MLMD_GEMM_BF16X3>(x, 1.f, p); }

// Eight FP32 values -> one 16-byte unit per bf16 part, stored at base + part * part_bytes + off.
__device__ __forceinline__ void store_unit(unsigned char* base, uint32_t part_bytes, uint32_t off, const float (&v)[8]) {
    uint16_t q[8][3];
#pragma unroll
    for (int e = 0; e < 8; ++e) bf16x3(v[e], q[e]);
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        uint4 u;
        u.x = (uint32_t)q[0][s] | ((uint32_t)q[1][s] << 16);
        u.y = (uint32_t)q[2][s] | ((uint32_t)q[3][s] << 16);
        u.z = (uint32_t)q[4][s] | ((uint32_t)q[5][s] << 16);
        u.w = (uint32_t)q[6][s] | ((uint32_t)q[7][s] << 16);
        *reinterpret_cast<uint4*>(base + (size_t)s * part_bytes + off) = u;
    }
}

// Grid coordinates of point p of brick (bx, by, bz); false outside the grid.
__device__ __forceinline__ bool brick_point(const TcGeo& G, int bx, int by, int bz, int p, int& x, int& y, int& z) {
    x = bx * BX + (p & 7);
    y = by * BY + ((p >> 3) & 3);
    z = bz * BZ + (p >> 5);
    return x < G.nx && y < G.ny && z < G.nz;
}

// Per-brick atom data staged in shared memory at kernel start (so that the
// producers' inner loops make no dependent global loads): position,
// membership set, projector normalisation and D of each of the brick's atoms,
// and its global index.
template <int NP> struct SAtoms {
    float4* pos;
    uint4* mask;
    float* nrm;                   // [na][NP]
    float* D;                     // [na][NP]
    int* id;
    static size_t bytes(int na) { return (size_t)na * (16 + 16 + 8 * NP + 4) + 64; }
};

template <int NP>
__device__ __forceinline__ SAtoms<NP> stage_atoms(const TcGeo& G, unsigned char* base, int a0, int na) {
    SAtoms<NP> S;
    S.pos = reinterpret_cast<float4*>(base);
    S.mask = reinterpret_cast<uint4*>(S.pos + na);
    S.nrm = reinterpret_cast<float*>(S.mask + na);
    S.D = S.nrm + (size_t)na * NP;
    S.id = reinterpret_cast<int*>(S.D + (size_t)na * NP);
    for (int k = threadIdx.x; k < na; k += blockDim.x) {
        const int a = G.batom[a0 + k];
        S.id[k] = a;
        S.pos[k] = G.apos[a];
        S.mask[k] = G.bmask[a0 + k];
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            S.nrm[k * NP + i] = G.anrm[(size_t)a * NP + i];
            S.D[k * NP + i] = G.aD[(size_t)a * NP + i];
        }
    }
    return S;
}

// The NP projector values of staged atom k at grid point (x, y, z),
// normalised; the caller masks them with the sphere membership.
template <int NP>
__device__ __forceinline__ void beta_at(const TcGeo& G, const SAtoms<NP>& S, int k, int x, int y, int z, float (&b)[NP]) {
    const float4 pa = S.pos[k];
    float dl[3] = {(float)x * G.h - pa.x, (float)y * G.h - pa.y, (float)z * G.h - pa.z};
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) dl[ax] -= G.L[ax] * floorf(dl[ax] * G.invL[ax] + 0.5f);
    const float d2 = dl[0] * dl[0] + dl[1] * dl[1] + dl[2] * dl[2];
#pragma unroll
    for (int set = 0; set < NP / 4; ++set) {
        const float e = exp2f(d2 * G.cexp[set]);
        const float* nr = S.nrm + k * NP + 4 * set;
        b[4 * set] = nr[0] * e;
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) b[4 * set + 1 + ax] = nr[1 + ax] * (dl[ax] * G.invrc[set]) * e;
    }
}

// Projector i of staged atom k at grid point (x, y, z), normalised.
template <int NP>
__device__ __forceinline__ float beta_one(const TcGeo& G, const SAtoms<NP>& S, int k, int i, int x, int y, int z) {
    const float4 pa = S.pos[k];
    float dl[3] = {(float)x * G.h - pa.x, (float)y * G.h - pa.y, (float)z * G.h - pa.z};
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) dl[ax] -= G.L[ax] * floorf(dl[ax] * G.invL[ax] + 0.5f);
    const float d2 = dl[0] * dl[0] + dl[1] * dl[1] + dl[2] * dl[2];
    const int set = i >> 2, c = i & 3;
    const float e = exp2f(d2 * G.cexp[set]);
    const float f = c == 0 ? 1.f : (c == 1 ? dl[0] : (c == 2 ? dl[1] : dl[2])) * G.invrc[set];
    return S.nrm[k * NP + i] * f * e;
}

__device__ __forceinline__ bool mask_bit(const uint4& m, int p) {
    const uint32_t w = p < 32 ? m.x : p < 64 ? m.y : p < 96 ? m.z : m.w;
    return (w >> (p & 31)) & 1u;
}

// Issue the MMAs of one ring stage: two K = 16 steps, six split products
// (smallest first), the N columns in one or two instructions.
__device__ __forceinline__ void issue_chunk(uint32_t tmem, uint32_t a_base, uint32_t b_base, uint32_t b_part, int ncols,
                                            bool first) {
    const int n0 = ncols <= 256 ? ncols : ((ncols / 2 + 15) / 16) * 16;
#pragma unroll
    for (int kk = 0; kk < 2; ++kk)
#pragma unroll
        for (int p = 0; p < 6; ++p) {
            const uint64_t ad = smem_desc(a_base + prod_a(p, 6) * A_PART + kk * 256, 128, 512);
            const uint32_t acc = (first && kk == 0 && p == 0) ? 0u : 1u;
            const uint32_t bp = b_base + prod_b(p, 6) * b_part + kk * 256;
            mma_f16(tmem, ad, smem_desc(bp, 128, 512), idesc_n(n0), acc);
            if (ncols > n0)
                mma_f16(tmem + (uint32_t)n0, ad, smem_desc(bp + (uint32_t)(n0 >> 3) * 512, 128, 512),
                        idesc_n(ncols - n0), acc);
        }
}

// Tensor memory for one accumulator of ncols FP32 columns: the smallest
// power of two >= ncols (at least 32), so that a small domain leaves room
// for other CTAs on the SM.
__device__ __forceinline__ uint32_t tmem_cols(int ncols) {
    uint32_t c = 32;
    while (c < (uint32_t)ncols) c <<= 1;
    return c;
}
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t cols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t t, uint32_t cols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(t), "r"(cols) : "memory");
}

// One B-operand item: 8 K-values (rows j*8 .. +7 of the chunk) x 4 orbital
// columns nq*4 .. +3, loaded as 8 float4 by the caller; stored as 4 units
// (one per column) of the K-major tile, each in three bf16 parts.
__device__ __forceinline__ void store_b_item(unsigned char* sb, uint32_t b_part, int j, int nq, const float4 (&c)[8],
                                             const float (&scale)[8]) {
    float v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = scale[e] * c[e].x;
    store_unit(sb, b_part, unit_off(4 * nq + 0, j), v);
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = scale[e] * c[e].y;
    store_unit(sb, b_part, unit_off(4 * nq + 1, j), v);
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = scale[e] * c[e].z;
    store_unit(sb, b_part, unit_off(4 * nq + 2, j), v);
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = scale[e] * c[e].w;
    store_unit(sb, b_part, unit_off(4 * nq + 3, j), v);
}

constexpr int BMAX = 2;                             // B items per thread per chunk (ncols <= 384)

// ---------------------------------------------------------------------------
// scatter: out[p] += gamma sum_r B[p][r] D_r P[r]   (one CTA per brick)
// ---------------------------------------------------------------------------
template <int NP>
__global__ void __launch_bounds__(NT, 1)
    k_nl_scatter_tc(TcGeo G, const float* __restrict__ P, float* __restrict__ out, float gre, float gim, int stages,
                    int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    __shared__ __align__(8) uint64_t full[4], empty[4], done;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_sh;
    constexpr int APC = KC / NP;                    // atoms per K-chunk
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int brick = blockIdx.x;
    const int bx = brick % G.nbx, by = (brick / G.nbx) % G.nby, bz = brick / (G.nbx * G.nby);
    const int a0 = G.bstart[brick], na = G.bstart[brick + 1] - a0;
    if (na == 0) return;
    const int nchunks = (na + APC - 1) / APC;
    const int ncols = G.ld2;
    const int nq4 = ncols / 4;
    const uint32_t b_part = (uint32_t)ncols * KC * 2;
    const uint32_t stage_bytes = 3 * A_PART + 3 * b_part;
    const SAtoms<NP> S = stage_atoms<NP>(G, smem + (size_t)stages * stage_bytes, a0, na);

    if (warp == 0) tmem_alloc(&tmem_base, tmem_cols(ncols));
    if (tid == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(&full[s], NT);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&done, 1);
        abort_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;

    for (int c = 0; c < nchunks; ++c) {
        const int st = c % stages;
        unsigned char* sa = smem + (size_t)st * stage_bytes;
        unsigned char* sb = sa + 3 * A_PART;
        if (c >= stages && !mbar_wait_bounded(&empty[st], (uint32_t)((c / stages - 1) & 1))) {
            abort_sh = 1;
            break;
        }
        // B loads first: P rows of the chunk's atoms, item = (K-octet j, column
        // quad nq) with nq fastest across the threads (coalesced rows); the
        // A generation below covers their latency
        float4 braw[BMAX][8];
#pragma unroll
        for (int u = 0; u < BMAX; ++u) {
            const int it = tid + u * NT;
            const int nq = it % nq4, j = it / nq4;
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int r = j * 8 + e, la = c * APC + r / NP;
                braw[u][e] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (j < KC / 8 && la < na)
                    braw[u][e] = __ldg(reinterpret_cast<const float4*>(P + ((size_t)S.id[la] * NP + r % NP) * ncols) + nq);
            }
        }
        // A: B[p][r] for the 128 points x the chunk's 32 rows; one unit = one
        // point x 8 rows (8 / NP atoms); points fastest across the threads
#pragma unroll 2
        for (int it = tid; it < BP * (KC / 8); it += NT) {
            const int p = it % BP, j = it / BP;
            float v[8];
            int x, y, z;
            const bool inside = brick_point(G, bx, by, bz, p, x, y, z);
#pragma unroll
            for (int u = 0; u < 8 / NP; ++u) {
                const int la = c * APC + j * (8 / NP) + u;
                float b[NP];
                const bool m = inside && la < na && mask_bit(S.mask[la], p);
                if (m) beta_at<NP>(G, S, la, x, y, z, b);
#pragma unroll
                for (int i = 0; i < NP; ++i) v[u * NP + i] = m ? b[i] : 0.f;
            }
            store_unit(sa, A_PART, unit_off(p, j), v);
        }
        // B: (D o P)[r][n] split into bf16 parts
#pragma unroll
        for (int u = 0; u < BMAX; ++u) {
            const int it = tid + u * NT;
            const int nq = it % nq4, j = it / nq4;
            if (j < KC / 8) {
                float dd[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const int r = j * 8 + e, la = c * APC + r / NP;
                    dd[e] = la < na ? S.D[la * NP + r % NP] : 0.f;
                }
                store_b_item(sb, b_part, j, nq, braw[u], dd);
            }
        }
        fence_async_smem();
        mbar_arrive(&full[st]);
        if (tid == 0) {
            if (!mbar_wait_bounded(&full[st], (uint32_t)((c / stages) & 1))) {
                abort_sh = 1;
                break;
            }
            tc_fence_after();
            issue_chunk(tmem, smem_u32(sa), smem_u32(sb), b_part, ncols, c == 0);
            mma_commit(&empty[st]);
        }
    }
    if (tid == 0) mma_commit(&done);                // fires when every MMA issued above has completed
    const bool ok = mbar_wait_bounded(&done, 0);
    tc_fence_after();
    if (!ok) abort_sh = 1;
    __syncthreads();
    if (abort_sh) {
        if (tid == 0) atomicExch(err, 1);
    } else {
        // epilogue in two passes through shared memory (the ring is free now):
        // warp w copies TMEM lanes 32 (w % 4) .. +31 (points), one half of the
        // columns, into a [point][column] array; then all threads add gamma D
        // to out row by row with coalesced 16-byte accesses
        const int ldd = ncols + 4;                  // padded row (floats) against bank conflicts
        float* sD = reinterpret_cast<float*>(smem);
        {
            const int p = (warp & 3) * 32 + lane;
            const int half = ((ncols / 2 + 31) / 32) * 32;
            const int c0 = (warp >> 2) ? half : 0, c1 = (warp >> 2) ? ncols : min(half, ncols);
            for (int cb = c0; cb < c1; cb += 32) {
                float v[32];
                tmem_ld32(tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)cb, v);
                const int nw = min(32, c1 - cb);
#pragma unroll
                for (int q = 0; q < 32; q += 4)
                    if (q < nw)
                        *reinterpret_cast<float4*>(sD + p * ldd + cb + q) = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
            }
        }
        __syncthreads();
        const int total = BP * nq4;
        for (int it0 = tid; it0 < total; it0 += 4 * NT) {
            float4 o[4];
            float4* dst[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int it = it0 + u * NT;
                dst[u] = nullptr;
                if (it < total) {
                    const int p = it / nq4, nq = it % nq4;
                    int x, y, z;
                    if (brick_point(G, bx, by, bz, p, x, y, z)) {
                        dst[u] = reinterpret_cast<float4*>(
                                     out + ((size_t)x + (size_t)G.nx * ((size_t)y + (size_t)G.ny * z)) * ncols) + nq;
                        o[u] = *dst[u];
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (!dst[u]) continue;
                const int it = it0 + u * NT, p = it / nq4, nq = it % nq4;
                const float4 dv = *reinterpret_cast<const float4*>(sD + p * ldd + 4 * nq);
                o[u].x += gre * dv.x - gim * dv.y;
                o[u].y += gre * dv.y + gim * dv.x;
                o[u].z += gre * dv.z - gim * dv.w;
                o[u].w += gre * dv.w + gim * dv.z;
                *dst[u] = o[u];
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, tmem_cols(ncols));
    }
}

// ---------------------------------------------------------------------------
// projection: P[r] += dV sum_p B[p][r] w[p]   (one CTA per brick; the rows of
// the brick's atoms in M-tiles of 128, each accumulated over the 128 points
// in four K-chunks and drained with vector atomics)
// ---------------------------------------------------------------------------
template <int NP>
__global__ void __launch_bounds__(NT, 1)
    k_nl_project_tc(TcGeo G, const float* __restrict__ w, float* __restrict__ P, float dV, int stages,
                    int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    __shared__ __align__(8) uint64_t full[4], empty[4], done;
    __shared__ __align__(8) uint64_t fin;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_sh;
    constexpr int APT = 128 / NP;                   // atoms per M-tile
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int brick = blockIdx.x;
    const int bx = brick % G.nbx, by = (brick / G.nbx) % G.nby, bz = brick / (G.nbx * G.nby);
    const int a0 = G.bstart[brick], na = G.bstart[brick + 1] - a0;
    if (na == 0) return;
    const int ntiles = (na + APT - 1) / APT;
    const int ncols = G.ld2;
    const int nq4 = ncols / 4;
    const uint32_t b_part = (uint32_t)ncols * KC * 2;
    const uint32_t stage_bytes = 3 * A_PART + 3 * b_part;
    const SAtoms<NP> S = stage_atoms<NP>(G, smem + (size_t)stages * stage_bytes, a0, na);

    if (warp == 0) tmem_alloc(&tmem_base, tmem_cols(ncols));
    if (tid == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(&full[s], NT);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&done, 1);
        mbar_init(&fin, 1);
        abort_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;

    for (int t = 0; t < ntiles; ++t) {
        for (int kc = 0; kc < BP / KC; ++kc) {
            const int c = t * (BP / KC) + kc;
            const int st = c % stages;
            unsigned char* sa = smem + (size_t)st * stage_bytes;
            unsigned char* sb = sa + 3 * A_PART;
            bool ok_e = true;
            if (c >= stages) ok_e = mbar_wait_bounded(&empty[st], (uint32_t)((c / stages - 1) & 1));
            if (!ok_e) abort_sh = 1;
            if (ok_e) {
                // B loads first: w on one brick x-row of 8 points (= K-octet j:
                // plane kc, row j of the brick) x 4 columns, columns fastest
                float4 braw[BMAX][8];
#pragma unroll
                for (int u = 0; u < BMAX; ++u) {
                    const int it = tid + u * NT;
                    const int nq = it % nq4, j = it / nq4;
                    int x, y, z;
                    const bool row_in = j < KC / 8 && brick_point(G, bx, by, bz, kc * KC + j * 8, x, y, z);
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        braw[u][e] = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (row_in && x + e < G.nx)
                            braw[u][e] = __ldg(reinterpret_cast<const float4*>(
                                                   w + ((size_t)(x + e) + (size_t)G.nx * ((size_t)y + (size_t)G.ny * z)) *
                                                           ncols) + nq);
                    }
                }
                // A: B^T[r][p] for the tile's 128 rows x the chunk's 32 points;
                // one unit = one row (atom, projector) x one brick x-row of 8
                // points; rows fastest across the threads
#pragma unroll 2
                for (int it = tid; it < 128 * (KC / 8); it += NT) {
                    const int r = it % 128, j = it / 128;
                    const int la = t * APT + r / NP, i = r % NP;
                    const uint4 mk = la < na ? S.mask[la] : make_uint4(0, 0, 0, 0);
                    float v[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const int p = kc * KC + j * 8 + e;
                        int x, y, z;
                        const bool inside = brick_point(G, bx, by, bz, p, x, y, z);
                        const bool m = inside && mask_bit(mk, p);
                        v[e] = m ? beta_one<NP>(G, S, la, i, x, y, z) : 0.f;
                    }
                    store_unit(sa, A_PART, unit_off(r, j), v);
                }
                // B: w^T[n][p] split into bf16 parts
                const float one[8] = {1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f};
#pragma unroll
                for (int u = 0; u < BMAX; ++u) {
                    const int it = tid + u * NT;
                    const int nq = it % nq4, j = it / nq4;
                    if (j < KC / 8) store_b_item(sb, b_part, j, nq, braw[u], one);
                }
            }
            fence_async_smem();
            mbar_arrive(&full[st]);         // always, so that the issuing thread's wait ends
            if (tid == 0) {
                if (!abort_sh && mbar_wait_bounded(&full[st], (uint32_t)((c / stages) & 1))) {
                    tc_fence_after();
                    issue_chunk(tmem, smem_u32(sa), smem_u32(sb), b_part, ncols, kc == 0);
                    mma_commit(&empty[st]);
                } else {
                    abort_sh = 1;
                }
                if (kc == BP / KC - 1) mma_commit(&done);   // one phase of `done` per tile
            }
        }
        // drain the tile: lane = row (warp % 4), half of the columns per warp group
        const bool ok = mbar_wait_bounded(&done, (uint32_t)(t & 1));
        tc_fence_after();
        if (!ok) abort_sh = 1;
        __syncthreads();
        if (abort_sh) break;                // the same decision in every thread
        const int r = (warp & 3) * 32 + lane;
        const int la = t * APT + r / NP;
        const int half = ((ncols / 2 + 31) / 32) * 32;
        const int c0 = (warp >> 2) ? half : 0, c1 = (warp >> 2) ? ncols : min(half, ncols);
        float* dst = la < na ? P + ((size_t)S.id[la] * NP + r % NP) * ncols : nullptr;
        for (int cb = c0; cb < c1; cb += 32) {
            float v[32];
            tmem_ld32(tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)cb, v);
            if (dst) {
                const int nw = min(32, c1 - cb);
#pragma unroll
                for (int q = 0; q < 32; q += 4)
                    if (q < nw)
                        atomicAdd(reinterpret_cast<float4*>(dst + cb + q),
                                  make_float4(dV * v[q], dV * v[q + 1], dV * v[q + 2], dV * v[q + 3]));
            }
        }
        tc_fence_before();
        __syncthreads();                    // TMEM read before the next tile's MMAs overwrite it
        tc_fence_after();
    }
    // every MMA this CTA issued has completed before its tensor memory is freed
    if (tid == 0) {
        mma_commit(&fin);
        if (!mbar_wait_bounded(&fin, 0)) abort_sh = 1;
        if (abort_sh) atomicExch(err, 1);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, tmem_cols(ncols));
    }
}

// row[1] += sum_{a,i,n} f_n D_ai |P_ai,n|^2: the nonlocal energy
// <psi|v_nl|psi> from the projections of psi (one block, fixed order, FP64).
__global__ void __launch_bounds__(512) k_nl_energy(const float* __restrict__ P, const double* __restrict__ f,
                                                   const float* __restrict__ D, int64_t n_rows, int ld,
                                                   double* __restrict__ row) {
    double s = 0.0;
    const int64_t n = n_rows * ld;
    for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
        const int64_t r = e / ld;
        const int o = (int)(e - r * ld);
        const float2 v = reinterpret_cast<const float2*>(P)[e];
        s += f[o] * (double)D[r] * ((double)v.x * v.x + (double)v.y * v.y);
    }
    __shared__ double sh[16];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        row[1] += t;
    }
}

// Minimum-image displacement along one axis as the list builder computes it
// (FP64; the host copy of the formula, for the normalisation constants).
double host_min_image(int c, double h, double p, double L) {
    const double t = (double)c * h - p;
    return t - L * std::floor(t / L + 0.5);
}

// -log2(e) / (2 w^2) and 1 / w of the two projector widths r_c, r_c / sqrt(2)
void widths(double r_c, float (&cexp)[2], float (&invrc)[2]) {
    for (int s = 0; s < 2; ++s) {
        const double rc = s == 0 ? r_c : r_c / std::sqrt(2.0);
        cexp[s] = (float)(-1.0 / (2.0 * rc * rc) / std::log(2.0));
        invrc[s] = (float)(1.0 / rc);
    }
}

// Ring stages that fit beside the staged atom data in 225 KB of shared memory.
size_t stage_bytes_for(int ld2) { return 3 * (size_t)A_PART + 3 * (size_t)ld2 * KC * 2; }
size_t atom_bytes_for(int max_atoms, int np) { return (size_t)max_atoms * (16 + 16 + 8 * np + 4) + 64; }
int stages_for(int ld2, int max_atoms, int np) {
    const size_t atoms = atom_bytes_for(max_atoms, np);
    if (atoms >= 225 * 1024) return 0;
    return (int)std::min<size_t>(4, (225 * 1024 - atoms) / stage_bytes_for(ld2));
}
// The ring and the staged atoms; the scatter's epilogue reuses the same space
// for its [128][ld2 + 4] FP32 copy of the accumulator.
size_t smem_for(int ld2, int max_atoms, int np) {
    const size_t used = (size_t)stages_for(ld2, max_atoms, np) * stage_bytes_for(ld2) + atom_bytes_for(max_atoms, np);
    return std::max(used, (size_t)128 * (ld2 + 4) * sizeof(float)) + 1024;
}

TcGeo geo_for(const Domain& d) {
    const NlTc& t = *d.nltc;
    TcGeo G;
    G.nx = d.desc.n[0]; G.ny = d.desc.n[1]; G.nz = d.desc.n[2];
    G.nbx = t.nbx; G.nby = t.nby;
    G.ld2 = 2 * d.ld;
    G.h = (float)d.desc.h;
    for (int ax = 0; ax < 3; ++ax) {
        const double L = (double)d.desc.n[ax] * d.desc.h;
        G.L[ax] = (float)L;
        G.invL[ax] = (float)(1.0 / L);
    }
    widths(d.nl_rc, G.cexp, G.invrc);
    G.bstart = t.bstart; G.batom = t.batom; G.bmask = t.bmask;
    G.apos = t.apos; G.anrm = t.anrm; G.aD = t.aD;
    return G;
}

}  // namespace

// The tensor-core path serves complex64 domains whose projector spheres
// cover every grid point many times over (MLMD_NL_TC=1 forces it, =0 turns
// it off): below about eight list entries per grid point the fused scatter
// of the stage kernels is cheaper than 128-point dense tiles.
bool nl_tc_wanted(const Domain& d) {
    if (!d.c64() || !d.has_nl() || d.ld > 192) return false;
    if (const char* e = std::getenv("MLMD_NL_TC")) return e[0] == '1';
    return (double)d.nl.n_list >= 8.0 * (double)d.ng;
}

void nl_tc_release(Domain& d) {
    if (!d.nltc) return;
    NlTc& t = *d.nltc;
    for (void* p : {(void*)t.bstart, (void*)t.batom, (void*)t.bmask, (void*)t.apos, (void*)t.anrm, (void*)t.aD})
        if (p) d.mem.put(p);
    delete d.nltc;
    d.nltc = nullptr;
}

// Brick tables from the exact neighbour lists (set-up, on the host): per
// brick the atoms touching it (ascending) and each one's 128-bit membership
// set; per atom its position, the normalisation of its projectors (the FP64
// sum over its list, as the list builder normalises) and D.
void nl_tc_build(Domain& d, const double* pos_host, double r_c, const double* D_host) {
    nl_tc_release(d);
    if (!nl_tc_wanted(d)) return;
    const Nonlocal& nl = d.nl;
    const int np = nl.n_proj, na = nl.n_atoms;
    const int nx = d.desc.n[0], ny = d.desc.n[1], nz = d.desc.n[2];
    const double h = d.desc.h, dV = h * h * h;
    d.nl_rc = r_c;
    NlTc* t = new NlTc();
    d.nltc = t;
    t->nbx = (nx + BX - 1) / BX;
    t->nby = (ny + BY - 1) / BY;
    t->nbz = (nz + BZ - 1) / BZ;
    t->nbricks = t->nbx * t->nby * t->nbz;
    std::vector<int32_t> idx(nl.n_list);
    MLMD_CUDA(cudaMemcpyAsync(idx.data(), nl.idx, sizeof(int32_t) * nl.n_list, cudaMemcpyDeviceToHost, d.stream));
    MLMD_CUDA(cudaStreamSynchronize(d.stream));
    std::vector<std::vector<std::pair<int32_t, uint4>>> per(t->nbricks);
    std::vector<float> nrm((size_t)na * np), Df((size_t)na * np);
    std::vector<float4> pos(na);
    const double L[3] = {nx * h, ny * h, nz * h};
    for (int a = 0; a < na; ++a) {
        double s2[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        const double* pa = pos_host + 3 * a;
        for (int64_t q = nl.h_off[a]; q < nl.h_off[a + 1]; ++q) {
            const int g = idx[q];
            const int x = g % nx, y = (g / nx) % ny, z = g / (nx * ny);
            const int b = x / BX + t->nbx * (y / BY + t->nby * (z / BZ));
            const int p = (x % BX) + BX * ((y % BY) + BY * (z % BZ));
            auto& v = per[b];
            if (v.empty() || v.back().first != a) v.push_back({a, make_uint4(0, 0, 0, 0)});
            uint32_t* m = reinterpret_cast<uint32_t*>(&v.back().second);
            m[p >> 5] |= 1u << (p & 31);
            const double dl[3] = {host_min_image(x, h, pa[0], L[0]), host_min_image(y, h, pa[1], L[1]),
                                  host_min_image(z, h, pa[2], L[2])};
            const double d2 = dl[0] * dl[0] + dl[1] * dl[1] + dl[2] * dl[2];
            for (int set = 0; set < np / 4; ++set) {
                const double rc = set == 0 ? r_c : r_c / std::sqrt(2.0);
                const double e = std::exp(-d2 / (2.0 * rc * rc));
                s2[4 * set] += e * e;
                for (int ax = 0; ax < 3; ++ax) s2[4 * set + 1 + ax] += (dl[ax] / rc * e) * (dl[ax] / rc * e);
            }
        }
        for (int i = 0; i < np; ++i) {
            const double s = dV * s2[i];
            nrm[(size_t)a * np + i] = (float)(s > 0.0 ? 1.0 / std::sqrt(s) : 0.0);
            Df[(size_t)a * np + i] = (float)D_host[(size_t)a * np + i];
        }
        pos[a] = make_float4((float)pa[0], (float)pa[1], (float)pa[2], 0.f);
    }
    std::vector<int32_t> bstart(t->nbricks + 1, 0), batom;
    std::vector<uint4> bmask;
    for (int b = 0; b < t->nbricks; ++b) {
        bstart[b + 1] = bstart[b] + (int32_t)per[b].size();
        t->max_atoms = std::max<int>(t->max_atoms, (int)per[b].size());
        for (const auto& e : per[b]) {
            batom.push_back(e.first);
            bmask.push_back(e.second);
        }
    }
    auto upload = [&](const void* src, size_t bytes) {
        void* p = d.mem.get(std::max<size_t>(bytes, 16));
        if (bytes) MLMD_CUDA(cudaMemcpyAsync(p, src, bytes, cudaMemcpyHostToDevice, d.stream));
        return p;
    };
    t->bstart = (int32_t*)upload(bstart.data(), sizeof(int32_t) * bstart.size());
    t->batom = (int32_t*)upload(batom.data(), sizeof(int32_t) * batom.size());
    t->bmask = (uint4*)upload(bmask.data(), sizeof(uint4) * bmask.size());
    t->apos = (float4*)upload(pos.data(), sizeof(float4) * pos.size());
    t->anrm = (float*)upload(nrm.data(), sizeof(float) * nrm.size());
    t->aD = (float*)upload(Df.data(), sizeof(float) * Df.size());
    MLMD_CUDA(cudaStreamSynchronize(d.stream));
    if (stages_for(2 * d.ld, t->max_atoms, np) < 2) {   // too many atoms on one brick for the ring: SIMT path
        nl_tc_release(d);
        return;
    }
    // raise the kernels' shared-memory limit now, outside any stream capture
    const size_t smem = smem_for(2 * d.ld, t->max_atoms, np);
    ensure_dynamic_smem(reinterpret_cast<const void*>(np == 4 ? k_nl_scatter_tc<4> : k_nl_scatter_tc<8>), smem);
    ensure_dynamic_smem(reinterpret_cast<const void*>(np == 4 ? k_nl_project_tc<4> : k_nl_project_tc<8>), smem);
}

void launch_nl_energy(Domain& d, const void* P, double* row) {
    k_nl_energy<<<1, 512, 0, d.stream>>>((const float*)P, d.f, d.nltc->aD, (int64_t)d.nl.n_atoms * d.nl.n_proj, d.ld,
                                         row);
    d.launches++;
    MLMD_CUDA(cudaGetLastError());
}

// out += gamma sum_r B (D o P): the nonlocal half of a stage, on top of the
// local part the stage kernel wrote to out.
void launch_nl_scatter_tc(Domain& d, const void* P, void* out, double gre, double gim) {
    const TcGeo G = geo_for(d);
    const int stages = stages_for(G.ld2, d.nltc->max_atoms, d.nl.n_proj);
    const size_t smem = smem_for(G.ld2, d.nltc->max_atoms, d.nl.n_proj);
    ProfScope ps(d.prof, MLMD_KERNEL_SCATTER, d.stream);
    if (d.nl.n_proj == 4) {
        ensure_dynamic_smem(reinterpret_cast<const void*>(k_nl_scatter_tc<4>), smem);
        k_nl_scatter_tc<4><<<d.nltc->nbricks, NT, smem, d.stream>>>(G, (const float*)P, (float*)out, (float)gre,
                                                                    (float)gim, stages, d.err_flag);
    } else {
        ensure_dynamic_smem(reinterpret_cast<const void*>(k_nl_scatter_tc<8>), smem);
        k_nl_scatter_tc<8><<<d.nltc->nbricks, NT, smem, d.stream>>>(G, (const float*)P, (float*)out, (float)gre,
                                                                    (float)gim, stages, d.err_flag);
    }
    d.launches++;
    MLMD_CUDA(cudaGetLastError());
}

// P = dV B^T w (P is zeroed here first, then accumulated by atomics).
void launch_nl_project_tc(Domain& d, const void* w, void* P) {
    const TcGeo G = geo_for(d);
    const int stages = stages_for(G.ld2, d.nltc->max_atoms, d.nl.n_proj);
    const size_t smem = smem_for(G.ld2, d.nltc->max_atoms, d.nl.n_proj);
    MLMD_CUDA(cudaMemsetAsync(P, 0, (size_t)d.nl.n_atoms * d.nl.n_proj * G.ld2 * sizeof(float), d.stream));
    const float dV = (float)(d.desc.h * d.desc.h * d.desc.h);
    ProfScope ps(d.prof, MLMD_KERNEL_PROJECT, d.stream);
    if (d.nl.n_proj == 4) {
        ensure_dynamic_smem(reinterpret_cast<const void*>(k_nl_project_tc<4>), smem);
        k_nl_project_tc<4><<<d.nltc->nbricks, NT, smem, d.stream>>>(G, (const float*)w, (float*)P, dV, stages,
                                                                    d.err_flag);
    } else {
        ensure_dynamic_smem(reinterpret_cast<const void*>(k_nl_project_tc<8>), smem);
        k_nl_project_tc<8><<<d.nltc->nbricks, NT, smem, d.stream>>>(G, (const float*)w, (float*)P, dV, stages,
                                                                    d.err_flag);
    }
    d.launches++;
    MLMD_CUDA(cudaGetLastError());
}

}  // namespace mlmd
