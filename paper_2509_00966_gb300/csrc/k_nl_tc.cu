// Nonlocal term of Eq. 3 on the tcgen05 tensor cores, for domains where
// many projector spheres overlap every grid point (Sec. V.B.5: projection
// and scatter-back as GEMMs; Sec. V.B.7: BF16 split products).
//
// The grid is cut into bricks of 8 x 4 x 4 = 128 points.  For one brick the
// atoms whose spheres touch it give the projector rows, and the two halves
// of the nonlocal term are dense GEMMs over the brick:
//
//   scatter     out[p][n] += gamma sum_r B[p][r] (D o P)[r][n]     (M = points, K = rows,   N = orbital reals)
//   projection  P[r][n]   += dV    sum_p B[p][r] w[p][n]           (M = rows,   K = points, N = orbital reals)
//
// with B[p][r] = beta_r(p) if p lies in the sphere of r's atom, else 0.
// Complex orbitals enter as interleaved (re, im) real columns (B is real).
// B is not stored: the producer threads evaluate the projector values of
// the brick's atoms in FP32 (min-image displacement, Gaussian, normalisation
// from the FP64 lists) and mask them with a per-(brick, atom) 128-bit
// membership set taken from the exact FP64 neighbour lists, so sphere
// membership is the lists' own.
//
// Every FP32 operand x is split exactly into three bf16 parts by truncation
// (x0 = the top 8 significand bits of x, x1 those of x - x0, x2 = x - x0 -
// x1, which has at most 8 significant bits), and the six products x_i y_j
// with i + j <= 2 are accumulated in FP32 in tensor memory, smallest first.
// The operands that do not depend on the brick's geometry are split once per
// stage, not once per CTA: D o P (small) by k_nl_split_P into one 16-byte
// slab per (atom, column) -- the NP projector values, padded to 8 -- and the
// stage output w by the scatter's epilogue (or k_nl_split_w) into one 16-byte
// slab per (brick x-row of 8 points, column).  Both reach shared memory by
// bulk copies in a layout whose 8 x 16-byte core matrices are 8 consecutive
// columns of one K-octet ([K-octet][column][8 values]).
//
// Pipeline of one CTA (256 threads): thread 0 issues the bulk copies of a
// K-chunk into a ring stage; every thread generates its share of the
// projector tile into the same stage, fences the writes into the async proxy
// and arrives on the stage's `full` barrier; thread 0 waits for `full`,
// issues the MMAs of the chunk and commits them to the stage's `empty`
// barrier, which guards the next refill.  Every wait is bounded (~2 s); on
// expiry the CTA raises the domain's error word, waits (bounded) for its
// copies and MMAs and frees its tensor memory.
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
    uint16_t* P3a = nullptr;      // split D o P of the projections in Pa: [3][n_atoms][2 ld][8] bf16
    uint16_t* P3b = nullptr;      // the same for Pb
    uint16_t* w3 = nullptr;       // split stage output: [3][nbricks][16][2 ld][8] bf16
    // projector tiles built once per projector set (null: generated in every
    // launch): one image of three bf16 parts per K-chunk, scatter chunks of
    // brick b from soff[b], projection chunks (M-tile, plane) from poff[b]
    unsigned char* As = nullptr;
    unsigned char* Ap = nullptr;
    int64_t* soff = nullptr;
    int64_t* poff = nullptr;
};

namespace {

using namespace tc;

constexpr int BX = 8, BY = 4, BZ = 4, BP = BX * BY * BZ;   // brick of 128 points
constexpr int KC = 32;                                      // K elements per ring stage (4 K-octets)
constexpr uint32_t A_PART = 128 * KC * 2;                   // one 16-bit part of a 128-row A tile
constexpr int NT = 256;                                     // generator threads per CTA
constexpr uint32_t IMG = 3 * A_PART;                        // one K-chunk of A: its three bf16 parts

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
    const unsigned char* As;      // projector tile images or null (NlTc)
    const unsigned char* Ap;
    const int64_t* soff;
    const int64_t* poff;
};

// A tiles (128 rows x K = 32): byte offset of the 16-byte unit (row, K-octet
// j); core matrices of 8 rows x 16 bytes, the four K-cores of a row group
// adjacent (LBO = 128 B), row groups 512 B apart (SBO).
__device__ __forceinline__ uint32_t unit_off(int row, int j) { return (uint32_t)((row >> 3) * 512 + j * 128 + (row & 7) * 16); }

// B tiles (ncols rows x K = 32) are [K-octet j][column n][16 bytes]: the core
// matrix of columns 8g .. 8g+7 is 128 contiguous bytes (SBO = 128 B), and
// the K-octets are ncols x 16 bytes apart (LBO).

// tcgen05.mma kind::f16 instruction descriptor: FP32 accumulator, BF16 A and
// B, K-major, M = 128, N given (a multiple of 16, at most 256).
__device__ __forceinline__ uint32_t idesc_n(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

// Exact split of two FP32 values into three bf16 parts each (truncation: the
// top 16 bits of x, then of the remainders), packed pairwise into 32-bit
// words (part of x0 in the low half).
__device__ __forceinline__ void split2(float x0, float x1, uint32_t& h, uint32_t& m, uint32_t& l) {
    const uint32_t u0 = __float_as_uint(x0), u1 = __float_as_uint(x1);
    h = __byte_perm(u0, u1, 0x7632);
    const float r0 = x0 - __uint_as_float(u0 & 0xffff0000u), r1 = x1 - __uint_as_float(u1 & 0xffff0000u);
    const uint32_t v0 = __float_as_uint(r0), v1 = __float_as_uint(r1);
    m = __byte_perm(v0, v1, 0x7632);
    const float s0 = r0 - __uint_as_float(v0 & 0xffff0000u), s1 = r1 - __uint_as_float(v1 & 0xffff0000u);
    l = __byte_perm(__float_as_uint(s0), __float_as_uint(s1), 0x7632);
}

// Eight FP32 values -> one 16-byte unit per bf16 part.
__device__ __forceinline__ void split8(const float (&v)[8], uint4 (&q)[3]) {
    split2(v[0], v[1], q[0].x, q[1].x, q[2].x);
    split2(v[2], v[3], q[0].y, q[1].y, q[2].y);
    split2(v[4], v[5], q[0].z, q[1].z, q[2].z);
    split2(v[6], v[7], q[0].w, q[1].w, q[2].w);
}
__device__ __forceinline__ void store_unit(unsigned char* base, uint32_t part_bytes, uint32_t off, const float (&v)[8]) {
    uint4 q[3];
    split8(v, q);
#pragma unroll
    for (int s = 0; s < 3; ++s) *reinterpret_cast<uint4*>(base + (size_t)s * part_bytes + off) = q[s];
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
// membership set and projector normalisation of each of the brick's atoms,
// and its global index.
template <int NP> struct SAtoms {
    float4* pos;
    uint4* mask;
    float* nrm;                   // [na][NP]
    int* id;
};

template <int NP>
__device__ __forceinline__ SAtoms<NP> stage_atoms(const TcGeo& G, unsigned char* base, int a0, int na) {
    SAtoms<NP> S;
    S.pos = reinterpret_cast<float4*>(base);
    S.mask = reinterpret_cast<uint4*>(S.pos + na);
    S.nrm = reinterpret_cast<float*>(S.mask + na);
    S.id = reinterpret_cast<int*>(S.nrm + (size_t)na * NP);
    for (int k = threadIdx.x; k < na; k += blockDim.x) {
        const int a = G.batom[a0 + k];
        S.id[k] = a;
        S.pos[k] = G.apos[a];
        S.mask[k] = G.bmask[a0 + k];
#pragma unroll
        for (int i = 0; i < NP; ++i) S.nrm[k * NP + i] = G.anrm[(size_t)a * NP + i];
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

__device__ __forceinline__ bool mask_bit(const uint4& m, int p) {
    const uint32_t w = p < 32 ? m.x : p < 64 ? m.y : p < 96 ? m.z : m.w;
    return (w >> (p & 31)) & 1u;
}

// Issue the MMAs of one ring stage: two K = 16 steps, six split products
// (smallest first), the N columns in one or two instructions.
__device__ __forceinline__ void issue_chunk(uint32_t tmem, uint32_t a_base, uint32_t b_base, uint32_t b_part, int ncols,
                                            bool first) {
    const int n0 = ncols <= 256 ? ncols : ((ncols / 2 + 15) / 16) * 16;
    const uint32_t lbo_b = (uint32_t)ncols * 16;
#pragma unroll
    for (int kk = 0; kk < 2; ++kk)
#pragma unroll
        for (int p = 0; p < 6; ++p) {
            const uint64_t ad = smem_desc(a_base + prod_a(p, 6) * A_PART + kk * 256, 128, 512);
            const uint32_t acc = (first && kk == 0 && p == 0) ? 0u : 1u;
            const uint32_t bp = b_base + prod_b(p, 6) * b_part + kk * 2 * lbo_b;
            mma_f16(tmem, ad, smem_desc(bp, lbo_b, 128), idesc_n(n0), acc);
            if (ncols > n0)
                mma_f16(tmem + (uint32_t)n0, ad, smem_desc(bp + (uint32_t)n0 * 16, lbo_b, 128), idesc_n(ncols - n0), acc);
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

// Offsets (bf16 elements) of the split arrays' 16-byte slab rows.
__device__ __forceinline__ size_t p3_off(int part, int n_atoms, int atom, int ncols) {
    return (((size_t)part * n_atoms + atom) * ncols) * 8;
}
__device__ __forceinline__ size_t w3_off(int part, int nbricks, int brick, int xrow, int ncols) {
    return ((((size_t)part * nbricks + brick) * 16 + xrow) * ncols) * 8;
}

// Projector tile of scatter chunk c (the brick's 128 points x the chunk's 4
// atoms, one unit = one point x one atom's NP projectors padded to 8,
// points fastest) into the three-part image at `dst` (a ring stage in
// shared memory, or a device-memory image); threads tid, tid + nthr, ...
template <int NP>
__device__ __forceinline__ void gen_scatter_chunk(const TcGeo& G, const SAtoms<NP>& S, int bx, int by, int bz, int na,
                                                  int c, unsigned char* dst, int tid, int nthr) {
#pragma unroll 2
    for (int it = tid; it < BP * 4; it += nthr) {
        const int p = it % BP, j = it / BP;
        const int la = c * 4 + j;
        int x, y, z;
        const bool inside = brick_point(G, bx, by, bz, p, x, y, z);
        float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (inside && la < na && mask_bit(S.mask[la], p)) {
            float bv[NP];
            beta_at<NP>(G, S, la, x, y, z, bv);
#pragma unroll
            for (int i = 0; i < NP; ++i) v[i] = bv[i];
        }
        store_unit(dst, A_PART, unit_off(p, j), v);
    }
}

// Projector tile of projection chunk (M-tile t, brick z-plane kc): B^T for
// the tile's 128 rows x the plane's 32 points; one item = one atom x one
// x-row of 8 points (NP units).
template <int NP>
__device__ __forceinline__ void gen_project_chunk(const TcGeo& G, const SAtoms<NP>& S, int bx, int by, int bz, int na,
                                                  int t, int kc, unsigned char* dst, int tid, int nthr) {
    constexpr int APT = 128 / NP;
    for (int it = tid; it < APT * 4; it += nthr) {
        const int ra = it % APT, j = it / APT;
        const int la = t * APT + ra;
        float b[8][NP];
        const uint4 mk = la < na ? S.mask[la] : make_uint4(0, 0, 0, 0);
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int p = kc * KC + j * 8 + e;
            int x, y, z;
            const bool m = brick_point(G, bx, by, bz, p, x, y, z) && mask_bit(mk, p);
            if (m) {
                beta_at<NP>(G, S, la, x, y, z, b[e]);
            } else {
#pragma unroll
                for (int i = 0; i < NP; ++i) b[e][i] = 0.f;
            }
        }
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            float v[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) v[e] = b[e][i];
            store_unit(dst, A_PART, unit_off(ra * NP + i, j), v);
        }
    }
}

// The images of both kernels' projector tiles for one brick (one CTA per
// brick), built once per projector set: the same bytes the generators would
// write into a ring stage in every launch.
template <int NP>
__global__ void __launch_bounds__(NT) k_nl_tiles(TcGeo G, unsigned char* __restrict__ As, unsigned char* __restrict__ Ap) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int brick = blockIdx.x;
    const int bx = brick % G.nbx, by = (brick / G.nbx) % G.nby, bz = brick / (G.nbx * G.nby);
    const int a0 = G.bstart[brick], na = G.bstart[brick + 1] - a0;
    if (na == 0) return;
    const SAtoms<NP> S = stage_atoms<NP>(G, smem_raw, a0, na);
    __syncthreads();
    const int nchunks = (na + 3) / 4;
    for (int c = 0; c < nchunks; ++c)
        gen_scatter_chunk<NP>(G, S, bx, by, bz, na, c, As + ((size_t)G.soff[brick] + c) * IMG, threadIdx.x, NT);
    constexpr int APT = 128 / NP;
    const int ntiles = (na + APT - 1) / APT;
    for (int t = 0; t < ntiles; ++t)
        for (int kc = 0; kc < BP / KC; ++kc)
            gen_project_chunk<NP>(G, S, bx, by, bz, na, t, kc,
                                  Ap + ((size_t)G.poff[brick] + (size_t)t * (BP / KC) + kc) * IMG, threadIdx.x, NT);
}

// ---------------------------------------------------------------------------
// scatter: out[p] += gamma sum_r B[p][r] D_r P[r]   (one CTA per brick)
// K-octet j of chunk c is atom c*4 + j (its NP projectors, padded to 8).
// The epilogue also writes the split, transposed output of the brick (the
// projection's B operand).
// ---------------------------------------------------------------------------
template <int NP>
__global__ void __launch_bounds__(NT + 32, 1)
    k_nl_scatter_tc(TcGeo G, const uint16_t* __restrict__ P3, int n_atoms, float* __restrict__ out,
                    uint16_t* __restrict__ w3, int nbricks, float gre, float gim, int stages, int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    __shared__ __align__(8) uint64_t full[4], empty[4], done;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_sh;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int brick = blockIdx.x;
    const int bx = brick % G.nbx, by = (brick / G.nbx) % G.nby, bz = brick / (G.nbx * G.nby);
    const int a0 = G.bstart[brick], na = G.bstart[brick + 1] - a0;
    if (na == 0) return;                            // nothing to add; the projection skips the brick too
    const int ncols = G.ld2;
    const uint32_t b_part = (uint32_t)ncols * KC * 2;
    const uint32_t stage_bytes = 3 * A_PART + 3 * b_part;
    const uint32_t slab = (uint32_t)ncols * 16;     // one K-octet of one B part
    const int nchunks = (na + 3) / 4;
    const SAtoms<NP> S = stage_atoms<NP>(G, smem + (size_t)stages * stage_bytes, a0, na);

    if (warp == 0) tmem_alloc(&tmem_base, tmem_cols(ncols));
    if (tid == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(&full[s], G.As ? 1 : NT + 1);   // the issuer's expect_tx, plus every generator without images
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

    if (warp == NT / 32) {
        // issuer warp: lane 0 waits on the barriers and issues the MMAs; the
        // bulk copies of a chunk (the tile image and the 3 x 4 D o P slabs)
        // are spread over the lanes, up to `stages` chunks ahead
        int issued = 0, consumed = 0;               // chunks whose copies were issued / landed
        bool stop = false;
        for (int c = 0; c < nchunks && !stop; ++c) {
            for (; issued < nchunks && issued < c + stages; ++issued) {
                const int cc = issued, st = cc % stages;
                int ok = 1;
                if (lane == 0 && cc >= stages) ok = mbar_wait_bounded(&empty[st], (uint32_t)((cc / stages - 1) & 1));
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (!ok) {
                    stop = true;
                    break;
                }
                unsigned char* sa = smem + (size_t)st * stage_bytes;
                unsigned char* sb = sa + 3 * A_PART;
                const int nv = min(4, na - cc * 4);
                if (lane == 0) mbar_expect_tx(&full[st], (uint32_t)nv * 3 * slab + (G.As ? IMG : 0u));
                __syncwarp();
                if (lane < nv * 3) {
                    const int jj = lane / 3, s = lane % 3;
                    bulk_load(sb + (size_t)s * b_part + (size_t)jj * slab,
                              P3 + p3_off(s, n_atoms, S.id[cc * 4 + jj], ncols), slab, &full[st]);
                }
                if (G.As && lane == 31) bulk_load(sa, G.As + ((size_t)G.soff[brick] + cc) * IMG, IMG, &full[st]);
                if (G.As && nv < 4) {               // K-octets of missing atoms (last chunk) are zero in B
                    for (int e = lane; e < (4 - nv) * 3 * ncols; e += 32) {
                        const int s = e / ((4 - nv) * ncols), r = e % ((4 - nv) * ncols);
                        *reinterpret_cast<uint4*>(sb + (size_t)s * b_part + (size_t)(nv + r / ncols) * slab +
                                                  (size_t)(r % ncols) * 16) = make_uint4(0, 0, 0, 0);
                    }
                    fence_async_smem();
                }
                __syncwarp();
            }
            if (stop) break;
            const int st = c % stages;
            int ok = 1;
            if (lane == 0) {
                ok = mbar_wait_bounded(&full[st], (uint32_t)((c / stages) & 1));
                if (ok) {
                    consumed = c + 1;
                    tc_fence_after();
                    const uint32_t sa = smem_u32(smem + (size_t)st * stage_bytes);
                    issue_chunk(tmem, sa, sa + 3 * A_PART, b_part, ncols, c == 0);
                    mma_commit(&empty[st]);
                }
            }
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) stop = true;
        }
        if (lane == 0) {
            if (stop) abort_sh = 1;
            mma_commit(&done);                      // fires when every MMA issued above has completed
            for (int c = consumed; c < issued; ++c) // after an abort: copies still in flight land first
                (void)mbar_wait_bounded(&full[c % stages], (uint32_t)((c / stages) & 1));
        }
    } else if (tid < NT && !G.As) {
        // generators (warps 0-7): the projector tile of each chunk
        for (int c = 0; c < nchunks; ++c) {
            const int st = c % stages;
            unsigned char* sa = smem + (size_t)st * stage_bytes;
            unsigned char* sb = sa + 3 * A_PART;
            if (c >= stages && !mbar_wait_bounded(&empty[st], (uint32_t)((c / stages - 1) & 1))) {
                abort_sh = 1;
                break;
            }
            const int nv = min(4, na - c * 4);      // atoms of this chunk
            // K-octets of missing atoms (last chunk) are zero in B
            for (int e = tid; e < (4 - nv) * 3 * ncols; e += NT) {
                const int s = e / ((4 - nv) * ncols), r = e % ((4 - nv) * ncols);
                *reinterpret_cast<uint4*>(sb + (size_t)s * b_part + (size_t)(nv + r / ncols) * slab +
                                          (size_t)(r % ncols) * 16) = make_uint4(0, 0, 0, 0);
            }
            // A: the chunk's projector tile (copied by the issuer when prebuilt)
            if (!G.As) gen_scatter_chunk<NP>(G, S, bx, by, bz, na, c, sa, tid, NT);
            fence_async_smem();
            mbar_arrive(&full[st]);
        }
    }
    const bool ok = mbar_wait_bounded(&done, 0);
    tc_fence_after();
    if (!ok) abort_sh = 1;
    __syncthreads();
    if (abort_sh) {
        if (tid == 0) atomicExch(err, 1);
    } else {
        // epilogue (the ring is free now): warp w reads TMEM lanes 32 (w % 4) ..
        // +31 (one grid point per lane) over one half of the columns, adds
        // gamma D to the point's output row with eight 16-byte loads in flight
        // per lane, and keeps the new values in a [point][column] array for
        // the split, transposed copy that the projection reads
        const int ldd = ncols + 4;                  // padded row (floats) against bank conflicts
        float* sD = reinterpret_cast<float*>(smem);
        if (tid < NT) {
            const int p = (warp & 3) * 32 + lane;
            int x, y, z;
            const bool inside = brick_point(G, bx, by, bz, p, x, y, z);
            float* orow = inside ? out + ((size_t)x + (size_t)G.nx * ((size_t)y + (size_t)G.ny * z)) * ncols : nullptr;
            const int half = ((ncols / 2 + 31) / 32) * 32;
            const int c0 = (warp >> 2) ? half : 0, c1 = (warp >> 2) ? ncols : min(half, ncols);
            for (int cb = c0; cb < c1; cb += 32) {
                const int nw = min(32, c1 - cb);
                float v[32];
                if (nchunks > 0) {
                    tmem_ld32(tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)cb, v);
                } else {
#pragma unroll
                    for (int q = 0; q < 32; ++q) v[q] = 0.f;
                }
                float4 o[8];
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    o[q] = (orow && 4 * q < nw) ? *reinterpret_cast<const float4*>(orow + cb + 4 * q)
                                                : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    if (4 * q >= nw) continue;
                    const float* d4 = v + 4 * q;
                    o[q].x += gre * d4[0] - gim * d4[1];
                    o[q].y += gre * d4[1] + gim * d4[0];
                    o[q].z += gre * d4[2] - gim * d4[3];
                    o[q].w += gre * d4[3] + gim * d4[2];
                    if (orow) *reinterpret_cast<float4*>(orow + cb + 4 * q) = o[q];
                    *reinterpret_cast<float4*>(sD + p * ldd + cb + 4 * q) = o[q];   // zero outside the grid
                }
            }
        }
        __syncthreads();
        // split output: item = (x-row r, column n), columns fastest
        for (int it = tid; it < (tid < NT ? 16 * ncols : 0); it += NT) {
            const int r = it / ncols, n = it % ncols;
            float v[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) v[e] = sD[(r * 8 + e) * ldd + n];
            uint4 q[3];
            split8(v, q);
#pragma unroll
            for (int s = 0; s < 3; ++s)
                *reinterpret_cast<uint4*>(w3 + w3_off(s, nbricks, brick, r, ncols) + (size_t)n * 8) = q[s];
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
// in four K-chunks -- chunk kc is the brick's z-plane kc, K-octet j its
// x-row y = j -- and drained with vector atomics)
// ---------------------------------------------------------------------------
template <int NP>
__global__ void __launch_bounds__(NT + 32, 1)
    k_nl_project_tc(TcGeo G, const uint16_t* __restrict__ w3, int nbricks, float* __restrict__ P, float dV, int stages,
                    int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    __shared__ __align__(8) uint64_t full[4], empty[4], done[2], drained[2];
    __shared__ __align__(8) uint64_t fin;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_sh;
    constexpr int APT = 128 / NP;                   // atoms per M-tile
    constexpr int KCH = BP / KC;                    // K-chunks (z-planes) per tile
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int brick = blockIdx.x;
    const int bx = brick % G.nbx, by = (brick / G.nbx) % G.nby, bz = brick / (G.nbx * G.nby);
    const int a0 = G.bstart[brick], na = G.bstart[brick + 1] - a0;
    if (na == 0) return;
    const int ntiles = (na + APT - 1) / APT;
    const int nch = ntiles * KCH;
    const int ncols = G.ld2;
    const uint32_t b_part = (uint32_t)ncols * KC * 2;
    const uint32_t stage_bytes = 3 * A_PART + 3 * b_part;
    const SAtoms<NP> S = stage_atoms<NP>(G, smem + (size_t)stages * stage_bytes, a0, na);
    // two accumulators when they fit in tensor memory: tile t drains while
    // tile t+1 accumulates
    const uint32_t tcols = tmem_cols(ncols);
    const int nbuf = 2 * tcols <= 512 ? 2 : 1;

    if (warp == 0) tmem_alloc(&tmem_base, tcols * (uint32_t)nbuf);
    if (tid == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(&full[s], G.Ap ? 1 : NT + 1);   // the issuer's expect_tx, plus every generator without images
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&done[b], 1);
            mbar_init(&drained[b], NT / 32);        // one arrival per generator warp
        }
        mbar_init(&fin, 1);
        abort_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;

    if (tid == NT) {
        // issuer: copies of the split output (the same four x-row groups for
        // every tile) up to `stages` chunks ahead; the MMAs of a tile once
        // its accumulator has been drained
        int issued = 0, consumed = 0;
        for (int c = 0; c < nch && !abort_sh; ++c) {
            for (; issued < nch && issued < c + stages; ++issued) {
                const int cc = issued, st = cc % stages, kc = cc % KCH;
                if (cc >= stages && !mbar_wait_bounded(&empty[st], (uint32_t)((cc / stages - 1) & 1))) {
                    abort_sh = 1;
                    break;
                }
                unsigned char* sa = smem + (size_t)st * stage_bytes;
                unsigned char* sb = sa + 3 * A_PART;
                mbar_expect_tx(&full[st], 3 * b_part + (G.Ap ? IMG : 0u));
                if (G.Ap) bulk_load(sa, G.Ap + ((size_t)G.poff[brick] + cc) * IMG, IMG, &full[st]);
#pragma unroll
                for (int s = 0; s < 3; ++s)
                    bulk_load(sb + (size_t)s * b_part, w3 + w3_off(s, nbricks, brick, kc * 4, ncols), b_part, &full[st]);
            }
            if (abort_sh) break;
            const int t = c / KCH, kc = c % KCH, buf = t % nbuf, st = c % stages;
            if (kc == 0 && t >= nbuf &&
                !mbar_wait_bounded(&drained[buf], (uint32_t)((t / nbuf - 1) & 1))) {
                abort_sh = 1;
                break;
            }
            if (!mbar_wait_bounded(&full[st], (uint32_t)((c / stages) & 1))) {
                abort_sh = 1;
                break;
            }
            consumed = c + 1;
            tc_fence_after();
            const uint32_t sa = smem_u32(smem + (size_t)st * stage_bytes);
            issue_chunk(tmem + (uint32_t)buf * tcols, sa, sa + 3 * A_PART, b_part, ncols, kc == 0);
            mma_commit(&empty[st]);
            if (kc == KCH - 1) mma_commit(&done[buf]);
        }
        for (int c = consumed; c < issued; ++c)     // every copy lands before the memory is freed
            (void)mbar_wait_bounded(&full[c % stages], (uint32_t)((c / stages) & 1));
        mma_commit(&fin);
        if (!mbar_wait_bounded(&fin, 0)) abort_sh = 1;
    } else if (tid < NT) {
        // generators (warps 0-7): B^T tiles; after tile t, the drain of tile t-1
        const int r = (warp & 3) * 32 + lane;       // TMEM lane = row of the tile
        const int half = ((ncols / 2 + 31) / 32) * 32;
        const int c0 = (warp >> 2) ? half : 0, c1 = (warp >> 2) ? ncols : min(half, ncols);
        auto drain = [&](int t) {
            const int buf = t % nbuf;
            const bool ok = mbar_wait_bounded(&done[buf], (uint32_t)((t / nbuf) & 1));
            tc_fence_after();
            if (!ok) { abort_sh = 1; return false; }
            const int la = t * APT + r / NP;
            float* dst = la < na ? P + ((size_t)S.id[la] * NP + r % NP) * ncols : nullptr;
            for (int cb = c0; cb < c1; cb += 32) {
                float v[32];
                tmem_ld32(tmem + (uint32_t)buf * tcols + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)cb, v);
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
            __syncwarp();
            if (lane == 0) mbar_arrive(&drained[buf]);
            return true;
        };
        bool live = true;
        for (int t = 0; t < ntiles && live; ++t) {
            if (nbuf == 1 && t > 0) live = drain(t - 1);       // one accumulator: drain before refilling it
            for (int kc = 0; kc < KCH && live && !G.Ap; ++kc) {   // (with images the issuer fills the stages alone)
                const int c = t * KCH + kc;
                const int st = c % stages;
                unsigned char* sa = smem + (size_t)st * stage_bytes;
                if (c >= stages && !mbar_wait_bounded(&empty[st], (uint32_t)((c / stages - 1) & 1))) {
                    abort_sh = 1;
                    live = false;
                    break;
                }
                // A: the chunk's projector tile (copied by the issuer when prebuilt)
                if (!G.Ap) gen_project_chunk<NP>(G, S, bx, by, bz, na, t, kc, sa, tid, NT);
                fence_async_smem();
                mbar_arrive(&full[st]);
            }
            if (live && nbuf == 2 && t > 0) live = drain(t - 1);   // overlaps tile t's MMAs
        }
        if (live) drain(ntiles - 1);
    }
    tc_fence_before();
    __syncthreads();
    if (tid == 0 && abort_sh) atomicExch(err, 1);
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, tcols * (uint32_t)nbuf);
    }
}

// P3[s][a][n][0..7] = part s of D_ai P[a][i][n] for i < NP (zero for i >= NP)
template <int NP>
__global__ void __launch_bounds__(256) k_nl_split_P(const float* __restrict__ P, const float* __restrict__ D, int n_atoms,
                                                    int ncols, uint16_t* __restrict__ P3) {
    const int64_t total = (int64_t)n_atoms * ncols;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int a = (int)(e / ncols), n = (int)(e % ncols);
        float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int i = 0; i < NP; ++i) v[i] = D[(size_t)a * NP + i] * P[((size_t)a * NP + i) * ncols + n];
        uint4 q[3];
        split8(v, q);
#pragma unroll
        for (int s = 0; s < 3; ++s) *reinterpret_cast<uint4*>(P3 + p3_off(s, n_atoms, a, ncols) + (size_t)n * 8) = q[s];
    }
}

// w3 of a state that did not come out of the scatter kernel: one CTA per
// brick, item = (x-row r, column n), columns fastest; zero outside the grid.
__global__ void __launch_bounds__(256) k_nl_split_w(TcGeo G, const float* __restrict__ w, int nbricks,
                                                    uint16_t* __restrict__ w3) {
    const int brick = blockIdx.x, ncols = G.ld2;
    const int bx = brick % G.nbx, by = (brick / G.nbx) % G.nby, bz = brick / (G.nbx * G.nby);
    for (int it = threadIdx.x; it < 16 * ncols; it += blockDim.x) {
        const int r = it / ncols, n = it % ncols;
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            int x, y, z;
            v[e] = brick_point(G, bx, by, bz, r * 8 + e, x, y, z)
                       ? w[((size_t)x + (size_t)G.nx * ((size_t)y + (size_t)G.ny * z)) * ncols + n]
                       : 0.f;
        }
        uint4 q[3];
        split8(v, q);
#pragma unroll
        for (int s = 0; s < 3; ++s) *reinterpret_cast<uint4*>(w3 + w3_off(s, nbricks, brick, r, ncols) + (size_t)n * 8) = q[s];
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
size_t atom_bytes_for(int max_atoms, int np) { return (size_t)max_atoms * (16 + 16 + 4 * np + 4) + 64; }
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
    G.As = t.As; G.Ap = t.Ap; G.soff = t.soff; G.poff = t.poff;
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
    for (void* p : {(void*)t.bstart, (void*)t.batom, (void*)t.bmask, (void*)t.apos, (void*)t.anrm, (void*)t.aD,
                    (void*)t.P3a, (void*)t.P3b, (void*)t.w3, (void*)t.As, (void*)t.Ap, (void*)t.soff, (void*)t.poff})
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
    const size_t p3 = (size_t)3 * na * 2 * d.ld * 8 * sizeof(uint16_t);
    t->P3a = (uint16_t*)d.mem.get(p3);
    t->P3b = (uint16_t*)d.mem.get(p3);
    t->w3 = (uint16_t*)d.mem.get((size_t)3 * t->nbricks * 16 * 2 * d.ld * 8 * sizeof(uint16_t));
    MLMD_CUDA(cudaStreamSynchronize(d.stream));
    if (stages_for(2 * d.ld, t->max_atoms, np) < 2) {   // too many atoms on one brick for the ring: SIMT path
        nl_tc_release(d);
        return;
    }
    // raise the kernels' shared-memory limit now, outside any stream capture
    const size_t smem = smem_for(2 * d.ld, t->max_atoms, np);
    ensure_dynamic_smem(reinterpret_cast<const void*>(np == 4 ? k_nl_scatter_tc<4> : k_nl_scatter_tc<8>), smem);
    ensure_dynamic_smem(reinterpret_cast<const void*>(np == 4 ? k_nl_project_tc<4> : k_nl_project_tc<8>), smem);

    // projector tile images, built once here when they fit in half of the
    // free device memory (MLMD_NL_TILES=0 keeps generating them per launch)
    const char* te = std::getenv("MLMD_NL_TILES");
    if (te && te[0] == '0') return;
    const int apt = 128 / np;
    std::vector<int64_t> soff(t->nbricks + 1, 0), poff(t->nbricks + 1, 0);
    for (int b = 0; b < t->nbricks; ++b) {
        const int nab = bstart[b + 1] - bstart[b];
        soff[b + 1] = soff[b] + (nab + 3) / 4;
        poff[b + 1] = poff[b] + (int64_t)((nab + apt - 1) / apt) * (BP / KC);
    }
    const size_t bytes_s = (size_t)soff[t->nbricks] * IMG, bytes_p = (size_t)poff[t->nbricks] * IMG;
    size_t free_b = 0, total_b = 0;
    MLMD_CUDA(cudaMemGetInfo(&free_b, &total_b));
    if (bytes_s + bytes_p == 0 || bytes_s + bytes_p > free_b / 2) return;
    t->soff = (int64_t*)upload(soff.data(), sizeof(int64_t) * soff.size());
    t->poff = (int64_t*)upload(poff.data(), sizeof(int64_t) * poff.size());
    t->As = (unsigned char*)d.mem.get(std::max<size_t>(bytes_s, 16));
    t->Ap = (unsigned char*)d.mem.get(std::max<size_t>(bytes_p, 16));
    TcGeo G = geo_for(d);
    G.As = G.Ap = nullptr;
    const size_t asm_bytes = atom_bytes_for(t->max_atoms, np) + 16;
    const void* bk = reinterpret_cast<const void*>(np == 4 ? k_nl_tiles<4> : k_nl_tiles<8>);
    ensure_dynamic_smem(bk, asm_bytes);
    if (np == 4) k_nl_tiles<4><<<t->nbricks, NT, asm_bytes, d.stream>>>(G, t->As, t->Ap);
    else k_nl_tiles<8><<<t->nbricks, NT, asm_bytes, d.stream>>>(G, t->As, t->Ap);
    d.launches++;
    MLMD_CUDA(cudaGetLastError());
    MLMD_CUDA(cudaStreamSynchronize(d.stream));
}

void launch_nl_energy(Domain& d, const void* P, double* row) {
    k_nl_energy<<<1, 512, 0, d.stream>>>((const float*)P, d.f, d.nltc->aD, (int64_t)d.nl.n_atoms * d.nl.n_proj, d.ld,
                                         row);
    d.launches++;
    MLMD_CUDA(cudaGetLastError());
}

// out += gamma sum_r B (D o P): the nonlocal half of a stage, on top of the
// local part the stage kernel wrote to out; P is Pa or Pb, whose split copy
// (P3a / P3b) the projection left behind.  Also leaves the split output in
// w3 for the projection of out.
void launch_nl_scatter_tc(Domain& d, const void* P, void* out, double gre, double gim) {
    const TcGeo G = geo_for(d);
    NlTc& t = *d.nltc;
    const int np = d.nl.n_proj;
    const int stages = stages_for(G.ld2, t.max_atoms, np);
    const size_t smem = smem_for(G.ld2, t.max_atoms, np);
    const uint16_t* P3 = P == d.Pa ? t.P3a : t.P3b;
    ProfScope ps(d.prof, MLMD_KERNEL_SCATTER, d.stream);
    auto kern = np == 4 ? k_nl_scatter_tc<4> : k_nl_scatter_tc<8>;
    kern<<<t.nbricks, NT + 32, smem, d.stream>>>(G, P3, d.nl.n_atoms, (float*)out, t.w3, t.nbricks, (float)gre, (float)gim,
                                            stages, d.err_flag);
    d.launches++;
    MLMD_CUDA(cudaGetLastError());
}

// P = dV B^T w (zeroed first, accumulated by atomics), then its split copy
// D o P for the next scatter.  w3_ready: the scatter just wrote w's split
// copy; otherwise it is made here.
void launch_nl_project_tc(Domain& d, const void* w, void* P, bool w3_ready) {
    const TcGeo G = geo_for(d);
    NlTc& t = *d.nltc;
    const int np = d.nl.n_proj;
    const int stages = stages_for(G.ld2, t.max_atoms, np);
    const size_t smem = smem_for(G.ld2, t.max_atoms, np);
    ProfScope ps(d.prof, MLMD_KERNEL_PROJECT, d.stream);
    if (!w3_ready) {
        k_nl_split_w<<<t.nbricks, 256, 0, d.stream>>>(G, (const float*)w, t.nbricks, t.w3);
        d.launches++;
    }
    MLMD_CUDA(cudaMemsetAsync(P, 0, (size_t)d.nl.n_atoms * np * G.ld2 * sizeof(float), d.stream));
    const float dV = (float)(d.desc.h * d.desc.h * d.desc.h);
    auto kern = np == 4 ? k_nl_project_tc<4> : k_nl_project_tc<8>;
    kern<<<t.nbricks, NT + 32, smem, d.stream>>>(G, t.w3, t.nbricks, (float*)P, dV, stages, d.err_flag);
    uint16_t* P3 = P == d.Pa ? t.P3a : t.P3b;
    const int64_t items = (int64_t)d.nl.n_atoms * G.ld2;
    const int blocks = (int)std::min<int64_t>((items + 255) / 256, 4096);
    if (np == 4) k_nl_split_P<4><<<blocks, 256, 0, d.stream>>>((const float*)P, t.aD, d.nl.n_atoms, G.ld2, P3);
    else k_nl_split_P<8><<<blocks, 256, 0, d.stream>>>((const float*)P, t.aD, d.nl.n_atoms, G.ld2, P3);
    d.launches += 2;
    MLMD_CUDA(cudaGetLastError());
}

}  // namespace mlmd
