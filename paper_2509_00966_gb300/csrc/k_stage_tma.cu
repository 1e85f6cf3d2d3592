// TMA-staged stage kernel: out = psi + gamma * h(A) w with the Hamiltonian
// of Eq. 3, 2.5-D blocked, with the nonlocal scatter-back of Sec. V.B.5
// fused, and the column projection kernel that prepares its input.
//
// A CTA owns an 8 x 8 tile of grid points in x-y, one 128-byte chunk of the
// orbital row (16 complex64 or 8 complex128 orbitals; 64-byte chunks when the
// padded row is not a multiple of 128 bytes) and a range of z planes (its
// "column").  It streams along z: every plane of w is brought into shared
// memory by five TMA tile loads (the 8 x 8 centre and the four 2-deep
// star-halo slabs, at periodically wrapped coordinates, so no corner is
// loaded), through a ring of slots kept ahead of the plane being computed.
// The x-y neighbours come from shared memory; the z neighbours of each
// thread's own points stay in registers as the window slides.
//
// Nonlocal part: the projections <b|w> of the atoms whose spheres touch the
// column are staged in shared memory once per CTA for the scatter-back
// B (D o P).  The projections of the output, <b|out>, which the next stage
// needs, come from k_nl_project_cols over the same columns right after the
// stage: summing them inside the plane loop put a reduction behind every
// per-plane barrier, which cost more than reading the output once more.
//
// Every mbarrier wait is bounded: on expiry the CTA raises the domain's
// error word, waits (bounded) for its copies in flight, and stops.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <type_traits>

#include "mlmd_internal.cuh"

namespace mlmd {

struct TmaMaps {
    const void* base = nullptr;
    CUtensorMap centre{}, xslab{}, yslab{};
};

struct TmaState {
    bool ok = false;          // tiles divide the grid and the row splits into chunks
    int vp = 0;               // 16-byte vectors per point per chunk (8 or 4)
    int tpp = 4;              // threads per grid point of the stage kernel (4, or 8 with vp = 8)
    bool vp8_ok = false;      // the row splits into 128-byte chunks
    bool tuned = false;       // tile shape chosen by timing
    int zc = 0;               // planes per CTA
    int zc_full = 0;          // planes per CTA without projectors (zc <= zc_full)
    int ncols = 0;            // tiles x z-chunks
    std::vector<TmaMaps> maps;
    // nonlocal tables of the fused path (device, owned by the domain's allocator)
    bool nl_ok = false;
    int maxs = 0;             // most atoms touching one column
    int32_t* col_start = nullptr;
    int32_t* col_atom = nullptr;
    // scatter-back entries, one 16-byte aligned block per (column, plane):
    // int32 header [68] = entry offsets of the 64 points (65 values), the
    // entry count n and n rounded up to 4; then the slots [n4] int32, then
    // beta * D [n][NP] in the working real type
    unsigned char* sblk = nullptr;
    int64_t* sblk_off = nullptr;      // [ncols * zc + 1] byte offsets
    int scap = 0;                     // largest block, bytes
    // projection tables: half-height columns of PZC planes, entries slot-major
    int pzc = 0;              // planes per projection column
    int pcap = 0;             // most entries of one projection column, a multiple of 4
    int32_t* pp_seg = nullptr;        // [slots + 1] first entry of each (column, slot)
    int32_t* pp_atom_start = nullptr; // [ncols_p + 1] ranges of pp_atom
    int32_t* pp_atom = nullptr;       // atoms of each projection column, ascending
    int32_t* pp_key = nullptr;        // [n_list + 8] point | plane << 6 | slot << 10
    void* pp_beta = nullptr;          // [n_list][NP]
};

namespace {

constexpr int TX = 8, TY = 8;
// most z planes one CTA computes
constexpr int kMaxZc = 32;
constexpr long long kWaitCycles = 4000000000LL;   // ~2 s at 2 GHz

template <typename R> struct V16;
template <> struct V16<float> { static constexpr int NC = 2; };
template <> struct V16<double> { static constexpr int NC = 1; };

template <typename R> struct Cv {
    R re[V16<R>::NC];
    R im[V16<R>::NC];
};

__device__ __forceinline__ void unpack(const float4 t, Cv<float>& c) {
    c.re[0] = t.x; c.im[0] = t.y; c.re[1] = t.z; c.im[1] = t.w;
}
__device__ __forceinline__ void unpack(const float4 t, Cv<double>& c) {
    double2 d = *reinterpret_cast<const double2*>(&t);
    c.re[0] = d.x; c.im[0] = d.y;
}
__device__ __forceinline__ float4 pack(const Cv<float>& c) { return make_float4(c.re[0], c.im[0], c.re[1], c.im[1]); }
__device__ __forceinline__ float4 pack(const Cv<double>& c) {
    double2 d = make_double2(c.re[0], c.im[0]);
    return *reinterpret_cast<const float4*>(&d);
}

// ---- PTX wrappers ---------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
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

// Bounded wait on one phase of an mbarrier: false after ~kWaitCycles.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;     // the usual case: no clock read
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > kWaitCycles) return false;
    return true;
}

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3),
          "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

template <typename R> struct TGeo {
    R kc0, kc1, kc2, gk1, gk2;
    int nx, ny, nz, ld;
    int ntx;       // tiles along x
    int zc;        // planes per CTA
};

// Shared-memory slot of w: centre [TY][TX][VP], xm/xp [TY][2][VP], ym/yp
// [2][TX][VP] (16-byte vectors).
template <int VP> struct Slot {
    static constexpr int C = 0;
    static constexpr int XM = C + TY * TX * VP;
    static constexpr int XP = XM + TY * 2 * VP;
    static constexpr int YM = XP + TY * 2 * VP;
    static constexpr int YP = YM + 2 * TX * VP;
    static constexpr int N = YP + 2 * TX * VP;    // vectors per slot
    static constexpr uint32_t BYTES = N * 16;
    static constexpr int PN = TY * TX * VP;       // vectors of a psi tile
    static constexpr uint32_t PSI_BYTES = PN * 16;
};
// The scatter entry block and (when it comes by TMA) psi's centre tile of
// computed plane j share a ring of XSL slots and one mbarrier per slot; they
// are brought one plane ahead of their use into slot j % XSL.  One plane of
// look-ahead is enough; the shared memory goes to a fifth w slot instead
// (two planes of w in flight).
constexpr int XSL = 2;

// Vector (x+dx, y+dy) of the plane in slot s, one of dx, dy zero, |d| <= 2.
template <int VP>
__device__ __forceinline__ const float4* nb_ptr(const float4* s, int x, int y, int j) {
    if (x < 0) return s + Slot<VP>::XM + (y * 2 + (x + 2)) * VP + j;
    if (x >= TX) return s + Slot<VP>::XP + (y * 2 + (x - TX)) * VP + j;
    if (y < 0) return s + Slot<VP>::YM + ((y + 2) * TX + x) * VP + j;
    if (y >= TY) return s + Slot<VP>::YP + ((y - TY) * TX + x) * VP + j;
    return s + Slot<VP>::C + (y * TX + x) * VP + j;
}

// With 128-byte chunks (VP = 8) the tiles arrive with TMA's 128-byte swizzle:
// the 16-byte vector v of a 128-byte row at float4 offset o (a multiple of 8,
// measured from a 1024-byte aligned base) sits at o + (v ^ (o / 8 mod 8)).
// That spreads the same vector of eight consecutive points over all banks.
template <int VP>
__device__ __forceinline__ int swz(int o, int v) {
    if constexpr (VP == 8) return o + (v ^ ((o >> 3) & 7));
    else return o + v;
}


// Nonlocal tables of the fused path (see the file comment).
template <typename R> struct TNl {
    const unsigned char* sblk; // scatter-back entry blocks (see TmaState)
    const int64_t* sblk_off;
    int scap;
    const int32_t* col_start;  // [ncols + 1]
    const int32_t* col_atom;   // global atom ids of each column, ascending
    const R* Pin;              // <b|w>: [n_atoms][NP] rows of 2 ld reals
    R* Pout;                   // <b|out> accumulated (zeroed by the caller), or null
    // projection of the output: projection columns (PZC planes), entries
    // ordered by (slot, plane, point) within a column
    const int32_t* pp_seg;     // [slots + 1] first entry of each (column, slot)
    const int32_t* pp_atom_start;
    const int32_t* pp_atom;
    const int32_t* pp_key;     // W row in the column's planes: plane * 64 + y * 8 + x
    const R* pp_beta;          // [..][NP]
    R dV;
    int maxs;                  // staging capacity (atoms per column)
};

template <typename R, int NP>
__device__ __forceinline__ void load_beta(const R* p, R (&b)[NP]) {
    constexpr int PER = 16 / (int)sizeof(R);
#pragma unroll
    for (int v = 0; v < NP / PER; ++v) {
        const float4 t = __ldg(reinterpret_cast<const float4*>(p) + v);
        const R* tr = reinterpret_cast<const R*>(&t);
#pragma unroll
        for (int k = 0; k < PER; ++k) b[v * PER + k] = tr[k];
    }
}

__device__ __forceinline__ void global_add(float* p, float4 v, float s) {
    atomicAdd(reinterpret_cast<float4*>(p), make_float4(s * v.x, s * v.y, s * v.z, s * v.w));
}
__device__ __forceinline__ void global_add(double* p, float4 v, double s) {
    const double2 d = *reinterpret_cast<const double2*>(&v);
    atomicAdd(p, s * d.x);
    atomicAdd(p + 1, s * d.y);
}

// NP projector values of one entry from shared memory, 16 bytes at a time
template <typename R, int NP>
__device__ __forceinline__ void load_beta_s(const R* p, R (&b)[NP]) {
    constexpr int PER = 16 / (int)sizeof(R);
#pragma unroll
    for (int v = 0; v < NP / PER; ++v) {
        const float4 t = reinterpret_cast<const float4*>(p)[v];
        const R* tr = reinterpret_cast<const R*>(&t);
#pragma unroll
        for (int k = 0; k < PER; ++k) b[v * PER + k] = tr[k];
    }
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// packed pairs of FP32 (Blackwell f32x2 arithmetic): one complex64 value
__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) { return __ffma2_rn(make_float2(-1.f, -1.f), b, a); }
__device__ __forceinline__ float2 f2s(float x) { return make_float2(x, x); }
__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float2 swp(float2 v) { return make_float2(v.y, v.x); }

template <typename R, int ORDER, int VP, int NP, int NSLOT, int TPP, bool OBS>
__global__ void __launch_bounds__(64 * TPP, 2)
    k_stage_tma(const __grid_constant__ CUtensorMap tm_c, const __grid_constant__ CUtensorMap tm_x,
                const __grid_constant__ CUtensorMap tm_y, const __grid_constant__ CUtensorMap tm_p, int psi_mode,
                TGeo<R> G, R* out,
                const R* __restrict__ V, const R* __restrict__ f, const double* __restrict__ Ak, TNl<R> N,
                R gre, R gim, double* __restrict__ obs, int* err) {
    constexpr int NC = V16<R>::NC;
    constexpr int NVT = VP / TPP;                   // 16-byte vectors of its point per thread
    constexpr int NT = 64 * TPP;                    // threads
    constexpr int OCR = VP * 16 / sizeof(R);        // reals per chunk row
    constexpr int NPV = (NP > 0 ? NP : 1);
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // TMA destinations on a 128-byte boundary (the launch adds 128 bytes of slack)
    // TMA destinations on a 1024-byte boundary (the launch adds 1024 bytes of
    // slack): the swizzle pattern is a function of the address bits
    float4* ring = reinterpret_cast<float4*>(smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u));
    float4* sPsi = ring + NSLOT * Slot<VP>::N;      // [XSL][TY][TX][VP] psi tiles
    float4* sP = sPsi + XSL * Slot<VP>::PN;         // [maxs][NP][VP] staged <b|w>
    unsigned char* sE = reinterpret_cast<unsigned char*>(sP + N.maxs * NPV * VP);   // [XSL][scap] entry blocks
    __shared__ __align__(8) uint64_t bars[NSLOT];
    __shared__ __align__(8) uint64_t xbars[XSL];
    __shared__ int64_t soff[kMaxZc + 1];            // entry-block offsets of the column's planes
    __shared__ R sA[4];
    __shared__ int abort_sh;
    __shared__ int iss[8];                          // copy-issue state (see issue)

    const int tid = threadIdx.x;
    // point of the tile and first vector (then jv + TPP k); with 4 threads per
    // point a warp holds a 4 x 2 block of points (its scatter loop runs as
    // long as its busiest point, and compact blocks see more even sphere
    // counts than a row of 8); two consecutive points are x neighbours, so
    // the swizzled 16-byte loads stay free of bank conflicts
    const int wp = tid / TPP, jv = tid % TPP;
    const int lx = (wp & 3) + ((wp >> 3) & 1) * 4, ly = ((wp >> 2) & 1) + (wp >> 4) * 2;
    const int pt = ly * TX + lx;                    // row-major index in the tile
    // grid (chunk, tile, z range): the chunks of one tile run side by side,
    // so each grid point's orbital row is read from DRAM in one stretch
    const int tile = blockIdx.y;
    const int x0 = (tile % G.ntx) * TX, y0 = (tile / G.ntx) * TY;
    const int chunk = blockIdx.x;
    const int z0 = blockIdx.z * G.zc;
    const int nzc = min(G.zc, G.nz - z0);           // planes computed by this CTA
    const int nplanes = nzc + 4;                    // planes z0-2 .. z0+nzc+1
    const int c0 = chunk * OCR;                     // first real of the chunk within a row
    // psi_mode 0: out = gamma h w; 1: psi is w itself (its centre tile is in
    // the ring already); 2: psi's centre tile comes by TMA with each plane
    const bool has_psi = psi_mode != 0;
    // complex64 launches take the packed path: h w as sum_n c_n w_n with the
    // complex coefficient c_n = k_n - i a_n of each stencil neighbour (k from
    // the Laplacian, a = A . gradient weight), evaluated as f32x2
    // multiply-adds on (re, im) pairs; with observables the gradient is kept
    // per axis for the current and the sums run on packed pairs too
    constexpr bool FAST = std::is_same<R, float>::value;
    const int col = tile + gridDim.y * blockIdx.z;

    if (tid == 0) {
        iss[0] = (x0 - 2 + G.nx) % G.nx;
        iss[1] = (x0 + TX) % G.nx;
        iss[2] = (y0 - 2 + G.ny) % G.ny;
        iss[3] = (y0 + TY) % G.ny;
        iss[4] = ((z0 - 2) % G.nz + G.nz) % G.nz;
        iss[5] = 0;
        iss[6] = iss[7] = 0;
        for (int s = 0; s < NSLOT; ++s) mbar_init(&bars[s], 1);
        for (int s = 0; s < XSL; ++s) mbar_init(&xbars[s], 1);
        abort_sh = 0;
        fence_proxy_async();
    }
    // TMA of the next plane, p = 0, 1, 2, ... in turn (z = z0 - 2 + p, slot
    // p % NSLOT).  One thread issues right after each plane barrier (lane 0
    // of warp i mod the warp count at plane i, so no warp carries the issue
    // work every plane); the issue state lives in shared memory: the wrapped
    // halo origins and the running (z, slot) pair, so no thread divides by
    // the grid size per plane, and the copies issued so far on each ring
    // (iss[]: x-2, x+8, y-2, y+8, z, slot, planes, entry / psi pairs).
    auto issue = [&]() {
        const int s = iss[5], zz = iss[4];
        float4* d = ring + s * Slot<VP>::N;
        uint64_t* b = &bars[s];
        mbar_expect_tx(b, Slot<VP>::BYTES);
        tma_load_4d(d + Slot<VP>::C, &tm_c, c0, x0, y0, zz, b);
        tma_load_4d(d + Slot<VP>::XM, &tm_x, c0, iss[0], y0, zz, b);
        tma_load_4d(d + Slot<VP>::XP, &tm_x, c0, iss[1], y0, zz, b);
        tma_load_4d(d + Slot<VP>::YM, &tm_y, c0, x0, iss[2], zz, b);
        tma_load_4d(d + Slot<VP>::YP, &tm_y, c0, x0, iss[3], zz, b);
        iss[4] = zz + 1 == G.nz ? 0 : zz + 1;
        iss[5] = s + 1 == NSLOT ? 0 : s + 1;
        iss[6] += 1;
    };
    auto wait_plane = [&](int p) -> bool { return mbar_wait_bounded(&bars[p % NSLOT], (uint32_t)((p / NSLOT) & 1)); };
    // entry block and psi tile of computed plane j (z = z0 + j) into slot
    // j % XSL, both on that slot's barrier (nothing when neither is used)
    const bool has_x = NP > 0 || psi_mode == 2;
    auto issue_x = [&](int j) {
        if (!has_x || j >= nzc) return;
        uint64_t* b = &xbars[j % XSL];
        int64_t eo = 0;
        uint32_t eb = 0;
        if (NP > 0) {
            eo = soff[j];
            eb = (uint32_t)(soff[j + 1] - eo);      // >= the 272-byte header
        }
        mbar_expect_tx(b, eb + (psi_mode == 2 ? Slot<VP>::PSI_BYTES : 0u));
        if (NP > 0) bulk_g2s(sE + (size_t)(j % XSL) * N.scap, N.sblk + eo, eb, b);
        if (psi_mode == 2) tma_load_4d(sPsi + (j % XSL) * Slot<VP>::PN, &tm_p, c0, x0, y0, z0 + j, b);
        iss[7] = j + 1;
    };

    // shared-memory offsets (16-byte vectors) of this thread's first vector and
    // of its x-y neighbours within a slot; vector k adds 4 k
    // this thread's vectors of its point: vb + k, k < NVT (NVT is 1 or 2, vb
    // even when NVT = 2, so the vector k of a row sits at the row's vector-0
    // address XOR k)
    static_assert(NVT == 1 || NVT == 2, "one or two vectors per thread");
    const int vb = jv * NVT;
    const int offC = swz<VP>(Slot<VP>::C + (ly * TX + lx) * VP, vb);
    const int offPs = swz<VP>(pt * VP, vb);        // within a psi tile
    int offN[8];
    {
        const int dx[8] = {1, -1, 0, 0, 2, -2, 0, 0}, dy[8] = {0, 0, 1, -1, 0, 0, 2, -2};
#pragma unroll
        for (int n = 0; n < 8; ++n) offN[n] = swz<VP>((int)(nb_ptr<VP>(ring, lx + dx[n], ly + dy[n], 0) - ring), vb);
    }

    // the first planes and psi tiles are in flight while the column's
    // projections are staged; the entry blocks need the staged offsets
    if (tid == 0) {
        for (int p = 0; p < NSLOT && p < nplanes; ++p) issue();
    }
    if (tid < 3) sA[tid] = (R)Ak[tid];
    if (tid == 3) sA[3] = (R)(0.5 * (Ak[0] * Ak[0] + Ak[1] * Ak[1] + Ak[2] * Ak[2]));
    int cs = 0, na = 0;
    if (NP > 0) {
        if (tid <= nzc) soff[tid] = N.sblk_off[(int64_t)col * G.zc + tid];
        cs = N.col_start[col];
        na = N.col_start[col + 1] - cs;
        for (int idx = tid; idx < na * NPV * VP; idx += NT) {
            const int s = idx / (NPV * VP), r = idx - s * (NPV * VP), i = r / VP, jj = r - i * VP;
            const int64_t a = N.col_atom[cs + s];
            sP[idx] = __ldg(reinterpret_cast<const float4*>(N.Pin + (a * NPV + i) * 2 * G.ld + c0) + jj);
        }
    }
    __syncthreads();

    if (tid == 0)
        for (int j = 0; j < XSL - 1; ++j) issue_x(j);
    // register window of the thread's vectors: q[k][0..4] = planes z-2 .. z+2
    float4 q[NVT][5];
    bool ok = true;
    for (int p = 0; p < 4; ++p) ok = ok && wait_plane(p);
    if (!ok) abort_sh = 1;
    __syncthreads();
    const bool aborted0 = abort_sh != 0;
    if (!aborted0) {
        for (int p = 0; p < 4; ++p) {
            const float4* s = ring + (p % NSLOT) * Slot<VP>::N;
#pragma unroll
            for (int k = 0; k < NVT; ++k) q[k][p] = s[offC ^ k];
        }
    }
    __syncthreads();
    if (tid == 0 && !aborted0 && iss[6] < nplanes) {   // slot 0 (plane z0-2) is free again
        fence_proxy_async();
        issue();
    }

    R acc[5] = {0, 0, 0, 0, 0};
    // packed observable sums (the two halves add up at the end): norm,
    // energy and the three current components
    float2 aN = f2s(0.f), aE = f2s(0.f), aJ[3] = {f2s(0.f), f2s(0.f), f2s(0.f)};
    // occupations of the thread's orbitals, loop invariant
    R fo[NVT][NC];
    if constexpr (OBS) {
#pragma unroll
        for (int k = 0; k < NVT; ++k)
#pragma unroll
            for (int e = 0; e < NC; ++e) fo[k][e] = f[c0 / 2 + (vb + k) * NC + e];
    }
    const int64_t plane_stride = (int64_t)G.nx * G.ny;
    int64_t g = (x0 + lx) + (int64_t)G.nx * (y0 + ly) + plane_stride * z0;
    const int64_t row = 2 * (int64_t)G.ld;
    R vnext = nzc > 0 ? V[g] : (R)0;       // V one plane ahead
    // running ring positions (no division per plane): slots of planes z and
    // z+2 and the phase parity of the latter's barrier; the output row
    int s2 = 2 % NSLOT, s4i = 4 % NSLOT;
    uint32_t ph4 = (uint32_t)((4 / NSLOT) & 1);
    R* orow = out + g * row + c0;
    const int64_t orow_step = plane_stride * row;
    for (int i = 0; i < nzc && !aborted0; ++i, g += plane_stride, orow += orow_step) {
        // per-point global loads first, so that they overlap the plane wait
        // and the shared-memory stencil
        const R vv = vnext;
        if (i + 1 < nzc) vnext = V[g + plane_stride];
        float4 ps_cur[NVT];
        // plane z+2 (p = i+4) must have landed
        ok = mbar_wait_bounded(&bars[s4i], ph4);
        if (!ok) abort_sh = 1;
        __syncthreads();                    // also: all reads of the slot of plane z-1 are done
        if (abort_sh) break;
        if (tid == ((i & (NT / 32 - 1)) << 5)) {
            fence_proxy_async();
            if (iss[6] < nplanes) issue();  // next plane into the slot of plane z-1
            issue_x(i + XSL - 1);           // into the entry / psi slot of plane z-1
        }
        const float4* sc = ring + s2 * Slot<VP>::N;     // plane z
        const float4* s4 = ring + s4i * Slot<VP>::N;    // plane z+2
        s2 = s2 + 1 == NSLOT ? 0 : s2 + 1;
        if (++s4i == NSLOT) { s4i = 0; ph4 ^= 1u; }
        Cv<R> hw[NVT], dd[NVT][OBS ? 3 : 1];
        float2 hp[NVT][2];                  // packed path: h w of the vector's two complex values
        float2 dlp[NVT][2][OBS ? 3 : 1];    // packed path with observables: gradient per axis
        if constexpr (FAST) {
            const float2 kk1 = f2s((float)G.kc1), kk2 = f2s((float)G.kc2);
            const float2 cd = f2s((float)(G.kc0 + sA[3] + vv));
            float2 a1[3], a2[3];
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) { a1[ax] = f2s((float)(sA[ax] * G.gk1)); a2[ax] = f2s((float)(sA[ax] * G.gk2)); }
#pragma unroll
            for (int k = 0; k < NVT; ++k) {
                q[k][4] = s4[offC ^ k];
                float4 p1[3], m1[3], p2[3], m2[3];
#pragma unroll
                for (int ax = 0; ax < 2; ++ax) {
                    p1[ax] = sc[(offN[2 * ax]) ^ k];
                    m1[ax] = sc[(offN[2 * ax + 1]) ^ k];
                    if (ORDER == 4) {
                        p2[ax] = sc[(offN[4 + 2 * ax]) ^ k];
                        m2[ax] = sc[(offN[5 + 2 * ax]) ^ k];
                    }
                }
                p1[2] = q[k][3]; m1[2] = q[k][1]; p2[2] = q[k][4]; m2[2] = q[k][0];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    auto part = [&](float4 v) { return h == 0 ? lo2(v) : hi2(v); };
                    float2 s1 = f2add(f2add(part(p1[0]), part(m1[0])), f2add(part(p1[1]), part(m1[1])));
                    s1 = f2add(s1, f2add(part(p1[2]), part(m1[2])));
                    float2 hk = f2mul(kk1, s1);
                    float2 ha;
                    if constexpr (OBS) {
                        // gradient per axis, dl = gk1 (w+1 - w-1) + gk2 (w+2 - w-2), then A . dl
#pragma unroll
                        for (int ax = 0; ax < 3; ++ax) {
                            float2 dl = f2mul(f2s((float)G.gk1), f2sub(part(p1[ax]), part(m1[ax])));
                            if (ORDER == 4) dl = f2fma(f2s((float)G.gk2), f2sub(part(p2[ax]), part(m2[ax])), dl);
                            dlp[k][h][ax] = dl;
                        }
                        ha = f2mul(f2s((float)sA[0]), dlp[k][h][0]);
                        ha = f2fma(f2s((float)sA[1]), dlp[k][h][1], ha);
                        ha = f2fma(f2s((float)sA[2]), dlp[k][h][2], ha);
                    } else {
                        ha = f2mul(a1[0], f2sub(part(p1[0]), part(m1[0])));
                        ha = f2fma(a1[1], f2sub(part(p1[1]), part(m1[1])), ha);
                        ha = f2fma(a1[2], f2sub(part(p1[2]), part(m1[2])), ha);
                        if (ORDER == 4)
#pragma unroll
                            for (int ax = 0; ax < 3; ++ax) ha = f2fma(a2[ax], f2sub(part(p2[ax]), part(m2[ax])), ha);
                    }
                    if (ORDER == 4) {
                        float2 s2 = f2add(f2add(part(p2[0]), part(m2[0])), f2add(part(p2[1]), part(m2[1])));
                        s2 = f2add(s2, f2add(part(p2[2]), part(m2[2])));
                        hk = f2fma(kk2, s2, hk);
                    }
                    hk = f2fma(cd, part(q[k][2]), hk);
                    // h w = hk - i ha
                    hp[k][h] = f2fma(make_float2(1.f, -1.f), swp(ha), hk);
                }
            }
        } else {
#pragma unroll
        for (int k = 0; k < NVT; ++k) {
            q[k][4] = s4[offC ^ k];
            Cv<R> qq[5];
#pragma unroll
            for (int w = 0; w < 5; ++w) unpack(q[k][w], qq[w]);
            const Cv<R>& c = qq[2];
            Cv<R> lap, t1, t2, t3, t4;
            Cv<R> dl[3];
#pragma unroll
            for (int e = 0; e < NC; ++e) { lap.re[e] = G.kc0 * c.re[e]; lap.im[e] = G.kc0 * c.im[e]; }
#pragma unroll
            for (int ax = 0; ax < 2; ++ax) {
                unpack(sc[(offN[2 * ax]) ^ k], t1);
                unpack(sc[(offN[2 * ax + 1]) ^ k], t2);
                if (ORDER == 4) {
                    unpack(sc[(offN[4 + 2 * ax]) ^ k], t3);
                    unpack(sc[(offN[5 + 2 * ax]) ^ k], t4);
                }
#pragma unroll
                for (int e = 0; e < NC; ++e) {
                    lap.re[e] += G.kc1 * (t1.re[e] + t2.re[e]);
                    lap.im[e] += G.kc1 * (t1.im[e] + t2.im[e]);
                    dl[ax].re[e] = G.gk1 * (t1.re[e] - t2.re[e]);
                    dl[ax].im[e] = G.gk1 * (t1.im[e] - t2.im[e]);
                    if (ORDER == 4) {
                        lap.re[e] += G.kc2 * (t3.re[e] + t4.re[e]);
                        lap.im[e] += G.kc2 * (t3.im[e] + t4.im[e]);
                        dl[ax].re[e] += G.gk2 * (t3.re[e] - t4.re[e]);
                        dl[ax].im[e] += G.gk2 * (t3.im[e] - t4.im[e]);
                    }
                }
            }
#pragma unroll
            for (int e = 0; e < NC; ++e) {
                lap.re[e] += G.kc1 * (qq[3].re[e] + qq[1].re[e]);
                lap.im[e] += G.kc1 * (qq[3].im[e] + qq[1].im[e]);
                dl[2].re[e] = G.gk1 * (qq[3].re[e] - qq[1].re[e]);
                dl[2].im[e] = G.gk1 * (qq[3].im[e] - qq[1].im[e]);
                if (ORDER == 4) {
                    lap.re[e] += G.kc2 * (qq[4].re[e] + qq[0].re[e]);
                    lap.im[e] += G.kc2 * (qq[4].im[e] + qq[0].im[e]);
                    dl[2].re[e] += G.gk2 * (qq[4].re[e] - qq[0].re[e]);
                    dl[2].im[e] += G.gk2 * (qq[4].im[e] - qq[0].im[e]);
                }
            }
            const R diag = vv + sA[3];
#pragma unroll
            for (int e = 0; e < NC; ++e) {
                const R gr = sA[0] * dl[0].re[e] + sA[1] * dl[1].re[e] + sA[2] * dl[2].re[e];
                const R gi = sA[0] * dl[0].im[e] + sA[1] * dl[1].im[e] + sA[2] * dl[2].im[e];
                hw[k].re[e] = lap.re[e] + diag * c.re[e] + gi;
                hw[k].im[e] = lap.im[e] + diag * c.im[e] - gr;
            }
            if constexpr (OBS) {
#pragma unroll
                for (int ax = 0; ax < 3; ++ax) dd[k][ax] = dl[ax];
            }
        }
        }
        // the entry block and psi tile of this plane must have landed; on a
        // timeout the scatter is skipped (the CTA aborts) rather than read a
        // stale block
        bool e_ok = true;
        if (has_x) {
            e_ok = mbar_wait_bounded(&xbars[i % XSL], (uint32_t)((i / XSL) & 1));
            if (!e_ok) abort_sh = 1;
        }
        if (NP > 0 && e_ok) {   // scatter-back: sum_(a,i) b_ai(r) D_ai <b_ai|w>
            const unsigned char* eb = sE + (size_t)(i % XSL) * N.scap;
            const int32_t* hdr = reinterpret_cast<const int32_t*>(eb);
            const int32_t* eslot = hdr + 68;
            const R* ebd = reinterpret_cast<const R*>(eb + 272 + 4 * hdr[66]);
            const int e0 = hdr[pt], e1 = hdr[pt + 1];
            for (int e = e0; e < e1; ++e) {
                const int s = eslot[e];
                R b[NPV];
                load_beta_s<R, NPV>(ebd + (int64_t)e * NPV, b);   // beta * D
#pragma unroll
                for (int pi = 0; pi < NPV; ++pi) {
                    const R bd = b[pi];
#pragma unroll
                    for (int k = 0; k < NVT; ++k) {
                        const float4 pv4 = sP[(s * NPV + pi) * VP + vb + k];
                        if constexpr (FAST) {
                            hp[k][0] = f2fma(f2s((float)bd), lo2(pv4), hp[k][0]);
                            hp[k][1] = f2fma(f2s((float)bd), hi2(pv4), hp[k][1]);
                        } else {
                            Cv<R> pv;
                            unpack(pv4, pv);
#pragma unroll
                            for (int u = 0; u < NC; ++u) {
                                hw[k].re[u] += bd * pv.re[u];
                                hw[k].im[u] += bd * pv.im[u];
                            }
                        }
                    }
                }
            }
        }
        if (psi_mode == 2) {                // psi tile of this plane (landed with the entry block)
#pragma unroll
            for (int k = 0; k < NVT; ++k) ps_cur[k] = sPsi[(i % XSL) * Slot<VP>::PN + (offPs ^ k)];
        }
#pragma unroll
        for (int k = 0; k < NVT; ++k) {
            if constexpr (FAST) {
                const float4 ps = psi_mode == 1 ? q[k][2]
                                  : psi_mode == 2 ? ps_cur[k]
                                                  : make_float4(0.f, 0.f, 0.f, 0.f);
                // out = psi + gamma h w, gamma = gre + i gim
                const float2 gr2 = f2s((float)gre), gi2 = make_float2(-(float)gim, (float)gim);
                const float2 o0 = f2fma(gi2, swp(hp[k][0]), f2fma(gr2, hp[k][0], lo2(ps)));
                const float2 o1 = f2fma(gi2, swp(hp[k][1]), f2fma(gr2, hp[k][1], hi2(ps)));
                *(reinterpret_cast<float4*>(orow) + vb + k) = make_float4(o0.x, o0.y, o1.x, o1.y);
                if constexpr (OBS) {
                    // f |c|^2, f Re(c* h w) and f Re(c* (-i) dl_a), each as a packed
                    // pair whose halves add up to the term
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const float2 c = h == 0 ? lo2(q[k][2]) : hi2(q[k][2]);
                        const float2 f2 = f2s((float)fo[k][h]), f2m = make_float2((float)fo[k][h], -(float)fo[k][h]);
                        aN = f2fma(f2, f2mul(c, c), aN);
                        aE = f2fma(f2, f2mul(c, hp[k][h]), aE);
#pragma unroll
                        for (int ax = 0; ax < 3; ++ax) aJ[ax] = f2fma(f2m, f2mul(c, swp(dlp[k][h][ax])), aJ[ax]);
                    }
                }
#pragma unroll
                for (int w = 0; w < 4; ++w) q[k][w] = q[k][w + 1];
                continue;
            }
            Cv<R> o;
            if (has_psi) {
                Cv<R> ps;
                if (psi_mode == 1) unpack(q[k][2], ps);
                else unpack(ps_cur[k], ps);
#pragma unroll
                for (int e = 0; e < NC; ++e) {
                    o.re[e] = ps.re[e] + gre * hw[k].re[e] - gim * hw[k].im[e];
                    o.im[e] = ps.im[e] + gre * hw[k].im[e] + gim * hw[k].re[e];
                }
            } else {
#pragma unroll
                for (int e = 0; e < NC; ++e) {
                    o.re[e] = gre * hw[k].re[e] - gim * hw[k].im[e];
                    o.im[e] = gre * hw[k].im[e] + gim * hw[k].re[e];
                }
            }
            const float4 ov = pack(o);
            *(reinterpret_cast<float4*>(orow) + vb + k) = ov;
            if constexpr (OBS) {
                Cv<R> c;
                unpack(q[k][2], c);
#pragma unroll
                for (int e = 0; e < NC; ++e) {
                    const R cr = c.re[e], ci = c.im[e];
                    acc[0] += fo[k][e] * (cr * cr + ci * ci);
                    acc[1] += fo[k][e] * (cr * hw[k].re[e] + ci * hw[k].im[e]);
#pragma unroll
                    for (int ax = 0; ax < 3; ++ax)
                        acc[2 + ax] += fo[k][e] * (cr * dd[k][ax].im[e] - ci * dd[k][ax].re[e]);
                }
            }
#pragma unroll
            for (int w = 0; w < 4; ++w) q[k][w] = q[k][w + 1];
        }
    }
    __syncthreads();                        // the issue counters and abort_sh are final
    if (abort_sh) {
        if (tid == 0) {
            atomicExch(err, 1);
            // let the copies still in flight land before the CTA's shared
            // memory goes away: the latest copy issued into each slot of
            // each ring (earlier ones into the same slot completed before it
            // was issued; waiting on a completed phase returns at once)
            for (int p = max(0, iss[6] - NSLOT); p < iss[6]; ++p) (void)wait_plane(p);
            for (int j = max(0, iss[7] - XSL); j < iss[7]; ++j)
                (void)mbar_wait_bounded(&xbars[j % XSL], (uint32_t)((j / XSL) & 1));
        }
    }
    if constexpr (OBS) {
        if constexpr (FAST) {
            acc[0] = aN.x + aN.y;
            acc[1] = aE.x + aE.y;
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) acc[2 + ax] = aJ[ax].x + aJ[ax].y;
        }
        __shared__ double sh[NT / 32][5];
        const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
        for (int v = 0; v < 5; ++v)
            for (int o = 16; o > 0; o >>= 1) acc[v] += __shfl_xor_sync(0xffffffffu, acc[v], o);
        if (lane == 0)
#pragma unroll
            for (int v = 0; v < 5; ++v) sh[warp][v] = (double)acc[v];
        __syncthreads();
        if (tid < 5) {
            double t = 0.0;
            for (int w = 0; w < NT / 32; ++w) t += sh[w][tid];
            const int64_t blin = blockIdx.x + (int64_t)gridDim.x * (blockIdx.y + (int64_t)gridDim.y * blockIdx.z);
            obs[blin * 5 + tid] = t;
        }
    }
}



// <b|W> for every atom, by projection columns (an 8 x 8 tile of points, one
// orbital chunk, PZC planes).  Thread 0 brings the column's W planes (one
// TMA each, issued before the column's index loads) and its entries -- W
// row (plane * 64 + point) and beta, ordered by (slot, plane, point) -- (two
// bulk copies) into shared memory, all on one mbarrier.  The entries are cut into eight equal runs, one per warp;
// a warp walks the atoms (slots) its run overlaps and, for each, the
// entries in both, with the lanes split over (entry group, projector,
// 16-byte vector), then adds the atom's sum to Pout with one vector atomic.
// Every warp does the same work whatever the sizes of the atoms' spheres in
// the column.
template <typename R, int VP, int NP>
__global__ void __launch_bounds__(256) k_nl_project_cols(const __grid_constant__ CUtensorMap tm_c, TNl<R> N, int nx,
                                                         int ny, int nz, int ntx, int pzc, int ld, int pcap,
                                                         int* err) {
    constexpr int OCR = VP * 16 / sizeof(R);
    constexpr int NC = V16<R>::NC;
    constexpr int EG = 32 / VP;                              // entry groups per warp
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    // W [pzc][64][VP] float4 (swizzled like the stage kernel's tiles), rows [pcap + 8] int32, beta [pcap][NP] R
    const uint32_t wbytes = (uint32_t)pzc * 64 * VP * 16;
    const uint32_t kbytes = (uint32_t)(pcap + 8) * 4;
    const float4* sW = reinterpret_cast<const float4*>(base);
    __shared__ __align__(8) uint64_t bar;
    __shared__ int abort_sh;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int pcol = blockIdx.y + gridDim.y * blockIdx.z;    // grid (chunk, tile, z range)
    const int x0 = (blockIdx.y % ntx) * TX, y0 = (blockIdx.y / ntx) * TY;
    const int z0 = blockIdx.z * pzc;
    const int nzc = min(pzc, nz - z0);
    const int c0 = blockIdx.x * OCR;
    // the W planes go out first (they need no index), two arrivals on the
    // barrier: the planes' and, once the column's ranges are known, the
    // entries'
    if (tid == 0) {
        mbar_init(&bar, 2);
        abort_sh = 0;
        fence_proxy_async();
        mbar_expect_tx(&bar, (uint32_t)nzc * 64 * VP * 16);
        for (int iz = 0; iz < nzc; ++iz) tma_load_4d(base + (size_t)iz * 64 * VP * 16, &tm_c, c0, x0, y0, z0 + iz, &bar);
    }
    const int k0 = N.pp_atom_start[pcol], k1 = N.pp_atom_start[pcol + 1];   // the column's slots
    const int e0 = N.pp_seg[k0], e1 = N.pp_seg[k1];
    const int a0 = e0 & ~3, a1 = (e1 + 3) & ~3;
    const int32_t* sRow = reinterpret_cast<const int32_t*>(base + wbytes) - a0;
    const R* sB = reinterpret_cast<const R*>(base + wbytes + kbytes) - (int64_t)e0 * NP;
    if (tid == 0) {
        // (an empty column expects no entry bytes: its barrier completes with the planes)
        mbar_expect_tx(&bar, e1 > e0 ? (uint32_t)(a1 - a0) * 4 + (uint32_t)(e1 - e0) * NP * sizeof(R) : 0u);
        if (e1 > e0) {
            bulk_g2s(base + wbytes, N.pp_key + a0, (uint32_t)(a1 - a0) * 4, &bar);
            bulk_g2s(base + wbytes + kbytes, N.pp_beta + (int64_t)e0 * NP, (uint32_t)(e1 - e0) * NP * sizeof(R),
                     &bar);
        }
    }
    __syncthreads();
    const bool ok = mbar_wait_bounded(&bar, 0);
    const int T = e1 - e0;
    const int r0 = e0 + (int)(((int64_t)T * warp) / 8), r1 = e0 + (int)(((int64_t)T * (warp + 1)) / 8);
    const int eg = lane / VP, jj = lane % VP;
    const int64_t row = 2 * (int64_t)ld;
    if (ok && r1 > r0) {
        for (int k = k0; k < k1; ++k) {
            const int lo = max(r0, N.pp_seg[k]), hi = min(r1, N.pp_seg[k + 1]);
            if (lo >= hi) continue;                  // the same for the whole warp
            Cv<R> acc[NP];
#pragma unroll
            for (int pi = 0; pi < NP; ++pi)
#pragma unroll
                for (int u = 0; u < NC; ++u) { acc[pi].re[u] = 0; acc[pi].im[u] = 0; }
            if constexpr (sizeof(R) == 4) {
                // complex64: (re, im) pairs on packed f32x2 FMAs
                float2 a2[NP][2];
#pragma unroll
                for (int pi = 0; pi < NP; ++pi) a2[pi][0] = a2[pi][1] = make_float2(0.f, 0.f);
                for (int e = lo + eg; e < hi; e += EG) {
                    const int r = sRow[e];
                    const int K = r * VP + (VP == 8 ? (r & 7) : 0);
                    const float4 w4 = sW[K ^ jj];
                    R b[NP];
                    load_beta_s<R, NP>(sB + (int64_t)e * NP, b);
#pragma unroll
                    for (int pi = 0; pi < NP; ++pi) {
                        const float2 bb = f2s((float)b[pi]);
                        a2[pi][0] = f2fma(bb, lo2(w4), a2[pi][0]);
                        a2[pi][1] = f2fma(bb, hi2(w4), a2[pi][1]);
                    }
                }
#pragma unroll
                for (int pi = 0; pi < NP; ++pi) {
                    acc[pi].re[0] = a2[pi][0].x; acc[pi].im[0] = a2[pi][0].y;
                    acc[pi].re[NC - 1] = a2[pi][1].x; acc[pi].im[NC - 1] = a2[pi][1].y;
                }
            } else {
                for (int e = lo + eg; e < hi; e += EG) {
                    const int r = sRow[e];
                    // swizzled row start r*VP + (r mod 8): vector jj sits at that XOR jj
                    const int K = r * VP + (VP == 8 ? (r & 7) : 0);
                    Cv<R> w;
                    unpack(sW[K ^ jj], w);
                    R b[NP];
                    load_beta_s<R, NP>(sB + (int64_t)e * NP, b);
#pragma unroll
                    for (int pi = 0; pi < NP; ++pi)
#pragma unroll
                        for (int u = 0; u < NC; ++u) {
                            acc[pi].re[u] += b[pi] * w.re[u];
                            acc[pi].im[u] += b[pi] * w.im[u];
                        }
                }
            }
            // sum the entry groups (lanes jj, jj + VP, ...)
#pragma unroll
            for (int off = VP; off < 32; off <<= 1)
#pragma unroll
                for (int pi = 0; pi < NP; ++pi)
#pragma unroll
                    for (int u = 0; u < NC; ++u) {
                        acc[pi].re[u] += __shfl_xor_sync(0xffffffffu, acc[pi].re[u], off);
                        acc[pi].im[u] += __shfl_xor_sync(0xffffffffu, acc[pi].im[u], off);
                    }
            if (eg == 0) {
                const int64_t at = N.pp_atom[k];
#pragma unroll
                for (int pi = 0; pi < NP; ++pi)
                    global_add(N.Pout + (at * NP + pi) * row + c0 + jj * (16 / (int)sizeof(R)), pack(acc[pi]), N.dV);
            }
        }
    }
    if (!ok) abort_sh = 1;
    __syncthreads();
    if (tid == 0 && abort_sh) {
        atomicExch(err, 1);
        (void)mbar_wait_bounded(&bar, 0);     // copies still in flight land before the CTA exits
    }
}

template <typename R, int VP>
size_t project_smem(int np, int pcap, int pzc) {
    return (size_t)pzc * 64 * VP * 16 + (size_t)(pcap + 8) * 4 + (size_t)pcap * np * sizeof(R) + 1024;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
// dynamic shared memory per CTA that lets two CTAs share an SM (228 KB,
// less 1 KB the runtime keeps per CTA)
constexpr size_t kTwoCtaSmem = 113 * 1024;

template <typename R, int VP, int NP>
size_t smem_bytes(int maxs, int nslot, int scap) {
    const int npv = NP > 0 ? NP : 1;
    size_t b = (size_t)nslot * Slot<VP>::N * 16 + (size_t)XSL * Slot<VP>::PSI_BYTES;
    if (NP > 0) b += (size_t)maxs * npv * VP * 16 + (size_t)XSL * scap;
    return b + 1024;
}

TmaMaps maps_for(Domain& d, const void* base);

template <typename R, int ORDER, int VP, int NP>
void tma_launch(Domain& d, const StageArgs& a, const TmaMaps& m, dim3 grid, bool proj) {
    const TmaState& t = *d.tma;
    const Geo G0 = geo_of(d);
    TGeo<R> G;
    G.kc0 = (R)G0.kc0; G.kc1 = (R)G0.kc1; G.kc2 = (R)G0.kc2; G.gk1 = (R)G0.gk1; G.gk2 = (R)G0.gk2;
    G.nx = d.desc.n[0]; G.ny = d.desc.n[1]; G.nz = d.desc.n[2]; G.ld = d.ld;
    G.ntx = d.desc.n[0] / TX;
    G.zc = t.zc;
    TNl<R> N{};
    if (NP > 0) {
        N.sblk = t.sblk;
        N.sblk_off = t.sblk_off;
        N.scap = t.scap;
        N.col_start = t.col_start;
        N.col_atom = t.col_atom;
        N.Pin = static_cast<const R*>(a.P);
        N.Pout = proj ? static_cast<R*>(a.P_out) : nullptr;
        N.pp_seg = t.pp_seg;
        N.pp_atom_start = t.pp_atom_start;
        N.pp_atom = t.pp_atom;
        N.pp_key = t.pp_key;
        N.pp_beta = static_cast<const R*>(t.pp_beta);
        N.dV = (R)(d.desc.h * d.desc.h * d.desc.h);
        N.maxs = t.maxs;
    }
    const int maxs = NP > 0 ? t.maxs : 0;
    // five w slots (a deeper prefetch) when two CTAs still fit on an SM
    const int scap = NP > 0 ? t.scap : 0;
    const int nslot = smem_bytes<R, VP, NP>(maxs, 5, scap) <= kTwoCtaSmem ? 5 : 4;
    const size_t smem = smem_bytes<R, VP, NP>(maxs, nslot, scap);
    constexpr int TPP_WIDE = VP == 8 ? 8 : 4;       // one 16-byte vector per thread
    const int tpp = t.tpp == 8 ? TPP_WIDE : 4;
    const bool obs = a.obs != nullptr;
    decltype(&k_stage_tma<R, ORDER, VP, NP, 4, 4, false>) kern;
    if (nslot == 5)
        kern = obs ? (tpp == 8 ? k_stage_tma<R, ORDER, VP, NP, 5, TPP_WIDE, true> : k_stage_tma<R, ORDER, VP, NP, 5, 4, true>)
                   : (tpp == 8 ? k_stage_tma<R, ORDER, VP, NP, 5, TPP_WIDE, false> : k_stage_tma<R, ORDER, VP, NP, 5, 4, false>);
    else
        kern = obs ? (tpp == 8 ? k_stage_tma<R, ORDER, VP, NP, 4, TPP_WIDE, true> : k_stage_tma<R, ORDER, VP, NP, 4, 4, true>)
                   : (tpp == 8 ? k_stage_tma<R, ORDER, VP, NP, 4, TPP_WIDE, false> : k_stage_tma<R, ORDER, VP, NP, 4, 4, false>);
    ensure_dynamic_smem(reinterpret_cast<const void*>(kern), smem);
    N.Pout = nullptr;
    {
        ProfScope ps(d.prof, MLMD_KERNEL_STAGE, d.stream);
        const int psi_mode = a.psi == nullptr ? 0 : (a.psi == a.w ? 1 : 2);
        const CUtensorMap tm_p = psi_mode == 2 ? maps_for(d, a.psi).centre : m.centre;
        kern<<<grid, 64 * tpp, smem, d.stream>>>(m.centre, m.xslab, m.yslab, tm_p, psi_mode, G,
                                           static_cast<R*>(a.out), static_cast<const R*>(d.V),
                                           static_cast<const R*>(d.fR), a.A, N, (R)a.gamma_re, (R)a.gamma_im, a.obs,
                                           d.err_flag);
    }
    if constexpr (NP > 0) {
        if (!proj) return;
        N.Pout = static_cast<R*>(a.P_out);
        const TmaMaps mo = maps_for(d, a.out);
        const size_t psm = project_smem<R, VP>(NP, t.pcap, t.pzc);
        const dim3 pgrid(grid.x, grid.y, (G.nz + t.pzc - 1) / t.pzc);
        auto pk = k_nl_project_cols<R, VP, NP>;
        ensure_dynamic_smem(reinterpret_cast<const void*>(pk), psm);
        ProfScope ps(d.prof, MLMD_KERNEL_PROJECT, d.stream);
        pk<<<pgrid, 256, psm, d.stream>>>(mo.centre, N, G.nx, G.ny, G.nz, G.ntx, t.pzc, G.ld, t.pcap, d.err_flag);
        d.launches++;
    }
}

template <typename R, int VP, int NP>
void tma_order(Domain& d, const StageArgs& a, const TmaMaps& m, dim3 grid, bool proj) {
    if (d.desc.fd_order == 4) tma_launch<R, 4, VP, NP>(d, a, m, grid, proj);
    else tma_launch<R, 2, VP, NP>(d, a, m, grid, proj);
}

template <typename R, int VP>
void tma_np(Domain& d, const StageArgs& a, const TmaMaps& m, dim3 grid, bool nl, bool proj) {
    if (!nl) tma_order<R, VP, 0>(d, a, m, grid, false);
    else if (d.nl.n_proj == 4) tma_order<R, VP, 4>(d, a, m, grid, proj);
    else tma_order<R, VP, 8>(d, a, m, grid, proj);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        MLMD_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
        MLMD_REQUIRE(q == cudaDriverEntryPointSuccess && p, MLMD_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
        fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

void encode(CUtensorMap* map, const Domain& d, const void* base, uint32_t bx, uint32_t by) {
    const size_t rs = d.c64() ? sizeof(float) : sizeof(double);
    const cuuint64_t dims[4] = {(cuuint64_t)2 * d.ld, (cuuint64_t)d.desc.n[0], (cuuint64_t)d.desc.n[1],
                                (cuuint64_t)d.desc.n[2]};
    const cuuint64_t row = (cuuint64_t)2 * d.ld * rs;
    const cuuint64_t strides[3] = {row, row * d.desc.n[0], row * d.desc.n[0] * d.desc.n[1]};
    const cuuint32_t box[4] = {(cuuint32_t)(d.tma->vp * 16 / rs), bx, by, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = encode_fn()(map, d.c64() ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4,
                             const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                             d.tma->vp == 8 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    MLMD_REQUIRE(r == CUDA_SUCCESS, MLMD_ERR_CUDA, "cuTensorMapEncodeTiled failed");
}

TmaMaps maps_for(Domain& d, const void* base) {
    for (const auto& m : d.tma->maps)
        if (m.base == base) return m;
    if (d.tma->maps.size() >= 64) d.tma->maps.clear();
    TmaMaps m;
    m.base = base;
    encode(&m.centre, d, base, TX, TY);
    encode(&m.xslab, d, base, 2, TY);
    encode(&m.yslab, d, base, TX, 2);
    d.tma->maps.push_back(m);
    return m;
}

int chunks_of(const Domain& d) { return (int)((size_t)d.ld * d.elem / (d.tma->vp * 16)); }

void set_zc(Domain& d, int zc) {
    TmaState& t = *d.tma;
    t.zc = zc;
    t.ncols = (d.desc.n[0] / TX) * (d.desc.n[1] / TY) * ((d.desc.n[2] + zc - 1) / zc);
}

// Does the stage kernel with projectors keep five w slots at two CTAs per SM
// in one of the chunk widths the tile tuner may pick?
bool five_slots_fit(const Domain& d, int np, int maxs, int scap) {
    if (!d.c64())
        return (np == 4 ? smem_bytes<double, 8, 4>(maxs, 5, scap) : smem_bytes<double, 8, 8>(maxs, 5, scap)) <=
               kTwoCtaSmem;
    const size_t b4 = np == 4 ? smem_bytes<float, 4, 4>(maxs, 5, scap) : smem_bytes<float, 4, 8>(maxs, 5, scap);
    const size_t b8 = np == 4 ? smem_bytes<float, 8, 4>(maxs, 5, scap) : smem_bytes<float, 8, 8>(maxs, 5, scap);
    return b4 <= kTwoCtaSmem || (d.tma->vp == 8 && b8 <= kTwoCtaSmem);
}

}  // namespace

void tma_setup(Domain& d) {
    if (!d.tma) d.tma = new TmaState();
    TmaState& t = *d.tma;
    t.maps.clear();
    const int nx = d.desc.n[0], ny = d.desc.n[1], nz = d.desc.n[2];
    const size_t row_bytes = (size_t)d.ld * d.elem;
    t.vp8_ok = row_bytes % 128 == 0;
    t.vp = t.vp8_ok ? 8 : ((row_bytes % 64 == 0 && d.c64()) ? 4 : 0);
    t.ok = t.vp != 0 && nx % TX == 0 && ny % TY == 0 && std::getenv("MLMD_NO_TMA") == nullptr;
    t.tuned = false;
    if (!t.ok) return;
    // z range per CTA: enough CTAs to fill the GPU, at most kMaxZc planes
    // (longer columns spread each CTA's start-up and its 4-plane z halo over
    // more planes; the projector tables may cut this to 16, see tma_build_nl)
    const int base = (nx / TX) * (ny / TY) * chunks_of(d);
    const int nzch = std::max(1, std::min((608 + base - 1) / base, std::max(1, nz / 4)));
    t.zc_full = std::min((nz + nzch - 1) / nzch, kMaxZc);
    // MLMD_STAGE_ZC (1..32) fixes the planes per column instead (tests and
    // profiles; the projector tables may still cut it to 16)
    if (const char* e = std::getenv("MLMD_STAGE_ZC")) {
        const int v = std::atoi(e);
        if (v >= 1 && v <= kMaxZc) t.zc_full = std::min(v, nz);
    }
    set_zc(d, t.zc_full);
}

void tma_release(Domain& d) {
    delete d.tma;
    d.tma = nullptr;
}

// Per-column tables of the fused nonlocal path, built on the host from the
// device lists (set-up, not on the time-step path).
void tma_build_nl(Domain& d, const double* D_host, int zc_cap) {
    if (!d.tma || !d.tma->ok) return;
    TmaState& t = *d.tma;
    for (void* p : {(void*)t.col_start, (void*)t.col_atom, (void*)t.sblk, (void*)t.sblk_off, (void*)t.pp_seg,
                    (void*)t.pp_atom_start, (void*)t.pp_atom, (void*)t.pp_key, t.pp_beta})
        if (p) d.mem.put(p);
    t.col_start = t.col_atom = t.pp_seg = t.pp_atom_start = t.pp_atom = t.pp_key = nullptr;
    t.sblk = nullptr;
    t.sblk_off = nullptr;
    t.pp_beta = nullptr;
    t.scap = 0;
    t.nl_ok = false;
    t.maxs = 0;
    if (zc_cap == 0) set_zc(d, t.zc_full);
    const Nonlocal& nl = d.nl;
    if (nl.n_atoms == 0 || nl.n_list == 0) return;
    const int nx = d.desc.n[0], ny = d.desc.n[1];
    const int ntx = nx / TX, ntiles = ntx * (ny / TY);
    const int np = nl.n_proj;
    std::vector<int32_t> idx(nl.n_list), pstart_dev(d.ng + 1);
    std::vector<double> beta((size_t)nl.n_list * np);
    MLMD_CUDA(cudaMemcpyAsync(idx.data(), nl.idx, sizeof(int32_t) * nl.n_list, cudaMemcpyDeviceToHost, d.stream));
    MLMD_CUDA(cudaMemcpyAsync(beta.data(), nl.beta64, sizeof(double) * beta.size(), cudaMemcpyDeviceToHost, d.stream));
    MLMD_CUDA(cudaMemcpyAsync(pstart_dev.data(), nl.pstart, sizeof(int32_t) * (d.ng + 1), cudaMemcpyDeviceToHost,
                              d.stream));
    MLMD_CUDA(cudaStreamSynchronize(d.stream));
    auto col_of = [&](int64_t g) {
        const int x = (int)(g % nx), y = (int)((g / nx) % ny), z = (int)(g / ((int64_t)nx * ny));
        return (x / TX + ntx * (y / TY)) + ntiles * (z / t.zc);
    };
    std::vector<std::vector<int32_t>> catoms(t.ncols);
    std::vector<int32_t> last(t.ncols, -1);
    std::vector<int32_t> qslot(nl.n_list);
    std::vector<int32_t> pcount(d.ng, 0);
    for (int a = 0; a < nl.n_atoms; ++a)
        for (int64_t q = nl.h_off[a]; q < nl.h_off[a + 1]; ++q) {
            const int c = col_of(idx[q]);
            if (last[c] != a) { catoms[c].push_back(a); last[c] = a; }
            qslot[q] = (int32_t)catoms[c].size() - 1;
            pcount[idx[q]]++;
        }
    std::vector<int32_t> pstart(d.ng + 1, 0), cur(d.ng, 0);
    for (int64_t g = 0; g < d.ng; ++g) pstart[g + 1] = pstart[g] + pcount[g];
    MLMD_REQUIRE(pstart == pstart_dev, MLMD_ERR_STATE, "per-point projector ranges disagree");
    const size_t rs = d.c64() ? sizeof(float) : sizeof(double);
    std::vector<int32_t> ent_slot(nl.n_list);
    std::vector<unsigned char> ent_beta((size_t)nl.n_list * np * rs);
    for (int a = 0; a < nl.n_atoms; ++a)
        for (int64_t q = nl.h_off[a]; q < nl.h_off[a + 1]; ++q) {
            const int64_t g = idx[q];
            const int64_t e = pstart[g] + cur[g]++;
            ent_slot[e] = qslot[q];
            for (int i = 0; i < np; ++i) {
                const double bd = beta[q * np + i] * D_host[(int64_t)a * np + i];
                if (rs == 4) reinterpret_cast<float*>(ent_beta.data())[e * np + i] = (float)bd;
                else reinterpret_cast<double*>(ent_beta.data())[e * np + i] = bd;
            }
        }
    std::vector<int32_t> col_start(t.ncols + 1, 0), col_atom;
    for (int c = 0; c < t.ncols; ++c) {
        col_start[c + 1] = col_start[c] + (int32_t)catoms[c].size();
        t.maxs = std::max<int>(t.maxs, (int)catoms[c].size());
        col_atom.insert(col_atom.end(), catoms[c].begin(), catoms[c].end());
    }
    // scatter-back blocks, one per (column, plane) in column-major order:
    // header [68] int32 (point offsets 0..64, n, n4, 0), slots [n4], beta * D [n][np]
    std::vector<unsigned char> sblk;
    std::vector<int64_t> sblk_off((size_t)t.ncols * t.zc + 1, 0);
    {
        const int nzch = (d.desc.n[2] + t.zc - 1) / t.zc;
        for (int zc_i = 0; zc_i < nzch; ++zc_i)
            for (int tile = 0; tile < ntiles; ++tile)
                for (int iz = 0; iz < t.zc; ++iz) {
                    const int64_t blk = (int64_t)(tile + ntiles * zc_i) * t.zc + iz;
                    const int z = zc_i * t.zc + iz;
                    const int x0 = (tile % ntx) * TX, y0 = (tile / ntx) * TY;
                    int32_t hdr[68] = {0};
                    std::vector<int32_t> sl;
                    std::vector<unsigned char> bd;
                    if (z < d.desc.n[2])
                        for (int pt = 0; pt < 64; ++pt) {
                            hdr[pt] = (int32_t)sl.size();
                            const int64_t g = (x0 + pt % TX) + (int64_t)nx * (y0 + pt / TX) + (int64_t)nx * ny * z;
                            for (int32_t e = pstart[g]; e < pstart[g + 1]; ++e) {
                                sl.push_back(ent_slot[e]);
                                bd.insert(bd.end(), ent_beta.begin() + (size_t)e * np * rs,
                                          ent_beta.begin() + (size_t)(e + 1) * np * rs);
                            }
                        }
                    const int n = (int)sl.size(), n4 = (n + 3) / 4 * 4;
                    for (int pt = (z < d.desc.n[2] ? 64 : 0); pt <= 64; ++pt) hdr[pt] = n;
                    hdr[65] = n;
                    hdr[66] = n4;
                    sl.resize(n4, 0);
                    bd.resize((bd.size() + 15) / 16 * 16, 0);
                    sblk_off[blk] = (int64_t)sblk.size();
                    const unsigned char* hp = reinterpret_cast<const unsigned char*>(hdr);
                    sblk.insert(sblk.end(), hp, hp + sizeof(hdr));
                    const unsigned char* sp = reinterpret_cast<const unsigned char*>(sl.data());
                    sblk.insert(sblk.end(), sp, sp + sl.size() * sizeof(int32_t));
                    sblk.insert(sblk.end(), bd.begin(), bd.end());
                    t.scap = std::max<int>(t.scap, (int)(sblk.size() - sblk_off[blk]));
                }
        sblk_off[(size_t)t.ncols * t.zc] = (int64_t)sblk.size();
    }
    // long columns gather more atoms: where their staged projections would
    // cost the fifth w slot, build the tables again for 16-plane columns
    if (t.zc > 16 && !five_slots_fit(d, np, t.maxs, t.scap)) {
        set_zc(d, 16);
        tma_build_nl(d, D_host, 16);
        return;
    }
    // projection tables: projection columns of pzc planes, entries ordered by
    // (slot, plane, point); slots number a column's atoms in ascending order
    // MLMD_PROJ_PLANES (1..16) overrides the 4 planes per projection column
    // (profiling)
    int pz = 4;
    if (const char* e = std::getenv("MLMD_PROJ_PLANES")) {
        const int v = std::atoi(e);
        if (v >= 1 && v <= 16) pz = v;
    }
    t.pzc = std::min(pz, t.zc);
    const int nzp = (d.desc.n[2] + t.pzc - 1) / t.pzc;
    const int64_t ncp = (int64_t)ntiles * nzp;
    auto pcol_of = [&](int64_t g) {
        const int x = (int)(g % nx), y = (int)((g / nx) % ny), z = (int)(g / ((int64_t)nx * ny));
        return (int64_t)(x / TX + ntx * (y / TY)) + ntiles * (z / t.pzc);
    };
    std::vector<std::vector<int32_t>> patoms(ncp);
    std::vector<int32_t> plast(ncp, -1), pslot(nl.n_list);
    for (int a = 0; a < nl.n_atoms; ++a)
        for (int64_t q = nl.h_off[a]; q < nl.h_off[a + 1]; ++q) {
            const int64_t c = pcol_of(idx[q]);
            if (plast[c] != a) { patoms[c].push_back(a); plast[c] = a; }
            pslot[q] = (int32_t)patoms[c].size() - 1;
        }
    // atoms are visited in ascending order and each atom's points in ascending
    // grid order, so counting by (column, slot, plane) gives the wanted order
    std::vector<int32_t> pp_atom_start(ncp + 1, 0), pp_atom;
    for (int64_t c = 0; c < ncp; ++c) {
        pp_atom_start[c + 1] = pp_atom_start[c] + (int32_t)patoms[c].size();
        pp_atom.insert(pp_atom.end(), patoms[c].begin(), patoms[c].end());
    }
    auto pkey_of = [&](int64_t q) {     // (column, slot, plane) bucket
        const int64_t g = idx[q];
        const int z = (int)(g / ((int64_t)nx * ny));
        return ((int64_t)pp_atom_start[pcol_of(g)] + pslot[q]) * t.pzc + (z % t.pzc);
    };
    const int64_t nbk = (int64_t)pp_atom_start[ncp] * t.pzc;
    std::vector<int32_t> bcnt(nbk + 1, 0);
    for (int64_t q = 0; q < nl.n_list; ++q) bcnt[pkey_of(q) + 1]++;
    for (int64_t k = 0; k < nbk; ++k) bcnt[k + 1] += bcnt[k];
    const int64_t nslots = pp_atom_start[ncp];
    std::vector<int32_t> pp_seg(nslots + 1, 0);
    for (int64_t k = 0; k <= nslots; ++k) pp_seg[k] = bcnt[k * t.pzc];
    std::vector<int32_t> pp_key(nl.n_list + 8, 0);
    std::vector<unsigned char> pp_beta((size_t)nl.n_list * np * rs);
    for (int a = 0; a < nl.n_atoms; ++a)
        for (int64_t q = nl.h_off[a]; q < nl.h_off[a + 1]; ++q) {
            const int64_t g = idx[q];
            const int64_t e = bcnt[pkey_of(q)]++;
            const int z = (int)(g / ((int64_t)nx * ny));
            pp_key[e] = (int32_t)((((g / nx) % ny) % TY) * TX + (g % nx) % TX) + (z % t.pzc) * 64;
            for (int i = 0; i < np; ++i) {
                if (rs == 4) reinterpret_cast<float*>(pp_beta.data())[e * np + i] = (float)beta[q * np + i];
                else reinterpret_cast<double*>(pp_beta.data())[e * np + i] = beta[q * np + i];
            }
        }
    int pcap = 0;
    for (int64_t c = 0; c < ncp; ++c) pcap = std::max(pcap, pp_seg[pp_atom_start[c + 1]] - pp_seg[pp_atom_start[c]]);
    t.pcap = (pcap + 3) / 4 * 4;
    size_t sm8 = 0, sm4 = 0;
    if (d.c64()) {
        sm8 = std::max(np == 4 ? smem_bytes<float, 8, 4>(t.maxs, 4, t.scap) : smem_bytes<float, 8, 8>(t.maxs, 4, t.scap),
                       project_smem<float, 8>(np, t.pcap, t.pzc));
        sm4 = std::max(np == 4 ? smem_bytes<float, 4, 4>(t.maxs, 4, t.scap) : smem_bytes<float, 4, 8>(t.maxs, 4, t.scap),
                       project_smem<float, 4>(np, t.pcap, t.pzc));
    } else {
        sm8 = sm4 = std::max(np == 4 ? smem_bytes<double, 8, 4>(t.maxs, 4, t.scap) : smem_bytes<double, 8, 8>(t.maxs, 4, t.scap),
                             project_smem<double, 8>(np, t.pcap, t.pzc));
    }
    const size_t kMaxSmem = 200 * 1024;
    if (sm4 > kMaxSmem) return;   // too many atoms per column for the staging: plain kernel
    if (t.vp == 8 && (sm8 > kMaxSmem || !d.c64())) {
        if (!d.c64()) return;
        t.vp = 4;                 // only the narrower chunks fit
        t.vp8_ok = false;
        t.maps.clear();
    }
    t.col_start = (int32_t*)d.mem.get(sizeof(int32_t) * col_start.size());
    t.col_atom = (int32_t*)d.mem.get(sizeof(int32_t) * std::max<size_t>(col_atom.size(), 1));
    MLMD_CUDA(cudaMemcpyAsync(t.col_start, col_start.data(), sizeof(int32_t) * col_start.size(), cudaMemcpyHostToDevice, d.stream));
    if (!col_atom.empty())
        MLMD_CUDA(cudaMemcpyAsync(t.col_atom, col_atom.data(), sizeof(int32_t) * col_atom.size(), cudaMemcpyHostToDevice, d.stream));
    auto upload = [&](const void* src, size_t bytes) {
        void* p = d.mem.get(std::max<size_t>(bytes, 16));
        if (bytes) MLMD_CUDA(cudaMemcpyAsync(p, src, bytes, cudaMemcpyHostToDevice, d.stream));
        return p;
    };
    t.pp_seg = (int32_t*)upload(pp_seg.data(), sizeof(int32_t) * pp_seg.size());
    t.pp_atom_start = (int32_t*)upload(pp_atom_start.data(), sizeof(int32_t) * pp_atom_start.size());
    t.pp_atom = (int32_t*)upload(pp_atom.data(), sizeof(int32_t) * pp_atom.size());
    t.pp_key = (int32_t*)upload(pp_key.data(), sizeof(int32_t) * pp_key.size());
    t.pp_beta = upload(pp_beta.data(), pp_beta.size());
    t.sblk = (unsigned char*)upload(sblk.data(), sblk.size());
    t.sblk_off = (int64_t*)upload(sblk_off.data(), sizeof(int64_t) * sblk_off.size());
    MLMD_CUDA(cudaStreamSynchronize(d.stream));
    t.nl_ok = true;
}

bool tma_fused_nl(const Domain& d) {
    return d.tma && d.tma->ok && d.has_nl() && d.tma->nl_ok && !gauge_on(d);
}

int tma_blocks(const Domain& d) {
    if (!d.tma || !d.tma->ok) return 0;
    return (d.desc.n[0] / TX) * (d.desc.n[1] / TY) * chunks_of(d) * ((d.desc.n[2] + d.tma->zc - 1) / d.tma->zc);
}

bool launch_stage_tma(Domain& d, const StageArgs& a, bool* proj_done) {
    if (proj_done) *proj_done = false;
    if (!d.tma || !d.tma->ok) return false;
    const bool nl = d.has_nl() && a.P != nullptr;
    // the fused scatter holds real projector tables: velocity-gauge
    // projectors take the per-point kernel
    if (nl && (!d.tma->nl_ok || gauge_on(d))) return false;
    const bool proj = nl && a.P_out != nullptr;
    const TmaState& t = *d.tma;
    const TmaMaps m = maps_for(d, a.w);
    dim3 grid(chunks_of(d), (d.desc.n[0] / TX) * (d.desc.n[1] / TY), (d.desc.n[2] + t.zc - 1) / t.zc);
    if (proj)
        MLMD_CUDA(cudaMemsetAsync(a.P_out, 0, (size_t)d.nl.n_atoms * d.nl.n_proj * d.ld * d.elem, d.stream));
    if (d.c64()) {
        if (t.vp == 8) tma_np<float, 8>(d, a, m, grid, nl, proj);
        else tma_np<float, 4>(d, a, m, grid, nl, proj);
    } else {
        tma_np<double, 8>(d, a, m, grid, nl, proj);
    }
    d.launches++;
    MLMD_CUDA(cudaGetLastError());
    if (proj_done) *proj_done = proj;
    return true;
}

// Pick the tile shape of the TMA stage kernel -- orbital-chunk width (128- or
// 64-byte rows per CTA) and threads per grid point (4, or 8 with 128-byte
// chunks) -- by timing a few launches of each on the domain's own buffers.
// The timed launches read psi and the work buffer wa (as the later stages of
// a step do) and write only the work buffer wb and the projection buffer Pb,
// which every step overwrites before reading.
void tma_autotune(Domain& d, const double* Ak) {
    if (!d.tma || !d.tma->ok || d.tma->tuned) return;
    TmaState& t = *d.tma;
    t.tuned = true;
    // full-scheme steps without projectors run as one sweep (k_sweep.cu)
    if (d.sweep.ok && d.sweep.use == 1 && !d.has_nl() && d.desc.scheme == MLMD_SCHEME_FULL) return;
    // tensor-core nonlocal domains run the stage kernel for the local part only
    const bool nl = d.has_nl() && !nltc_on(d);
    if (nl && (!t.nl_ok || gauge_on(d))) return;
    // MLMD_STAGE_TILE="vp,tpp" (e.g. "8,4") fixes the shape instead, for
    // reproducible profiles; ignored unless it names a valid shape here
    if (const char* fix = std::getenv("MLMD_STAGE_TILE")) {
        int vp = 0, tpp = 0;
        if (std::sscanf(fix, "%d,%d", &vp, &tpp) == 2 && (tpp == 4 || (tpp == 8 && vp == 8)) &&
            ((vp == 8 && t.vp == 8) || (vp == 4 && d.c64() && (t.vp == 4 || t.vp8_ok)))) {
            t.vp = vp;
            t.tpp = tpp;
            t.maps.clear();
            return;
        }
    }
    std::vector<std::pair<int, int>> cand;
    if (t.vp == 8) {
        cand.push_back({8, 4});
        cand.push_back({8, 8});
    }
    if (d.c64() && (t.vp == 4 || t.vp8_ok)) cand.push_back({4, 4});
    if (cand.size() < 2) return;
    StageArgs a;
    a.w = d.wa;
    a.psi = d.psi;
    a.out = d.wb;
    a.P = nl ? d.Pa : nullptr;
    a.P_out = nl ? d.Pb : nullptr;
    a.A = Ak;
    a.gamma_re = 0.0;
    a.gamma_im = -d.desc.dt;
    cudaEvent_t e0, e1;
    MLMD_CUDA(cudaEventCreate(&e0));
    MLMD_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    std::pair<int, int> pick = cand[0];
    for (const auto& c : cand) {
        t.vp = c.first;
        t.tpp = c.second;
        t.maps.clear();
        launch_stage_tma(d, a, nullptr);      // warm-up (also sets the kernel attribute)
        MLMD_CUDA(cudaEventRecord(e0, d.stream));
        for (int r = 0; r < 3; ++r) launch_stage_tma(d, a, nullptr);
        MLMD_CUDA(cudaEventRecord(e1, d.stream));
        MLMD_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        MLMD_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best) { best = ms; pick = c; }
    }
    (void)cudaEventDestroy(e0);
    (void)cudaEventDestroy(e1);
    t.vp = pick.first;
    t.tpp = pick.second;
    t.maps.clear();
}

int tma_chunk_bytes(const Domain& d) { return d.tma && d.tma->ok ? d.tma->vp * 16 : 0; }

}  // namespace mlmd
