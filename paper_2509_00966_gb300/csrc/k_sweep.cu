// One-sweep local Taylor-4: psi <- sum_{j=0..4} (-i dt)^j / j! h_loc^j psi
// (Eq. 2's exp(-i dt h_loc / hbar) to fourth order, h_loc of Eq. 3 with the
// finite-difference stencils) in a single pass over HBM: psi is read once
// and written once (16 B per orbital-gridpoint for complex64), against 88 B
// for four staged passes.  Used when the step has no nonlocal term (no
// projectors) and for the local factor of the split scheme.
//
// Decomposition.  A thread-block cluster of CX x CY CTAs covers a whole x-y
// plane of the domain for one chunk of VPC orbitals (VPC x 8 or x 16 bytes
// per grid point, so global accesses stay in whole 32-byte sectors); each CTA
// owns a TX x TY tile of every plane and streams z.  One thread owns one
// (grid point, orbital) of the tile for the whole sweep.
//
// Pipeline.  With stencil radius r = order / 2, u_0 = psi and
// u_j = h u_{j-1}, step t of the sweep loads psi on plane t and evaluates
// stage j on plane p_j(t) = t - j (r + 1): stage j+1 then reads only planes of
// u_j that were finished at step t-1, so each step needs one cluster barrier.
// The z neighbours of a thread's own point are its own earlier results and
// stay in a register window of 2r+1 planes per u_j; the x-y neighbours of the
// plane each stage reads are published once per step in shared memory (double
// buffered) and read across CTA boundaries through distributed shared memory
// (mapa + ld.shared::cluster).  The Taylor sum
// psi + c1 u1 + c2 u2 + c3 u3 + c4 u4 accumulates per plane in a shared-
// memory ring of 3(r+1) planes; stage 4 writes the finished plane back in
// place.  Planes 0..4r-1 of psi are read again at the end of the periodic
// sweep, after their outputs were written, so their original values are kept
// in shared memory.
#include <algorithm>
#include <cstdlib>

#include "mlmd_internal.cuh"

namespace mlmd {
namespace {

template <typename R> struct C2T;
template <> struct C2T<float> { using T = float2; };
template <> struct C2T<double> { using T = double2; };

// Threads per CTA at most, by working type and stencil order (bounded by the
// register windows: 4 (2r+1) + scratch complex values per thread).
template <typename R, int ORDER> constexpr int sweep_max_threads() {
    return sizeof(R) == 4 ? (ORDER == 4 ? 576 : 768) : (ORDER == 4 ? 384 : 512);
}

struct SweepArgs {
    int nx, ny, nz, ld;
    int TX, TY, CX, VPC;
    int t_begin, t_end;                 // steps [t_begin, t_end), t_begin a multiple of 2r+1
    double kc0, kc1, kc2, gk1, gk2;     // stencil weights (h_loc of Eq. 3)
    double cre[5], cim[5];              // Taylor coefficients c_j = (-i dt)^j / j!
};

// The same weights in the working type, read by the kernel straight from its
// parameter space (constant-bank operands, no registers).
template <typename R> struct SweepCoef {
    R kc0, kc1, kc2, gk1, gk2;
    R cre[5], cim[5];
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint32_t cluster_map(uint32_t addr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_arrive() {
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Neighbour loads from the published planes (kept between the cluster
// barriers; the loads of one batch are issued back to back).
__device__ __forceinline__ float2 ld_cluster(uint32_t a, float2) {
    float2 v;
    asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ double2 ld_cluster(uint32_t a, double2) {
    double2 v;
    asm volatile("ld.shared::cluster.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ float2 ld_local(uint32_t a, float2) {
    float2 v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ double2 ld_local(uint32_t a, double2) {
    double2 v;
    asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "r"(a) : "memory");
    return v;
}

// Complex helpers: (re, im) pairs; complex64 runs on packed f32x2 FMAs.
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return double2{a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return double2{a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ double2 smul(double k, double2 a) { return double2{k * a.x, k * a.y}; }
__device__ __forceinline__ double2 sfma(double k, double2 b, double2 a) { return double2{a.x + k * b.x, a.y + k * b.y}; }
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return __ffma2_rn(make_float2(-1.f, -1.f), b, a); }
__device__ __forceinline__ float2 smul(float k, float2 a) { return __fmul2_rn(make_float2(k, k), a); }
__device__ __forceinline__ float2 sfma(float k, float2 b, float2 a) { return __ffma2_rn(make_float2(k, k), b, a); }
// a + c b for complex c = (cr, ci)
__device__ __forceinline__ double2 cfma(double cr, double ci, double2 b, double2 a) {
    return double2{a.x + cr * b.x - ci * b.y, a.y + cr * b.y + ci * b.x};
}
__device__ __forceinline__ float2 cfma(float cr, float ci, float2 b, float2 a) {
    return __ffma2_rn(make_float2(cr, cr), b, __ffma2_rn(make_float2(-ci, ci), make_float2(b.y, b.x), a));
}
// a - i b
__device__ __forceinline__ double2 sub_ib(double2 a, double2 b) { return double2{a.x + b.y, a.y - b.x}; }
__device__ __forceinline__ float2 sub_ib(float2 a, float2 b) {
    return __ffma2_rn(make_float2(1.f, -1.f), make_float2(b.y, b.x), a);
}

constexpr int pmod(int a, int n) { return ((a % n) + n) % n; }

// Per-thread state of the sweep.
template <typename R, int ORDER, bool OBS>
struct Sweep {
    static constexpr int r = ORDER / 2;
    static constexpr int NW = 2 * r + 1;     // register window per u_j
    static constexpr int NA = 3 * (r + 1);   // accumulator ring (planes)
    using T = typename C2T<R>::T;

    const SweepArgs& A;
    const SweepCoef<R>& K;
    R* psi;
    const R* V;
    T* sp;        // [2][4][PE] published planes
    T* sacc;      // [NA][PE]
    T* ssave;     // [4r][PE]
    int PE, tid;
    int gx, gy, orb;
    int64_t vbase, pstride, qbase, qstride;   // V and psi offsets of this thread's point, plane strides
    uint32_t nb[4 * r];   // neighbour addresses (buffer 0, array 0); bit 0 set = remote (cluster address)
    R A0, A1, A2, half_a2;
    T W[4][NW];
    double obs[5];
    R fo;

    // plane p wrapped into [0, nz) (every plane the sweep touches lies in
    // [-nz, 2 nz))
    __device__ __forceinline__ int wrapz(int p) const {
        return p < 0 ? p + A.nz : (p >= A.nz ? p - A.nz : p);
    }
    __device__ __forceinline__ int64_t gidx(int p) const { return qbase + (int64_t)wrapz(p) * qstride; }
    __device__ __forceinline__ T load_psi(int t) const {
        const T* q = reinterpret_cast<const T*>(psi) + gidx(t);
        return *q;
    }

    __device__ __forceinline__ T nbr(int k, uint32_t off) const {
        const uint32_t a = nb[k];
        if (a & 1u) return ld_cluster((a & ~1u) + off, T{});
        return ld_local(a + off, T{});
    }

    // The part of h u_WA on plane p that needs no neighbour of another
    // thread: centre, z neighbours (register window; S0 = slot of plane p),
    // diagonal.
    struct Part { T ctr, lap, gz; R diag; };
    template <int WA, int S0>
    __device__ __forceinline__ Part zpart(R v) const {
        Part z;
        z.ctr = W[WA][S0];
        const T zp1 = W[WA][pmod(S0 + 1, NW)], zm1 = W[WA][pmod(S0 - 1, NW)];
        z.lap = sfma(K.kc1, cadd(zp1, zm1), smul(K.kc0, z.ctr));
        z.gz = smul(K.gk1, csub(zp1, zm1));
        if constexpr (ORDER == 4) {
            const T zp2 = W[WA][pmod(S0 + 2, NW)], zm2 = W[WA][pmod(S0 - 2, NW)];
            z.lap = sfma(K.kc2, cadd(zp2, zm2), z.lap);
            z.gz = sfma(K.gk2, csub(zp2, zm2), z.gz);
        }
        z.diag = v + half_a2;
        return z;
    }
    // x-y neighbours of array WA in buffer b: +x, -x, +y, -y (then at distance 2)
    __device__ __forceinline__ void load_xy(int WA, int b, T (&v)[4 * r]) const {
        const uint32_t off = (uint32_t)((b * 4 + WA) * PE) * (uint32_t)sizeof(T);
#pragma unroll
        for (int k = 0; k < 4 * r; ++k) v[k] = nbr(k, off);
    }
    // h u = lap + diag u - i A . grad u
    __device__ __forceinline__ T finish(const Part& z, const T (&v)[4 * r], T* grad_out) const {
        T lap = sfma(K.kc1, cadd(cadd(v[0], v[1]), cadd(v[2], v[3])), z.lap);
        T gx = smul(K.gk1, csub(v[0], v[1])), gy = smul(K.gk1, csub(v[2], v[3]));
        if constexpr (ORDER == 4) {
            lap = sfma(K.kc2, cadd(cadd(v[4], v[5]), cadd(v[6], v[7])), lap);
            gx = sfma(K.gk2, csub(v[4], v[5]), gx);
            gy = sfma(K.gk2, csub(v[6], v[7]), gy);
        }
        const T ag = sfma(A0, gx, sfma(A1, gy, smul(A2, z.gz)));
        if (grad_out) { grad_out[0] = gx; grad_out[1] = gy; grad_out[2] = z.gz; }
        return sub_ib(sfma(z.diag, z.ctr, lap), ag);
    }

    // a + c_j h
    __device__ __forceinline__ T add_term(int j, T h, T a) const { return cfma(K.cre[j], K.cim[j], h, a); }
    __device__ __forceinline__ int64_t vidx(int p) const { return vbase + (int64_t)wrapz(p) * pstride; }

    // One step of the pipeline at t = base + U (base a multiple of NW).
    template <int U>
    __device__ __forceinline__ void step(int t, T& pending) {
        constexpr int S1 = pmod(U - (r + 1), NW), S2 = pmod(U - 2 * (r + 1), NW);
        constexpr int S3 = pmod(U - 3 * (r + 1), NW), S4 = pmod(U - 4 * (r + 1), NW);
        const int b = t & 1;
        const int nz = A.nz;
        const int p1 = t - (r + 1), p2 = t - 2 * (r + 1), p3 = t - 3 * (r + 1), p4 = t - 4 * (r + 1);
        const bool a1 = p1 >= -3 * r && p1 < nz + 3 * r, a2 = p2 >= -2 * r && p2 < nz + 2 * r;
        const bool a3 = p3 >= -r && p3 < nz + r, a4 = p4 >= 0 && p4 < nz;
        const R v1 = a1 ? __ldg(V + vidx(p1)) : (R)0, v2 = a2 ? __ldg(V + vidx(p2)) : (R)0;
        const R v3 = a3 ? __ldg(V + vidx(p3)) : (R)0, v4 = a4 ? __ldg(V + vidx(p4)) : (R)0;
        // publish the centre planes the four stages read this step: u_j on
        // plane p_{j+1}(t), the middle of u_j's window
        sp[(b * 4 + 0) * PE + tid] = W[0][S1];
        sp[(b * 4 + 1) * PE + tid] = W[1][S2];
        sp[(b * 4 + 2) * PE + tid] = W[2][S3];
        sp[(b * 4 + 3) * PE + tid] = W[3][S4];
        cluster_arrive();
        const T ps1 = W[0][S1];
        cluster_wait();
        // stages in descending order (stage j+1 reads u_j's window before
        // stage j writes it), neighbour loads two stages at a time
        T x[2][4 * r];
        if (a4) load_xy(3, b, x[0]);
        if (a4) {   // stage 4: plane p4 in [0, nz) -> output
            const T h = finish(zpart<3, S4>(v4), x[0], nullptr);
            const T o = add_term(4, h, sacc[(p4 % NA) * PE + tid]);
            reinterpret_cast<T*>(psi)[gidx(p4)] = o;
        }
        if (a3) load_xy(2, b, x[1]);
        if (a3) {   // stage 3: planes [-r, nz + r)
            const T h = finish(zpart<2, S3>(v3), x[1], nullptr);
            W[3][S3] = h;
            if (p3 >= 0 && p3 < nz) {
                T* acc = sacc + (p3 % NA) * PE + tid;
                *acc = add_term(3, h, *acc);
            }
        }
        if (a2) load_xy(1, b, x[0]);
        if (a2) {   // stage 2: planes [-2r, nz + 2r)
            const T h = finish(zpart<1, S2>(v2), x[0], nullptr);
            W[2][S2] = h;
            if (p2 >= 0 && p2 < nz) {
                T* acc = sacc + (p2 % NA) * PE + tid;
                *acc = add_term(2, h, *acc);
            }
        }
        if (a1) load_xy(0, b, x[1]);
        if (a1) {   // stage 1: planes [-3r, nz + 3r); observables of psi on [0, nz)
            const bool own = p1 >= 0 && p1 < nz;
            T g[3];
            const T h = finish(zpart<0, S1>(v1), x[1], (OBS && own) ? g : nullptr);
            W[1][S1] = h;
            if (own) {
                sacc[(p1 % NA) * PE + tid] = add_term(1, h, ps1);
                if constexpr (OBS) {
                    obs[0] += (double)(fo * (ps1.x * ps1.x + ps1.y * ps1.y));
                    obs[1] += (double)(fo * (ps1.x * h.x + ps1.y * h.y));
#pragma unroll
                    for (int ax = 0; ax < 3; ++ax) obs[2 + ax] += (double)(fo * (ps1.x * g[ax].y - ps1.y * g[ax].x));
                }
            }
        }
        // psi on plane t joins the window; plane t+1 is requested now
        if (t >= -4 * r && t < nz + 4 * r) {
            W[0][U] = pending;
            if (t >= 0 && t < 4 * r) ssave[t * PE + tid] = pending;
        }
        const int tn = t + 1;
        if (tn >= -4 * r && tn < nz + 4 * r) pending = (tn >= nz) ? ssave[(tn - nz) * PE + tid] : load_psi(tn);
    }
};

template <typename R, int ORDER, bool OBS>
__global__ void __launch_bounds__(sweep_max_threads<R, ORDER>(), 1)
k_t4_sweep(const SweepArgs A, const SweepCoef<R> K, R* psi, const R* __restrict__ V, const double* __restrict__ Ak,
           const R* __restrict__ f, double* __restrict__ obs_part) {
    using S = Sweep<R, ORDER, OBS>;
    using T = typename S::T;
    constexpr int r = S::r;
    constexpr int NW = S::NW;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int PE = blockDim.x;
    S s{A, K, psi, V};
    s.PE = PE;
    s.tid = threadIdx.x;
    s.sp = reinterpret_cast<T*>(smem_raw);
    s.sacc = s.sp + 8 * PE;
    s.ssave = s.sacc + S::NA * PE;
    const int ol = threadIdx.x % A.VPC, pt = threadIdx.x / A.VPC;
    const int xl = pt % A.TX, yl = pt / A.TX;
    const int cx = blockIdx.x, cy = blockIdx.y;
    const int CY = gridDim.y;
    s.gx = cx * A.TX + xl;
    s.gy = cy * A.TY + yl;
    s.orb = blockIdx.z * A.VPC + ol;
    s.pstride = (int64_t)A.nx * A.ny;
    s.vbase = (int64_t)s.gx + (int64_t)A.nx * s.gy;
    s.qstride = s.pstride * A.ld;
    s.qbase = s.vbase * A.ld + s.orb;
    s.A0 = (R)Ak[0]; s.A1 = (R)Ak[1]; s.A2 = (R)Ak[2];
    s.half_a2 = (R)(0.5 * (Ak[0] * Ak[0] + Ak[1] * Ak[1] + Ak[2] * Ak[2]));
    s.fo = OBS ? f[s.orb] : (R)0;
#pragma unroll
    for (int k = 0; k < 5; ++k) s.obs[k] = 0.0;
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int w = 0; w < NW; ++w) s.W[j][w] = T{0, 0};
    // in-plane neighbours: +-1 along x and y (then +-2), each in this CTA's
    // tile or in the neighbouring CTA's (periodic across the cluster)
    {
        const uint32_t base = smem_u32(s.sp);
        uint32_t my_rank;
        asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(my_rank));
#pragma unroll
        for (int k = 0; k < 4 * r; ++k) {
            const int dist = k / 4 + 1;
            const int kind = k % 4;          // 0: +x, 1: -x, 2: +y, 3: -y
            int nxl = xl, nyl = yl, ncx = cx, ncy = cy;
            if (kind == 0) nxl += dist; else if (kind == 1) nxl -= dist; else if (kind == 2) nyl += dist; else nyl -= dist;
            if (nxl >= A.TX) { nxl -= A.TX; ncx = (cx + 1) % A.CX; }
            if (nxl < 0) { nxl += A.TX; ncx = (cx + A.CX - 1) % A.CX; }
            if (nyl >= A.TY) { nyl -= A.TY; ncy = (cy + 1) % CY; }
            if (nyl < 0) { nyl += A.TY; ncy = (cy + CY - 1) % CY; }
            const uint32_t e = base + (uint32_t)(((nyl * A.TX + nxl) * A.VPC + ol) * (int)sizeof(T));
            const uint32_t rank = (uint32_t)(ncx + ncy * A.CX);
            s.nb[k] = rank == my_rank ? e : (cluster_map(e, rank) | 1u);
        }
    }
    T pending = T{0, 0};
    if (A.t_begin >= -4 * r) pending = s.load_psi(A.t_begin);
    for (int t = A.t_begin; t < A.t_end; t += NW) {
        s.template step<0>(t, pending);
        if (t + 1 < A.t_end) s.template step<1 % NW>(t + 1, pending);
        if (t + 2 < A.t_end) s.template step<2 % NW>(t + 2, pending);
        if constexpr (NW > 3) {
            if (t + 3 < A.t_end) s.template step<3 % NW>(t + 3, pending);
            if (t + 4 < A.t_end) s.template step<4 % NW>(t + 4, pending);
        }
    }
    // no CTA leaves while a neighbour may still read its shared memory
    cluster_sync_all();
    if constexpr (OBS) {
        __shared__ double red[32][5];
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            double v = s.obs[k];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) red[warp][k] = v;
        }
        __syncthreads();
        if (warp == 0) {
            const int nw = (blockDim.x + 31) >> 5;
            const int64_t blin = blockIdx.x + (int64_t)gridDim.x * (blockIdx.y + (int64_t)gridDim.y * blockIdx.z);
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                double v = lane < nw ? red[lane][k] : 0.0;
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 0) obs_part[blin * 5 + k] = v;
            }
        }
    }
}

template <typename R, int ORDER, bool OBS>
const void* sweep_kernel() {
    return reinterpret_cast<const void*>(&k_t4_sweep<R, ORDER, OBS>);
}

const void* sweep_kernel_for(const Domain& d, bool obs) {
    if (d.c64()) {
        if (d.desc.fd_order == 4) return obs ? sweep_kernel<float, 4, true>() : sweep_kernel<float, 4, false>();
        return obs ? sweep_kernel<float, 2, true>() : sweep_kernel<float, 2, false>();
    }
    if (d.desc.fd_order == 4) return obs ? sweep_kernel<double, 4, true>() : sweep_kernel<double, 4, false>();
    return obs ? sweep_kernel<double, 2, true>() : sweep_kernel<double, 2, false>();
}

int max_threads_for(const Domain& d) {
    if (d.c64()) return d.desc.fd_order == 4 ? sweep_max_threads<float, 4>() : sweep_max_threads<float, 2>();
    return d.desc.fd_order == 4 ? sweep_max_threads<double, 4>() : sweep_max_threads<double, 2>();
}

size_t sweep_smem(int r, int threads, size_t tsz) {
    return (size_t)(8 + 3 * (r + 1) + 4 * r) * threads * tsz;
}

}  // namespace

// Choose the cluster tiling of one domain (or none): enough CTAs to fill the
// GPU first (up to 152), then the widest orbital chunk (whole 32-byte sectors),
// then the smallest cluster, then the fewest CTAs along x.
SweepPlan plan_sweep(const Domain& d) {
    SweepPlan best;
    const int nx = d.desc.n[0], ny = d.desc.n[1], nz = d.desc.n[2];
    const int r = d.desc.fd_order / 2;
    if (nz < 4 * (r + 1)) return best;
    const size_t tsz = d.c64() ? 8 : 16;
    const int maxt = max_threads_for(d);
    const int vpcs[2] = {d.c64() ? 4 : 2, d.c64() ? 2 : 1};
    long best_key[4] = {-1, 0, 0, 0};
    for (int vpc : vpcs) {
        if (d.ld % vpc) continue;
        for (int cs = 1; cs <= 16; ++cs)
            for (int cx = 1; cx <= cs; ++cx) {
                if (cs % cx) continue;
                const int cy = cs / cx;
                if (nx % cx || ny % cy) continue;
                const int tx = nx / cx, ty = ny / cy;
                if (tx < r || ty < r) continue;
                const int threads = tx * ty * vpc;
                if (threads > maxt || threads % 32) continue;
                const size_t smem = sweep_smem(r, threads, tsz);
                if (smem > 220 * 1024) continue;
                const long ctas = (long)cs * (d.ld / vpc);
                const long key[4] = {std::min<long>(ctas, 152), vpc, -cs, -cx};
                bool better = false;
                for (int k = 0; k < 4; ++k)
                    if (key[k] != best_key[k]) { better = key[k] > best_key[k]; break; }
                if (!better) continue;
                for (int k = 0; k < 4; ++k) best_key[k] = key[k];
                best.ok = true;
                best.CX = cx; best.CY = cy; best.TX = tx; best.TY = ty; best.VPC = vpc;
                best.threads = threads;
                best.smem = smem;
            }
    }
    return best;
}

namespace {

cudaLaunchConfig_t sweep_config(const Domain& d, const SweepPlan& P, cudaLaunchAttribute* attr) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)P.CX, (unsigned)P.CY, (unsigned)(d.ld / P.VPC));
    cfg.blockDim = dim3((unsigned)P.threads, 1, 1);
    cfg.dynamicSmemBytes = P.smem;
    cfg.stream = d.stream;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)P.CX;
    attr[0].val.clusterDim.y = (unsigned)P.CY;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

void prepare_kernel(const void* k, const SweepPlan& P) {
    ensure_dynamic_smem(k, P.smem);
    if (P.CX * P.CY > 8) MLMD_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
}

}  // namespace

// Plan, prepare both kernel variants and confirm that one cluster of the plan
// fits on the device; the plan is dropped otherwise.  MLMD_SWEEP=0 drops it,
// MLMD_SWEEP=1 uses it whenever it exists; by default the first propagate
// times it against the staged passes (sweep_autotune) and keeps the faster.
void sweep_setup(Domain& d) {
    d.sweep = SweepPlan{};
    const char* e = std::getenv("MLMD_SWEEP");
    if (e && e[0] == '0') return;
    SweepPlan P = plan_sweep(d);
    if (!P.ok) return;
    cudaLaunchAttribute attr[1];
    for (bool obs : {false, true}) {
        const void* k = sweep_kernel_for(d, obs);
        prepare_kernel(k, P);
        cudaLaunchConfig_t cfg = sweep_config(d, P, attr);
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, k, &cfg) != cudaSuccess || n < 1) {
            (void)cudaGetLastError();
            return;
        }
    }
    P.use = (e && e[0] == '1') ? 1 : 0;
    d.sweep = P;
}

// buf <- T4(h_loc(A)) buf in place (buf: psi or a work copy); obs (per-CTA
// partials of the observables, as the stage kernel's) when obs_part is set.
// Returns the number of partial rows.
int launch_sweep(Domain& d, void* buf, const double* Ak, double* obs_part) {
    const SweepPlan& P = d.sweep;
    MLMD_REQUIRE(P.ok, MLMD_ERR_STATE, "no one-sweep plan for this domain");
    const int r = d.desc.fd_order / 2;
    const int NW = 2 * r + 1;
    SweepArgs A{};
    A.nx = d.desc.n[0]; A.ny = d.desc.n[1]; A.nz = d.desc.n[2]; A.ld = d.ld;
    A.TX = P.TX; A.TY = P.TY; A.CX = P.CX; A.VPC = P.VPC;
    const int t0 = -4 * r;
    A.t_begin = (t0 - (NW - 1)) / NW * NW;     // round down to a multiple of NW
    if (A.t_begin > t0) A.t_begin -= NW;
    A.t_end = A.nz + 4 * (r + 1);
    const Geo G = geo_of(d);
    A.kc0 = G.kc0; A.kc1 = G.kc1; A.kc2 = G.kc2; A.gk1 = G.gk1; A.gk2 = G.gk2;
    // c_j = (-i dt)^j / j!
    const double dt = d.desc.dt;
    double cr = 1.0, ci = 0.0;
    A.cre[0] = 1.0; A.cim[0] = 0.0;
    for (int j = 1; j <= 4; ++j) {
        const double nr = ci * dt / j, ni = -cr * dt / j;     // (cr + i ci) * (-i dt / j)
        cr = nr; ci = ni;
        A.cre[j] = cr; A.cim[j] = ci;
    }
    const bool obs = obs_part != nullptr;
    const void* k = sweep_kernel_for(d, obs);
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = sweep_config(d, P, attr);
    ProfScope ps(d.prof, MLMD_KERNEL_STAGE, d.stream);
    SweepCoef<float> Kf{};
    SweepCoef<double> Kd{};
    Kf.kc0 = (float)A.kc0; Kf.kc1 = (float)A.kc1; Kf.kc2 = (float)A.kc2; Kf.gk1 = (float)A.gk1; Kf.gk2 = (float)A.gk2;
    Kd.kc0 = A.kc0; Kd.kc1 = A.kc1; Kd.kc2 = A.kc2; Kd.gk1 = A.gk1; Kd.gk2 = A.gk2;
    for (int j = 0; j < 5; ++j) {
        Kf.cre[j] = (float)A.cre[j]; Kf.cim[j] = (float)A.cim[j];
        Kd.cre[j] = A.cre[j]; Kd.cim[j] = A.cim[j];
    }
    void* args[7];
    void* psi = buf;
    const void* V = d.V;
    const void* f = d.fR;
    args[0] = &A;
    args[1] = d.c64() ? (void*)&Kf : (void*)&Kd;
    args[2] = &psi; args[3] = &V; args[4] = &Ak; args[5] = &f; args[6] = &obs_part;
    MLMD_CUDA(cudaLaunchKernelExC(&cfg, k, args));
    d.launches++;
    return P.CX * P.CY * (d.ld / P.VPC);
}

// Time one sweep against one step of staged passes on the domain's own
// buffers (psi is copied to the work buffer wb first; psi itself is not
// written) and keep the faster for the full-scheme steps without projectors
// and the split form's local factor.
void sweep_autotune(Domain& d, const double* Ak) {
    SweepPlan& P = d.sweep;
    if (!P.ok || P.use != 0) return;
    P.use = -1;
    const bool local_steps = !d.has_nl() || d.desc.scheme == MLMD_SCHEME_SPLIT;
    if (!local_steps) return;
    cudaEvent_t e0, e1;
    MLMD_CUDA(cudaEventCreate(&e0));
    MLMD_CUDA(cudaEventCreate(&e1));
    float t_sweep = 0.f, t_staged = 0.f;
    for (int rep = 0; rep < 3; ++rep) {
        MLMD_CUDA(cudaMemcpyAsync(d.wb, d.psi, d.state_bytes, cudaMemcpyDeviceToDevice, d.stream));
        MLMD_CUDA(cudaEventRecord(e0, d.stream));
        launch_sweep(d, d.wb, Ak, nullptr);
        MLMD_CUDA(cudaEventRecord(e1, d.stream));
        MLMD_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        MLMD_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (rep) t_sweep += ms;
        MLMD_CUDA(cudaEventRecord(e0, d.stream));
        for (int s = 0; s < 4; ++s) {
            StageArgs a;
            a.w = s == 0 ? d.psi : d.wa;
            a.psi = d.psi;
            a.out = s == 0 ? d.wa : d.wb;
            a.A = Ak;
            a.gamma_re = 0.0;
            a.gamma_im = -d.desc.dt / (double)(4 - s);
            launch_stage(d, a);
        }
        MLMD_CUDA(cudaEventRecord(e1, d.stream));
        MLMD_CUDA(cudaEventSynchronize(e1));
        MLMD_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (rep) t_staged += ms;
    }
    (void)cudaEventDestroy(e0);
    (void)cudaEventDestroy(e1);
    P.use = t_sweep < t_staged ? 1 : -1;
    P.t_sweep_ms = t_sweep / 2;
    P.t_staged_ms = t_staged / 2;
}

}  // namespace mlmd
