// Local kernels of the LFD step: the finite-difference Hamiltonian of Eq. 3
// applied with the nonlocal scatter fused in, the Taylor-4 nested combine,
// the observable partial sums, the density/current reduction with warp
// shuffles, and the adjoint contractions.
//
// Layout (Sec. V.B.2): psi[g][o] complex, orbital fastest, rows padded to
// `ld` orbitals.  A thread owns one 16-byte vector of a row: two complex64
// or one complex128 orbital, so every neighbour row is read with fully
// coalesced 16-byte loads.
#include <algorithm>

#include "mlmd_internal.cuh"

namespace mlmd {
namespace {

template <typename R> struct Vec;
template <> struct Vec<float> { static constexpr int NC = 2; };
template <> struct Vec<double> { static constexpr int NC = 1; };

template <typename R> struct Cx {
    R re[Vec<R>::NC];
    R im[Vec<R>::NC];
};

__device__ __forceinline__ Cx<float> ldg_c(const float* p) {
    float4 t = __ldg(reinterpret_cast<const float4*>(p));
    Cx<float> c;
    c.re[0] = t.x; c.im[0] = t.y; c.re[1] = t.z; c.im[1] = t.w;
    return c;
}
__device__ __forceinline__ Cx<double> ldg_c(const double* p) {
    double2 t = __ldg(reinterpret_cast<const double2*>(p));
    Cx<double> c;
    c.re[0] = t.x; c.im[0] = t.y;
    return c;
}
__device__ __forceinline__ Cx<float> ld_c(const float* p) {
    float4 t = *reinterpret_cast<const float4*>(p);
    Cx<float> c;
    c.re[0] = t.x; c.im[0] = t.y; c.re[1] = t.z; c.im[1] = t.w;
    return c;
}
__device__ __forceinline__ Cx<double> ld_c(const double* p) {
    double2 t = *reinterpret_cast<const double2*>(p);
    Cx<double> c;
    c.re[0] = t.x; c.im[0] = t.y;
    return c;
}
__device__ __forceinline__ void st_c(float* p, const Cx<float>& c) {
    *reinterpret_cast<float4*>(p) = make_float4(c.re[0], c.im[0], c.re[1], c.im[1]);
}
__device__ __forceinline__ void st_c(double* p, const Cx<double>& c) {
    *reinterpret_cast<double2*>(p) = make_double2(c.re[0], c.im[0]);
}

}  // namespace

Geo geo_of(const Domain& d) {
    Geo G;
    G.nx = d.desc.n[0]; G.ny = d.desc.n[1]; G.nz = d.desc.n[2];
    G.ld = d.ld;
    G.nv = d.c64() ? d.ld / 2 : d.ld;
    G.ng = d.ng;
    const double h = d.desc.h, ih2 = 1.0 / (h * h), ih = 1.0 / h;
    double l0, l1, l2, g1, g2;
    if (d.desc.fd_order == 2) { l0 = -2.0; l1 = 1.0; l2 = 0.0; g1 = 0.5; g2 = 0.0; }
    else { l0 = -2.5; l1 = 4.0 / 3.0; l2 = -1.0 / 12.0; g1 = 2.0 / 3.0; g2 = -1.0 / 12.0; }
    G.kc0 = -0.5 * 3.0 * l0 * ih2;
    G.kc1 = -0.5 * l1 * ih2;
    G.kc2 = -0.5 * l2 * ih2;
    G.gk1 = g1 * ih;
    G.gk2 = g2 * ih;
    G.dV = h * h * h;
    return G;
}

namespace {

Geo make_geo(const Domain& d) { return geo_of(d); }

// Row offsets (in grid points) of the +-1 and +-2 neighbours along one axis
// with periodic wrap.
struct Nb { int64_t p1, m1, p2, m2; };
__device__ __forceinline__ Nb nbr(int c, int n, int64_t s) {
    Nb r;
    r.p1 = (c + 1 < n) ? s : s - (int64_t)n * s;
    r.m1 = (c >= 1) ? -s : (int64_t)(n - 1) * s;
    r.p2 = (c + 2 < n) ? 2 * s : 2 * s - (int64_t)n * s;
    r.m2 = (c >= 2) ? -2 * s : (int64_t)(n - 2) * s;
    return r;
}

template <typename R>
__device__ __forceinline__ const R* rowp(const R* base, int64_t g, int ld, int j) {
    return base + (g * ld + (int64_t)j * Vec<R>::NC) * 2;
}
template <typename R>
__device__ __forceinline__ R* rowp(R* base, int64_t g, int ld, int j) {
    return base + (g * ld + (int64_t)j * Vec<R>::NC) * 2;
}

// Block-wide sum of W doubles; thread 0 of the block gets the totals.
template <int W>
__device__ __forceinline__ void block_sum(double (&v)[W], double* out) {
    __shared__ double sh[32][W];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < W; ++i)
        for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < W; ++i) sh[warp][i] = v[i];
    __syncthreads();
    if (warp == 0) {
        const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
        for (int i = 0; i < W; ++i) {
            double t = lane < nw ? sh[lane][i] : 0.0;
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (lane == 0) out[i] = t;
        }
    }
}

// Block-wide sum of W values of the working type: warp shuffles in R, then
// the per-warp partials in FP64; thread 0 writes the totals.
template <typename R, int W>
__device__ __forceinline__ void block_sum_r(R (&v)[W], double* out) {
    __shared__ double sh[32][W];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < W; ++i)
        for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < W; ++i) sh[warp][i] = (double)v[i];
    __syncthreads();
    if (warp == 0) {
        const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
        for (int i = 0; i < W; ++i) {
            double t = lane < nw ? sh[lane][i] : 0.0;
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (lane == 0) out[i] = t;
        }
    }
}

// Stencil constants in the working type (computed on the host so that no
// thread converts from FP64).
template <typename R> struct GeoR {
    R kc0, kc1, kc2, gk1, gk2;
    int nx, ny, nz, ld, nv;
};

template <typename R>
GeoR<R> make_geo_r(const Domain& d) {
    const Geo G = make_geo(d);
    GeoR<R> g;
    g.kc0 = (R)G.kc0; g.kc1 = (R)G.kc1; g.kc2 = (R)G.kc2; g.gk1 = (R)G.gk1; g.gk2 = (R)G.gk2;
    g.nx = G.nx; g.ny = G.ny; g.nz = G.nz; g.ld = G.ld; g.nv = G.nv;
    return g;
}

// ---------------------------------------------------------------------------
// stage: out = psi + gamma * h(A) w
// Launch: grid (ceil(nx*nv/256), ny, nz), 256 threads; thread t of a block
// row covers point x = t / nv of line (y, z) and 16-byte vector j = t % nv.
// ---------------------------------------------------------------------------
// NLP: projectors per atom of the scatter-back (0: no nonlocal term, 4 or 8)
// GAUGE: velocity-gauge projectors; each entry's sum over its NLP projectors
// is multiplied by the entry's phase ph[e] = e^{-i A.(r - R_a)}.
template <typename R, int ORDER, int NLP, bool OBS, bool HAS_PSI, bool GAUGE>
__global__ void __launch_bounds__(256) k_stage(GeoR<R> G, const R* __restrict__ w, const R* psi, R* out,
                                               const R* __restrict__ V, const R* __restrict__ f,
                                               const double* __restrict__ Ak,
                                               const int32_t* __restrict__ pstart,
                                               const int32_t* __restrict__ patom, const R* __restrict__ pbd,
                                               const R* __restrict__ ph,
                                               const R* __restrict__ P, int n_proj, R gre, R gim,
                                               double* __restrict__ obs) {
    constexpr int NC = Vec<R>::NC;
    __shared__ R sA[4];
    if (threadIdx.x < 3) sA[threadIdx.x] = (R)Ak[threadIdx.x];
    if (threadIdx.x == 3) sA[3] = (R)(0.5 * (Ak[0] * Ak[0] + Ak[1] * Ak[1] + Ak[2] * Ak[2]));
    __syncthreads();
    const unsigned t = blockIdx.x * 256u + threadIdx.x;
    const int x = (int)(t / (unsigned)G.nv);
    const int j = (int)(t - (unsigned)x * (unsigned)G.nv);
    const int y = blockIdx.y, z = blockIdx.z;
    R acc[5] = {0, 0, 0, 0, 0};
    if (x < G.nx) {
        const int64_t sy = G.nx, sz = (int64_t)G.nx * G.ny;
        const int64_t g = x + sy * y + sz * z;
        const Nb b[3] = {nbr(x, G.nx, 1), nbr(y, G.ny, sy), nbr(z, G.nz, sz)};
        const R A0 = sA[0], A1 = sA[1], A2 = sA[2];
        const R diag = V[g] + sA[3];

        const Cx<R> c = ldg_c(rowp(w, g, G.ld, j));
        Cx<R> lap, dd[3];
#pragma unroll
        for (int k = 0; k < NC; ++k) { lap.re[k] = G.kc0 * c.re[k]; lap.im[k] = G.kc0 * c.im[k]; }
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            const Cx<R> p1 = ldg_c(rowp(w, g + b[ax].p1, G.ld, j));
            const Cx<R> m1 = ldg_c(rowp(w, g + b[ax].m1, G.ld, j));
#pragma unroll
            for (int k = 0; k < NC; ++k) {
                lap.re[k] += G.kc1 * (p1.re[k] + m1.re[k]);
                lap.im[k] += G.kc1 * (p1.im[k] + m1.im[k]);
                dd[ax].re[k] = G.gk1 * (p1.re[k] - m1.re[k]);
                dd[ax].im[k] = G.gk1 * (p1.im[k] - m1.im[k]);
            }
            if (ORDER == 4) {
                const Cx<R> p2 = ldg_c(rowp(w, g + b[ax].p2, G.ld, j));
                const Cx<R> m2 = ldg_c(rowp(w, g + b[ax].m2, G.ld, j));
#pragma unroll
                for (int k = 0; k < NC; ++k) {
                    lap.re[k] += G.kc2 * (p2.re[k] + m2.re[k]);
                    lap.im[k] += G.kc2 * (p2.im[k] + m2.im[k]);
                    dd[ax].re[k] += G.gk2 * (p2.re[k] - m2.re[k]);
                    dd[ax].im[k] += G.gk2 * (p2.im[k] - m2.im[k]);
                }
            }
        }
        // h w = lap + diag c - i sum_a A_a d_a (+ nonlocal)
        Cx<R> hw;
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            const R gr = A0 * dd[0].re[k] + A1 * dd[1].re[k] + A2 * dd[2].re[k];
            const R gi = A0 * dd[0].im[k] + A1 * dd[1].im[k] + A2 * dd[2].im[k];
            hw.re[k] = lap.re[k] + diag * c.re[k] + gi;
            hw.im[k] = lap.im[k] + diag * c.im[k] - gr;
        }
        if constexpr (NLP > 0) {
            // EU entries at a time: their atoms, beta * D and projection rows
            // are all requested before any is used
            constexpr int EU = NLP == 4 ? 2 : 1;
            const int e0 = pstart[g], e1 = pstart[g + 1];
            for (int e = e0; e < e1; e += EU) {
                int a[EU];
                R bd[EU][NLP], pc[EU], ps[EU];
                Cx<R> pv[EU][NLP];
#pragma unroll
                for (int u = 0; u < EU; ++u) a[u] = e + u < e1 ? patom[e + u] : -1;
#pragma unroll
                for (int u = 0; u < EU; ++u)
                    if (a[u] >= 0) {
                        if constexpr (GAUGE) {
                            pc[u] = ph[2 * (int64_t)(e + u)];
                            ps[u] = ph[2 * (int64_t)(e + u) + 1];
                        }
#pragma unroll
                        for (int i = 0; i < NLP; ++i) {
                            bd[u][i] = pbd[(int64_t)(e + u) * NLP + i];
                            pv[u][i] = ldg_c(rowp(P, (int64_t)a[u] * NLP + i, G.ld, j));
                        }
                    }
#pragma unroll
                for (int u = 0; u < EU; ++u)
                    if (a[u] >= 0) {
                        if constexpr (GAUGE) {
                            Cx<R> t;
#pragma unroll
                            for (int k = 0; k < NC; ++k) { t.re[k] = 0; t.im[k] = 0; }
#pragma unroll
                            for (int i = 0; i < NLP; ++i)
#pragma unroll
                                for (int k = 0; k < NC; ++k) {
                                    t.re[k] += bd[u][i] * pv[u][i].re[k];
                                    t.im[k] += bd[u][i] * pv[u][i].im[k];
                                }
#pragma unroll
                            for (int k = 0; k < NC; ++k) {
                                hw.re[k] += pc[u] * t.re[k] - ps[u] * t.im[k];
                                hw.im[k] += pc[u] * t.im[k] + ps[u] * t.re[k];
                            }
                        } else {
#pragma unroll
                            for (int i = 0; i < NLP; ++i)
#pragma unroll
                                for (int k = 0; k < NC; ++k) {
                                    hw.re[k] += bd[u][i] * pv[u][i].re[k];
                                    hw.im[k] += bd[u][i] * pv[u][i].im[k];
                                }
                        }
                    }
            }
        }
        Cx<R> o;
        if (HAS_PSI) {
            const Cx<R> p = ld_c(rowp(psi, g, G.ld, j));
#pragma unroll
            for (int k = 0; k < NC; ++k) {
                o.re[k] = p.re[k] + gre * hw.re[k] - gim * hw.im[k];
                o.im[k] = p.im[k] + gre * hw.im[k] + gim * hw.re[k];
            }
        } else {
#pragma unroll
            for (int k = 0; k < NC; ++k) {
                o.re[k] = gre * hw.re[k] - gim * hw.im[k];
                o.im[k] = gre * hw.im[k] + gim * hw.re[k];
            }
        }
        st_c(rowp(out, g, G.ld, j), o);
        if (OBS) {
#pragma unroll
            for (int k = 0; k < NC; ++k) {
                const R fo = f[j * NC + k];
                const R cr = c.re[k], ci = c.im[k];
                acc[0] += fo * (cr * cr + ci * ci);
                acc[1] += fo * (cr * hw.re[k] + ci * hw.im[k]);
#pragma unroll
                for (int ax = 0; ax < 3; ++ax) acc[2 + ax] += fo * (cr * dd[ax].im[k] - ci * dd[ax].re[k]);
            }
        }
    }
    if (OBS) {
        const int64_t blin = blockIdx.x + (int64_t)gridDim.x * (blockIdx.y + (int64_t)gridDim.y * blockIdx.z);
        block_sum_r<R, 5>(acc, obs + blin * 5);
    }
}

template <typename R, int ORDER>
void stage_dispatch(Domain& d, const StageArgs& a, dim3 grid) {
    const GeoR<R> G = make_geo_r<R>(d);
    const bool nl = d.has_nl() && a.P != nullptr;
    const bool obs = a.obs != nullptr;
    const bool hp = a.psi != nullptr;
    const R* w = static_cast<const R*>(a.w);
    const R* psi = static_cast<const R*>(a.psi);
    R* out = static_cast<R*>(a.out);
    const R* V = static_cast<const R*>(d.V);
    const R* f = static_cast<const R*>(d.fR);
    const R* pbd = static_cast<const R*>(d.nl.pbd);
    const R* P = static_cast<const R*>(a.P);
    const bool gauge = nl && gauge_on(d);
    const R* ph = gauge ? static_cast<const R*>(d.nl.ph_pt) : nullptr;
#define MLMD_STAGE(NLv, OBSv, HPv, GAv)                                                              \
    k_stage<R, ORDER, NLv, OBSv, HPv, GAv><<<grid, 256, 0, d.stream>>>(                              \
        G, w, psi, out, V, f, a.A, d.nl.pstart, d.nl.patom, pbd, ph, P, d.nl.n_proj, (R)a.gamma_re,  \
        (R)a.gamma_im, a.obs)
#define MLMD_STAGE_NL(NLv, GAv)                                                                       \
    if (obs) { if (hp) MLMD_STAGE(NLv, true, true, GAv); else MLMD_STAGE(NLv, true, false, GAv); }   \
    else { if (hp) MLMD_STAGE(NLv, false, true, GAv); else MLMD_STAGE(NLv, false, false, GAv); }
    if (nl && d.nl.n_proj == 4) {
        if (gauge) { MLMD_STAGE_NL(4, true) } else { MLMD_STAGE_NL(4, false) }
    } else if (nl) {
        if (gauge) { MLMD_STAGE_NL(8, true) } else { MLMD_STAGE_NL(8, false) }
    } else {
        MLMD_STAGE_NL(0, false)
    }
#undef MLMD_STAGE_NL
#undef MLMD_STAGE
}

// ---------------------------------------------------------------------------
// final observables: fixed-order FP64 sum of the per-block partials
// ---------------------------------------------------------------------------
__global__ void k_obs_finish(const double* __restrict__ part, int nblk, double dV, const double* __restrict__ A,
                             double* __restrict__ row) {
    double v[5] = {0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblk; b += blockDim.x)
#pragma unroll
        for (int i = 0; i < 5; ++i) v[i] += part[(int64_t)b * 5 + i];
    __shared__ double tot[5];
    block_sum<5>(v, tot);
    __syncthreads();
    if (threadIdx.x == 0) {
        const double n = dV * tot[0];
        row[0] = n;
        row[1] = dV * tot[1];
        for (int a = 0; a < 3; ++a) row[2 + a] = dV * tot[2 + a] + A[a] * n;
    }
}

__global__ void k_reduce_partials(const double* __restrict__ part, int nblk, int width, double* __restrict__ out) {
    // one block per output column, fixed order
    const int col = blockIdx.x;
    double v[1] = {0.0};
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) v[0] += part[(int64_t)b * width + col];
    __shared__ double tot[1];
    block_sum<1>(v, tot);
    __syncthreads();
    if (threadIdx.x == 0) out[col] = tot[0];
}

// ---------------------------------------------------------------------------
// density and current: one warp per grid point, lanes over the orbital row,
// warp-shuffle reduction over orbitals.  Complex64 rows sum each lane's
// orbitals in FP32 (the occupations in the working type fR; a lane holds
// ld/64 vectors, 16 at N_o = 1024) and reduce across the lanes in FP64:
// FP64 arithmetic per orbital value cost milliseconds per call at Blackwell
// Ultra's reduced FP64 rate.  Complex128 sums in FP64 throughout.
// ---------------------------------------------------------------------------
template <typename R, int ORDER>
__global__ void __launch_bounds__(256) k_density_current(Geo G, const R* __restrict__ psi,
                                                         const double* __restrict__ f, const R* __restrict__ fR,
                                                         const double* __restrict__ Ak, R* __restrict__ rho,
                                                         R* __restrict__ jcur, double* __restrict__ Jpart) {
    constexpr int NC = Vec<R>::NC;
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double Jacc[3] = {0, 0, 0};
    const R gk1 = (R)G.gk1, gk2 = (R)G.gk2;
    for (int64_t g = warp; g < G.ng; g += nwarps) {
        const int x = (int)(g % G.nx);
        const int64_t gyz = g / G.nx;
        const int y = (int)(gyz % G.ny);
        const int z = (int)(gyz / G.ny);
        const Nb b[3] = {nbr(x, G.nx, 1), nbr(y, G.ny, G.nx), nbr(z, G.nz, (int64_t)G.nx * G.ny)};
        double r = 0.0, jj[3] = {0.0, 0.0, 0.0};
        if constexpr (std::is_same<R, float>::value) {
            float rf = 0.f, jf[3] = {0.f, 0.f, 0.f};
            for (int j = lane; j < G.nv; j += 32) {
                const Cx<R> c = ldg_c(rowp(psi, g, G.ld, j));
                float fo[NC];
#pragma unroll
                for (int k = 0; k < NC; ++k) {
                    fo[k] = fR[j * NC + k];
                    rf += fo[k] * (c.re[k] * c.re[k] + c.im[k] * c.im[k]);
                }
#pragma unroll
                for (int ax = 0; ax < 3; ++ax) {
                    const Cx<R> p1 = ldg_c(rowp(psi, g + b[ax].p1, G.ld, j));
                    const Cx<R> m1 = ldg_c(rowp(psi, g + b[ax].m1, G.ld, j));
                    Cx<R> dd;
#pragma unroll
                    for (int k = 0; k < NC; ++k) {
                        dd.re[k] = gk1 * (p1.re[k] - m1.re[k]);
                        dd.im[k] = gk1 * (p1.im[k] - m1.im[k]);
                    }
                    if (ORDER == 4) {
                        const Cx<R> p2 = ldg_c(rowp(psi, g + b[ax].p2, G.ld, j));
                        const Cx<R> m2 = ldg_c(rowp(psi, g + b[ax].m2, G.ld, j));
#pragma unroll
                        for (int k = 0; k < NC; ++k) {
                            dd.re[k] += gk2 * (p2.re[k] - m2.re[k]);
                            dd.im[k] += gk2 * (p2.im[k] - m2.im[k]);
                        }
                    }
#pragma unroll
                    for (int k = 0; k < NC; ++k) jf[ax] += fo[k] * (c.re[k] * dd.im[k] - c.im[k] * dd.re[k]);
                }
            }
            r = rf;
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) jj[ax] = jf[ax];
        } else
        for (int j = lane; j < G.nv; j += 32) {
            const Cx<R> c = ldg_c(rowp(psi, g, G.ld, j));
#pragma unroll
            for (int k = 0; k < NC; ++k) r += f[j * NC + k] * ((double)c.re[k] * c.re[k] + (double)c.im[k] * c.im[k]);
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) {
                const Cx<R> p1 = ldg_c(rowp(psi, g + b[ax].p1, G.ld, j));
                const Cx<R> m1 = ldg_c(rowp(psi, g + b[ax].m1, G.ld, j));
                Cx<R> dd;
#pragma unroll
                for (int k = 0; k < NC; ++k) {
                    dd.re[k] = gk1 * (p1.re[k] - m1.re[k]);
                    dd.im[k] = gk1 * (p1.im[k] - m1.im[k]);
                }
                if (ORDER == 4) {
                    const Cx<R> p2 = ldg_c(rowp(psi, g + b[ax].p2, G.ld, j));
                    const Cx<R> m2 = ldg_c(rowp(psi, g + b[ax].m2, G.ld, j));
#pragma unroll
                    for (int k = 0; k < NC; ++k) {
                        dd.re[k] += gk2 * (p2.re[k] - m2.re[k]);
                        dd.im[k] += gk2 * (p2.im[k] - m2.im[k]);
                    }
                }
#pragma unroll
                for (int k = 0; k < NC; ++k)
                    jj[ax] += f[j * NC + k] * ((double)c.re[k] * dd.im[k] - (double)c.im[k] * dd.re[k]);
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            r += __shfl_xor_sync(0xffffffffu, r, o);
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) jj[ax] += __shfl_xor_sync(0xffffffffu, jj[ax], o);
        }
        if (lane == 0) {
            if (rho) rho[g] = (R)r;
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) {
                const double ja = jj[ax] + Ak[ax] * r;
                if (jcur) jcur[ax * G.ng + g] = (R)ja;
                Jacc[ax] += ja;
            }
        }
    }
    block_sum<3>(Jacc, Jpart + (int64_t)blockIdx.x * 3);
}

// ---------------------------------------------------------------------------
// out = sum_t coef_t in_t
// ---------------------------------------------------------------------------
struct LinArgs {
    const void* in[5];
    double cre[5], cim[5];
    int n;
};

template <typename R>
__global__ void __launch_bounds__(256) k_lincomb(LinArgs L, int64_t nvec, R* __restrict__ out) {
    constexpr int NC = Vec<R>::NC;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nvec; t += (int64_t)gridDim.x * blockDim.x) {
        Cx<R> o;
#pragma unroll
        for (int k = 0; k < NC; ++k) { o.re[k] = 0; o.im[k] = 0; }
        for (int s = 0; s < L.n; ++s) {
            const Cx<R> c = ld_c(static_cast<const R*>(L.in[s]) + t * NC * 2);
            const R a = (R)L.cre[s], b = (R)L.cim[s];
#pragma unroll
            for (int k = 0; k < NC; ++k) {
                o.re[k] += a * c.re[k] - b * c.im[k];
                o.im[k] += a * c.im[k] + b * c.re[k];
            }
        }
        st_c(out + t * NC * 2, o);
    }
}

// ---------------------------------------------------------------------------
// adjoint contractions (one warp per grid point)
// ---------------------------------------------------------------------------
struct ContractArgs {
    const void* z[4];
    const void* u[4];
};

template <typename R, int ORDER>
__global__ void __launch_bounds__(256) k_adjoint_contract(Geo G, ContractArgs C, double* __restrict__ part,
                                                          double* __restrict__ gV) {
    constexpr int NC = Vec<R>::NC;
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double acc[4] = {0, 0, 0, 0};
    const R gk1 = (R)G.gk1, gk2 = (R)G.gk2;
    for (int64_t g = warp; g < G.ng; g += nwarps) {
        const int x = (int)(g % G.nx);
        const int64_t gyz = g / G.nx;
        const int y = (int)(gyz % G.ny);
        const int z = (int)(gyz / G.ny);
        const Nb b[3] = {nbr(x, G.nx, 1), nbr(y, G.ny, G.nx), nbr(z, G.nz, (int64_t)G.nx * G.ny)};
        double pv = 0.0, pa[3] = {0, 0, 0};
        for (int p = 0; p < 4; ++p) {
            const R* zp = static_cast<const R*>(C.z[p]);
            const R* up = static_cast<const R*>(C.u[p]);
            for (int j = lane; j < G.nv; j += 32) {
                const Cx<R> zc = ldg_c(rowp(zp, g, G.ld, j));
                const Cx<R> uc = ldg_c(rowp(up, g, G.ld, j));
#pragma unroll
                for (int k = 0; k < NC; ++k) pv += 2.0 * ((double)zc.re[k] * uc.re[k] + (double)zc.im[k] * uc.im[k]);
#pragma unroll
                for (int ax = 0; ax < 3; ++ax) {
                    const Cx<R> p1 = ldg_c(rowp(up, g + b[ax].p1, G.ld, j));
                    const Cx<R> m1 = ldg_c(rowp(up, g + b[ax].m1, G.ld, j));
                    Cx<R> dd;
#pragma unroll
                    for (int k = 0; k < NC; ++k) {
                        dd.re[k] = gk1 * (p1.re[k] - m1.re[k]);
                        dd.im[k] = gk1 * (p1.im[k] - m1.im[k]);
                    }
                    if (ORDER == 4) {
                        const Cx<R> p2 = ldg_c(rowp(up, g + b[ax].p2, G.ld, j));
                        const Cx<R> m2 = ldg_c(rowp(up, g + b[ax].m2, G.ld, j));
#pragma unroll
                        for (int k = 0; k < NC; ++k) {
                            dd.re[k] += gk2 * (p2.re[k] - m2.re[k]);
                            dd.im[k] += gk2 * (p2.im[k] - m2.im[k]);
                        }
                    }
                    // 2 Re(conj(z) (-i d)) = 2 Im(conj(z) d)
#pragma unroll
                    for (int k = 0; k < NC; ++k)
                        pa[ax] += 2.0 * ((double)zc.re[k] * dd.im[k] - (double)zc.im[k] * dd.re[k]);
                }
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            pv += __shfl_xor_sync(0xffffffffu, pv, o);
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) pa[ax] += __shfl_xor_sync(0xffffffffu, pa[ax], o);
        }
        if (lane == 0) {
            gV[g] += pv;
            acc[0] += pa[0]; acc[1] += pa[1]; acc[2] += pa[2]; acc[3] += pv;
        }
    }
    block_sum<4>(acc, part + (int64_t)blockIdx.x * 4);
}

// ---------------------------------------------------------------------------
// split scheme (Eq. 2): per-orbital norms, the nonlocal factor, the rescale
// ---------------------------------------------------------------------------
// part[b][o] = sum over the block's grid rows of |psi[g][o]|^2 (o < ld)
template <typename R>
__global__ void __launch_bounds__(256) k_orbital_norms(const R* __restrict__ psi, int64_t ng, int ld, int rows_per_block,
                                                       double* __restrict__ part) {
    const int o = blockIdx.y * blockDim.x + threadIdx.x;
    if (o >= ld) return;
    const int64_t g0 = (int64_t)blockIdx.x * rows_per_block;
    const int64_t g1 = min(ng, g0 + rows_per_block);
    double s = 0.0;
    for (int64_t g = g0; g < g1; ++g) {
        const R re = psi[(g * ld + o) * 2], im = psi[(g * ld + o) * 2 + 1];
        s += (double)re * re + (double)im * im;
    }
    part[(int64_t)blockIdx.x * ld + o] = s;
}

__global__ void k_sum_rows(const double* __restrict__ part, int nrow, int ld, double* __restrict__ out) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= ld) return;
    double s = 0.0;
    for (int r = 0; r < nrow; ++r) s += part[(int64_t)r * ld + o];
    out[o] = s;
}

template <typename R>
__global__ void __launch_bounds__(256) k_scale_orbitals(R* __restrict__ psi, int64_t n, int ld,
                                                        const double* __restrict__ before,
                                                        const double* __restrict__ after) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const int o = (int)(t % ld);
        const double a = after[o];
        const R sc = (R)(a > 0.0 ? sqrt(before[o] / a) : 1.0);
        psi[t * 2] *= sc;
        psi[t * 2 + 1] *= sc;
    }
}

// out = in + i gamma_im * v_nl in   (v_nl from the projections P of in;
// ph: null, or the per-entry velocity-gauge phases e^{-i A.(r - R_a)})
template <typename R>
__global__ void __launch_bounds__(256) k_nl_apply(Geo G, const R* __restrict__ in, const int32_t* __restrict__ pstart,
                                                  const int32_t* __restrict__ patom, const R* __restrict__ pbd,
                                                  const R* __restrict__ ph,
                                                  const R* __restrict__ P, int n_proj, R gim, R* out) {
    constexpr int NC = Vec<R>::NC;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t g = t / G.nv;
    const int j = (int)(t - g * G.nv);
    if (g >= G.ng) return;
    Cx<R> acc;
#pragma unroll
    for (int k = 0; k < NC; ++k) { acc.re[k] = 0; acc.im[k] = 0; }
    for (int e = pstart[g]; e < pstart[g + 1]; ++e) {
        const int a = patom[e];
        Cx<R> t;
#pragma unroll
        for (int k = 0; k < NC; ++k) { t.re[k] = 0; t.im[k] = 0; }
        for (int i = 0; i < n_proj; ++i) {
            const R bd = pbd[(int64_t)e * n_proj + i];
            const Cx<R> pv = ldg_c(rowp(P, (int64_t)a * n_proj + i, G.ld, j));
#pragma unroll
            for (int k = 0; k < NC; ++k) { t.re[k] += bd * pv.re[k]; t.im[k] += bd * pv.im[k]; }
        }
        if (ph) {
            const R pc = ph[2 * (int64_t)e], ps = ph[2 * (int64_t)e + 1];
#pragma unroll
            for (int k = 0; k < NC; ++k) {
                acc.re[k] += pc * t.re[k] - ps * t.im[k];
                acc.im[k] += pc * t.im[k] + ps * t.re[k];
            }
        } else {
#pragma unroll
            for (int k = 0; k < NC; ++k) { acc.re[k] += t.re[k]; acc.im[k] += t.im[k]; }
        }
    }
    const Cx<R> c = ld_c(rowp(in, g, G.ld, j));
    Cx<R> o;
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        o.re[k] = c.re[k] - gim * acc.im[k];
        o.im[k] = c.im[k] + gim * acc.re[k];
    }
    st_c(rowp(out, g, G.ld, j), o);
}

}  // namespace

// ---------------------------------------------------------------------------
// launch wrappers
// ---------------------------------------------------------------------------
dim3 stage_grid(const Domain& d) {
    const unsigned nv = d.c64() ? d.ld / 2 : d.ld;
    return dim3((unsigned)((d.desc.n[0] * nv + 255) / 256), (unsigned)d.desc.n[1], (unsigned)d.desc.n[2]);
}

int stage_blocks(const Domain& d) {
    const dim3 g = stage_grid(d);
    return (int)(g.x * g.y * g.z);
}

int launch_stage(Domain& d, const StageArgs& a, bool* proj_done) {
    if (launch_stage_tma(d, a, proj_done)) return tma_blocks(d);
    const dim3 grid = stage_grid(d);
    ProfScope ps(d.prof, MLMD_KERNEL_STAGE, d.stream);
    if (d.c64()) {
        if (d.desc.fd_order == 4) stage_dispatch<float, 4>(d, a, grid);
        else stage_dispatch<float, 2>(d, a, grid);
    } else {
        if (d.desc.fd_order == 4) stage_dispatch<double, 4>(d, a, grid);
        else stage_dispatch<double, 2>(d, a, grid);
    }
    d.launches++;
    MLMD_CUDA(cudaGetLastError());
    return stage_blocks(d);
}

void launch_obs_finish(Domain& d, const double* partials, int nblk, const double* A, double* row) {
    k_obs_finish<<<1, 256, 0, d.stream>>>(partials, nblk, d.desc.h * d.desc.h * d.desc.h, A, row);
    d.launches++;
    MLMD_CUDA(cudaGetLastError());
}

void launch_reduce_partials(Domain& d, const double* part, int nblk, int width, double* out) {
    k_reduce_partials<<<width, 256, 0, d.stream>>>(part, nblk, width, out);
    d.launches++;
    MLMD_CUDA(cudaGetLastError());
}

int density_blocks(const Domain& d) {
    int64_t b = (d.ng + 7) / 8;
    return (int)(b < 152 * 16 ? b : 152 * 16);
}

void launch_density_current(Domain& d, const double* A, void* rho, void* j, double* Jpart, int nblk) {
    const Geo G = make_geo(d);
    if (d.c64()) {
        if (d.desc.fd_order == 4)
            k_density_current<float, 4><<<nblk, 256, 0, d.stream>>>(G, (const float*)d.psi, d.f, (const float*)d.fR, A, (float*)rho,
                                                                (float*)j, Jpart);
        else
            k_density_current<float, 2><<<nblk, 256, 0, d.stream>>>(G, (const float*)d.psi, d.f, (const float*)d.fR, A, (float*)rho,
                                                                (float*)j, Jpart);
    } else {
        if (d.desc.fd_order == 4)
            k_density_current<double, 4><<<nblk, 256, 0, d.stream>>>(G, (const double*)d.psi, d.f, (const double*)d.fR, A,
                                                                 (double*)rho, (double*)j, Jpart);
        else
            k_density_current<double, 2><<<nblk, 256, 0, d.stream>>>(G, (const double*)d.psi, d.f, (const double*)d.fR, A,
                                                                 (double*)rho, (double*)j, Jpart);
    }
    d.launches++;
    MLMD_CUDA(cudaGetLastError());
}

void launch_lincomb(Domain& d, int n, const void* const* in, const double* cre, const double* cim, void* out) {
    LinArgs L;
    L.n = n;
    for (int i = 0; i < 5; ++i) {
        L.in[i] = i < n ? in[i] : nullptr;
        L.cre[i] = i < n ? cre[i] : 0.0;
        L.cim[i] = i < n ? cim[i] : 0.0;
    }
    const int64_t nvec = d.ng * (d.c64() ? d.ld / 2 : d.ld);
    const int blocks = (int)std::min<int64_t>((nvec + 255) / 256, 152 * 32);
    if (d.c64()) k_lincomb<float><<<blocks, 256, 0, d.stream>>>(L, nvec, (float*)out);
    else k_lincomb<double><<<blocks, 256, 0, d.stream>>>(L, nvec, (double*)out);
    d.launches++;
    MLMD_CUDA(cudaGetLastError());
}

int contract_blocks(const Domain& d) { return density_blocks(d); }

void launch_adjoint_contract(Domain& d, const void* const* z, const void* const* u, double* part, int nblk,
                             double* gV) {
    const Geo G = make_geo(d);
    ContractArgs C;
    for (int p = 0; p < 4; ++p) { C.z[p] = z[p]; C.u[p] = u[p]; }
    if (d.c64()) {
        if (d.desc.fd_order == 4) k_adjoint_contract<float, 4><<<nblk, 256, 0, d.stream>>>(G, C, part, gV);
        else k_adjoint_contract<float, 2><<<nblk, 256, 0, d.stream>>>(G, C, part, gV);
    } else {
        if (d.desc.fd_order == 4) k_adjoint_contract<double, 4><<<nblk, 256, 0, d.stream>>>(G, C, part, gV);
        else k_adjoint_contract<double, 2><<<nblk, 256, 0, d.stream>>>(G, C, part, gV);
    }
    d.launches++;
    MLMD_CUDA(cudaGetLastError());
}

void launch_orbital_norms(Domain& d, const void* psi, double* nrm) {
    const int rows = 512;
    const int nrow = (int)((d.ng + rows - 1) / rows);
    double* part = (double*)d.mem.get(sizeof(double) * (size_t)nrow * d.ld);
    dim3 grid(nrow, (d.ld + 255) / 256);
    const int bx = std::min(d.ld, 256);
    if (d.c64()) k_orbital_norms<float><<<grid, bx, 0, d.stream>>>((const float*)psi, d.ng, d.ld, rows, part);
    else k_orbital_norms<double><<<grid, bx, 0, d.stream>>>((const double*)psi, d.ng, d.ld, rows, part);
    k_sum_rows<<<(d.ld + 255) / 256, 256, 0, d.stream>>>(part, nrow, d.ld, nrm);
    d.launches += 2;
    MLMD_CUDA(cudaGetLastError());
    d.mem.put(part);
}

void launch_scale_orbitals(Domain& d, void* psi, const double* before, const double* after) {
    const int64_t n = d.ng * d.ld;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 32);
    if (d.c64()) k_scale_orbitals<float><<<blocks, 256, 0, d.stream>>>((float*)psi, n, d.ld, before, after);
    else k_scale_orbitals<double><<<blocks, 256, 0, d.stream>>>((double*)psi, n, d.ld, before, after);
    d.launches++;
    MLMD_CUDA(cudaGetLastError());
}

void launch_nl_apply(Domain& d, const void* in, const void* P, void* out, double gamma_im) {
    const Geo G = make_geo(d);
    const int blocks = stage_blocks(d);
    const void* ph = gauge_on(d) ? d.nl.ph_pt : nullptr;
    if (d.c64())
        k_nl_apply<float><<<blocks, 256, 0, d.stream>>>(G, (const float*)in, d.nl.pstart, d.nl.patom, (const float*)d.nl.pbd,
                                                        (const float*)ph, (const float*)P, d.nl.n_proj, (float)gamma_im,
                                                        (float*)out);
    else
        k_nl_apply<double><<<blocks, 256, 0, d.stream>>>(G, (const double*)in, d.nl.pstart, d.nl.patom,
                                                         (const double*)d.nl.pbd, (const double*)ph, (const double*)P,
                                                         d.nl.n_proj, gamma_im, (double*)out);
    d.launches++;
    MLMD_CUDA(cudaGetLastError());
}

}  // namespace mlmd
