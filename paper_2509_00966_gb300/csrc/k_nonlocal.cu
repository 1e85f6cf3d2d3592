// Nonlocal projector term of Eq. 3, applied in the GEMM form of Sec. V.B.5:
// a projection P = dV B^T w (per atom, over its sphere of grid points)
// followed by a scatter-back B (D o P) that the stage kernel fuses per grid
// point.  This file builds the tables on the device (neighbour lists with a
// bit-exact FP64 membership test, projector values, the per-point transpose)
// and runs the projection.
#include <algorithm>
#include <cmath>

#include "mlmd_internal.cuh"

namespace mlmd {
namespace {

constexpr int kMaxAxis = 1024;  // grid points per axis served by the list builder

struct NLGeo {
    int n[3];
    double h;
    double L[3];
    double rc2;
    int m;          // candidate half-width per axis (grid points)
};

// Minimum-image displacement of grid coordinate c from position p along one
// axis, every operation rounded separately (no contraction into FMA):
//   t = c*h - p;  delta = t - L*floor(t/L + 1/2)
__device__ __forceinline__ double min_image(int c, double h, double p, double L) {
    const double t = __dsub_rn(__dmul_rn((double)c, h), p);
    const double k = floor(__dadd_rn(__ddiv_rn(t, L), 0.5));
    return __dsub_rn(t, __dmul_rn(L, k));
}

__device__ __forceinline__ double dist2(double dx, double dy, double dz) {
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// One block per atom.  Candidate coordinates per axis are the grid lines
// within m of the atom (all lines if the window covers the axis), kept in
// ascending order; candidates are enumerated z, y, x (x fastest), so the
// members come out in ascending linear index.  Pass 1 (idx == null) counts,
// pass 2 writes the list with a block-wide ordered compaction.
__global__ void __launch_bounds__(256) k_nl_lists(NLGeo G, const double* __restrict__ pos,
                                                  const int64_t* __restrict__ off, int64_t* __restrict__ counts,
                                                  int32_t* __restrict__ idx) {
    __shared__ int cand[3][kMaxAxis];
    __shared__ int ncand[3];
    __shared__ int warp_tot[8];
    __shared__ int64_t running;
    const int a = blockIdx.x;
    if (threadIdx.x < 3) {
        const int ax = threadIdx.x, n = G.n[ax];
        int k = 0;
        if (2 * G.m + 1 >= n) {
            for (int i = 0; i < n; ++i) cand[ax][k++] = i;
        } else {
            double p = pos[3 * a + ax];
            p = p - G.L[ax] * floor(p / G.L[ax]);
            int c0 = (int)floor(p / G.h);
            c0 = ((c0 % n) + n) % n;
            for (int i = 0; i < n; ++i) {
                int dd = i - c0;
                dd = ((dd % n) + n) % n;
                const int cd = dd < n - dd ? dd : n - dd;
                if (cd <= G.m) cand[ax][k++] = i;
            }
        }
        ncand[ax] = k;
    }
    if (threadIdx.x == 0) running = 0;
    __syncthreads();
    const int64_t nx = ncand[0], ny = ncand[1];
    const int64_t total = nx * ny * ncand[2];
    const double px = pos[3 * a], py = pos[3 * a + 1], pz = pos[3 * a + 2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t base = idx ? off[a] : 0;
    for (int64_t t0 = 0; t0 < total; t0 += blockDim.x) {
        const int64_t t = t0 + threadIdx.x;
        int flag = 0;
        int32_t gi = 0;
        if (t < total) {
            const int ix = (int)(t % nx);
            const int64_t r = t / nx;
            const int iy = (int)(r % ny);
            const int iz = (int)(r / ny);
            const int x = cand[0][ix], y = cand[1][iy], z = cand[2][iz];
            const double d2 = dist2(min_image(x, G.h, px, G.L[0]), min_image(y, G.h, py, G.L[1]),
                                    min_image(z, G.h, pz, G.L[2]));
            flag = d2 <= G.rc2;
            gi = x + G.n[0] * (y + G.n[1] * z);
        }
        const unsigned bal = __ballot_sync(0xffffffffu, flag);
        if (lane == 0) warp_tot[warp] = __popc(bal);
        __syncthreads();
        int before = 0, tot = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            if (w < warp) before += warp_tot[w];
            tot += warp_tot[w];
        }
        if (idx && flag) idx[base + running + before + __popc(bal & ((1u << lane) - 1u))] = gi;
        __syncthreads();
        if (threadIdx.x == 0) running += tot;
        __syncthreads();
    }
    if (!idx && threadIdx.x == 0) counts[a] = running;
}

// Projector values on the lists (one block per atom), then the normalisation
// dV sum_r b^2 = 1 of each projector over its support.
__global__ void __launch_bounds__(256) k_nl_values(NLGeo G, const double* __restrict__ pos,
                                                   const int64_t* __restrict__ off,
                                                   const int32_t* __restrict__ idx, int n_proj, double r_c,
                                                   double dV, double* __restrict__ beta) {
    const int a = blockIdx.x;
    const int64_t q0 = off[a], q1 = off[a + 1];
    const double px = pos[3 * a], py = pos[3 * a + 1], pz = pos[3 * a + 2];
    for (int64_t q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
        const int g = idx[q];
        const int x = g % G.n[0], y = (g / G.n[0]) % G.n[1], z = g / (G.n[0] * G.n[1]);
        const double dl[3] = {min_image(x, G.h, px, G.L[0]), min_image(y, G.h, py, G.L[1]),
                              min_image(z, G.h, pz, G.L[2])};
        const double d2 = dist2(dl[0], dl[1], dl[2]);
        for (int set = 0; set < n_proj / 4; ++set) {
            const double rc = set == 0 ? r_c : r_c / sqrt(2.0);
            const double s = exp(-d2 / (2.0 * rc * rc));
            beta[q * n_proj + 4 * set] = s;
            for (int ax = 0; ax < 3; ++ax) beta[q * n_proj + 4 * set + 1 + ax] = dl[ax] / rc * s;
        }
    }
    __syncthreads();
    __shared__ double red[8][256 / 32];
    __shared__ double scale[8];
    for (int i = 0; i < n_proj; ++i) {
        double s = 0.0;
        for (int64_t q = q0 + threadIdx.x; q < q1; q += blockDim.x) s += beta[q * n_proj + i] * beta[q * n_proj + i];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if ((threadIdx.x & 31) == 0) red[i][threadIdx.x >> 5] = s;
    }
    __syncthreads();
    if (threadIdx.x < n_proj) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[threadIdx.x][w];
        s *= dV;
        scale[threadIdx.x] = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
    }
    __syncthreads();
    for (int64_t q = q0 + threadIdx.x; q < q1; q += blockDim.x)
        for (int i = 0; i < n_proj; ++i) beta[q * n_proj + i] *= scale[i];
}

// ---- per-point transpose of the lists (for the fused scatter) ------------
__global__ void k_pt_count(const int32_t* __restrict__ idx, int64_t n, int32_t* __restrict__ cnt) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&cnt[idx[q]], 1);
}

// Exclusive scan of cnt[0..n) into start[0..n] by one block, chunk by chunk.
__global__ void k_scan(const int32_t* __restrict__ cnt, int64_t n, int32_t* __restrict__ start) {
    __shared__ int32_t buf[1024];
    __shared__ int32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t c0 = 0; c0 < n; c0 += 1024) {
        const int64_t i = c0 + threadIdx.x;
        int32_t v = i < n ? cnt[i] : 0;
        buf[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {
            int32_t t = threadIdx.x >= o ? buf[threadIdx.x - o] : 0;
            __syncthreads();
            buf[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < n) start[i] = carry + buf[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry += buf[1023];
        __syncthreads();
    }
    if (threadIdx.x == 0) start[n] = carry;
}

__global__ void k_pt_fill(const int64_t* __restrict__ off, const int32_t* __restrict__ idx,
                          const int32_t* __restrict__ start, int32_t* __restrict__ cursor,
                          int32_t* __restrict__ ent_q) {
    const int a = blockIdx.x;
    for (int64_t q = off[a] + threadIdx.x; q < off[a + 1]; q += blockDim.x) {
        const int g = idx[q];
        const int slot = atomicAdd(&cursor[g], 1);
        ent_q[start[g] + slot] = (int32_t)q;
    }
}

// Sort each point's entries by list index (atoms in order), fill atom ids and
// beta * D in the working type.
template <typename R>
__global__ void k_pt_finish(int64_t ng, const int32_t* __restrict__ start, int32_t* __restrict__ ent_q,
                            const int64_t* __restrict__ off, int n_atoms, const double* __restrict__ beta,
                            const double* __restrict__ D, int n_proj, int32_t* __restrict__ patom,
                            R* __restrict__ pbd) {
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < ng; g += (int64_t)gridDim.x * blockDim.x) {
        const int e0 = start[g], e1 = start[g + 1];
        for (int e = e0 + 1; e < e1; ++e) {
            const int32_t v = ent_q[e];
            int k = e - 1;
            while (k >= e0 && ent_q[k] > v) { ent_q[k + 1] = ent_q[k]; --k; }
            ent_q[k + 1] = v;
        }
        for (int e = e0; e < e1; ++e) {
            const int64_t q = ent_q[e];
            int lo = 0, hi = n_atoms - 1;  // atom with off[a] <= q < off[a+1]
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (off[mid] <= q) lo = mid; else hi = mid - 1;
            }
            patom[e] = lo;
            for (int i = 0; i < n_proj; ++i) pbd[(int64_t)e * n_proj + i] = (R)(beta[q * n_proj + i] * D[lo * n_proj + i]);
        }
    }
}

template <typename R>
__global__ void k_cast(const double* __restrict__ in, int64_t n, R* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (R)in[i];
}

// ---- velocity-gauge tables --------------------------------------------------
// Minimum-image displacement r - R_a of every list entry (one block per atom),
// the same FP64 wrap as the list test, stored per axis in the working type.
template <typename R>
__global__ void __launch_bounds__(256) k_nl_disp(NLGeo G, const double* __restrict__ pos,
                                                 const int64_t* __restrict__ off, const int32_t* __restrict__ idx,
                                                 int64_t n_list, R* __restrict__ disp) {
    const int a = blockIdx.x;
    const double px = pos[3 * a], py = pos[3 * a + 1], pz = pos[3 * a + 2];
    for (int64_t q = off[a] + threadIdx.x; q < off[a + 1]; q += blockDim.x) {
        const int g = idx[q];
        const int x = g % G.n[0], y = (g / G.n[0]) % G.n[1], z = g / (G.n[0] * G.n[1]);
        disp[q] = (R)min_image(x, G.h, px, G.L[0]);
        disp[n_list + q] = (R)min_image(y, G.h, py, G.L[1]);
        disp[2 * n_list + q] = (R)min_image(z, G.h, pz, G.L[2]);
    }
}

// pq[e] = the atom-list entry of per-point entry e: the position of point g
// in its atom's list (ascending), found by bisection.
__global__ void k_nl_pq(int64_t ng, const int32_t* __restrict__ pstart, const int32_t* __restrict__ patom,
                        const int64_t* __restrict__ off, const int32_t* __restrict__ idx, int32_t* __restrict__ pq) {
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < ng; g += (int64_t)gridDim.x * blockDim.x) {
        for (int e = pstart[g]; e < pstart[g + 1]; ++e) {
            const int a = patom[e];
            int64_t lo = off[a], hi = off[a + 1] - 1;
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if (idx[mid] < g) lo = mid + 1; else hi = mid;
            }
            pq[e] = (int32_t)lo;
        }
    }
}

// Phases of step k: theta = A_k . (r - R_a) in FP64;
// ph_at[q] = e^{+i theta_q} (projection, atom-list order) and
// ph_pt[e] = e^{-i theta_pq[e]} (scatter, per-point order).
template <typename R>
__global__ void __launch_bounds__(256) k_nl_phase(int64_t n_list, const R* __restrict__ disp,
                                                  const int32_t* __restrict__ pq, const double* __restrict__ Ak,
                                                  R* __restrict__ ph_at, R* __restrict__ ph_pt) {
    const double A0 = Ak[0], A1 = Ak[1], A2 = Ak[2];
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n_list; q += (int64_t)gridDim.x * blockDim.x) {
        double sn, cs;
        const double th = A0 * (double)disp[q] + A1 * (double)disp[n_list + q] + A2 * (double)disp[2 * n_list + q];
        sincos(th, &sn, &cs);
        ph_at[2 * q] = (R)cs;
        ph_at[2 * q + 1] = (R)sn;
        const int64_t r = pq[q];
        const double tr = A0 * (double)disp[r] + A1 * (double)disp[n_list + r] + A2 * (double)disp[2 * n_list + r];
        sincos(tr, &sn, &cs);
        ph_pt[2 * q] = (R)cs;
        ph_pt[2 * q + 1] = (R)(-sn);
    }
}

// Nonlocal commutator current (one block): row[2 + x] +=
//   sum_(r,o) f_o D_r 2 Re(i conj(P_ro) Q^x_ro) = -2 sum f_o D_r (Pre Q^x_im - Pim Q^x_re)
// over projector rows r = (atom, i) and orbitals o, summed in FP64.
template <typename R>
__global__ void __launch_bounds__(1024) k_nl_current(const R* __restrict__ P, const R* __restrict__ Q, int64_t qstride,
                                                     const double* __restrict__ D, const double* __restrict__ f,
                                                     int n_rows, int ld, int n_orb, double* __restrict__ row) {
    double s[3] = {0.0, 0.0, 0.0};
    const int64_t n = (int64_t)n_rows * n_orb;
    for (int64_t t = threadIdx.x; t < n; t += blockDim.x) {
        const int r = (int)(t / n_orb);
        const int o = (int)(t - (int64_t)r * n_orb);
        const int64_t e = ((int64_t)r * ld + o) * 2;
        const double pr = (double)P[e], pi = (double)P[e + 1];
        const double w = -2.0 * f[o] * D[r];
#pragma unroll
        for (int ax = 0; ax < 3; ++ax)
            s[ax] += w * (pr * (double)Q[ax * qstride + e + 1] - pi * (double)Q[ax * qstride + e]);
    }
    __shared__ double red[3][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        for (int o = 16; o > 0; o >>= 1) s[ax] += __shfl_xor_sync(0xffffffffu, s[ax], o);
        if (lane == 0) red[ax][warp] = s[ax];
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = (int)(blockDim.x >> 5);
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            double t = lane < nw ? red[ax][lane] : 0.0;
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (lane == 0) row[2 + ax] += t;
        }
    }
}

// ---- projection -----------------------------------------------------------
template <typename R> struct V16;
template <> struct V16<float> { static constexpr int NC = 2; };
template <> struct V16<double> { static constexpr int NC = 1; };

// Block (segment s, atom a, orbital chunk c): thread j owns one 16-byte
// vector of the orbital row; loops over the segment's points and keeps the
// NP projections in registers.  Pseg[s][a][i][o] = sum_{q in seg} beta[q][i] w[idx[q]][o].
// GAUGE: each row is first multiplied by the complex phase ph[q] (and by the
// displacement component mom[q] when mom is set).
template <typename R, int NP, bool GAUGE>
__global__ void __launch_bounds__(128) k_project(const R* __restrict__ w, int ld, int nv,
                                                 const int64_t* __restrict__ off,
                                                 const int32_t* __restrict__ idx, const R* __restrict__ beta,
                                                 const R* __restrict__ ph, const R* __restrict__ mom,
                                                 int seg_len, int n_atoms, R* __restrict__ Pseg) {
    constexpr int NC = V16<R>::NC;
    const int s = blockIdx.x, a = blockIdx.y;
    const int j = blockIdx.z * blockDim.x + threadIdx.x;
    const int64_t q0 = off[a] + (int64_t)s * seg_len;
    const int64_t q1 = min(off[a + 1], q0 + seg_len);
    R acc[NP][2 * NC];
#pragma unroll
    for (int i = 0; i < NP; ++i)
#pragma unroll
        for (int k = 0; k < 2 * NC; ++k) acc[i][k] = 0;
    if (j < nv) {
        // two points at a time: both rows and both beta vectors are in
        // flight before either is used
        for (int64_t q = q0; q < q1; q += 2) {
            const bool two = q + 1 < q1;
            R v[2][2 * NC], b[2][NP], pc[2], ps[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                if (u == 1 && !two) break;
                if constexpr (GAUGE) {
                    pc[u] = ph[2 * (q + u)];
                    ps[u] = ph[2 * (q + u) + 1];
                    if (mom) {
                        const R m = mom[q + u];
                        pc[u] *= m;
                        ps[u] *= m;
                    }
                }
                const R* row = w + ((int64_t)idx[q + u] * ld + (int64_t)j * NC) * 2;
                if (NC == 2) {
                    const float4 t = __ldg(reinterpret_cast<const float4*>(row));
                    v[u][0] = t.x; v[u][1] = t.y; v[u][2 % (2 * NC)] = t.z; v[u][3 % (2 * NC)] = t.w;
                } else {
                    const double2 t = __ldg(reinterpret_cast<const double2*>(row));
                    v[u][0] = t.x; v[u][1] = t.y;
                }
#pragma unroll
                for (int i = 0; i < NP; ++i) b[u][i] = __ldg(beta + (q + u) * NP + i);
            }
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                if (u == 1 && !two) break;
                if constexpr (GAUGE) {
#pragma unroll
                    for (int k = 0; k < NC; ++k) {
                        const R vr = v[u][2 * k], vi = v[u][2 * k + 1];
                        v[u][2 * k] = pc[u] * vr - ps[u] * vi;
                        v[u][2 * k + 1] = pc[u] * vi + ps[u] * vr;
                    }
                }
#pragma unroll
                for (int i = 0; i < NP; ++i)
#pragma unroll
                    for (int k = 0; k < 2 * NC; ++k) acc[i][k] += b[u][i] * v[u][k];
            }
        }
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            R* dst = Pseg + ((((int64_t)s * n_atoms + a) * NP + i) * ld + (int64_t)j * NC) * 2;
#pragma unroll
            for (int k = 0; k < 2 * NC; ++k) dst[k] = acc[i][k];
        }
    }
}

// P[e] = dV * sum_s Pseg[s][e] over the flattened [n_atoms][NP][ld] complex.
template <typename R>
__global__ void k_project_reduce(const R* __restrict__ Pseg, int n_seg, int64_t n_real, R dV, R* __restrict__ P) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n_real; e += (int64_t)gridDim.x * blockDim.x) {
        R s = 0;
        for (int k = 0; k < n_seg; ++k) s += Pseg[(int64_t)k * n_real + e];
        P[e] = dV * s;
    }
}

}  // namespace

void build_projectors(Domain& d, int n_atoms, const double* pos_host, int n_proj, double r_c, double r_cut,
                      const double* D_host) {
    Nonlocal& nl = d.nl;
    // drop the previous tables
    gauge_release(d);
    for (void* p : {(void*)nl.off, (void*)nl.idx, (void*)nl.beta64, nl.beta, (void*)nl.pstart, (void*)nl.patom,
                    nl.pbd, (void*)nl.D, d.Pa, d.Pb, d.Pseg})
        if (p) d.mem.put(p);
    nl = Nonlocal{};
    d.Pa = d.Pb = d.Pseg = nullptr;
    d.pa_psi = false;
    nl_tc_release(d);
    if (n_atoms == 0) {
        tma_build_nl(d, nullptr);
        return;
    }
    for (int ax = 0; ax < 3; ++ax)
        MLMD_REQUIRE(d.desc.n[ax] <= kMaxAxis, MLMD_ERR_UNSUPPORTED, "projectors need n <= 1024 per axis");
    const cudaStream_t st = d.stream;
    NLGeo G;
    for (int ax = 0; ax < 3; ++ax) {
        G.n[ax] = d.desc.n[ax];
        G.L[ax] = (double)d.desc.n[ax] * d.desc.h;
    }
    G.h = d.desc.h;
    G.rc2 = r_cut * r_cut;
    G.m = (int)floor(r_cut / d.desc.h) + 2;

    double* pos = (double*)d.mem.get(sizeof(double) * 3 * n_atoms);
    nl.D = (double*)d.mem.get(sizeof(double) * n_atoms * n_proj);
    MLMD_CUDA(cudaMemcpyAsync(pos, pos_host, sizeof(double) * 3 * n_atoms, cudaMemcpyHostToDevice, st));
    MLMD_CUDA(cudaMemcpyAsync(nl.D, D_host, sizeof(double) * n_atoms * n_proj, cudaMemcpyHostToDevice, st));
    int64_t* counts = (int64_t*)d.mem.get(sizeof(int64_t) * n_atoms);
    k_nl_lists<<<n_atoms, 256, 0, st>>>(G, pos, nullptr, counts, nullptr);
    d.launches++;
    MLMD_CUDA(cudaGetLastError());
    std::vector<int64_t> hc(n_atoms);
    MLMD_CUDA(cudaMemcpyAsync(hc.data(), counts, sizeof(int64_t) * n_atoms, cudaMemcpyDeviceToHost, st));
    MLMD_CUDA(cudaStreamSynchronize(st));
    nl.h_off.assign(n_atoms + 1, 0);
    for (int a = 0; a < n_atoms; ++a) {
        nl.h_off[a + 1] = nl.h_off[a] + hc[a];
        nl.max_count = std::max<int>(nl.max_count, (int)hc[a]);
    }
    nl.n_atoms = n_atoms;
    nl.n_proj = n_proj;
    nl.n_list = nl.h_off[n_atoms];
    nl.h_pos.assign(pos_host, pos_host + 3 * (size_t)n_atoms);
    MLMD_REQUIRE(nl.n_list < (int64_t)INT32_MAX, MLMD_ERR_UNSUPPORTED, "projector lists too long");
    const int64_t nlist = std::max<int64_t>(nl.n_list, 1);
    nl.off = (int64_t*)d.mem.get(sizeof(int64_t) * (n_atoms + 1));
    nl.idx = (int32_t*)d.mem.get(sizeof(int32_t) * nlist);
    nl.beta64 = (double*)d.mem.get(sizeof(double) * nlist * n_proj);
    MLMD_CUDA(cudaMemcpyAsync(nl.off, nl.h_off.data(), sizeof(int64_t) * (n_atoms + 1), cudaMemcpyHostToDevice, st));
    k_nl_lists<<<n_atoms, 256, 0, st>>>(G, pos, nl.off, nullptr, nl.idx);
    d.launches++;
    MLMD_CUDA(cudaGetLastError());
    const double dV = d.desc.h * d.desc.h * d.desc.h;
    k_nl_values<<<n_atoms, 256, 0, st>>>(G, pos, nl.off, nl.idx, n_proj, r_c, dV, nl.beta64);
    d.launches++;
    MLMD_CUDA(cudaGetLastError());

    // working-type copy of beta for the projection
    const size_t rsz = d.c64() ? sizeof(float) : sizeof(double);
    nl.beta = d.mem.get(rsz * nlist * n_proj);
    if (d.c64()) k_cast<float><<<256, 256, 0, st>>>(nl.beta64, nl.n_list * n_proj, (float*)nl.beta);
    else k_cast<double><<<256, 256, 0, st>>>(nl.beta64, nl.n_list * n_proj, (double*)nl.beta);
    d.launches++;

    // per-point transpose
    int32_t* cnt = (int32_t*)d.mem.get(sizeof(int32_t) * d.ng);
    int32_t* cursor = (int32_t*)d.mem.get(sizeof(int32_t) * d.ng);
    nl.pstart = (int32_t*)d.mem.get(sizeof(int32_t) * (d.ng + 1));
    int32_t* ent_q = (int32_t*)d.mem.get(sizeof(int32_t) * nlist);
    nl.patom = (int32_t*)d.mem.get(sizeof(int32_t) * nlist);
    nl.pbd = d.mem.get(rsz * nlist * n_proj);
    MLMD_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * d.ng, st));
    MLMD_CUDA(cudaMemsetAsync(cursor, 0, sizeof(int32_t) * d.ng, st));
    k_pt_count<<<512, 256, 0, st>>>(nl.idx, nl.n_list, cnt);
    k_scan<<<1, 1024, 0, st>>>(cnt, d.ng, nl.pstart);
    k_pt_fill<<<n_atoms, 256, 0, st>>>(nl.off, nl.idx, nl.pstart, cursor, ent_q);
    if (d.c64())
        k_pt_finish<float><<<(int)((d.ng + 255) / 256), 256, 0, st>>>(d.ng, nl.pstart, ent_q, nl.off, n_atoms, nl.beta64,
                                                                     nl.D, n_proj, nl.patom, (float*)nl.pbd);
    else
        k_pt_finish<double><<<(int)((d.ng + 255) / 256), 256, 0, st>>>(d.ng, nl.pstart, ent_q, nl.off, n_atoms,
                                                                      nl.beta64, nl.D, n_proj, nl.patom, (double*)nl.pbd);
    d.launches += 4;
    MLMD_CUDA(cudaGetLastError());

    // projection buffers
    nl.seg_len = 256;
    nl.n_seg = std::max(1, (nl.max_count + nl.seg_len - 1) / nl.seg_len);
    const size_t pbytes = (size_t)n_atoms * n_proj * d.ld * d.elem;
    d.Pa = d.mem.get(pbytes);
    d.Pb = d.mem.get(pbytes);
    d.Pseg = d.mem.get(pbytes * nl.n_seg);
    MLMD_CUDA(cudaStreamSynchronize(st));
    d.mem.put(pos);
    d.mem.put(counts);
    d.mem.put(cnt);
    d.mem.put(cursor);
    d.mem.put(ent_q);
    tma_build_nl(d, D_host);
    nl_tc_build(d, pos_host, r_c, D_host);
    if (d.nl_gauge == MLMD_NL_GAUGE_VELOCITY) gauge_build(d);
}

void gauge_release(Domain& d) {
    Nonlocal& nl = d.nl;
    for (void* p : {nl.disp, (void*)nl.pq, nl.ph_at, nl.ph_pt, nl.Qm})
        if (p) d.mem.put(p);
    nl.disp = nl.ph_at = nl.ph_pt = nl.Qm = nullptr;
    nl.pq = nullptr;
}

void gauge_build(Domain& d) {
    gauge_release(d);
    if (!d.has_nl()) return;
    Nonlocal& nl = d.nl;
    const cudaStream_t st = d.stream;
    NLGeo G{};
    for (int ax = 0; ax < 3; ++ax) {
        G.n[ax] = d.desc.n[ax];
        G.L[ax] = (double)d.desc.n[ax] * d.desc.h;
    }
    G.h = d.desc.h;
    const size_t rsz = d.c64() ? sizeof(float) : sizeof(double);
    const int64_t nlist = std::max<int64_t>(nl.n_list, 1);
    nl.disp = d.mem.get(rsz * 3 * nlist);
    nl.pq = (int32_t*)d.mem.get(sizeof(int32_t) * nlist);
    nl.ph_at = d.mem.get(rsz * 2 * nlist);
    nl.ph_pt = d.mem.get(rsz * 2 * nlist);
    nl.Qm = d.mem.get((size_t)3 * nl.n_atoms * nl.n_proj * d.ld * d.elem);
    double* pos = (double*)d.mem.get(sizeof(double) * 3 * nl.n_atoms);
    MLMD_CUDA(cudaMemcpyAsync(pos, nl.h_pos.data(), sizeof(double) * 3 * nl.n_atoms, cudaMemcpyHostToDevice, st));
    if (d.c64()) k_nl_disp<float><<<nl.n_atoms, 256, 0, st>>>(G, pos, nl.off, nl.idx, nl.n_list, (float*)nl.disp);
    else k_nl_disp<double><<<nl.n_atoms, 256, 0, st>>>(G, pos, nl.off, nl.idx, nl.n_list, (double*)nl.disp);
    k_nl_pq<<<(int)std::min<int64_t>((d.ng + 255) / 256, 152 * 16), 256, 0, st>>>(d.ng, nl.pstart, nl.patom, nl.off,
                                                                                   nl.idx, nl.pq);
    d.launches += 2;
    MLMD_CUDA(cudaGetLastError());
    MLMD_CUDA(cudaStreamSynchronize(st));
    d.mem.put(pos);
}

void launch_nl_phase(Domain& d, const double* Ak) {
    const Nonlocal& nl = d.nl;
    MLMD_REQUIRE(nl.ph_at != nullptr, MLMD_ERR_STATE, "velocity-gauge tables missing");
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((nl.n_list + 255) / 256, 152 * 8));
    if (d.c64())
        k_nl_phase<float><<<blocks, 256, 0, d.stream>>>(nl.n_list, (const float*)nl.disp, nl.pq, Ak,
                                                        (float*)nl.ph_at, (float*)nl.ph_pt);
    else
        k_nl_phase<double><<<blocks, 256, 0, d.stream>>>(nl.n_list, (const double*)nl.disp, nl.pq, Ak,
                                                         (double*)nl.ph_at, (double*)nl.ph_pt);
    d.launches++;
    MLMD_CUDA(cudaGetLastError());
}

void* moment_buffer(Domain& d, int ax) {
    const size_t bytes = (size_t)d.nl.n_atoms * d.nl.n_proj * d.ld * d.elem;
    return static_cast<char*>(d.nl.Qm) + bytes * ax;
}

void launch_nl_current(Domain& d, const void* P, double* obs_row) {
    const Nonlocal& nl = d.nl;
    const int n_rows = nl.n_atoms * nl.n_proj;
    const int64_t qstride = (int64_t)n_rows * d.ld * 2;
    if (d.c64())
        k_nl_current<float><<<1, 1024, 0, d.stream>>>((const float*)P, (const float*)nl.Qm, qstride, nl.D, d.f, n_rows,
                                                      d.ld, d.desc.n_orb, obs_row);
    else
        k_nl_current<double><<<1, 1024, 0, d.stream>>>((const double*)P, (const double*)nl.Qm, qstride, nl.D, d.f,
                                                       n_rows, d.ld, d.desc.n_orb, obs_row);
    d.launches++;
    MLMD_CUDA(cudaGetLastError());
}

void launch_project(Domain& d, const void* w, void* P, int moment_axis) {
    const Nonlocal& nl = d.nl;
    const bool gauge = gauge_on(d);
    MLMD_REQUIRE(gauge || moment_axis < 0, MLMD_ERR_STATE, "moment projection without velocity-gauge tables");
    const int nv = d.c64() ? d.ld / 2 : d.ld;
    const int bx = std::min(nv, 128);
    dim3 grid(nl.n_seg, nl.n_atoms, (nv + bx - 1) / bx);
    const int64_t n_real = (int64_t)nl.n_atoms * nl.n_proj * d.ld * 2;
    const double dV = d.desc.h * d.desc.h * d.desc.h;
    const int rb = (int)std::min<int64_t>((n_real + 255) / 256, 152 * 8);
    ProfScope ps(d.prof, MLMD_KERNEL_PROJECT, d.stream);
    auto run = [&](auto zero) {
        using R = decltype(zero);
        const R* ph = static_cast<const R*>(nl.ph_at);
        const R* mom = moment_axis >= 0 ? static_cast<const R*>(nl.disp) + (int64_t)moment_axis * nl.n_list : nullptr;
        const R* beta = static_cast<const R*>(nl.beta);
        R* seg = static_cast<R*>(d.Pseg);
        const R* wr = static_cast<const R*>(w);
        if (nl.n_proj == 4) {
            if (gauge) k_project<R, 4, true><<<grid, bx, 0, d.stream>>>(wr, d.ld, nv, nl.off, nl.idx, beta, ph, mom,
                                                                        nl.seg_len, nl.n_atoms, seg);
            else k_project<R, 4, false><<<grid, bx, 0, d.stream>>>(wr, d.ld, nv, nl.off, nl.idx, beta, nullptr, nullptr,
                                                                   nl.seg_len, nl.n_atoms, seg);
        } else {
            if (gauge) k_project<R, 8, true><<<grid, bx, 0, d.stream>>>(wr, d.ld, nv, nl.off, nl.idx, beta, ph, mom,
                                                                        nl.seg_len, nl.n_atoms, seg);
            else k_project<R, 8, false><<<grid, bx, 0, d.stream>>>(wr, d.ld, nv, nl.off, nl.idx, beta, nullptr, nullptr,
                                                                   nl.seg_len, nl.n_atoms, seg);
        }
        k_project_reduce<R><<<rb, 256, 0, d.stream>>>(seg, nl.n_seg, n_real, (R)dV, static_cast<R*>(P));
    };
    if (d.c64()) run(0.0f);
    else run(0.0);
    d.launches += 2;
    MLMD_CUDA(cudaGetLastError());
}

}  // namespace mlmd
