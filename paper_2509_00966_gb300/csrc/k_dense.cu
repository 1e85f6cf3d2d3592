// Dense orbital-space algebra: the overlap (Gram) product Psi^dagger Psi of
// Eq. 5, the update Psi <- Psi M, and the FP64 factorisations used for
// re-orthonormalisation (Cholesky with L^{-H}, Loewdin S^{-1/2}).
#include <algorithm>
#include <cmath>

#include "mlmd_internal.cuh"

namespace mlmd {
namespace {

// ---- overlap: S[n][m] = scale * sum_g conj(X[g][n]) Y[g][m] ----------------
// Block tile 32x32 of (n, m), 256 threads, each owning a 2x2 sub-tile; the
// grid-point loop is split across blockIdx.z.  Products accumulate in the
// working type over 256 points, then in FP64.
template <typename R>
__global__ void __launch_bounds__(256) k_overlap(const R* __restrict__ X, const R* __restrict__ Y, int64_t ng, int ld,
                                                 int n_orb, int64_t kchunk, double* __restrict__ part) {
    __shared__ R xs[32][33][2];
    __shared__ R ys[32][33][2];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int n0 = blockIdx.y * 32, m0 = blockIdx.x * 32;
    const int64_t g0 = blockIdx.z * kchunk;
    const int64_t g1 = std::min<int64_t>(ng, g0 + kchunk);
    double acc[2][2][2] = {};
    R racc[2][2][2] = {};
    int cnt = 0;
    for (int64_t gb = g0; gb < g1; gb += 32) {
        for (int e = threadIdx.x; e < 32 * 32; e += 256) {
            const int r = e >> 5, c = e & 31;
            const int64_t g = gb + r;
            R xr = 0, xi = 0, yr = 0, yi = 0;
            if (g < g1) {
                if (n0 + c < n_orb) { xr = X[(g * ld + n0 + c) * 2]; xi = X[(g * ld + n0 + c) * 2 + 1]; }
                if (m0 + c < n_orb) { yr = Y[(g * ld + m0 + c) * 2]; yi = Y[(g * ld + m0 + c) * 2 + 1]; }
            }
            xs[r][c][0] = xr; xs[r][c][1] = xi;
            ys[r][c][0] = yr; ys[r][c][1] = yi;
        }
        __syncthreads();
#pragma unroll 8
        for (int r = 0; r < 32; ++r) {
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                const R xr = xs[r][ty + 16 * a][0], xi = xs[r][ty + 16 * a][1];
#pragma unroll
                for (int b = 0; b < 2; ++b) {
                    const R yr = ys[r][tx + 16 * b][0], yi = ys[r][tx + 16 * b][1];
                    // conj(x) * y
                    racc[a][b][0] += xr * yr + xi * yi;
                    racc[a][b][1] += xr * yi - xi * yr;
                }
            }
        }
        __syncthreads();
        if (++cnt == 8) {
            for (int a = 0; a < 2; ++a)
                for (int b = 0; b < 2; ++b)
                    for (int k = 0; k < 2; ++k) { acc[a][b][k] += (double)racc[a][b][k]; racc[a][b][k] = 0; }
            cnt = 0;
        }
    }
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            const int n = n0 + ty + 16 * a, m = m0 + tx + 16 * b;
            if (n < n_orb && m < n_orb) {
                double* dst = part + (((int64_t)blockIdx.z * n_orb + n) * n_orb + m) * 2;
                dst[0] = acc[a][b][0] + (double)racc[a][b][0];
                dst[1] = acc[a][b][1] + (double)racc[a][b][1];
            }
        }
}

__global__ void k_overlap_reduce(const double* __restrict__ part, int nsplit, int64_t n, double scale,
                                 double* __restrict__ S) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int k = 0; k < nsplit; ++k) s += part[(int64_t)k * n + e];
        S[e] = scale * s;
    }
}

// ---- update: Y[g][m] = sum_n X[g][n] M[n][m] -------------------------------
// Block tile 64 points x 32 orbitals, 256 threads; thread (ty, tx) owns the
// points ty + 16 a (a < 4) and the orbitals tx + 16 b (b < 2) of the tile.
template <typename R>
__global__ void __launch_bounds__(256) k_update(const R* __restrict__ X, const double* __restrict__ M, int64_t ng,
                                                int ld, int n_orb, R* __restrict__ Y) {
    __shared__ R xs[64][33][2];
    __shared__ R ms[32][33][2];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t gb = blockIdx.y * (int64_t)64;
    const int m0 = blockIdx.x * 32;
    R acc[4][2][2] = {};
    for (int n0 = 0; n0 < n_orb; n0 += 32) {
        for (int e = threadIdx.x; e < 64 * 32; e += 256) {
            const int r = e >> 5, c = e & 31;
            const int64_t g = gb + r;
            R xr = 0, xi = 0;
            if (g < ng && n0 + c < n_orb) { xr = X[(g * ld + n0 + c) * 2]; xi = X[(g * ld + n0 + c) * 2 + 1]; }
            xs[r][c][0] = xr; xs[r][c][1] = xi;
        }
        for (int e = threadIdx.x; e < 32 * 32; e += 256) {
            const int r = e >> 5, c = e & 31;
            R mr = 0, mi = 0;
            if (n0 + r < n_orb && m0 + c < n_orb) {
                mr = (R)M[((int64_t)(n0 + r) * n_orb + m0 + c) * 2];
                mi = (R)M[((int64_t)(n0 + r) * n_orb + m0 + c) * 2 + 1];
            }
            ms[r][c][0] = mr; ms[r][c][1] = mi;
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < 32; ++k) {
            R mr[2], mi[2];
#pragma unroll
            for (int b = 0; b < 2; ++b) { mr[b] = ms[k][tx + 16 * b][0]; mi[b] = ms[k][tx + 16 * b][1]; }
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const R xr = xs[ty + 16 * a][k][0], xi = xs[ty + 16 * a][k][1];
#pragma unroll
                for (int b = 0; b < 2; ++b) {
                    acc[a][b][0] += xr * mr[b] - xi * mi[b];
                    acc[a][b][1] += xr * mi[b] + xi * mr[b];
                }
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int64_t g = gb + ty + 16 * a;
            const int m = m0 + tx + 16 * b;
            if (g < ng && m < ld) {
                Y[(g * ld + m) * 2] = m < n_orb ? acc[a][b][0] : (R)0;
                Y[(g * ld + m) * 2 + 1] = m < n_orb ? acc[a][b][1] : (R)0;
            }
        }
}

// ---- FP64 complex Cholesky, column by column (right-looking) ----------------
// S is row-major complex [n][n]; on exit its lower triangle holds L.
__global__ void k_chol_col(double* __restrict__ S, int n, int j, int* __restrict__ info) {
    __shared__ double dj;
    if (threadIdx.x == 0) {
        const double a = S[((int64_t)j * n + j) * 2];
        if (!(a > 0.0) || !isfinite(a)) { if (*info == 0) *info = j + 1; dj = 1.0; }
        else dj = sqrt(a);
        S[((int64_t)j * n + j) * 2] = dj;
        S[((int64_t)j * n + j) * 2 + 1] = 0.0;
    }
    __syncthreads();
    const double inv = 1.0 / dj;
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) {
        S[((int64_t)i * n + j) * 2] *= inv;
        S[((int64_t)i * n + j) * 2 + 1] *= inv;
    }
}

// S[i][k] -= L[i][j] conj(L[k][j]) for j < k <= i
__global__ void k_chol_update(double* __restrict__ S, int n, int j) {
    const int i = j + 1 + blockIdx.y * blockDim.y + threadIdx.y;
    const int k = j + 1 + blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || k > i) return;
    const double ar = S[((int64_t)i * n + j) * 2], ai = S[((int64_t)i * n + j) * 2 + 1];
    const double br = S[((int64_t)k * n + j) * 2], bi = -S[((int64_t)k * n + j) * 2 + 1];
    S[((int64_t)i * n + k) * 2] -= ar * br - ai * bi;
    S[((int64_t)i * n + k) * 2 + 1] -= ar * bi + ai * br;
}

// Row i of X = L^{-1} by forward substitution: X[i][c] = (delta_ic - sum_{c<=k<i} L[i][k] X[k][c]) / L[i][i]
__global__ void k_trinv_row(const double* __restrict__ L, double* __restrict__ X, int n, int i) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        double sr = (c == i) ? 1.0 : 0.0, si = 0.0;
        if (c < i) {
            for (int k = c; k < i; ++k) {
                const double lr = L[((int64_t)i * n + k) * 2], li = L[((int64_t)i * n + k) * 2 + 1];
                const double xr = X[((int64_t)k * n + c) * 2], xi = X[((int64_t)k * n + c) * 2 + 1];
                sr -= lr * xr - li * xi;
                si -= lr * xi + li * xr;
            }
        }
        const double d = L[((int64_t)i * n + i) * 2];
        X[((int64_t)i * n + c) * 2] = c <= i ? sr / d : 0.0;
        X[((int64_t)i * n + c) * 2 + 1] = c <= i ? si / d : 0.0;
    }
}

// Minv[r][c] = conj(X[c][r])
__global__ void k_conj_transpose(const double* __restrict__ X, int n, double* __restrict__ Y) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * n; e += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / n), c = (int)(e % n);
        Y[e * 2] = X[((int64_t)c * n + r) * 2];
        Y[e * 2 + 1] = -X[((int64_t)c * n + r) * 2 + 1];
    }
}

// ---- FP64 complex GEMM for Newton-Schulz: C = alpha A B + beta_diag I ------
__global__ void k_zgemm(const double* __restrict__ A, const double* __restrict__ B, int n, double alpha,
                        double diag, double* __restrict__ C) {
    __shared__ double as[16][17][2], bs[16][17][2];
    const int r = blockIdx.y * 16 + threadIdx.y, c = blockIdx.x * 16 + threadIdx.x;
    double sr = 0.0, si = 0.0;
    for (int k0 = 0; k0 < n; k0 += 16) {
        const int ka = k0 + threadIdx.x, kb = k0 + threadIdx.y;
        as[threadIdx.y][threadIdx.x][0] = (r < n && ka < n) ? A[((int64_t)r * n + ka) * 2] : 0.0;
        as[threadIdx.y][threadIdx.x][1] = (r < n && ka < n) ? A[((int64_t)r * n + ka) * 2 + 1] : 0.0;
        bs[threadIdx.y][threadIdx.x][0] = (kb < n && c < n) ? B[((int64_t)kb * n + c) * 2] : 0.0;
        bs[threadIdx.y][threadIdx.x][1] = (kb < n && c < n) ? B[((int64_t)kb * n + c) * 2 + 1] : 0.0;
        __syncthreads();
        for (int k = 0; k < 16; ++k) {
            const double ar = as[threadIdx.y][k][0], ai = as[threadIdx.y][k][1];
            const double br = bs[k][threadIdx.x][0], bi = bs[k][threadIdx.x][1];
            sr += ar * br - ai * bi;
            si += ar * bi + ai * br;
        }
        __syncthreads();
    }
    if (r < n && c < n) {
        C[((int64_t)r * n + c) * 2] = alpha * sr + (r == c ? diag : 0.0);
        C[((int64_t)r * n + c) * 2 + 1] = alpha * si;
    }
}

__global__ void k_identity(double* __restrict__ X, int n) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * n; e += (int64_t)gridDim.x * blockDim.x) {
        X[e * 2] = (e / n == e % n) ? 1.0 : 0.0;
        X[e * 2 + 1] = 0.0;
    }
}

// ||I - Z Y||_max into err (FP64), for the Newton-Schulz stopping test.
__global__ void k_offdiag_err(const double* __restrict__ T, int n, double* __restrict__ err) {
    double m = 0.0;
    for (int64_t e = threadIdx.x; e < (int64_t)n * n; e += blockDim.x) {
        const double re = T[e * 2] - ((e / n == e % n) ? 1.0 : 0.0), im = T[e * 2 + 1];
        m = fmax(m, fabs(re) + fabs(im));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ double sh[32];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmax(t, sh[w]);
        *err = t;
    }
}

}  // namespace

void launch_overlap(Domain& d, const void* X, const void* Y, double scale, double* S) {
    if (launch_overlap_tc(d, X, Y, scale, S)) return;    // tensor cores for the 16-bit GEMM modes
    const int no = d.desc.n_orb;
    const int tiles = (no + 31) / 32;
    // split the grid so that the launch fills the GPU
    int64_t nsplit = std::max<int64_t>(1, std::min<int64_t>((152 * 8) / (tiles * tiles) + 1, (d.ng + 255) / 256));
    const int64_t kchunk = ((d.ng + nsplit - 1) / nsplit + 31) / 32 * 32;
    nsplit = (d.ng + kchunk - 1) / kchunk;
    const size_t need = (size_t)nsplit * no * no * 2 * sizeof(double);
    double* part = (double*)d.mem.get(need);
    dim3 grid(tiles, tiles, (unsigned)nsplit);
    if (d.c64())
        k_overlap<float><<<grid, 256, 0, d.stream>>>((const float*)X, (const float*)Y, d.ng, d.ld, no, kchunk, part);
    else
        k_overlap<double><<<grid, 256, 0, d.stream>>>((const double*)X, (const double*)Y, d.ng, d.ld, no, kchunk, part);
    const int64_t n = (int64_t)no * no * 2;
    k_overlap_reduce<<<(int)std::min<int64_t>((n + 255) / 256, 2048), 256, 0, d.stream>>>(part, (int)nsplit, n, scale, S);
    d.launches += 2;
    MLMD_CUDA(cudaGetLastError());
    d.mem.put(part);
}

void launch_update(Domain& d, const void* X, const double* M, void* Y) {
    const int no = d.desc.n_orb;
    dim3 grid((d.ld + 31) / 32, (unsigned)((d.ng + 63) / 64));
    if (d.c64()) k_update<float><<<grid, 256, 0, d.stream>>>((const float*)X, M, d.ng, d.ld, no, (float*)Y);
    else k_update<double><<<grid, 256, 0, d.stream>>>((const double*)X, M, d.ng, d.ld, no, (double*)Y);
    d.launches++;
    MLMD_CUDA(cudaGetLastError());
}

void cholesky_inverse_upper(Domain& d, double* S, double* Minv, int* d_info) {
    const int n = d.desc.n_orb;
    MLMD_CUDA(cudaMemsetAsync(d_info, 0, sizeof(int), d.stream));
    for (int j = 0; j < n; ++j) {
        k_chol_col<<<1, 256, 0, d.stream>>>(S, n, j, d_info);
        d.launches++;
        const int m = n - j - 1;
        if (m > 0) {
            dim3 blk(16, 16), grd((m + 15) / 16, (m + 15) / 16);
            k_chol_update<<<grd, blk, 0, d.stream>>>(S, n, j);
            d.launches++;
        }
    }
    // X = L^{-1} row by row into Minv's storage, then Minv = X^H
    double* X = (double*)d.mem.get((size_t)n * n * 2 * sizeof(double));
    for (int i = 0; i < n; ++i) {
        k_trinv_row<<<(n + 255) / 256, 256, 0, d.stream>>>(S, X, n, i);
        d.launches++;
    }
    k_conj_transpose<<<(int)std::min<int64_t>(((int64_t)n * n + 255) / 256, 4096), 256, 0, d.stream>>>(X, n, Minv);
    d.launches++;
    MLMD_CUDA(cudaGetLastError());
    d.mem.put(X);
}

void lowdin_inverse_sqrt(Domain& d, double* S, double* Minv, double* work, int* d_info) {
    // Coupled Newton-Schulz: Y0 = S, Z0 = I; T = (3I - Z Y)/2; Y <- Y T; Z <- T Z.
    // Z -> S^{-1/2} quadratically when ||I - S|| < 1.
    const int n = d.desc.n_orb;
    const size_t mat = (size_t)n * n * 2;
    double* Y = work;
    double* T = work + mat;
    double* W = work + 2 * mat;
    double* err = work + 3 * mat;
    MLMD_CUDA(cudaMemsetAsync(d_info, 0, sizeof(int), d.stream));
    MLMD_CUDA(cudaMemcpyAsync(Y, S, mat * sizeof(double), cudaMemcpyDeviceToDevice, d.stream));
    k_identity<<<256, 256, 0, d.stream>>>(Minv, n);
    d.launches++;
    dim3 blk(16, 16), grd((n + 15) / 16, (n + 15) / 16);
    double h_err = 1.0;
    for (int it = 0; it < 40 && h_err > 1e-14; ++it) {
        k_zgemm<<<grd, blk, 0, d.stream>>>(Minv, Y, n, -0.5, 1.5, T);   // T = 1.5 I - 0.5 Z Y
        k_zgemm<<<grd, blk, 0, d.stream>>>(Y, T, n, 1.0, 0.0, W);       // Y <- Y T
        MLMD_CUDA(cudaMemcpyAsync(Y, W, mat * sizeof(double), cudaMemcpyDeviceToDevice, d.stream));
        k_zgemm<<<grd, blk, 0, d.stream>>>(T, Minv, n, 1.0, 0.0, W);    // Z <- T Z
        MLMD_CUDA(cudaMemcpyAsync(Minv, W, mat * sizeof(double), cudaMemcpyDeviceToDevice, d.stream));
        k_zgemm<<<grd, blk, 0, d.stream>>>(Minv, Y, n, 1.0, 0.0, W);    // Z Y -> I
        k_offdiag_err<<<1, 1024, 0, d.stream>>>(W, n, err);
        d.launches += 5;
        MLMD_CUDA(cudaMemcpyAsync(&h_err, err, sizeof(double), cudaMemcpyDeviceToHost, d.stream));
        MLMD_CUDA(cudaStreamSynchronize(d.stream));
        MLMD_REQUIRE(std::isfinite(h_err) && h_err < 1.0, MLMD_ERR_NUMERIC,
                     "Loewdin iteration diverged (overlap too far from identity)");
    }
    MLMD_CUDA(cudaGetLastError());
}

}  // namespace mlmd
