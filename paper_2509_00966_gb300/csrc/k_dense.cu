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
                                                int ld, int n_orb, const R* __restrict__ Z, R* __restrict__ Y) {
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
                const R zr = Z ? Z[(g * ld + m) * 2] : (R)0, zi = Z ? Z[(g * ld + m) * 2 + 1] : (R)0;
                Y[(g * ld + m) * 2] = m < n_orb ? zr + acc[a][b][0] : (R)0;
                Y[(g * ld + m) * 2 + 1] = m < n_orb ? zi + acc[a][b][1] : (R)0;
            }
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

// ---- blocked FP64 complex Cholesky (panel width 32) ---------------------------
constexpr int CB = 32;

// Block column kb, diagonal block only (one CTA): A11 = L11 L11^H, right-
// looking in shared memory with all threads on each column's updates; L11
// goes to Ld[kb] (the side array the panel solve and the triangular inverse
// read, so that A11 in S stays untouched).  info > 0 marks a non-positive
// pivot.
__global__ void __launch_bounds__(256) k_chol_diag(const double* __restrict__ S, int n, int kb, double* __restrict__ Ld,
                                                   int* __restrict__ info) {
    __shared__ double L[CB][CB + 1][2];
    const int c0 = kb * CB;
    const int nb = min(CB, n - c0);
    for (int e = threadIdx.x; e < CB * CB; e += blockDim.x) {
        const int i = e / CB, j = e % CB;
        const bool in = i < nb && j < nb;
        L[i][j][0] = in ? S[((int64_t)(c0 + i) * n + c0 + j) * 2] : (i == j ? 1.0 : 0.0);
        L[i][j][1] = in ? S[((int64_t)(c0 + i) * n + c0 + j) * 2 + 1] : 0.0;
    }
    __shared__ double inv_sh;
    __syncthreads();
    for (int j = 0; j < nb; ++j) {
        if (threadIdx.x == 0) {           // one FP64 square root and reciprocal per pivot
            double a = L[j][j][0];
            if (!(a > 0.0) || !isfinite(a)) { atomicCAS(info, 0, c0 + j + 1); a = 1.0; }
            const double r = sqrt(a);
            L[j][j][0] = r;
            L[j][j][1] = 0.0;
            inv_sh = 1.0 / r;
        }
        __syncthreads();
        const double inv = inv_sh;
        for (int i = j + 1 + threadIdx.x; i < nb; i += blockDim.x) { L[i][j][0] *= inv; L[i][j][1] *= inv; }
        __syncthreads();
        const int m = nb - j - 1;
        for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
            const int i = j + 1 + e / m, k = j + 1 + e % m;
            if (k <= i) {
                const double ar = L[i][j][0], ai = L[i][j][1], br = L[k][j][0], bi = -L[k][j][1];
                L[i][k][0] -= ar * br - ai * bi;
                L[i][k][1] -= ar * bi + ai * br;
            }
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < CB * CB; e += blockDim.x) {
        const int i = e / CB, j = e % CB;
        Ld[((int64_t)kb * CB * CB + e) * 2] = (j <= i) ? L[i][j][0] : 0.0;
        Ld[((int64_t)kb * CB * CB + e) * 2 + 1] = (j <= i) ? L[i][j][1] : 0.0;
    }
}

// Panel rows below the diagonal block: x L11^H = a for every row, one warp
// per row with lane j holding column j: x_j = a_j / L_jj, then
// a_k -= x_j conj(L_kj) for k > j (the same operations per element as the
// right-looking block solve, without a block-wide barrier per column).
__global__ void __launch_bounds__(256) k_chol_rows(double* __restrict__ S, int n, int kb, const double* __restrict__ Ld) {
    __shared__ double L[CB][CB + 1][2];
    __shared__ double dinv[CB];
    const int c0 = kb * CB;
    const int nb = min(CB, n - c0);
    for (int e = threadIdx.x; e < CB * CB; e += blockDim.x) {
        const int i = e / CB, j = e % CB;
        L[i][j][0] = Ld[((int64_t)kb * CB * CB + e) * 2];
        L[i][j][1] = Ld[((int64_t)kb * CB * CB + e) * 2 + 1];
    }
    if (threadIdx.x < CB)
        dinv[threadIdx.x] = 1.0 / Ld[((int64_t)kb * CB * CB + threadIdx.x * CB + threadIdx.x) * 2];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int row = c0 + nb + blockIdx.x * (int)(blockDim.x >> 5) + (int)(threadIdx.x >> 5);
    if (row >= n) return;                           // whole warps leave together
    double* a = S + ((int64_t)row * n + c0) * 2;
    double ar = lane < nb ? a[lane * 2] : 0.0, ai = lane < nb ? a[lane * 2 + 1] : 0.0;
    for (int j = 0; j < nb; ++j) {
        if (lane == j) {
            ar *= dinv[j];
            ai *= dinv[j];
        }
        const double xr = __shfl_sync(0xffffffffu, ar, j), xi = __shfl_sync(0xffffffffu, ai, j);
        if (lane > j && lane < nb) {
            const double lr = L[lane][j][0], li = -L[lane][j][1];
            ar -= xr * lr - xi * li;
            ai -= xr * li + xi * lr;
        }
    }
    if (lane < nb) {
        a[lane * 2] = ar;
        a[lane * 2 + 1] = ai;
    }
}

// Trailing update after block column kb: S[i][k] -= sum_j L[i][j] conj(L[k][j])
// for i >= k >= (kb+1)*32 (lower triangle), j over the panel.  16 x 16 output
// tiles, one output per thread: the late panels' small trailing matrices
// still spread over many SMs (a 32 x 32 tile took ~55 us however few tiles
// a panel had).
constexpr int TT = 16;
// (tk0, ti0): first tile column and row of the launch, so that the next
// block column (tile columns 0 and 1) and the rest can go separately.
__global__ void __launch_bounds__(256) k_chol_trail(double* __restrict__ S, int n, int kb, int tk0, int ti0) {
    const int c0 = kb * CB, nb = min(CB, n - c0);
    const int base = c0 + nb;
    const int ti = ti0 + blockIdx.y, tk = tk0 + blockIdx.x;
    if (tk > ti) return;
    const int i0 = base + ti * TT, k0 = base + tk * TT;
    if (i0 >= n || k0 >= n) return;
    __shared__ double Li[TT][CB + 1][2], Lk[TT][CB + 1][2];
    for (int e = threadIdx.x; e < TT * CB; e += blockDim.x) {
        const int r = e / CB, j = e % CB;
        const bool ini = i0 + r < n && j < nb, ink = k0 + r < n && j < nb;
        Li[r][j][0] = ini ? S[((int64_t)(i0 + r) * n + c0 + j) * 2] : 0.0;
        Li[r][j][1] = ini ? S[((int64_t)(i0 + r) * n + c0 + j) * 2 + 1] : 0.0;
        Lk[r][j][0] = ink ? S[((int64_t)(k0 + r) * n + c0 + j) * 2] : 0.0;
        Lk[r][j][1] = ink ? S[((int64_t)(k0 + r) * n + c0 + j) * 2 + 1] : 0.0;
    }
    __syncthreads();
    const int r = threadIdx.x / TT, c = threadIdx.x % TT;
    const int i = i0 + r, k = k0 + c;
    if (i >= n || k >= n || k > i) return;
    double sr = 0.0, si = 0.0;
    for (int j = 0; j < nb; ++j) {
        const double ar = Li[r][j][0], ai = Li[r][j][1], br = Lk[c][j][0], bi = -Lk[c][j][1];
        sr += ar * br - ai * bi;
        si += ar * bi + ai * br;
    }
    S[((int64_t)i * n + k) * 2] -= sr;
    S[((int64_t)i * n + k) * 2 + 1] -= si;
}

// X = L^{-1} (lower), recursively by blocks.  First every 32 x 32 diagonal
// block X_ii = L_ii^{-1} (k_trinv_diag, from the stored L11 blocks); then for
// block size b = 32, 64, ...: pair p joins the finished inverses of
// A = [2pb, 2pb + b) and C = [2pb + b, 2pb + 2b) into one of size 2b through
//     X_CA = -X_CC (L_CA X_AA)
// (k_trinv_t: T = L_CA X_AA, then k_trinv_x: X_CA = -X_CC T), two batched
// GEMMs over all pairs of the level, each skipping the zero triangles.
__global__ void __launch_bounds__(256) k_trinv_diag(const double* __restrict__ Ld, double* __restrict__ X, int n) {
    __shared__ double Lb[CB][CB + 1][2];
    __shared__ double Xb[CB][CB + 1][2];
    const int kb = blockIdx.x, b0 = kb * CB, nb = min(CB, n - b0);
    for (int e = threadIdx.x; e < CB * CB; e += blockDim.x) {
        const int i = e / CB, j = e % CB;
        Lb[i][j][0] = Ld[((int64_t)kb * CB * CB + e) * 2];
        Lb[i][j][1] = Ld[((int64_t)kb * CB * CB + e) * 2 + 1];
        Xb[i][j][0] = (i == j) ? 1.0 : 0.0;     // right-hand sides: the identity
        Xb[i][j][1] = 0.0;
    }
    __syncthreads();
    // forward substitution on all 32 columns at once: row i of X is final
    // after step i, then rows below take their update
    for (int i = 0; i < CB; ++i) {
        const double dinv = 1.0 / Lb[i][i][0];
        if (threadIdx.x < CB) { Xb[i][threadIdx.x][0] *= dinv; Xb[i][threadIdx.x][1] *= dinv; }
        __syncthreads();
        const int m = CB - i - 1;
        for (int e = threadIdx.x; e < m * CB; e += blockDim.x) {
            const int r = i + 1 + e / CB, c = e % CB;
            const double lr = Lb[r][i][0], li = Lb[r][i][1], xr = Xb[i][c][0], xi = Xb[i][c][1];
            Xb[r][c][0] -= lr * xr - li * xi;
            Xb[r][c][1] -= lr * xi + li * xr;
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
        const int i = e / nb, c = e % nb;
        X[((int64_t)(b0 + i) * n + b0 + c) * 2] = Xb[i][c][0];
        X[((int64_t)(b0 + i) * n + b0 + c) * 2 + 1] = Xb[i][c][1];
    }
}

// acc += A[r0.., k0..k0+31] B[k0..k0+31, c0..] for one 32 x 32 output tile,
// each of the 256 threads holding a 2 x 2 block of outputs (rows ty, ty+16;
// columns tx, tx+16).  Out-of-range entries load as zero.
struct Tile32 {
    double a[CB][CB + 1][2];
    double b[CB][CB + 1][2];
};

__device__ __forceinline__ void tile_mac(Tile32& t, const double* A, int lda, int ar, int ac, int arows, int acols,
                                         const double* B, int ldb, int br, int bc, int brows, int bcols,
                                         double (&acc)[2][2][2]) {
    for (int e = threadIdx.x; e < CB * CB; e += blockDim.x) {
        const int r = e / CB, c = e % CB;
        const bool ina = r < arows && c < acols, inb = r < brows && c < bcols;
        t.a[r][c][0] = ina ? A[((int64_t)(ar + r) * lda + ac + c) * 2] : 0.0;
        t.a[r][c][1] = ina ? A[((int64_t)(ar + r) * lda + ac + c) * 2 + 1] : 0.0;
        t.b[r][c][0] = inb ? B[((int64_t)(br + r) * ldb + bc + c) * 2] : 0.0;
        t.b[r][c][1] = inb ? B[((int64_t)(br + r) * ldb + bc + c) * 2 + 1] : 0.0;
    }
    __syncthreads();
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll 4
    for (int k = 0; k < CB; ++k) {
        double xr[2], xi[2], yr[2], yi[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            xr[q] = t.a[ty + 16 * q][k][0]; xi[q] = t.a[ty + 16 * q][k][1];
            yr[q] = t.b[k][tx + 16 * q][0]; yi[q] = t.b[k][tx + 16 * q][1];
        }
#pragma unroll
        for (int p = 0; p < 2; ++p)
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                acc[p][q][0] += xr[p] * yr[q] - xi[p] * yi[q];
                acc[p][q][1] += xr[p] * yi[q] + xi[p] * yr[q];
            }
    }
    __syncthreads();
}

// T_p = L_CA X_AA for every pair p of level b (T_p: [nc][b], leading dim b,
// zeroed by the caller).  X_AA is lower triangular: only k >= the output
// column tile contributes.  Split over K: each CTA adds one 32-wide K-tile's
// product to its output tile with FP64 atomics, so that a level's work
// spreads over as many CTAs as it has (tile, K-tile) pairs instead of
// running each tile's K-tiles one after another (~55 us each).  Grid (b/32,
// b/32, pairs * b/32): z = pair * (b/32) + K-tile.
__global__ void __launch_bounds__(256) k_trinv_t(const double* __restrict__ L, const double* __restrict__ X, int n,
                                                 int b, double* __restrict__ T) {
    __shared__ Tile32 t;
    const int nkt = b / CB;
    const int p = blockIdx.z / nkt, kt = blockIdx.z % nkt;
    const int a0 = 2 * p * b, cc0 = a0 + b;
    const int nc = min(b, n - cc0);
    const int ti = blockIdx.y * CB, tj = blockIdx.x * CB;
    const int k0 = kt * CB;
    if (ti >= nc || k0 < tj) return;
    double acc[2][2][2] = {};
    tile_mac(t, L, n, cc0 + ti, a0 + k0, min(CB, nc - ti), CB, X, n, a0 + k0, a0 + tj, CB, CB, acc);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double* Tp = T + (int64_t)p * b * b * 2;
#pragma unroll
    for (int pp = 0; pp < 2; ++pp)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int r = ti + ty + 16 * pp, c = tj + tx + 16 * q;
            if (r < nc) {
                atomicAdd(&Tp[((int64_t)r * b + c) * 2], acc[pp][q][0]);
                atomicAdd(&Tp[((int64_t)r * b + c) * 2 + 1], acc[pp][q][1]);
            }
        }
}

// X_CA = -X_CC T_p; X_CC is lower triangular: only k < the end of the output
// row tile contributes.  X_CA is zero before (X starts zeroed and each block
// is written at one level only); split over K like k_trinv_t.  Grid (b/32,
// b/32, pairs * b/32).
__global__ void __launch_bounds__(256) k_trinv_x(const double* __restrict__ T, double* __restrict__ X, int n, int b) {
    __shared__ Tile32 t;
    const int nkt = b / CB;
    const int p = blockIdx.z / nkt, kt = blockIdx.z % nkt;
    const int a0 = 2 * p * b, cc0 = a0 + b;
    const int nc = min(b, n - cc0);
    const int ti = blockIdx.y * CB, tj = blockIdx.x * CB;
    const int k0 = kt * CB;
    const int kend = min(nc, ti + CB);
    if (ti >= nc || k0 >= kend) return;
    const double* Tp = T + (int64_t)p * b * b * 2;
    double acc[2][2][2] = {};
    tile_mac(t, X, n, cc0 + ti, cc0 + k0, min(CB, nc - ti), min(CB, nc - k0), Tp, b, k0, tj, min(CB, nc - k0), CB,
             acc);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
    for (int pp = 0; pp < 2; ++pp)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int r = ti + ty + 16 * pp, c = tj + tx + 16 * q;
            if (r < nc) {
                atomicAdd(&X[((int64_t)(cc0 + r) * n + a0 + c) * 2], -acc[pp][q][0]);
                atomicAdd(&X[((int64_t)(cc0 + r) * n + a0 + c) * 2 + 1], -acc[pp][q][1]);
            }
        }
}

}  // namespace

void launch_overlap(Domain& d, const void* X, const void* Y, double scale, double* S) {
    ProfScope ps(d.prof, MLMD_KERNEL_GEMM, d.stream);
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

void launch_update(Domain& d, const void* X, const double* M, void* Y, const void* Z) {
    const int no = d.desc.n_orb;
    dim3 grid((d.ld + 31) / 32, (unsigned)((d.ng + 63) / 64));
    if (d.c64())
        k_update<float><<<grid, 256, 0, d.stream>>>((const float*)X, M, d.ng, d.ld, no, (const float*)Z, (float*)Y);
    else
        k_update<double><<<grid, 256, 0, d.stream>>>((const double*)X, M, d.ng, d.ld, no, (const double*)Z,
                                                     (double*)Y);
    d.launches++;
    MLMD_CUDA(cudaGetLastError());
}

// M <- s M for a complex FP64 [n][n] matrix and complex s.
__global__ void k_scale_complex(double* __restrict__ M, int64_t nn, double sr, double si) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nn; e += (int64_t)gridDim.x * blockDim.x) {
        const double a = M[2 * e], b = M[2 * e + 1];
        M[2 * e] = sr * a - si * b;
        M[2 * e + 1] = sr * b + si * a;
    }
}

void launch_scale_complex(Domain& d, double* M, int64_t nn, double sr, double si) {
    k_scale_complex<<<(int)std::min<int64_t>((nn + 255) / 256, 1024), 256, 0, d.stream>>>(M, nn, sr, si);
    d.launches++;
    MLMD_CUDA(cudaGetLastError());
}

// Occupations of the reference orbitals (Sec. V.A.3, V.A.8) from the
// overlap C[s][m] = <psi_s(0)|psi_m(t)> (complex double [n][n]): one warp
// per row s, fs[s] = sum_m f_m |C_sm|^2 and rs[s] = sum_m |C_sm|^2, lanes
// striding over m, then a butterfly (a fixed order, so the sums repeat
// bit for bit).
__global__ void k_occ_rows(const double* __restrict__ C, const double* __restrict__ f, int n,
                           double* __restrict__ fs, double* __restrict__ rs) {
    const int lane = threadIdx.x & 31;
    const int s = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (s >= n) return;
    const double* row = C + (int64_t)2 * s * n;
    double af = 0.0, a1 = 0.0;
    for (int m = lane; m < n; m += 32) {
        const double re = row[2 * m], im = row[2 * m + 1];
        const double p = re * re + im * im;
        af += f[m] * p;
        a1 += p;
    }
    for (int o = 16; o > 0; o >>= 1) {
        af += __shfl_xor_sync(0xffffffffu, af, o);
        a1 += __shfl_xor_sync(0xffffffffu, a1, o);
    }
    if (lane == 0) {
        fs[s] = af;
        rs[s] = a1;
    }
}

// out[0] = sum_m f_m - sum_s fs[s] (n_exc), out[1] = sum_s rs[s]; one block,
// thread-strided partials then a shared-memory tree (fixed order).
__global__ void k_occ_total(const double* __restrict__ fs, const double* __restrict__ rs,
                            const double* __restrict__ f, int n, double* __restrict__ out) {
    __shared__ double sh[2][256];
    double a = 0.0, b = 0.0;
    for (int s = threadIdx.x; s < n; s += blockDim.x) {
        a += f[s] - fs[s];
        b += rs[s];
    }
    sh[0][threadIdx.x] = a;
    sh[1][threadIdx.x] = b;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = sh[0][0];
        out[1] = sh[1][0];
    }
}

void launch_occupations(Domain& d, const double* C, double* fs, double* rs, double* out) {
    const int n = d.desc.n_orb;
    k_occ_rows<<<(n + 7) / 8, 256, 0, d.stream>>>(C, d.f, n, fs, rs);
    k_occ_total<<<1, 256, 0, d.stream>>>(fs, rs, d.f, n, out);
    d.launches += 2;
    MLMD_CUDA(cudaGetLastError());
}

void cholesky_inverse_upper(Domain& d, double* S, double* Minv, int* d_info) {
    const int n = d.desc.n_orb;
    MLMD_CUDA(cudaMemsetAsync(d_info, 0, sizeof(int), d.stream));
    const int nblk = (n + CB - 1) / CB;
    double* Ld = (double*)d.mem.get((size_t)nblk * CB * CB * 2 * sizeof(double));
    // Look-ahead: the trailing update of panel kb is split into the next
    // block column (tile columns 0 and 1, main stream: the next diagonal
    // block and panel rows need it) and the rest (side stream), so that the
    // next panel's serial factorisation runs beside the bulk of the update.
    // Ordering: the side update of panel kb starts after panel kb's rows;
    // the main stream waits for it before panel kb+1's trailing update (both
    // touch block column kb+2), which precedes every later diagonal block.
    if (!d.side) {
        MLMD_CUDA(cudaStreamCreateWithFlags(&d.side, cudaStreamNonBlocking));
        MLMD_CUDA(cudaEventCreateWithFlags(&d.ev_rows, cudaEventDisableTiming));
        MLMD_CUDA(cudaEventCreateWithFlags(&d.ev_trail, cudaEventDisableTiming));
    }
    bool side_pending = false;
    for (int kb = 0; kb < nblk; ++kb) {
        const int below = n - (kb * CB + std::min(CB, n - kb * CB));
        k_chol_diag<<<1, 256, 0, d.stream>>>(S, n, kb, Ld, d_info);
        d.launches++;
        if (below <= 0) continue;
        k_chol_rows<<<(below + 7) / 8, 256, 0, d.stream>>>(S, n, kb, Ld);
        d.launches++;
        const int t = (below + TT - 1) / TT;
        if (t > 2) {
            MLMD_CUDA(cudaEventRecord(d.ev_rows, d.stream));
            MLMD_CUDA(cudaStreamWaitEvent(d.side, d.ev_rows, 0));
        }
        if (side_pending) {               // the previous panel's side update reaches block column kb+1
            MLMD_CUDA(cudaStreamWaitEvent(d.stream, d.ev_trail, 0));
            side_pending = false;
        }
        k_chol_trail<<<dim3(std::min(t, 2), t), 256, 0, d.stream>>>(S, n, kb, 0, 0);
        d.launches++;
        if (t > 2) {
            k_chol_trail<<<dim3(t - 2, t - 2), 256, 0, d.side>>>(S, n, kb, 2, 2);
            d.launches++;
            MLMD_CUDA(cudaEventRecord(d.ev_trail, d.side));
            side_pending = true;
        }
    }
    if (side_pending) MLMD_CUDA(cudaStreamWaitEvent(d.stream, d.ev_trail, 0));
    // X = L^{-1} by recursive doubling of inverted diagonal blocks, then Minv = X^H
    double* X = (double*)d.mem.get((size_t)n * n * 2 * sizeof(double));
    double* T = (double*)d.mem.get((size_t)n * n * 2 * sizeof(double));
    MLMD_CUDA(cudaMemsetAsync(X, 0, (size_t)n * n * 2 * sizeof(double), d.stream));
    k_trinv_diag<<<nblk, 256, 0, d.stream>>>(Ld, X, n);
    d.launches++;
    for (int b = CB; b < n; b *= 2) {
        const int pairs = (n - b + 2 * b - 1) / (2 * b);      // pairs whose C block is non-empty
        const dim3 grid(b / CB, b / CB, pairs * (b / CB));    // (tile column, tile row, pair x K-tile)
        MLMD_CUDA(cudaMemsetAsync(T, 0, (size_t)pairs * b * b * 2 * sizeof(double), d.stream));
        k_trinv_t<<<grid, 256, 0, d.stream>>>(S, X, n, b, T);
        k_trinv_x<<<grid, 256, 0, d.stream>>>(T, X, n, b);
        d.launches += 2;
    }
    k_conj_transpose<<<(int)std::min<int64_t>(((int64_t)n * n + 255) / 256, 4096), 256, 0, d.stream>>>(X, n, Minv);
    d.launches++;
    MLMD_CUDA(cudaGetLastError());
    d.mem.put(T);
    d.mem.put(X);
    d.mem.put(Ld);
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
