// Overlap matrix without any device allocation.
//
// Some callers cannot call cudaMalloc (or anything that allocates) at the
// point where they need an overlap: code running while a caller-owned memory
// pool is frozen or fully reserved, code inside a framework that forbids
// allocation on its hot path, or a host thread that must not contend for the
// allocator while other work is in flight.  mlmd_overlap_noalloc serves them:
// the caller passes the orbital arrays and the output, and the split sums
// that the overlap kernel needs live in one fixed array that the library
// declares at file scope.
//
// The array is `kScratchBytes` (4 MiB) of device memory that every GPU which
// loads this library holds until the process exits.  All calls share it: two
// calls whose kernels overlap on the GPU (for example on different streams)
// race on it and give wrong results; calls ordered on one stream are safe.
// Every split sum a call reads is written by that same call first, so the
// array keeps the previous call's contents without harm and is never cleared.
#include <algorithm>
#include <mutex>

#include "mlmd_internal.cuh"

namespace {

constexpr size_t kScratchBytes = size_t(4) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_overlap_scratch[kScratchBytes];

std::mutex g_mutex;
int g_sm_count[kMaxDevices] = {};

// The device address of the scratch array on the current device.  In host
// code the array's name is only a host-side stand-in, so the address is
// looked up with the device current.  The lookup is host-side and allocates
// nothing; it is repeated on every call rather than cached, so that a call
// after the caller reset the device (which reloads the module and may move
// the array) still gets the array's current address.
cudaError_t scratch_address(void** out) { return cudaGetSymbolAddress(out, g_overlap_scratch); }

// Streaming multiprocessors of a device (queried once per device).
cudaError_t sm_count(int dev, int* out) {
    std::lock_guard<std::mutex> lock(g_mutex);
    if (g_sm_count[dev] <= 0) {
        int n = 0;
        const cudaError_t e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        g_sm_count[dev] = n > 0 ? n : 1;
    }
    *out = g_sm_count[dev];
    return cudaSuccess;
}

// part[z][n][m] = sum over the z-th slab of grid points of conj(X[g][n]) Y[g][m]
// (32 x 32 output tile per block, each thread a 2 x 2 sub-tile; products in
// the working type over 256 points, then FP64).
template <typename R>
__global__ void __launch_bounds__(256) k_overlap_partials(const R* __restrict__ X, const R* __restrict__ Y,
                                                          int64_t ng, int n_orb, int64_t kchunk,
                                                          double* __restrict__ part) {
    __shared__ R xs[32][33][2];
    __shared__ R ys[32][33][2];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int n0 = blockIdx.y * 32, m0 = blockIdx.x * 32;
    const int64_t g0 = blockIdx.z * kchunk;
    const int64_t g1 = g0 + kchunk < ng ? g0 + kchunk : ng;
    double acc[2][2][2] = {};
    R racc[2][2][2] = {};
    int cnt = 0;
    for (int64_t gb = g0; gb < g1; gb += 32) {
        for (int e = threadIdx.x; e < 32 * 32; e += 256) {
            const int r = e >> 5, c = e & 31;
            const int64_t g = gb + r;
            R xr = 0, xi = 0, yr = 0, yi = 0;
            if (g < g1) {
                if (n0 + c < n_orb) { xr = X[(g * n_orb + n0 + c) * 2]; xi = X[(g * n_orb + n0 + c) * 2 + 1]; }
                if (m0 + c < n_orb) { yr = Y[(g * n_orb + m0 + c) * 2]; yi = Y[(g * n_orb + m0 + c) * 2 + 1]; }
            }
            xs[r][c][0] = xr; xs[r][c][1] = xi;
            ys[r][c][0] = yr; ys[r][c][1] = yi;
        }
        __syncthreads();
        for (int r = 0; r < 32; ++r)
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                const R xr = xs[r][ty + 16 * a][0], xi = xs[r][ty + 16 * a][1];
#pragma unroll
                for (int b = 0; b < 2; ++b) {
                    const R yr = ys[r][tx + 16 * b][0], yi = ys[r][tx + 16 * b][1];
                    racc[a][b][0] += xr * yr + xi * yi;
                    racc[a][b][1] += xr * yi - xi * yr;
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

// S[e] = scale * sum_z part[z][e], fixed order
__global__ void k_overlap_finish(const double* __restrict__ part, int nsplit, int64_t n, double scale,
                                 double* __restrict__ S) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int k = 0; k < nsplit; ++k) s += part[(int64_t)k * n + e];
        S[e] = scale * s;
    }
}

}  // namespace

extern "C" mlmd_status mlmd_overlap_noalloc(int32_t precision, int64_t n_grid, int32_t n_orb, const void* X,
                                            const void* Y, double scale, double* S, void* stream) {
    if (precision != MLMD_C64 && precision != MLMD_C128) return MLMD_ERR_INVALID;
    if (n_grid < 1 || n_orb < 1 || !X || !Y || !S) return MLMD_ERR_INVALID;
    const size_t per_split = (size_t)n_orb * n_orb * 2 * sizeof(double);
    if (per_split > kScratchBytes) return MLMD_ERR_INVALID;   // n_orb above MLMD_OVERLAP_NOALLOC_MAX_ORB
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MLMD_ERR_CUDA;
    void* scratch = nullptr;
    int sms = 0;
    if (scratch_address(&scratch) != cudaSuccess || sm_count(dev, &sms) != cudaSuccess) return MLMD_ERR_CUDA;
    // split the grid points so that the launch fills the GPU (about eight
    // blocks per SM), within the scratch
    const int tiles = (n_orb + 31) / 32;
    int64_t nsplit = ((int64_t)sms * 8) / ((int64_t)tiles * tiles) + 1;
    nsplit = std::min<int64_t>(nsplit, (n_grid + 255) / 256);
    nsplit = std::min<int64_t>(nsplit, (int64_t)(kScratchBytes / per_split));
    nsplit = std::max<int64_t>(nsplit, 1);
    const int64_t kchunk = ((n_grid + nsplit - 1) / nsplit + 31) / 32 * 32;
    nsplit = (n_grid + kchunk - 1) / kchunk;
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    double* part = static_cast<double*>(scratch);
    dim3 grid(tiles, tiles, (unsigned)nsplit);
    if (precision == MLMD_C64)
        k_overlap_partials<float><<<grid, 256, 0, st>>>(static_cast<const float*>(X), static_cast<const float*>(Y),
                                                         n_grid, n_orb, kchunk, part);
    else
        k_overlap_partials<double><<<grid, 256, 0, st>>>(static_cast<const double*>(X), static_cast<const double*>(Y),
                                                          n_grid, n_orb, kchunk, part);
    const int64_t n = (int64_t)n_orb * n_orb * 2;
    k_overlap_finish<<<(int)std::min<int64_t>((n + 255) / 256, 2048), 256, 0, st>>>(part, (int)nsplit, n, scale, S);
    return cudaGetLastError() == cudaSuccess ? MLMD_OK : MLMD_ERR_CUDA;
}
