// Internal declarations of libmlmd (CUDA, sm_103a).  Not part of the ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "mlmd.h"

namespace mlmd {

// ---------------------------------------------------------------------------
// error plumbing: every entry point converts failures into an mlmd_status
// ---------------------------------------------------------------------------
struct Error {
    mlmd_status status;
    std::string msg;
};

#define MLMD_CUDA(call)                                                                      \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            throw ::mlmd::Error{MLMD_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_) + \
                                " (" + __FILE__ + ":" + std::to_string(__LINE__) + ")"};                \
    } while (0)

#define MLMD_REQUIRE(cond, code, text)                                      \
    do {                                                                    \
        if (!(cond)) throw ::mlmd::Error{code, std::string(text)};          \
    } while (0)

// The library's stream-ordered memory pool on a device (freed blocks stay
// mapped for reuse; trimmed when a domain is destroyed).
cudaMemPool_t library_pool(int dev);

// Padded orbital stride: orbitals are stored in rows of `ld` complex values
// with ld a multiple of 8 (64-byte rows for complex64), padding orbitals zero.
inline int padded_orbitals(int n_orb) { return (n_orb + 7) / 8 * 8; }

// ---------------------------------------------------------------------------
// device memory through the caller's allocator or cudaMallocAsync
// ---------------------------------------------------------------------------
struct Alloc {
    mlmd_allocator a{};
    bool custom = false;
    cudaStream_t stream = nullptr;
    int device = 0;
    struct Blk { void* p; size_t bytes; };
    std::vector<Blk> live;

    void* get(size_t bytes);
    void put(void* p);
    void release_all();
};

// Stencil geometry of one domain (FP64; kernels convert once on the host).
struct Geo {
    int nx, ny, nz;
    int ld;        // padded orbitals per row
    int nv;        // 16-byte vectors per row
    int64_t ng;
    double kc0;    // -1/2 * 3 * lap_0 / h^2   (centre weight of the three axes)
    double kc1;    // -1/2 * lap_1 / h^2
    double kc2;    // -1/2 * lap_2 / h^2
    double gk1;    // grad_1 / h
    double gk2;    // grad_2 / h
    double dV;
};

// Cluster tiling of the one-sweep local Taylor-4 kernel (k_sweep.cu): a
// cluster of CX x CY CTAs covers a whole x-y plane for a chunk of VPC
// orbitals, each CTA a TX x TY tile; ok = false when the domain does not fit.
struct SweepPlan {
    bool ok = false;
    int CX = 0, CY = 0, TX = 0, TY = 0, VPC = 0, threads = 0;
    size_t smem = 0;
    int use = 0;                     // 1: sweep, -1: staged passes, 0: not yet timed
    float t_sweep_ms = 0.f, t_staged_ms = 0.f;   // the timing that decided it
};

struct TmaState;   // TMA stage-kernel state (tensor maps, tiling), k_stage_tma.cu
struct NlTc;       // brick tables of the tensor-core nonlocal path, k_nl_tc.cu

// Projector tables built on the device by set_projectors.
struct Nonlocal {
    int n_atoms = 0;
    int n_proj = 0;
    int64_t n_list = 0;            // total (atom, point) entries
    int max_count = 0;             // longest atom list
    int64_t* off = nullptr;        // [n_atoms + 1] list offsets
    int32_t* idx = nullptr;        // [n_list] grid index, ascending per atom
    double* beta64 = nullptr;      // [n_list][n_proj] FP64 projector values
    void* beta = nullptr;          // [n_list][n_proj] in the working real type
    int32_t* pstart = nullptr;     // [N_g + 1] per-point entry ranges
    int32_t* patom = nullptr;      // [n_list] atom of each per-point entry
    void* pbd = nullptr;           // [n_list][n_proj] beta * D (working real type)
    double* D = nullptr;           // [n_atoms][n_proj]
    std::vector<int64_t> h_off;    // host copy of off
    std::vector<double> h_pos;     // host copy of the atom positions [n_atoms][3]
    int n_seg = 0;                 // projection segments per atom
    int seg_len = 0;
    // velocity-gauge tables (present while the domain's nonlocal gauge is
    // MLMD_NL_GAUGE_VELOCITY)
    void* disp = nullptr;          // [3][n_list] minimum-image displacement r - R_a (working real type)
    int32_t* pq = nullptr;         // [n_list] atom-list entry of each per-point entry
    void* ph_at = nullptr;         // [n_list] complex e^{+i A.(r - R_a)}, atom-list order (projection)
    void* ph_pt = nullptr;         // [n_list] complex e^{-i A.(r - R_a)}, per-point order (scatter)
    void* Qm = nullptr;            // [3][n_atoms][n_proj][ld] complex moment projections
};

// CUDA-event timing of selected kernel kinds (enabled by mlmd_profile_enable).
struct Profiler {
    bool on = false;
    struct Rec { int kind; cudaEvent_t a, b; };
    std::vector<Rec> pending;
    std::vector<cudaEvent_t> pool;
    double total_ms[MLMD_KERNEL_KINDS] = {};
    uint64_t count[MLMD_KERNEL_KINDS] = {};
    cudaEvent_t take();
    void begin(int kind, cudaStream_t s, Rec& r);
    void end(Rec& r, cudaStream_t s);
    void collect();              // caller synchronised the stream
    void reset();
    void destroy();
};

// RAII bracket around one launch of a timed kind.
struct ProfScope {
    Profiler& p;
    cudaStream_t s;
    Profiler::Rec r{};
    bool on;
    ProfScope(Profiler& pp, int kind, cudaStream_t st) : p(pp), s(st), on(pp.on) { if (on) p.begin(kind, s, r); }
    ~ProfScope() { if (on) p.end(r, s); }
};

struct Domain {
    mlmd_domain_desc desc{};
    int64_t ng = 0;                // grid points
    int ld = 0;                    // padded orbital stride
    size_t elem = 0;               // bytes per complex value
    size_t state_bytes = 0;        // ng * ld * elem
    int device = 0;
    cudaStream_t stream = nullptr;
    Alloc mem;

    void* psi = nullptr;           // current orbitals
    void* psi0 = nullptr;          // reference orbitals Psi(0)
    void* wa = nullptr;            // Taylor work buffers
    void* wb = nullptr;
    void* V = nullptr;             // [ng] local potential (working real type)
    double* V64 = nullptr;         // [ng] FP64 copy (adjoint, batch)
    double* f = nullptr;           // [ld] occupations, zero on padding
    void* fR = nullptr;            // [ld] occupations in the working real type
    Nonlocal nl;
    void* Pa = nullptr;            // projections [n_atoms][n_proj][ld] complex
    void* Pb = nullptr;
    void* Pseg = nullptr;          // segment partials [n_seg][n_atoms][n_proj][ld]
    double* obs_part = nullptr;    // per-block observable partials
    int obs_blocks = 0;
    double* obs_dev = nullptr;     // [cap][5]
    int obs_cap = 0;
    double* A_dev = nullptr;       // [cap][3]
    int A_cap = 0;
    double* dense = nullptr;       // scratch for N_o x N_o FP64 work
    size_t dense_bytes = 0;
    // look-ahead Cholesky: side stream for the trailing updates beyond the
    // next block column, and its two ordering events (created on first use)
    cudaStream_t side = nullptr;
    cudaEvent_t ev_rows = nullptr, ev_trail = nullptr;

    int64_t step = 0;              // steps since set_orbitals
    bool pa_psi = false;           // Pa holds <b|psi> of the current orbitals
    bool psi0_valid = false;
    uint64_t launches = 0;
    Profiler prof;
    TmaState* tma = nullptr;
    NlTc* nltc = nullptr;          // tensor-core nonlocal tables (dense-projector domains), or null
    int nl_gauge = MLMD_NL_GAUGE_REAL;   // projector gauge (mlmd_set_nonlocal_gauge)
    SweepPlan sweep;               // one-sweep local Taylor-4 tiling (ok = false: staged passes)
    double nl_rc = 0.0;            // projector width r_c of the current projectors
    int* err_flag = nullptr;       // device word raised by a kernel whose bounded wait expired
    mlmd_status latched = MLMD_OK;
    std::string err;

    bool c64() const { return desc.precision == MLMD_C64; }
    bool has_nl() const { return nl.n_atoms > 0 && nl.n_proj > 0; }
};

// The velocity-gauge projectors are in use (they run on the per-point
// projection and scatter kernels).
inline bool gauge_on(const Domain& d) { return d.nl_gauge == MLMD_NL_GAUGE_VELOCITY && d.has_nl(); }
// The tensor-core nonlocal path is in use (real projectors only).
inline bool nltc_on(const Domain& d) { return d.nltc != nullptr && d.nl_gauge == MLMD_NL_GAUGE_REAL; }

// ---------------------------------------------------------------------------
// kernels (launch wrappers count launches into dom.launches)
// ---------------------------------------------------------------------------

// out = psi + gamma * (h(A) w) with h of Eq. 3; psi may be null (then out =
// gamma * h w).  P: projections of w (may be null when there are no
// projectors).  When obs != null, also writes per-block partial observables
// of w (which must then equal psi's state) into obs.
struct StageArgs {
    const void* w = nullptr;
    const void* psi = nullptr;
    void* out = nullptr;
    const void* P = nullptr;       // <b|w> for the scatter-back
    void* P_out = nullptr;         // if set: <b|out> wanted (the TMA path fuses it)
    const double* A = nullptr;     // device [3]
    double gamma_re = 0.0, gamma_im = 0.0;
    double* obs = nullptr;         // per-block partials [blocks][5] or null
};
// Returns the number of thread blocks of the launch (= rows of obs partials).
// *proj_done (if given) tells whether <b|out> was written to a.P_out.
int launch_stage(Domain& d, const StageArgs& a, bool* proj_done = nullptr);
int stage_blocks(const Domain& d);

Geo geo_of(const Domain& d);

// Raise a kernel's dynamic shared-memory limit to at least `bytes` on the
// current device.  The attribute belongs to the kernel function on each
// device, not to a launch site, so the cache is keyed by (device, kernel).
void ensure_dynamic_smem(const void* kernel, size_t bytes);

// TMA-staged stage kernel (k_stage_tma.cu): set up at domain creation; the
// launch returns false when the grid or row does not tile (then the plain
// kernel runs).
void tma_setup(Domain& d);
void tma_release(Domain& d);
int tma_blocks(const Domain& d);
bool launch_stage_tma(Domain& d, const StageArgs& a, bool* proj_done);
// Tables of the fused nonlocal path (after the projector lists are built).
void tma_build_nl(Domain& d, const double* D_host, int zc_cap = 0);   // zc_cap: internal (16 on the rebuild)
bool tma_fused_nl(const Domain& d);
// Time both orbital-chunk widths of the TMA stage kernel once per domain and
// keep the faster (no-op after the first call).  Must not run during stream
// capture.  Ak: device [3].
void tma_autotune(Domain& d, const double* Ak);
int tma_chunk_bytes(const Domain& d);

// P[a][i][o] = dV sum_q beta[q][i] w[idx[q]][o]
// P = <b|w> (dV included); with the velocity-gauge projectors <b~|w> at the
// phases of the last launch_nl_phase, and for moment_axis >= 0 the moment
// projection <(r - R_a)_axis b~|w>.
void launch_project(Domain& d, const void* w, void* P, int moment_axis = -1);
// Velocity-gauge tables: build (lists present) / drop; per-step phases at A_k.
void gauge_build(Domain& d);
void gauge_release(Domain& d);
void launch_nl_phase(Domain& d, const double* Ak);
// Moment projection buffer of axis ax (velocity gauge).
void* moment_buffer(Domain& d, int ax);
// obs_row[2 + x] += the nonlocal commutator current from P = <b~|psi> and
// the moment projections in Qm (velocity gauge).
void launch_nl_current(Domain& d, const void* P, double* obs_row);

// One-sweep local Taylor-4 (k_sweep.cu): plan at domain creation; launch
// buf <- T4(h_loc(A_k)) buf in place, with observable partials when obs_part
// is set (returns their row count).
SweepPlan plan_sweep(const Domain& d);
void sweep_setup(Domain& d);
int launch_sweep(Domain& d, void* buf, const double* Ak, double* obs_part);
// First-propagate timing of the sweep against the staged passes (sets sweep.use).
void sweep_autotune(Domain& d, const double* Ak);
inline bool sweep_on(const Domain& d) { return d.sweep.ok && d.sweep.use == 1; }

// Tensor-core nonlocal path (k_nl_tc.cu) for complex64 domains whose
// projector spheres cover each grid point many times: brick tables built
// from the exact lists at set_projectors; the scatter adds gamma v_nl w (from
// P = <b|w>, P being Pa or Pb) to a stage output that holds the local part
// and leaves the output's split copy for the projection; the projection
// writes P = <b|w> (zeroing P first; w3_ready says the scatter just made w's
// split copy) and the split copy of D o P; the energy adds <psi|v_nl|psi>
// from P = <b|psi> to an observable row.
bool nl_tc_wanted(const Domain& d);
void nl_tc_build(Domain& d, const double* pos_host, double r_c, const double* D_host);
void nl_tc_release(Domain& d);
void launch_nl_scatter_tc(Domain& d, const void* P, void* out, double gre, double gim);
void launch_nl_project_tc(Domain& d, const void* w, void* P, bool w3_ready);
void launch_nl_energy(Domain& d, const void* P, double* row);

// obs_dev[row][0..4] = final observables from the per-block partials
void launch_obs_finish(Domain& d, const double* partials, int nblocks, const double* A, double* row);

// density / current
void launch_density_current(Domain& d, const double* A, void* rho, void* j, double* Jpart, int nblk);
int density_blocks(const Domain& d);

// out = sum_t coef[t] * in[t] over whole states (t < n <= 5)
void launch_lincomb(Domain& d, int n, const void* const* in, const double* coef_re, const double* coef_im,
                    void* out);

// adjoint contractions: for p < 4, with z_p, u_p states:
//   gA[a]  += 2 Re sum <z_p | -i G_a u_p>   (per-block partials, a = 0..2)
//   gZ     += 2 Re sum <z_p | u_p>           (partial index 3)
//   gV[r]  += 2 Re sum_o conj(z_p) u_p       (FP64 [ng], accumulated)
void launch_adjoint_contract(Domain& d, const void* const* z, const void* const* u, double* part, int nblk,
                             double* gV);
int contract_blocks(const Domain& d);

// neighbour lists and projector tables (a1)
void build_projectors(Domain& d, int n_atoms, const double* pos_host, int n_proj, double r_c, double r_cut,
                      const double* D_host);

// dense orbital-space algebra (FP64 results)
// S[n][m] = scale * sum_g conj(X[g][n]) Y[g][m] for n, m < n_orb; S is
// complex double [n_orb][n_orb] on the device.
void launch_overlap(Domain& d, const void* X, const void* Y, double scale, double* S);
// The same on the tcgen05 tensor cores with split 16-bit operands, for
// complex64 domains whose gemm_mode is not FP32 (returns false otherwise).
bool launch_overlap_tc(Domain& d, const void* X, const void* Y, double scale, double* S);
// Y[g][m] = sum_n X[g][n] M[n][m] (M complex double [n_orb][n_orb], device)
// Y = Z + X M (Z = null: Y = X M), SIMT, FP32 or FP64 accumulation per the domain.
void launch_update(Domain& d, const void* X, const double* M, void* Y, const void* Z = nullptr);
// From C[s][m] = <psi_s(0)|psi_m(t)> (device complex double [n_orb][n_orb]):
// fs[s] = sum_m f_m |C_sm|^2, rs[s] = sum_m |C_sm|^2 (device [n_orb]) and
// out[0] = sum f - sum fs, out[1] = sum rs (device [2]); FP64, fixed order.
void launch_occupations(Domain& d, const double* C, double* fs, double* rs, double* out);
// M <- (sr + i si) M for a complex FP64 matrix of nn entries.
void launch_scale_complex(Domain& d, double* M, int64_t nn, double sr, double si);
// Y = X M on the tensor cores in the domain's split mode (c64, non-FP32 GEMM
// modes); false if the domain does not use them.
// upper: M is upper triangular (a Cholesky L^{-H}); the zero K-tiles are skipped.
bool launch_update_tc(Domain& d, const void* X, const double* M, void* Y, bool upper);
// Y = Z + X Mc on the tensor cores in the domain's split mode (Mc complex
// FP64 [n_orb][n_orb]); false if the domain does not use them.
bool launch_gemm_add_tc(Domain& d, const void* X, const double* Mc, const void* Z, void* Y);
// In place: S -> lower Cholesky factor L (S = L L^H); returns false if S is
// not positive definite.  Then Minv = L^{-H} (upper).
void cholesky_inverse_upper(Domain& d, double* S, double* Minv, int* d_info);
// Minv = S^{-1/2} by coupled Newton-Schulz iterations in FP64.
void lowdin_inverse_sqrt(Domain& d, double* S, double* Minv, double* work, int* d_info);

// One full-scheme Taylor-4 step of the domain's orbitals under A (device
// [3]); writes the pre-step observables to obs_row (device [5]) if non-null.
// Allocates nothing, so it can be captured into a CUDA graph.
void step_full(Domain& d, const double* Ak, double* obs_row);

// Raise MLMD_ERR_TIMEOUT if a kernel of the domain gave up a bounded
// device-side wait (reads the error word in stream order; synchronises).
void check_err_flag(Domain& d);

// final reduce of per-block partials (fixed order, FP64)
void launch_reduce_partials(Domain& d, const double* part, int nblk, int width, double* out);

}  // namespace mlmd

// The opaque handles of the ABI.
struct mlmd_domain : public mlmd::Domain {};

struct mlmd_batch {
    std::vector<mlmd_domain*> doms;
    cudaStream_t stream = nullptr;
    int device = 0;
};
