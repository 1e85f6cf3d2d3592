// C-ABI entry points of libmlmd (declared in include/mlmd.h) and the host
// orchestration of the time loop.  Every step of the path runs in the
// kernels of this library; the host only validates, allocates and launches.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <new>
#include <vector>

#include <map>
#include <mutex>

#include "mlmd_internal.cuh"

using mlmd::Domain;
using mlmd::Error;


namespace mlmd {

void ensure_dynamic_smem(const void* kernel, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, size_t> set;
    int dev = 0;
    MLMD_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    size_t& cur = set[{dev, kernel}];
    if (bytes > cur) {
        MLMD_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
        cur = bytes;
    }
}

// ---------------------------------------------------------------------------
// allocator
// ---------------------------------------------------------------------------
// The library's own stream-ordered memory pool on a device.  Its release
// threshold is unbounded, so memory freed by one call (the split-operand
// tile images of the tensor-core GEMMs are gigabytes at the largest
// workloads) stays mapped for the next instead of going back to the driver
// at every synchronisation; mlmd_domain_destroy trims the pool.
cudaMemPool_t library_pool(int dev) {
    static std::mutex mu;
    static std::map<int, cudaMemPool_t> pools;
    std::lock_guard<std::mutex> lock(mu);
    auto it = pools.find(dev);
    if (it != pools.end()) return it->second;
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool;
    MLMD_CUDA(cudaMemPoolCreate(&pool, &props));
    uint64_t thr = UINT64_MAX;
    MLMD_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
    pools[dev] = pool;
    return pool;
}

void* Alloc::get(size_t bytes) {
    bytes = std::max<size_t>(bytes, 256);
    void* p = nullptr;
    if (custom) {
        p = a.alloc(bytes, (void*)stream, a.ctx);
        MLMD_REQUIRE(p != nullptr, MLMD_ERR_OOM, "device allocation failed (caller allocator)");
    } else {
        cudaError_t e = cudaMallocFromPoolAsync(&p, bytes, library_pool(device), stream);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            throw Error{MLMD_ERR_OOM, std::string("cudaMallocFromPoolAsync: ") + cudaGetErrorString(e)};
        }
    }
    live.push_back({p, bytes});
    return p;
}

void Alloc::put(void* p) {
    if (!p) return;
    for (size_t i = 0; i < live.size(); ++i)
        if (live[i].p == p) {
            if (custom) a.free(p, live[i].bytes, (void*)stream, a.ctx);
            else (void)cudaFreeAsync(p, stream);
            live.erase(live.begin() + i);
            return;
        }
}

void Alloc::release_all() {
    for (auto& b : live) {
        if (custom) a.free(b.p, b.bytes, (void*)stream, a.ctx);
        else (void)cudaFreeAsync(b.p, stream);
    }
    live.clear();
}

// One FULL-scheme Taylor-4 step in nested form:
//   w <- psi + (-i dt/4) h psi;  w <- psi + (-i dt/3) h w;
//   w <- psi + (-i dt/2) h w;    psi <- psi + (-i dt) h w
// each h = local stencil + scatter-back of the projections of its input.
// When the TMA stage kernel fuses the projection of its output, the four
// stages pass the projections along (Pa -> Pb -> Pa -> Pb -> Pa) and Pa holds
// <b|psi> of the new orbitals for the next step; otherwise each stage is
// preceded by a projection pass over its input.
void step_full(Domain& d, const double* Ak, double* obs_row) {
    const double dt = d.desc.dt;
    if (nltc_on(d)) {
        // tensor-core nonlocal path: each stage is the local stencil kernel
        // (out = psi + gamma h_loc w), the scatter GEMM (out += gamma v_nl w
        // from P = <b|w>) and the projection GEMM of out for the next stage;
        // the projections pass along Pa -> Pb -> Pa -> Pb -> Pa
        if (!d.pa_psi) launch_nl_project_tc(d, d.psi, d.Pa, false);
        const void* in = d.psi;
        void* outs[4] = {d.wa, d.wb, d.wa, d.psi};
        void* Pin[4] = {d.Pa, d.Pb, d.Pa, d.Pb};
        void* Pout[4] = {d.Pb, d.Pa, d.Pb, d.Pa};
        for (int s = 0; s < 4; ++s) {
            StageArgs a;
            a.w = in;
            a.psi = d.psi;
            a.out = outs[s];
            a.A = Ak;
            a.gamma_re = 0.0;
            a.gamma_im = -dt / (double)(4 - s);
            a.obs = (s == 0 && obs_row) ? d.obs_part : nullptr;
            const int nblk = launch_stage(d, a);
            if (s == 0 && obs_row) {
                launch_obs_finish(d, d.obs_part, nblk, Ak, obs_row);
                launch_nl_energy(d, d.Pa, obs_row);      // <psi|v_nl|psi> from P = <b|psi>
            }
            launch_nl_scatter_tc(d, Pin[s], outs[s], a.gamma_re, a.gamma_im);
            launch_nl_project_tc(d, outs[s], Pout[s], true);   // the scatter left the split output
            in = outs[s];
        }
        d.pa_psi = true;
        return;
    }
    const bool nl = d.has_nl();
    if (!nl && sweep_on(d)) {
        // no nonlocal term: all four Taylor terms in one sweep over psi
        const int nblk = launch_sweep(d, d.psi, Ak, obs_row ? d.obs_part : nullptr);
        if (obs_row) launch_obs_finish(d, d.obs_part, nblk, Ak, obs_row);
        d.pa_psi = false;
        return;
    }
    const bool fused = nl && tma_fused_nl(d);
    const bool gauge = gauge_on(d);
    if (gauge) launch_nl_phase(d, Ak);       // projector phases at this step's A
    if (fused && !d.pa_psi) launch_project(d, d.psi, d.Pa);
    const void* in = d.psi;
    void* outs[4] = {d.wa, d.wb, d.wa, d.psi};
    void* Pin[4] = {d.Pa, d.Pb, d.Pa, d.Pb};
    void* Pout[4] = {d.Pb, d.Pa, d.Pb, d.Pa};
    bool chain = fused;
    for (int s = 0; s < 4; ++s) {
        if (nl && !chain) launch_project(d, in, Pin[s]);
        StageArgs a;
        a.w = in;
        a.psi = d.psi;
        a.out = outs[s];
        a.P = nl ? Pin[s] : nullptr;
        a.P_out = fused ? Pout[s] : nullptr;
        a.A = Ak;
        a.gamma_re = 0.0;
        a.gamma_im = -dt / (double)(4 - s);
        a.obs = (s == 0 && obs_row) ? d.obs_part : nullptr;
        bool done = false;
        const int nblk = launch_stage(d, a, &done);
        chain = fused && done;
        if (s == 0 && obs_row) {
            launch_obs_finish(d, d.obs_part, nblk, Ak, obs_row);
            if (gauge) {
                // the nonlocal commutator current of psi (Pin[0] = <b~|psi>)
                for (int ax = 0; ax < 3; ++ax) launch_project(d, d.psi, moment_buffer(d, ax), ax);
                launch_nl_current(d, Pin[0], obs_row);
            }
        }
        in = outs[s];
    }
    d.pa_psi = chain;
}

// Raise MLMD_ERR_TIMEOUT if a kernel's bounded device-side wait expired:
// reads the domain's error word in stream order and synchronises the stream.
void check_err_flag(Domain& d) {
    int h = 0;
    MLMD_CUDA(cudaMemcpyAsync(&h, d.err_flag, sizeof(int), cudaMemcpyDeviceToHost, d.stream));
    MLMD_CUDA(cudaStreamSynchronize(d.stream));
    MLMD_REQUIRE(h == 0, MLMD_ERR_TIMEOUT, "a device-side wait timed out");
}

// ---------------------------------------------------------------------------
// kernel timing
// ---------------------------------------------------------------------------
cudaEvent_t Profiler::take() {
    if (!pool.empty()) {
        cudaEvent_t e = pool.back();
        pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    MLMD_CUDA(cudaEventCreate(&e));
    return e;
}

void Profiler::begin(int kind, cudaStream_t s, Rec& r) {
    r.kind = kind;
    r.a = take();
    r.b = take();
    MLMD_CUDA(cudaEventRecord(r.a, s));
}

void Profiler::end(Rec& r, cudaStream_t s) {
    if (cudaEventRecord(r.b, s) == cudaSuccess) pending.push_back(r);
}

void Profiler::collect() {
    for (auto& r : pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            total_ms[r.kind] += ms;
            count[r.kind] += 1;
        }
        pool.push_back(r.a);
        pool.push_back(r.b);
    }
    pending.clear();
}

void Profiler::reset() {
    for (auto& r : pending) { pool.push_back(r.a); pool.push_back(r.b); }
    pending.clear();
    for (int k = 0; k < MLMD_KERNEL_KINDS; ++k) { total_ms[k] = 0.0; count[k] = 0; }
}

void Profiler::destroy() {
    reset();
    for (cudaEvent_t e : pool) (void)cudaEventDestroy(e);
    pool.clear();
}

namespace {

template <typename F>
mlmd_status guarded(Domain* d, F&& fn) {
    if (!d) return MLMD_ERR_INVALID;
    if (d->latched != MLMD_OK) return MLMD_ERR_STATE;
    try {
        fn();
        d->err.clear();
        return MLMD_OK;
    } catch (const Error& e) {
        d->err = e.msg;
        if (e.status == MLMD_ERR_CUDA || e.status == MLMD_ERR_NUMERIC || e.status == MLMD_ERR_TIMEOUT)
            d->latched = e.status;
        return e.status;
    } catch (const std::bad_alloc&) {
        d->err = "host allocation failed";
        return MLMD_ERR_OOM;
    } catch (...) {
        d->err = "unexpected failure";
        d->latched = MLMD_ERR_STATE;
        return MLMD_ERR_STATE;
    }
}

void ensure_obs(Domain& d, int n) {
    if (d.obs_cap >= n) return;
    if (d.obs_dev) d.mem.put(d.obs_dev);
    d.obs_cap = std::max(n, 16);
    d.obs_dev = (double*)d.mem.get(sizeof(double) * 5 * d.obs_cap);
}

void ensure_A(Domain& d, int n) {
    if (d.A_cap >= n) return;
    if (d.A_dev) d.mem.put(d.A_dev);
    d.A_cap = std::max(n, 16);
    d.A_dev = (double*)d.mem.get(sizeof(double) * 3 * d.A_cap);
}

double* ensure_dense(Domain& d, size_t doubles) {
    const size_t bytes = doubles * sizeof(double);
    if (d.dense_bytes < bytes) {
        if (d.dense) d.mem.put(d.dense);
        d.dense = (double*)d.mem.get(bytes);
        d.dense_bytes = bytes;
    }
    return d.dense;
}

// out = h(A) in
void apply_h(Domain& d, const void* in, void* out, const double* Ak, double* obs_row = nullptr) {
    const bool nl = d.has_nl();
    if (gauge_on(d)) launch_nl_phase(d, Ak);
    if (nl) launch_project(d, in, d.Pa);
    StageArgs a;
    a.w = in;
    a.psi = nullptr;
    a.out = out;
    a.P = nl ? d.Pa : nullptr;
    a.A = Ak;
    a.gamma_re = 1.0;
    a.gamma_im = 0.0;
    a.obs = obs_row ? d.obs_part : nullptr;
    const int nblk = launch_stage(d, a);
    if (obs_row) {
        launch_obs_finish(d, d.obs_part, nblk, Ak, obs_row);
        if (gauge_on(d)) {
            for (int ax = 0; ax < 3; ++ax) launch_project(d, in, moment_buffer(d, ax), ax);
            launch_nl_current(d, d.Pa, obs_row);
        }
    }
}

void reorth(Domain& d, int kind);

}  // namespace
}  // namespace mlmd

// ---- split scheme helpers (Eq. 2) -----------------------------------------
namespace mlmd {
void launch_orbital_norms(Domain& d, const void* psi, double* nrm);
void launch_scale_orbitals(Domain& d, void* psi, const double* before, const double* after);
void launch_nl_apply(Domain& d, const void* in, const void* P, void* out, double gamma_im);
namespace {

// psi <- (1 - i dt/2 v_nl) psi, then each orbital back to its previous norm.
void apply_nnl(Domain& d) {
    double* nb = (double*)d.mem.get(sizeof(double) * d.ld * 2);
    double* na = nb + d.ld;
    launch_orbital_norms(d, d.psi, nb);
    launch_project(d, d.psi, d.Pa);
    launch_nl_apply(d, d.psi, d.Pa, d.psi, -0.5 * d.desc.dt);
    launch_orbital_norms(d, d.psi, na);
    launch_scale_orbitals(d, d.psi, nb, na);
    d.mem.put(nb);
}

void step_split(Domain& d, const double* Ak, double* obs_row) {
    d.pa_psi = false;
    if (obs_row) apply_h(d, d.psi, d.wb, Ak, obs_row);
    else if (gauge_on(d)) launch_nl_phase(d, Ak);     // N_nl at this step's A
    if (d.has_nl()) apply_nnl(d);
    if (sweep_on(d)) {
        // the local factor T4(h_loc) in one sweep
        launch_sweep(d, d.psi, Ak, nullptr);
        if (d.has_nl()) apply_nnl(d);
        return;
    }
    const double dt = d.desc.dt;
    const void* in = d.psi;
    void* outs[4] = {d.wa, d.wb, d.wa, d.psi};
    for (int s = 0; s < 4; ++s) {
        StageArgs a;
        a.w = in;
        a.psi = d.psi;
        a.out = outs[s];
        a.P = nullptr;
        a.A = Ak;
        a.gamma_re = 0.0;
        a.gamma_im = -dt / (double)(4 - s);
        a.obs = nullptr;
        launch_stage(d, a);
        in = outs[s];
    }
    if (d.has_nl()) apply_nnl(d);
}

void reorth(Domain& d, int kind) {
    d.pa_psi = false;
    const int n = d.desc.n_orb;
    const size_t mat = (size_t)n * n * 2;
    double* base = ensure_dense(d, mat * (kind == MLMD_ORTHO_LOWDIN ? 6 : 2) + 8);
    double* S = base;
    double* M = base + mat;
    int* info = (int*)(base + mat * (kind == MLMD_ORTHO_LOWDIN ? 6 : 2));
    const double dV = d.desc.h * d.desc.h * d.desc.h;
    launch_overlap(d, d.psi, d.psi, dV, S);
    if (kind == MLMD_ORTHO_LOWDIN) lowdin_inverse_sqrt(d, S, M, base + 2 * mat, info);
    else cholesky_inverse_upper(d, S, M, info);
    int h_info = 0;
    MLMD_CUDA(cudaMemcpyAsync(&h_info, info, sizeof(int), cudaMemcpyDeviceToHost, d.stream));
    MLMD_CUDA(cudaStreamSynchronize(d.stream));
    MLMD_REQUIRE(h_info == 0, MLMD_ERR_NUMERIC, "overlap matrix is not positive definite");
    {
        ProfScope ps(d.prof, MLMD_KERNEL_GEMM, d.stream);
        if (!launch_update_tc(d, d.psi, M, d.wa, kind == MLMD_ORTHO_CHOL)) launch_update(d, d.psi, M, d.wa);
    }
    std::swap(d.psi, d.wa);
}

// f (padded to ld with zeros) into the FP64 and working-type copies.
void upload_occupations(Domain& d, const std::vector<double>& f) {
    MLMD_CUDA(cudaMemcpyAsync(d.f, f.data(), sizeof(double) * d.ld, cudaMemcpyHostToDevice, d.stream));
    if (d.c64()) {
        std::vector<float> ff(f.begin(), f.end());
        MLMD_CUDA(cudaMemcpyAsync(d.fR, ff.data(), sizeof(float) * d.ld, cudaMemcpyHostToDevice, d.stream));
        MLMD_CUDA(cudaStreamSynchronize(d.stream));
    } else {
        MLMD_CUDA(cudaMemcpyAsync(d.fR, f.data(), sizeof(double) * d.ld, cudaMemcpyHostToDevice, d.stream));
        MLMD_CUDA(cudaStreamSynchronize(d.stream));
    }
}

void check_desc(const mlmd_domain_desc* s) {
    MLMD_REQUIRE(s != nullptr, MLMD_ERR_INVALID, "null descriptor");
    for (int i = 0; i < 3; ++i) MLMD_REQUIRE(s->n[i] >= 4 && s->n[i] <= 4096, MLMD_ERR_INVALID, "grid size out of range");
    MLMD_REQUIRE(std::isfinite(s->h) && s->h > 0.0, MLMD_ERR_INVALID, "h must be positive");
    MLMD_REQUIRE(s->n_orb >= 1 && s->n_orb <= 65536, MLMD_ERR_INVALID, "n_orb out of range");
    MLMD_REQUIRE(s->fd_order == 2 || s->fd_order == 4, MLMD_ERR_INVALID, "fd_order must be 2 or 4");
    MLMD_REQUIRE(s->precision == MLMD_C128 || s->precision == MLMD_C64, MLMD_ERR_INVALID, "bad precision");
    MLMD_REQUIRE(s->gemm_mode >= MLMD_GEMM_FP32 && s->gemm_mode <= MLMD_GEMM_FP16, MLMD_ERR_INVALID, "bad gemm_mode");
    MLMD_REQUIRE(s->scheme == MLMD_SCHEME_FULL || s->scheme == MLMD_SCHEME_SPLIT, MLMD_ERR_INVALID, "bad scheme");
    MLMD_REQUIRE(std::isfinite(s->dt) && s->dt > 0.0, MLMD_ERR_INVALID, "dt must be positive");
    MLMD_REQUIRE(s->ortho_every >= 0, MLMD_ERR_INVALID, "ortho_every must be >= 0");
    MLMD_REQUIRE(s->ortho_kind == MLMD_ORTHO_CHOL || s->ortho_kind == MLMD_ORTHO_LOWDIN, MLMD_ERR_INVALID,
                 "bad ortho_kind");
    const int64_t ng = (int64_t)s->n[0] * s->n[1] * s->n[2];
    MLMD_REQUIRE(ng < ((int64_t)1 << 31), MLMD_ERR_INVALID, "grid too large");
    const int64_t nv = (int64_t)(s->n_orb + 7) / 8 * 8 / (s->precision == MLMD_C64 ? 2 : 1);
    MLMD_REQUIRE((int64_t)s->n[0] * nv < ((int64_t)1 << 31), MLMD_ERR_INVALID, "grid line too long");
}

}  // namespace
}  // namespace mlmd

using namespace mlmd;

extern "C" {

int32_t mlmd_abi_version(void) { return 1; }

const char* mlmd_status_string(mlmd_status s) {
    switch (s) {
        case MLMD_OK: return "ok";
        case MLMD_ERR_INVALID: return "invalid argument";
        case MLMD_ERR_OOM: return "out of device memory";
        case MLMD_ERR_CUDA: return "CUDA error";
        case MLMD_ERR_NUMERIC: return "numeric failure";
        case MLMD_ERR_TIMEOUT: return "device wait timed out";
        case MLMD_ERR_STATE: return "invalid state";
        case MLMD_ERR_UNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

mlmd_status mlmd_domain_create(const mlmd_domain_desc* desc, const mlmd_allocator* allocator, void* stream,
                               mlmd_domain_t* out) {
    if (!out) return MLMD_ERR_INVALID;
    *out = nullptr;
    mlmd_domain* d = nullptr;
    try {
        check_desc(desc);
        if (allocator) MLMD_REQUIRE(allocator->alloc && allocator->free, MLMD_ERR_INVALID, "allocator needs alloc and free");
        d = new mlmd_domain();
    } catch (const Error& e) {
        return e.status;
    } catch (...) {
        return MLMD_ERR_OOM;
    }
    d->desc = *desc;
    mlmd_status st = guarded(d, [&] {
        MLMD_CUDA(cudaGetDevice(&d->device));
        d->stream = (cudaStream_t)stream;
        d->mem.stream = d->stream;
        d->mem.device = d->device;
        if (allocator) { d->mem.a = *allocator; d->mem.custom = true; }
        d->ng = (int64_t)desc->n[0] * desc->n[1] * desc->n[2];
        d->ld = padded_orbitals(desc->n_orb);
        d->elem = desc->precision == MLMD_C64 ? 8 : 16;
        d->state_bytes = (size_t)d->ng * d->ld * d->elem;
        d->psi = d->mem.get(d->state_bytes);
        d->wa = d->mem.get(d->state_bytes);
        d->wb = d->mem.get(d->state_bytes);
        const size_t rsz = d->c64() ? sizeof(float) : sizeof(double);
        d->V = d->mem.get(rsz * d->ng);
        d->V64 = (double*)d->mem.get(sizeof(double) * d->ng);
        d->f = (double*)d->mem.get(sizeof(double) * d->ld);
        d->fR = d->mem.get(rsz * d->ld);
        d->obs_blocks = stage_blocks(*d);
        d->err_flag = (int*)d->mem.get(sizeof(int));
        MLMD_CUDA(cudaMemsetAsync(d->err_flag, 0, sizeof(int), d->stream));
        tma_setup(*d);
        sweep_setup(*d);
        if (d->sweep.ok)
            d->obs_blocks = std::max(d->obs_blocks, d->sweep.CX * d->sweep.CY * (d->ld / d->sweep.VPC));
        d->obs_part = (double*)d->mem.get(sizeof(double) * 5 * (size_t)std::max(d->obs_blocks, density_blocks(*d) * 2));
        MLMD_CUDA(cudaMemsetAsync(d->psi, 0, d->state_bytes, d->stream));
        MLMD_CUDA(cudaMemsetAsync(d->V, 0, rsz * d->ng, d->stream));
        MLMD_CUDA(cudaMemsetAsync(d->V64, 0, sizeof(double) * d->ng, d->stream));
        std::vector<double> f(d->ld, 0.0);
        for (int i = 0; i < desc->n_orb; ++i) f[i] = 2.0;
        upload_occupations(*d, f);
    });
    if (st != MLMD_OK) {
        d->mem.release_all();
        (void)cudaStreamSynchronize(d->stream);
        delete d;
        return st;
    }
    *out = d;
    return MLMD_OK;
}

mlmd_status mlmd_domain_destroy(mlmd_domain_t dom) {
    if (!dom) return MLMD_ERR_INVALID;
    dom->mem.release_all();
    cudaError_t e = cudaStreamSynchronize(dom->stream);
    if (!dom->mem.custom && e == cudaSuccess) (void)cudaMemPoolTrimTo(library_pool(dom->device), 0);
    dom->prof.destroy();
    tma_release(*dom);
    nl_tc_release(*dom);
    if (dom->side) {
        if (cudaStreamSynchronize(dom->side) != cudaSuccess) e = cudaErrorUnknown;
        (void)cudaStreamDestroy(dom->side);
    }
    if (dom->ev_rows) (void)cudaEventDestroy(dom->ev_rows);
    if (dom->ev_trail) (void)cudaEventDestroy(dom->ev_trail);
    delete dom;
    return e == cudaSuccess ? MLMD_OK : MLMD_ERR_CUDA;
}

mlmd_status mlmd_set_orbitals(mlmd_domain_t d, const void* psi, int32_t on_device) {
    return guarded(d, [&] {
        MLMD_REQUIRE(psi != nullptr, MLMD_ERR_INVALID, "null orbitals");
        d->pa_psi = false;
        const size_t src_pitch = (size_t)d->desc.n_orb * d->elem, dst_pitch = (size_t)d->ld * d->elem;
        const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        if (src_pitch == dst_pitch) {
            // no padding orbitals: the rows are contiguous, one flat copy
            MLMD_CUDA(cudaMemcpyAsync(d->psi, psi, d->state_bytes, kind, d->stream));
        } else {
            MLMD_CUDA(cudaMemsetAsync(d->psi, 0, d->state_bytes, d->stream));     // padding orbitals stay zero
            const void* src = psi;
            if (!on_device) {
                // from the host as one flat copy into the work buffer, then
                // into the padded rows on the device
                MLMD_CUDA(cudaMemcpyAsync(d->wa, psi, src_pitch * (size_t)d->ng, cudaMemcpyHostToDevice, d->stream));
                src = d->wa;
            }
            MLMD_CUDA(cudaMemcpy2DAsync(d->psi, dst_pitch, src, src_pitch, src_pitch, (size_t)d->ng,
                                        cudaMemcpyDeviceToDevice, d->stream));
        }
        if (!d->psi0) d->psi0 = d->mem.get(d->state_bytes);
        MLMD_CUDA(cudaMemcpyAsync(d->psi0, d->psi, d->state_bytes, cudaMemcpyDeviceToDevice, d->stream));
        if (!on_device) MLMD_CUDA(cudaStreamSynchronize(d->stream));
        d->psi0_valid = true;
        d->step = 0;
    });
}

mlmd_status mlmd_get_orbitals(mlmd_domain_t d, void* psi_out, int32_t on_device) {
    return guarded(d, [&] {
        MLMD_REQUIRE(psi_out != nullptr, MLMD_ERR_INVALID, "null output");
        const size_t dst_pitch = (size_t)d->desc.n_orb * d->elem, src_pitch = (size_t)d->ld * d->elem;
        const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        if (src_pitch == dst_pitch) {
            MLMD_CUDA(cudaMemcpyAsync(psi_out, d->psi, d->state_bytes, kind, d->stream));
        } else if (on_device) {
            MLMD_CUDA(cudaMemcpy2DAsync(psi_out, dst_pitch, d->psi, src_pitch, dst_pitch, (size_t)d->ng, kind, d->stream));
        } else {
            // packed on the device into the work buffer, then one flat copy to the host
            MLMD_CUDA(cudaMemcpy2DAsync(d->wa, dst_pitch, d->psi, src_pitch, dst_pitch, (size_t)d->ng,
                                        cudaMemcpyDeviceToDevice, d->stream));
            MLMD_CUDA(cudaMemcpyAsync(psi_out, d->wa, dst_pitch * (size_t)d->ng, cudaMemcpyDeviceToHost, d->stream));
        }
        if (!on_device) MLMD_CUDA(cudaStreamSynchronize(d->stream));
    });
}

mlmd_status mlmd_set_occupations(mlmd_domain_t d, const double* f) {
    return guarded(d, [&] {
        MLMD_REQUIRE(f != nullptr, MLMD_ERR_INVALID, "null occupations");
        std::vector<double> h(d->ld, 0.0);
        for (int i = 0; i < d->desc.n_orb; ++i) {
            MLMD_REQUIRE(std::isfinite(f[i]), MLMD_ERR_INVALID, "occupation not finite");
            h[i] = f[i];
        }
        upload_occupations(*d, h);
    });
}

mlmd_status mlmd_set_potential(mlmd_domain_t d, const double* v) {
    return guarded(d, [&] {
        MLMD_REQUIRE(v != nullptr, MLMD_ERR_INVALID, "null potential");
        for (int64_t g = 0; g < d->ng; ++g) MLMD_REQUIRE(std::isfinite(v[g]), MLMD_ERR_INVALID, "potential not finite");
        MLMD_CUDA(cudaMemcpyAsync(d->V64, v, sizeof(double) * d->ng, cudaMemcpyHostToDevice, d->stream));
        if (d->c64()) {
            std::vector<float> h(d->ng);
            for (int64_t g = 0; g < d->ng; ++g) h[g] = (float)v[g];
            MLMD_CUDA(cudaMemcpyAsync(d->V, h.data(), sizeof(float) * d->ng, cudaMemcpyHostToDevice, d->stream));
            MLMD_CUDA(cudaStreamSynchronize(d->stream));
        } else {
            MLMD_CUDA(cudaMemcpyAsync(d->V, v, sizeof(double) * d->ng, cudaMemcpyHostToDevice, d->stream));
            MLMD_CUDA(cudaStreamSynchronize(d->stream));
        }
    });
}

mlmd_status mlmd_set_projectors(mlmd_domain_t d, int32_t n_atoms, const double* pos, int32_t n_proj, double r_c,
                                double r_cut, const double* D) {
    return guarded(d, [&] {
        MLMD_REQUIRE(n_atoms >= 0, MLMD_ERR_INVALID, "n_atoms < 0");
        if (n_atoms > 0) {
            MLMD_REQUIRE(pos && D, MLMD_ERR_INVALID, "null positions or strengths");
            MLMD_REQUIRE(n_proj == 4 || n_proj == 8, MLMD_ERR_INVALID, "n_proj_per_atom must be 4 or 8");
            MLMD_REQUIRE(std::isfinite(r_c) && r_c > 0 && std::isfinite(r_cut) && r_cut > 0, MLMD_ERR_INVALID,
                         "r_c and r_cut must be positive");
            for (int i = 0; i < 3 * n_atoms; ++i) MLMD_REQUIRE(std::isfinite(pos[i]), MLMD_ERR_INVALID, "position not finite");
            for (int i = 0; i < n_atoms * n_proj; ++i) MLMD_REQUIRE(std::isfinite(D[i]), MLMD_ERR_INVALID, "D not finite");
        }
        build_projectors(*d, n_atoms, pos, n_proj, r_c, r_cut, D);
    });
}

mlmd_status mlmd_set_nonlocal_gauge(mlmd_domain_t d, int32_t gauge) {
    return guarded(d, [&] {
        MLMD_REQUIRE(gauge == MLMD_NL_GAUGE_REAL || gauge == MLMD_NL_GAUGE_VELOCITY, MLMD_ERR_INVALID,
                     "unknown nonlocal gauge");
        if (gauge == d->nl_gauge) return;
        d->nl_gauge = gauge;
        d->pa_psi = false;       // carried projections were taken with the other projectors
        if (gauge == MLMD_NL_GAUGE_VELOCITY) gauge_build(*d);
        else gauge_release(*d);
    });
}

mlmd_status mlmd_get_projector_lists(mlmd_domain_t d, int64_t* off, int32_t* idx, size_t idx_cap, double* beta) {
    return guarded(d, [&] {
        MLMD_REQUIRE(off != nullptr, MLMD_ERR_INVALID, "null off");
        const Nonlocal& nl = d->nl;
        if (nl.n_atoms == 0) { off[0] = 0; return; }
        std::memcpy(off, nl.h_off.data(), sizeof(int64_t) * (nl.n_atoms + 1));
        if (idx) {
            MLMD_REQUIRE(idx_cap >= (size_t)nl.n_list, MLMD_ERR_INVALID, "idx capacity too small");
            MLMD_CUDA(cudaMemcpyAsync(idx, nl.idx, sizeof(int32_t) * nl.n_list, cudaMemcpyDeviceToHost, d->stream));
            if (beta)
                MLMD_CUDA(cudaMemcpyAsync(beta, nl.beta64, sizeof(double) * nl.n_list * nl.n_proj,
                                          cudaMemcpyDeviceToHost, d->stream));
            MLMD_CUDA(cudaStreamSynchronize(d->stream));
        }
    });
}

mlmd_status mlmd_propagate(mlmd_domain_t d, int32_t n_steps, const double* A, double* obs_out) {
    return guarded(d, [&] {
        MLMD_REQUIRE(n_steps >= 0, MLMD_ERR_INVALID, "n_steps < 0");
        if (n_steps == 0) return;
        MLMD_REQUIRE(A != nullptr, MLMD_ERR_INVALID, "null A");
        for (int i = 0; i < 3 * n_steps; ++i) MLMD_REQUIRE(std::isfinite(A[i]), MLMD_ERR_INVALID, "A not finite");
        ensure_A(*d, n_steps);
        MLMD_CUDA(cudaMemcpyAsync(d->A_dev, A, sizeof(double) * 3 * n_steps, cudaMemcpyHostToDevice, d->stream));
        if (obs_out) ensure_obs(*d, n_steps);
        tma_autotune(*d, d->A_dev);
        sweep_autotune(*d, d->A_dev);
        for (int k = 0; k < n_steps; ++k) {
            const double* Ak = d->A_dev + 3 * k;
            double* row = obs_out ? d->obs_dev + 5 * k : nullptr;
            if (d->desc.scheme == MLMD_SCHEME_FULL) step_full(*d, Ak, row);
            else step_split(*d, Ak, row);
            d->step++;
            if (d->desc.ortho_every > 0 && d->step % d->desc.ortho_every == 0) reorth(*d, d->desc.ortho_kind);
        }
        if (obs_out) {
            MLMD_CUDA(cudaMemcpyAsync(obs_out, d->obs_dev, sizeof(double) * 5 * n_steps, cudaMemcpyDeviceToHost, d->stream));
        }
        int h_err = 0;
        MLMD_CUDA(cudaMemcpyAsync(&h_err, d->err_flag, sizeof(int), cudaMemcpyDeviceToHost, d->stream));
        MLMD_CUDA(cudaStreamSynchronize(d->stream));
        MLMD_CUDA(cudaGetLastError());
        MLMD_REQUIRE(h_err == 0, MLMD_ERR_TIMEOUT, "a device-side wait timed out");
        if (obs_out)
            for (int i = 0; i < 5 * n_steps; ++i)
                MLMD_REQUIRE(std::isfinite(obs_out[i]), MLMD_ERR_NUMERIC, "observable is NaN or Inf");
    });
}

mlmd_status mlmd_density_current(mlmd_domain_t d, const double* A, void* rho, void* j, double* J, int32_t on_device) {
    return guarded(d, [&] {
        MLMD_REQUIRE(A != nullptr, MLMD_ERR_INVALID, "null A");
        const size_t rsz = d->c64() ? sizeof(float) : sizeof(double);
        ensure_A(*d, 1);
        double* Ad = d->A_dev;
        MLMD_CUDA(cudaMemcpyAsync(Ad, A, sizeof(double) * 3, cudaMemcpyHostToDevice, d->stream));
        void* rho_d = rho;
        void* j_d = j;
        if (!on_device) {
            rho_d = rho ? d->wa : nullptr;                               // reuse work buffers as staging
            j_d = j ? (void*)((char*)d->wb) : nullptr;
        }
        const int nb = density_blocks(*d);
        double* part = d->obs_part;
        launch_density_current(*d, Ad, rho_d, j_d, part, nb);
        double* tot = d->obs_part + 3 * (size_t)nb;
        launch_reduce_partials(*d, part, nb, 3, tot);
        double Jh[3];
        MLMD_CUDA(cudaMemcpyAsync(Jh, tot, sizeof(double) * 3, cudaMemcpyDeviceToHost, d->stream));
        if (!on_device) {
            if (rho) MLMD_CUDA(cudaMemcpyAsync(rho, rho_d, rsz * d->ng, cudaMemcpyDeviceToHost, d->stream));
            if (j) MLMD_CUDA(cudaMemcpyAsync(j, j_d, rsz * 3 * d->ng, cudaMemcpyDeviceToHost, d->stream));
        }
        MLMD_CUDA(cudaStreamSynchronize(d->stream));
        const double dV = d->desc.h * d->desc.h * d->desc.h;
        if (J)
            for (int a = 0; a < 3; ++a) J[a] = dV * Jh[a];
    });
}

mlmd_status mlmd_overlap(mlmd_domain_t d, double* S_out) {
    return guarded(d, [&] {
        MLMD_REQUIRE(S_out != nullptr, MLMD_ERR_INVALID, "null output");
        const int n = d->desc.n_orb;
        double* S = ensure_dense(*d, (size_t)n * n * 2);
        launch_overlap(*d, d->psi, d->psi, d->desc.h * d->desc.h * d->desc.h, S);
        MLMD_CUDA(cudaMemcpyAsync(S_out, S, sizeof(double) * n * n * 2, cudaMemcpyDeviceToHost, d->stream));
        MLMD_CUDA(cudaStreamSynchronize(d->stream));
        check_err_flag(*d);
    });
}

mlmd_status mlmd_reorthonormalize(mlmd_domain_t d, int32_t kind) {
    return guarded(d, [&] {
        MLMD_REQUIRE(kind == MLMD_ORTHO_CHOL || kind == MLMD_ORTHO_LOWDIN, MLMD_ERR_INVALID, "bad kind");
        reorth(*d, kind);
        MLMD_CUDA(cudaStreamSynchronize(d->stream));
        check_err_flag(*d);
    });
}

// C = dV Psi(0)^H Psi(t) and its occupation sums on the device; fills
// fs (device [n_orb]) and tot (device [2], see launch_occupations).
static void reference_occupations(Domain& d, double** fs, double** tot) {
    const int n = d.desc.n_orb;
    double* base = ensure_dense(d, (size_t)n * n * 2 + 2 * (size_t)n + 2);
    double* C = base;
    *fs = base + (size_t)n * n * 2;
    double* rs = *fs + n;
    *tot = rs + n;
    launch_overlap(d, d.psi0, d.psi, d.desc.h * d.desc.h * d.desc.h, C);
    launch_occupations(d, C, *fs, rs, *tot);
}

mlmd_status mlmd_excitation(mlmd_domain_t d, double* n_exc) {
    return guarded(d, [&] {
        MLMD_REQUIRE(n_exc != nullptr, MLMD_ERR_INVALID, "null output");
        MLMD_REQUIRE(d->psi0_valid, MLMD_ERR_STATE, "no reference orbitals (call mlmd_set_orbitals)");
        double *fs = nullptr, *tot = nullptr;
        reference_occupations(*d, &fs, &tot);
        double t[2];
        MLMD_CUDA(cudaMemcpyAsync(t, tot, sizeof(t), cudaMemcpyDeviceToHost, d->stream));
        MLMD_CUDA(cudaStreamSynchronize(d->stream));
        check_err_flag(*d);
        *n_exc = 2.0 * ((double)d->desc.n_orb - t[1]);
    });
}

mlmd_status mlmd_occupations(mlmd_domain_t d, double* f_out, double* n_exc) {
    return guarded(d, [&] {
        MLMD_REQUIRE(f_out != nullptr || n_exc != nullptr, MLMD_ERR_INVALID, "no output");
        MLMD_REQUIRE(d->psi0_valid, MLMD_ERR_STATE, "no reference orbitals (call mlmd_set_orbitals)");
        double *fs = nullptr, *tot = nullptr;
        reference_occupations(*d, &fs, &tot);
        double t[2];
        if (f_out)
            MLMD_CUDA(cudaMemcpyAsync(f_out, fs, sizeof(double) * d->desc.n_orb, cudaMemcpyDeviceToHost, d->stream));
        MLMD_CUDA(cudaMemcpyAsync(t, tot, sizeof(t), cudaMemcpyDeviceToHost, d->stream));
        MLMD_CUDA(cudaStreamSynchronize(d->stream));
        check_err_flag(*d);
        if (n_exc) *n_exc = t[0];
    });
}

mlmd_status mlmd_ks_correction(mlmd_domain_t d, const double* delta) {
    return guarded(d, [&] {
        MLMD_REQUIRE(delta != nullptr && std::isfinite(delta[0]) && std::isfinite(delta[1]), MLMD_ERR_INVALID,
                     "delta must be two finite numbers");
        MLMD_REQUIRE(d->psi0_valid, MLMD_ERR_STATE, "no reference orbitals (call mlmd_set_orbitals)");
        const int n = d->desc.n_orb;
        double* C = ensure_dense(*d, (size_t)n * n * 2);
        // C = dV Psi(0)^H Psi(t), then C <- -delta C, then Psi(t) + Psi(0) C
        launch_overlap(*d, d->psi0, d->psi, d->desc.h * d->desc.h * d->desc.h, C);
        launch_scale_complex(*d, C, (int64_t)n * n, -delta[0], -delta[1]);
        if (!launch_gemm_add_tc(*d, d->psi0, C, d->psi, d->wa)) launch_update(*d, d->psi0, C, d->wa, d->psi);
        std::swap(d->psi, d->wa);
        d->pa_psi = false;
        MLMD_CUDA(cudaStreamSynchronize(d->stream));
        check_err_flag(*d);
    });
}

mlmd_status mlmd_profile_enable(mlmd_domain_t d, int32_t enable) {
    return guarded(d, [&] {
        MLMD_CUDA(cudaStreamSynchronize(d->stream));
        d->prof.reset();
        d->prof.on = enable != 0;
    });
}

mlmd_status mlmd_profile_read(mlmd_domain_t d, int32_t kind, double* total_ms, uint64_t* launches) {
    return guarded(d, [&] {
        MLMD_REQUIRE(kind >= 0 && kind < MLMD_KERNEL_KINDS && total_ms && launches, MLMD_ERR_INVALID,
                     "bad profile query");
        MLMD_CUDA(cudaStreamSynchronize(d->stream));
        d->prof.collect();
        *total_ms = d->prof.total_ms[kind];
        *launches = d->prof.count[kind];
    });
}

uint64_t mlmd_launch_count(mlmd_domain_t d) { return d ? d->launches : 0; }

const char* mlmd_last_error(mlmd_domain_t d) { return d ? d->err.c_str() : "null handle"; }

}  // extern "C"
