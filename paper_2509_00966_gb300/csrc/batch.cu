// Batched form: many uneven DC domains (Sec. V.A.1) stepped together on one
// GPU.  One time step of all domains is captured once as a CUDA graph; the
// graph reads each domain's vector potential from a device table through a
// device step counter, so the same graph is replayed for every step.  The
// domains are spread over kBranches parallel branches of the graph (forked
// after the step counter is read, joined before it advances), so kernels of
// different domains can run side by side and fill each other's tails.
#include <algorithm>
#include <cmath>
#include <vector>

#include "mlmd_internal.cuh"

namespace mlmd {
namespace {

constexpr int kBranches = 8;

// A_cur[d] = A_all[d][ctr]
__global__ void k_batch_begin(int n_dom, int n_steps, const double* __restrict__ A_all, const int* __restrict__ ctr,
                              double* __restrict__ A_cur) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_dom * 3) return;
    const int d = i / 3, a = i % 3;
    const int k = *ctr;
    A_cur[i] = k < n_steps ? A_all[((int64_t)d * n_steps + k) * 3 + a] : 0.0;
}

// obs_all[d][ctr] = obs_cur[d]; ctr += 1
__global__ void k_batch_end(int n_dom, int n_steps, const double* __restrict__ obs_cur, int* __restrict__ ctr,
                            double* __restrict__ obs_all) {
    const int k = *ctr;
    for (int i = threadIdx.x; i < n_dom * 5; i += blockDim.x) {
        const int d = i / 5, c = i % 5;
        if (obs_all && k < n_steps) obs_all[((int64_t)d * n_steps + k) * 5 + c] = obs_cur[i];
    }
    __syncthreads();
    if (threadIdx.x == 0) *ctr = k + 1;
}

}  // namespace
}  // namespace mlmd

using namespace mlmd;

extern "C" {

mlmd_status mlmd_batch_create(int32_t n_domains, const mlmd_domain_t* doms, mlmd_batch_t* out) {
    if (!out || n_domains < 1 || !doms) return MLMD_ERR_INVALID;
    *out = nullptr;
    cudaStream_t st = doms[0] ? doms[0]->stream : nullptr;
    for (int i = 0; i < n_domains; ++i) {
        Domain* d = doms[i];
        if (!d) return MLMD_ERR_INVALID;
        if (d->latched != MLMD_OK) return MLMD_ERR_STATE;
        if (d->desc.precision != MLMD_C64 || d->desc.scheme != MLMD_SCHEME_FULL || d->desc.ortho_every != 0)
            return MLMD_ERR_UNSUPPORTED;
        if (d->stream != st || d->desc.dt != doms[0]->desc.dt) return MLMD_ERR_INVALID;
    }
    mlmd_batch* b = new (std::nothrow) mlmd_batch();
    if (!b) return MLMD_ERR_OOM;
    b->doms.assign(doms, doms + n_domains);
    b->stream = st;
    (void)cudaGetDevice(&b->device);
    *out = b;
    return MLMD_OK;
}

mlmd_status mlmd_batch_destroy(mlmd_batch_t b) {
    if (!b) return MLMD_ERR_INVALID;
    delete b;
    return MLMD_OK;
}

mlmd_status mlmd_batch_propagate(mlmd_batch_t b, int32_t n_steps, const double* A, double* obs_out) {
    if (!b) return MLMD_ERR_INVALID;
    if (n_steps < 0) return MLMD_ERR_INVALID;
    if (n_steps == 0) return MLMD_OK;
    if (!A) return MLMD_ERR_INVALID;
    const int nd = (int)b->doms.size();
    for (int64_t i = 0; i < (int64_t)nd * n_steps * 3; ++i)
        if (!std::isfinite(A[i])) return MLMD_ERR_INVALID;
    Domain& d0 = *b->doms[0];
    for (auto* d : b->doms)
        if (d->latched != MLMD_OK) return MLMD_ERR_STATE;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    double *A_all = nullptr, *A_cur = nullptr, *obs_cur = nullptr, *obs_all = nullptr;
    int* ctr = nullptr;
    try {
        const cudaStream_t st = b->stream;
        A_all = (double*)d0.mem.get(sizeof(double) * 3 * (size_t)nd * n_steps);
        A_cur = (double*)d0.mem.get(sizeof(double) * 3 * nd);
        obs_cur = (double*)d0.mem.get(sizeof(double) * 5 * nd);
        obs_all = obs_out ? (double*)d0.mem.get(sizeof(double) * 5 * (size_t)nd * n_steps) : nullptr;
        ctr = (int*)d0.mem.get(sizeof(int));
        MLMD_CUDA(cudaMemcpyAsync(A_all, A, sizeof(double) * 3 * (size_t)nd * n_steps, cudaMemcpyHostToDevice, st));
        MLMD_CUDA(cudaMemsetAsync(ctr, 0, sizeof(int), st));
        MLMD_CUDA(cudaMemsetAsync(obs_cur, 0, sizeof(double) * 5 * nd, st));
        // tile choice and projections of the current orbitals, outside the
        // graph, so that the captured step is the steady-state one
        for (auto* d : b->doms) {
            tma_autotune(*d, A_all);
            sweep_autotune(*d, A_all);
        }
        for (auto* d : b->doms)
            if (d->has_nl() && !d->pa_psi && (nltc_on(*d) || tma_fused_nl(*d))) {
                if (nltc_on(*d)) launch_nl_project_tc(*d, d->psi, d->Pa, false);
                else launch_project(*d, d->psi, d->Pa);
                d->pa_psi = true;
            }
        MLMD_CUDA(cudaStreamSynchronize(st));
        // Capture one step of every domain on a private stream (the legacy
        // default stream cannot be captured), ordered after the caller's
        // stream by an event and joined back the same way.
        cudaStream_t cap = nullptr;
        cudaEvent_t ev_in = nullptr, ev_out = nullptr, ev_fork = nullptr;
        const int nbr = std::min(nd, kBranches);
        std::vector<cudaStream_t> br(nbr, nullptr);
        std::vector<cudaEvent_t> ev_join(nbr, nullptr);
        struct Restore {
            std::vector<mlmd_domain*>& ds;
            cudaStream_t orig;
            cudaStream_t& cap;
            std::vector<cudaStream_t>& br;
            std::vector<cudaEvent_t>& joins;
            cudaEvent_t &a, &b, &f;
            ~Restore() {
                for (auto* d : ds) { d->stream = orig; d->mem.stream = orig; }
                if (cap) (void)cudaStreamSynchronize(cap);
                for (auto s : br) if (s) (void)cudaStreamDestroy(s);
                for (auto e : joins) if (e) (void)cudaEventDestroy(e);
                if (cap) (void)cudaStreamDestroy(cap);
                if (a) (void)cudaEventDestroy(a);
                if (b) (void)cudaEventDestroy(b);
                if (f) (void)cudaEventDestroy(f);
            }
        } restore{b->doms, st, cap, br, ev_join, ev_in, ev_out, ev_fork};
        MLMD_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        MLMD_CUDA(cudaEventCreateWithFlags(&ev_in, cudaEventDisableTiming));
        MLMD_CUDA(cudaEventCreateWithFlags(&ev_out, cudaEventDisableTiming));
        MLMD_CUDA(cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming));
        for (int k = 0; k < nbr; ++k) {
            MLMD_CUDA(cudaStreamCreateWithFlags(&br[k], cudaStreamNonBlocking));
            MLMD_CUDA(cudaEventCreateWithFlags(&ev_join[k], cudaEventDisableTiming));
        }
        std::vector<uint64_t> before;
        std::vector<bool> prof_on;
        for (int i = 0; i < nd; ++i) {
            mlmd_domain* d = b->doms[i];
            d->stream = br[i % nbr];
            d->mem.stream = br[i % nbr];
            before.push_back(d->launches);
            prof_on.push_back(d->prof.on);
            d->prof.on = false;   // no timing events inside the graph
        }
        MLMD_CUDA(cudaEventRecord(ev_in, st));
        MLMD_CUDA(cudaStreamWaitEvent(cap, ev_in, 0));
        MLMD_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
        try {
            k_batch_begin<<<(nd * 3 + 255) / 256, 256, 0, cap>>>(nd, n_steps, A_all, ctr, A_cur);
            MLMD_CUDA(cudaEventRecord(ev_fork, cap));
            for (int k = 0; k < nbr; ++k) MLMD_CUDA(cudaStreamWaitEvent(br[k], ev_fork, 0));
            for (int i = 0; i < nd; ++i)
                step_full(*b->doms[i], A_cur + 3 * i, obs_out ? obs_cur + 5 * i : nullptr);
            for (int k = 0; k < nbr; ++k) {
                MLMD_CUDA(cudaEventRecord(ev_join[k], br[k]));
                MLMD_CUDA(cudaStreamWaitEvent(cap, ev_join[k], 0));
            }
            k_batch_end<<<1, 256, 0, cap>>>(nd, n_steps, obs_cur, ctr, obs_all);
        } catch (...) {
            cudaGraph_t g = nullptr;
            (void)cudaStreamEndCapture(cap, &g);
            if (g) (void)cudaGraphDestroy(g);
            throw;
        }
        MLMD_CUDA(cudaStreamEndCapture(cap, &graph));
        MLMD_CUDA(cudaGraphInstantiate(&exec, graph, 0));
        // every captured kernel runs once per replay
        for (int i = 0; i < nd; ++i) {
            const uint64_t captured = b->doms[i]->launches - before[i];
            b->doms[i]->launches = before[i] + captured * (uint64_t)n_steps;
            b->doms[i]->prof.on = prof_on[i];
        }
        for (int k = 0; k < n_steps; ++k) MLMD_CUDA(cudaGraphLaunch(exec, cap));
        MLMD_CUDA(cudaEventRecord(ev_out, cap));
        MLMD_CUDA(cudaStreamWaitEvent(st, ev_out, 0));
        if (obs_out)
            MLMD_CUDA(cudaMemcpyAsync(obs_out, obs_all, sizeof(double) * 5 * (size_t)nd * n_steps,
                                      cudaMemcpyDeviceToHost, st));
        MLMD_CUDA(cudaStreamSynchronize(st));
        MLMD_CUDA(cudaGetLastError());
        // a stage or projection kernel inside the graph that gave up a bounded
        // wait has left its domain's orbitals wrong: report it per domain
        for (auto* d : b->doms) {
            d->stream = st;
            check_err_flag(*d);
        }
        (void)cudaGraphExecDestroy(exec);
        (void)cudaGraphDestroy(graph);
        exec = nullptr;
        graph = nullptr;
        d0.launches += 2ull * (uint64_t)n_steps;
        for (auto* d : b->doms) d->step += n_steps;
        d0.mem.put(A_all);
        d0.mem.put(A_cur);
        d0.mem.put(obs_cur);
        d0.mem.put(obs_all);
        d0.mem.put(ctr);
        if (obs_out)
            for (int64_t i = 0; i < (int64_t)nd * n_steps * 5; ++i)
                if (!std::isfinite(obs_out[i])) {
                    d0.err = "observable is NaN or Inf";
                    return MLMD_ERR_NUMERIC;
                }
        return MLMD_OK;
    } catch (const Error& e) {
        if (exec) (void)cudaGraphExecDestroy(exec);
        if (graph) (void)cudaGraphDestroy(graph);
        d0.err = e.msg;
        if (e.status == MLMD_ERR_CUDA || e.status == MLMD_ERR_TIMEOUT)
            for (auto* d : b->doms) d->latched = e.status;
        return e.status;
    } catch (...) {
        return MLMD_ERR_STATE;
    }
}

}  // extern "C"
