// Discrete adjoint of the Taylor-4 map with checkpointing.
//
// Forward: psi_{k+1} = T_k psi_k, T_k = sum_j c_j h_k^j, c_j = (-i dt)^j / j!.
// Loss L = 2 (N_o - sum_{n,m} |C_nm|^2), C = dV Psi(0)^dagger Psi(T), the
// per-domain excited-electron count of Sec. V.A.8.  With Euclidean inner
// products and lam = dL/dpsi*:
//   lam_N = -2 dV Psi(0) C,   lam_k = T_k^dagger lam_{k+1} = sum_j conj(c_j) h_k^j lam_{k+1},
//   dL/dA_{k,a} = 2 Re sum_p <z_p | (-i G_a + A_a) u_p>,
//   dL/dV(r)   += 2 Re sum_p sum_o conj(z_p)(r) u_p(r),
// where u_p = h^p psi_k (p < 4), w_q = h^q lam_{k+1} and
// z_p = sum_{q <= 3-p} conj(c_{q+p+1}) w_q (the double sum over j and p
// regrouped by p).
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include "mlmd_internal.cuh"

namespace mlmd {
namespace {

struct Scratch {
    Domain& d;
    std::vector<void*> blocks;
    explicit Scratch(Domain& dd) : d(dd) {}
    void* get(size_t b) { void* p = d.mem.get(b); blocks.push_back(p); return p; }
    ~Scratch() { for (void* p : blocks) d.mem.put(p); }
};

// out = h(A) in, projections through d.Pa
void apply_h_plain(Domain& d, const void* in, void* out, const double* Ak) {
    const bool nl = d.has_nl();
    if (nl) launch_project(d, in, d.Pa);
    StageArgs a;
    a.w = in;
    a.psi = nullptr;
    a.out = out;
    a.P = nl ? d.Pa : nullptr;
    a.A = Ak;
    a.gamma_re = 1.0;
    a.gamma_im = 0.0;
    a.obs = nullptr;
    launch_stage(d, a);
}

// psi_out = T4(h(A)) psi_in in nested form (psi_out may equal psi_in; wa/wb
// are clobbered)
void taylor_step(Domain& d, const void* psi_in, void* psi_out, const double* Ak) {
    const double dt = d.desc.dt;
    const bool nl = d.has_nl();
    if (psi_out != psi_in)
        MLMD_CUDA(cudaMemcpyAsync(psi_out, psi_in, d.state_bytes, cudaMemcpyDeviceToDevice, d.stream));
    const void* in = psi_out;
    void* outs[4] = {d.wa, d.wb, d.wa, psi_out};
    void* Ps[4] = {d.Pa, d.Pb, d.Pa, d.Pb};
    for (int s = 0; s < 4; ++s) {
        if (nl) launch_project(d, in, Ps[s]);
        StageArgs a;
        a.w = in;
        a.psi = psi_out;
        a.out = outs[s];
        a.P = nl ? Ps[s] : nullptr;
        a.A = Ak;
        a.gamma_re = 0.0;
        a.gamma_im = -dt / (double)(4 - s);
        a.obs = nullptr;
        launch_stage(d, a);
        in = outs[s];
    }
}

}  // namespace
}  // namespace mlmd

using namespace mlmd;


extern "C" mlmd_status mlmd_propagate_adjoint(mlmd_domain_t dom, int32_t n_steps, const double* A, int32_t ckpt_every,
                                              double* loss, double* dL_dA, void* dL_dV, int32_t on_device) {
    Domain* d = dom;
    if (!d) return MLMD_ERR_INVALID;
    if (d->latched != MLMD_OK) return MLMD_ERR_STATE;
    try {
        MLMD_REQUIRE(n_steps >= 1 && A && loss && dL_dA, MLMD_ERR_INVALID, "bad adjoint arguments");
        MLMD_REQUIRE(ckpt_every >= 1, MLMD_ERR_INVALID, "ckpt_every must be >= 1");
        MLMD_REQUIRE(d->desc.scheme == MLMD_SCHEME_FULL && d->desc.ortho_every == 0, MLMD_ERR_UNSUPPORTED,
                     "adjoint needs the full scheme without re-orthonormalisation");
        MLMD_REQUIRE(d->psi0_valid, MLMD_ERR_STATE, "no reference orbitals (call mlmd_set_orbitals)");
        MLMD_REQUIRE(!gauge_on(*d), MLMD_ERR_UNSUPPORTED,
                     "adjoint of the velocity-gauge projectors (dh/dA has the nonlocal commutator)");
        for (int i = 0; i < 3 * n_steps; ++i) MLMD_REQUIRE(std::isfinite(A[i]), MLMD_ERR_INVALID, "A not finite");
        Scratch S(*d);
        d->pa_psi = false;
        const size_t sb = d->state_bytes;
        const int K = ckpt_every;
        const int nck = (n_steps + K - 1) / K;
        double* Ad = (double*)S.get(sizeof(double) * 3 * n_steps);
        MLMD_CUDA(cudaMemcpyAsync(Ad, A, sizeof(double) * 3 * n_steps, cudaMemcpyHostToDevice, d->stream));
        // checkpoints: ck[c] = psi at step c*K
        std::vector<void*> ck(nck);
        for (int c = 0; c < nck; ++c) ck[c] = S.get(sb);
        MLMD_CUDA(cudaMemcpyAsync(ck[0], d->psi, sb, cudaMemcpyDeviceToDevice, d->stream));
        for (int k = 0; k < n_steps; ++k) {
            taylor_step(*d, d->psi, d->psi, Ad + 3 * k);
            if ((k + 1) % K == 0 && (k + 1) / K < nck)
                MLMD_CUDA(cudaMemcpyAsync(ck[(k + 1) / K], d->psi, sb, cudaMemcpyDeviceToDevice, d->stream));
        }
        d->step += n_steps;
        // loss and lam_N
        const int no = d->desc.n_orb;
        const double dV = d->desc.h * d->desc.h * d->desc.h;
        double* C = (double*)S.get(sizeof(double) * 2 * no * no);
        launch_overlap(*d, d->psi0, d->psi, dV, C);
        std::vector<double> hC((size_t)2 * no * no);
        MLMD_CUDA(cudaMemcpyAsync(hC.data(), C, sizeof(double) * hC.size(), cudaMemcpyDeviceToHost, d->stream));
        MLMD_CUDA(cudaStreamSynchronize(d->stream));
        check_err_flag(*d);       // a forward stage that gave up a wait leaves psi(T) and the loss wrong
        double s2 = 0.0;
        for (double v : hC) s2 += v * v;
        *loss = 2.0 * ((double)no - s2);
        MLMD_REQUIRE(std::isfinite(*loss), MLMD_ERR_NUMERIC, "loss is NaN or Inf");
        for (double& v : hC) v *= -2.0 * dV;
        MLMD_CUDA(cudaMemcpyAsync(C, hC.data(), sizeof(double) * hC.size(), cudaMemcpyHostToDevice, d->stream));
        void* lam = S.get(sb);
        launch_update(*d, d->psi0, C, lam);

        // backward
        void* seg[1024];
        MLMD_REQUIRE(K <= 1024, MLMD_ERR_UNSUPPORTED, "ckpt_every must be <= 1024");
        for (int i = 0; i < K; ++i) seg[i] = S.get(sb);
        void* u[4];
        void* w[5];
        void* z[4];
        for (int i = 1; i < 4; ++i) u[i] = S.get(sb);
        w[0] = lam;
        for (int i = 1; i < 5; ++i) w[i] = S.get(sb);
        for (int i = 0; i < 4; ++i) z[i] = S.get(sb);
        double* gV = (double*)S.get(sizeof(double) * d->ng);
        MLMD_CUDA(cudaMemsetAsync(gV, 0, sizeof(double) * d->ng, d->stream));
        const int nblk = contract_blocks(*d);
        double* part = (double*)S.get(sizeof(double) * 4 * nblk);
        double* gA = (double*)S.get(sizeof(double) * 4 * n_steps);
        const double dt = d->desc.dt;
        std::complex<double> c[5];
        c[0] = 1.0;
        for (int j = 1; j < 5; ++j) c[j] = c[j - 1] * std::complex<double>(0.0, -dt) / (double)j;
        for (int c0 = nck - 1; c0 >= 0; --c0) {
            const int s0 = c0 * K, s1 = std::min(n_steps, s0 + K);
            MLMD_CUDA(cudaMemcpyAsync(seg[0], ck[c0], sb, cudaMemcpyDeviceToDevice, d->stream));
            for (int k = s0; k < s1 - 1; ++k) taylor_step(*d, seg[k - s0], seg[k - s0 + 1], Ad + 3 * k);
            for (int k = s1 - 1; k >= s0; --k) {
                const double* Ak = Ad + 3 * k;
                u[0] = seg[k - s0];
                for (int p = 1; p < 4; ++p) apply_h_plain(*d, u[p - 1], u[p], Ak);
                for (int q = 1; q < 5; ++q) apply_h_plain(*d, w[q - 1], w[q], Ak);
                for (int p = 0; p < 4; ++p) {
                    const void* in[5];
                    double cre[5], cim[5];
                    int n = 0;
                    for (int q = 0; q + p + 1 <= 4; ++q) {
                        in[n] = w[q];
                        const std::complex<double> cc = std::conj(c[q + p + 1]);
                        cre[n] = cc.real();
                        cim[n] = cc.imag();
                        ++n;
                    }
                    launch_lincomb(*d, n, in, cre, cim, z[p]);
                }
                launch_adjoint_contract(*d, (const void* const*)z, (const void* const*)u, part, nblk, gV);
                launch_reduce_partials(*d, part, nblk, 4, gA + 4 * k);
                // lam_k = sum_j conj(c_j) w_j (written over w_0 = lam)
                const void* in[5] = {w[0], w[1], w[2], w[3], w[4]};
                double cre[5], cim[5];
                for (int j = 0; j < 5; ++j) { cre[j] = std::conj(c[j]).real(); cim[j] = std::conj(c[j]).imag(); }
                launch_lincomb(*d, 5, in, cre, cim, w[0]);
            }
        }
        std::vector<double> hg((size_t)4 * n_steps);
        MLMD_CUDA(cudaMemcpyAsync(hg.data(), gA, sizeof(double) * hg.size(), cudaMemcpyDeviceToHost, d->stream));
        if (dL_dV)
            MLMD_CUDA(cudaMemcpyAsync(dL_dV, gV, sizeof(double) * d->ng,
                                      on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, d->stream));
        MLMD_CUDA(cudaStreamSynchronize(d->stream));
        MLMD_CUDA(cudaGetLastError());
        check_err_flag(*d);       // recompute and backward sweep launch the same bounded-wait kernels
        for (int k = 0; k < n_steps; ++k)
            for (int a = 0; a < 3; ++a) {
                dL_dA[3 * k + a] = hg[4 * k + a] + A[3 * k + a] * hg[4 * k + 3];
                MLMD_REQUIRE(std::isfinite(dL_dA[3 * k + a]), MLMD_ERR_NUMERIC, "gradient is NaN or Inf");
            }
        d->err.clear();
        return MLMD_OK;
    } catch (const Error& e) {
        d->err = e.msg;
        if (e.status == MLMD_ERR_CUDA || e.status == MLMD_ERR_NUMERIC || e.status == MLMD_ERR_TIMEOUT)
            d->latched = e.status;
        return e.status;
    } catch (...) {
        d->err = "unexpected failure";
        d->latched = MLMD_ERR_STATE;
        return MLMD_ERR_STATE;
    }
}
