/*
 * FP64 CPU oracle for the DC-MESH local-field-dynamics (LFD) step.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg use it.  It shares no code, header, table or
 * helper with the CUDA path.
 *
 * Plain, slow and literal on purpose: every routine is the textbook
 * definition written out in double precision, with no blocking or fusion.
 *
 *   Hamiltonian (Eq. 3, atomic units, velocity gauge, e/c absorbed into A):
 *     h = 1/2 (-i grad + A)^2 + v_loc(r) + v_nl
 *       = -1/2 lap - i A.grad + 1/2 |A|^2 + v_loc + sum_{a,i} |b_ai> D_ai <b_ai|
 *     with <b|psi> = dV sum_r b(r) psi(r) (b real).
 *   Velocity-gauge projectors (optional, nl_gauge = 1): for uniform A the
 *   minimal coupling of Eq. 3 is the unitary map h(A) = e^{-iA.r} h(0) e^{iA.r}
 *   of the kinetic term; carried onto v_nl it gives each projector the
 *   factor e^{-i A.(r - R_a)}, referred to the atom by the minimum image:
 *     v_nl(A) = sum_{a,i} |b~_ai> D_ai <b~_ai|,  b~_ai(r) = e^{-i A.(r - R_a)} b_ai(r),
 *   and the current J = dE/dA then has the nonlocal commutator part
 *     dE_nl/dA_x = sum_o f_o sum_ai D_ai 2 Re( i conj(P_aio) Q_aio^x ),
 *     P = <b~|psi>,  Q^x = <(r - R_a)_x b~|psi>
 *   (the nonlocal correction to energy and current of Sec. V.B.5, last
 *   paragraph).
 *   Periodic finite differences of order p (p = 2 or 4) for lap and grad.
 *   Time step: 4th-order Taylor expansion of exp(-i dt h(t_k)), A taken at
 *   the step midpoint t_k = (k + 1/2) dt as in Eq. 2.
 *   Split form (Eq. 2): N_nl T4(h_loc) N_nl with N_nl = (1 - i dt/2 v_nl)
 *   followed by a per-orbital rescale to the orbital's norm before N_nl.
 *
 * Layout (Sec. V.B.2): psi[g][o] complex (re, im interleaved), orbital index
 * fastest; grid index g = x + nx (y + ny z).
 *
 * Compile with -ffp-contract=off: the neighbour-list distance test must
 * round every product and sum separately.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double _Complex cplx;

typedef struct {
    int32_t n[3];
    double h;
    int32_t n_orb;
    int32_t fd_order;        /* 2 or 4 */
    const double* V;         /* [N_g] local potential */
    int32_t n_atoms;
    int32_t n_proj;          /* projectors per atom */
    const int64_t* off;      /* [n_atoms + 1] list offsets */
    const int32_t* idx;      /* [off[n_atoms]] grid indices */
    const double* beta;      /* [off[n_atoms]][n_proj] projector values */
    const double* D;         /* [n_atoms][n_proj] strengths */
    int32_t nl_gauge;        /* 1: velocity-gauge projectors b e^{-i A.(r - R_a)} */
    const double* pos;       /* [n_atoms][3] atom positions (read when nl_gauge) */
} orc_domain;

static int64_t n_grid(const orc_domain* d) { return (int64_t)d->n[0] * d->n[1] * d->n[2]; }

/* ---- finite-difference coefficients ----------------------------------
 * Second derivative (per axis, offsets 0, +-1, +-2, divided by h^2):
 *   p=2: [1, -2, 1]            p=4: [-1/12, 4/3, -5/2, 4/3, -1/12]
 * First derivative (central, offsets -2..2, divided by h):
 *   p=2: [-1/2, 0, 1/2]         p=4: [1/12, -2/3, 0, 2/3, -1/12]      */
static void fd_coeffs(int order, double lap[3], double grad[3]) {
    if (order == 2) {
        lap[0] = -2.0; lap[1] = 1.0; lap[2] = 0.0;
        grad[0] = 0.0; grad[1] = 0.5; grad[2] = 0.0;
    } else {
        lap[0] = -2.5; lap[1] = 4.0 / 3.0; lap[2] = -1.0 / 12.0;
        grad[0] = 0.0; grad[1] = 2.0 / 3.0; grad[2] = -1.0 / 12.0;
    }
}

static inline int64_t wrap(int64_t i, int64_t n) { i %= n; return i < 0 ? i + n : i; }

static inline int64_t lin(const orc_domain* d, int64_t x, int64_t y, int64_t z) {
    return wrap(x, d->n[0]) + (int64_t)d->n[0] * (wrap(y, d->n[1]) + (int64_t)d->n[1] * wrap(z, d->n[2]));
}

/* out = G_axis psi (periodic central difference) for every orbital. */
void orc_gradient(const orc_domain* d, int axis, const double* psi_in, double* out_) {
    const cplx* in = (const cplx*)psi_in;
    cplx* out = (cplx*)out_;
    double lap[3], grad[3];
    fd_coeffs(d->fd_order, lap, grad);
    const int no = d->n_orb;
    const double ih = 1.0 / d->h;
#pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < d->n[2]; ++z)
        for (int y = 0; y < d->n[1]; ++y)
            for (int x = 0; x < d->n[0]; ++x) {
                int64_t g = lin(d, x, y, z);
                for (int o = 0; o < no; ++o) {
                    cplx acc = 0.0;
                    for (int k = 1; k <= 2; ++k) {
                        int e[3] = {0, 0, 0};
                        e[axis] = k;
                        int64_t gp = lin(d, x + e[0], y + e[1], z + e[2]);
                        int64_t gm = lin(d, x - e[0], y - e[1], z - e[2]);
                        acc += grad[k] * (in[gp * no + o] - in[gm * no + o]);
                    }
                    out[g * no + o] = acc * ih;
                }
            }
}

/* out = h_loc(A) psi = -1/2 lap psi - i sum_a A_a G_a psi + (V + |A|^2/2) psi */
void orc_apply_hloc(const orc_domain* d, const double A[3], const double* psi_in, double* out_) {
    const cplx* in = (const cplx*)psi_in;
    cplx* out = (cplx*)out_;
    double lap[3], grad[3];
    fd_coeffs(d->fd_order, lap, grad);
    const int no = d->n_orb;
    const double ih2 = 1.0 / (d->h * d->h), ih = 1.0 / d->h;
    const double a2 = 0.5 * (A[0] * A[0] + A[1] * A[1] + A[2] * A[2]);
#pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < d->n[2]; ++z)
        for (int y = 0; y < d->n[1]; ++y)
            for (int x = 0; x < d->n[0]; ++x) {
                int64_t g = lin(d, x, y, z);
                for (int o = 0; o < no; ++o) {
                    cplx c = in[g * no + o];
                    cplx lp = 3.0 * lap[0] * c;
                    cplx ag = 0.0;
                    for (int ax = 0; ax < 3; ++ax) {
                        cplx gr = 0.0;
                        for (int k = 1; k <= 2; ++k) {
                            int e[3] = {0, 0, 0};
                            e[ax] = k;
                            cplx p = in[lin(d, x + e[0], y + e[1], z + e[2]) * no + o];
                            cplx m = in[lin(d, x - e[0], y - e[1], z - e[2]) * no + o];
                            lp += lap[k] * (p + m);
                            gr += grad[k] * (p - m);
                        }
                        ag += A[ax] * gr;
                    }
                    out[g * no + o] = -0.5 * ih2 * lp - I * ih * ag + (d->V[g] + a2) * c;
                }
            }
}

/* Minimum-image displacement r_g - R_a of grid point g from atom a, with
 * the wrap of the neighbour lists. */
static void entry_delta(const orc_domain* d, int a, int32_t g, double dl[3]) {
    const int coord[3] = {g % d->n[0], (g / d->n[0]) % d->n[1], g / (d->n[0] * d->n[1])};
    for (int ax = 0; ax < 3; ++ax) {
        const double L = (double)d->n[ax] * d->h;
        const double t = (double)coord[ax] * d->h - d->pos[3 * a + ax];
        dl[ax] = t - L * floor(t / L + 0.5);
    }
}

/* Gauge factor of projector a at grid point g: e^{-i A.(r_g - R_a)} in the
 * velocity gauge, 1 for real projectors (or A == NULL). */
static cplx gauge_factor(const orc_domain* d, const double* A, int a, int32_t g) {
    if (!d->nl_gauge || !A) return 1.0;
    double dl[3];
    entry_delta(d, a, g, dl);
    const double th = A[0] * dl[0] + A[1] * dl[1] + A[2] * dl[2];
    return cos(th) - I * sin(th);
}

/* proj[a][i][o] = <b~_ai|w_o psi_o> = dV sum_r conj(b~_ai(r)) w(r) psi_o(r)
 * (Eq. 5 form: one projection GEMM per atom), w = 1, or the displacement
 * component (r - R_a)_axis when axis >= 0.  proj: complex [n_atoms][n_proj][n_orb]. */
static void project_impl(const orc_domain* d, const double* A, int axis, const double* psi_in, double* proj_) {
    const cplx* in = (const cplx*)psi_in;
    cplx* proj = (cplx*)proj_;
    const int no = d->n_orb, np = d->n_proj;
    const double dV = d->h * d->h * d->h;
#pragma omp parallel for schedule(dynamic)
    for (int a = 0; a < d->n_atoms; ++a) {
        for (int i = 0; i < np; ++i)
            for (int o = 0; o < no; ++o) proj[((int64_t)a * np + i) * no + o] = 0.0;
        for (int64_t q = d->off[a]; q < d->off[a + 1]; ++q) {
            const cplx* row = in + (int64_t)d->idx[q] * no;
            cplx wq = conj(gauge_factor(d, A, a, d->idx[q]));
            if (axis >= 0) {
                double dl[3];
                entry_delta(d, a, d->idx[q], dl);
                wq *= dl[axis];
            }
            for (int i = 0; i < np; ++i) {
                double b = d->beta[q * np + i];
                cplx* pr = proj + ((int64_t)a * np + i) * no;
                for (int o = 0; o < no; ++o) pr[o] += b * wq * row[o];
            }
        }
        for (int i = 0; i < np; ++i)
            for (int o = 0; o < no; ++o) proj[((int64_t)a * np + i) * no + o] *= dV;
    }
}

/* proj = <b~|psi> at field A (A may be NULL for real projectors). */
void orc_project(const orc_domain* d, const double* A, const double* psi_in, double* proj_) {
    project_impl(d, A, -1, psi_in, proj_);
}

/* proj = <(r - R_a)_axis b~|psi>: the moment projection of the nonlocal current. */
void orc_project_moment(const orc_domain* d, const double* A, int axis, const double* psi_in, double* proj_) {
    project_impl(d, A, axis, psi_in, proj_);
}

/* out += sum_{a,i} b~_ai D_ai proj[a][i]   (scatter-back GEMM). */
void orc_scatter(const orc_domain* d, const double* A, const double* proj_, double* out_) {
    const cplx* proj = (const cplx*)proj_;
    cplx* out = (cplx*)out_;
    const int no = d->n_orb, np = d->n_proj;
    /* parallel over orbitals so that overlapping spheres never race */
#pragma omp parallel for schedule(static)
    for (int o = 0; o < no; ++o)
        for (int a = 0; a < d->n_atoms; ++a)
            for (int64_t q = d->off[a]; q < d->off[a + 1]; ++q) {
                cplx acc = 0.0;
                for (int i = 0; i < np; ++i)
                    acc += d->beta[q * np + i] * d->D[(int64_t)a * np + i] * proj[((int64_t)a * np + i) * no + o];
                out[(int64_t)d->idx[q] * no + o] += gauge_factor(d, A, a, d->idx[q]) * acc;
            }
}

/* out = v_nl(A) psi */
void orc_apply_vnl(const orc_domain* d, const double* A, const double* psi_in, double* out_, double* work_proj) {
    memset(out_, 0, sizeof(cplx) * (size_t)n_grid(d) * d->n_orb);
    if (d->n_atoms == 0 || d->n_proj == 0) return;
    orc_project(d, A, psi_in, work_proj);
    orc_scatter(d, A, work_proj, out_);
}

/* out = h(A) psi (local + nonlocal), Eq. 3.  work_proj: [n_atoms*n_proj*n_orb] complex. */
void orc_apply_h(const orc_domain* d, const double A[3], const double* psi_in, double* out_, double* work_proj) {
    orc_apply_hloc(d, A, psi_in, out_);
    if (d->n_atoms == 0 || d->n_proj == 0) return;
    orc_project(d, A, psi_in, work_proj);
    orc_scatter(d, A, work_proj, out_);
}

/* psi_out = sum_{j=0..4} (-i dt)^j / j! h^j psi_in, with u_j = h u_{j-1}
 * evaluated term by term (not in nested form).  local_only != 0 drops v_nl.
 * work: 2 * N_g * n_orb complex; work_proj as above.  psi_out may alias psi_in. */
void orc_taylor4(const orc_domain* d, const double A[3], double dt, int local_only,
                 const double* psi_in, double* psi_out, double* work, double* work_proj) {
    const int64_t N = n_grid(d) * d->n_orb;
    cplx* u = (cplx*)work;
    cplx* v = u + N;
    cplx* acc = (cplx*)psi_out;
    memcpy(u, psi_in, sizeof(cplx) * (size_t)N);
    if (psi_out != psi_in) memcpy(acc, psi_in, sizeof(cplx) * (size_t)N);
    cplx c = 1.0;
    for (int j = 1; j <= 4; ++j) {
        if (local_only) orc_apply_hloc(d, A, (const double*)u, (double*)v);
        else orc_apply_h(d, A, (const double*)u, (double*)v, work_proj);
        c *= (-I * dt) / (double)j;
#pragma omp parallel for schedule(static)
        for (int64_t t = 0; t < N; ++t) acc[t] += c * v[t];
        cplx* tmp = u; u = v; v = tmp;
    }
}

/* psi_out = sum_{j=0..4} (+i dt)^j / j! h^j lam_in: the Hermitian adjoint of
 * the Taylor map (h is Hermitian in the Euclidean inner product). */
void orc_taylor4_adjoint(const orc_domain* d, const double A[3], double dt,
                         const double* lam_in, double* lam_out, double* work, double* work_proj) {
    const int64_t N = n_grid(d) * d->n_orb;
    cplx* u = (cplx*)work;
    cplx* v = u + N;
    cplx* acc = (cplx*)lam_out;
    memcpy(u, lam_in, sizeof(cplx) * (size_t)N);
    if (lam_out != lam_in) memcpy(acc, lam_in, sizeof(cplx) * (size_t)N);
    cplx c = 1.0;
    for (int j = 1; j <= 4; ++j) {
        orc_apply_h(d, A, (const double*)u, (double*)v, work_proj);
        c *= (I * dt) / (double)j;
#pragma omp parallel for schedule(static)
        for (int64_t t = 0; t < N; ++t) acc[t] += c * v[t];
        cplx* tmp = u; u = v; v = tmp;
    }
}

/* Per-orbital squared norms nrm[o] = <psi_o|psi_o>. */
void orc_orbital_norms(const orc_domain* d, const double* psi_in, double* nrm) {
    const cplx* in = (const cplx*)psi_in;
    const int no = d->n_orb;
    const int64_t ng = n_grid(d);
    const double dV = d->h * d->h * d->h;
    for (int o = 0; o < no; ++o) {
        double s = 0.0;
        for (int64_t g = 0; g < ng; ++g) { cplx c = in[g * no + o]; s += creal(c) * creal(c) + cimag(c) * cimag(c); }
        nrm[o] = dV * s;
    }
}

/* N_nl psi = (1 - i dt/2 v_nl(A)) psi, then each orbital rescaled to the norm
 * it had before the factor (the normalising denominator of Eq. 2). */
static void apply_nnl(const orc_domain* d, const double A[3], double dt, cplx* psi, cplx* tmp, double* work_proj,
                      double* nrm_before, double* nrm_after) {
    const int no = d->n_orb;
    const int64_t ng = n_grid(d);
    orc_orbital_norms(d, (const double*)psi, nrm_before);
    orc_apply_vnl(d, A, (const double*)psi, (double*)tmp, work_proj);
    for (int64_t t = 0; t < ng * no; ++t) psi[t] += (-0.5 * I * dt) * tmp[t];
    orc_orbital_norms(d, (const double*)psi, nrm_after);
    for (int64_t g = 0; g < ng; ++g)
        for (int o = 0; o < no; ++o)
            psi[g * no + o] *= (nrm_after[o] > 0.0) ? sqrt(nrm_before[o] / nrm_after[o]) : 1.0;
}

/* One split step of Eq. 2: N_nl T4(h_loc) N_nl.  work: 2*N_g*n_orb complex. */
void orc_split_step(const orc_domain* d, const double A[3], double dt, const double* psi_in,
                    double* psi_out, double* work, double* work_proj, double* nrm_before, double* nrm_after) {
    const int64_t N = n_grid(d) * d->n_orb;
    cplx* out = (cplx*)psi_out;
    const int has_nl = d->n_atoms > 0 && d->n_proj > 0;
    if (psi_out != psi_in) memcpy(out, psi_in, sizeof(cplx) * (size_t)N);
    if (has_nl) apply_nnl(d, A, dt, out, (cplx*)work, work_proj, nrm_before, nrm_after);
    orc_taylor4(d, A, dt, 1, (const double*)out, (double*)out, work, work_proj);
    if (has_nl) apply_nnl(d, A, dt, out, (cplx*)work, work_proj, nrm_before, nrm_after);
}

/* Observables of psi under h(A):
 *   obs[0] = sum_o f_o <psi_o|psi_o>                 (electron count)
 *   obs[1] = sum_o f_o Re <psi_o| h |psi_o>            (energy)
 *   obs[2+a] = sum_o f_o Re <psi_o| -i G_a + A_a |psi_o>  (current J = dE/dA)
 *              + the nonlocal commutator part with velocity-gauge projectors
 * work: N_g*n_orb complex. */
void orc_observables(const orc_domain* d, const double A[3], const double* f, const double* psi_in,
                     double* obs, double* work, double* work_proj) {
    const cplx* in = (const cplx*)psi_in;
    const cplx* hp = (const cplx*)work;   /* h psi, later G_a psi */
    const int no = d->n_orb;
    const int64_t ng = n_grid(d);
    const double dV = d->h * d->h * d->h;
    double nrm = 0.0, e = 0.0;
    orc_apply_h(d, A, psi_in, work, work_proj);
    for (int64_t g = 0; g < ng; ++g)
        for (int o = 0; o < no; ++o) {
            cplx c = in[g * no + o];
            nrm += f[o] * creal(conj(c) * c);
            e += f[o] * creal(conj(c) * hp[g * no + o]);
        }
    obs[0] = dV * nrm;
    obs[1] = dV * e;
    for (int ax = 0; ax < 3; ++ax) {
        orc_gradient(d, ax, psi_in, work);
        const cplx* gp = (const cplx*)work;
        double s = 0.0;
        for (int64_t g = 0; g < ng; ++g)
            for (int o = 0; o < no; ++o) {
                cplx c = in[g * no + o];
                s += f[o] * creal(conj(c) * (-I * gp[g * no + o] + A[ax] * c));
            }
        obs[2 + ax] = dV * s;
    }
    if (d->nl_gauge && d->n_atoms > 0 && d->n_proj > 0) {
        /* dv_nl/dA_x = -i [(r - R)_x, v_nl(A)], so
         * <psi|dv_nl/dA_x|psi> = sum_ai D_ai 2 Re(i conj(P_ai) Q^x_ai) */
        const int64_t np = (int64_t)d->n_atoms * d->n_proj;
        cplx* P = (cplx*)work_proj;
        cplx* Q = (cplx*)malloc(sizeof(cplx) * (size_t)np * no);
        if (!Q) abort();
        orc_project(d, A, psi_in, (double*)P);
        for (int ax = 0; ax < 3; ++ax) {
            orc_project_moment(d, A, ax, psi_in, (double*)Q);
            double s = 0.0;
            for (int64_t r = 0; r < np; ++r)
                for (int o = 0; o < no; ++o)
                    s += f[o] * d->D[r] * 2.0 * creal(I * conj(P[r * no + o]) * Q[r * no + o]);
            obs[2 + ax] += s;
        }
        free(Q);
    }
}

/* rho(r) = sum_o f_o |psi_o(r)|^2 ;  j_a(r) = sum_o f_o Im(conj(psi_o) G_a psi_o)(r) + A_a rho(r);
 * J_a = dV sum_r j_a(r).  j: [3][N_g].  work: N_g*n_orb complex. */
void orc_density_current(const orc_domain* d, const double A[3], const double* f, const double* psi_in,
                         double* rho, double* jcur, double* Jtot, double* work) {
    const cplx* in = (const cplx*)psi_in;
    const cplx* gp = (const cplx*)work;
    const int no = d->n_orb;
    const int64_t ng = n_grid(d);
    const double dV = d->h * d->h * d->h;
    for (int64_t g = 0; g < ng; ++g) {
        double s = 0.0;
        for (int o = 0; o < no; ++o) { cplx c = in[g * no + o]; s += f[o] * creal(conj(c) * c); }
        rho[g] = s;
    }
    for (int ax = 0; ax < 3; ++ax) {
        orc_gradient(d, ax, psi_in, work);
        double tot = 0.0;
        for (int64_t g = 0; g < ng; ++g) {
            double s = 0.0;
            for (int o = 0; o < no; ++o) s += f[o] * cimag(conj(in[g * no + o]) * gp[g * no + o]);
            jcur[ax * ng + g] = s + A[ax] * rho[g];
            tot += jcur[ax * ng + g];
        }
        Jtot[ax] = dV * tot;
    }
}

/* S[n][m] = dV sum_r conj(a_n(r)) b_m(r)   (overlap / Gram matrix, Eq. 5's
 * Psi^dagger(0) Psi(t)).  a: [N_g][na], b: [N_g][nb], S: [na][nb] complex. */
void orc_overlap(int64_t ng, int na, int nb, double dV, const double* a_, const double* b_, double* S_) {
    const cplx* a = (const cplx*)a_;
    const cplx* b = (const cplx*)b_;
    cplx* S = (cplx*)S_;
#pragma omp parallel for schedule(dynamic)
    for (int n = 0; n < na; ++n)
        for (int m = 0; m < nb; ++m) {
            cplx s = 0.0;
            for (int64_t g = 0; g < ng; ++g) s += conj(a[g * na + n]) * b[g * nb + m];
            S[(int64_t)n * nb + m] = dV * s;
        }
}

/* Neighbour lists of the projector spheres: every grid point r_i = i*h with
 * minimum-image distance d <= r_cut from the atom, by brute force over the
 * whole grid in ascending linear order.  The wrap is
 * delta -= L * floor(delta / L + 1/2), so an exact tie lands on -L/2.
 * If idx is NULL only counts[a] are written; otherwise idx receives each
 * atom's list, atoms concatenated in order (caller sized it from counts). */
void orc_neighbor_lists(const int32_t n[3], double h, int32_t n_atoms, const double* pos,
                        double r_cut, int64_t* counts, int32_t* idx) {
    const double L[3] = {(double)n[0] * h, (double)n[1] * h, (double)n[2] * h};
    const double rc2 = r_cut * r_cut;
    int64_t w = 0;
    for (int a = 0; a < n_atoms; ++a) {
        int64_t c = 0;
        for (int z = 0; z < n[2]; ++z)
            for (int y = 0; y < n[1]; ++y)
                for (int x = 0; x < n[0]; ++x) {
                    const int coord[3] = {x, y, z};
                    double dl[3];
                    for (int ax = 0; ax < 3; ++ax) {
                        double t = (double)coord[ax] * h - pos[3 * a + ax];
                        double k = floor(t / L[ax] + 0.5);
                        double s = L[ax] * k;
                        dl[ax] = t - s;
                    }
                    double xx = dl[0] * dl[0];
                    double yy = dl[1] * dl[1];
                    double zz = dl[2] * dl[2];
                    double d2 = xx + yy;
                    d2 = d2 + zz;
                    if (d2 <= rc2) {
                        if (idx) idx[w++] = (int32_t)(x + n[0] * (y + n[1] * z));
                        ++c;
                    }
                }
        counts[a] = c;
    }
}

/* Projector values on the lists.  For shape 4: s, p_x, p_y, p_z with
 *   s(r) = exp(-d^2 / (2 rc^2)),  p_a(r) = (delta_a / rc) s(r);
 * shape 8 appends the same four with rc / sqrt(2).  Each projector is then
 * scaled so that dV sum_r b(r)^2 = 1 over its truncated support (left at zero
 * if that sum vanishes).  beta: [sum counts][n_proj]. */
void orc_projector_values(const int32_t n[3], double h, int32_t n_atoms, const double* pos,
                          const int64_t* off, const int32_t* idx, int32_t n_proj, double r_c, double* beta) {
    const double L[3] = {(double)n[0] * h, (double)n[1] * h, (double)n[2] * h};
    const double dV = h * h * h;
    for (int a = 0; a < n_atoms; ++a) {
        for (int64_t q = off[a]; q < off[a + 1]; ++q) {
            int32_t g = idx[q];
            int coord[3] = {g % n[0], (g / n[0]) % n[1], g / (n[0] * n[1])};
            double dl[3];
            for (int ax = 0; ax < 3; ++ax) {
                double t = (double)coord[ax] * h - pos[3 * a + ax];
                dl[ax] = t - L[ax] * floor(t / L[ax] + 0.5);
            }
            double d2 = dl[0] * dl[0] + dl[1] * dl[1] + dl[2] * dl[2];
            for (int set = 0; set < n_proj / 4; ++set) {
                double rc = set == 0 ? r_c : r_c / sqrt(2.0);
                double s = exp(-d2 / (2.0 * rc * rc));
                beta[q * n_proj + 4 * set + 0] = s;
                for (int ax = 0; ax < 3; ++ax) beta[q * n_proj + 4 * set + 1 + ax] = dl[ax] / rc * s;
            }
        }
        for (int i = 0; i < n_proj; ++i) {
            double s = 0.0;
            for (int64_t q = off[a]; q < off[a + 1]; ++q) s += beta[q * n_proj + i] * beta[q * n_proj + i];
            s *= dV;
            double scale = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
            for (int64_t q = off[a]; q < off[a + 1]; ++q) beta[q * n_proj + i] *= scale;
        }
    }
}

int orc_abi_version(void) { return 2; }
