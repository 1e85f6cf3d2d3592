/*
 * mlmd.h -- C ABI of the GB300 local-field-dynamics (LFD) propagator.
 *
 * The library propagates many Kohn-Sham orbitals of one divide-and-conquer
 * domain on a periodic real-space grid (the LFD part of DC-MESH, Sec. V.A.3-5
 * of the paper).  Each time step applies the 4th-order Taylor expansion of
 * exp(-i dt h(t_k)) with the Hamiltonian of Eq. 3 in atomic units,
 *
 *   h = 1/2 (-i grad + A(t))^2 + v_loc(r) + sum_{a,i} |b_ai> D_ai <b_ai|,
 *
 * finite-difference Laplacian and gradient of order 2 or 4 on the periodic
 * grid, A(t) taken at the step midpoint t_k = (k + 1/2) dt as in Eq. 2, and
 * the nonlocal term applied as a projection GEMM followed by a scatter-back
 * GEMM (Sec. V.B.5).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Grid: n[0] x n[1] x n[2] points, spacing h (bohr), point r = (x, y, z) h,
 *   linear index g = x + n[0] (y + n[1] z).  dV = h^3.
 * - Orbitals: a [N_g][N_o] complex array, orbital index fastest (the
 *   structure-of-arrays layout of Sec. V.B.2), real and imaginary parts
 *   interleaved.  Precision MLMD_C128 uses double pairs, MLMD_C64 float pairs.
 * - Inner product <a|b> = dV sum_r conj(a(r)) b(r).
 * - Host pointers are plain CPU memory (pinned or not); "on_device" pointers
 *   are device memory of the domain's current device.  The caller owns every
 *   buffer it passes; the library copies what it keeps.
 * - Calls are ordered on the domain's CUDA stream.  Host outputs are valid
 *   on return (the call synchronises that stream); device outputs are valid
 *   in stream order.
 * - A handle is not thread-safe; distinct handles are independent.
 * - No C++ exception crosses this interface.  Every call returns an
 *   mlmd_status; after a CUDA or numeric failure the handle latches
 *   MLMD_ERR_STATE for every later call except destroy and last_error.
 */
#ifndef MLMD_H
#define MLMD_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define MLMD_API __attribute__((visibility("default")))
#else
#define MLMD_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mlmd_domain* mlmd_domain_t;
typedef struct mlmd_batch* mlmd_batch_t;

typedef enum {
    MLMD_OK = 0,
    MLMD_ERR_INVALID = 1,      /* bad argument, size or descriptor field   */
    MLMD_ERR_OOM = 2,          /* device allocation failed                 */
    MLMD_ERR_CUDA = 3,         /* a CUDA runtime call or launch failed     */
    MLMD_ERR_NUMERIC = 4,      /* NaN/Inf or blow-up in a norm/energy      */
    MLMD_ERR_TIMEOUT = 5,      /* a bounded device-side wait gave up       */
    MLMD_ERR_STATE = 6,        /* call out of order, or handle latched     */
    MLMD_ERR_UNSUPPORTED = 7   /* valid request this build does not serve */
} mlmd_status;

enum { MLMD_C128 = 0, MLMD_C64 = 1 };

/* Arithmetic of the orbital-space GEMMs of MLMD_C64 domains (Sec. V.B.7,
 * Sec. VI.C): the overlap Psi^H Psi or Psi(0)^H Psi (re-orthonormalisation,
 * mlmd_overlap, mlmd_excitation, mlmd_occupations, Eq. 5) and the orbital
 * updates Psi M (re-orthonormalisation, Eq. 5).  The split modes run on the
 * tensor cores:
 *   FP32    plain FP32 products and sums (SIMT);
 *   BF16    each FP32 operand rounded to one bf16, FP32 accumulation;
 *   BF16X2  operand = two bf16 parts, 3 cross products, FP32 accumulation;
 *   BF16X3  operand = three bf16 parts, 6 cross products, FP32 accumulation;
 *   FP16    each operand rounded to fp16 after one power-of-two scale that
 *           brings a normalised orbital's entries to O(1).
 * The atom-projector products inside the time step (Eq. 3's nonlocal term)
 * are FP32 in every mode.  MLMD_C128 domains always use FP64. */
enum { MLMD_GEMM_FP32 = 0, MLMD_GEMM_BF16 = 1, MLMD_GEMM_BF16X2 = 2, MLMD_GEMM_BF16X3 = 3, MLMD_GEMM_FP16 = 4 };

/* FULL: Taylor-4 of the whole h (v_nl inside the expansion).
 * SPLIT: Eq. 2, N_nl T4(h_loc) N_nl with N_nl = (1 - i dt/2 v_nl) followed
 *        by a per-orbital rescale to the orbital's norm before the factor. */
enum { MLMD_SCHEME_FULL = 0, MLMD_SCHEME_SPLIT = 1 };

enum { MLMD_ORTHO_CHOL = 0, MLMD_ORTHO_LOWDIN = 1 };

/* Optional device allocator (e.g. a framework's caching allocator).  alloc
 * returns device memory of at least `bytes`, 256-byte aligned, or NULL;
 * free releases it.  Both are called only from create/set_* /destroy and the
 * first propagate call, on the caller's thread, with the domain's stream. */
typedef struct {
    void* (*alloc)(size_t bytes, void* stream, void* ctx);
    void (*free)(void* ptr, size_t bytes, void* stream, void* ctx);
    void* ctx;
} mlmd_allocator;

typedef struct {
    int32_t n[3];          /* grid points per axis, each in [4, 4096]       */
    double h;              /* grid spacing, bohr, > 0                       */
    int32_t n_orb;         /* orbitals, >= 1                                */
    int32_t fd_order;      /* 2 or 4                                         */
    int32_t precision;     /* MLMD_C128 or MLMD_C64                          */
    int32_t gemm_mode;     /* MLMD_GEMM_*                                    */
    int32_t scheme;        /* MLMD_SCHEME_*                                  */
    double dt;             /* time step, a.u., > 0                           */
    int32_t ortho_every;   /* re-orthonormalise after every k-th step; 0 off */
    int32_t ortho_kind;    /* MLMD_ORTHO_*                                   */
} mlmd_domain_desc;

/* Version of this interface (bumped on any signature change). */
MLMD_API int32_t mlmd_abi_version(void);

/* Create a domain on the current CUDA device.  allocator may be NULL (then
 * device memory comes stream-ordered from a memory pool the library keeps per
 * device, which holds freed blocks for reuse and is trimmed whenever a domain
 * is destroyed); stream may be NULL (the legacy default stream).  Orbitals start at zero, occupations at 2, v_loc at 0, and no
 * projectors.  Returns MLMD_ERR_INVALID for a bad descriptor, MLMD_ERR_OOM
 * when device memory runs out. */
MLMD_API mlmd_status mlmd_domain_create(const mlmd_domain_desc* desc, const mlmd_allocator* allocator,
                               void* stream, mlmd_domain_t* out);

/* Release every device buffer of the domain (stream-ordered) and the handle. */
MLMD_API mlmd_status mlmd_domain_destroy(mlmd_domain_t dom);

/* Copy orbitals in: psi is [N_g][N_o] interleaved complex in the domain's
 * precision, host or device memory.  The copy also becomes the reference
 * Psi(0) of mlmd_excitation and mlmd_propagate_adjoint, and resets the
 * domain's step counter to 0. */
MLMD_API mlmd_status mlmd_set_orbitals(mlmd_domain_t dom, const void* psi, int32_t on_device);

/* Copy the current orbitals out, same layout as mlmd_set_orbitals. */
MLMD_API mlmd_status mlmd_get_orbitals(mlmd_domain_t dom, void* psi_out, int32_t on_device);

/* Occupations f_n, host double [N_o], each finite. */
MLMD_API mlmd_status mlmd_set_occupations(mlmd_domain_t dom, const double* f);

/* Local potential v_loc(r), host double [N_g], each finite (Ha). */
MLMD_API mlmd_status mlmd_set_potential(mlmd_domain_t dom, const double* v);

/* Nonlocal projectors (Sec. V.A.2's nonlocal pseudopotential, Sec. V.B.5).
 * pos: host double [n_atoms][3] (bohr, any real value; wrapped periodically).
 * n_proj_per_atom: 4 (s, p_x, p_y, p_z) or 8 (the same four at r_c and at
 * r_c/sqrt(2)).  Projector shapes: s(r) = exp(-d^2/(2 rc^2)),
 * p_a(r) = (delta_a/rc) s(r), each truncated at d <= r_cut and normalised
 * to dV sum b^2 = 1 over its grid support.  Membership uses the minimum
 * image delta -= L floor(delta/L + 1/2) and d^2 = dx*dx + dy*dy + dz*dz
 * rounded after every operation (no fused multiply-add).  D: host double
 * [n_atoms][n_proj_per_atom] (Ha).  n_atoms = 0 removes the projectors.
 * The lists and values are built on the device. */
MLMD_API mlmd_status mlmd_set_projectors(mlmd_domain_t dom, int32_t n_atoms, const double* pos,
                                int32_t n_proj_per_atom, double r_c, double r_cut, const double* D);

/* Read back the projector index maps built by mlmd_set_projectors: off is
 * host int64 [n_atoms + 1] (list offsets), idx host int32 [off[n_atoms]]
 * (grid indices, ascending within each atom), beta (may be NULL) host double
 * [off[n_atoms]][n_proj].  Pass idx = NULL to read only off.  idx_cap is the
 * capacity of idx in elements; MLMD_ERR_INVALID if it is too small. */
MLMD_API mlmd_status mlmd_get_projector_lists(mlmd_domain_t dom, int64_t* off, int32_t* idx, size_t idx_cap,
                                     double* beta);

/* Gauge of the nonlocal projectors (Eq. 3 with Sec. V.B.5's nonlocal
 * energy and current).  MLMD_NL_GAUGE_REAL (the default): v_nl = sum
 * |b_ai> D_ai <b_ai| with the real projectors of mlmd_set_projectors,
 * independent of A.  MLMD_NL_GAUGE_VELOCITY: the minimal coupling of Eq. 3
 * carried onto v_nl -- for uniform A, h(A) = e^{-iA.r} h(0) e^{iA.r}, so
 * each projector becomes b~_ai(r) = e^{-i A.(r - R_a)} b_ai(r), with r - R_a
 * the minimum-image displacement of the projector lists, re-evaluated at
 * every step's A.  Then dh/dA_x gains the commutator -i[(r - R)_x, v_nl],
 * and the current column of mlmd_propagate's observables (J = dE/dA) adds
 *   sum_n f_n sum_ai D_ai 2 Re(i conj(<b~_ai|psi_n>) <(r - R_a)_x b~_ai|psi_n>),
 * computed from three moment projections of the orbitals.  The
 * velocity-gauge form runs on the per-point projection and scatter kernels
 * (the TMA-staged and tensor-core nonlocal forms keep real projector tables
 * and are not used while it is on).  mlmd_density_current's fields and J
 * stay the local current density and its integral (the commutator term has
 * no local density).  mlmd_propagate_adjoint returns MLMD_ERR_UNSUPPORTED
 * for a domain with projectors in the velocity gauge.  May be called at any
 * time; the setting survives mlmd_set_projectors.  MLMD_ERR_INVALID for an
 * unknown gauge. */
enum { MLMD_NL_GAUGE_REAL = 0, MLMD_NL_GAUGE_VELOCITY = 1 };
MLMD_API mlmd_status mlmd_set_nonlocal_gauge(mlmd_domain_t dom, int32_t gauge);

/* Propagate n_steps >= 0 Taylor-4 steps.  A: host double [n_steps][3], the
 * vector potential at each step's midpoint.  obs_out: NULL or host double
 * [n_steps][5]; row k holds, for the state before step k under h(A_k):
 *   [0] sum_n f_n <psi_n|psi_n>          (electron count)
 *   [1] sum_n f_n Re <psi_n|h|psi_n>      (energy, Ha)
 *   [2..4] J_a = sum_n f_n Re <psi_n|-i d_a + A_a|psi_n> = dE/dA_a.
 * The excited-electron count n_exc is not a sixth column by design: it needs
 * the N_o x N_o overlap with Psi(0), a GEMM of N_g N_o^2 work (at 1024
 * orbitals ten times a Taylor step's stencil work), which a per-step row
 * would add to every step; mlmd_excitation / mlmd_occupations compute it
 * when the caller asks (Sec. V.A.8 hands n_exc over once per MD step).
 * If desc.ortho_every > 0 the orbitals are re-orthonormalised after every
 * step whose count since set_orbitals is a multiple of it.
 * MLMD_ERR_NUMERIC if an observable comes out NaN or Inf. */
MLMD_API mlmd_status mlmd_propagate(mlmd_domain_t dom, int32_t n_steps, const double* A, double* obs_out);

/* Density and current of the current orbitals under A (host double [3]):
 * rho(r) = sum_n f_n |psi_n(r)|^2, j_a(r) = sum_n f_n Im(conj(psi_n) d_a psi_n)(r)
 * + A_a rho(r), and J_a = dV sum_r j_a(r).  rho: [N_g], j: [3][N_g], both in
 * the domain's real type (double for C128, float for C64), host or device;
 * either may be NULL.  J: host double [3] or NULL. */
MLMD_API mlmd_status mlmd_density_current(mlmd_domain_t dom, const double* A, void* rho, void* j, double* J,
                                 int32_t on_device);

/* Overlap S = dV Psi^dagger Psi of the current orbitals, host complex double
 * [N_o][N_o] (S[n][m] = <psi_n|psi_m>), computed with the Gram GEMM in the
 * domain's gemm_mode. */
MLMD_API mlmd_status mlmd_overlap(mlmd_domain_t dom, double* S_out);

/* Re-orthonormalise the current orbitals now: Cholesky S = L L^H and
 * Psi <- Psi L^{-H} (Gram-Schmidt order), or Loewdin Psi <- Psi S^{-1/2}.
 * The factorisation runs in FP64 on the device. */
MLMD_API mlmd_status mlmd_reorthonormalize(mlmd_domain_t dom, int32_t kind);

/* Excited-electron count of the current orbitals against the reference
 * Psi(0) from mlmd_set_orbitals: n_exc = 2 (N_o - sum_{n,m} |<psi_n(0)|psi_m>|^2)
 * (the per-domain n_exc of Sec. V.A.8). */
MLMD_API mlmd_status mlmd_excitation(mlmd_domain_t dom, double* n_exc);

/* Shadow-dynamics occupations (Sec. V.A.3-4: LFD hands the occupation
 * numbers of the Kohn-Sham states back to QXMD; Sec. V.A.8: n_exc per domain
 * is computed from them).  The reference orbitals psi_s(0) from
 * mlmd_set_orbitals are the adiabatic states; the current orbitals psi_n(t)
 * carry the occupations f_n of mlmd_set_occupations.  f_out: host double
 * [N_o], f_s(t) = sum_n f_n |<psi_s(0)|psi_n(t)>|^2 (may be NULL).  n_exc:
 * host double, sum_n f_n - sum_s f_s(t), the electrons that have left the
 * span of the reference orbitals (may be NULL; with every f_n = 2 it equals
 * mlmd_excitation).  The overlap runs as a GEMM in the domain's gemm_mode;
 * the sums run on the device in FP64 in a fixed order.  MLMD_ERR_INVALID if
 * both outputs are NULL, MLMD_ERR_STATE without reference orbitals. */
MLMD_API mlmd_status mlmd_occupations(mlmd_domain_t dom, double* f_out, double* n_exc);

/* KS-space nonlocal correction of Eq. 5 (Sec. V.B.5) applied once to the
 * current orbitals: Psi(t) <- Psi(t) - delta Psi(0) C with C = dV Psi(0)^H
 * Psi(t), the overlap with the reference orbitals from mlmd_set_orbitals in
 * the grid's inner product (so delta is dimensionless).  delta: host double
 * [2] = (Re, Im).  Both products run as GEMMs in the domain's gemm_mode
 * (tcgen05 split operands for complex64 and non-FP32 modes).  Returns
 * MLMD_ERR_STATE without reference orbitals, MLMD_ERR_INVALID for a null or
 * non-finite delta. */
MLMD_API mlmd_status mlmd_ks_correction(mlmd_domain_t dom, const double* delta);

/* Gradients of L = n_exc(Psi(T)) after n_steps full-scheme steps from the
 * current orbitals, by the discrete adjoint of the Taylor map.  The forward
 * pass keeps every ckpt_every-th state and recomputes the others inside each
 * segment.  loss: host double.  dL_dA: host double [n_steps][3].  dL_dV: the
 * gradient with respect to each grid value v_loc(r), [N_g] double, host or
 * device per on_device.  On return the domain's orbitals are Psi(T).
 * Requires desc.scheme == FULL and desc.ortho_every == 0 (else
 * MLMD_ERR_UNSUPPORTED). */
MLMD_API mlmd_status mlmd_propagate_adjoint(mlmd_domain_t dom, int32_t n_steps, const double* A, int32_t ckpt_every,
                                   double* loss, double* dL_dA, void* dL_dV, int32_t on_device);

/* Batched form: n_domains MLMD_C64 FULL-scheme domains with uneven grids and
 * orbital counts stepped together; one step of all domains is one CUDA graph
 * launch.  The batch keeps references to the handles (do not destroy them
 * before the batch).  All domains must share dt and the caller's stream. */
MLMD_API mlmd_status mlmd_batch_create(int32_t n_domains, const mlmd_domain_t* doms, mlmd_batch_t* out);
MLMD_API mlmd_status mlmd_batch_destroy(mlmd_batch_t batch);

/* A: host double [n_domains][n_steps][3]; obs_out: NULL or host double
 * [n_domains][n_steps][5] with the per-domain rows of mlmd_propagate. */
MLMD_API mlmd_status mlmd_batch_propagate(mlmd_batch_t batch, int32_t n_steps, const double* A, double* obs_out);

/* Overlap without device allocation.  The paper has no counterpart: this
 * entry point serves callers that cannot allocate device memory at the point
 * of the call (a frozen or fully reserved memory pool, a framework that
 * forbids allocation on its hot path, a thread that must not contend for the
 * allocator).  It computes S[n][m] = scale * sum_g conj(X[g][n]) Y[g][m] for
 * caller-owned device arrays X, Y ([n_grid][n_orb] interleaved complex,
 * float pairs for MLMD_C64, double pairs for MLMD_C128, rows not padded) into
 * the caller-owned device array S (complex double [n_orb][n_orb]), on
 * `stream` (NULL: the legacy default stream); S is valid in stream order.
 * It calls no allocator: its split sums live in one 4 MiB device array that
 * the library declares at file scope and that every GPU loading the library
 * holds until exit, so n_orb may be at most MLMD_OVERLAP_NOALLOC_MAX_ORB
 * (larger values return MLMD_ERR_INVALID).  All calls share that array:
 * calls whose kernels overlap on the GPU (e.g. on two streams) race and give
 * wrong results.  Every call looks up the array's device address
 * (cudaGetSymbolAddress, a host-side lookup that allocates nothing) with the
 * current device, so a call after a device reset finds the array where the
 * reloaded library put it; the first call on a device may load the library's
 * device code, so make that first call before any stream capture. */
#define MLMD_OVERLAP_NOALLOC_MAX_ORB 512
MLMD_API mlmd_status mlmd_overlap_noalloc(int32_t precision, int64_t n_grid, int32_t n_orb, const void* X,
                                          const void* Y, double scale, double* S, void* stream);

/* Kernel timing hooks (measurement only).  While enabled, every launch of
 * the kinds below is bracketed by CUDA events recorded on the domain's
 * stream; mlmd_profile_read synchronises that stream and returns the summed
 * device time and launch count of one kind since the last enable.  Enabling
 * (enable != 0) resets the totals. */
/* MLMD_KERNEL_GEMM brackets a whole dense orbital GEMM (the Gram of
 * mlmd_overlap and of the re-orthonormalisation, the update Psi M), with its
 * operand split passes and partial-sum reductions. */
enum { MLMD_KERNEL_STAGE = 0, MLMD_KERNEL_PROJECT = 1, MLMD_KERNEL_SCATTER = 2, MLMD_KERNEL_GEMM = 3,
       MLMD_KERNEL_KINDS = 4 };
MLMD_API mlmd_status mlmd_profile_enable(mlmd_domain_t dom, int32_t enable);
MLMD_API mlmd_status mlmd_profile_read(mlmd_domain_t dom, int32_t kind, double* total_ms, uint64_t* launches);

/* Number of kernels this handle has launched since creation. */
MLMD_API uint64_t mlmd_launch_count(mlmd_domain_t dom);

/* Text of the last error on this handle ("" if none); owned by the handle. */
MLMD_API const char* mlmd_last_error(mlmd_domain_t dom);

/* Static text for a status code. */
MLMD_API const char* mlmd_status_string(mlmd_status s);

#ifdef __cplusplus
}
#endif

#endif /* MLMD_H */
