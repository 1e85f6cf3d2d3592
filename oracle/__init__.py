"""FP64 CPU oracle for the DC-MESH local-field-dynamics step.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg import this package; the product library never
does, and this package never imports the product library.  It shares no code
with the CUDA path: the heavy loops are plain C (``mlmd_oracle.c``, built with
gcc, OpenMP, ``-ffp-contract=off``) and the small dense linear algebra is
NumPy/LAPACK.

What each function follows (paper sections and equations):

* ``Domain.apply_h``         Eq. 3: h = 1/2(-i grad + A)^2 + v_loc + v_nl.
* ``Domain.taylor4``         exp(-i dt h(t_k)) to 4th order in dt, A at the
                             step midpoint (Eq. 2's t + (n + 1/2) dt).
* ``Domain.split_step``      Eq. 2: N_nl T4(h_loc) N_nl with normalised
                             N_nl = (1 - i dt/2 v_nl).
* ``Domain.project``         Sec. V.B.5 GEMM form of the nonlocal term.
* ``Domain.observables``     energy and current through the same projections
                             (Sec. V.B.5, last paragraph).
* ``nl_gauge=True``          velocity-gauge projectors b e^{-iA.(r-R_a)}: Eq. 3's
                             minimal coupling carried onto v_nl, whose current
                             gains the commutator part from the moment
                             projections ``Domain.project_moment`` (Sec. V.B.5,
                             last paragraph).
* ``overlap``/``reorth``     Eq. 5's Psi^dagger Psi product; Cholesky or
                             Loewdin re-orthonormalisation.
* ``ks_correction``          Eq. 5: Psi(t) -= delta Psi(0) Psi^dagger(0) Psi(t),
                             with the dV inner-product metric in Psi^dagger Psi.
* ``loss``/``adjoint``       excited-electron count 2(N_o - sum |<psi_n(0)|psi_m(T)>|^2)
                             (Sec. V.A.8's n_exc) and its discrete adjoint.
* ``occupations``            shadow-dynamics occupations f_s of the reference
                             orbitals and n_exc computed from them (Sec. V.A.3,
                             V.A.4 and V.A.8).

Parity pins: see ``tests/test_oracle_pins.py``; every function above is pinned
there against a dense eigendecomposition, closed forms, or brute force.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mlmd_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_CFLAGS = ["-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c11"]


def build(force: bool = False) -> str:
    """Compile the C part of the oracle with gcc (no-op when up to date)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", *_CFLAGS, "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _CDomain(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32 * 3), ("h", ctypes.c_double), ("n_orb", ctypes.c_int32),
        ("fd_order", ctypes.c_int32), ("V", ctypes.c_void_p), ("n_atoms", ctypes.c_int32),
        ("n_proj", ctypes.c_int32), ("off", ctypes.c_void_p), ("idx", ctypes.c_void_p),
        ("beta", ctypes.c_void_p), ("D", ctypes.c_void_p), ("nl_gauge", ctypes.c_int32),
        ("pos", ctypes.c_void_p),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            # a test may point the oracle at a deliberately broken build of
            # the same source to check that the pins catch the mistake
            path = os.environ.get("MLMD_ORACLE_LIB") or build()
            L = ctypes.CDLL(path)
            P = ctypes.c_void_p
            D = ctypes.POINTER(_CDomain)
            L.orc_gradient.argtypes = [D, ctypes.c_int, P, P]
            L.orc_apply_hloc.argtypes = [D, P, P, P]
            L.orc_project.argtypes = [D, P, P, P]
            L.orc_project_moment.argtypes = [D, P, ctypes.c_int, P, P]
            L.orc_scatter.argtypes = [D, P, P, P]
            L.orc_apply_vnl.argtypes = [D, P, P, P, P]
            L.orc_apply_h.argtypes = [D, P, P, P, P]
            L.orc_taylor4.argtypes = [D, P, ctypes.c_double, ctypes.c_int, P, P, P, P]
            L.orc_taylor4_adjoint.argtypes = [D, P, ctypes.c_double, P, P, P, P]
            L.orc_split_step.argtypes = [D, P, ctypes.c_double, P, P, P, P, P, P]
            L.orc_observables.argtypes = [D, P, P, P, P, P, P]
            L.orc_density_current.argtypes = [D, P, P, P, P, P, P, P]
            L.orc_overlap.argtypes = [ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_double, P, P, P]
            L.orc_neighbor_lists.argtypes = [P, ctypes.c_double, ctypes.c_int32, P, ctypes.c_double, P, P]
            L.orc_projector_values.argtypes = [P, ctypes.c_double, ctypes.c_int32, P, P, P, ctypes.c_int32,
                                               ctypes.c_double, P]
            L.orc_orbital_norms.argtypes = [D, P, P]
            _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.flags.c_contiguous
    return a.ctypes.data


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


# ---------------------------------------------------------------------------
# neighbour lists and projector values
# ---------------------------------------------------------------------------

def neighbor_lists(n, h, pos, r_cut):
    """Per-atom sorted lists of grid indices within the minimum-image
    distance r_cut (brute force over the whole grid).  Returns (off, idx)."""
    n3 = np.ascontiguousarray(n, dtype=np.int32)
    pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
    na = pos.shape[0]
    counts = np.zeros(max(na, 1), dtype=np.int64)
    lib().orc_neighbor_lists(_p(n3), h, na, _p(pos), r_cut, _p(counts), None)
    off = np.zeros(na + 1, dtype=np.int64)
    off[1:] = np.cumsum(counts[:na])
    idx = np.zeros(max(int(off[-1]), 1), dtype=np.int32)
    lib().orc_neighbor_lists(_p(n3), h, na, _p(pos), r_cut, _p(counts), _p(idx))
    return off, idx[: int(off[-1])]


def projector_values(n, h, pos, off, idx, n_proj, r_c):
    """beta[q][i] on the concatenated lists; each projector normalised to
    dV sum beta^2 = 1 over its truncated support."""
    n3 = np.ascontiguousarray(n, dtype=np.int32)
    pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
    off = np.ascontiguousarray(off, dtype=np.int64)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    beta = np.zeros((max(len(idx), 1), n_proj), dtype=np.float64)
    lib().orc_projector_values(_p(n3), h, pos.shape[0], _p(pos), _p(off), _p(idx if len(idx) else np.zeros(1, np.int32)),
                               n_proj, r_c, _p(beta))
    return beta[: len(idx)]


# ---------------------------------------------------------------------------
# one domain
# ---------------------------------------------------------------------------

class Domain:
    """One periodic domain: grid, local potential, projectors."""

    def __init__(self, n, h, n_orb, fd_order, V, atoms=None, n_proj=0, r_c=1.2, r_cut=3.0, D=None,
                 nl_gauge=False):
        self.n = tuple(int(v) for v in n)
        self.h = float(h)
        self.n_orb = int(n_orb)
        self.fd_order = int(fd_order)
        self.n_grid = self.n[0] * self.n[1] * self.n[2]
        self.dV = self.h ** 3
        self.V = np.ascontiguousarray(V, dtype=np.float64).reshape(self.n_grid)
        atoms = np.zeros((0, 3)) if atoms is None else np.asarray(atoms, np.float64).reshape(-1, 3)
        self.atoms = np.ascontiguousarray(atoms)
        self.n_proj = int(n_proj) if len(atoms) else 0
        if self.n_proj:
            self.off, self.idx = neighbor_lists(self.n, self.h, self.atoms, r_cut)
            self.beta = projector_values(self.n, self.h, self.atoms, self.off, self.idx, self.n_proj, r_c)
            self.D = np.ascontiguousarray(D, dtype=np.float64).reshape(len(atoms), self.n_proj)
        else:
            self.off = np.zeros(1, np.int64)
            self.idx = np.zeros(1, np.int32)
            self.beta = np.zeros((1, 1))
            self.D = np.zeros((1, 1))
        self._c = _CDomain()
        self._c.n = (ctypes.c_int32 * 3)(*self.n)
        self._c.h = self.h
        self._c.n_orb = self.n_orb
        self._c.fd_order = self.fd_order
        self._c.V = _p(self.V)
        self._c.n_atoms = len(self.atoms) if self.n_proj else 0
        self._c.n_proj = self.n_proj
        self._c.off = _p(self.off)
        self._c.idx = _p(self.idx)
        self._c.beta = _p(np.ascontiguousarray(self.beta))
        self._c.D = _p(self.D)
        self.nl_gauge = bool(nl_gauge)
        self._c.nl_gauge = int(self.nl_gauge)
        self._c.pos = _p(self.atoms) if len(self.atoms) else None
        self._beta_keep = self.beta
        self._proj = np.zeros(max(1, self._c.n_atoms * max(self.n_proj, 1) * self.n_orb), np.complex128)

    @classmethod
    def from_spec(cls, spec, V=None, n_orb=None, nl_gauge=False):
        from paper_2509_00966_gb300.inputs import gaussian_wells
        if V is None:
            V = gaussian_wells(spec.n, spec.h, spec.wells, spec.well_depth, spec.well_width)
        return cls(spec.n, spec.h, n_orb or spec.n_orb, spec.fd_order, V, spec.atoms, spec.n_proj,
                   spec.r_c, spec.r_cut, spec.D, nl_gauge=nl_gauge)

    # -- helpers ---------------------------------------------------------
    def _check(self, psi):
        psi = _c128(psi)
        assert psi.shape == (self.n_grid, self.n_orb), psi.shape
        return psi

    def _like(self, psi):
        return np.zeros_like(psi)

    def _A(self, A):
        return np.ascontiguousarray(A, dtype=np.float64).reshape(3)

    # -- operators ---------------------------------------------------------
    def gradient(self, psi, axis):
        psi = self._check(psi)
        out = self._like(psi)
        lib().orc_gradient(ctypes.byref(self._c), int(axis), _p(psi), _p(out))
        return out

    def apply_hloc(self, psi, A):
        psi = self._check(psi)
        out = self._like(psi)
        lib().orc_apply_hloc(ctypes.byref(self._c), _p(self._A(A)), _p(psi), _p(out))
        return out

    def apply_vnl(self, psi, A=None):
        """v_nl psi; with velocity-gauge projectors at field A (None: A = 0)."""
        psi = self._check(psi)
        out = self._like(psi)
        Ac = None if A is None else self._A(A)
        lib().orc_apply_vnl(ctypes.byref(self._c), None if Ac is None else _p(Ac), _p(psi), _p(out), _p(self._proj))
        return out

    def apply_h(self, psi, A):
        psi = self._check(psi)
        out = self._like(psi)
        lib().orc_apply_h(ctypes.byref(self._c), _p(self._A(A)), _p(psi), _p(out), _p(self._proj))
        return out

    def project(self, psi, A=None):
        """<beta~_ai|psi_o> as complex [n_atoms, n_proj, n_orb] (beta~ = beta,
        or beta e^{-iA.(r-R_a)} with velocity-gauge projectors at field A)."""
        psi = self._check(psi)
        out = np.zeros((self._c.n_atoms, self.n_proj, self.n_orb), np.complex128)
        if self.n_proj:
            Ac = None if A is None else self._A(A)
            lib().orc_project(ctypes.byref(self._c), None if Ac is None else _p(Ac), _p(psi), _p(out))
        return out

    def project_moment(self, psi, A, axis):
        """<(r - R_a)_axis beta~_ai|psi_o>, complex [n_atoms, n_proj, n_orb]."""
        psi = self._check(psi)
        out = np.zeros((self._c.n_atoms, self.n_proj, self.n_orb), np.complex128)
        if self.n_proj:
            Ac = self._A(A)
            lib().orc_project_moment(ctypes.byref(self._c), _p(Ac), int(axis), _p(psi), _p(out))
        return out

    def taylor4(self, psi, A, dt, local_only=False):
        psi = self._check(psi)
        out = self._like(psi)
        work = np.zeros((2,) + psi.shape, np.complex128)
        lib().orc_taylor4(ctypes.byref(self._c), _p(self._A(A)), float(dt), int(bool(local_only)),
                          _p(psi), _p(out), _p(work), _p(self._proj))
        return out

    def taylor4_adjoint(self, lam, A, dt):
        lam = self._check(lam)
        out = self._like(lam)
        work = np.zeros((2,) + lam.shape, np.complex128)
        lib().orc_taylor4_adjoint(ctypes.byref(self._c), _p(self._A(A)), float(dt), _p(lam), _p(out),
                                  _p(work), _p(self._proj))
        return out

    def split_step(self, psi, A, dt):
        psi = self._check(psi)
        out = self._like(psi)
        work = np.zeros((2,) + psi.shape, np.complex128)
        nb = np.zeros(self.n_orb)
        na = np.zeros(self.n_orb)
        lib().orc_split_step(ctypes.byref(self._c), _p(self._A(A)), float(dt), _p(psi), _p(out), _p(work),
                             _p(self._proj), _p(nb), _p(na))
        return out

    def orbital_norms(self, psi):
        psi = self._check(psi)
        out = np.zeros(self.n_orb)
        lib().orc_orbital_norms(ctypes.byref(self._c), _p(psi), _p(out))
        return out

    def observables(self, psi, A, f):
        """[electron count, energy, Jx, Jy, Jz] of psi under h(A)."""
        psi = self._check(psi)
        f = np.ascontiguousarray(f, np.float64)
        obs = np.zeros(5)
        work = self._like(psi)
        lib().orc_observables(ctypes.byref(self._c), _p(self._A(A)), _p(f), _p(psi), _p(obs), _p(work),
                              _p(self._proj))
        return obs

    def density_current(self, psi, A, f):
        """(rho[N_g], j[3, N_g], J[3])."""
        psi = self._check(psi)
        f = np.ascontiguousarray(f, np.float64)
        rho = np.zeros(self.n_grid)
        j = np.zeros((3, self.n_grid))
        J = np.zeros(3)
        work = self._like(psi)
        lib().orc_density_current(ctypes.byref(self._c), _p(self._A(A)), _p(f), _p(psi), _p(rho), _p(j),
                                  _p(J), _p(work))
        return rho, j, J

    def dense_h(self, A, n_orb_probe=None):
        """h(A) as a dense N_g x N_g matrix, column g = h e_g (tiny grids only)."""
        ng = self.n_grid
        assert ng <= 1000
        cols = np.zeros((ng, ng), np.complex128)
        save = self.n_orb
        self.n_orb = ng
        self._c.n_orb = ng
        self._proj = np.zeros(max(1, self._c.n_atoms * max(self.n_proj, 1) * ng), np.complex128)
        try:
            cols = self.apply_h(np.eye(ng, dtype=np.complex128), A)
        finally:
            self.n_orb = save
            self._c.n_orb = save
            self._proj = np.zeros(max(1, self._c.n_atoms * max(self.n_proj, 1) * save), np.complex128)
        return cols


# ---------------------------------------------------------------------------
# dense orbital-space linear algebra (NumPy / LAPACK)
# ---------------------------------------------------------------------------

def overlap(a, b, dV):
    """S[n][m] = dV sum_r conj(a_n(r)) b_m(r)."""
    a = _c128(a)
    b = _c128(b)
    S = np.zeros((a.shape[1], b.shape[1]), np.complex128)
    lib().orc_overlap(a.shape[0], a.shape[1], b.shape[1], float(dV), _p(a), _p(b), _p(S))
    return S


def reorth(psi, dV, kind="chol"):
    """Cholesky: S = L L^H, psi <- psi L^{-H}.  Loewdin: psi <- psi S^{-1/2}."""
    import scipy.linalg as sla
    psi = _c128(psi)
    S = overlap(psi, psi, dV)
    if kind == "chol":
        L = np.linalg.cholesky(S)
        return np.ascontiguousarray(sla.solve_triangular(L.conj(), psi.T, lower=True).T)
    w, U = np.linalg.eigh(S)
    return np.ascontiguousarray(psi @ ((U * (1.0 / np.sqrt(w))) @ U.conj().T))


def ks_correction(psi_t, psi_0, delta, dV):
    """Eq. 5, the nonlocal correction in the space of the Kohn-Sham orbitals:
    Psi(t) <- Psi(t) - delta Psi(0) C with C = dV Psi(0)^H Psi(t) (the
    overlap in the grid's inner product, so delta is dimensionless).
    Two matrix products, as the equation is written."""
    psi_t = _c128(psi_t)
    psi_0 = _c128(psi_0)
    C = overlap(psi_0, psi_t, dV)
    return np.ascontiguousarray(psi_t - complex(delta) * (psi_0 @ C))


def loss(psi_ref, psi_T, dV):
    """n_exc = 2 (N_o - sum_{n,m} |<psi_n(0)|psi_m(T)>|^2)."""
    C = overlap(psi_ref, psi_T, dV)
    return 2.0 * (psi_ref.shape[1] - float(np.sum(np.abs(C) ** 2)))


def occupations(psi_ref, psi_t, f, dV):
    """Occupation numbers handed from LFD back to QXMD (Sec. V.A.3-4) and the
    excited-electron count computed from them (Sec. V.A.8).  The reference
    orbitals psi_s(0) are the adiabatic states; the propagated orbitals
    psi_n(t) carry the occupations f_n.  The occupation of reference state s
    at time t is f_s(t) = sum_n f_n |<psi_s(0)|psi_n(t)>|^2, and
    n_exc = sum_n f_n - sum_s f_s(t), the electrons that have left the span
    of the reference orbitals.  Returns (f_s(t) [N_o], n_exc)."""
    C = overlap(psi_ref, psi_t, dV)          # C[s][n] = <psi_s(0)|psi_n(t)>
    f = np.asarray(f, np.float64)
    f_s = (np.abs(C) ** 2) @ f
    return f_s, float(np.sum(f) - np.sum(f_s))


def propagate(dom: Domain, psi, A, dt, f, scheme="full", ortho_every=0, ortho_kind="chol", step0=0):
    """Run len(A) steps.  Row k of the returned observables describes the
    state before step k under h(A_k).  Re-orthonormalisation follows every
    step whose 1-based global count t = step0 + k + 1 is a multiple of
    ortho_every."""
    psi = _c128(psi)
    A = np.asarray(A, np.float64).reshape(-1, 3)
    obs = np.zeros((len(A), 5))
    for k in range(len(A)):
        obs[k] = dom.observables(psi, A[k], f)
        psi = dom.taylor4(psi, A[k], dt) if scheme == "full" else dom.split_step(psi, A[k], dt)
        t = step0 + k + 1
        if ortho_every and t % ortho_every == 0:
            psi = reorth(psi, dom.dV, ortho_kind)
    return psi, obs


def adjoint(dom: Domain, psi_init, psi_ref, A, dt, ckpt_every):
    """Loss n_exc(psi(T)) and its gradients by the discrete adjoint of the
    Taylor map.  psi is checkpointed every ckpt_every steps and recomputed
    inside each segment.  With c_j = (-i dt)^j / j!, per step k:
      lam_k = sum_j conj(c_j) h_k^j lam_{k+1}
      dL/dA_{k,a} = 2 Re sum_j c_j sum_{p<j} <h^{j-1-p} lam_{k+1} | (-i G_a + A_a) h^p psi_k>
      dL/dV(r)   += 2 Re sum_j c_j sum_{p<j} sum_o conj(h^{j-1-p} lam)(r) (h^p psi_k)(r)
    with Euclidean inner products (no dV) and lam_N = dL/dpsi*(T) = -2 dV psi_ref C.
    Returns (loss, dL_dA [n_steps, 3], dL_dV [N_g]).  Real projectors only:
    with velocity-gauge projectors dh/dA gains the nonlocal commutator, which
    this contraction does not carry."""
    if dom.nl_gauge and dom.n_proj:
        raise NotImplementedError("adjoint with velocity-gauge projectors")
    psi_init = _c128(psi_init)
    psi_ref = _c128(psi_ref)
    A = np.asarray(A, np.float64).reshape(-1, 3)
    N = len(A)
    K = max(1, int(ckpt_every))
    ckpt = {0: psi_init.copy()}
    psi = psi_init
    for k in range(N):
        psi = dom.taylor4(psi, A[k], dt)
        if (k + 1) % K == 0 and k + 1 < N:
            ckpt[k + 1] = psi.copy()
    C = overlap(psi_ref, psi, dom.dV)
    L = 2.0 * (psi_ref.shape[1] - float(np.sum(np.abs(C) ** 2)))
    lam = -2.0 * dom.dV * (psi_ref @ C)
    c = [1.0 + 0j]
    for j in range(1, 5):
        c.append(c[-1] * (-1j * dt) / j)
    dA = np.zeros((N, 3))
    dVg = np.zeros(dom.n_grid)
    for s0 in reversed(range(0, N, K)):
        s1 = min(s0 + K, N)
        states = [ckpt[s0]]
        for k in range(s0, s1 - 1):
            states.append(dom.taylor4(states[-1], A[k], dt))
        for k in reversed(range(s0, s1)):
            u = [states[k - s0]]
            for p in range(3):
                u.append(dom.apply_h(u[-1], A[k]))
            w = [lam]
            for q in range(4):
                w.append(dom.apply_h(w[-1], A[k]))
            Gu = [[dom.gradient(u[p], ax) for ax in range(3)] for p in range(4)]
            for j in range(1, 5):
                for p in range(j):
                    q = j - 1 - p
                    wu = np.vdot(w[q], u[p])
                    for ax in range(3):
                        dA[k, ax] += 2.0 * np.real(c[j] * (-1j * np.vdot(w[q], Gu[p][ax]) + A[k, ax] * wu))
                    dVg += 2.0 * np.real(c[j] * np.sum(np.conj(w[q]) * u[p], axis=1))
            lam = sum(np.conj(c[j]) * w[j] for j in range(5))
    return L, dA, dVg
