"""Pins of the FP64 oracle against things other than itself.

Every check below compares the oracle with an independent route to the same
number: a dense eigendecomposition (LAPACK), closed-form plane-wave phases of
the finite-difference operators, exact central differences of a quadratic,
brute-force lattice counts, invariants (Hermiticity, translation, norms).
A dropped term, a flipped sign, a wrong coefficient or a transposed axis in
the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest
import scipy.linalg as sla

import oracle
from paper_2509_00966_gb300 import inputs


def _pw(n, h, m):
    """Plane wave exp(i k.r) / sqrt(N dV), k = 2 pi m / L, on the linear grid."""
    nx, ny, nz = n
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ph = 2 * np.pi * (m[0] * x.ravel() / nx + m[1] * y.ravel() / ny + m[2] * z.ravel() / nz)
    return np.exp(1j * ph) / math.sqrt(nx * ny * nz * h ** 3)


def _s(order, th):
    return 2 - 2 * np.cos(th) if order == 2 else 2.5 - 8.0 / 3.0 * np.cos(th) + np.cos(2 * th) / 6.0


def _kappa(order, th, h):
    return np.sin(th) / h if order == 2 else (4.0 / 3.0 * np.sin(th) - np.sin(2 * th) / 6.0) / h


def _g(x):
    return 1 - 1j * x - x ** 2 / 2 + 1j * x ** 3 / 6 + x ** 4 / 24


def _tiny_domain(order=4, n=(4, 5, 6), h=0.6, n_orb=3, with_nl=True, seed=7):
    rng = np.random.default_rng(seed)
    V = rng.uniform(-1, 0.5, n[0] * n[1] * n[2])
    L = np.array(n) * h
    atoms = rng.uniform(0, 1, (2, 3)) * L if with_nl else None
    D = rng.uniform(-1, 1, (2, 4)) if with_nl else None
    return oracle.Domain(n, h, n_orb, order, V, atoms, 4 if with_nl else 0, r_c=0.7, r_cut=1.3, D=D)


def _rand_psi(ng, no, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((ng, no)) + 1j * rng.standard_normal((ng, no))


# ---------------------------------------------------------------------------
# stencils: plane waves are exact eigenvectors with a closed-form eigenvalue
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("order", [2, 4])
def test_plane_wave_eigenvalue_and_phase(order):
    n, h = (6, 8, 10), 0.45
    A = np.array([0.03, -0.07, 0.11])
    dom = oracle.Domain(n, h, 3, order, np.zeros(n[0] * n[1] * n[2]))
    ms = [(1, 0, 0), (0, -2, 1), (2, 3, -4)]
    psi = np.stack([_pw(n, h, m) for m in ms], axis=1)
    hpsi = dom.apply_h(psi, A)
    E = []
    for m in ms:
        th = 2 * np.pi * np.array(m) / np.array(n)
        E.append(sum(0.5 * _s(order, th[a]) / h ** 2 + A[a] * _kappa(order, th[a], h) for a in range(3))
                 + 0.5 * A @ A)
    E = np.array(E)
    np.testing.assert_allclose(hpsi, psi * E[None, :], atol=1e-12, rtol=0)
    # Taylor-4 phase after several steps: g(dt E)^n
    dt, nsteps = 0.05, 7
    out = psi.copy()
    for _ in range(nsteps):
        out = dom.taylor4(out, A, dt)
    np.testing.assert_allclose(out, psi * (_g(dt * E) ** nsteps)[None, :], atol=1e-13, rtol=0)


def test_constant_potential_shifts_energy():
    n, h = (5, 5, 6), 0.5
    ng = n[0] * n[1] * n[2]
    psi = _pw(n, h, (1, 1, 0))[:, None]
    d0 = oracle.Domain(n, h, 1, 4, np.zeros(ng))
    d1 = oracle.Domain(n, h, 1, 4, np.full(ng, -0.37))
    A = np.zeros(3)
    np.testing.assert_allclose(d1.apply_h(psi, A) - d0.apply_h(psi, A), -0.37 * psi, atol=1e-14)


def test_local_potential_is_diagonal():
    dom = _tiny_domain(with_nl=False)
    dom0 = oracle.Domain(dom.n, dom.h, dom.n_orb, dom.fd_order, np.zeros(dom.n_grid))
    A = np.array([0.1, 0.0, -0.2])
    diff = dom.dense_h(A) - dom0.dense_h(A)
    np.testing.assert_allclose(diff, np.diag(dom.V).astype(np.complex128), atol=1e-13, rtol=0)


# ---------------------------------------------------------------------------
# Hermiticity of the whole operator (local + A.grad + projectors)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("order", [2, 4])
def test_hermitian(order):
    dom = _tiny_domain(order=order)
    H = dom.dense_h(np.array([0.2, -0.1, 0.05]))
    assert np.max(np.abs(H - H.conj().T)) < 1e-13 * np.max(np.abs(H))
    # and on a larger grid through inner products
    spec = inputs.config("c4", n=12, n_orb=2)
    d = oracle.Domain.from_spec(spec)
    phi = _rand_psi(d.n_grid, 2, 1)
    psi = _rand_psi(d.n_grid, 2, 2)
    A = np.array([0.01, 0.02, 0.05])
    lhs = np.vdot(phi, d.apply_h(psi, A))
    rhs = np.conj(np.vdot(psi, d.apply_h(phi, A)))
    assert abs(lhs - rhs) < 1e-13 * abs(lhs)


# ---------------------------------------------------------------------------
# whole Taylor step against the dense eigendecomposition
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("order", [2, 4])
def test_taylor4_matches_dense_eigendecomposition(order):
    dom = _tiny_domain(order=order)
    A = np.array([0.05, -0.02, 0.08])
    dt = 0.04
    H = dom.dense_h(A)
    lam, U = np.linalg.eigh(H)
    psi = _rand_psi(dom.n_grid, dom.n_orb, 3)
    ref = U @ (_g(dt * lam)[:, None] * (U.conj().T @ psi))
    out = dom.taylor4(psi, A, dt)
    assert np.max(np.abs(out - ref)) < 1e-13 * np.max(np.abs(psi))
    # truncation against the exact exponential: |T4(-ix) - e^{-ix}| <= x^5/120
    exact = sla.expm(-1j * dt * H) @ psi
    bound = np.max(np.abs(dt * lam)) ** 5 / 120 * np.linalg.norm(psi, axis=0).max()
    assert np.max(np.linalg.norm(out - exact, axis=0)) <= bound * 1.0001 + 1e-14
    # the adjoint map is the conjugate transpose of the Taylor matrix
    T = U @ np.diag(_g(dt * lam)) @ U.conj().T
    lam_v = _rand_psi(dom.n_grid, dom.n_orb, 4)
    np.testing.assert_allclose(dom.taylor4_adjoint(lam_v, A, dt), T.conj().T @ lam_v, atol=1e-13, rtol=0)


def test_norm_and_energy_follow_spectral_prediction():
    """Static h: Taylor-4 damps each eigencomponent by |g(dt lam)|^2 per step
    (|g(x)|^2 = 1 - x^6/72 + x^8/576), so the norm and energy after n steps are
    sums over the dense spectrum."""
    dom = _tiny_domain(order=4, n_orb=2)
    A = np.array([0.0, 0.03, 0.0])
    dt, n = 0.08, 12
    H = dom.dense_h(A)
    lam, U = np.linalg.eigh(H)
    x = dt * lam
    np.testing.assert_allclose(np.abs(_g(x)) ** 2, 1 - x ** 6 / 72 + x ** 8 / 576, rtol=1e-13)
    psi = _rand_psi(dom.n_grid, 2, 5)
    psi /= np.sqrt(dom.dV) * np.linalg.norm(psi, axis=0)
    f = np.array([2.0, 1.0])
    out, obs = oracle.propagate(dom, psi, np.tile(A, (n, 1)), dt, f)
    c = U.conj().T @ psi
    for k in (0, 5, n - 1):
        damp = (1 - x ** 6 / 72 + x ** 8 / 576) ** k
        nrm = dom.dV * np.sum(f[None, :] * (np.abs(c) ** 2) * damp[:, None])
        en = dom.dV * np.sum(f[None, :] * (np.abs(c) ** 2) * (damp * lam)[:, None])
        assert abs(obs[k, 0] - nrm) < 1e-12 * abs(nrm)
        assert abs(obs[k, 1] - en) < 1e-12 * max(1.0, abs(en))


def test_plane_wave_norm_decay_closed_form():
    """A plane wave keeps its shape; its norm decays by exactly
    |g(x)|^2 = 1 - x^6/72 + x^8/576 per step, x = dt E_k."""
    n, h = (8, 8, 8), 0.5
    dom = oracle.Domain(n, h, 1, 4, np.zeros(512))
    psi = _pw(n, h, (1, 0, 0))[:, None]
    out, obs = oracle.propagate(dom, psi, np.zeros((20, 3)), 0.02, np.array([2.0]))
    x = 0.02 * 0.5 * _s(4, 2 * np.pi / 8) / h ** 2
    r = 1 - x ** 6 / 72 + x ** 8 / 576
    pred = 2.0 * r ** np.arange(20)
    np.testing.assert_allclose(obs[:, 0], pred, rtol=0, atol=1e-13)
    # the decay itself (~1e-11 over the run) is resolved to a few per cent
    np.testing.assert_allclose(2.0 - obs[10:, 0], 2.0 - pred[10:], rtol=5e-2)
    assert 1.0 - r < 1e-11  # a smooth state conserves the norm to O(x^6)


# ---------------------------------------------------------------------------
# projectors and neighbour lists
# ---------------------------------------------------------------------------

def test_neighbor_list_brute_force_count():
    """Atom exactly on a grid point: the list is the set of integer offsets with
    h^2 |m|^2 <= r_cut^2, counted here by direct enumeration."""
    n, h, rcut = (20, 22, 24), 0.4, 2.05
    pos = np.array([[5 * h, 7 * h, 11 * h], [0.0, 0.0, 0.0]])
    off, idx = oracle.neighbor_lists(n, h, pos, rcut)
    r = int(rcut / h) + 1
    cnt = sum(1 for i in range(-r, r + 1) for j in range(-r, r + 1) for k in range(-r, r + 1)
              if (i * h) ** 2 + (j * h) ** 2 + (k * h) ** 2 <= rcut ** 2 + 1e-12)
    assert off[1] - off[0] == cnt and off[2] - off[1] == cnt
    for a in range(2):
        lst = idx[off[a]:off[a + 1]]
        assert np.all(np.diff(lst) > 0)
    # the atom at the origin wraps: its list holds both ends of every axis
    lst = idx[off[1]:off[2]]
    xs = lst % n[0]
    assert 0 in xs and n[0] - 1 in xs


def test_neighbor_list_exact_tie_is_member():
    """A point at exactly r_cut belongs to the sphere (d^2 <= r_cut^2): with
    h = 0.5 and r_cut = 1.5 (both exact in binary) and the atom on a grid
    point, every offset with |m|^2 = 9 -- (3,0,0) and (2,2,1) up to signs and
    order, 30 points -- lies exactly on the sphere."""
    n, h, rcut = (16, 16, 16), 0.5, 1.5
    pos = np.array([[4 * h, 5 * h, 6 * h]])
    off, idx = oracle.neighbor_lists(n, h, pos, rcut)
    inside = sum(1 for i in range(-3, 4) for j in range(-3, 4) for k in range(-3, 4) if i * i + j * j + k * k <= 9)
    on = sum(1 for i in range(-3, 4) for j in range(-3, 4) for k in range(-3, 4) if i * i + j * j + k * k == 9)
    assert on == 30
    assert off[1] - off[0] == inside
    lst = set(idx[off[0]:off[1]].tolist())
    assert (4 + 3) + 16 * (5 + 16 * 6) in lst                   # offset (3, 0, 0)
    assert (4 + 2) + 16 * ((5 - 2) + 16 * (6 + 1)) in lst       # offset (2, -2, 1)


def test_neighbor_list_translation_and_wrap():
    n, h, rcut = (16, 16, 16), 0.5, 1.6
    pos = np.array([[3.25, 4.125, 7.5]])
    off, idx = oracle.neighbor_lists(n, h, pos, rcut)
    off2, idx2 = oracle.neighbor_lists(n, h, pos + np.array([[3 * h, -2 * h, 9 * h]]), rcut)
    x, y, z = idx % 16, (idx // 16) % 16, idx // 256
    shifted = np.sort(((x + 3) % 16) + 16 * (((y - 2) % 16) + 16 * ((z + 9) % 16)))
    np.testing.assert_array_equal(shifted, idx2)


def test_single_atom_projector_spectrum():
    """One atom on a grid point: s, px, py, pz are mutually orthogonal by parity
    and normalised, so v_nl has eigenvalues {D_i} plus zeros, and trace D."""
    n, h = (9, 9, 9), 0.5
    ng = 729
    pos = np.array([[4 * h, 4 * h, 4 * h]])
    D = np.array([[0.7, -0.3, 0.2, -0.9]])
    dom = oracle.Domain(n, h, 1, 2, np.zeros(ng), pos, 4, r_c=0.6, r_cut=1.6, D=D)
    d0 = oracle.Domain(n, h, 1, 2, np.zeros(ng))
    Vnl = dom.dense_h(np.zeros(3)) - d0.dense_h(np.zeros(3))
    ev = np.linalg.eigvalsh(Vnl)
    big = np.sort(ev[np.abs(ev) > 1e-10])
    np.testing.assert_allclose(big, np.sort(D[0]), atol=1e-12)
    # p_y does not see a wave that is constant along y; p_x does
    pw = _pw(n, h, (1, 0, 0))[:, None]
    P = dom.project(pw)
    assert abs(P[0, 2, 0]) < 1e-13 and abs(P[0, 3, 0]) < 1e-13 and abs(P[0, 1, 0]) > 1e-3


def test_projector_trace_any_position_8_shapes():
    n, h = (8, 9, 10), 0.45
    rng = np.random.default_rng(11)
    pos = rng.uniform(0, 1, (3, 3)) * np.array(n) * h
    D = rng.uniform(-1, 1, (3, 8))
    dom = oracle.Domain(n, h, 1, 4, np.zeros(720), pos, 8, r_c=0.8, r_cut=1.5, D=D)
    d0 = oracle.Domain(n, h, 1, 4, np.zeros(720))
    Vnl = dom.dense_h(np.zeros(3)) - d0.dense_h(np.zeros(3))
    assert abs(np.trace(Vnl).real - D.sum()) < 1e-12
    assert np.max(np.abs(Vnl - Vnl.T)) < 1e-14 and np.max(np.abs(Vnl.imag)) == 0.0


def test_projector_radial_profile_ratios():
    """The radial shape of every projector, free of its normalisation: with
    the atom on a grid point the displacement to a point is exactly m h for
    an integer offset m, so within one projector the ratio of two values is
    fixed by the Gaussian width alone,
        s(m) / s(m')     = exp(-(|m|^2 - |m'|^2) h^2 / (2 w^2)),
        p_x(m) / p_x(m') = (m_x / m'_x) exp(-(|m|^2 - |m'|^2) h^2 / (2 w^2)),
    with w = r_c for the first four projectors and w = r_c / sqrt(2) for the
    second four of the 8-projector set.  The normalisation constant cancels,
    so this pins the width, the second shell's width and the sign and axis of
    the p factor independently of the trace and spectrum pins."""
    n, h, r_c, r_cut = (14, 13, 12), 0.5, 0.9, 1.6
    c = np.array([5, 6, 7])
    pos = (c * h)[None, :].astype(np.float64)
    off, idx = oracle.neighbor_lists(n, h, pos, r_cut)
    beta = oracle.projector_values(n, h, pos, off, idx, 8, r_c)
    where = {int(g): q for q, g in enumerate(idx[off[0]:off[1]])}

    def val(m, i):
        x, y, z = (c + np.array(m)) % np.array(n)
        return beta[where[int(x + n[0] * (y + n[1] * z))], i]

    shells = [(1, 0, 0), (1, 1, 0), (2, 0, 0), (1, 1, 1), (2, 1, 1), (3, 0, 0)]
    for st, w in ((0, r_c), (4, r_c / math.sqrt(2.0))):
        for a in range(len(shells)):
            for b in range(a + 1, len(shells)):
                ma, mb = np.array(shells[a]), np.array(shells[b])
                ratio = math.exp(-(ma @ ma - mb @ mb) * h * h / (2.0 * w * w))
                assert abs(val(ma, st) / val(mb, st) - ratio) < 1e-12 * ratio
                # p_x, p_y, p_z: the same Gaussian times the displacement along its own axis
                for ax in range(3):
                    if ma[ax] != 0 and mb[ax] != 0:
                        r = ratio * ma[ax] / mb[ax]
                        assert abs(val(ma, st + 1 + ax) / val(mb, st + 1 + ax) - r) < 1e-12 * abs(r)
        for ax in range(3):
            e = np.zeros(3, int)
            e[ax] = 1
            assert val(e, st + 1 + ax) > 0.0                       # delta = r - R: positive on the + side
            np.testing.assert_allclose(val(-e, st + 1 + ax), -val(e, st + 1 + ax), rtol=1e-14)
            assert val(np.roll(e, 1), st + 1 + ax) == 0.0           # no displacement along the axis: zero
    # the two shells really differ in width: s(1,0,0) / s(2,0,0) is e^{3 h^2 / (2 r_c^2)} and e^{3 h^2 / r_c^2}
    assert abs(val((1, 0, 0), 0) / val((2, 0, 0), 0) - math.exp(3 * h * h / (2 * r_c * r_c))) < 1e-12 * 2
    assert abs(val((1, 0, 0), 4) / val((2, 0, 0), 4) - math.exp(3 * h * h / (r_c * r_c))) < 1e-12 * 3


# ---------------------------------------------------------------------------
# observables
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("order", [2, 4])
def test_current_is_exact_derivative_of_energy(order):
    """E(A) is a quadratic in A, so the central difference is exact up to rounding."""
    dom = _tiny_domain(order=order, n_orb=3)
    psi = _rand_psi(dom.n_grid, 3, 9)
    f = np.array([2.0, 2.0, 1.0])
    A = np.array([0.02, -0.04, 0.06])
    J = dom.observables(psi, A, f)[2:]
    for ax in range(3):
        e = np.zeros(3)
        e[ax] = 1e-3
        dE = (dom.observables(psi, A + e, f)[1] - dom.observables(psi, A - e, f)[1]) / 2e-3
        assert abs(dE - J[ax]) < 1e-9 * max(1.0, abs(J[ax]))
    rho, j, Jd = dom.density_current(psi, A, f)
    np.testing.assert_allclose(Jd, J, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(rho.sum() * dom.dV, dom.observables(psi, A, f)[0], rtol=1e-13)


def test_plane_wave_observables_closed_form():
    n, h, order = (6, 6, 8), 0.4, 4
    dom = oracle.Domain(n, h, 1, order, np.zeros(288))
    m = (1, -1, 2)
    psi = _pw(n, h, m)[:, None]
    A = np.array([0.01, 0.02, -0.03])
    th = 2 * np.pi * np.array(m) / np.array(n)
    kap = np.array([_kappa(order, th[a], h) for a in range(3)])
    obs = dom.observables(psi, A, np.array([2.0]))
    assert abs(obs[0] - 2.0) < 1e-13
    np.testing.assert_allclose(obs[2:], 2.0 * (kap + A), atol=1e-12)
    rho, j, J = dom.density_current(psi, A, np.array([2.0]))
    np.testing.assert_allclose(rho, 2.0 / (288 * h ** 3), rtol=1e-12)
    np.testing.assert_allclose(j, (2.0 * (kap + A) / (288 * h ** 3))[:, None] * np.ones((3, 288)), rtol=1e-11)


def test_real_orbitals_carry_no_current_at_zero_field():
    dom = _tiny_domain(n_orb=2)
    psi = np.random.default_rng(3).standard_normal((dom.n_grid, 2)).astype(np.complex128)
    rho, j, J = dom.density_current(psi, np.zeros(3), np.array([2.0, 2.0]))
    assert np.max(np.abs(j)) == 0.0


def test_translation_bit_exact_local():
    """Shifting V and psi by whole grid vectors shifts h_loc psi exactly."""
    n, h = (6, 7, 8), 0.5
    rng = np.random.default_rng(1)
    ng = 336
    V = rng.uniform(-1, 0, ng)
    psi = _rand_psi(ng, 2, 4)
    A = np.array([0.1, 0.2, 0.3])

    def shift(a):
        return np.roll(a.reshape(n[2], n[1], n[0], -1), (1, -2, 3), axis=(0, 1, 2)).reshape(ng, -1)

    d0 = oracle.Domain(n, h, 2, 4, V)
    d1 = oracle.Domain(n, h, 2, 4, shift(V[:, None])[:, 0])
    np.testing.assert_array_equal(d1.apply_hloc(shift(psi), A), shift(d0.apply_hloc(psi, A)))


# ---------------------------------------------------------------------------
# velocity-gauge projectors b e^{-iA.(r - R_a)} and their commutator current
# ---------------------------------------------------------------------------

def _gauge_domain(order=4, n=(6, 5, 7), h=0.55, n_orb=3, seed=5, atoms=None, gauge=True):
    rng = np.random.default_rng(seed)
    ng = n[0] * n[1] * n[2]
    V = rng.uniform(-1, 0.5, ng)
    L = np.array(n) * h
    # one atom near a corner so that its sphere wraps on every axis
    drawn = np.array([[0.3 * h, L[1] - 0.4 * h, 0.45 * h], rng.uniform(0, 1, 3) * L, rng.uniform(0, 1, 3) * L])
    atoms = drawn if atoms is None else atoms
    D = rng.uniform(-1, 1, (len(atoms), 4))
    return oracle.Domain(n, h, n_orb, order, V, atoms, 4, r_c=0.7, r_cut=1.4, D=D, nl_gauge=gauge)


def _grid_r(n, h):
    z, y, x = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1) * h


def test_gauge_projectors_equal_real_ones_at_zero_field():
    d0 = _gauge_domain(gauge=False)
    d1 = _gauge_domain(gauge=True)
    psi = _rand_psi(d0.n_grid, 3, 1)
    assert np.max(np.abs(d1.apply_h(psi, np.zeros(3)) - d0.apply_h(psi, np.zeros(3)))) == 0.0
    assert np.max(np.abs(d1.project(psi, np.zeros(3)) - d0.project(psi))) == 0.0


def test_gauge_covariance_at_reciprocal_lattice_field():
    """For A = 2 pi m / L the phase U = e^{-iA.r} is periodic on the grid and
    v_nl(A) = U v_nl(0) U^H exactly (the per-atom factor e^{iA.R_a} cancels
    inside each projector): v_nl(A) U phi = U v_nl(0) phi for any phi, and
    the nonlocal energy of U phi at A is that of phi at A = 0."""
    n, h = (6, 5, 7), 0.55
    dom = _gauge_domain(n=n, h=h)
    L = np.array(n) * h
    A = 2 * np.pi * np.array([1, -2, 1]) / L
    U = np.exp(-1j * (_grid_r(n, h) @ A))[:, None]
    phi = _rand_psi(dom.n_grid, 3, 2)
    lhs = dom.apply_vnl(U * phi, A)
    rhs = U * dom.apply_vnl(phi, np.zeros(3))
    assert np.max(np.abs(lhs - rhs)) < 1e-13 * np.max(np.abs(rhs))
    P_A = dom.project(U * phi, A)
    P_0 = dom.project(phi, np.zeros(3))
    e_A = np.einsum("ai,aio->", dom.D, np.abs(P_A) ** 2)
    e_0 = np.einsum("ai,aio->", dom.D, np.abs(P_0) ** 2)
    assert abs(e_A - e_0) < 1e-13 * abs(e_0)


def test_gauge_translation_across_the_wrap():
    """Shifting atoms and orbitals by whole grid vectors shifts v_nl(A) psi
    at any A: the phase is taken from the minimum-image displacement, which
    a shift carrying points across the box edge leaves unchanged."""
    n, h = (6, 5, 7), 0.55
    L = np.array(n) * h
    s = np.array([4, -3, 5])
    base = _gauge_domain(n=n, h=h)
    moved = np.mod(base.atoms + s * h, L)
    dom1 = _gauge_domain(n=n, h=h, atoms=moved)
    psi = _rand_psi(base.n_grid, 3, 3)
    A = np.array([0.31, -0.22, 0.17])

    def shift(a):
        return np.roll(a.reshape(n[2], n[1], n[0], -1), (s[2], s[1], s[0]), axis=(0, 1, 2)).reshape(base.n_grid, -1)

    out0 = shift(base.apply_vnl(psi, A))
    out1 = dom1.apply_vnl(shift(psi), A)
    assert np.max(np.abs(out1 - out0)) < 1e-12 * np.max(np.abs(out0))


@pytest.mark.parametrize("order", [2, 4])
def test_gauge_hamiltonian_hermitian(order):
    dom = _gauge_domain(order=order, n=(5, 4, 6), h=0.6)
    H = dom.dense_h(np.array([0.3, -0.15, 0.2]))
    assert np.max(np.abs(H - H.conj().T)) < 1e-13 * np.max(np.abs(H))


@pytest.mark.parametrize("order", [2, 4])
def test_gauge_current_is_derivative_of_energy(order):
    """With velocity-gauge projectors E(A) is no longer quadratic in A; the
    fourth-order central difference of E must match the current, which now
    carries the nonlocal commutator part."""
    dom = _gauge_domain(order=order)
    psi = _rand_psi(dom.n_grid, 3, 9)
    f = np.array([2.0, 2.0, 1.0])
    A = np.array([0.21, -0.34, 0.16])
    J = dom.observables(psi, A, f)[2:]
    J_loc = _gauge_domain(order=order, gauge=False).observables(psi, A, f)[2:]
    assert np.max(np.abs(J - J_loc)) > 1e-3 * np.max(np.abs(J))      # the nonlocal part is there
    eps = 2e-3
    for ax in range(3):
        e = np.zeros(3)
        e[ax] = eps
        E = [dom.observables(psi, A + k * e, f)[1] for k in (-2, -1, 1, 2)]
        dE = (E[0] - 8 * E[1] + 8 * E[2] - E[3]) / (12 * eps)
        assert abs(dE - J[ax]) < 1e-9 * max(1.0, abs(J[ax]))


# ---------------------------------------------------------------------------
# re-orthonormalisation and the loss
# ---------------------------------------------------------------------------

def test_reorth_cholesky_and_loewdin():
    ng, no, dV = 300, 6, 0.064
    psi = _rand_psi(ng, no, 21)
    q = oracle.reorth(psi, dV, "chol")
    np.testing.assert_allclose(dV * q.conj().T @ q, np.eye(no), atol=1e-13)
    # Gram-Schmidt order: q_m lies in span(psi_0..psi_m), q_0 parallel to psi_0
    for m in range(no):
        coef, *_ = np.linalg.lstsq(psi[:, :m + 1], q[:, m], rcond=None)
        assert np.linalg.norm(psi[:, :m + 1] @ coef - q[:, m]) < 1e-10
    # Loewdin: closest orthonormal set = polar factor of sqrt(dV) psi (SVD route)
    lw = oracle.reorth(psi, dV, "lowdin")
    U, s, Vh = np.linalg.svd(np.sqrt(dV) * psi, full_matrices=False)
    np.testing.assert_allclose(np.sqrt(dV) * lw, U @ Vh, atol=1e-12)
    np.testing.assert_allclose(oracle.reorth(q, dV, "lowdin"), q, atol=1e-12)


def test_loss_limits():
    ng, no, dV = 200, 4, 0.1
    psi = oracle.reorth(_rand_psi(ng, no, 2), dV)
    assert abs(oracle.loss(psi, psi, dV)) < 1e-12
    Uni = np.linalg.qr(_rand_psi(no, no, 5))[0]
    assert abs(oracle.loss(psi, psi @ Uni, dV)) < 1e-12
    full = oracle.reorth(_rand_psi(ng, 2 * no, 3), dV)
    assert abs(oracle.loss(full[:, :no], full[:, no:], dV) - 2 * no) < 1e-12


# ---------------------------------------------------------------------------
# split form (Eq. 2) against dense matrices
# ---------------------------------------------------------------------------

def test_split_step_dense():
    dom = _tiny_domain(order=4, n_orb=2)
    dloc = oracle.Domain(dom.n, dom.h, 2, 4, dom.V)
    A = np.array([0.0, 0.05, 0.02])
    dt = 0.05
    Hl = dloc.dense_h(A)
    Vn = dom.dense_h(A) - Hl
    lam, U = np.linalg.eigh(Hl)
    T = U @ np.diag(_g(dt * lam)) @ U.conj().T
    psi = _rand_psi(dom.n_grid, 2, 8)

    def nnl(p):
        q = p - 0.5j * dt * (Vn @ p)
        return q * (np.linalg.norm(p, axis=0) / np.linalg.norm(q, axis=0))[None, :]

    ref = nnl(T @ nnl(psi))
    np.testing.assert_allclose(dom.split_step(psi, A, dt), ref, atol=1e-13, rtol=0)
    # without projectors the split step is the plain local Taylor step
    np.testing.assert_allclose(dloc.split_step(psi, A, dt), T @ psi, atol=1e-13, rtol=0)


# ---------------------------------------------------------------------------
# adjoint: finite differences and the dot-product identity
# ---------------------------------------------------------------------------

def test_adjoint_against_central_differences():
    dom = _tiny_domain(order=4, n=(4, 4, 5), h=0.7, n_orb=2, seed=3)
    rng = np.random.default_rng(0)
    psi0 = oracle.reorth(_rand_psi(dom.n_grid, 2, 6), dom.dV)
    nsteps, dt = 9, 0.05
    A = rng.uniform(-0.05, 0.05, (nsteps, 3))
    L, dA, dVg = oracle.adjoint(dom, psi0, psi0, A, dt, ckpt_every=4)

    def run(Am, dm):
        p = psi0
        for k in range(nsteps):
            p = dm.taylor4(p, Am[k], dt)
        return oracle.loss(psi0, p, dom.dV)

    assert abs(L - run(A, dom)) < 1e-12
    eps = 1e-4
    for (k, ax) in [(0, 0), (4, 2), (8, 1), (3, 1)]:
        Ap, Am = A.copy(), A.copy()
        Ap[k, ax] += eps
        Am[k, ax] -= eps
        fd = (run(Ap, dom) - run(Am, dom)) / (2 * eps)
        assert abs(fd - dA[k, ax]) <= 1e-4 * max(abs(fd), 1e-6), (k, ax, fd, dA[k, ax])
    for g in [0, 17, 55]:
        Vp, Vm = dom.V.copy(), dom.V.copy()
        Vp[g] += eps
        Vm[g] -= eps
        dp = oracle.Domain(dom.n, dom.h, 2, 4, Vp, dom.atoms, 4, 0.7, 1.3, dom.D)
        dm = oracle.Domain(dom.n, dom.h, 2, 4, Vm, dom.atoms, 4, 0.7, 1.3, dom.D)
        fd = (run(A, dp) - run(A, dm)) / (2 * eps)
        assert abs(fd - dVg[g]) <= 1e-4 * max(abs(fd), 1e-6), (g, fd, dVg[g])


def test_adjoint_dot_product_identity():
    dom = _tiny_domain(order=2, n_orb=2)
    A = np.array([0.01, 0.03, -0.02])
    x = _rand_psi(dom.n_grid, 2, 1)
    y = _rand_psi(dom.n_grid, 2, 2)
    lhs = np.vdot(dom.taylor4_adjoint(y, A, 0.03), x)
    rhs = np.vdot(y, dom.taylor4(x, A, 0.03))
    assert abs(lhs - rhs) < 1e-13 * abs(lhs)


def test_ks_correction_closed_forms():
    """Eq. 5 pinned without retyping it: with Psi(0) orthonormal in the dV
    metric and Psi(t) = Psi(0) A + Q B, Q orthogonal to span Psi(0), the
    correction must give (1 - delta) Psi(0) A + Q B for general complex A, B
    (a transposed or conjugated overlap, a missing dV or a wrong sign of
    delta all break it); delta = 0 is the identity."""
    rng = np.random.default_rng(11)
    ng, no, dV = 300, 7, 0.064
    # an orthonormal basis of 12 columns: the first 7 span Psi(0), 5 span Q
    Z = rng.standard_normal((ng, 12)) + 1j * rng.standard_normal((ng, 12))
    Qf, _ = np.linalg.qr(Z)
    basis = Qf / np.sqrt(dV)
    psi0, Q = basis[:, :no], basis[:, no:]
    A = rng.standard_normal((no, no)) + 1j * rng.standard_normal((no, no))
    B = rng.standard_normal((5, no)) + 1j * rng.standard_normal((5, no))
    psit = psi0 @ A + Q @ B
    delta = 0.03 - 0.017j
    out = oracle.ks_correction(psit, psi0, delta, dV)
    np.testing.assert_allclose(out, (1 - delta) * (psi0 @ A) + Q @ B, rtol=0, atol=1e-12 * np.abs(psit).max())
    np.testing.assert_allclose(oracle.ks_correction(psit, psi0, 0.0, dV), psit, rtol=0, atol=0)
    # Psi(t) = Psi(0): every orbital scales by 1 - delta
    np.testing.assert_allclose(oracle.ks_correction(psi0, psi0, delta, dV), (1 - delta) * psi0, rtol=0,
                               atol=1e-12 * np.abs(psi0).max())


def test_occupations_closed_forms():
    """Shadow-dynamics occupations pinned by construction: with Psi(0)
    orthonormal in the dV metric, Psi(t) = cos(t) Psi(0) U + sin(t) Q W (U, W
    unitary, Q orthonormal and orthogonal to span Psi(0)) gives
    f_s(t) = cos^2(t) sum_n f_n |U_sn|^2 and n_exc = sin^2(t) sum_n f_n, for
    unequal occupations and a non-symmetric U (so a transposed overlap, a
    missing dV or a wrong sign of n_exc break it).  Diagonal phases keep
    every occupation; a state orthogonal to the reference has none."""
    rng = np.random.default_rng(12)
    ng, no, dV = 320, 6, 0.064
    Z = rng.standard_normal((ng, 2 * no)) + 1j * rng.standard_normal((ng, 2 * no))
    Qf, _ = np.linalg.qr(Z)
    basis = Qf / np.sqrt(dV)
    psi0, Q = basis[:, :no], basis[:, no:]

    def unitary():
        M = rng.standard_normal((no, no)) + 1j * rng.standard_normal((no, no))
        q, r = np.linalg.qr(M)
        return q * (np.diag(r) / np.abs(np.diag(r)))

    U, W = unitary(), unitary()
    assert np.abs(np.abs(U) - np.abs(U).T).max() > 0.1
    f = rng.uniform(0.2, 2.0, no)
    t = 0.37
    psit = np.cos(t) * (psi0 @ U) + np.sin(t) * (Q @ W)
    f_s, n_exc = oracle.occupations(psi0, psit, f, dV)
    np.testing.assert_allclose(f_s, np.cos(t) ** 2 * (np.abs(U) ** 2 @ f), rtol=1e-12, atol=1e-13)
    assert abs(n_exc - np.sin(t) ** 2 * f.sum()) < 1e-12 * f.sum()
    phases = np.exp(1j * rng.uniform(0, 2 * np.pi, no))
    f_s, n_exc = oracle.occupations(psi0, psi0 * phases, f, dV)
    np.testing.assert_allclose(f_s, f, rtol=1e-12)
    assert abs(n_exc) < 1e-12 * f.sum()
    f_s, n_exc = oracle.occupations(psi0, Q @ W, f, dV)
    assert np.abs(f_s).max() < 1e-12 and abs(n_exc - f.sum()) < 1e-12 * f.sum()
    # with f_n = 2 the count is the loss of Sec. V.A.8 (2 (N_o - sum |C|^2))
    _, n2 = oracle.occupations(psi0, psit, np.full(no, 2.0), dV)
    assert abs(n2 - oracle.loss(psi0, psit, dV)) < 1e-12 * no
