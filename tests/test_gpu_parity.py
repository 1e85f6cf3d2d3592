"""CUDA path (through the C ABI) against the FP64 oracle, element by element
on the same seeded inputs.

Tolerances:
* complex128 domains: max |psi - psi_ref| <= 1e-12 (same arithmetic up to
  summation order), observables relative 1e-11;
* complex64 domains (FP32 stencil arithmetic, FP64 reductions): max
  |psi - psi_ref| <= 1e-5 absolute with <psi|psi> = 1, electron count and
  energy relative 1e-6, current within 1e-6 of max(|J|, N_e);
* neighbour lists and index maps: identical.
"""
import numpy as np
import pytest

import oracle
from _helpers import gpu_domain, oracle_domain, orbitals, small_spec, to_device, to_numpy
from paper_2509_00966_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    from paper_2509_00966_gb300 import build
    build.build()
    torch.cuda.init()


def _run_both(spec, steps=None, scheme="full", ortho_every=0, psi=None):
    steps = steps or spec.n_steps
    d, V = gpu_domain(spec, scheme=scheme, ortho_every=ortho_every)
    od = oracle_domain(spec, V)
    psi = orbitals(spec) if psi is None else psi
    d.set_orbitals(to_device(psi, spec.precision))
    obs = d.propagate(spec.A[:steps])
    out = to_numpy(d.get_orbitals())
    ref, robs = oracle.propagate(od, psi, spec.A[:steps], spec.dt, np.full(spec.n_orb, 2.0), scheme=scheme,
                                 ortho_every=ortho_every)
    d.close()
    return out, obs, ref, robs


def _check_obs(obs, robs, rel):
    np.testing.assert_allclose(obs[:, 0], robs[:, 0], rtol=rel, atol=0)
    np.testing.assert_allclose(obs[:, 1], robs[:, 1], rtol=rel, atol=rel * np.abs(robs[:, 0]).max())
    scale = np.maximum(np.abs(robs[:, 2:]).max(), np.abs(robs[:, 0]).max())
    assert np.max(np.abs(obs[:, 2:] - robs[:, 2:])) <= rel * scale


def test_c0_complex128_100_steps():
    spec = inputs.config("c0")
    out, obs, ref, robs = _run_both(spec)
    assert np.max(np.abs(out - ref)) <= 1e-12
    _check_obs(obs, robs, 1e-11)


@pytest.mark.parametrize("order", [2, 4])
def test_full_scheme_complex128_all_terms(order):
    spec = small_spec(precision="c128", fd_order=order, steps=12)
    out, obs, ref, robs = _run_both(spec)
    assert np.max(np.abs(out - ref)) <= 1e-12
    _check_obs(obs, robs, 1e-11)


def test_full_scheme_complex64_all_terms():
    spec = small_spec(precision="c64", steps=100, n=(10, 12, 9), n_orb=13)
    out, obs, ref, robs = _run_both(spec)
    assert np.max(np.abs(out - ref)) <= 1e-5
    _check_obs(obs, robs, 1e-6)


@pytest.mark.parametrize("precision,n,n_orb,order", [
    ("c64", (16, 8, 12), 32, 4),     # TMA path, 128-byte orbital chunks
    ("c64", (8, 16, 5), 20, 4),      # TMA path, 64-byte chunks, short z
    ("c64", (16, 16, 9), 13, 2),     # TMA path, 2nd order, ragged orbital count
    ("c128", (8, 8, 11), 12, 4),     # TMA path, complex128
])
def test_tma_stage_path(precision, n, n_orb, order):
    """Grids whose x and y extents tile by 8 run the TMA-staged stage kernel;
    the same case with MLMD_NO_TMA set runs the plain kernel.  Both match the
    oracle."""
    import os
    spec = small_spec(precision=precision, n=n, n_orb=n_orb, fd_order=order, steps=12, n_atoms=5)
    tol = 1e-12 if precision == "c128" else 1e-5
    out, obs, ref, robs = _run_both(spec)
    assert np.max(np.abs(out - ref)) <= tol
    _check_obs(obs, robs, 1e-11 if precision == "c128" else 1e-6)
    os.environ["MLMD_NO_TMA"] = "1"
    try:
        out2, obs2, _, _ = _run_both(spec)
    finally:
        del os.environ["MLMD_NO_TMA"]
    assert np.max(np.abs(out2 - ref)) <= tol
    assert np.max(np.abs(out2 - out)) <= tol


@pytest.mark.parametrize("tile,precision,n_proj,order", [
    ("8,4", "c64", 4, 4), ("8,8", "c64", 4, 4), ("4,4", "c64", 4, 4),
    ("8,4", "c64", 8, 2), ("8,8", "c64", 8, 4), ("4,4", "c64", 8, 4),
    ("8,4", "c128", 4, 4), ("8,8", "c128", 8, 2),
])
def test_stage_tile_shapes(tile, precision, n_proj, order, monkeypatch):
    """Every tile shape of the TMA stage kernel (orbital chunk of 8 or 4
    16-byte vectors; 4 or 8 threads per grid point), fixed through
    MLMD_STAGE_TILE instead of the timing autotuner, on a grid with several
    tiles, z ranges and projection columns (the projection of the output is
    a separate kernel), against the oracle."""
    monkeypatch.setenv("MLMD_STAGE_TILE", tile)
    spec = small_spec(precision=precision, n=(16, 16, 20), n_orb=48, fd_order=order, steps=8, n_atoms=7,
                      n_proj=n_proj, r_cut=2.6)
    tol = 1e-12 if precision == "c128" else 1e-5
    out, obs, ref, robs = _run_both(spec)
    assert np.max(np.abs(out - ref)) <= tol
    _check_obs(obs, robs, 1e-11 if precision == "c128" else 1e-6)


def test_projector_lists_bit_exact():
    for spec in [small_spec(n_atoms=9, r_cut=1.7), inputs.config("c1", n_orb=8, n_steps=1),
                 inputs.config("c2", n_orb=8, n_steps=1), inputs.config("c4", n_orb=8, n_steps=1)]:
        d, V = gpu_domain(spec)
        od = oracle_domain(spec, V)
        off, idx, beta = d.projector_lists()
        np.testing.assert_array_equal(off, od.off)
        np.testing.assert_array_equal(idx, od.idx)
        np.testing.assert_allclose(beta, od.beta, rtol=0, atol=1e-13 * np.abs(od.beta).max())
        d.close()


def test_projector_lists_exact_tie():
    """Points exactly at r_cut belong to the sphere on both sides: h = 0.5,
    r_cut = 1.5 and atoms on grid points make d^2 = r_cut^2 exact in binary
    for 30 offsets per atom; the device lists equal the oracle's."""
    from paper_2509_00966_gb300 import mlmd
    n, h = (16, 16, 16), 0.5
    pos = np.array([[2.0, 2.5, 3.0], [0.0, 0.0, 0.0], [7.5, 7.5, 7.5]])
    D = np.ones((3, 4))
    d = mlmd.Domain(n, h, 4, 4, "c128", dt=0.02)
    d.set_projectors(pos, 4, 0.9, 1.5, D)
    off, idx, beta = d.projector_lists()
    V = np.zeros(int(np.prod(n)))
    od = oracle.Domain(n, h, 4, 4, V, pos, 4, 0.9, 1.5, D)
    np.testing.assert_array_equal(off, od.off)
    np.testing.assert_array_equal(idx, od.idx)
    assert all(off[a + 1] - off[a] == 123 for a in range(3))   # |m|^2 <= 9: 123 offsets
    d.close()


def test_projector_edge_cases():
    # an atom whose sphere holds no grid point, atoms far outside the box, 8 shapes
    spec = small_spec(n_atoms=3, n_proj=8, r_cut=1.5, precision="c128", steps=3)
    spec.atoms[0] = [0.2, 0.2, 0.2]
    spec.atoms[1] = [-37.3, 51.9, 1e3 + 0.1]
    d, V = gpu_domain(spec)
    d.set_projectors(np.vstack([spec.atoms, [[0.2, 0.2, 0.2]]]), 8, spec.r_c, 0.05,
                     np.vstack([spec.D, np.ones((1, 8))]))
    off, idx, beta = d.projector_lists()
    assert off[-1] - off[-2] == 0   # r_cut 0.05 around an off-grid point: empty list
    od = oracle.Domain(spec.n, spec.h, spec.n_orb, spec.fd_order, V, np.vstack([spec.atoms, [[0.2, 0.2, 0.2]]]),
                       8, spec.r_c, 0.05, np.vstack([spec.D, np.ones((1, 8))]))
    np.testing.assert_array_equal(off, od.off)
    np.testing.assert_array_equal(idx, od.idx)
    psi = orbitals(spec)
    d.set_orbitals(to_device(psi, "c128"))
    d.propagate(spec.A)
    ref, _ = oracle.propagate(od, psi, spec.A, spec.dt, np.full(spec.n_orb, 2.0))
    assert np.max(np.abs(to_numpy(d.get_orbitals()) - ref)) <= 1e-12
    d.close()


@pytest.mark.parametrize("precision,tol", [("c128", 1e-12), ("c64", 1e-5)])
def test_density_current(precision, tol):
    spec = small_spec(precision=precision)
    d, V = gpu_domain(spec)
    od = oracle_domain(spec, V)
    psi = orbitals(spec)
    d.set_orbitals(to_device(psi, precision))
    A = np.array([0.05, -0.02, 0.11])
    rho, j, J = d.density_current(A)
    rr, jr, Jr = od.density_current(psi, A, np.full(spec.n_orb, 2.0))
    rho = rho.cpu().numpy()
    j = j.cpu().numpy()
    assert np.max(np.abs(rho - rr)) <= tol * np.abs(rr).max()
    assert np.max(np.abs(j - jr)) <= tol * np.abs(jr).max()
    assert np.max(np.abs(J - Jr)) <= tol * max(np.abs(Jr).max(), 1.0)
    # host outputs
    rho_h, j_h, J_h = d.density_current(A, device=False)
    np.testing.assert_array_equal(rho_h.numpy(), rho)
    d.close()


@pytest.mark.parametrize("precision,tol", [("c128", 1e-12), ("c64", 2e-6)])
def test_overlap_reorth_excitation(precision, tol):
    spec = small_spec(precision=precision, n_orb=19)
    d, V = gpu_domain(spec)
    rng = np.random.default_rng(4)
    psi = rng.standard_normal((spec.n_grid, spec.n_orb)) + 1j * rng.standard_normal((spec.n_grid, spec.n_orb))
    psi *= 1.0 / np.sqrt(spec.dV * spec.n_grid)
    d.set_orbitals(to_device(psi, precision))
    S = d.overlap()
    Sr = oracle.overlap(psi, psi, spec.dV)
    assert np.max(np.abs(S - Sr)) <= tol * np.abs(Sr).max()
    for kind in ["chol", "lowdin"]:
        d.set_orbitals(to_device(psi, precision))
        d.reorthonormalize(kind)
        q = to_numpy(d.get_orbitals())
        qr = oracle.reorth(psi, spec.dV, kind)
        assert np.max(np.abs(q - qr)) <= 50 * tol * np.abs(qr).max(), kind
        assert np.max(np.abs(spec.dV * q.conj().T @ q - np.eye(spec.n_orb))) <= 50 * tol
    # excitation of the re-orthonormalised set against the raw set
    d.set_orbitals(to_device(qr, precision))
    assert abs(d.excitation()) <= 100 * tol * spec.n_orb
    d.close()


def test_reorth_every_k_steps_c128():
    spec = small_spec(precision="c128", steps=10)
    out, obs, ref, robs = _run_both(spec, ortho_every=3)
    assert np.max(np.abs(out - ref)) <= 1e-12
    _check_obs(obs, robs, 1e-11)


@pytest.mark.parametrize("precision,tol", [("c128", 1e-12), ("c64", 1e-5)])
def test_split_scheme(precision, tol):
    spec = small_spec(precision=precision, steps=8)
    out, obs, ref, robs = _run_both(spec, scheme="split")
    assert np.max(np.abs(out - ref)) <= tol
    _check_obs(obs, robs, 1e-6 if precision == "c64" else 1e-11)


@pytest.mark.parametrize("precision", ["c128", "c64"])
def test_adjoint_against_oracle(precision):
    spec = small_spec(precision=precision, n=(8, 9, 10), n_orb=6, steps=14, n_atoms=4)
    d, V = gpu_domain(spec)
    od = oracle_domain(spec, V)
    psi = orbitals(spec)
    d.set_orbitals(to_device(psi, precision))
    loss, dA, dV_ = d.propagate_adjoint(spec.A, ckpt_every=4)
    Lr, dAr, dVr = oracle.adjoint(od, psi, psi, spec.A, spec.dt, ckpt_every=4)
    if precision == "c128":
        assert abs(loss - Lr) <= 1e-10 * max(1.0, abs(Lr))
        assert np.max(np.abs(dA - dAr)) <= 1e-9 * np.abs(dAr).max()
        assert np.max(np.abs(dV_ - dVr)) <= 1e-9 * np.abs(dVr).max()
    else:
        assert abs(loss - Lr) <= 1e-4 * max(1.0, abs(Lr))
        assert np.linalg.norm(dA - dAr) <= 1e-3 * np.linalg.norm(dAr)
        assert np.linalg.norm(dV_ - dVr) <= 1e-3 * np.linalg.norm(dVr)
    # the orbitals are left at Psi(T)
    ref = psi
    for k in range(spec.n_steps):
        ref = od.taylor4(ref, spec.A[k], spec.dt)
    assert np.max(np.abs(to_numpy(d.get_orbitals()) - ref)) <= (1e-12 if precision == "c128" else 1e-5)
    d.close()


def test_adjoint_as_autograd_function():
    """The adjoint behind torch.autograd: from the same start, backward of
    excitation_loss leaves the direct mlmd_propagate_adjoint's dL/dV in V's
    gradient, and the chain rule through A = s A0 gives dL/ds = sum dL/dA A0."""
    import torch
    spec = small_spec(precision="c128", n=(8, 9, 10), n_orb=6, steps=10, n_atoms=4)
    d, V = gpu_domain(spec)
    psi = orbitals(spec)
    d.set_orbitals(to_device(psi, "c128"))
    loss0, dA0, dV0 = d.propagate_adjoint(spec.A, ckpt_every=4)
    d.set_orbitals(to_device(psi, "c128"))
    s = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    Vt = torch.from_numpy(np.ascontiguousarray(V)).cuda().requires_grad_(True)
    loss = d.excitation_loss(s * torch.from_numpy(spec.A), Vt, ckpt_every=4)
    loss.backward()
    assert abs(loss.item() - loss0) <= 1e-12 * max(1.0, abs(loss0))
    np.testing.assert_allclose(Vt.grad.cpu().numpy(), dV0, rtol=1e-12, atol=1e-14 * np.abs(dV0).max())
    ds = float(np.sum(dA0 * spec.A))
    assert abs(s.grad.item() - ds) <= 1e-10 * max(1.0, abs(ds))
    d.close()


def test_batch_matches_single_domains_and_oracle():
    specs = [small_spec(n=(10, 10, 10), n_orb=7, seed=1, steps=6), small_spec(n=(12, 9, 11), n_orb=16, seed=2, steps=6),
             small_spec(n=(8, 8, 12), n_orb=3, seed=3, steps=6, n_atoms=2)]
    from paper_2509_00966_gb300 import mlmd
    doms, refs = [], []
    for s in specs:
        d, V = gpu_domain(s)
        psi = orbitals(s)
        d.set_orbitals(to_device(psi, s.precision))
        doms.append(d)
        od = oracle_domain(s, V)
        refs.append(oracle.propagate(od, psi, s.A, s.dt, np.full(s.n_orb, 2.0)))
    b = mlmd.batch_create([d.handle for d in doms])
    A = np.stack([s.A for s in specs])
    obs = mlmd.batch_propagate(b, A, first_handle=doms[0].handle)
    for i, d in enumerate(doms):
        assert np.max(np.abs(to_numpy(d.get_orbitals()) - refs[i][0])) <= 1e-5
        _check_obs(obs[i], refs[i][1], 1e-6)
    mlmd.batch_destroy(b)
    for d in doms:
        d.close()


def test_batch_groups_of_plain_domains():
    """Plain-path domains of a batch run as persistent launches per group of
    equal FD order and projector count; a batch mixing 2nd/4th order, 4 and 8
    projectors per atom, a domain without projectors and a TMA-path domain
    matches the oracle domain by domain."""
    specs = [small_spec(n=(10, 10, 10), n_orb=7, seed=1, steps=5),
             small_spec(n=(12, 9, 11), n_orb=16, seed=2, steps=5, fd_order=2),
             small_spec(n=(9, 10, 11), n_orb=9, seed=4, steps=5, n_proj=8, n_atoms=3),
             small_spec(n=(10, 9, 8), n_orb=5, seed=5, steps=5, n_proj=0),
             small_spec(n=(11, 10, 9), n_orb=12, seed=6, steps=5, n_atoms=4),
             small_spec(n=(8, 8, 12), n_orb=3, seed=3, steps=5, n_atoms=2)]
    from paper_2509_00966_gb300 import mlmd
    doms, refs = [], []
    for s in specs:
        d, V = gpu_domain(s)
        psi = orbitals(s)
        d.set_orbitals(to_device(psi, s.precision))
        doms.append(d)
        od = oracle_domain(s, V)
        refs.append(oracle.propagate(od, psi, s.A, s.dt, np.full(s.n_orb, 2.0)))
    b = mlmd.batch_create([d.handle for d in doms])
    A = np.stack([s.A for s in specs])
    obs = mlmd.batch_propagate(b, A, first_handle=doms[0].handle)
    for i, d in enumerate(doms):
        assert np.max(np.abs(to_numpy(d.get_orbitals()) - refs[i][0])) <= 1e-5, i
        _check_obs(obs[i], refs[i][1], 1e-6)
    mlmd.batch_destroy(b)
    for d in doms:
        d.close()


def test_c1_full_size_sampled_orbitals():
    """The benchmark workload (48^3 grid, 256 complex64 orbitals, 64 atoms x 4
    projectors, pulse) for 100 steps in the benchmark's launch configuration;
    orbitals evolve independently, so the oracle runs a sample of them."""
    spec = inputs.config("c1", n_steps=100)
    d, V = gpu_domain(spec)
    psi = orbitals(spec)
    d.set_orbitals(to_device(psi, "c64"))
    d.propagate(spec.A, obs=False)
    out = to_numpy(d.get_orbitals())
    sample = [0, 77, 200, 255]
    od = oracle_domain(spec, V, n_orb=len(sample))
    ref, _ = oracle.propagate(od, psi[:, sample], spec.A, spec.dt, np.full(len(sample), 2.0))
    assert np.max(np.abs(out[:, sample] - ref)) <= 1e-5
    d.close()


def test_c2_full_size_sampled_orbitals_and_reorth():
    """The precision-form workload at full size (64^3 grid, 1024 complex64
    orbitals, 128 atoms x 8 projectors, BF16X3 GEMMs, re-orthonormalisation
    every 10 steps).  For 9 steps no re-orthonormalisation couples the
    orbitals, so the oracle runs a sample of them; then one BF16X3 Cholesky
    re-orthonormalisation of all 1024, whose result must be orthonormal as
    an independent FP32 SIMT overlap measures it.  The orbitals are seeded
    random vectors made on the device, each normalised."""
    import torch
    from paper_2509_00966_gb300 import mlmd
    spec = inputs.config("c2", n_steps=9)
    d, V = gpu_domain(spec, gemm_mode="bf16x3", ortho_every=10)
    g = torch.Generator(device="cuda").manual_seed(2)
    re = torch.randn(spec.n_grid, spec.n_orb, generator=g, device="cuda")
    im = torch.randn(spec.n_grid, spec.n_orb, generator=g, device="cuda")
    psi = torch.complex(re, im)
    del re, im
    psi = (psi / torch.sqrt(spec.dV * (psi.abs() ** 2).sum(0, keepdim=True))).contiguous()
    sample = [0, 333, 700, 1023]
    p0 = psi[:, sample].cpu().numpy().astype(np.complex128)
    d.set_orbitals(psi)
    del psi
    d.propagate(spec.A, obs=False)
    out = d.get_orbitals()[:, sample].cpu().numpy().astype(np.complex128)
    od = oracle_domain(spec, V, n_orb=len(sample))
    ref, _ = oracle.propagate(od, p0, spec.A, spec.dt, np.full(len(sample), 2.0))
    assert np.max(np.abs(out - ref)) <= 1e-5, np.max(np.abs(out - ref))
    d.reorthonormalize("chol")
    q = d.get_orbitals()
    d.close()
    d32 = mlmd.Domain(spec.n, spec.h, spec.n_orb, spec.fd_order, "c64", gemm_mode="fp32", dt=spec.dt)
    d32.set_orbitals(q)
    del q
    S = d32.overlap()
    d32.close()
    err = np.abs(S - np.eye(spec.n_orb))
    assert err.max() <= 2e-5 and abs(np.real(np.diag(S)).mean() - 1.0) <= 1e-5, (err.max(), np.diag(S).mean())


def test_zero_steps_and_single_orbital():
    spec = small_spec(precision="c128", n_orb=1, steps=4)
    out, obs, ref, robs = _run_both(spec)
    assert np.max(np.abs(out - ref)) <= 1e-12
    d, V = gpu_domain(spec)
    psi = orbitals(spec)
    d.set_orbitals(to_device(psi, "c128"))
    n0 = d.launches
    d.propagate(np.zeros((0, 3)))
    assert d.launches == n0
    assert np.array_equal(to_numpy(d.get_orbitals()), psi)
    d.close()


def test_invalid_calls_return_status():
    from paper_2509_00966_gb300 import mlmd
    spec = small_spec(precision="c64", steps=2)
    d, V = gpu_domain(spec)
    with pytest.raises(mlmd.MLMDError) as e:
        d.set_projectors(spec.atoms, 5, 1.0, 2.0, np.zeros((len(spec.atoms), 5)))
    assert e.value.status == 1
    with pytest.raises(mlmd.MLMDError) as e:
        d.propagate(np.array([[np.nan, 0, 0]]))
    assert e.value.status == 1
    with pytest.raises(mlmd.MLMDError) as e:
        d.excitation()     # no reference orbitals yet
    assert e.value.status == 6
    d.close()


@pytest.mark.parametrize("zc,precision,n_proj,n_atoms,r_cut", [
    (3, "c64", 4, 7, 2.6),       # many short columns, the last one ragged (20 = 6 x 3 + 2)
    (7, "c64", 8, 7, 2.6),       # odd column length, ragged last column
    (20, "c64", 8, 7, 2.6),      # one column over the whole z extent (above 16 planes)
    (32, "c128", 4, 7, 2.6),     # longer than the grid: clamped to it
    (20, "c64", 8, 40, 3.0),     # dense projectors: the tables may fall back to 16-plane columns
])
def test_stage_column_lengths(zc, precision, n_proj, n_atoms, r_cut, monkeypatch):
    """The z extent of the TMA stage kernel's columns (planes per CTA, up to
    32 where the staged projections leave room for five w slots), fixed
    through MLMD_STAGE_ZC, against the oracle: the plane ring, the entry and
    psi copies and the halo planes wrap the same way at any column length."""
    monkeypatch.setenv("MLMD_STAGE_ZC", str(zc))
    spec = small_spec(precision=precision, n=(16, 16, 20), n_orb=48, steps=6, n_atoms=n_atoms, n_proj=n_proj,
                      r_cut=r_cut)
    tol = 1e-12 if precision == "c128" else 1e-5
    out, obs, ref, robs = _run_both(spec)
    assert np.max(np.abs(out - ref)) <= tol
    _check_obs(obs, robs, 1e-11 if precision == "c128" else 1e-6)
