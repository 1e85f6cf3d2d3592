"""The tensor-core nonlocal path against the FP64 oracle.

Domains whose projector spheres cover each grid point many times over
(about 41 times in the batched workload) apply the nonlocal term as dense
brick GEMMs on tcgen05 with BF16x3 split operands: a scatter GEMM added to
the local stage output and a projection GEMM of that output.  Here the path
is forced (MLMD_NL_TC=1) on small domains whose grids cut the 8 x 4 x 4
bricks raggedly in every axis, with 4 and 8 projectors per atom and orbital
rows that take one or two MMAs per K-step, and chosen automatically on a
domain of the batched workload's density; every case is compared with the
oracle after several full-scheme steps, and the profiling hooks confirm
which kernels ran.
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


def _run(spec, psi):
    from paper_2509_00966_gb300 import mlmd
    d, V = gpu_domain(spec)
    d.set_orbitals(to_device(psi, "c64"))
    mlmd.profile_enable(d.handle, True)
    obs = d.propagate(spec.A)
    n_scatter = mlmd.profile_read(d.handle, "scatter")[1]
    mlmd.profile_enable(d.handle, False)
    out = to_numpy(d.get_orbitals())
    d.close()
    od = oracle_domain(spec, V)
    ref, robs = oracle.propagate(od, psi, spec.A, spec.dt, np.full(spec.n_orb, 2.0))
    return out, obs, ref, robs, n_scatter


def _check(out, obs, ref, robs, tag):
    err = np.max(np.abs(out - ref))
    e_n = np.max(np.abs(obs[:, 0] - robs[:, 0]) / np.abs(robs[:, 0]))
    e_E = np.max(np.abs(obs[:, 1] - robs[:, 1]) / np.abs(robs[:, 1]))
    scale = max(np.abs(robs[:, 2:]).max(), np.abs(robs[:, 0]).max())
    e_J = np.max(np.abs(obs[:, 2:] - robs[:, 2:])) / scale
    print(f"\n[errors] {tag}: psi={err:.3e} norm={e_n:.3e} energy={e_E:.3e} current={e_J:.3e}", flush=True)
    assert err <= 1e-5
    assert e_n <= 1e-6 and e_E <= 1e-6 and e_J <= 1e-6


@pytest.mark.parametrize("n,n_orb,n_proj,order,n_atoms", [
    ((10, 9, 11), 20, 4, 4, 30),     # ragged bricks on every axis; 48 orbital columns
    ((16, 8, 12), 37, 8, 4, 16),     # 8 projectors per atom; 80 columns
    ((12, 12, 9), 100, 4, 2, 40),    # 2nd order; 208 columns in one MMA
    ((9, 8, 8), 150, 4, 4, 24),      # 304 columns in two MMAs per K-step
])
def test_tensor_nonlocal_forced(n, n_orb, n_proj, order, n_atoms, monkeypatch):
    monkeypatch.setenv("MLMD_NL_TC", "1")
    spec = small_spec(precision="c64", n=n, n_orb=n_orb, fd_order=order, n_proj=n_proj, n_atoms=n_atoms,
                      r_cut=2.2, steps=6)
    out, obs, ref, robs, n_scatter = _run(spec, orbitals(spec))
    assert n_scatter == 4 * spec.n_steps          # the tensor path ran: one scatter GEMM per Taylor stage
    _check(out, obs, ref, robs, f"tensor nonlocal {n} x {n_orb}, {n_atoms}x{n_proj}")


def test_tensor_nonlocal_chosen_at_batched_density():
    """A domain of the batched workload's kind (N = 26, h = 0.35,
    round(N^3/64) atoms x 4 projectors, r_cut = 3: about 41 spheres over
    every point) takes the tensor path without being told to."""
    spec = inputs.batched_specs(n_domains=2, n_steps=3, seed=11)[1]
    assert spec.n == (26, 26, 26)
    psi = inputs.random_orbitals(spec.n_grid, spec.n_orb, spec.dV, 77)
    out, obs, ref, robs, n_scatter = _run(spec, psi)
    assert n_scatter == 4 * spec.n_steps
    _check(out, obs, ref, robs, f"tensor nonlocal c3 domain N=26 x {spec.n_orb}")


def test_tensor_nonlocal_off_matches_on(monkeypatch):
    """The same dense domain with the path switched off (per-point SIMT
    scatter and projection) gives the same orbitals within the FP32 bound."""
    spec = small_spec(precision="c64", n=(10, 9, 11), n_orb=20, n_proj=4, n_atoms=30, r_cut=2.2, steps=4)
    psi = orbitals(spec)
    monkeypatch.setenv("MLMD_NL_TC", "1")
    on, _, ref, _, n_on = _run(spec, psi)
    monkeypatch.setenv("MLMD_NL_TC", "0")
    off, _, _, _, n_off = _run(spec, psi)
    assert n_on > 0 and n_off == 0
    assert np.max(np.abs(on - off)) <= 1e-5 and np.max(np.abs(off - ref)) <= 1e-5


def test_prebuilt_tiles_match_generated(monkeypatch):
    """The projector tiles built once per projector set are the bytes the
    kernels would generate in every launch: orbitals and observables agree
    with the images on and off to the rounding of the projection's
    atomic accumulation (whose order varies from run to run)."""
    spec = small_spec(precision="c64", n=(16, 8, 12), n_orb=37, n_proj=8, n_atoms=16, r_cut=2.2, steps=4)
    psi = orbitals(spec)
    monkeypatch.setenv("MLMD_NL_TC", "1")
    a, oa, _, _, na_ = _run(spec, psi)
    monkeypatch.setenv("MLMD_NL_TILES", "0")
    b, ob, _, _, nb_ = _run(spec, psi)
    assert na_ == nb_ == 4 * spec.n_steps
    d_psi = np.max(np.abs(a - b))
    d_obs = np.max(np.abs(oa - ob)) / np.max(np.abs(ob))
    print(f"\n[errors] tiles on/off: psi={d_psi:.3e} obs={d_obs:.3e}", flush=True)
    assert d_psi <= 1e-6 and d_obs <= 1e-6
