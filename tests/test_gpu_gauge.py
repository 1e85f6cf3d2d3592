"""Velocity-gauge projectors on the GPU against the FP64 oracle.

With the gauge switched on, every projector carries the phase
e^{-i A.(r - R_a)} of its minimum-image displacement at each step's A (Eq. 3's
minimal coupling carried onto v_nl), and the current column of the
observables adds the nonlocal commutator term from three moment projections
(Sec. V.B.5, energy and current through the nonlocal GEMMs).  Each case runs
the same seeded inputs through the C ABI and through the oracle with
``nl_gauge=True`` and compares orbitals and observables; the A values of the
test pulse put phases of up to about 0.7 rad on the sphere edges.
"""
import numpy as np
import pytest

import oracle
from _helpers import gpu_domain, oracle_domain, orbitals, small_spec, to_device, to_numpy

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    from paper_2509_00966_gb300 import build
    build.build()
    torch.cuda.init()


def _oracle_gauge(spec, V):
    return oracle.Domain(spec.n, spec.h, spec.n_orb, spec.fd_order, V, spec.atoms, spec.n_proj, spec.r_c,
                         spec.r_cut, spec.D, nl_gauge=True)


def _check_obs(obs, robs, rel):
    np.testing.assert_allclose(obs[:, 0], robs[:, 0], rtol=rel, atol=0)
    np.testing.assert_allclose(obs[:, 1], robs[:, 1], rtol=rel, atol=rel * np.abs(robs[:, 0]).max())
    scale = np.maximum(np.abs(robs[:, 2:]).max(), np.abs(robs[:, 0]).max())
    assert np.max(np.abs(obs[:, 2:] - robs[:, 2:])) <= rel * scale


def _run(spec, scheme="full"):
    d, V = gpu_domain(spec, scheme=scheme)
    d.set_nonlocal_gauge("velocity")
    psi = orbitals(spec)
    d.set_orbitals(to_device(psi, spec.precision))
    obs = d.propagate(spec.A)
    out = to_numpy(d.get_orbitals())
    d.close()
    od = _oracle_gauge(spec, V)
    ref, robs = oracle.propagate(od, psi, spec.A, spec.dt, np.full(spec.n_orb, 2.0), scheme=scheme)
    return out, obs, ref, robs, od, psi


def _tol(spec):
    return (1e-12, 1e-11) if spec.precision == "c128" else (1e-5, 1e-6)


@pytest.mark.parametrize("precision,order,n_proj,n", [
    ("c128", 4, 4, (12, 10, 14)),
    ("c128", 2, 8, (9, 11, 10)),
    ("c64", 4, 4, (12, 10, 14)),
    ("c64", 4, 8, (16, 16, 16)),      # a grid the TMA-staged kernel would take with real projectors
    ("c64", 2, 4, (10, 9, 11)),
])
def test_gauge_full_scheme(precision, order, n_proj, n):
    spec = small_spec(precision=precision, fd_order=order, n_proj=n_proj, n=n, n_atoms=5, steps=8)
    out, obs, ref, robs, od, psi = _run(spec)
    psi_tol, obs_tol = _tol(spec)
    err = np.max(np.abs(out - ref))
    # the nonlocal commutator current is a visible part of J in these runs
    J_loc = oracle.propagate(oracle_domain(spec, od.V), psi, spec.A[:1], spec.dt, np.full(spec.n_orb, 2.0))[1][0, 2:]
    print(f"\n[errors] gauge {precision} p={order} np={n_proj} {n}: psi={err:.3e} "
          f"J_nl/J={np.max(np.abs(robs[0, 2:] - J_loc)) / np.max(np.abs(robs[0, 2:])):.3e}", flush=True)
    assert np.max(np.abs(robs[0, 2:] - J_loc)) > 1e-4 * np.max(np.abs(robs[0, 2:]))
    assert err <= psi_tol
    _check_obs(obs, robs, obs_tol)


@pytest.mark.parametrize("precision", ["c128", "c64"])
def test_gauge_split_scheme(precision):
    spec = small_spec(precision=precision, n=(10, 12, 9), n_atoms=6, steps=6)
    out, obs, ref, robs, _, _ = _run(spec, scheme="split")
    psi_tol, obs_tol = _tol(spec)
    assert np.max(np.abs(out - ref)) <= psi_tol
    _check_obs(obs, robs, obs_tol)


def test_gauge_switch_back_to_real_projectors():
    """velocity -> real mid-run: the second half follows the real-projector
    oracle from the state the first half reached."""
    spec = small_spec(precision="c128", n=(10, 9, 11), n_atoms=4, steps=8)
    d, V = gpu_domain(spec)
    psi = orbitals(spec)
    d.set_orbitals(to_device(psi, "c128"))
    d.set_nonlocal_gauge("velocity")
    d.propagate(spec.A[:4])
    d.set_nonlocal_gauge("real")
    obs2 = d.propagate(spec.A[4:])
    out = to_numpy(d.get_orbitals())
    d.close()
    mid, _ = oracle.propagate(_oracle_gauge(spec, V), psi, spec.A[:4], spec.dt, np.full(spec.n_orb, 2.0))
    ref, robs2 = oracle.propagate(oracle_domain(spec, V), mid, spec.A[4:], spec.dt, np.full(spec.n_orb, 2.0))
    assert np.max(np.abs(out - ref)) <= 1e-12
    _check_obs(obs2, robs2, 1e-11)


def test_gauge_survives_new_projectors():
    """The gauge setting stays on when the projectors are replaced."""
    spec = small_spec(precision="c128", n=(10, 10, 10), n_atoms=3, steps=4)
    d, V = gpu_domain(spec)
    d.set_nonlocal_gauge("velocity")
    d.set_projectors(spec.atoms, spec.n_proj, spec.r_c, spec.r_cut, spec.D)
    psi = orbitals(spec)
    d.set_orbitals(to_device(psi, "c128"))
    obs = d.propagate(spec.A)
    out = to_numpy(d.get_orbitals())
    d.close()
    ref, robs = oracle.propagate(_oracle_gauge(spec, V), psi, spec.A, spec.dt, np.full(spec.n_orb, 2.0))
    assert np.max(np.abs(out - ref)) <= 1e-12
    _check_obs(obs, robs, 1e-11)


def test_gauge_batch():
    """Batched domains, one in the velocity gauge and one with real
    projectors, each against its own oracle."""
    from paper_2509_00966_gb300 import mlmd
    specs = [small_spec(n=(10, 10, 10), n_orb=7, seed=1, steps=5), small_spec(n=(12, 9, 11), n_orb=16, seed=2, steps=5)]
    doms, refs = [], []
    for i, s in enumerate(specs):
        d, V = gpu_domain(s)
        if i == 0:
            d.set_nonlocal_gauge("velocity")
        psi = orbitals(s)
        d.set_orbitals(to_device(psi, s.precision))
        doms.append(d)
        od = _oracle_gauge(s, V) if i == 0 else oracle_domain(s, V)
        refs.append(oracle.propagate(od, psi, s.A, s.dt, np.full(s.n_orb, 2.0)))
    b = mlmd.batch_create([d.handle for d in doms])
    obs = mlmd.batch_propagate(b, np.stack([s.A for s in specs]), first_handle=doms[0].handle)
    for i, d in enumerate(doms):
        assert np.max(np.abs(to_numpy(d.get_orbitals()) - refs[i][0])) <= 1e-5, i
        _check_obs(obs[i], refs[i][1], 1e-6)
    mlmd.batch_destroy(b)
    for d in doms:
        d.close()


def test_gauge_adjoint_is_unsupported():
    from paper_2509_00966_gb300 import mlmd
    spec = small_spec(precision="c128", n=(8, 9, 10), n_orb=4, steps=4, n_atoms=2)
    d, V = gpu_domain(spec)
    d.set_nonlocal_gauge("velocity")
    d.set_orbitals(to_device(orbitals(spec), "c128"))
    with pytest.raises(mlmd.MLMDError) as e:
        d.propagate_adjoint(spec.A, ckpt_every=2)
    assert e.value.status == 7
    d.close()


def test_gauge_on_dense_projector_domain():
    """A domain of the batched workload's density (about 41 projector spheres
    over every point) in the velocity gauge: the tensor-core nonlocal path
    holds real projector tables, so the step falls back to the per-point
    kernels with phases and still matches the oracle."""
    from paper_2509_00966_gb300 import inputs, mlmd
    spec = inputs.batched_specs(n_domains=2, n_steps=3, seed=11)[1]
    d, V = gpu_domain(spec)
    d.set_nonlocal_gauge("velocity")
    psi = inputs.random_orbitals(spec.n_grid, spec.n_orb, spec.dV, 78)
    d.set_orbitals(to_device(psi, "c64"))
    mlmd.profile_enable(d.handle, True)
    obs = d.propagate(spec.A)
    n_scatter = mlmd.profile_read(d.handle, "scatter")[1]
    out = to_numpy(d.get_orbitals())
    d.close()
    assert n_scatter == 0                     # no tensor-core scatter launches
    ref, robs = oracle.propagate(_oracle_gauge(spec, V), psi, spec.A, spec.dt, np.full(spec.n_orb, 2.0))
    err = np.max(np.abs(out - ref))
    print(f"\n[errors] gauge dense domain N={spec.n[0]} x {spec.n_orb}: psi={err:.3e}", flush=True)
    assert err <= 1e-5
    _check_obs(obs, robs, 1e-6)
