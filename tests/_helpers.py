"""Shared set-up for the GPU parity tests: the same seeded inputs go to the
CUDA library (through the C ABI) and to the FP64 oracle."""
import numpy as np

import oracle
from paper_2509_00966_gb300 import inputs


def small_spec(n=(12, 10, 14), h=0.4, n_orb=20, fd_order=4, precision="c64", n_proj=4, n_atoms=6, steps=10,
               seed=5, pulse=True, r_cut=2.2, r_c=0.9, dt=0.02):
    """A small periodic domain with everything switched on: ragged grid,
    orbital count not a multiple of the padding, wells, projectors and a
    z-polarised pulse with x and y components added."""
    rng = np.random.Generator(np.random.PCG64(seed + 100))
    L = np.array(n) * h
    atoms = rng.uniform(0, 1, (n_atoms, 3)) * L if n_proj else None
    A = np.zeros((steps, 3))
    if pulse:
        A = inputs.envelope_pulse(steps, dt, A0=0.3, omega=0.5, fwhm=2.0)
        A[:, 0] = 0.05
        A[:, 1] = -0.03
    return inputs.make_domain(n, h, n_orb, fd_order, precision, dt, steps, seed=seed, geo_seed=seed + 100,
                              n_wells=5, atoms=atoms, n_proj=n_proj, r_c=r_c, r_cut=r_cut, A=A)


def orbitals(spec, seed=None):
    return inputs.random_orbitals(spec.n_grid, spec.n_orb, spec.dV, spec.seed if seed is None else seed)


def gpu_domain(spec, gemm_mode="fp32", scheme="full", ortho_every=None, ortho_kind="chol", n_orb=None):
    from paper_2509_00966_gb300 import mlmd
    d = mlmd.Domain(spec.n, spec.h, n_orb or spec.n_orb, spec.fd_order, spec.precision, gemm_mode, scheme, spec.dt,
                    spec.ortho_every if ortho_every is None else ortho_every, ortho_kind)
    V = inputs.gaussian_wells(spec.n, spec.h, spec.wells, spec.well_depth, spec.well_width)
    d.set_potential(V)
    d.set_occupations(np.full(d.n_orb, 2.0))
    if spec.n_proj and len(spec.atoms):
        d.set_projectors(spec.atoms, spec.n_proj, spec.r_c, spec.r_cut, spec.D)
    return d, V


def oracle_domain(spec, V, n_orb=None):
    return oracle.Domain(spec.n, spec.h, n_orb or spec.n_orb, spec.fd_order, V, spec.atoms if spec.n_proj else None,
                         spec.n_proj, spec.r_c, spec.r_cut, spec.D)


def to_device(psi, precision):
    import torch
    dt = torch.complex64 if precision == "c64" else torch.complex128
    return torch.from_numpy(np.ascontiguousarray(psi)).to(dt).cuda()


def to_numpy(t):
    return t.detach().cpu().numpy().astype(np.complex128)
