"""Seeded synthetic inputs for the local-field-dynamics (LFD) workloads.

This module only draws random numbers and lays out input arrays: grids,
local-potential wells, atom sites, projector strengths, laser pulses and
initial orbitals.  It holds none of the propagation arithmetic; both the CUDA
library and the FP64 oracle receive the arrays it returns.

The five workloads stand in for the paper's PbTiO3 domains (Sec. VI.A,
Sec. VII.A.1), whose structures and pseudopotentials are not available:

* ``c0``  16^3 grid, h=0.4, 32 complex128 orbitals, 2nd-order stencil,
          8 Gaussian wells, no projectors, A=0, 100 steps.
* ``c1``  48^3 grid, h=0.35, 256 complex64 orbitals, 4th-order stencil,
          64 wells on a perturbed 4x4x4 lattice, 64 atoms x 4 projectors,
          Gaussian-envelope pulse, 1000 steps.
* ``c2``  64^3 grid, h=0.35, 1024 orbitals, 128 atoms x 8 projectors,
          Cholesky re-orthonormalisation every 10 steps, 500 steps.
* ``c3``  216 domains, N ~ U{24..40}, N_o ~ U{32..192}, atoms = round(N^3/64).
* ``c4``  32^3 grid, h=0.4, 128 orbitals, 32 atoms x 4 projectors, random
          smooth 8-Gaussian pulse, 500 steps, checkpoints every 50.

Seeds: orbitals use the workload index, geometry index+100, pulses index+200;
every generator is NumPy PCG64.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

__all__ = [
    "DomainSpec", "make_domain", "config", "config_names", "gaussian_wells",
    "random_orbitals", "envelope_pulse", "random_smooth_pulse", "batched_specs",
]


@dataclasses.dataclass
class DomainSpec:
    """Everything needed to set up one periodic domain (atomic units)."""
    n: tuple                    # grid points per axis (nx, ny, nz)
    h: float                    # grid spacing, bohr
    n_orb: int
    fd_order: int               # 2 or 4
    precision: str              # "c128" or "c64"
    dt: float
    n_steps: int
    wells: np.ndarray           # [n_wells, 3] centres, bohr
    well_depth: np.ndarray      # [n_wells] U, Ha
    well_width: float           # sigma, bohr
    atoms: np.ndarray           # [n_atoms, 3] projector centres, bohr
    n_proj: int                 # projectors per atom (0, 4 or 8)
    r_c: float
    r_cut: float
    D: np.ndarray               # [n_atoms, n_proj] diagonal strengths, Ha
    occ: np.ndarray             # [n_orb] occupations f_n
    A: np.ndarray               # [n_steps, 3] vector potential at step midpoints
    ortho_every: int = 0
    ckpt_every: int = 0
    seed: int = 0
    name: str = ""

    @property
    def n_grid(self) -> int:
        return int(self.n[0] * self.n[1] * self.n[2])

    @property
    def L(self) -> np.ndarray:
        return np.array(self.n, dtype=np.float64) * self.h

    @property
    def dV(self) -> float:
        return self.h ** 3

    @property
    def units_per_step(self) -> int:
        return self.n_grid * self.n_orb


def _grid_coords(n, h):
    """Point coordinates r = (i*h, j*h, k*h) in linear order x fastest."""
    nx, ny, nz = n
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return (np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1).astype(np.float64) * h)


def gaussian_wells(n, h, centres, depth, width):
    """V(r) = -sum_w U_w exp(-d^2 / (2 sigma^2)), d summed over the 27 nearest
    periodic images so that V is periodic.  Returns float64 [N_g].

    The image set is the product {-1, 0, 1}^3, so each well's sum factorises
    into three one-dimensional periodic sums, g_x(x) g_y(y) g_z(z), and V is
    one contraction over the wells (x fastest in the result)."""
    n = tuple(int(v) for v in n)
    centres = np.asarray(centres, dtype=np.float64).reshape(-1, 3)
    depth = np.asarray(depth, dtype=np.float64).reshape(-1)
    if len(centres) == 0:
        return np.zeros(n[0] * n[1] * n[2])
    L = np.array(n, dtype=np.float64) * h
    g = []
    for ax in range(3):
        x = np.arange(n[ax], dtype=np.float64) * h                         # [n_ax]
        d = x[None, None, :] - (centres[:, ax][:, None, None] + np.array([-1.0, 0.0, 1.0])[None, :, None] * L[ax])
        g.append(np.exp(-d * d / (2.0 * width * width)).sum(axis=1))      # [wells, n_ax]
    V = -np.einsum("w,wz,wy,wx->zyx", depth, g[2], g[1], g[0], optimize=True)
    return np.ascontiguousarray(V).reshape(-1)


def random_orbitals(n_grid, n_orb, dV, seed, dtype=np.complex128):
    """Re and Im i.i.d. N(0,1) from PCG64(seed), orthonormalised in the dV
    metric by a Cholesky factorisation taken in orbital order.  [N_g, N_o]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    re = rng.standard_normal((n_grid, n_orb))
    im = rng.standard_normal((n_grid, n_orb))
    psi = re + 1j * im
    S = dV * (psi.conj().T @ psi)
    Lc = np.linalg.cholesky(S)
    # psi <- psi L^{-H}: solve L X^T = psi^T for the conjugate-transposed factor
    psi = np.linalg.solve(Lc.conj(), psi.T).T
    return np.ascontiguousarray(psi.astype(dtype))


def envelope_pulse(n_steps, dt, A0=0.05, omega=0.1, fwhm=200.0, t0=None, axis=2):
    """A(t) = e_axis A0 exp(-4 ln2 (t-t0)^2 / FWHM^2) sin(omega (t-t0)),
    sampled at step midpoints t_k = (k+1/2) dt; t0 defaults to the run's centre."""
    T = n_steps * dt
    if t0 is None:
        t0 = 0.5 * T
    t = (np.arange(n_steps) + 0.5) * dt
    a = A0 * np.exp(-4.0 * math.log(2.0) * (t - t0) ** 2 / fwhm ** 2) * np.sin(omega * (t - t0))
    A = np.zeros((n_steps, 3))
    A[:, axis] = a
    return A


def random_smooth_pulse(n_steps, dt, seed, n_gauss=8, amp=0.05, axis=2):
    """A_z(t) = sum_i a_i exp(-(t-t_i)^2 / (2 s_i^2)), t_i~U[0,T], s_i~U[0.5,2],
    a_i~U[-1,1], rescaled so that max|A_z| over the samples equals amp."""
    rng = np.random.Generator(np.random.PCG64(seed))
    T = n_steps * dt
    ti = rng.uniform(0.0, T, n_gauss)
    si = rng.uniform(0.5, 2.0, n_gauss)
    ai = rng.uniform(-1.0, 1.0, n_gauss)
    t = (np.arange(n_steps) + 0.5) * dt
    a = np.zeros(n_steps)
    for k in range(n_gauss):
        a += ai[k] * np.exp(-(t - ti[k]) ** 2 / (2.0 * si[k] ** 2))
    a *= amp / np.max(np.abs(a))
    A = np.zeros((n_steps, 3))
    A[:, axis] = a
    return A


def _lattice(cells, L, basis, rng=None, sigma=0.0):
    sites = []
    for k in range(cells):
        for j in range(cells):
            for i in range(cells):
                for b in basis:
                    sites.append((np.array([i, j, k], dtype=np.float64) + np.asarray(b)) * (L / cells))
    sites = np.array(sites)
    if rng is not None and sigma > 0:
        sites = sites + rng.normal(0.0, sigma, sites.shape)
    return np.mod(sites, L)


def make_domain(n, h, n_orb, fd_order, precision, dt, n_steps, *, seed, geo_seed,
                n_wells=None, wells=None, well_depth=None, well_width=0.8,
                atoms=None, n_proj=0, r_c=1.2, r_cut=3.0, D=None, A=None,
                ortho_every=0, ckpt_every=0, name=""):
    """Assemble a DomainSpec; unspecified wells are seeded uniformly in the box."""
    n = tuple(int(v) for v in (n if np.ndim(n) else (n, n, n)))
    L = np.array(n, dtype=np.float64) * h
    rng = np.random.Generator(np.random.PCG64(geo_seed))
    if wells is None:
        wells = rng.uniform(0.0, 1.0, (n_wells, 3)) * L
    if well_depth is None:
        well_depth = rng.uniform(0.5, 2.0, len(wells))
    if atoms is None:
        atoms = np.zeros((0, 3))
    if D is None:
        D = rng.uniform(-1.0, 1.0, (len(atoms), n_proj)) if n_proj else np.zeros((len(atoms), 0))
    if A is None:
        A = np.zeros((n_steps, 3))
    return DomainSpec(n=n, h=h, n_orb=n_orb, fd_order=fd_order, precision=precision, dt=dt,
                      n_steps=n_steps, wells=np.asarray(wells, np.float64),
                      well_depth=np.asarray(well_depth, np.float64), well_width=well_width,
                      atoms=np.asarray(atoms, np.float64), n_proj=n_proj, r_c=r_c, r_cut=r_cut,
                      D=np.asarray(D, np.float64), occ=np.full(n_orb, 2.0), A=np.asarray(A, np.float64),
                      ortho_every=ortho_every, ckpt_every=ckpt_every, seed=seed, name=name)


def config(name: str, *, n_orb: Optional[int] = None, n_steps: Optional[int] = None,
           n: Optional[int] = None) -> DomainSpec:
    """The single-domain workloads c0, c1, c2, c4 (optionally shrunk in
    orbitals, steps or grid for parity tests; geometry stays seeded the same)."""
    if name == "c0":
        idx, N, h, no, order, prec, steps = 0, 16, 0.4, 32, 2, "c128", 100
    elif name == "c1":
        idx, N, h, no, order, prec, steps = 1, 48, 0.35, 256, 4, "c64", 1000
    elif name == "c2":
        idx, N, h, no, order, prec, steps = 2, 64, 0.35, 1024, 4, "c64", 500
    elif name == "c4":
        idx, N, h, no, order, prec, steps = 4, 32, 0.4, 128, 4, "c64", 500
    else:
        raise ValueError(name)
    full_steps = steps
    N = n or N
    no = n_orb or no
    steps = n_steps or steps
    dt = 0.02
    L = N * h
    geo = np.random.Generator(np.random.PCG64(idx + 100))
    if name == "c0":
        return make_domain(N, h, no, order, prec, dt, steps, seed=idx, geo_seed=idx + 100,
                           n_wells=8, name=name)
    if name == "c1":
        sites = _lattice(4, L, [(0.5, 0.5, 0.5)], geo, 0.1)
        depth = geo.uniform(0.5, 2.0, len(sites))
        D = geo.uniform(-1.0, 1.0, (len(sites), 4))
        A = envelope_pulse(full_steps, dt)[:steps]
        return make_domain(N, h, no, order, prec, dt, steps, seed=idx, geo_seed=idx + 100,
                           wells=sites, well_depth=depth, atoms=sites, n_proj=4, D=D, A=A, name=name)
    if name == "c2":
        sites = _lattice(4, L, [(0.0, 0.0, 0.0), (0.5, 0.5, 0.5)], geo, 0.1)
        depth = geo.uniform(0.5, 2.0, len(sites))
        D = geo.uniform(-1.0, 1.0, (len(sites), 8))
        A = envelope_pulse(full_steps, dt)[:steps]
        return make_domain(N, h, no, order, prec, dt, steps, seed=idx, geo_seed=idx + 100,
                           wells=sites, well_depth=depth, atoms=sites, n_proj=8, D=D, A=A,
                           ortho_every=10, name=name)
    # c4
    sites = _lattice(2, L, [(0, 0, 0), (0.5, 0.5, 0.0), (0.5, 0.0, 0.5), (0.0, 0.5, 0.5)], geo, 0.1)
    depth = geo.uniform(0.5, 2.0, len(sites))
    D = geo.uniform(-1.0, 1.0, (len(sites), 4))
    A = random_smooth_pulse(full_steps, dt, seed=idx + 200)[:steps]
    return make_domain(N, h, no, order, prec, dt, steps, seed=idx, geo_seed=idx + 100,
                       wells=sites, well_depth=depth, atoms=sites, n_proj=4, D=D, A=A,
                       ckpt_every=50, name=name)


def config_names() -> List[str]:
    return ["c0", "c1", "c2", "c4"]


def batched_specs(n_domains=216, n_steps=200, seed=3, n_min=24, n_max=40,
                  orb_min=32, orb_max=192, h=0.35) -> List[DomainSpec]:
    """Workload c3: uneven domains, cubic N ~ U{n_min..n_max}, N_o ~ U{orb_min..orb_max}
    wells = atoms = round(N^3/64) at seeded uniform
    positions, 4 projectors per atom, the c1 pulse shape over n_steps."""
    rng = np.random.Generator(np.random.PCG64(seed + 100))
    A = envelope_pulse(1000, 0.02)[:n_steps]
    specs = []
    for d in range(n_domains):
        N = int(rng.integers(n_min, n_max + 1))
        no = int(rng.integers(orb_min, orb_max + 1))
        na = int(round(N ** 3 / 64))
        L = N * h
        sites = rng.uniform(0.0, 1.0, (na, 3)) * L
        depth = rng.uniform(0.5, 2.0, na)
        D = rng.uniform(-1.0, 1.0, (na, 4))
        specs.append(make_domain(N, h, no, 4, "c64", 0.02, n_steps, seed=seed * 1000 + d,
                                 geo_seed=seed + 100, wells=sites, well_depth=depth, atoms=sites,
                                 n_proj=4, D=D, A=A, name=f"c3/{d}"))
    return specs
