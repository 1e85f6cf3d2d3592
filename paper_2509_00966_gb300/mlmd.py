"""Thin Python binding of libmlmd's C ABI (include/mlmd.h).

Argument marshalling only: every function here passes plain pointers and
sizes to the library of the same name (``domain_create`` -> ``mlmd_domain_create``
and so on); all arithmetic runs in the library's CUDA kernels.  PyTorch is
used for device memory and the current CUDA stream.  If the compiled library
is missing, every call raises: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmlmd.so")

C128, C64 = 0, 1
GEMM = {"fp32": 0, "bf16": 1, "bf16x2": 2, "bf16x3": 3, "fp16": 4}
SCHEME = {"full": 0, "split": 1}
NL_GAUGE = {"real": 0, "velocity": 1}
ORTHO = {"chol": 0, "lowdin": 1}
STATUS = {0: "ok", 1: "invalid argument", 2: "out of device memory", 3: "CUDA error", 4: "numeric failure",
          5: "device wait timed out", 6: "invalid state", 7: "unsupported"}


class MLMDError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        super().__init__(f"libmlmd: {STATUS.get(status, status)}" + (f": {msg}" if msg else ""))


class Desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32 * 3), ("h", ctypes.c_double), ("n_orb", ctypes.c_int32),
                ("fd_order", ctypes.c_int32), ("precision", ctypes.c_int32), ("gemm_mode", ctypes.c_int32),
                ("scheme", ctypes.c_int32), ("dt", ctypes.c_double), ("ortho_every", ctypes.c_int32),
                ("ortho_kind", ctypes.c_int32)]


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class Allocator(ctypes.Structure):
    _fields_ = [("alloc", _ALLOC_FN), ("free", _FREE_FN), ("ctx", ctypes.c_void_p)]


# name -> (restype, argtypes)
_P = ctypes.c_void_p
_SIGS = {
    "mlmd_abi_version": (ctypes.c_int32, []),
    "mlmd_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "mlmd_domain_create": (ctypes.c_int, [ctypes.POINTER(Desc), ctypes.POINTER(Allocator), _P, ctypes.POINTER(_P)]),
    "mlmd_domain_destroy": (ctypes.c_int, [_P]),
    "mlmd_set_orbitals": (ctypes.c_int, [_P, _P, ctypes.c_int32]),
    "mlmd_get_orbitals": (ctypes.c_int, [_P, _P, ctypes.c_int32]),
    "mlmd_set_occupations": (ctypes.c_int, [_P, _P]),
    "mlmd_set_potential": (ctypes.c_int, [_P, _P]),
    "mlmd_set_projectors": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_int32, ctypes.c_double,
                                           ctypes.c_double, _P]),
    "mlmd_get_projector_lists": (ctypes.c_int, [_P, _P, _P, ctypes.c_size_t, _P]),
    "mlmd_set_nonlocal_gauge": (ctypes.c_int, [_P, ctypes.c_int32]),
    "mlmd_propagate": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P]),
    "mlmd_density_current": (ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.c_int32]),
    "mlmd_overlap": (ctypes.c_int, [_P, _P]),
    "mlmd_reorthonormalize": (ctypes.c_int, [_P, ctypes.c_int32]),
    "mlmd_excitation": (ctypes.c_int, [_P, _P]),
    "mlmd_occupations": (ctypes.c_int, [_P, _P, _P]),
    "mlmd_ks_correction": (ctypes.c_int, [_P, _P]),
    "mlmd_propagate_adjoint": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_int32, _P, _P, _P, ctypes.c_int32]),
    "mlmd_batch_create": (ctypes.c_int, [ctypes.c_int32, _P, ctypes.POINTER(_P)]),
    "mlmd_batch_destroy": (ctypes.c_int, [_P]),
    "mlmd_batch_propagate": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P]),
    "mlmd_overlap_noalloc": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, _P, _P,
                                            ctypes.c_double, _P, _P]),
    "mlmd_profile_enable": (ctypes.c_int, [_P, ctypes.c_int32]),
    "mlmd_profile_read": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P]),
    "mlmd_launch_count": (ctypes.c_uint64, [_P]),
    "mlmd_last_error": (ctypes.c_char_p, [_P]),
}

_lib = None


def lib():
    """The loaded libmlmd (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libmlmd is not built ({LIB_PATH} missing); run "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def declared_symbols():
    return list(_SIGS)


def _check(st, handle=None):
    if st != 0:
        msg = lib().mlmd_last_error(handle).decode() if handle else ""
        raise MLMDError(st, msg)


def _stream_ptr():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(x):
    """(pointer, on_device, keepalive) of a torch tensor or numpy array."""
    try:
        import torch
        if isinstance(x, torch.Tensor):
            assert x.is_contiguous()
            return ctypes.c_void_p(x.data_ptr()), int(x.is_cuda), x
    except ImportError:  # pragma: no cover
        pass
    x = np.ascontiguousarray(x)
    return ctypes.c_void_p(x.ctypes.data), 0, x


# ---------------------------------------------------------------------------
# functions with the ABI's names
# ---------------------------------------------------------------------------

def abi_version():
    return lib().mlmd_abi_version()


def domain_create(n, h, n_orb, fd_order=4, precision="c64", gemm_mode="fp32", scheme="full", dt=0.02,
                  ortho_every=0, ortho_kind="chol", stream=None):
    d = Desc()
    n = (n, n, n) if np.ndim(n) == 0 else tuple(n)
    d.n = (ctypes.c_int32 * 3)(*[int(v) for v in n])
    d.h = float(h)
    d.n_orb = int(n_orb)
    d.fd_order = int(fd_order)
    d.precision = C64 if precision == "c64" else C128
    d.gemm_mode = GEMM[gemm_mode]
    d.scheme = SCHEME[scheme]
    d.dt = float(dt)
    d.ortho_every = int(ortho_every)
    d.ortho_kind = ORTHO[ortho_kind]
    out = ctypes.c_void_p()
    st = lib().mlmd_domain_create(ctypes.byref(d), None, stream if stream is not None else _stream_ptr(),
                                  ctypes.byref(out))
    _check(st)
    return out


def domain_destroy(h):
    _check(lib().mlmd_domain_destroy(h))


def set_orbitals(h, psi):
    p, dev, keep = _ptr(psi)
    _check(lib().mlmd_set_orbitals(h, p, dev), h)


def get_orbitals(h, out):
    p, dev, keep = _ptr(out)
    _check(lib().mlmd_get_orbitals(h, p, dev), h)
    return out


def set_occupations(h, f):
    f = _f64(f)
    _check(lib().mlmd_set_occupations(h, ctypes.c_void_p(f.ctypes.data)), h)


def set_potential(h, v):
    v = _f64(v)
    _check(lib().mlmd_set_potential(h, ctypes.c_void_p(v.ctypes.data)), h)


def set_projectors(h, pos, n_proj, r_c, r_cut, D):
    pos = _f64(pos).reshape(-1, 3)
    na = pos.shape[0]
    D = _f64(D).reshape(na, -1) if na else np.zeros((0, max(n_proj, 1)))
    _check(lib().mlmd_set_projectors(h, na, ctypes.c_void_p(pos.ctypes.data), int(n_proj), float(r_c), float(r_cut),
                                     ctypes.c_void_p(D.ctypes.data)), h)


def set_nonlocal_gauge(h, gauge):
    """'real' (A-independent projectors) or 'velocity' (b e^{-iA.(r-R_a)})."""
    _check(lib().mlmd_set_nonlocal_gauge(h, NL_GAUGE[gauge]), h)


def projector_list_length(h, n_atoms):
    """Total number of (atom, grid point) list entries (reads only the offsets)."""
    off = np.zeros(n_atoms + 1, np.int64)
    _check(lib().mlmd_get_projector_lists(h, ctypes.c_void_p(off.ctypes.data), None, 0, None), h)
    return int(off[-1])


def get_projector_lists(h, n_atoms, n_proj):
    off = np.zeros(n_atoms + 1, np.int64)
    _check(lib().mlmd_get_projector_lists(h, ctypes.c_void_p(off.ctypes.data), None, 0, None), h)
    n = int(off[-1])
    idx = np.zeros(max(n, 1), np.int32)
    beta = np.zeros((max(n, 1), max(n_proj, 1)), np.float64)
    _check(lib().mlmd_get_projector_lists(h, ctypes.c_void_p(off.ctypes.data), ctypes.c_void_p(idx.ctypes.data),
                                          idx.size, ctypes.c_void_p(beta.ctypes.data)), h)
    return off, idx[:n], beta[:n]


def propagate(h, A, obs=True):
    A = _f64(A).reshape(-1, 3)
    out = np.zeros((A.shape[0], 5)) if obs else None
    _check(lib().mlmd_propagate(h, A.shape[0], ctypes.c_void_p(A.ctypes.data),
                                ctypes.c_void_p(out.ctypes.data) if obs else None), h)
    return out


def density_current(h, A, rho=None, j=None):
    """rho [N_g], j [3, N_g] (torch CUDA tensors or numpy arrays of the domain's
    real type, either may be None); returns (rho, j, J)."""
    A = _f64(A).reshape(3)
    J = np.zeros(3)
    pr, dr, kr = _ptr(rho) if rho is not None else (None, None, None)
    pj, dj, kj = _ptr(j) if j is not None else (None, None, None)
    on_dev = dr if dr is not None else (dj if dj is not None else 0)
    _check(lib().mlmd_density_current(h, ctypes.c_void_p(A.ctypes.data), pr, pj, ctypes.c_void_p(J.ctypes.data),
                                      on_dev), h)
    return rho, j, J


def overlap(h, n_orb):
    S = np.zeros((n_orb, n_orb), np.complex128)
    _check(lib().mlmd_overlap(h, ctypes.c_void_p(S.ctypes.data)), h)
    return S


def reorthonormalize(h, kind="chol"):
    _check(lib().mlmd_reorthonormalize(h, ORTHO[kind]), h)


def excitation(h):
    v = ctypes.c_double()
    _check(lib().mlmd_excitation(h, ctypes.byref(v)), h)
    return v.value


def occupations(h, n_orb):
    """(f_s(t) [N_o], n_exc): occupations of the reference orbitals and the
    electrons that left their span."""
    fs = np.zeros(n_orb, np.float64)
    v = ctypes.c_double()
    _check(lib().mlmd_occupations(h, ctypes.c_void_p(fs.ctypes.data), ctypes.byref(v)), h)
    return fs, v.value


def ks_correction(h, delta):
    """Eq. 5 once: Psi(t) -= delta Psi(0) (dV Psi(0)^H Psi(t)); delta complex."""
    dl = np.array([complex(delta).real, complex(delta).imag], np.float64)
    _check(lib().mlmd_ks_correction(h, ctypes.c_void_p(dl.ctypes.data)), h)


def propagate_adjoint(h, A, ckpt_every, n_grid, dL_dV=None):
    A = _f64(A).reshape(-1, 3)
    loss = ctypes.c_double()
    dA = np.zeros_like(A)
    if dL_dV is None:
        dL_dV = np.zeros(n_grid)
    p, dev, keep = _ptr(dL_dV)
    _check(lib().mlmd_propagate_adjoint(h, A.shape[0], ctypes.c_void_p(A.ctypes.data), int(ckpt_every),
                                        ctypes.byref(loss), ctypes.c_void_p(dA.ctypes.data), p, dev), h)
    return loss.value, dA, dL_dV


_EXC_LOSS = None


def _excitation_loss_fn():
    global _EXC_LOSS
    if _EXC_LOSS is None:
        import torch

        class ExcitationLoss(torch.autograd.Function):
            @staticmethod
            def forward(ctx, A, V, dom, ckpt_every):
                Ah = A.detach().to("cpu", torch.float64).contiguous().numpy()
                Vh = V.detach().to("cpu", torch.float64).contiguous().numpy()
                dom.set_potential(Vh)
                dV = torch.zeros(dom.n_grid, dtype=torch.float64, device=V.device)
                loss, dA, dV = propagate_adjoint(dom.handle, Ah, ckpt_every, dom.n_grid, dV)
                ctx.save_for_backward(torch.from_numpy(dA).to(A.device, A.dtype), dV.to(V.dtype))
                return torch.tensor(loss, dtype=torch.float64, device=A.device)

            @staticmethod
            def backward(ctx, g):
                dA, dV = ctx.saved_tensors
                return g.to(dA.device, dA.dtype) * dA, g.to(dV.device, dV.dtype) * dV, None, None

        _EXC_LOSS = ExcitationLoss
    return _EXC_LOSS


def excitation_loss(dom, A, V, ckpt_every):
    """n_exc(Psi(T)) (Sec. V.A.8) after len(A) full-scheme steps from the
    domain's current orbitals, as a torch function of the vector-potential
    samples A ([n_steps, 3]) and the local potential V ([N_g]); backward
    gives mlmd_propagate_adjoint's dL/dA and dL/dV.  V becomes the domain's
    potential and the orbitals are left at Psi(T), as the ABI call does."""
    return _excitation_loss_fn().apply(A, V, dom, int(ckpt_every))


def batch_create(handles):
    arr = (ctypes.c_void_p * len(handles))(*[h.value for h in handles])
    out = ctypes.c_void_p()
    _check(lib().mlmd_batch_create(len(handles), arr, ctypes.byref(out)))
    return out


def batch_destroy(b):
    _check(lib().mlmd_batch_destroy(b))


def batch_propagate(b, A, obs=True, first_handle=None):
    """A: [n_domains, n_steps, 3]; returns obs [n_domains, n_steps, 5] or None."""
    A = _f64(A)
    nd, ns = A.shape[0], A.shape[1]
    out = np.zeros((nd, ns, 5)) if obs else None
    _check(lib().mlmd_batch_propagate(b, ns, ctypes.c_void_p(A.ctypes.data),
                                      ctypes.c_void_p(out.ctypes.data) if obs else None), first_handle)
    return out


def overlap_noalloc(X, Y, scale, S, stream=None):
    """S = scale * X^dagger Y for device tensors X, Y [n_grid, n_orb] (complex64
    or complex128) into the device tensor S [n_orb, n_orb] complex128, without
    any device allocation by the library (see include/mlmd.h)."""
    import torch
    assert X.is_cuda and Y.is_cuda and S.is_cuda and X.shape == Y.shape and X.dtype == Y.dtype
    assert S.dtype == torch.complex128 and S.shape == (X.shape[1], X.shape[1])
    assert X.is_contiguous() and Y.is_contiguous() and S.is_contiguous()
    prec = C64 if X.dtype == torch.complex64 else C128
    st = lib().mlmd_overlap_noalloc(prec, X.shape[0], X.shape[1], ctypes.c_void_p(X.data_ptr()),
                                    ctypes.c_void_p(Y.data_ptr()), float(scale), ctypes.c_void_p(S.data_ptr()),
                                    stream if stream is not None else _stream_ptr())
    _check(st)
    return S


KERNEL = {"stage": 0, "project": 1, "scatter": 2, "gemm": 3}


def profile_enable(h, enable=True):
    _check(lib().mlmd_profile_enable(h, int(bool(enable))), h)


def profile_read(h, kind):
    """(total device ms, launches) of one kernel kind since profile_enable."""
    ms = ctypes.c_double()
    n = ctypes.c_uint64()
    _check(lib().mlmd_profile_read(h, KERNEL[kind], ctypes.byref(ms), ctypes.byref(n)), h)
    return ms.value, n.value


def launch_count(h):
    return int(lib().mlmd_launch_count(h))


def last_error(h):
    return lib().mlmd_last_error(h).decode()


# ---------------------------------------------------------------------------
# convenience wrapper owning a handle
# ---------------------------------------------------------------------------

class Domain:
    """One domain handle; methods forward to the functions above."""

    def __init__(self, n, h, n_orb, fd_order=4, precision="c64", gemm_mode="fp32", scheme="full", dt=0.02,
                 ortho_every=0, ortho_kind="chol"):
        self.n = (n, n, n) if np.ndim(n) == 0 else tuple(int(v) for v in n)
        self.h = float(h)
        self.n_orb = int(n_orb)
        self.n_grid = int(np.prod(self.n))
        self.precision = precision
        self.handle = domain_create(self.n, h, n_orb, fd_order, precision, gemm_mode, scheme, dt, ortho_every,
                                    ortho_kind)
        self.n_atoms = 0
        self.n_proj = 0

    @classmethod
    def from_spec(cls, spec, V=None, gemm_mode="fp32", scheme="full", ortho_every=None, n_orb=None):
        from .inputs import gaussian_wells
        d = cls(spec.n, spec.h, n_orb or spec.n_orb, spec.fd_order, spec.precision, gemm_mode, scheme, spec.dt,
                spec.ortho_every if ortho_every is None else ortho_every)
        if V is None:
            V = gaussian_wells(spec.n, spec.h, spec.wells, spec.well_depth, spec.well_width)
        d.set_potential(V)
        d.set_occupations(spec.occ[: d.n_orb] if len(spec.occ) >= d.n_orb else np.full(d.n_orb, 2.0))
        if spec.n_proj and len(spec.atoms):
            d.set_projectors(spec.atoms, spec.n_proj, spec.r_c, spec.r_cut, spec.D)
        return d

    @property
    def cdtype(self):
        import torch
        return torch.complex64 if self.precision == "c64" else torch.complex128

    def close(self):
        if self.handle is not None:
            domain_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_orbitals(self, psi):
        set_orbitals(self.handle, psi)

    def get_orbitals(self, device=True):
        import torch
        out = torch.empty((self.n_grid, self.n_orb), dtype=self.cdtype, device="cuda" if device else "cpu")
        return get_orbitals(self.handle, out)

    def set_occupations(self, f):
        set_occupations(self.handle, f)

    def set_potential(self, v):
        set_potential(self.handle, v)

    def set_projectors(self, pos, n_proj, r_c, r_cut, D):
        set_projectors(self.handle, pos, n_proj, r_c, r_cut, D)
        self.n_atoms = int(np.asarray(pos).reshape(-1, 3).shape[0])
        self.n_proj = int(n_proj) if self.n_atoms else 0

    def set_nonlocal_gauge(self, gauge):
        set_nonlocal_gauge(self.handle, gauge)

    def projector_lists(self):
        return get_projector_lists(self.handle, self.n_atoms, self.n_proj)

    def projector_list_length(self):
        return projector_list_length(self.handle, self.n_atoms) if self.n_atoms else 0

    def propagate(self, A, obs=True):
        return propagate(self.handle, A, obs)

    def density_current(self, A, device=True):
        import torch
        rdt = torch.float32 if self.precision == "c64" else torch.float64
        dev = "cuda" if device else "cpu"
        rho = torch.empty(self.n_grid, dtype=rdt, device=dev)
        j = torch.empty((3, self.n_grid), dtype=rdt, device=dev)
        return density_current(self.handle, A, rho, j)

    def overlap(self):
        return overlap(self.handle, self.n_orb)

    def reorthonormalize(self, kind="chol"):
        reorthonormalize(self.handle, kind)

    def excitation(self):
        return excitation(self.handle)

    def ks_correction(self, delta):
        ks_correction(self.handle, delta)

    def occupations(self):
        return occupations(self.handle, self.n_orb)

    def propagate_adjoint(self, A, ckpt_every, dL_dV=None):
        return propagate_adjoint(self.handle, A, ckpt_every, self.n_grid, dL_dV)

    def excitation_loss(self, A, V, ckpt_every):
        return excitation_loss(self, A, V, ckpt_every)

    @property
    def launches(self):
        return launch_count(self.handle)
