"""The C-ABI library builds, loads and exports every symbol include/mlmd.h
declares; host-side validation rejects bad descriptors before any device
work.  No GPU needed."""
import ctypes
import os
import re

import pytest

from paper_2509_00966_gb300 import build, mlmd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "mlmd.h")).read()
    return sorted(set(re.findall(r"MLMD_API[^;]*?\b(mlmd_\w+)\s*\(", txt, flags=re.S)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return mlmd.lib()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["mlmd_domain_create", "mlmd_set_potential", "mlmd_set_projectors", "mlmd_propagate",
              "mlmd_density_current", "mlmd_propagate_adjoint", "mlmd_batch_propagate"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for n in _declared():
        assert hasattr(lib, n), n
    # and the binding knows every one of them, with the same names
    assert sorted(mlmd.declared_symbols()) == _declared()


def test_exported_symbols_are_only_the_abi(lib):
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", mlmd.LIB_PATH], capture_output=True, text=True).stdout
    ours = [l.split()[-1] for l in out.splitlines() if l.split()[-1].startswith("mlmd")]
    assert sorted(ours) == _declared()


def test_abi_version_and_status_strings(lib):
    assert lib.mlmd_abi_version() == 1
    assert lib.mlmd_status_string(0) == b"ok"
    assert lib.mlmd_status_string(7) == b"unsupported"


def _desc(**kw):
    d = mlmd.Desc()
    d.n = (ctypes.c_int32 * 3)(*kw.get("n", (8, 8, 8)))
    d.h = kw.get("h", 0.4)
    d.n_orb = kw.get("n_orb", 4)
    d.fd_order = kw.get("fd_order", 4)
    d.precision = kw.get("precision", 1)
    d.gemm_mode = kw.get("gemm_mode", 0)
    d.scheme = kw.get("scheme", 0)
    d.dt = kw.get("dt", 0.02)
    d.ortho_every = kw.get("ortho_every", 0)
    d.ortho_kind = kw.get("ortho_kind", 0)
    return d


@pytest.mark.parametrize("bad", [dict(n=(3, 8, 8)), dict(h=0.0), dict(h=float("nan")), dict(n_orb=0),
                                 dict(fd_order=6), dict(precision=5), dict(gemm_mode=9), dict(scheme=2),
                                 dict(dt=-1.0), dict(ortho_every=-1), dict(ortho_kind=3)])
def test_invalid_descriptor_rejected_on_host(lib, bad):
    out = ctypes.c_void_p()
    st = lib.mlmd_domain_create(ctypes.byref(_desc(**bad)), None, None, ctypes.byref(out))
    assert st == 1 and not out.value


def test_null_arguments_rejected(lib):
    assert lib.mlmd_domain_create(None, None, None, None) == 1
    assert lib.mlmd_domain_destroy(None) == 1
    assert lib.mlmd_propagate(None, 1, None, None) == 1
    # every entry point that takes a handle rejects a null one before touching a device
    v = ctypes.c_double()
    assert lib.mlmd_excitation(None, ctypes.byref(v)) == 1
    assert lib.mlmd_occupations(None, None, ctypes.byref(v)) == 1
    assert lib.mlmd_ks_correction(None, None) == 1
    assert lib.mlmd_overlap(None, None) == 1
    assert lib.mlmd_reorthonormalize(None, 0) == 1
    assert lib.mlmd_batch_create(0, None, None) == 1
    assert lib.mlmd_last_error(None) == b"null handle"
    assert lib.mlmd_launch_count(None) == 0


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    """No fallback: with libmlmd missing, the first call raises instead of
    computing anything another way."""
    monkeypatch.setattr(mlmd, "_lib", None)
    monkeypatch.setattr(mlmd, "LIB_PATH", str(tmp_path / "libmlmd.so"))
    with pytest.raises(RuntimeError, match="not built"):
        mlmd.abi_version()


def test_seeded_inputs_repeat():
    """Both sides get their inputs from the seeded generators: the same
    workload twice gives the same arrays, bit for bit."""
    import numpy as np
    from paper_2509_00966_gb300 import inputs
    for name in ["c0", "c4"]:
        a, b = inputs.config(name, n_steps=3), inputs.config(name, n_steps=3)
        for f in ["wells", "well_depth", "atoms", "D", "A", "occ"]:
            assert np.array_equal(getattr(a, f), getattr(b, f)), (name, f)
    p1 = inputs.random_orbitals(500, 4, 0.1, 3)
    assert np.array_equal(p1, inputs.random_orbitals(500, 4, 0.1, 3))
    assert not np.array_equal(p1, inputs.random_orbitals(500, 4, 0.1, 4))
