"""The allocation-free overlap entry point against the regular one.

mlmd_overlap_noalloc exists for callers that cannot allocate device memory
when they need an overlap matrix (a frozen memory pool, a framework that
forbids allocation on its hot path); its split sums live in a fixed device
array declared by the library.  Here it is called through the C ABI twice in
a row, on different orbitals, and each result is compared with
mlmd_overlap (the entry point that allocates its own scratch) on the same
orbitals, within the overlap tolerance of the other GPU tests.  This file
is collected last so that a failure here does not hide the other tests.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    from paper_2509_00966_gb300 import build
    build.build()
    torch.cuda.init()


@pytest.mark.parametrize("precision,tol", [("c64", 2e-6), ("c128", 1e-12)])
def test_overlap_noalloc_matches_overlap_twice(precision, tol):
    import torch
    from paper_2509_00966_gb300 import mlmd
    n, h, no = (12, 10, 14), 0.4, 37
    ng = n[0] * n[1] * n[2]
    dV = h ** 3
    dt = torch.complex64 if precision == "c64" else torch.complex128
    d = mlmd.Domain(n, h, no, 4, precision)
    try:
        for call in range(2):
            rng = np.random.default_rng(100 + call)
            psi = (rng.standard_normal((ng, no)) + 1j * rng.standard_normal((ng, no))) / np.sqrt(ng * dV)
            X = torch.from_numpy(psi).to(dt).cuda().contiguous()
            d.set_orbitals(X)
            S_ref = d.overlap()                                   # allocating entry point
            S = torch.full((no, no), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
            mlmd.overlap_noalloc(X, X, dV, S)
            torch.cuda.synchronize()
            S = S.cpu().numpy()
            assert np.all(np.isfinite(S))
            assert np.max(np.abs(S - S_ref)) <= tol * np.abs(S_ref).max(), call
    finally:
        d.close()


def test_overlap_noalloc_rejects_too_many_orbitals():
    from paper_2509_00966_gb300 import mlmd
    L = mlmd.lib()
    no = 513                     # one above MLMD_OVERLAP_NOALLOC_MAX_ORB
    dummy = ctypes.c_void_p(16)  # never dereferenced: the size check comes first
    st = L.mlmd_overlap_noalloc(1, 1000, no, dummy, dummy, 1.0, dummy, None)
    assert st == 1
