"""The allocation-free overlap entry point against the regular one and the oracle.

mlmd_overlap_noalloc exists for callers that cannot allocate device memory
when they need an overlap matrix (a frozen memory pool, a framework that
forbids allocation on its hot path); its split sums live in a fixed device
array declared by the library.  Here it is called through the C ABI twice in
a row, on different orbitals, and each result is compared with
mlmd_overlap (the entry point that allocates its own scratch) and with the
FP64 oracle's overlap on the same orbitals, within the overlap tolerance of
the other GPU tests.  The sizes cover a small ragged case, an orbital count
whose split sums fill only part of the array (so that the array, not the
GPU, limits the number of grid-point slabs), and the largest accepted count,
whose one slab takes the whole array.  This file is collected last so that
a failure here does not hide the other tests.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    from paper_2509_00966_gb300 import build
    build.build()
    torch.cuda.init()


@pytest.mark.parametrize("precision,tol", [("c64", 2e-6), ("c128", 1e-12)])
@pytest.mark.parametrize("n,no", [((12, 10, 14), 37), ((16, 16, 24), 300), ((16, 16, 16), 512)])
def test_overlap_noalloc_matches_overlap_twice(precision, tol, n, no):
    import torch
    from paper_2509_00966_gb300 import mlmd
    h = 0.4
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
            scale = np.abs(S_ref).max()
            assert np.max(np.abs(S - S_ref)) <= tol * scale, call
            # the same orbitals as the device holds them, through the FP64 oracle
            S_orc = oracle.overlap(X.cpu().numpy().astype(np.complex128),
                                   X.cpu().numpy().astype(np.complex128), dV)
            assert np.max(np.abs(S - S_orc)) <= tol * scale, call
    finally:
        d.close()


def test_overlap_noalloc_rejects_too_many_orbitals():
    """One orbital above the limit is refused before any launch; the output
    buffer is left as it was."""
    import torch
    from paper_2509_00966_gb300 import mlmd
    L = mlmd.lib()
    no, ng = 513, 64             # one above MLMD_OVERLAP_NOALLOC_MAX_ORB
    X = torch.zeros((ng, no), dtype=torch.complex64, device="cuda")
    S = torch.full((no, no), 7.0, dtype=torch.complex128, device="cuda")
    st = L.mlmd_overlap_noalloc(1, ng, no, X.data_ptr(), X.data_ptr(), 1.0, S.data_ptr(), None)
    torch.cuda.synchronize()
    assert st == 1
    assert bool(torch.all(S == 7.0))
