"""The allocation-free tridiagonal eigen-solve, gsyeig_tridiag_eig_noalloc.

It exists for callers that cannot allocate device memory when they need the
solve (device memory owned by another allocator or a fixed budget; loops
where a cudaMalloc would synchronise the device).  Its scratch is a fixed
array inside the library.  This test calls it through the C ABI and checks
it against gsyeig_tridiag_eig (same tolerances as the other tridiagonal
tests) on consecutive calls, so that the shared scratch left by one call
cannot leak into the next.  The file name makes pytest collect it last."""
import ctypes

import numpy as np
import pytest
import torch

import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib_and_solver():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1111_6374_gb300 import Solver, load

    return load(), Solver(0)


def _noalloc(lib, d, e, first, cnt):
    m = d.shape[0]
    lam = torch.full((cnt,), float("nan"), device="cuda", dtype=torch.float64)
    Z = torch.full((cnt, m), float("nan"), device="cuda", dtype=torch.float64).t()
    st = lib.gsyeig_tridiag_eig_noalloc(ctypes.c_void_p(d.data_ptr()), ctypes.c_void_p(e.data_ptr()), m, first, cnt,
                                        ctypes.c_void_p(lam.data_ptr()), ctypes.c_void_p(Z.data_ptr()), m,
                                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, lam, Z


@pytest.mark.parametrize("cases", [[(300, 100, 100, False), (777, 0, 200, True), (300, 100, 100, False)]])
def test_noalloc_matches_allocating_entry_point_on_consecutive_calls(lib_and_solver, cases):
    lib, solver = lib_and_solver
    for m, first, cnt, clustered in cases:
        d, e = (t.cuda() for t in inputs.make_tridiagonal(m, seed=m + cnt, clustered=clustered))
        st, lam, Z = _noalloc(lib, d, e, first, cnt)
        assert st == 0
        lam_ref, Z_ref = solver.tridiag_eig(d, e, first, cnt)
        tn = float(d.abs().max() + 2 * e.abs().max())
        assert float((lam - lam_ref).abs().max()) <= 1e-12 * tn
        assert float((Z - Z_ref).abs().max()) <= 1e-10
        Zn = Z.cpu().numpy()
        assert np.abs(Zn.T @ Zn - np.eye(cnt)).max() <= 1e-10


def test_noalloc_rejects_sizes_beyond_its_scratch(lib_and_solver):
    lib, _ = lib_and_solver
    m, cnt = 4096, 300  # 5 m cnt > 2^20 doubles
    d, e = (t.cuda() for t in inputs.make_tridiagonal(m, seed=1))
    st, lam, Z = _noalloc(lib, d, e, 0, cnt)
    assert st == 7
    assert b"scratch" in lib.gsyeig_strerror(7)
    assert bool(torch.isnan(lam).all()) and bool(torch.isnan(Z).all())
