"""isdf_gemm_f64_noalloc: the tensor-core FP64-accurate product for callers
that cannot allocate device memory (its scratch is one static device array).

Called through the C ABI with device pointers, twice in a row with different
shapes (the second call reuses the array the first one left behind), and
checked against the allocating entry point isdf_gemm_f64 within the error
bound the GEMM tests use.  Oversized operands must be rejected, not run.
This file is collected last so a stop-at-first-failure run has already run
every other test; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _bound(A, B, slices=5):
    K = A.shape[1]
    return 2.0 ** -(7 * slices - 2) * K * np.abs(A).max(axis=1)[:, None] * np.abs(B).max(axis=1)[None, :]


def test_noalloc_matches_allocating_entry_point_on_two_calls():
    import torch

    from paper_2404_09373_gb300 import isdf as B_

    lib = B_.load_library()
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(20240409)
    for M, N, K in ((300, 200, 1500), (129, 97, 700)):
        A = rng.standard_normal((M, K)) * np.exp2(rng.integers(-20, 20, size=(M, 1)))
        Bm = rng.standard_normal((N, K)) * np.exp2(rng.integers(-20, 20, size=(N, 1)))
        a = torch.from_numpy(A).to(dev)
        b = torch.from_numpy(Bm).to(dev)
        c_ref = torch.full((M, N), np.nan, dtype=torch.float64, device=dev)
        c_new = torch.full((M, N), np.nan, dtype=torch.float64, device=dev)
        st = lib.isdf_gemm_f64(a.data_ptr(), b.data_ptr(), c_ref.data_ptr(), M, N, K, K, K, N, 1.0, 5, 1,
                               ctypes.c_void_p(stream))
        assert st == B_.ISDF_OK, lib.isdf_last_error(None)
        st = lib.isdf_gemm_f64_noalloc(a.data_ptr(), b.data_ptr(), c_new.data_ptr(), M, N, K, K, K, N, 1.0, 5,
                                       ctypes.c_void_p(stream))
        assert st == B_.ISDF_OK, lib.isdf_last_error(None)
        torch.cuda.synchronize()
        ref = c_ref.cpu().numpy()
        new = c_new.cpu().numpy()
        assert np.all(np.isfinite(new))
        assert np.all(np.abs(new - ref) <= _bound(A, Bm))
        assert np.all(np.abs(new - A @ Bm.T) <= _bound(A, Bm))


def test_noalloc_rejects_operands_beyond_the_static_array():
    import torch

    from paper_2404_09373_gb300 import isdf as B_

    lib = B_.load_library()
    cap = lib.isdf_gemm_f64_noalloc_capacity()
    assert cap == 32 << 20
    dev = torch.device("cuda:0")
    M, N, K = 2048, 2048, 1024  # ~42 MB of digit planes > 32 MiB
    a = torch.zeros((M, K), dtype=torch.float64, device=dev)
    b = torch.zeros((N, K), dtype=torch.float64, device=dev)
    c = torch.zeros((M, N), dtype=torch.float64, device=dev)
    st = lib.isdf_gemm_f64_noalloc(a.data_ptr(), b.data_ptr(), c.data_ptr(), M, N, K, K, K, N, 1.0, 5,
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == B_.ISDF_ERR_ARG
    assert b"static array holds" in lib.isdf_last_error(None)


def test_noalloc_refuses_host_pointers_and_huge_extents_before_any_launch():
    """A host pointer (here a NumPy buffer) would reach the kernels as an
    address; the call refuses it on the host.  Extents whose products would
    overflow the size arithmetic are refused before that arithmetic."""
    import torch

    from paper_2404_09373_gb300 import isdf as B_

    lib = B_.load_library()
    dev = torch.device("cuda:0")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    M, N, K = 64, 48, 96
    A = np.ones((M, K))
    a = torch.from_numpy(A).to(dev)
    b = torch.ones((N, K), dtype=torch.float64, device=dev)
    c = torch.zeros((M, N), dtype=torch.float64, device=dev)
    for pa, pb, pc in ((A.ctypes.data, b.data_ptr(), c.data_ptr()),
                       (a.data_ptr(), b.data_ptr(), np.zeros((M, N)).ctypes.data)):
        st = lib.isdf_gemm_f64_noalloc(pa, pb, pc, M, N, K, K, K, N, 1.0, 5, stream)
        assert st == B_.ISDF_ERR_ARG
        assert b"device pointers" in lib.isdf_last_error(None)
    huge = 1 << 40
    st = lib.isdf_gemm_f64_noalloc(a.data_ptr(), b.data_ptr(), c.data_ptr(), huge, N, huge, huge, huge, N, 1.0, 5,
                                   stream)
    assert st == B_.ISDF_ERR_ARG
    assert b"static array" in lib.isdf_last_error(None)
    torch.cuda.synchronize()
    assert float(c.abs().max()) == 0.0  # nothing ran
    # the entry point still works afterwards
    st = lib.isdf_gemm_f64_noalloc(a.data_ptr(), b.data_ptr(), c.data_ptr(), M, N, K, K, K, N, 1.0, 5, stream)
    assert st == B_.ISDF_OK, lib.isdf_last_error(None)
    torch.cuda.synchronize()
    assert np.array_equal(c.cpu().numpy(), np.full((M, N), float(K)))
