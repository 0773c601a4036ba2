"""The tensor-core FP64-accurate GEMM (sliced BF16 digits on tcgen05) against
NumPy FP64, through the C ABI entry point isdf_gemm_f64.

Bound per element (documented in include/isdf.h):
    |C - A B^T| <= 2^-(7 S - 2) * K * max_k|A[m,k]| * max_k|B[n,k]|.
Shapes cover one tile, ragged tails in every dimension, k ranges that cross
the 1024-wide exact chunk, split-K, both digit counts, rows spanning many
binades, and integer data where the product must be exact.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _run(A, B, slices, splits, alpha=1.0):
    import torch

    from paper_2404_09373_gb300 import isdf as B_

    dev = torch.device("cuda:0")
    a = torch.from_numpy(A).to(dev)
    b = torch.from_numpy(B).to(dev)
    c = torch.full((A.shape[0], B.shape[0]), np.nan, dtype=torch.float64, device=dev)
    B_.isdf_gemm_f64(a, b, c, alpha=alpha, slices=slices, splits=splits)
    torch.cuda.synchronize()
    return c.cpu().numpy()


@pytest.mark.parametrize(
    "M,N,K,splits,slices",
    [
        (128, 96, 32, 1, 5),
        (129, 97, 33, 1, 5),
        (300, 200, 1500, 1, 5),
        (300, 200, 1500, 3, 5),
        (257, 130, 2100, 2, 6),
        (40, 20, 5000, 1, 5),
        (1000, 64, 64, 1, 6),
        (300, 200, 1500, 1, 7),
        (129, 97, 700, 2, 7),
    ],
)
def test_ozgemm_within_bound(M, N, K, splits, slices):
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    A = rng.standard_normal((M, K)) * np.exp2(rng.integers(-30, 30, size=(M, 1)))
    B = rng.standard_normal((N, K)) * np.exp2(rng.integers(-30, 30, size=(N, 1)))
    A[:, ::7] *= 1e-6  # mixed magnitudes within a row
    C = _run(A, B, slices, splits)
    ref = A @ B.T
    bound = 2.0 ** -(7 * slices - 2) * K * np.abs(A).max(axis=1)[:, None] * np.abs(B).max(axis=1)[None, :]
    assert np.all(np.isfinite(C))
    assert np.all(np.abs(C - ref) <= bound)


def test_ozgemm_integer_data_is_exact():
    rng = np.random.default_rng(3)
    A = rng.integers(-100, 100, size=(200, 700)).astype(np.float64)
    B = rng.integers(-100, 100, size=(150, 700)).astype(np.float64)
    C = _run(A, B, 5, 1)
    np.testing.assert_array_equal(C, A @ B.T)


def test_ozgemm_zero_rows_and_alpha():
    rng = np.random.default_rng(4)
    A = rng.standard_normal((130, 64))
    B = rng.standard_normal((50, 64))
    A[5] = 0.0
    B[7] = 0.0
    C = _run(A, B, 5, 1, alpha=-2.5)
    ref = -2.5 * (A @ B.T)
    assert np.all(C[5] == 0.0) and np.all(C[:, 7] == 0.0)
    bound = 2.5 * 2.0 ** -33 * 64 * np.abs(A).max(axis=1)[:, None] * np.abs(B).max(axis=1)[None, :]
    assert np.all(np.abs(C - ref) <= bound)


@pytest.mark.parametrize("slices", [5, 8])
def test_expired_pipeline_wait_reports_timeout_and_the_next_call_succeeds(monkeypatch, slices):
    """Failure detection without a GPU fault: ISDF_FAULT=oz_wait makes every
    pipeline wait of the tensor-core kernel give up at once (the host passes
    a zero limit).  The launch records an error code, lets its copies and
    MMAs in flight finish, frees tensor memory and exits; the call returns
    ISDF_ERR_TIMEOUT.  The context stays usable: the same product without
    the injection is correct."""
    from paper_2404_09373_gb300 import isdf as B_

    rng = np.random.default_rng(11)
    A = rng.standard_normal((1024, 4096))
    B = rng.standard_normal((96, 4096))
    monkeypatch.setenv("ISDF_FAULT", "oz_wait")
    with pytest.raises(B_.IsdfError) as e:
        _run(A, B, slices, 1)
    assert e.value.status == B_.ISDF_ERR_TIMEOUT
    monkeypatch.delenv("ISDF_FAULT")
    C = _run(A, B, slices, 1)
    bound = 2.0 ** -(7 * slices - 2) * 4096 * np.abs(A).max(axis=1)[:, None] * np.abs(B).max(axis=1)[None, :]
    assert np.all(np.abs(C - A @ B.T) <= bound)
