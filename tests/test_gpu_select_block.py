"""Speculative-block selection (options.select_block > 0) and the FP64-grade
8-digit tensor-core product it is built on.

The block form must give the greedy pivots of Section II.A exactly: every
case compares pivots element by element with the FP64 oracle (or, at full
size, with the step-by-step GPU loop) and the pivot values and K within the
FP64 bars of the parity tests.
"""
import numpy as np
import pytest

import oracle
from paper_2404_09373_gb300 import isdf as B
from paper_2404_09373_gb300 import systems as S
from parity_util import assert_parity, gpu_run

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).to(torch.device("cuda:0"))


@pytest.mark.parametrize("M,N,K", [(200, 70, 700), (129, 64, 33), (1, 1, 1), (300, 5, 1500)])
def test_gemm_8_slices_is_fp64_grade(M, N, K):
    """8 digits, exact level sums: |C - AB^T| <= 2^-52 K max|A_m| max|B_n| + 2^-52 |C|
    against an extended-precision product (long double).  Rows span 40
    binades, K crosses several 256-wide exact chunks and a ragged tail."""
    import torch

    rng = np.random.default_rng(M + 7 * N + 13 * K)
    A = rng.standard_normal((M, K)) * np.exp2(rng.integers(-20, 20, size=(M, 1)))
    Bm = rng.standard_normal((N, K)) * np.exp2(rng.integers(-20, 20, size=(N, 1)))
    A[:, ::7] *= 1e-9  # wide range inside a row as well
    C = torch.zeros((M, N), dtype=torch.float64, device="cuda:0")
    B.isdf_gemm_f64(_dev(A), _dev(Bm), C, alpha=1.0, slices=8)
    got = C.cpu().numpy()
    ref = (A.astype(np.longdouble) @ Bm.T.astype(np.longdouble)).astype(np.float64)
    bound = 2.0 ** -52 * K * np.abs(A).max(axis=1)[:, None] * np.abs(Bm).max(axis=1)[None, :] + 2.0 ** -52 * np.abs(ref)
    assert np.all(np.abs(got - ref) <= bound)


@pytest.fixture(scope="module")
def small():
    sysd, C = S.small_multigrid(per_cell=(16, 8, 4), seed=5)
    o = oracle.run(sysd, C, 300)
    return sysd, C, o


def _stats(sysd, nip, opts, cand=None):
    plan = B.isdf_plan(sysd, opts)
    try:
        piv, dv = B.isdf_select_points(plan, nip, cand=cand)
        st = B.isdf_get(plan, B.GET_SELECT_STATS)
    finally:
        plan.close()
    return piv, dv, st


@pytest.mark.parametrize("sb", [64, 16, 1, 256])
def test_blocked_selection_matches_oracle(small, sb):
    sysd, C, o = small
    g = gpu_run(sysd, C, 300, opts={"select_block": sb})
    assert_parity(g, o, natom=8)
    _, _, st = _stats(sysd, 300, {"select_block": sb})
    assert st[0] >= 1 and st[0] + st[1] <= 300
    if sb >= 16:
        assert st[0] < 300 // 3  # several pivots per block


def test_blocked_selection_ragged_prefilter_and_ties():
    rng = np.random.default_rng(9)
    sysd = S.make_system((1, 1, 2), 0.07, rng, ((10, 12, 9), (6, 6, 5), (2, 4, 3)), (1.6, 0.4))
    C = S.make_orbitals(sysd, 12, rng)
    o = oracle.run(sysd, C, 350)
    g = gpu_run(sysd, C, 350, opts={"select_block": 64, "prefilter": 1})
    assert_parity(g, o, natom=16)
    # exact symmetric ties of the undisplaced single-grid cell
    sysd, C, nip = S.config(1)
    o = oracle.run(sysd, C, nip)
    g = gpu_run(sysd, C, nip, opts={"select_block": 64, "precision": 1})
    assert_parity(g, o, natom=8, k_tol=1e-6, tc=True)


def test_blocked_selection_candidates_and_tol_stop():
    sysd, C = S.small_multigrid(per_cell=(16, 8, 4), seed=31)
    rng = np.random.default_rng(2)
    offs = np.concatenate([[0], np.cumsum([int(np.prod(g)) for g in sysd["grids"]])])
    cand = []
    for lev in range(3):
        n = offs[lev + 1] - offs[lev]
        keep = np.sort(rng.choice(n, size=max(1, n // 3), replace=False))
        cand.append((np.int64(lev) << 40) | keep.astype(np.int64))
    cand = np.concatenate(cand)
    o = oracle.run(sysd, C, 200, cand=cand)
    g = gpu_run(sysd, C, 200, cand=cand, opts={"select_block": 32})
    assert_parity(g, o, natom=8)
    # tolerance stop inside a block (this cell stops before 500 pivots)
    sysd, C = S.small_multigrid(per_cell=(12, 6, 4), seed=8)
    o = oracle.run(sysd, C, 500, tol=1e-4)
    g = gpu_run(sysd, C, 500, tol=1e-4, opts={"select_block": 32})
    assert g["pivots"].size == o["pivots"].size < 500
    assert_parity(g, o, natom=8)


def test_blocked_equals_stepwise_at_benchmark_density():
    """1x1x1 cell of the benchmark family (48^3/24^3/12^3, N_ip = 6N), exact
    prefilter on: the block form returns the step-by-step pivots."""
    rng = np.random.default_rng(S.SEED_BASE + 2)
    sysd = S.make_system((1, 1, 1), 0.05, rng, ((48, 48, 48), (24, 24, 24), (12, 12, 12)), S.LEVEL_EDGES_3)
    nip = 6 * S.nbasis(sysd)
    p0, d0, _ = _stats(sysd, nip, {"prefilter": 1})
    p1, d1, st = _stats(sysd, nip, {"prefilter": 1, "select_block": 64, "precision": 1})
    np.testing.assert_array_equal(p1, p0)
    np.testing.assert_allclose(d1, d0, rtol=1e-9, atol=1e-14 * d0[0])
    assert st[0] < nip // 5


def test_blocked_selection_time_budget(small):
    sysd, _, _ = small
    plan = B.isdf_plan(sysd, {"select_block": 8, "timeout_ms": 1})
    try:
        with pytest.raises(B.IsdfError) as e:
            B.isdf_select_points(plan, 600)
        assert e.value.status == B.ISDF_ERR_TIMEOUT
    finally:
        plan.close()
    # the plan's context stays usable: a fresh plan runs to the end
    plan = B.isdf_plan(sysd, {"select_block": 8})
    try:
        piv, _ = B.isdf_select_points(plan, 100)
        assert piv.size == 100
    finally:
        plan.close()


def test_blocked_full_size_equals_stepwise():
    """2x2x2 diamond (96^3/48^3/24^3, N_ip = 4992) in the benchmark's launch
    configuration: identical pivots to the step-by-step loop."""
    sysd, C, nip = S.config(2)
    p0, d0, _ = _stats(sysd, nip, {"prefilter": 1, "precision": 1})
    p1, d1, st = _stats(sysd, nip, {"prefilter": 1, "precision": 1, "select_block": 64})
    print(f"\nblocked selection: {st[0]} blocks, {st[1]} single steps for {nip} pivots")
    np.testing.assert_array_equal(p1, p0)
    np.testing.assert_allclose(d1, d0, rtol=1e-9, atol=1e-14 * d0[0])
