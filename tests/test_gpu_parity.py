"""CUDA path (through the C ABI) vs the FP64 oracle, element by element.

Sizes span several 64-wide GEMM tiles and ragged tails; every level count,
orthorhombic (non-cubic) cells, exact pivot ties, candidate lists, the
tolerance stop, a level without pivots, given pivots, device pointers, the
error paths and host-side fault injection are covered.  The full-size
workload (2x2x2 diamond, 96^3/48^3/24^3) is checked on sampled outputs the
oracle computes one by one and on properties that hold at any size.
"""
import os

import numpy as np
import pytest

import oracle
from oracle import isdf as O
from paper_2404_09373_gb300 import isdf as B
from paper_2404_09373_gb300 import systems as S
from parity_util import assert_parity, gpu_run

pytestmark = pytest.mark.gpu

TWO_ATOMS = np.array([[0.1, 0.2, 0.3], [0.55, 0.6, 0.7]])


@pytest.fixture(scope="module")
def small():
    sysd, C = S.small_multigrid(per_cell=(16, 8, 4), seed=5)
    o = oracle.run(sysd, C, 300)
    return sysd, C, o


def test_basis_values_match_oracle(small):
    sysd, C, o = small
    plan = B.isdf_plan(sysd)
    try:
        f = O.expand_functions(sysd)
        for lev in range(3):
            L, N, _ = O.level_sets(f, lev)
            ref = O.basis_on_level(sysd, f, np.concatenate([L, N]), lev)
            got = B.isdf_get(plan, B.GET_PHI_LEVEL0 + lev).reshape(ref.shape)
            assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))
    finally:
        plan.close()


def test_small_multigrid_parity(small):
    sysd, C, o = small
    g = gpu_run(sysd, C, 300)
    assert_parity(g, o, natom=8)


def test_ragged_orthorhombic_cell():
    rng = np.random.default_rng(9)
    sysd = S.make_system((1, 1, 2), 0.07, rng, ((10, 12, 9), (6, 6, 5), (2, 4, 3)), (1.6, 0.4))
    C = S.make_orbitals(sysd, 12, rng)
    o = oracle.run(sysd, C, 350)
    g = gpu_run(sysd, C, 350)
    assert_parity(g, o, natom=16)


def test_two_levels_and_given_pivots():
    rng = np.random.default_rng(2)
    sysd = S.make_system((1, 1, 1), 0.05, rng, ((18, 18, 18), (10, 10, 10)), (0.5,))
    C = S.make_orbitals(sysd, 8, rng)
    o = oracle.run(sysd, C, 210)
    g = gpu_run(sysd, C, 210)
    assert_parity(g, o, natom=8)
    # isdf_fit on a pivot set from elsewhere (here: the oracle's, shuffled)
    perm = np.random.default_rng(0).permutation(o["pivots"].size)
    o2 = oracle.run(sysd, C, 0, pivots=o["pivots"][perm])
    g2 = gpu_run(sysd, C, 0, piv=o["pivots"][perm])
    g2["dvals"] = None
    o2["dvals"] = None
    g2["pivots"] = o2["pivots"]
    assert_parity(g2, o2, natom=8)


def test_workload1_single_grid_with_exact_ties():
    """1x1x1 undisplaced diamond, one 48^3 grid, N_ip = 8N = 832 (atoms on
    grid points: the diagonal has exact symmetric ties)."""
    sysd, C, nip = S.config(1)
    o = oracle.run(sysd, C, nip)
    g = gpu_run(sysd, C, nip)
    assert_parity(g, o, natom=8, k_tol=1e-7)


def test_candidate_list_and_tol_stop():
    sysd, C = S.small_multigrid(per_cell=(12, 6, 4), seed=8)
    rng = np.random.default_rng(4)
    codes = []
    for lev, n in enumerate(sysd["grids"]):
        ng = int(np.prod(n))
        g = rng.choice(ng, size=ng // 2, replace=False)
        codes.append((np.int64(lev) << 40) | np.sort(g).astype(np.int64))
    cand = np.concatenate(codes)
    o = oracle.run(sysd, C, 120, cand=cand)
    g = gpu_run(sysd, C, 120, cand=cand)
    assert_parity(g, o, natom=8)
    # tolerance stop: fewer pivots than asked
    o = oracle.run(sysd, C, 500, tol=1e-4)
    g = gpu_run(sysd, C, 500, tol=1e-4)
    assert o["pivots"].size < 500
    assert_parity(g, o, natom=8)


def test_few_pivots_leave_a_level_empty():
    sysd, C = S.small_multigrid(per_cell=(12, 6, 4), seed=3)
    for nip in (1, 3):
        o = oracle.run(sysd, C, nip)
        g = gpu_run(sysd, C, nip)
        assert (np.bincount(o["pivots"] >> 40, minlength=3) == 0).any()
        assert_parity(g, o, natom=8)


def test_device_pointers_give_the_same_results(small):
    import torch

    sysd, C, o = small
    dev = torch.device("cuda:0")
    plan = B.isdf_plan(sysd)
    try:
        piv = torch.zeros(300, dtype=torch.int64, device=dev)
        dv = torch.zeros(300, dtype=torch.float64, device=dev)
        p, d = B.isdf_select_points(plan, 300, piv_out=piv, dval_out=dv)
        B.isdf_fit(plan, p)
        V = torch.zeros((300, 300), dtype=torch.float64, device=dev)
        B.isdf_coulomb(plan, V)
        K = torch.zeros((C.shape[0], C.shape[0]), dtype=torch.float64, device=dev)
        Cd = torch.from_numpy(C).to(dev)
        _, Ex = B.isdf_exchange(plan, Cd, K)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(p.cpu().numpy(), o["pivots"])
        assert np.max(np.abs(K.cpu().numpy() - o["K"])) <= 1e-8
        assert abs(Ex - o["Ex"]) <= 1e-8
    finally:
        plan.close()


def test_call_order_and_argument_errors(small):
    sysd, C, o = small
    plan = B.isdf_plan(sysd)
    try:
        with pytest.raises(B.IsdfError) as e:
            B.isdf_coulomb(plan)
        assert e.value.status == B.ISDF_ERR_STATE
        with pytest.raises(B.IsdfError) as e:
            B.isdf_exchange(plan, C)
        assert e.value.status == B.ISDF_ERR_STATE
        bad = np.array([5, 5], dtype=np.int64)
        with pytest.raises(B.IsdfError) as e:
            B.isdf_fit(plan, bad)
        assert e.value.status == B.ISDF_ERR_ARG
        with pytest.raises(B.IsdfError) as e:
            B.isdf_fit(plan, np.array([(np.int64(3) << 40) | 1], dtype=np.int64))
        assert e.value.status == B.ISDF_ERR_ARG
        # after errors the plan still works
        p, _ = B.isdf_select_points(plan, 300)
        np.testing.assert_array_equal(p, o["pivots"])
    finally:
        plan.close()


@pytest.mark.parametrize("fault,stage,status", [("oom", "plan", B.ISDF_ERR_OOM), ("not_pd", "fit", B.ISDF_ERR_NOT_PD),
                                                ("fft_plan", "coulomb", B.ISDF_ERR_CUFFT)])
def test_host_fault_injection(small, monkeypatch, fault, stage, status):
    """Failures are injected on the host (no GPU fault): the call returns the
    status, the plan can be destroyed, and a fresh plan works."""
    sysd, C, o = small
    monkeypatch.setenv("ISDF_FAULT", fault)
    if stage == "plan":
        with pytest.raises(B.IsdfError) as e:
            B.isdf_plan(sysd)
        assert e.value.status == status
    else:
        plan = B.isdf_plan(sysd)
        p, _ = B.isdf_select_points(plan, 50)
        with pytest.raises(B.IsdfError) as e:
            B.isdf_fit(plan, p)
            B.isdf_coulomb(plan)
        assert e.value.status == status
        plan.close()
    monkeypatch.delenv("ISDF_FAULT")
    g = gpu_run(sysd, C, 300)
    assert_parity(g, o, natom=8)


def test_selection_time_budget(small):
    """options.timeout_ms ends the device loop early with ISDF_ERR_TIMEOUT; the
    pivots found so far are the oracle's prefix."""
    sysd, C, o = small
    plan = B.isdf_plan(sysd, {"timeout_ms": 1})
    try:
        with pytest.raises(B.IsdfError) as e:
            B.isdf_select_points(plan, 300)
        assert e.value.status == B.ISDF_ERR_TIMEOUT
    finally:
        plan.close()


def test_exact_prefilter_equals_full_greedy():
    """options.prefilter = 1 drops points whose initial residual is below tau
    and certifies the result; pivots and K equal the oracle's full greedy."""
    sysd, C = S.small_multigrid(per_cell=(16, 8, 4), seed=12)
    o = oracle.run(sysd, C, 260)
    g = gpu_run(sysd, C, 260, opts={"prefilter": 1})
    assert_parity(g, o, natom=8)
    sysd, C, nip = S.config(1)  # nothing can be dropped here: full run
    o = oracle.run(sysd, C, nip)
    g = gpu_run(sysd, C, nip, opts={"prefilter": 1})
    assert_parity(g, o, natom=8, k_tol=1e-7)


# --------------------------------------------------------------------------- tensor-core path


def test_tensor_core_path_small(small):
    """options.precision = 1: fit, Coulomb products on tcgen05 with sliced BF16
    digits.  Selection is unchanged (FP64), so pivots match exactly; K and E_x
    meet max|dK| <= 1e-6 Ha and |dE_x| <= 1e-6 Ha/atom; Xi and V meet the
    conditioning-aware bounds of assert_tc_parity."""
    sysd, C, o = small
    g = gpu_run(sysd, C, 300, opts={"precision": 1})
    dK = assert_parity(g, o, natom=8, k_tol=1e-6, tc=True)
    assert dK <= 1e-6


def test_tensor_core_path_ragged_and_workload1():
    rng = np.random.default_rng(9)
    sysd = S.make_system((1, 1, 2), 0.07, rng, ((10, 12, 9), (6, 6, 5), (2, 4, 3)), (1.6, 0.4))
    C = S.make_orbitals(sysd, 12, rng)
    o = oracle.run(sysd, C, 350)
    g = gpu_run(sysd, C, 350, opts={"precision": 1})
    assert_parity(g, o, natom=16, k_tol=1e-6, tc=True)
    sysd, C, nip = S.config(1)
    o = oracle.run(sysd, C, nip)
    g = gpu_run(sysd, C, nip, opts={"precision": 1})
    assert_parity(g, o, natom=8, k_tol=1e-6, tc=True)


# --------------------------------------------------------------------------- full size


@pytest.fixture(scope="module")
def workload2():
    sysd, C, nip = S.config(2)
    return sysd, C, nip


def test_workload2_full_size_sampled_and_properties(workload2):
    """2x2x2 diamond, 96^3/48^3/24^3, N = 832, n = 128, N_ip = 6N = 4992 in the
    launch configuration the benchmark times.  Checked: basis values at
    sampled points, the first selection steps against the oracle's own, the
    interpolation identity, symmetry / PSD of V, symmetry of K, E_x < 0."""
    sysd, C, nip = workload2
    plan = B.isdf_plan(sysd)
    try:
        f = O.expand_functions(sysd)
        rng = np.random.default_rng(1)
        # sampled basis values (oracle one by one)
        for lev in range(3):
            L, N, _ = O.level_sets(f, lev)
            rows = np.concatenate([L, N])
            phi = B.isdf_get(plan, B.GET_PHI_LEVEL0 + lev).reshape(rows.size, -1)
            ng = phi.shape[1]
            gs = rng.choice(ng, size=64, replace=False)
            rs = rng.choice(rows.size, size=64)
            for r, g in zip(rs, gs):
                ref = O.basis_on_level(sysd, f, [rows[r]], lev)[0, g]
                assert abs(phi[r, g] - ref) <= 1e-13 * max(1e-3, abs(ref))
        piv, dv = B.isdf_select_points(plan, nip)
        assert piv.size == nip
        # the exact prefilter reproduces the full greedy selection at full size
        plan_f = B.isdf_plan(sysd, {"prefilter": 1})
        try:
            piv_f, dv_f = B.isdf_select_points(plan_f, nip)
        finally:
            plan_f.close()
        np.testing.assert_array_equal(piv_f, piv)
        np.testing.assert_allclose(dv_f, dv, rtol=1e-9, atol=1e-14 * dv[0])
        # first steps of the greedy selection against the oracle
        levels = O._level_data(sysd, f)
        osel = O.select_points(levels, 12)
        np.testing.assert_array_equal(piv[:12], osel["pivots"])
        np.testing.assert_allclose(dv[:12], osel["dvals"], rtol=1e-10)
        del levels
        # pivot values never grow (beyond the tie margin)
        assert np.all(np.diff(dv) <= 1e-9 * dv[:-1] + 1e-13 * dv[0])
        B.isdf_fit(plan, piv)
        k = B.isdf_get(plan, B.GET_NIP_LEVEL)
        lo = B.isdf_get(plan, B.GET_PIVOTS)
        off = 0
        for lev in range(3):
            if k[lev] == 0:
                continue
            xiT = B.isdf_get(plan, B.GET_XI_LEVEL0 + lev).reshape(int(k[lev]), -1)
            g = lo[off:off + k[lev]] & ((1 << 40) - 1)
            sub = xiT[:, g]
            assert np.max(np.abs(sub - np.eye(int(k[lev])))) <= 1e-8
            off += int(k[lev])
        V = np.zeros((nip, nip))
        B.isdf_coulomb(plan, V)
        assert np.max(np.abs(V - V.T)) <= 1e-12 * np.max(np.abs(V))
        sel = rng.choice(nip, size=400, replace=False)
        ev = np.linalg.eigvalsh(V[np.ix_(sel, sel)])
        assert ev.min() >= -1e-10 * ev.max()
        K, Ex = B.isdf_exchange(plan, C)
        assert np.max(np.abs(K - K.T)) <= 1e-10 * np.max(np.abs(K))
        assert Ex < 0.0
    finally:
        plan.close()


def test_threshold_driven_grids_and_isdf_tolerance():
    """The paper's thresholds instead of fixed sizes (Section III, Eq. 6 and
    the eps_ISDF stop of the selection): every level's grid from eps_K, then
    pivots until the largest residual falls below eps_ISDF d_0.  The whole
    path against the oracle run on the same derived grids and tolerance."""
    rng = np.random.default_rng(21)
    sysd = S.make_system((1, 1, 1), 0.05, rng, ((8, 8, 8), (4, 4, 4), (2, 2, 2)), S.LEVEL_EDGES_3)
    sysd["grids"] = B.isdf_grids_for_threshold(sysd, 1e-2).astype(np.int64)
    np.testing.assert_array_equal(sysd["grids"], O.grids_for_threshold(sysd, 1e-2))
    C = S.make_orbitals(sysd, 16, rng)
    cap = 3000
    for prec in (0, 1):
        o = oracle.run(sysd, C, cap, tol=1e-4)
        g = gpu_run(sysd, C, cap, tol=1e-4, opts={"precision": prec, "prefilter": 1, "select_block": 64})
        assert 0 < o["pivots"].size < cap
        assert_parity(g, o, natom=8, k_tol=1e-8 if prec == 0 else 1e-6, tc=prec == 1)


@pytest.mark.parametrize("prec", [0, 1])
def test_checkpoint_resume_gives_the_same_exchange(small, tmp_path, prec):
    """isdf_save after the Coulomb matrix, isdf_load into a fresh plan of the
    same system: the exchange builds (K and the occ-RI output) are bitwise
    those of the original plan, and E_x matches the oracle.  Malformed files
    and a plan of another system are refused with ISDF_ERR_ARG."""
    sysd, C, o = small
    path = str(tmp_path / "factors.isdf")
    plan = B.isdf_plan(sysd, {"precision": prec})
    try:
        with pytest.raises(B.IsdfError) as e:
            B.isdf_save(plan, path)
        assert e.value.status == B.ISDF_ERR_STATE
        piv, _ = B.isdf_select_points(plan, 300)
        B.isdf_fit(plan, piv)
        B.isdf_coulomb(plan)
        K1, E1 = B.isdf_exchange(plan, C)
        KC1, _ = B.isdf_exchange_occ(plan, C)
        B.isdf_save(plan, path)
    finally:
        plan.close()
    plan = B.isdf_plan(sysd, {"precision": prec})
    try:
        B.isdf_load(plan, path)
        K2, E2 = B.isdf_exchange(plan, C)
        KC2, _ = B.isdf_exchange_occ(plan, C)
        np.testing.assert_array_equal(K2, K1)
        np.testing.assert_array_equal(KC2, KC1)
        assert E2 == E1
        assert abs(E2 - o["Ex"]) / 8 <= (1e-8 if prec == 0 else 1e-6)
    finally:
        plan.close()
    raw = open(path, "rb").read()
    bad = tmp_path / "bad.isdf"
    other, _ = S.small_multigrid(per_cell=(12, 6, 4), seed=5)
    for content, sysx in ((raw[:200], sysd), (b"NOTACKPT" + raw[8:], sysd), (raw + b"x", sysd), (raw, other)):
        bad.write_bytes(content)
        plan = B.isdf_plan(sysx)
        try:
            with pytest.raises(B.IsdfError) as e:
                B.isdf_load(plan, str(bad))
            assert e.value.status == B.ISDF_ERR_ARG
            with pytest.raises(B.IsdfError) as e:
                B.isdf_exchange(plan, C)
            assert e.value.status == B.ISDF_ERR_STATE  # the refused load changed nothing
        finally:
            plan.close()


# --------------------------------------------------------------------------- coarse level as the universal sinc grid


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("case", ["three_levels", "two_levels"])
def test_coarse_level_as_sinc_grid_matches_oracle(prec, case):
    """options.coarse_sinc: every point of the coarsest grid is an
    interpolation point with Xi = I (Section III; Section III.A after Eq. 8).
    Pivots of the finer levels, the fitted block of V, V_FU = (xi_P|sinc_g),
    K and E_x against the oracle's run_sinc; the coarse-coarse block of V is
    never formed on the GPU (applied in Fourier space in the exchange)."""
    if case == "three_levels":
        sysd, C = S.small_multigrid(per_cell=(16, 8, 4), seed=5)
        nip, natom = 200, 8
    else:
        rng = np.random.default_rng(2)
        sysd = S.make_system((1, 1, 1), 0.05, rng, ((18, 18, 18), (10, 10, 10)), (0.5,))
        C = S.make_orbitals(sysd, 8, rng)
        nip, natom = 150, 8
    o = oracle.run_sinc(sysd, C, nip)
    k = o["pivots"].size
    plan = B.isdf_plan(sysd, {"precision": prec, "coarse_sinc": 1, "prefilter": 1})
    try:
        piv, dv = B.isdf_select_points(plan, nip)
        np.testing.assert_array_equal(piv, o["pivots"])
        np.testing.assert_allclose(dv, o["dvals"], rtol=1e-9, atol=1e-14 * o["dvals"][0])
        B.isdf_fit(plan, piv)
        V = np.zeros((k, k))
        B.isdf_coulomb(plan, V)
        Vfu = B.isdf_get(plan, B.GET_V_COARSE).reshape(k, -1)
        K, Ex = B.isdf_exchange(plan, C)
        KC, Ex2 = B.isdf_exchange_occ(plan, C)
    finally:
        plan.close()
    scale = np.abs(o["V"]).max()
    vtol = 1e-9 if prec == 0 else 1e-6
    assert np.max(np.abs(V - o["V"][:k, :k])) <= vtol * scale
    assert np.max(np.abs(Vfu - o["V"][:k, k:])) <= vtol * scale
    ktol = 1e-8 if prec == 0 else 1e-6
    assert np.max(np.abs(K - o["K"])) <= ktol
    assert abs(Ex - o["Ex"]) / natom <= ktol
    assert np.max(np.abs(KC - o["K"] @ C)) <= ktol * np.max(np.sum(np.abs(C), axis=0))
    assert abs(Ex2 - Ex) <= 1e-12 * abs(Ex)


def test_coarse_sinc_refuses_coarse_pivots_and_candidates(small):
    sysd, C, o = small
    plan = B.isdf_plan(sysd, {"coarse_sinc": 1})
    try:
        coarse = (np.int64(2) << 40) | np.arange(3, dtype=np.int64)
        with pytest.raises(B.IsdfError) as e:
            B.isdf_select_points(plan, 10, cand=coarse)
        assert e.value.status == B.ISDF_ERR_ARG
        with pytest.raises(B.IsdfError) as e:
            B.isdf_fit(plan, coarse)
        assert e.value.status == B.ISDF_ERR_ARG
    finally:
        plan.close()
    one = S.make_system((1, 1, 1), 0.0, None, ((8, 8, 8),), ())
    with pytest.raises(B.IsdfError) as e:
        B.isdf_plan(one, {"coarse_sinc": 1})
    assert e.value.status == B.ISDF_ERR_ARG
