"""Atom-centred local dense grids (options.local_grids, Section III, Eq. 5)
against the oracle's run_local: the atoms' pivot sequences and the coarser
levels' pivots exactly, the box and r_max, X^L / X^N, V, K, K C and E_x."""
import numpy as np
import pytest

import oracle
from paper_2404_09373_gb300 import isdf as B
from paper_2404_09373_gb300 import systems as S

pytestmark = pytest.mark.gpu


def cell(per_cell=(24, 12, 6), reps=(1, 1, 1), seed=11, sigma=0.05, n_occ_per_atom=2):
    rng = np.random.default_rng(S.SEED_BASE + seed)
    sysd = S.make_system(reps, sigma, rng, tuple((p, p, p) for p in per_cell), S.LEVEL_EDGES_3)
    C = S.make_orbitals(sysd, n_occ_per_atom * sysd["xyz"].shape[0], rng)
    return sysd, C


def gpu_local(sysd, C, nip, opts):
    plan = B.isdf_plan(sysd, opts)
    try:
        piv, dv = B.isdf_select_points(plan, nip)
        piv, dv = piv.copy(), dv.copy()
        B.isdf_fit(plan, piv)
        k = B.isdf_get(plan, B.GET_NIP_LEVEL)
        npiv = int(k.sum())
        V = np.zeros((npiv, npiv))
        B.isdf_coulomb(plan, V)
        K, Ex = B.isdf_exchange(plan, C)
        KC, Ex_occ = B.isdf_exchange_occ(plan, C)
        N = S.nbasis(sysd)
        return {"pivots": piv, "dvals": dv, "nip_level": k, "V": V, "K": K, "Ex": Ex, "KC": KC, "Ex_occ": Ex_occ,
                "XL": B.isdf_get(plan, B.GET_XL).reshape(N, npiv), "XN": B.isdf_get(plan, B.GET_XN).reshape(N, npiv),
                "box": B.isdf_get(plan, B.GET_LOCAL_BOX), "per_atom": B.isdf_get(plan, B.GET_LOCAL_NIP),
                "pivots_lo": B.isdf_get(plan, B.GET_PIVOTS)}
    finally:
        plan.close()


def pivot_gram(o, sysd):
    """Block-diagonal CC^T = M[P, P] over the level-ordered pivots: every
    atom's local block, then every coarser level's, from the oracle's own
    basis values at the pivots."""
    from oracle import isdf as O

    blocks = []
    atoms = o["local_pivots"] >> B.LOCAL_ATOM_SHIFT
    for A, blk in enumerate(o["blocks"]):
        b = o["local_pivots"][atoms == A] & ((1 << B.LOCAL_ATOM_SHIFT) - 1)
        P = np.searchsorted(blk["box_index"], b)
        sub = {"PhiL": blk["PhiL"][:, P], "PhiN": blk["PhiN"][:, P]}
        blocks.append(O.m_columns(sub, np.arange(P.size)))
    funcs = o["funcs"]
    main = o["pivots"]
    for lev in range(1, int(main.max() >> B.PIVOT_SHIFT) + 1 if main.size else 1):
        P = main[(main >> B.PIVOT_SHIFT) == lev] & ((1 << B.PIVOT_SHIFT) - 1)
        if not P.size:
            continue
        L, N, _ = O.level_sets(funcs, lev)
        sub = {"PhiL": O.basis_on_level(sysd, funcs, L, lev)[:, P], "PhiN": O.basis_on_level(sysd, funcs, N, lev)[:, P]}
        blocks.append(O.m_columns(sub, np.arange(P.size)))
    n = sum(b.shape[0] for b in blocks)
    M = np.zeros((n, n))
    c = 0
    for b in blocks:
        M[c:c + b.shape[0], c:c + b.shape[0]] = b
        c += b.shape[0]
    return M


def check(g, o, C, natom, precision, sinc=False, sysd=None):
    nloc = o["local_pivots"].size
    # pivots: every atom's sequence, then the coarser levels' greedy ones
    assert np.array_equal(g["pivots"][:nloc], o["local_pivots"])
    assert np.array_equal(g["pivots"][nloc:], o["pivots"])
    # a pivot value is a difference d_0 - sum L^2: its rounding is relative to
    # the atom's (level's) largest initial residual, not to itself
    atoms = o["local_pivots"] >> B.LOCAL_ATOM_SHIFT
    for A in range(natom):
        ga, oa = g["dvals"][:nloc][atoms == A], o["local_dvals"][atoms == A]
        assert np.max(np.abs(ga - oa), initial=0.0) <= 1e-12 * oa.max()
    assert np.max(np.abs(g["dvals"][nloc:] - o["dvals"])) <= 1e-12 * o["dvals"].max()
    assert np.array_equal(g["per_atom"], np.bincount(o["local_pivots"] >> B.LOCAL_ATOM_SHIFT, minlength=natom))
    b = o["blocks"][0]["box"]
    assert g["box"][0] == pytest.approx(o["r_max"], rel=1e-15) and list(g["box"][1:]) == list(b)
    # the fitted columns (the sinc grid's columns are implicit on the device)
    nf = g["XL"].shape[1]
    assert np.max(np.abs(g["XL"] - o["XL"][:, :nf])) <= 1e-13 and np.max(np.abs(g["XN"] - o["XN"][:, :nf])) <= 1e-13
    if not sinc:
        dV = g["V"] - o["V"]
        if precision == 0:
            vr = np.max(np.abs(dV)) / np.max(np.abs(o["V"]))
            assert vr <= 1e-9, vr
        else:
            # the atoms' Xi = ZC (CC^T)^-1 come from fits conditioned up to
            # ~1e9 (and the coarser levels' V from W (ZC^T v ZC) W): the
            # forward error of V carries that conditioning, so V is compared
            # in the conditioning-free form CC^T dV CC^T (the Coulomb matrix
            # of the pair-density columns ZC)
            M = pivot_gram(o, sysd)
            vr = np.max(np.abs(M @ dV @ M)) / np.max(np.abs(M @ o["V"] @ M))
            assert vr <= 1e-7, vr
    dk = np.max(np.abs(g["K"] - o["K"]))
    assert dk <= 1e-6, dk
    assert abs(g["Ex"] - o["Ex"]) <= 1e-6 * natom
    # the occ-RI route and K C from the dense K: two 5-digit product chains
    assert np.max(np.abs(g["KC"] - g["K"] @ C)) <= 1e-8 * max(1.0, np.max(np.abs(g["KC"])))
    assert abs(g["Ex_occ"] - g["Ex"]) <= 1e-9 * abs(g["Ex"])
    return dk


@pytest.mark.parametrize("precision,block", [(0, 0), (1, 0), (1, 96)])
def test_local_grids_match_oracle(precision, block):
    """1x1x1 displaced cell, grids 24^3/12^3/6^3: per atom a box of 21^3 points
    (r_max = 2.68 bohr at eps_r = 1e-5, alpha_min = 1.6), atoms on the cell
    corner wrap around the cell."""
    sysd, C = cell()
    N = S.nbasis(sysd)
    o = oracle.run_local(sysd, C, 3 * N, local_tol=1e-6, local_cap=64)
    g = gpu_local(sysd, C, 3 * N, {"precision": precision, "local_grids": 1, "local_tol": 1e-6, "local_cap": 64,
                                   "prefilter": 1, "select_block": block})
    check(g, o, C, 8, precision, sysd=sysd)


def test_local_grids_two_cells_and_cap():
    """A 1x1x2 cell with a per-atom cap that binds (16 pivots on every atom)."""
    sysd, C = cell(reps=(1, 1, 2), seed=12)
    N = S.nbasis(sysd)
    o = oracle.run_local(sysd, C, 2 * N, local_tol=1e-9, local_cap=16)
    assert np.all(np.bincount(o["local_pivots"] >> B.LOCAL_ATOM_SHIFT) == 16)
    g = gpu_local(sysd, C, 2 * N, {"precision": 1, "local_grids": 1, "local_tol": 1e-9, "local_cap": 16,
                                   "prefilter": 1, "select_block": 96})
    check(g, o, C, 16, 1, sysd=sysd)


def test_local_grids_with_the_sinc_coarse_level():
    """The paper's full layout: local grids for the sharp functions, the
    coarsest level as the universal sinc grid, a fitted level between."""
    sysd, C = cell(seed=13)
    N = S.nbasis(sysd)
    o = oracle.run_local(sysd, C, 2 * N, local_tol=1e-6, local_cap=64, sinc=True)
    g = gpu_local(sysd, C, 2 * N, {"precision": 1, "local_grids": 1, "coarse_sinc": 1, "local_tol": 1e-6,
                                   "local_cap": 64, "prefilter": 1})
    check(g, o, C, 8, 1, sinc=True, sysd=sysd)


def test_local_grids_at_the_full_resolution():
    """Grids 48^3/24^3/12^3 per cell (the resolution of the 2x2x2 workload):
    boxes of 41^3 points, about 29,000 sphere points per atom; the bench's
    options (tensor-core precision, prefilter, speculative blocks of 96)."""
    sysd, C = cell(per_cell=(48, 24, 12), seed=11)
    N = S.nbasis(sysd)
    o = oracle.run_local(sysd, C, 3 * N, local_tol=1e-8, local_cap=128)
    g = gpu_local(sysd, C, 3 * N, {"precision": 1, "local_grids": 1, "local_tol": 1e-8, "local_cap": 128,
                                   "prefilter": 1, "select_block": 96})
    check(g, o, C, 8, 1, sysd=sysd)


def test_local_grids_refusals():
    sysd, C = cell()
    with pytest.raises(B.IsdfError, match="wider than the cell"):
        B.isdf_plan(sysd, {"local_grids": 1, "local_eps_r": 1e-14})
    one = S.make_system((1, 1, 1), 0.0, None, ((24, 24, 24),), ())
    with pytest.raises(B.IsdfError, match="two grid levels"):
        B.isdf_plan(one, {"local_grids": 1})
    plan = B.isdf_plan(sysd, {"local_grids": 1})
    try:
        # box point 0 (a corner) lies outside the sphere: refused as a pivot
        with pytest.raises(B.IsdfError, match="outside its atom's sphere"):
            B.isdf_fit(plan, np.array([0], dtype=np.int64))
        with pytest.raises(B.IsdfError, match="out of range"):
            B.isdf_fit(plan, np.array([8 << B.LOCAL_ATOM_SHIFT], dtype=np.int64))
        # level-0 candidates of the greedy are refused (the atoms select their own)
        with pytest.raises(B.IsdfError, match="level 0 has no candidates"):
            B.isdf_select_points(plan, 10, cand=np.array([5], dtype=np.int64))
        piv, _ = B.isdf_select_points(plan, 20)
        assert piv.size > 20 and np.all(piv[:-20] >> B.PIVOT_SHIFT == 0)
        with pytest.raises(B.IsdfError, match="learned proposal"):
            B.isdf_features(plan)
    finally:
        plan.close()


def test_local_grids_release_keeps_the_exchange():
    """isdf_release_fit on a local-grid plan frees the atoms' boxes too; the
    exchange afterwards is bitwise the one before and the box stays known."""
    sysd, C = cell(seed=14)
    N = S.nbasis(sysd)
    plan = B.isdf_plan(sysd, {"precision": 1, "local_grids": 1, "prefilter": 1})
    try:
        piv, _ = B.isdf_select_points(plan, 2 * N)
        B.isdf_fit(plan, piv)
        B.isdf_coulomb(plan)
        K1, E1 = B.isdf_exchange(plan, C)
        box = B.isdf_get(plan, B.GET_LOCAL_BOX)
        B.isdf_release_fit(plan)
        K2, E2 = B.isdf_exchange(plan, C)
        assert np.array_equal(K1, K2) and E1 == E2
        assert np.array_equal(B.isdf_get(plan, B.GET_LOCAL_BOX), box)
        with pytest.raises(B.IsdfError):
            B.isdf_select_points(plan, 2 * N)
    finally:
        plan.close()


def test_local_grids_in_a_batch_and_one_exchange_graph():
    """Local-grid plans made by isdf_plan_batch (the atoms' boxes evaluated in
    the batch's one basis launch) and their exchange builds captured into one
    graph give the results of the same cells planned and run one by one."""
    cells = [cell(seed=21), cell(reps=(1, 1, 2), seed=22)]
    opts = {"precision": 1, "local_grids": 1, "prefilter": 1}
    alone = [gpu_local(sysd, C, 2 * S.nbasis(sysd), opts) for sysd, C in cells]
    plans = B.isdf_plan_batch([c[0] for c in cells], opts)
    try:
        for (sysd, C), p, a in zip(cells, plans, alone):
            piv, _ = B.isdf_select_points(p, 2 * S.nbasis(sysd))
            assert np.array_equal(piv, a["pivots"])
            B.isdf_fit(p, piv)
            B.isdf_coulomb(p)
        g = B.ExchangeGraph(plans, [C.shape[1] for _, C in cells])
        try:
            Ks, exs = g.run([C for _, C in cells])
        finally:
            g.close()
        for K, ex, a in zip(Ks, exs, alone):
            # same kernels; a captured product may take another split-K factor
            assert np.max(np.abs(K - a["K"])) <= 1e-9 and abs(ex - a["Ex"]) <= 1e-9 * abs(a["Ex"])
    finally:
        for p in plans:
            p.close()
