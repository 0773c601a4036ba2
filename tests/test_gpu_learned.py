"""Learned point proposer: kernels against the FP64 oracle network, features
against NumPy, exact top-K, and what the trained network gains.

The gain test trains on seeded displaced cells (labels = the full greedy
selection's picks), then selects on a held-out cell from 4 N_ip candidates.
Measure: the oracle's exchange error |K - K_nofit| (exact no-fit exchange), for
the learned selection against the full one; an untrained network must trip
the fallback check instead.
"""
import numpy as np
import pytest

import oracle
from oracle import isdf as O
from oracle import mlp as OM
from paper_2404_09373_gb300 import isdf as B
from paper_2404_09373_gb300 import learn as Lr
from paper_2404_09373_gb300 import systems as S

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).to(torch.device("cuda:0"))


def test_mlp_gradient_and_adam_match_fp64_oracle():
    import torch

    rng = np.random.default_rng(3)
    theta = OM.init_params(rng)
    X = rng.standard_normal((3000, 8))
    y = (rng.random(3000) < 0.1).astype(float)
    w = np.where(y > 0, 9.0, 1.0)
    L_ref, g_ref = OM.loss_and_grad(theta, X, y, w)
    p = _dev(theta.astype(np.float32))
    grad = torch.zeros_like(p)
    loss = B.isdf_mlp_train_step(p, None, None, 1, 0.0, _dev(X.astype(np.float32)), _dev(y.astype(np.float32)),
                                 _dev(w.astype(np.float32)), grad_out=grad)
    g = grad.cpu().numpy().astype(np.float64)
    assert abs(loss - L_ref) <= 1e-5 * max(1.0, abs(L_ref))
    assert np.max(np.abs(g - g_ref)) <= 2e-5 * max(1e-3, np.max(np.abs(g_ref)))
    # one Adam step
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    B.isdf_mlp_train_step(p, m, v, 1, 1e-3, _dev(X.astype(np.float32)), _dev(y.astype(np.float32)),
                          _dev(w.astype(np.float32)))
    t_ref, _, _ = OM.adam_step(theta, np.zeros_like(theta), np.zeros_like(theta), g_ref, 1, 1e-3)
    assert np.max(np.abs(p.cpu().numpy() - t_ref)) <= 1e-5


def test_bf16_scores_close_to_fp64_logits():
    import torch

    rng = np.random.default_rng(4)
    theta = OM.init_params(rng)
    X = rng.standard_normal((5000, 8))
    z_ref, _ = OM.forward(theta, X)
    out = torch.zeros(5000, dtype=torch.float32, device="cuda:0")
    B.isdf_mlp_score(_dev(theta.astype(np.float32)), _dev(X.astype(np.float32)), out)
    z = out.cpu().numpy()
    # BF16 weights and activations: relative error of a few 2^-8 of the logit scale
    assert np.max(np.abs(z - z_ref)) <= 0.05 * max(1.0, np.max(np.abs(z_ref)))
    assert np.corrcoef(z, z_ref)[0, 1] > 0.999


def _numpy_features(sysd):
    f = O.expand_functions(sysd)
    feats, d0all = [], []
    levs = O._level_data(sysd, f)
    for lev, ld in enumerate(levs):
        aL = np.sum(ld["PhiL"] ** 2, axis=0)
        aN = np.sum(ld["PhiN"] ** 2, axis=0)
        d0all.append(ld["w"] * aL * (aL + 2 * aN))
    d0max = max(d.max() for d in d0all)
    nlev = len(levs)
    for lev, ld in enumerate(levs):
        n = sysd["grids"][lev]
        aL = np.sum(ld["PhiL"] ** 2, axis=0)
        aN = np.sum(ld["PhiN"] ** 2, axis=0)
        rho = (aL + aN).reshape(n[2], n[1], n[0])
        h = sysd["edges"] / n
        gx = (np.roll(rho, -1, 2) - np.roll(rho, 1, 2)) / (2 * h[0])
        gy = (np.roll(rho, -1, 1) - np.roll(rho, 1, 1)) / (2 * h[1])
        gz = (np.roll(rho, -1, 0) - np.roll(rho, 1, 0)) / (2 * h[2])
        gn = np.sqrt(gx ** 2 + gy ** 2 + gz ** 2).ravel()
        Z, Y, X = np.meshgrid(np.arange(n[2]) * h[2], np.arange(n[1]) * h[1], np.arange(n[0]) * h[0], indexing="ij")
        P = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
        d = P[:, None, :] - sysd["xyz"][None, :, :]
        d -= sysd["edges"] * np.rint(d / sysd["edges"])
        r = np.sort(np.sqrt(np.sum(d * d, axis=2)), axis=1)
        F = np.stack([np.log10(np.maximum(d0all[lev], 1e-300) / d0max) / 10, np.log10(aL + 1e-30) / 10,
                      np.log10(aN + 1e-30) / 10, np.log10(gn + 1e-30) / 10, r[:, 0] / 4, r[:, 1] / 4,
                      aL / (aL + aN + 1e-300), np.full(aL.shape, lev / max(1, nlev - 1))], axis=1)
        feats.append(F)
    return np.concatenate(feats)


def test_features_match_numpy():
    sysd, _ = S.small_multigrid(per_cell=(12, 6, 4), seed=21)
    plan = B.isdf_plan(sysd)
    try:
        got = B.isdf_features(plan)
    finally:
        plan.close()
    ref = _numpy_features(sysd)
    assert got.shape == ref.shape
    assert np.max(np.abs(got - ref)) <= 1e-5


def test_propose_returns_exact_top_k_in_order():
    import torch

    sysd, _ = S.small_multigrid(per_cell=(12, 6, 4), seed=22)
    params = Lr.init_params(5)
    plan = B.isdf_plan(sysd)
    try:
        feat = torch.zeros((int(B.isdf_get(plan, B.GET_NPOINTS)[0]), 8), dtype=torch.float32, device="cuda:0")
        B.isdf_features(plan, feat)
        sc = torch.zeros(feat.shape[0], dtype=torch.float32, device="cuda:0")
        B.isdf_mlp_score(params, feat, sc)
        quota = [200, 90, 0]
        got = B.isdf_propose(plan, params, quota)
    finally:
        plan.close()
    s = sc.cpu().numpy()
    offs = np.concatenate([[0], np.cumsum([int(np.prod(g)) for g in sysd["grids"]])])
    ref = []
    for lev, K in enumerate(quota):
        sl = s[offs[lev]:offs[lev + 1]]
        order = np.lexsort((np.arange(sl.size), -sl))  # score descending, index ascending
        ref.append((np.int64(lev) << 40) | np.sort(order[:K]).astype(np.int64))
    np.testing.assert_array_equal(got, np.concatenate(ref))


def test_learned_proposer_gain_measured_by_oracle_exchange_error():
    per_cell = (24, 12, 6)
    cells = Lr.training_cells(12, per_cell=per_cell)
    stats = {}
    X, y, w = Lr.collect(cells, neg_per_pos=20, stats=stats)
    params, losses = Lr.train(X, y, w, epochs=40, batch=32768, lr=3e-3)
    assert losses[-1] < 0.7 * losses[0]
    # held-out evaluation cell of the same family
    rng = np.random.default_rng(S.SEED_BASE + 4)
    sysd = S.make_system((1, 1, 1), 0.05, rng, tuple((p, p, p) for p in per_cell), S.LEVEL_EDGES_3)
    C = S.make_orbitals(sysd, 16, rng)
    nip = 6 * S.nbasis(sysd)
    Kn, _ = oracle.nofit_exchange(sysd, C)

    def finish(plan):
        B.isdf_coulomb(plan)
        return B.isdf_exchange(plan, C)[0]

    plan = B.isdf_plan(sysd, {"precision": 1, "prefilter": 1})
    try:
        piv_full, _ = B.isdf_select_points(plan, nip)
        B.isdf_fit(plan, piv_full)
        K_full = finish(plan)
        piv_l, info = Lr.select_learned(plan, params, nip, stats["level_density"], factor=4)
        K_l = finish(plan)
        untrained = Lr.init_params(123)
        _, info_u = Lr.select_learned(plan, untrained, nip, stats["level_density"], factor=4)
    finally:
        plan.close()
    err_full = np.max(np.abs(K_full - Kn))
    err_l = np.max(np.abs(K_l - Kn))
    print(f"\nlearned proposer: ncand {info['ncand']} of {info['n_points']} points, residual ratio "
          f"{info['residual_ratio']:.3g}, repairs {info['repairs']}, fallback {info['fallback']}; "
          f"|K - K_nofit|: full {err_full:.3e}, "
          f"learned {err_l:.3e}; untrained ratio {info_u['residual_ratio']:.3g} fallback {info_u['fallback']}")
    assert not info["fallback"]
    assert info["ncand"] * 5 < info["n_points"]
    assert err_l <= 2.0 * err_full + 1e-5
    assert info_u["fallback"] or info_u["residual_ratio"] > info["residual_ratio"]


def test_propose_residual_returns_the_worst_represented_points():
    """After the fit, isdf_propose_residual returns per level the points with
    the largest residual w (M(g,g) - M(g,P) M_PP^-1 M(P,g)) (Section II.A),
    checked against the oracle's residual of the same pivots (FP32 ordering:
    every returned point is within 1e-5 of the K-th largest)."""
    sysd, _ = S.small_multigrid(per_cell=(12, 6, 4), seed=23)
    f = O.expand_functions(sysd)
    levels = O._level_data(sysd, f)
    plan = B.isdf_plan(sysd)
    try:
        piv, _ = B.isdf_select_points(plan, 60)
        B.isdf_fit(plan, piv)
        quota = [25, 10, 5]
        got = B.isdf_propose_residual(plan, quota)
    finally:
        plan.close()
    assert np.all(np.diff(got) > 0)
    per = O.split_pivots(piv, len(levels))
    off = 0
    for lev, ld in enumerate(levels):
        P = per[lev]
        d = O.initial_diagonal(ld)
        if P.size:
            Mc = ld["w"] * O.m_columns(ld, P)
            d = d - np.einsum("gp,gp->g", Mc, np.linalg.solve(Mc[P, :], Mc.T).T)
        g = got[off:off + quota[lev]]
        off += quota[lev]
        assert np.all(g >> 40 == lev)
        kth = np.sort(d)[-quota[lev]]
        assert np.all(d[g & ((1 << 40) - 1)] >= kth - 1e-5 * abs(d).max())
