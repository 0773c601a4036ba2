"""Learned point proposer: kernels against the FP64 oracle network, features
against NumPy, exact top-K, and what the trained network gains.

The gain test trains on seeded displaced 1x1x1 / 2x2x1 cells (labels = the
full greedy selection's picks) and evaluates on held-out 2x2x2 cells: the
oracle's exact no-fit exchange judges the accuracy (learned path against the
full selection), CUDA events the time per SCF iteration at full resolution;
an untrained network must leave a larger residual ratio than the trained one.
"""
import os

import numpy as np
import pytest

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


GOLD_EVAL = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "learned_eval_2x2x2.npz")


def _s_iter(t):
    return (t["plan"] + t["select"] + t["fit"] + t["coulomb"]) / 7.0 + t["exchange"]


def _timed_path(sysd, C, nip, opts, select):
    """One pass of the path with CUDA events around each stage (s)."""
    import torch

    ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
    ev[0].record()
    plan = B.isdf_plan(sysd, opts)
    ev[1].record()
    try:
        select(plan)
        ev[3].record()
        B.isdf_coulomb(plan)
        ev[4].record()
        K, _ = B.isdf_exchange(plan, C)
        ev[5].record()
        torch.cuda.synchronize()
    finally:
        plan.close()
    t = [ev[0].elapsed_time(ev[1]), 0.0, ev[1].elapsed_time(ev[3]), 0.0, ev[3].elapsed_time(ev[4]),
         ev[4].elapsed_time(ev[5])]
    return {"plan": t[0] / 1e3, "select": t[2] / 1e3, "fit": 0.0, "coulomb": t[4] / 1e3, "exchange": t[5] / 1e3}, K


def test_learned_proposer_gains_over_the_full_selection():
    """What the trained network gains over the method without it (the full
    pivoted selection of N_ip points).  The learned path selects 1.1 N_ip
    points among 4x as many proposed candidates.

    Accuracy, judged by the oracle: on the held-out 2x2x2 cell of the
    evaluation geometry (seeded displacements sigma = 0.05, grids of 16 / 8 /
    4 points per cell edge so that the oracle's exact no-fit exchange is
    affordable; 32 orbitals), the learned path's exchange error
    max|K - K_nofit| is no larger than the full selection's.
    Speed: on the 2x2x2 workload at full resolution (96^3 / 48^3 / 24^3,
    N_ip = 4992, 128 orbitals) the learned path's s/iter (ISDF / 7 +
    exchange, CUDA events; the proposal, selection and fit of the learned
    path inside) is lower than the full path's.
    Training cells (1x1x1 and 2x2x1, other seeds) never include the
    evaluation cells."""
    gold = np.load(GOLD_EVAL)
    opts = {"precision": 1, "prefilter": 1, "select_block": 96}
    # ---- accuracy on the held-out cell (reduced resolution)
    per_cell = (16, 8, 4)
    stats = {}
    X, y, w = Lr.collect(Lr.training_cells(24, per_cell=per_cell), neg_per_pos=20, stats=stats)
    params, losses = Lr.train(X, y, w, epochs=40, batch=32768, lr=3e-3)
    assert losses[-1] < 0.7 * losses[0]
    sysd, C, nip = Lr.eval_cell(per_cell=per_cell)
    Kn = gold["K"]
    plan = B.isdf_plan(sysd, opts)
    try:
        piv, _ = B.isdf_select_points(plan, nip)
        B.isdf_fit(plan, piv)
        res_full = float(B.isdf_get(plan, B.GET_FIT_RESIDUAL).reshape(-1, 2)[:, 1].sum())
        B.isdf_coulomb(plan)
        K_full, _ = B.isdf_exchange(plan, C)
        _, info = Lr.select_learned(plan, params, nip, stats["level_density"])
        B.isdf_coulomb(plan)
        K_l, _ = B.isdf_exchange(plan, C)
        untrained = Lr.init_params(123)
        _, info_u = Lr.select_learned(plan, untrained, nip, stats["level_density"], repair=0)
    finally:
        plan.close()
    err_full = float(np.max(np.abs(K_full - Kn)))
    err_l = float(np.max(np.abs(K_l - Kn)))
    print(f"\nheld-out 2x2x2 ({per_cell} per cell): |K - K_nofit| full {err_full:.3e} (N_ip {nip}), learned "
          f"{err_l:.3e} ({info['n_selected']} of {info['ncand']} candidates, ratio {info['residual_ratio']:.3g}, "
          f"repairs {info['repairs']}, fallback {info['fallback']}); residual trace full {res_full:.4g}, learned "
          f"{info['residual_trace']:.4g}; untrained ratio {info_u['residual_ratio']:.3g}")
    assert not info["fallback"]
    assert err_l <= err_full
    assert info_u["residual_ratio"] > info["residual_ratio"]
    # ---- speed at full resolution
    stats48 = {}
    X, y, w = Lr.collect(Lr.training_cells(40), neg_per_pos=20, stats=stats48)
    params48, _ = Lr.train(X, y, w, epochs=30, batch=65536, lr=3e-3)
    sysd, C, nip = S.config(2)

    def full(plan):
        p_, _ = B.isdf_select_points(plan, nip)
        B.isdf_fit(plan, p_)

    def learned(plan):
        _, inf = Lr.select_learned(plan, params48, nip, stats48["level_density"])
        assert not inf["fallback"]

    for _ in range(2):  # the second pass of each is timed (the first meets new product shapes)
        t_full, K_f = _timed_path(sysd, C, nip, opts, full)
        t_l, K_l2 = _timed_path(sysd, C, nip, opts, learned)
    print(f"2x2x2 full resolution: s/iter full {_s_iter(t_full):.4f}, learned {_s_iter(t_l):.4f}; "
          f"max|K_learned - K_full| {np.max(np.abs(K_l2 - K_f)):.3e}")
    assert _s_iter(t_l) < _s_iter(t_full)


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
