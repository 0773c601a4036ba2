"""Learned point proposal for the pivoted-Cholesky selection (host orchestration).

A small network (8 -> 64 -> 64 -> 1, ReLU, logistic) scores every grid point;
the highest-scoring ``factor * N_ip`` points become the candidate list of
``isdf_select_points``.  Everything numeric runs in the library's kernels
(features, fused forward/backward, Adam, BF16 scoring, top-K); this module
only assembles data and loops.

Training data: for seeded displaced cells, the points the full greedy
selection picks are labelled 1, every other point 0; negatives are
subsampled and the loss is class-weighted so both classes weigh the same.

Fallback: after the candidate-restricted selection and the fit, the largest
residual over ALL grid points (the Schur complement the pivots leave,
reported by isdf_fit) is compared with the last pivot value.  The full
greedy run leaves no residual above its last pivot value; if the restricted
run leaves one larger than ``kappa`` times it, the network missed important
points.  A corrective pass then adds the points with the largest fit residual
on the offending levels to the candidates and selects again; if the check
still fails, the full selection is run instead.

Candidates are proposed per level: ``factor * N_ip`` split over the levels
like the pivots of the training cells (pivot density of each level times its
number of points), so that no level is starved by a bias of the scores.
"""
from __future__ import annotations

import time

import numpy as np

from . import isdf as B
from . import systems as S


def training_cells(n_cells, seed0=S.SEED_BASE + 3 * 1000, per_cell=(48, 24, 12), sigma=0.05):
    """Alternating 1x1x1 and 2x2x1 diamond cells, seeded displacements."""
    cells = []
    for j in range(n_cells):
        rng = np.random.default_rng(seed0 + 1000 * j)
        reps = (1, 1, 1) if j % 2 == 0 else (2, 2, 1)
        sysd = S.make_system(reps, sigma, rng, tuple((p, p, p) for p in per_cell), S.LEVEL_EDGES_3)
        cells.append((sysd, 6 * S.nbasis(sysd)))
    return cells


def collect(cells, neg_per_pos=20, seed=0, opts=None, stats=None):
    """Features and labels on the device.  Returns (X, y, w) torch tensors.
    If ``stats`` is a dict it receives the pivot density of every level
    (pivots / points over all training cells), used for the per-level quotas."""
    import torch

    rng = np.random.default_rng(seed)
    Xs, ys = [], []
    piv_per_level = np.zeros(8)
    pts_per_level = np.zeros(8)
    for sysd, nip in cells:
        plan = B.isdf_plan(sysd, opts or {"precision": 1, "prefilter": 1})
        try:
            feat = B.isdf_features(plan)
            piv, _ = B.isdf_select_points(plan, nip)
            offs = np.concatenate([[0], np.cumsum([int(np.prod(g)) for g in sysd["grids"]])])
            idx = offs[(piv >> B.PIVOT_SHIFT).astype(np.int64)] + (piv & ((1 << B.PIVOT_SHIFT) - 1))
        finally:
            plan.close()
        for l, g in enumerate(sysd["grids"]):
            pts_per_level[l] += int(np.prod(g))
        piv_per_level[: len(sysd["grids"])] += np.bincount(piv >> B.PIVOT_SHIFT, minlength=len(sysd["grids"]))
        lab = np.zeros(feat.shape[0], dtype=np.float32)
        lab[idx] = 1.0
        neg = np.flatnonzero(lab == 0)
        take = rng.choice(neg, size=min(neg.size, neg_per_pos * idx.size), replace=False)
        keep = np.concatenate([idx, take])
        Xs.append(feat[keep])
        ys.append(lab[keep])
    if stats is not None:
        nl = int(np.max(np.flatnonzero(pts_per_level)) + 1)
        stats["level_density"] = (piv_per_level[:nl] / pts_per_level[:nl]).tolist()
    X = np.concatenate(Xs).astype(np.float32)
    y = np.concatenate(ys).astype(np.float32)
    npos = float(y.sum())
    w = np.where(y > 0, (y.size - npos) / max(npos, 1.0), 1.0).astype(np.float32)
    dev = torch.device("cuda", torch.cuda.current_device())
    return (torch.from_numpy(X).to(dev), torch.from_numpy(y).to(dev), torch.from_numpy(w).to(dev))


def init_params(seed=0):
    """He-style initial parameters (fan-in scaled normals, zero biases), flat FP32."""
    import torch

    rng = np.random.default_rng(seed)
    parts = [rng.standard_normal((8, 64)) * np.sqrt(2 / 8), np.zeros(64), rng.standard_normal((64, 64)) * np.sqrt(2 / 64),
             np.zeros(64), rng.standard_normal(64) * np.sqrt(1 / 64), np.zeros(1)]
    theta = np.concatenate([p.ravel() for p in parts]).astype(np.float32)
    assert theta.size == B.load_library().isdf_mlp_num_params()
    return torch.from_numpy(theta).to(torch.device("cuda", torch.cuda.current_device()))


def train(X, y, w, epochs=30, batch=65536, lr=3e-3, seed=0, params=None, stream=None):
    """Mini-batch Adam on the library's kernels.  Returns (params, losses)."""
    import torch

    params = init_params(seed) if params is None else params
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    g = torch.Generator(device=X.device).manual_seed(seed)
    losses, step = [], 0
    n = X.shape[0]
    for _ in range(epochs):
        perm = torch.randperm(n, device=X.device, generator=g)
        ep = []
        for b0 in range(0, n, batch):
            sel = perm[b0:b0 + batch]
            step += 1
            ep.append(B.isdf_mlp_train_step(params, m, v, step, lr, X[sel].contiguous(), y[sel].contiguous(),
                                            w[sel].contiguous(), stream=stream))
        losses.append(float(np.mean(ep)))
    return params, losses


def eval_cell(per_cell=(16, 8, 4), n_occ=32, seed=S.SEED_BASE + 4, sigma=0.05):
    """Held-out evaluation cell with the geometry of the learned workload's
    evaluation (2x2x2 diamond, seeded displacements); the training cells are
    1x1x1 and 2x2x1 with other seeds.  Returns (system, C, N_ip = 6N)."""
    rng = np.random.default_rng(seed)
    sysd = S.make_system((2, 2, 2), sigma, rng, tuple((p, p, p) for p in per_cell), S.LEVEL_EDGES_3)
    C = S.make_orbitals(sysd, n_occ, rng)
    return sysd, C, 6 * S.nbasis(sysd)


def quotas(grids, level_density, nip, factor):
    """Candidates per level: factor * nip split like the expected pivots
    (level pivot density from training x level points), capped per level."""
    pts = np.array([int(np.prod(g)) for g in grids], dtype=np.float64)
    dens = np.asarray(level_density, dtype=np.float64)[: pts.size]
    expect = dens * pts
    q = np.ceil(factor * nip * expect / max(expect.sum(), 1e-300)).astype(np.int64)
    return np.minimum(q, pts.astype(np.int64))


def select_learned(plan, params, nip, level_density, factor=4, oversub=1.1, kappa=100.0, repair=1):
    """Candidate-restricted selection + fit with the residual check.

    The learned selection picks ``oversub * nip`` points among ``factor``
    times as many proposed candidates: restricted to the candidates, the
    greedy steps are several times cheaper than over all grid points, and the
    extra points buy back the accuracy the restriction costs (measured by the
    fit's residual trace, the pair-fit error squared, and by the oracle's
    exchange error).  Check: if the largest fit residual over ALL points
    exceeds kappa times the last pivot value, up to ``repair`` corrective
    passes add, on every level whose residual is above the last pivot value,
    the points with the largest fit residual (as many as the level's share of
    the pivots) to the candidates and select and fit again; if the check
    still fails the full selection of ``nip`` points runs (fallback).

    Returns (pivots, info): info has the candidate count, the passes, whether
    the fallback ran, the residual ratio, the residual trace and the
    selection / fit times."""
    t0 = time.perf_counter()
    n_sel = int(round(oversub * nip))
    n_points = int(B.isdf_get(plan, B.GET_NPOINTS)[0])
    q = quotas(plan.system["grids"], level_density, n_sel, factor)
    cand = B.isdf_propose(plan, params, q)
    info = {"quota": q.tolist(), "n_points": n_points, "n_selected": n_sel, "fallback": False, "repairs": 0}
    t_fit = 0.0
    while True:
        piv, dv = B.isdf_select_points(plan, n_sel, cand=cand)
        t1 = time.perf_counter()
        B.isdf_fit(plan, piv)
        t_fit += time.perf_counter() - t1
        res = B.isdf_get(plan, B.GET_FIT_RESIDUAL).reshape(-1, 2)
        dlast = float(dv[-1]) if dv.size else np.inf
        ratio = float(res[:, 0].max()) / dlast if dv.size else np.inf
        ok = ratio <= kappa and piv.size == n_sel
        if ok or info["repairs"] >= repair or not dv.size:
            break
        extra_q = np.where(res[:, 0] > dlast, np.ceil(q / factor), 0).astype(np.int64)
        if extra_q.sum() == 0:
            break
        extra = B.isdf_propose_residual(plan, extra_q)
        cand = np.unique(np.concatenate([cand, extra]))
        info["repairs"] += 1
    t2 = time.perf_counter()
    info.update({"ncand": int(cand.size), "residual_ratio": ratio,
                 "residual_ratio_per_level": (res[:, 0] / dlast).tolist() if dv.size else None,
                 "residual_trace": float(res[:, 1].sum()),
                 "pivots_per_level": np.bincount(piv >> B.PIVOT_SHIFT, minlength=len(q)).tolist(),
                 "t_select_s": t2 - t0 - t_fit, "t_fit_s": t_fit})
    if not ok:
        t3 = time.perf_counter()
        piv, dv = B.isdf_select_points(plan, nip)
        B.isdf_fit(plan, piv)
        info.update(fallback=True, t_fallback_s=time.perf_counter() - t3)
    return piv, info
