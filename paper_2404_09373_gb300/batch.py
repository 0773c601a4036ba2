"""Batched execution of many independent cells (host orchestration).

1. ``isdf_plan_batch``: one plan per cell; the basis values of every cell
   and every level are evaluated by one launch of each basis kernel.
2. ISDF per cell (selection, fit, Coulomb matrix), every cell on its own
   CUDA stream: a pool of ``n_streams`` host threads keeps cells in flight so that
   small cells, whose kernels cannot fill the GPU, overlap with each other
   and with the large ones; a device-memory budget bounds how many are in
   flight at once, and a finished cell keeps only its exchange inputs
   (``isdf_release_fit``: its basis values, fit and spectra are freed).
3. The exchange builds of all cells -- the per-SCF-iteration part -- are
   captured once into one CUDA graph (``isdf_exchange_graph``, one branch per
   cell) and replayed with each iteration's orbitals.

Every cell keeps its own plan, so results are those of running the cells one
by one up to the rounding of the exchange products (the captured build uses
the same kernels and shapes).
"""
from __future__ import annotations

import threading
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from . import isdf as B


def peak_bytes(system, nip, prefilter=True):
    """Device-memory peak of one cell's ISDF, used only for admission: the
    larger of (a) the selection -- factor columns (FP64) and their 8-digit
    planes, nip columns over the candidates of every level (about half the
    points after the exact prefilter), the candidates' basis-value digit
    planes -- and (b) the Coulomb stage on the finest level, with about half
    the pivots there: ZC (FP64), its half spectra and the two 7-digit operands
    of the spectra product."""
    grids = np.asarray(system["grids"]).reshape(-1, 3)
    ng = [int(np.prod(g)) for g in grids]
    nfun = int(sum(1 if l == 0 else 3 for l in system["shell_l"]))
    frac = 0.5 if prefilter else 1.0
    sel = sum(24 * min(nip, n) * n * frac + 16 * nfun * n * frac for n in ng)
    k = max(1, nip // 2)
    nq = (int(grids[0][0]) // 2 + 1) * int(grids[0][1]) * int(grids[0][2])
    coul = 8 * k * ng[0] + 16 * k * nq + 2 * 14 * k * 2 * nq
    return int(max(sel, coul) + 2 ** 30)


def run_cell(system, C, nip, opts, stream):
    """One cell alone: plan, ISDF, exchange (the reference for the batch)."""
    t0 = time.perf_counter()
    plan = B.isdf_plan(system, opts, stream=stream)
    try:
        piv, _ = B.isdf_select_points(plan, nip)
        B.isdf_fit(plan, piv)
        B.isdf_coulomb(plan)
        t1 = time.perf_counter()
        K, ex = B.isdf_exchange(plan, C)
        t2 = time.perf_counter()
    finally:
        plan.close()
    return {"pivots": piv, "K": K, "Ex": ex, "t_isdf_s": t1 - t0, "t_exchange_s": t2 - t1}


def run_batch(cells, opts=None, n_streams=4, mem_budget=120 * 2 ** 30, iterations=1):
    """Run every (system, C, nip) cell.  Returns (results in input order,
    timings): per cell pivots, K, E_x; timings of the batch plan, the ISDF
    stages, the graph capture and each exchange replay (``iterations`` SCF
    iterations with the cells' orbitals)."""
    import torch

    opts = opts or {"precision": 1, "prefilter": 1}
    dev = torch.cuda.current_device()
    streams = [torch.cuda.Stream(device=dev) for _ in cells]  # one per cell: cells in flight never share one
    t0 = time.perf_counter()
    plans = B.isdf_plan_batch([c[0] for c in cells], opts, streams=[st.cuda_stream for st in streams])
    t_plan = time.perf_counter() - t0
    # the budget never exceeds what the device has free once every cell's
    # basis values are resident (other work of the process holds the rest)
    torch.cuda.empty_cache()
    free_after_plans = torch.cuda.mem_get_info(dev)[0]
    mem_budget = min(mem_budget, int(0.8 * free_after_plans))
    lock = threading.Condition()
    state = {"bytes": 0}
    piv = [None] * len(cells)

    def isdf(i):
        sysd, C, nip = cells[i]
        need = min(peak_bytes(sysd, nip, bool(opts.get("prefilter", 0))), mem_budget)
        with lock:
            while state["bytes"] + need > mem_budget and state["bytes"] > 0:
                lock.wait()
            state["bytes"] += need
        try:
            torch.cuda.set_device(dev)
            p, _ = B.isdf_select_points(plans[i], nip)
            B.isdf_fit(plans[i], p)
            B.isdf_coulomb(plans[i])
            # only the exchange's inputs (X^L, X^N, V) stay for the SCF iterations
            B.isdf_release_fit(plans[i])
            piv[i] = p
        finally:
            with lock:
                state["bytes"] -= need
                lock.notify_all()

    try:
        # largest cells first, so the small ones fill the gaps at the end
        order = sorted(range(len(cells)), key=lambda i: -peak_bytes(cells[i][0], cells[i][2]))
        t1 = time.perf_counter()
        with ThreadPoolExecutor(max_workers=n_streams) as ex:
            for f in [ex.submit(isdf, i) for i in order]:
                f.result()
        torch.cuda.synchronize()
        t_isdf = time.perf_counter() - t1
        t2 = time.perf_counter()
        graph = B.ExchangeGraph(plans, [c[1].shape[1] for c in cells])
        t_capture = time.perf_counter() - t2
        try:
            reps = []
            for _ in range(max(1, iterations)):
                t3 = time.perf_counter()
                Ks, exs = graph.run([c[1] for c in cells])
                reps.append(time.perf_counter() - t3)
        finally:
            graph.close()
    finally:
        for p in plans:
            p.close()
    res = [{"pivots": piv[i], "K": Ks[i], "Ex": exs[i]} for i in range(len(cells))]
    return res, {"plan_s": t_plan, "isdf_s": t_isdf, "capture_s": t_capture, "exchange_replay_s": reps,
                 "wall_s": t_plan + t_isdf + t_capture + reps[0], "device_free_gb_after_plans": free_after_plans / 2 ** 30,
                 "mem_budget_gb": mem_budget / 2 ** 30}
