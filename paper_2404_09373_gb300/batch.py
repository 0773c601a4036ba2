"""Batched execution of many independent cells (host orchestration).

Each cell runs the whole path (plan -> select -> fit -> Coulomb -> exchange)
on its own CUDA stream; a pool of host threads keeps ``n_streams`` cells in
flight so that small cells, whose kernels cannot fill the GPU, overlap with
each other and with the large ones.  A device-memory budget bounds how many
cells are in flight at once.  Results are the same as running the cells one
by one: every cell has its own plan and stream, and no kernel is shared.
"""
from __future__ import annotations

import threading
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from . import isdf as B


def peak_bytes(system, nip):
    """Rough device-memory peak of one cell (basis values, selection factor,
    fit buffers and digit planes, spectra), used only for admission."""
    grids = np.asarray(system["grids"]).reshape(-1, 3)
    ng = [int(np.prod(g)) for g in grids]
    nfun = int(sum(1 if l == 0 else 3 for l in system["shell_l"]))
    k = max(1, nip // len(ng))
    return int(8 * nfun * sum(ng) + 8 * 2 * k * ng[0] + 8 * 2 * nip * ng[0] + 2 * 10 * k * ng[0] + 2 ** 30)


def run_cell(system, C, nip, opts, stream):
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


def run_batch(cells, opts=None, n_streams=4, mem_budget=200 * 2 ** 30):
    """Run every (system, C, nip) cell; returns (results in input order, wall s)."""
    import torch

    opts = opts or {"precision": 1, "prefilter": 1}
    dev = torch.cuda.current_device()
    streams = [torch.cuda.Stream(device=dev) for _ in range(n_streams)]
    free = list(range(n_streams))
    lock = threading.Condition()
    state = {"bytes": 0}

    def work(i):
        sysd, C, nip = cells[i]
        need = min(peak_bytes(sysd, nip), mem_budget)
        with lock:
            while state["bytes"] + need > mem_budget and state["bytes"] > 0:
                lock.wait()
            state["bytes"] += need
            sid = free.pop()
        try:
            torch.cuda.set_device(dev)
            return run_cell(sysd, C, nip, opts, streams[sid].cuda_stream)
        finally:
            with lock:
                state["bytes"] -= need
                free.append(sid)
                lock.notify_all()

    # largest cells first, so the small ones fill the gaps at the end
    order = sorted(range(len(cells)), key=lambda i: -peak_bytes(cells[i][0], cells[i][2]))
    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=n_streams) as ex:
        futs = {i: ex.submit(work, i) for i in order}
        res = {i: f.result() for i, f in futs.items()}
    torch.cuda.synchronize()
    return [res[i] for i in range(len(cells))], time.perf_counter() - t0
