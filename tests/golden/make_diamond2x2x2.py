"""Write the FP64 oracle's results on the 2x2x2 diamond workload.

Workload: 64 C atoms (2x2x2 conventional diamond cells, a = 6.74 bohr, seeded
Gaussian displacements sigma = 0.05 bohr), uncontracted s {0.1, 0.4, 1.6, 6.4}
and p {0.15, 0.6, 2.4} per atom (N = 832), three grid levels 96^3 / 48^3 /
24^3 split at exponents 1.6 and 0.4, n = 128 occupied orbitals, N_ip = 6N =
4992 (inputs from ``systems.config(2)``).

This script calls only ``oracle`` (and the seeded input generator); nothing
here comes from the CUDA path.  It stores, in ``diamond2x2x2_oracle.npz``:
the pivots and pivot values of the greedy selection (Section II.A, Eq. 2),
the number of pivots per level, the exchange matrix K and E_x (Section III.A,
Eq. 8), seeded samples of the Coulomb matrix V (Section II, Eq. 1) and of the
interpolation vectors Xi of every level (Eq. 3), with their indices.  The
wall time of each stage and the host it ran on go to
``diamond2x2x2_oracle.json``.

Run:  python tests/golden/make_diamond2x2x2.py   (about 60 GB of host memory)
      python tests/golden/make_diamond2x2x2.py --augment   (adds cond(CC^T) per
      level to an existing result)
      python tests/golden/make_diamond2x2x2.py --time-sample   (records the time
      of oracle/sample.py's bounded sample on this host beside the full run,
      with all BLAS threads and with one)
"""
from __future__ import annotations

import json
import os
import platform
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import isdf as O  # noqa: E402
from paper_2404_09373_gb300 import systems as S  # noqa: E402

SAMPLE_SEED = 17
N_V_SAMPLES = 20000
N_XI_SAMPLES = 4096


def pivot_conditioning(levels, pivots):
    """cond(CC^T) per level: eigenvalues of M_l[P, P], formed by the oracle's
    own M columns on the basis values at the pivots only."""
    out = []
    for ld, P in zip(levels, O.split_pivots(pivots, len(levels))):
        if P.size == 0:
            out.append(1.0)
            continue
        sub = {"PhiL": ld["PhiL"][:, P], "PhiN": ld["PhiN"][:, P]}
        ev = np.linalg.eigvalsh(O.m_columns(sub, np.arange(P.size)))
        out.append(float(ev[-1] / ev[0]))
    return np.array(out)


def augment(prefix):
    """Add the per-level conditioning to a stored result (same pivots)."""
    sysd, _, _ = S.config(2)
    z = dict(np.load(prefix + ".npz"))
    levels = O._level_data(sysd, O.expand_functions(sysd))
    z["cond_level"] = pivot_conditioning(levels, z["pivots"])
    np.savez_compressed(prefix + ".npz", **z)
    return z["cond_level"]


def make(sysd, C, nip, prefix, col_batch=256, log=print):
    funcs = O.expand_functions(sysd)
    t = {}
    t0 = time.perf_counter()
    levels = O._level_data(sysd, funcs)
    t["basis_s"] = time.perf_counter() - t0
    log(f"basis {t['basis_s']:.1f} s")
    t0 = time.perf_counter()
    sel = O.select_points(levels, nip)
    pivots, dvals = sel["pivots"], sel["dvals"]
    del sel
    t["select_s"] = time.perf_counter() - t0
    nlev = len(levels)
    per = np.bincount(pivots >> O.PIVOT_SHIFT, minlength=nlev)
    log(f"select {t['select_s']:.1f} s, pivots per level {per.tolist()}")
    t0 = time.perf_counter()
    Xi = O.fit(levels, pivots, 0.0, col_batch=col_batch)
    t["fit_s"] = time.perf_counter() - t0
    log(f"fit {t['fit_s']:.1f} s")
    cond = pivot_conditioning(levels, pivots)
    del levels
    t0 = time.perf_counter()
    V = O.coulomb(sysd, Xi, col_batch=col_batch)
    t["coulomb_s"] = time.perf_counter() - t0
    log(f"coulomb {t['coulomb_s']:.1f} s")
    t0 = time.perf_counter()
    XL, XN = O.pivot_factors(sysd, funcs, pivots)
    t["pivot_factors_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    K, Ex = O.exchange(XL, XN, V, C)
    t["exchange_s"] = time.perf_counter() - t0
    log(f"exchange {t['exchange_s']:.1f} s, E_x = {Ex!r}")

    rng = np.random.default_rng(SAMPLE_SEED)
    nv = V.shape[0]
    vi = rng.integers(0, nv, size=N_V_SAMPLES)
    vj = rng.integers(0, nv, size=N_V_SAMPLES)
    xi_idx, xi_val = [], []
    for lev in range(nlev):
        k = Xi[lev].shape[1]
        if k == 0:
            xi_idx.append(np.zeros((0, 2), dtype=np.int64))
            xi_val.append(np.zeros(0))
            continue
        g = rng.integers(0, Xi[lev].shape[0], size=N_XI_SAMPLES)
        c = rng.integers(0, k, size=N_XI_SAMPLES)
        xi_idx.append(np.stack([g, c], axis=1).astype(np.int64))
        xi_val.append(Xi[lev][g, c])
    arrays = {"pivots": pivots, "dvals": dvals, "nip_level": per.astype(np.int64), "K": K,
              "Ex": np.array(Ex), "V_diag": np.diag(V).copy(), "V_i": vi, "V_j": vj, "V_val": V[vi, vj],
              "V_absmax": np.array(np.abs(V).max()), "cond_level": cond}
    for lev in range(nlev):
        arrays[f"xi{lev}_idx"] = xi_idx[lev]
        arrays[f"xi{lev}_val"] = xi_val[lev]
        arrays[f"xi{lev}_absmax"] = np.array(np.abs(Xi[lev]).max() if Xi[lev].size else 0.0)
    np.savez_compressed(prefix + ".npz", **arrays)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    t_isdf = t["basis_s"] + t["select_s"] + t["fit_s"] + t["coulomb_s"] + t["pivot_factors_s"]
    meta = {"workload": "diamond 2x2x2 (64 C), N=832, n=128, grids 96^3/48^3/24^3, N_ip=6N=4992",
            "seed": S.SEED_BASE + 2, "sample_seed": SAMPLE_SEED, "stages": t,
            "s_iter": t_isdf / 7.0 + t["exchange_s"], "host": platform.machine(),
            "cpu_threads": cores, "blas_threads": os.environ.get("OPENBLAS_NUM_THREADS", "all"),
            "numpy": np.__version__, "Ex": Ex, "Ex_per_atom": Ex / sysd["xyz"].shape[0],
            "nip_level": per.tolist()}
    with open(prefix + ".json", "w") as fh:
        json.dump(meta, fh, indent=1)
    return meta


def time_sample(prefix, reps=3):
    """Time the bounded sample of oracle/sample.py on this host (median of
    ``reps``) and record it beside the full run, so that other hosts can
    scale their own sample time to the full run; also the same sample with
    the BLAS limited to one thread (threadpoolctl), for a one-core estimate."""
    from threadpoolctl import threadpool_limits

    from oracle import sample as OS

    sysd, C, _ = S.config(2)
    smp = OS.Sample(sysd, C)
    t = OS.median_seconds(smp, reps)
    with threadpool_limits(limits=1):
        t1 = OS.median_seconds(smp, reps)
    meta = json.load(open(prefix + ".json"))
    meta["sample_s"] = t
    meta["sample_threads"] = OS.threads()
    meta["sample_s_1thread"] = t1
    with open(prefix + ".json", "w") as fh:
        json.dump(meta, fh, indent=1)
    return t


def main():
    args = [a for a in sys.argv[1:] if not a.startswith("--")]
    prefix = args[0] if args else os.path.join(HERE, "diamond2x2x2_oracle")
    if "--augment" in sys.argv:
        print(augment(prefix))
        return
    if "--time-sample" in sys.argv:
        print(time_sample(prefix))
        return
    sysd, C, nip = S.config(2)
    make(sysd, C, nip, prefix, log=lambda m: print(m, flush=True))


if __name__ == "__main__":
    main()
