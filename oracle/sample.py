"""A bounded timing sample of the oracle on one workload (test infrastructure).

TEST INFRASTRUCTURE ONLY: used by the CPU-baseline leg of ``bench.py`` and
by the script that records the oracle's full run.  It adds no arithmetic of
its own: every timed line calls an oracle function as it stands.

A full oracle run of the 2x2x2 diamond workload takes tens of minutes, so the
CPU baseline times a bounded sample of the same work on the same inputs and
scales it by the ratio (full run / sample) measured once on a reference host:
    estimate(host) = T_full(ref) * T_sample(host) / T_sample(ref).
The sample, per call of ``run()``:
  * basis values of every ``stride``-th function on its levels (Section IV,
    AO evaluation);
  * the first ``steps`` greedy steps of the selection over all grid points
    (Section II.A, Eq. 2), using basis values prepared once, untimed;
  * the fit (Eq. 3), Coulomb matrix (Eq. 1), pivot factors and exchange build
    (Section III.A, Eq. 8) on those pivots.
"""
from __future__ import annotations

import time

import numpy as np

from . import isdf as O


class Sample:
    def __init__(self, system, C, steps=8, stride=8):
        self.system, self.C, self.steps, self.stride = system, C, steps, stride
        self.funcs = O.expand_functions(system)
        self.levels = O._level_data(system, self.funcs)  # untimed set-up

    def run(self):
        """Seconds of one sample (wall clock)."""
        sysd, f = self.system, self.funcs
        t0 = time.perf_counter()
        for lev in range(len(sysd["grids"])):
            _, _, G = O.level_sets(f, lev)
            O.basis_on_level(sysd, f, G[:: self.stride], lev)
        sel = O.select_points(self.levels, self.steps)
        Xi = O.fit(self.levels, sel["pivots"], 0.0)
        V = O.coulomb(sysd, Xi)
        XL, XN = O.pivot_factors(sysd, f, sel["pivots"])
        O.exchange(XL, XN, V, self.C)
        return time.perf_counter() - t0


def threads():
    """Host threads this process may use (BLAS uses all of them)."""
    import os

    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()


def median_seconds(sample, reps=3):
    return float(np.median([sample.run() for _ in range(reps)]))
