"""Write the exact (no-fit) exchange of the learned proposer's held-out cell.

Cell: ``learn.eval_cell()`` -- 2x2x2 diamond (64 C, seeded displacements
sigma = 0.05 bohr, seed 20240413), the workload's basis (N = 832), grids
32^3 / 16^3 / 8^3 (16 / 8 / 4 points per cell edge), 32 occupied orbitals.
K_nofit is the exchange matrix without any fit, by the occ-RI route of
Section II.A over the multigrid pair densities of Section II.B (the oracle's
``nofit_exchange``); it judges the exchange error of the full and of the
learned selection.  This script calls only the oracle and the seeded input
generators.  Output: ``learned_eval_2x2x2.npz`` (K, E_x).

Run:  python tests/golden/make_learned_eval.py
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2404_09373_gb300 import learn as Lr  # noqa: E402


def main():
    sysd, C, _ = Lr.eval_cell()
    t0 = time.perf_counter()
    K, Ex = oracle.nofit_exchange(sysd, C)
    print(f"no-fit exchange {time.perf_counter() - t0:.1f} s, E_x = {Ex!r}", flush=True)
    np.savez_compressed(os.path.join(HERE, "learned_eval_2x2x2.npz"), K=K, Ex=np.array(Ex))


if __name__ == "__main__":
    main()
