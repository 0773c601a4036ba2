"""The benchmarked workload against the FP64 oracle, at full size.

2x2x2 diamond (64 C, seeded displacements sigma = 0.05 bohr), N = 832,
n = 128, grids 96^3 / 48^3 / 24^3, N_ip = 6N = 4992, in the launch
configuration bench.py times: tensor-core sliced-BF16 products (precision 1),
the exact prefilter, speculative selection blocks of 96.

Expected values: ``golden/diamond2x2x2_oracle.npz``, written by
``golden/make_diamond2x2x2.py`` from the oracle alone (nothing in it comes
from the CUDA path).  Checked:
  * pivots (order and set) and pivot values of the greedy selection (Eq. 2);
  * K element by element, max|dK| <= 1e-6 Ha, and |dE_x| <= 1e-6 Ha per atom
    (Eq. 8);
  * 20,000 sampled entries of V (Eq. 1) and 4,096 sampled values of Xi per
    level (Eq. 3), within the conditioning-aware bound of the tensor-core
    path, U5 |G| cond(CC^T) relative to the largest entry (parity_util).
"""
import os

import numpy as np
import pytest

from paper_2404_09373_gb300 import isdf as B
from paper_2404_09373_gb300 import systems as S
from parity_util import U5

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "diamond2x2x2_oracle.npz")
BENCH_OPTS = {"precision": 1, "prefilter": 1, "select_block": 96}


@pytest.fixture(scope="module")
def gold():
    return dict(np.load(GOLD))


def test_workload2_in_the_benchmark_configuration_matches_the_oracle(gold):
    import torch

    sysd, C, nip = S.config(2)
    natom = sysd["xyz"].shape[0]
    plan = B.isdf_plan(sysd, BENCH_OPTS)
    try:
        piv, dv = B.isdf_select_points(plan, nip)
        np.testing.assert_array_equal(np.sort(piv), np.sort(gold["pivots"]))
        np.testing.assert_array_equal(piv, gold["pivots"])
        np.testing.assert_allclose(dv, gold["dvals"], rtol=1e-9, atol=1e-14 * gold["dvals"][0])
        B.isdf_fit(plan, piv)
        k = B.isdf_get(plan, B.GET_NIP_LEVEL).astype(np.int64)
        np.testing.assert_array_equal(k, gold["nip_level"])
        V = np.zeros((nip, nip))
        B.isdf_coulomb(plan, V)
        K, Ex = B.isdf_exchange(plan, C)
        dK = float(np.max(np.abs(K - gold["K"])))
        dEx = abs(Ex - float(gold["Ex"])) / natom
        assert dK <= 1e-6, dK
        assert dEx <= 1e-6, dEx
        gmax = S.nbasis(sysd)  # |G_l| <= N on every level (N on the finest)
        cond = float(np.max(gold["cond_level"]))
        dV = float(np.max(np.abs(V[gold["V_i"], gold["V_j"]] - gold["V_val"])) / gold["V_absmax"])
        np.testing.assert_allclose(np.diag(V), gold["V_diag"], rtol=0, atol=U5 * gmax * cond * gold["V_absmax"])
        assert dV <= U5 * gmax * cond, (dV, cond)
        dev = torch.device("cuda", torch.cuda.current_device())
        for lev in range(len(sysd["grids"])):
            if k[lev] == 0:
                continue
            ng = int(np.prod(sysd["grids"][lev]))
            xi = torch.empty(int(k[lev]) * ng, dtype=torch.float64, device=dev)
            B.isdf_get(plan, B.GET_XI_LEVEL0 + lev, xi)
            idx = torch.from_numpy(gold[f"xi{lev}_idx"]).to(dev)
            got = xi.view(int(k[lev]), ng)[idx[:, 1], idx[:, 0]].cpu().numpy()
            del xi
            dxi = float(np.max(np.abs(got - gold[f"xi{lev}_val"])) / gold[f"xi{lev}_absmax"])
            assert dxi <= U5 * gmax * float(gold["cond_level"][lev]), (lev, dxi)
    finally:
        plan.close()
