"""The batched path: isdf_plan_batch (one basis launch for every cell and
level), ISDF per cell on concurrent streams, and the exchange builds of all
cells captured into one CUDA graph and replayed.

Checked against the FP64 oracle cell by cell on a reduced batch that holds
every cell size of the batched workload (1x1x1, 1x1x2, 1x2x2, 2x2x2 diamond
supercells, seeded displacements sigma = 0.1 bohr, three levels scaled with
the cell), and against running each cell alone."""
import numpy as np
import pytest

import oracle
from paper_2404_09373_gb300 import batch as Bt
from paper_2404_09373_gb300 import isdf as B
from paper_2404_09373_gb300 import systems as S

pytestmark = pytest.mark.gpu


def reduced_batch(nip_per_n=2):
    """One cell of each size, 16/8/4 points per cell edge, N_ip = 2N."""
    cells = S.batch_cells(sigma=0.1, n_each=1, per_cell=(16, 8, 4))
    return [(sysd, C, nip_per_n * S.nbasis(sysd)) for sysd, C, _ in cells]


@pytest.fixture(scope="module")
def batch_and_oracle():
    cells = reduced_batch()
    res, timing = Bt.run_batch(cells, opts={"precision": 1, "prefilter": 1, "select_block": 64}, n_streams=3,
                               iterations=2)
    refs = [oracle.run(sysd, C, nip) for sysd, C, nip in cells]
    return cells, res, timing, refs


def test_batched_cells_match_the_oracle(batch_and_oracle):
    cells, res, timing, refs = batch_and_oracle
    assert sorted({tuple(c[0]["grids"][0]) for c in cells}) == [(16, 16, 16), (16, 16, 32), (16, 32, 32), (32, 32, 32)]
    for (sysd, C, nip), r, o in zip(cells, res, refs):
        natom = sysd["xyz"].shape[0]
        np.testing.assert_array_equal(r["pivots"], o["pivots"])
        assert np.max(np.abs(r["K"] - o["K"])) <= 1e-6
        assert abs(r["Ex"] - o["Ex"]) / natom <= 1e-6
    assert len(timing["exchange_replay_s"]) == 2


def test_batch_equals_cell_by_cell(batch_and_oracle):
    import torch

    cells, res, _, _ = batch_and_oracle
    stream = torch.cuda.Stream()
    opts = {"precision": 1, "prefilter": 1, "select_block": 64}
    for (sysd, C, nip), r in zip(cells, res):
        ref = Bt.run_cell(sysd, C, nip, opts, stream.cuda_stream)
        np.testing.assert_array_equal(r["pivots"], ref["pivots"])
        assert np.max(np.abs(r["K"] - ref["K"])) <= 1e-12 * max(1.0, np.max(np.abs(ref["K"])))
        assert abs(r["Ex"] - ref["Ex"]) <= 1e-12 * abs(ref["Ex"])


def test_plan_batch_basis_equals_single_plans():
    """One k_tab1d and one k_phi launch for all cells and levels give the same
    basis values as plan-by-plan evaluation, bit for bit."""
    cells = reduced_batch()
    plans = B.isdf_plan_batch([c[0] for c in cells])
    try:
        for (sysd, _, _), pb in zip(cells, plans):
            p1 = B.isdf_plan(sysd)
            try:
                for lev in range(3):
                    np.testing.assert_array_equal(B.isdf_get(pb, B.GET_PHI_LEVEL0 + lev),
                                                  B.isdf_get(p1, B.GET_PHI_LEVEL0 + lev))
            finally:
                p1.close()
    finally:
        for p in plans:
            p.close()


@pytest.mark.parametrize("occ", [False, True])
def test_exchange_graph_replays_with_new_orbitals(occ):
    """A captured graph of several cells' exchange builds, replayed with
    scaled orbitals: K is quadratic in C (K(2C) = 4K(C)), and each replay
    equals the plan's own isdf_exchange / isdf_exchange_occ."""
    cells = reduced_batch()[:3]
    plans = B.isdf_plan_batch([c[0] for c in cells], {"precision": 1})
    try:
        for p, (sysd, C, nip) in zip(plans, cells):
            piv, _ = B.isdf_select_points(p, nip)
            B.isdf_fit(p, piv)
            B.isdf_coulomb(p)
        g = B.ExchangeGraph(plans, [c[1].shape[1] for c in cells], occ=occ)
        try:
            out1, ex1 = g.run([c[1] for c in cells])
            out2, ex2 = g.run([2.0 * c[1] for c in cells])
        finally:
            g.close()
        for p, (sysd, C, nip), o1, e1, o2, e2 in zip(plans, cells, out1, ex1, out2, ex2):
            ref, eref = B.isdf_exchange_occ(p, C) if occ else B.isdf_exchange(p, C)
            np.testing.assert_allclose(o1, ref, rtol=0, atol=1e-13 * np.abs(ref).max())
            assert abs(e1 - eref) <= 1e-13 * abs(eref)
            scale = 8.0 if occ else 4.0  # K C is cubic in C, K quadratic
            np.testing.assert_allclose(o2, scale * o1, rtol=0, atol=1e-13 * scale * np.abs(o1).max())
            assert abs(e2 - 16.0 * e1) <= 1e-13 * abs(16.0 * e1)
    finally:
        for p in plans:
            p.close()


def test_autotuner_records_measured_split_choices(batch_and_oracle):
    """After the batch, the split-K autotuner holds a measured choice for
    every product shape it met: a power of two between 1 and 64 and a
    positive time."""
    table = B.isdf_autotune_table()
    assert len(table) > 0
    for row in table:
        assert row["splits"] in (1, 2, 4, 8, 16, 32, 64) or row["splits"] >= 1
        assert row["ms"] > 0.0 and row["M"] > 0 and row["N"] > 0 and row["k_tiles"] > 0


@pytest.mark.parametrize("sinc", [0, 1])
def test_release_fit_keeps_the_exchange(sinc, tmp_path):
    """isdf_release_fit frees the basis values, fit and spectra: the exchange
    builds afterwards are bitwise those before, saving still works, and the
    stages that need the basis values refuse with ISDF_ERR_STATE."""
    sysd, C, nip = reduced_batch()[1]
    plan = B.isdf_plan(sysd, {"precision": 1, "prefilter": 1, "coarse_sinc": sinc})
    try:
        nsel = nip // 2 if sinc else nip
        piv, _ = B.isdf_select_points(plan, nsel)
        B.isdf_fit(plan, piv)
        B.isdf_coulomb(plan)
        K1, E1 = B.isdf_exchange(plan, C)
        KC1, _ = B.isdf_exchange_occ(plan, C)
        assert B.load_library().isdf_get_size(plan.handle, B.GET_PHI_LEVEL0) > 0
        B.isdf_release_fit(plan)
        assert B.load_library().isdf_get_size(plan.handle, B.GET_PHI_LEVEL0) == 0
        K2, E2 = B.isdf_exchange(plan, C)
        KC2, _ = B.isdf_exchange_occ(plan, C)
        assert np.array_equal(K1, K2) and E1 == E2 and np.array_equal(KC1, KC2)
        if not sinc:
            B.isdf_save(plan, str(tmp_path / "f.isdf"))
        for call in (lambda: B.isdf_select_points(plan, nsel), lambda: B.isdf_fit(plan, piv),
                     lambda: B.isdf_coulomb(plan)):
            with pytest.raises(B.IsdfError) as e:
                call()
            assert e.value.status == B.ISDF_ERR_STATE
    finally:
        plan.close()
