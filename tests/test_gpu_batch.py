"""Batched execution of uneven cells on concurrent streams gives the same
pivots, exchange matrices and energies as running each cell alone."""
import numpy as np
import pytest

from paper_2404_09373_gb300 import batch as Bt
from paper_2404_09373_gb300 import systems as S

pytestmark = pytest.mark.gpu


def test_batch_equals_cell_by_cell():
    import torch

    cells = S.batch_cells(sigma=0.1, n_each=2, per_cell=(16, 8, 4))  # 8 cells of four sizes
    res, wall = Bt.run_batch(cells, n_streams=3)
    stream = torch.cuda.Stream()
    for (sysd, C, nip), r in zip(cells, res):
        ref = Bt.run_cell(sysd, C, nip, {"precision": 1, "prefilter": 1}, stream.cuda_stream)
        np.testing.assert_array_equal(r["pivots"], ref["pivots"])
        np.testing.assert_array_equal(r["K"], ref["K"])
        assert r["Ex"] == ref["Ex"]
    assert len({r["K"].shape for r in res}) == 4
