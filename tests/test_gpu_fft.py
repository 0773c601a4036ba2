"""The double-float 3-D real-to-half-complex transform behind the Coulomb
integrals (Section II, Eq. 1) against numpy.fft.rfftn (FP64), through the C ABI.

Shapes cover radix-4, -2 and -3 stages, one-point axes, several lines per
CTA and a ragged last tile; an unsupported axis (a factor 5) is refused.
The Coulomb and exchange parity tests with options.precision = 1 exercise the
same transform inside the pipeline.
"""
import numpy as np
import pytest

from paper_2404_09373_gb300 import isdf as B

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape,batch", [((96, 96, 96), 3), ((48, 24, 12), 5), ((16, 8, 4), 7), ((2, 4, 6), 11),
                                         ((128, 9, 1), 2), ((3, 3, 3), 1)])
def test_rfft3_matches_numpy(shape, batch):
    import torch

    nx, ny, nz = shape
    rng = np.random.default_rng(nx * 7 + ny * 3 + nz)
    f = rng.standard_normal((batch, nz, ny, nx)) * np.exp2(rng.integers(-10, 10, size=(batch, 1, 1, 1)))
    S = B.isdf_rfft3(torch.from_numpy(f).to("cuda:0")).cpu().numpy()
    ref = np.fft.rfftn(f, axes=(1, 2, 3))
    for b in range(batch):
        # double-float arithmetic: a few 2^-48 per stage, relative to the grid's magnitude
        assert np.max(np.abs(S[b] - ref[b])) <= 1e-12 * np.abs(f[b]).sum()


def test_rfft3_refuses_unsupported_axes():
    import torch

    f = torch.zeros((1, 9, 12, 10), dtype=torch.float64, device="cuda:0")
    with pytest.raises(B.IsdfError) as e:
        B.isdf_rfft3(f)
    assert e.value.status == B.ISDF_ERR_ARG
