"""Pins of the oracle's grid resampling (progressive grid scaling, Sec. 5.4):
an affine field stays the same affine field at any resolution, equal sizes
give the grid back, a refinement by an integer factor keeps every source
point, and the result equals PyTorch's trilinear interpolation with corner
alignment (an independent implementation of the same textbook operation)."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.filterwarnings("ignore")


def _affine_grid(G, coef):
    """Affine field a + b x + c y + d z sampled at the grid points of [-1, 1]^3."""
    axes = [np.linspace(-1.0, 1.0, g) for g in G]   # x, y, z
    z, y, x = np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")
    return coef[0] + coef[1] * x + coef[2] * y + coef[3] * z


@pytest.mark.parametrize("Gs,Gd", [((9, 12, 7), (17, 23, 13)), ((33, 33, 33), (20, 25, 41)),
                                   ((5, 5, 5), (160, 3, 9))])
def test_resample_keeps_an_affine_field(orc, Gs, Gd):
    coef = np.array([0.25, 1.5, -2.0, 0.75])
    src = _affine_grid(Gs, coef).astype(np.float32)
    # trilinear weights sum to 1 and reproduce affine functions, so the result
    # is the field at the new points up to the float32 rounding of the inputs
    out = orc.grid_resample(src, Gd)
    ref = _affine_grid(Gd, coef)
    assert np.max(np.abs(out - ref)) < 4 * np.finfo(np.float32).eps * np.max(np.abs(ref))


def test_resample_equal_size_is_identity(orc):
    rng = np.random.default_rng(70)
    src = rng.normal(size=(11, 7, 13, 5)).astype(np.float32)
    out = orc.grid_resample(src, (13, 7, 11))
    assert np.array_equal(out, src.astype(np.float64))


def test_resample_integer_refinement_keeps_source_points(orc):
    rng = np.random.default_rng(71)
    src = rng.normal(size=(6, 9, 5, 3)).astype(np.float32)   # G = (5, 9, 6)
    out = orc.grid_resample(src, (4 * 4 + 1, 3 * 8 + 1, 2 * 5 + 1))
    assert np.array_equal(out[::2, ::3, ::4], src.astype(np.float64))


@pytest.mark.parametrize("Gd", [(21, 14, 30), (6, 5, 4)])
def test_resample_matches_torch_trilinear_align_corners(orc, Gd):
    rng = np.random.default_rng(72)
    src = rng.normal(size=(10, 9, 12, 4)).astype(np.float32)   # [z, y, x, C], G = (12, 9, 10)
    out = orc.grid_resample(src, Gd)
    t = torch.from_numpy(src.astype(np.float64)).permute(3, 0, 1, 2)[None]   # [1, C, D, H, W]
    ref = torch.nn.functional.interpolate(t, size=(Gd[2], Gd[1], Gd[0]), mode="trilinear",
                                          align_corners=True)[0].permute(1, 2, 3, 0).numpy()
    assert np.max(np.abs(out - ref)) < 1e-12
