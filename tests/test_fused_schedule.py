"""The two-step pass's work order, checked on the host with the library's own order and tile
window functions (lbm_fused_schedule_check): every phase once, every wait on an earlier item,
ring slots rewritten only after their readers, and tile windows that cover every pulled cell
(brute force over the plane, periodic wrap included). No GPU."""
import pytest

from paper_2309_08068_gb300 import build as lbm_build
from paper_2309_08068_gb300.lbm import load_library


@pytest.fixture(scope="module")
def lib():
    lbm_build.build()
    return load_library()


SHAPES = [(256, 160), (256, 256), (300, 137), (1024, 64), (17, 500), (255, 300), (7, 7), (1000, 3), (96, 96),
          (2048, 20), (5, 2000), (256, 2)]


@pytest.mark.parametrize("nx,ny", SHAPES)
@pytest.mark.parametrize("tile", [256, 512, 768])
def test_windows_cover_every_pulled_cell(lib, nx, ny, tile):
    assert lib.lbm_fused_schedule_check(nx, ny, 8, 5, 3, tile) == 0


@pytest.mark.parametrize("L", [2, 3, 4, 6])
def test_order_and_waits_for_every_depth(lib, L):
    for R in (L + 1, L + 2, L + 4):
        for nz in range(max(3, L + 1), 48):
            assert lib.lbm_fused_schedule_check(64, 8, nz, R, L, 256) == 0, (nz, R, L)


def test_the_defaults(lib):
    assert lib.lbm_fused_schedule_check(256, 256, 256, 5, 3, 256) == 0  # MM
    assert lib.lbm_fused_schedule_check(256, 256, 256, 6, 4, 512) == 0  # HV


def test_invalid_shapes_are_rejected(lib):
    assert lib.lbm_fused_schedule_check(16, 16, 16, 2, 2, 256) < 0   # R < L + 1
    assert lib.lbm_fused_schedule_check(16, 16, 16, 5, 1, 256) < 0   # L < 2: B(k) would precede A(k+1)
    assert lib.lbm_fused_schedule_check(16, 16, 2, 5, 3, 256) < 0    # nz < 3


@pytest.mark.parametrize("nx,ny", [(16, 16), (17, 16), (28, 28), (29, 30), (31, 45), (256, 256), (300, 137),
                                   (208, 208), (1024, 16), (16, 999), (128, 128), (272, 272)])
def test_tiled_pass_layout(lib, nx, ny):
    """The tiled pass: an extended tile's 16 x 16 positions are distinct cells, a tile cell's
    neighbours lie in its extended tile, and the tiles cover the plane once (ragged last tiles
    included)."""
    assert lib.lbm_tiled_layout_check(nx, ny) == 0


def test_tiled_pass_layout_rejects_small_planes(lib):
    assert lib.lbm_tiled_layout_check(15, 64) < 0
    assert lib.lbm_tiled_layout_check(64, 15) < 0
