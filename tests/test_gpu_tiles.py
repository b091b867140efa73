"""The 2D tile shape (rows per warp item, warps per block) changes only the schedule: every shape
the autotuner may pick, 1-warp blocks and the library's default schedule (0, 0) give bitwise the
same state."""
import numpy as np
import pytest

from paper_2407_19169_gb300 import _native as N
from paper_2407_19169_gb300 import inputs as I

pytestmark = pytest.mark.gpu
TILES = [(8, 2), (16, 4), (32, 8), (64, 2), (128, 4), (8, 1), (0, 0)]


def run(tile, precision, k):
    s = N.Solver(dim=2, nx=90, ny=70, k=k, eq=N.EQ_EULER, bc=(N.BC_OUTFLOW,) * 4, precision=precision,
                 tile_rows=tile[0], tile_warps=tile[1])
    s.set_initial(N.IC_QUADRANT2D, I.quadrant_params(1))
    s.advance_steps(12)
    st, t, n = s.sync()
    assert st == 0 and n == 12
    u, t = s.read_state()
    s.close()
    return u, t


@pytest.mark.parametrize("precision", [N.PREC_FP32_MIXED, N.PREC_FP64])
@pytest.mark.parametrize("k", [1, 2, 3])
def test_tile_shape_does_not_change_the_result(precision, k):
    ref, t_ref = run(TILES[0], precision, k)
    for tile in TILES[1:]:
        u, t = run(tile, precision, k)
        assert t == t_ref, tile
        np.testing.assert_array_equal(u, ref, err_msg=str(tile))
