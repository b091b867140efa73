"""Sizes where the 1D stage kernel's warps loop over several strips (more strips than the bounded
grid has warps: > 152 x 8 x 4 x 28 cells) and where batched warps take several items of one
instance, against the oracle and against solo runs."""
import numpy as np
import pytest

import oracle as O
from paper_2407_19169_gb300 import _native as N
from paper_2407_19169_gb300 import inputs as I

from _helpers import rel_l1

pytestmark = pytest.mark.gpu
INF = float("inf")
NX = 300_007                      # about 10.7k strips for 4864 warps; a ragged last strip


@pytest.mark.parametrize("k", [1, 3])
def test_strip_loop_matches_oracle(k):
    p = O.Problem(dim=1, nx=NX, x0=0.0, x1=1.0, k=k, eq=O.EQ_EULER, bc=(O.BC_PERIODIC,) * 4)
    u0 = I.random_modal_state(p.shape, 40 + k, [(1.0, 2.0), (-0.5, 0.5), (4.0, 6.0)], high_scale=0.02)
    s = N.Solver(dim=1, nx=NX, k=k, eq=N.EQ_EULER, bc=(N.BC_PERIODIC,) * 4)
    s.write_state(u0)
    s.advance_steps(6)
    st, t, n = s.sync()
    assert st == 0 and n == 6
    ug, tg = s.read_state()
    uo, to, _ = O.advance(p, u0, 0.0, INF, 6)
    assert abs(tg - to) <= 1e-12 * to
    assert rel_l1(p, ug, uo) <= 1e-11


def test_batched_item_ranges_equal_solo_runs():
    def make(n, seed):
        s = N.Solver(dim=1, nx=n, k=2, eq=N.EQ_EULER, bc=(N.BC_OUTFLOW,) * 4, precision=N.PREC_FP32_MIXED)
        s.set_initial(N.IC_RIEMANN1D, I.riemann1d_params(seed))
        return s
    sizes = [(200_000, 1), (1_000, 2), (150_002, 4), (37, 1)]
    batch = [make(n, sd) for n, sd in sizes]
    assert N.batch_run(batch, 15) == 0
    for (n, sd), sb in zip(sizes, batch):
        alone = make(n, sd)
        alone.advance_steps(15)
        assert alone.sync()[0] == 0
        ua, ta = alone.read_state()
        ub, tb = sb.read_state()
        assert tb == ta
        assert np.abs(ub - ua).sum() <= 1e-12 * np.abs(ua).sum()
