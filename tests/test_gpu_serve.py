"""Served solves with continuous batching: every result equals the same solve run alone, the
memory budget is respected, and requests arriving during earlier solves are admitted."""
import numpy as np
import pytest

from paper_2407_19169_gb300 import _native as N
from paper_2407_19169_gb300 import inputs as I
from paper_2407_19169_gb300 import serve as S

pytestmark = pytest.mark.gpu
SEEDS = [1, 4, 7, 8, 11, 13]


def test_served_results_equal_alone_under_budget():
    reqs = S.poisson_requests(rate=400.0, n=8, seed=5, seeds=SEEDS, sides=(32, 64), t_range=(0.01, 0.04))
    one = N.Solver.workspace_size(dim=2, nx=64, ny=64, bc=(N.BC_OUTFLOW,) * 4, k=2, eq=N.EQ_EULER,
                                  precision=N.PREC_FP32_MIXED)
    eng = S.Engine(budget_bytes=2.5 * one, chunk_steps=8, keep_states=True, positivity=1)
    results, stats = eng.run(reqs)
    assert len(results) == len(reqs) and all(r.status == 0 for r in results)
    assert stats["peak_bytes"] <= 2.5 * one
    assert stats["peak_active"] >= 2                      # solves overlapped on the device
    for r in results:
        req = reqs[r.rid]
        alone = N.Solver(dim=2, nx=req.side, ny=req.side, bc=(N.BC_OUTFLOW,) * 4, k=2, eq=N.EQ_EULER,
                         precision=N.PREC_FP32_MIXED, positivity=1)
        alone.set_initial(N.IC_QUADRANT2D, I.quadrant_params(req.seed))
        alone.advance_to(req.T)
        ua, ta = alone.read_state()
        assert ta == req.T
        assert np.abs(r.state - ua).sum() <= 1e-12 * np.abs(ua).sum()
    summary = S.summarize(results, max(r.done for r in results))
    assert summary["completed"] == 8 and summary["p99_s"] >= summary["p50_s"] > 0


def test_served_fp64_results_equal_alone():
    # the plain FP64 path steps each resident solve on its own: results equal solo runs bitwise
    reqs = S.poisson_requests(rate=400.0, n=4, seed=6, seeds=SEEDS, sides=(32, 48), t_range=(0.01, 0.03))
    eng = S.Engine(budget_bytes=1e9, chunk_steps=8, keep_states=True, positivity=1, precision=N.PREC_FP64)
    results, stats = eng.run(reqs)
    assert len(results) == len(reqs) and all(r.status == 0 for r in results)
    for r in results:
        req = reqs[r.rid]
        alone = N.Solver(dim=2, nx=req.side, ny=req.side, bc=(N.BC_OUTFLOW,) * 4, k=2, eq=N.EQ_EULER,
                         precision=N.PREC_FP64, positivity=1)
        alone.set_initial(N.IC_QUADRANT2D, I.quadrant_params(req.seed))
        alone.advance_to(req.T)
        ua, ta = alone.read_state()
        assert ta == req.T
        np.testing.assert_array_equal(r.state, ua)
