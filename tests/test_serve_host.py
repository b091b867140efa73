"""Host-side logic of the serving loop (no GPU): the seeded Poisson stream and the summary."""
import math

from paper_2407_19169_gb300 import serve as S


def test_poisson_stream_is_seeded_and_shaped():
    a = S.poisson_requests(rate=50.0, n=4000, seed=9, seeds=[1, 4, 7])
    b = S.poisson_requests(rate=50.0, n=4000, seed=9, seeds=[1, 4, 7])
    assert [(r.arrival, r.side, r.T, r.seed) for r in a] == [(r.arrival, r.side, r.T, r.seed) for r in b]
    gaps = [a[0].arrival] + [a[i].arrival - a[i - 1].arrival for i in range(1, len(a))]
    assert all(g > 0 for g in gaps)
    mean = sum(gaps) / len(gaps)
    assert abs(mean - 1 / 50.0) < 0.1 / 50.0               # exponential with mean 1/rate
    var = sum((g - mean) ** 2 for g in gaps) / len(gaps)
    assert abs(math.sqrt(var) - mean) < 0.1 * mean        # exponential: std = mean
    assert {r.side for r in a} == set(S.SIDES)
    assert all(0.05 <= r.T <= 0.25 for r in a)
    assert [r.seed for r in a[:6]] == [1, 4, 7, 1, 4, 7]


def test_summary_percentiles():
    rs = [S.Result(i, 128, 0.1, 0.0, 0.0, float(i + 1), 10, 100, 0) for i in range(100)]
    s = S.summarize(rs, 100.0)
    assert s["p50_s"] == 50.0 and s["p99_s"] == 99.0 and s["completed"] == 100
    assert abs(s["dof_stage_per_s"] - 3.0 * 100 * 10 * 100 / 100.0) < 1e-9


def test_srpt_round_picks_shortest_until_the_gpu_is_filled():
    remaining = [50.0, 1.0, 7.0, 3.0, 100.0]
    cells = [1 << 20, 1 << 14, 1 << 16, 1 << 16, 1 << 20]
    # the three shortest hold 2^14 + 2 * 2^16 cells < 2^19: the next shortest (50) completes the fill
    assert S.pick_round(remaining, cells, 1 << 19) == [0, 1, 2, 3]
    assert S.pick_round(remaining, cells, 1 << 15) == [1, 3]
    assert S.pick_round(remaining, cells, 1 << 40) == [0, 1, 2, 3, 4]
    assert S.pick_round([2.0, 2.0], [10, 10], 5) == [0]           # ties: the earlier request
