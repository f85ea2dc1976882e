"""Training schedule of mars_training_step_ends (host logic, no GPU): one
fixed-point update after each warm-up render, then after training iterations
of 1, 2, 4, ... renders that grow in duration (Sec. 4.1 "Fixed-point
iteration", Sec. 5.1), the last one taking what is left."""
import pytest

import paper_2410_20429_gb300 as M


@pytest.mark.parametrize("n,warmup,expected", [
    (32, 3, [1, 1, 1, 1, 2, 4, 8, 14]),
    (35, 3, [1, 1, 1, 1, 2, 4, 8, 17]),
    (16, 3, [1, 1, 1, 1, 2, 4, 6]),
    (64, 3, [1, 1, 1, 1, 2, 4, 8, 16, 30]),
    (4, 1, [1, 1, 2]),
    (16, 1, [1, 1, 2, 4, 8]),
    (3, 3, [1, 1, 1]),
    (1, 0, [1]),
])
def test_schedules(n, warmup, expected):
    assert M.training_schedule(n, warmup) == expected


def test_invariants_over_many_jobs():
    for n in range(1, 200):
        for w in range(0, min(n, 5) + 1):
            s = M.training_schedule(n, w)
            assert sum(s) == n
            assert s[:w] == [1] * w
            rest = s[w:]
            # doubling, and a last iteration at least as long as the one before
            for a, b in zip(rest[:-2], rest[1:-1]):
                assert b == 2 * a
            if len(rest) >= 2:
                assert rest[-1] >= rest[-2]
            if rest:
                assert rest[0] == 1 or len(rest) == 1


def test_out_of_range_renders_close_nothing():
    assert not M.training_step_ends(-1, 3, 10)
    assert not M.training_step_ends(10, 3, 10)
    assert not M.training_step_ends(0, -1, 10)
    assert M.training_step_ends(9, 3, 10)
