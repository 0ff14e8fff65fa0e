"""Autotuner selection logic on the CPU (timing replaced by a fake)."""
from paper_2307_03760_gb300.autotune import choose, sweep


def test_choose_fastest_median_with_small_tie_break():
    assert choose({1: [5.0, 5.1, 9.0], 2: [4.0, 4.2, 4.1], 4: [4.0, 4.1, 4.2]})[0] == 2
    assert choose({8: [1.0], 16: [1.0]})[0] == 8


def test_sweep_sets_each_candidate_before_timing():
    state = {}
    seen = []

    def setter(c):
        state["c"] = c

    def run():
        seen.append(state["c"])

    fake = {1: 3.0, 2: 1.0, 4: 2.0}
    t = sweep(run, [1, 2, 4], setter, reps=3, warmup=1, timer=lambda fn: (fn(), fake[state["c"]])[1])
    assert choose(t)[0] == 2
    assert seen == [1] * 4 + [2] * 4 + [4] * 4
