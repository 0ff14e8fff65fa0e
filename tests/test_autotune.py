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


def test_apply_loads_every_knob(tmp_path):
    """apply() sets batch CTAs, RLE parts (matching chunk count) and input
    staging; no GPU needed (the setters only record the choice)."""
    import json

    import paper_2307_03760_gb300 as codag
    from paper_2307_03760_gb300 import autotune
    table = {"batch_ctas_per_sm": {"best": 2}, "rle_parts": {"rle_v2": {"chunks": 10, "best": 8}},
             "input_staging": {"deflate": {"format": 3, "best": 1}, "byte_rle": {"format": 6, "best": 1}}}
    p = tmp_path / "t.json"
    p.write_text(json.dumps(table))
    try:
        done = autotune.apply(str(p), n_chunks=10, family="rle_v2")
        assert done["batch_ctas_per_sm"] == 2 and done["parts_per_chunk"] == 8
        assert codag.codag_get_input_staging(3) == 1 and codag.codag_get_input_staging(7) == 1
        done = autotune.apply(str(p), n_chunks=11, family="rle_v2")
        assert "parts_per_chunk" not in done
    finally:
        codag.codag_set_batch_ctas_per_sm(0)
        codag.codag_set_parts_per_chunk(0)
        for f in (3, 6, 7):
            codag.codag_set_input_staging(f, 0)
