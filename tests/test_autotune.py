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
             "input_staging": {"deflate": {"format": 3, "best": 1}, "byte_rle": {"format": 6, "best": 1}},
             "staging_depth": {"best": [2048, 4]}, "chunk_mapping": {"best": [14, 32]}}
    p = tmp_path / "t.json"
    p.write_text(json.dumps(table))
    try:
        done = autotune.apply(str(p), n_chunks=10, family="rle_v2")
        assert done["batch_ctas_per_sm"] == 2 and done["parts_per_chunk"] == 8
        assert done["staging_depth"] == [2048, 4] and codag.codag_get_batch_staging() == (2048, 4)
        assert done["chunk_mapping"] == [14, 32] and codag.codag_get_batch_split() == (14, 32)
        assert codag.codag_get_input_staging(3) == 1 and codag.codag_get_input_staging(7) == 1
        done = autotune.apply(str(p), n_chunks=11, family="rle_v2")
        assert "parts_per_chunk" not in done
    finally:
        codag.codag_set_batch_ctas_per_sm(0)
        codag.codag_set_batch_staging(0, 0)
        codag.codag_set_batch_split(0, 0)
        codag.codag_set_parts_per_chunk(0)
        for f in (3, 6, 7):
            codag.codag_set_input_staging(f, 0)


def test_joint_batch_selection_over_shape_and_ctas():
    """The batch sweep's candidates are (slot, slots, ctas) triples; the
    fastest median wins and a near-tie goes to the smaller ring."""
    import paper_2307_03760_gb300 as codag
    from paper_2307_03760_gb300 import autotune
    shapes = codag.codag_batch_staging_shapes()
    cands = [(a, b, k) for a, b in shapes for k in autotune.BATCH_CTAS]
    fake = {c: 10.0 + abs(c[2] - 4) + (0.5 if c[0] == 1024 else 1.0) for c in cands}
    state = {}
    t = autotune.sweep(lambda: None, cands, lambda c: state.update(c=c), reps=3, warmup=0,
                       timer=lambda fn: fake[state["c"]])
    assert autotune.choose(t)[0] == (1024, 4, 4)
    fake[(512, 8, 4)] = fake[(1024, 4, 4)]
    t = autotune.sweep(lambda: None, cands, lambda c: state.update(c=c), reps=3, warmup=0,
                       timer=lambda fn: fake[state["c"]])
    assert autotune.choose(t)[0] == (512, 8, 4)
    assert autotune._key((1024, 4, 4)) == "1024x4x4"


def test_split_rules_offered_are_accepted():
    """Every split rule the sweep offers is one the library takes."""
    import paper_2307_03760_gb300 as codag
    from paper_2307_03760_gb300 import autotune
    assert (16, 16) in autotune.SPLIT_RULES and (16, 1) in autotune.SPLIT_RULES
    try:
        for r in autotune.SPLIT_RULES:
            codag.codag_set_batch_split(*r)
            assert codag.codag_get_batch_split() == r
    finally:
        codag.codag_set_batch_split(0, 0)


def test_committed_table_entries_are_valid():
    """The committed GB300 table names a compiled ring shape and a valid
    split rule, and records the sweeps they came from."""
    import json
    import os

    import paper_2307_03760_gb300 as codag
    from paper_2307_03760_gb300 import autotune
    if not os.path.exists(autotune.DEFAULT_TABLE):
        return
    table = json.load(open(autotune.DEFAULT_TABLE))
    if "staging_depth" not in table:
        return
    assert tuple(table["staging_depth"]["best"]) in codag.codag_batch_staging_shapes()
    assert tuple(table["chunk_mapping"]["best"]) in autotune.SPLIT_RULES
    assert len(table["sweeps"]["batch_staging_x_ctas"]) == \
        len(codag.codag_batch_staging_shapes()) * len(autotune.BATCH_CTAS)
    assert len(table["sweeps"]["batch_split"]) == len(autotune.SPLIT_RULES)


def test_reselect_applies_choose_to_recorded_sweeps():
    """Near-ties (within 1%) go to the smaller setting, from the medians a
    tuning table records; no GPU involved."""
    from paper_2307_03760_gb300 import autotune
    table = {
        "rle_parts": {"rle_v2": {"chunks": 10, "best": 0, "ms": 0}},
        "input_staging": {"deflate": {"format": 3, "best": 1, "ms": 0}},
        "staging_depth": {"best": [0, 0], "ms": 0}, "batch_ctas_per_sm": {"best": 0, "ms": 0},
        "chunk_mapping": {"best": [0, 0], "ms": 0},
        "sweeps": {
            "rle_v2_parts": {"4": 0.999, "5": 0.995, "6": 0.990, "8": 1.2},
            "deflate_input_staging": {"0": 12.5, "1": 29.5},
            "batch_staging_x_ctas": {"1024x4x3": 76.0, "1024x4x8": 75.5, "2048x4x2": 80.0, "256x8x1": 130.0},
            "batch_split": {"16x1": 72.6, "16x16": 72.9, "12x32": 79.0},
        },
    }
    t = autotune.reselect(table)
    assert t["rle_parts"]["rle_v2"]["best"] == 4  # 0.999 is within 1% of 0.990
    assert t["input_staging"]["deflate"]["best"] == 0
    assert t["staging_depth"]["best"] == [1024, 4] and t["batch_ctas_per_sm"]["best"] == 3
    assert t["chunk_mapping"]["best"] == [16, 1]
    assert autotune.choose({1: [1.0], 2: [0.95]})[0] == 2  # 5% apart: not a tie
