"""Host logic of the autotuner: the staged candidate sets (no GPU)."""

from paper_2404_19706_b300.api import Tuning
from paper_2404_19706_b300.tune import SORTS, stage1, stage2


def valid(t: Tuning) -> bool:
    ok_tile = (t.tile_w, t.tile_h) in {(8, 8), (8, 16), (16, 8), (16, 16), (32, 8)}
    return (ok_tile and t.batch in (32, 64) and t.schedule in (0, 1) and 1 <= t.persist_ctas_per_sm <= 8
            and t.sort_digit_bits in (4, 8) and 0 <= t.sort_rank_max <= 2048)


def test_stage1_covers_tile_batch_schedule_grid():
    c = stage1()
    assert len(c) == len(set(c)) == 40
    assert all(valid(t) for t in c)
    assert {(t.tile_w, t.tile_h) for t in c} == {(8, 8), (8, 16), (16, 8), (16, 16), (32, 8)}
    assert {t.batch for t in c} == {32, 64} and {t.schedule for t in c} == {0, 1}
    assert all(t.sort_digit_bits == 8 and t.sort_rank_max == 256 for t in c)  # ranking sort in stage 1


def test_stage2_varies_only_the_sort():
    base = Tuning(16, 8, 64, 1, 2, 8, 0)
    c = stage2(base)
    assert len(c) == len(SORTS) and all(valid(t) for t in c)
    assert all((t.tile_w, t.tile_h, t.batch, t.schedule, t.persist_ctas_per_sm) == (16, 8, 64, 1, 2) for t in c)
    assert {(t.sort_digit_bits, t.sort_rank_max) for t in c} == set(SORTS)
