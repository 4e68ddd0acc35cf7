"""Wave planning of streamed runs (host logic, CPU only)."""
import random

import pytest

from paper_1409_2700_gb300.stream import block_elems, plan_waves


def test_block_elems():
    assert block_elems(32, 32) == 2 * 32 ** 4
    assert block_elems(16, 96) == 2 * 16 * 16 * 96 * 96


@pytest.mark.parametrize("seed", range(5))
def test_plan_waves_cover_in_order_within_budget(seed):
    rng = random.Random(seed)
    elems = [block_elems(rng.choice(range(16, 97, 8)), rng.choice(range(16, 97, 8))) for _ in range(300)]
    budget = max(elems) * 3 + 17
    waves, offs = plan_waves(elems, budget)
    # waves tile the list in order
    assert waves[0][0] == 0
    for (f0, c0), (f1, _) in zip(waves, waves[1:]):
        assert f0 + c0 == f1
    assert waves[-1][0] + waves[-1][1] == len(elems)
    for first, count in waves:
        used = 0
        for d in range(first, first + count):
            assert offs[d] == used and offs[d] % 32 == 0        # 256-byte aligned, packed
            used += (elems[d] + 31) // 32 * 32
        assert used <= budget
        # a wave closes only when the next dimer would not fit
        if first + count < len(elems):
            assert used + (elems[first + count] + 31) // 32 * 32 > budget


def test_plan_waves_rejects_a_dimer_above_the_budget():
    with pytest.raises(ValueError):
        plan_waves([100, 5000, 100], 4096)


def test_plan_waves_empty():
    assert plan_waves([], 1000) == ([], [])
