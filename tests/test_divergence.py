"""The warp divergence measure D (Section 3.1) and the lane efficiency of a
fixed cell-to-thread mapping, on the CPU."""
import itertools

import numpy as np
import pytest

from paper_1309_2710_gb300 import divergence as dv


def test_equal_work_is_one():
    assert np.allclose(dv.warp_D(np.full(96, 7)), 1.0)
    assert dv.lane_efficiency(np.full(96, 7)) == 1.0


def test_one_thread_does_all_work():
    d = np.zeros(32, dtype=int)
    d[5] = 40
    assert dv.warp_D(d)[0] == pytest.approx(1.0 / 32)


def test_worked_example():
    # d_i = i for i = 1..32: sum 528, max 32 -> D = 528 / 1024
    assert dv.warp_D(np.arange(1, 33))[0] == pytest.approx(528.0 / 1024.0)
    # two warps: constant, then 1..32
    D = dv.warp_D(np.concatenate([np.full(32, 3), np.arange(1, 33)]))
    assert D == pytest.approx([1.0, 0.515625])


def test_partial_last_warp_uses_its_own_size():
    d = np.concatenate([np.full(32, 2), [4, 2, 2, 4]])
    D = dv.warp_D(d)
    assert D.shape == (2,)
    assert D[1] == pytest.approx(12.0 / (4 * 4))
    # the lane efficiency counts the partial warp as a full warp slot
    assert dv.lane_efficiency(d) == pytest.approx((64 + 12) / (32 * (2 + 4)))


def test_idle_warp_and_empty_input():
    assert dv.warp_D(np.zeros(40))[0] == 1.0
    assert dv.warp_D([]).shape == (0,)
    assert dv.lane_efficiency([]) == 1.0
    with pytest.raises(ValueError):
        dv.warp_D([1, -1])


def test_other_widths_against_the_definition():
    rng = np.random.default_rng(5)
    d = rng.integers(0, 1000, size=50)
    for w in (1, 4, 16, 50, 64):
        D = dv.warp_D(d, w)
        for g in range(D.size):
            part = d[g * w:(g + 1) * w]
            ref = part.sum() / (part.size * part.max()) if part.max() > 0 else 1.0
            assert D[g] == pytest.approx(ref)


@pytest.mark.parametrize("n,w", [(6, 2), (6, 3), (7, 3), (8, 4)])
def test_sorted_cut_is_the_best_fixed_mapping(n, w):
    """Brute force over every mapping of a few cells onto threads: no order
    has a higher lane efficiency than the cells sorted by count."""
    rng = np.random.default_rng(n * 10 + w)
    for _ in range(3):
        d = rng.integers(1, 50, size=n)
        best = dv.lane_efficiency(np.sort(d)[::-1], w)
        brute = max(dv.lane_efficiency(np.array(p), w) for p in itertools.permutations(d))
        assert best == pytest.approx(brute)


def test_summary_and_histogram():
    rng = np.random.default_rng(9)
    d = rng.integers(100, 400, size=2048 * 32 // 16)
    s = dv.summary(d)
    g, b = s["given_order"], s["sorted_by_count"]
    assert g["warps"] == b["warps"] == d.size // 32
    assert sum(g["hist"]) == g["warps"] and len(g["hist"]) == 20
    assert b["lane_efficiency"] >= g["lane_efficiency"]
    assert b["mean"] > g["mean"]
    assert dv.histogram(np.array([0.0, 0.5, 1.0]), 2).tolist() == [1, 2]
