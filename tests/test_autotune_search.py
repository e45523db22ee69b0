"""The autotuner's coordinate descent on a fake cost (no GPU): it starts at
the defaults, changes one knob at a time keeping the best, never proposes
decreasing bin bounds, and runs each setting once."""
from paper_2502_18497_gb300.autotune import DEFAULT_BINS, SEARCH, coordinate_descent


def test_descends_to_the_cheapest_reachable_setting():
    calls = []

    def cost(bins, cl):
        calls.append((tuple(bins), cl))
        assert all(bins[i] <= bins[i + 1] for i in range(3))
        # separable: cheapest at bins (32, 96, 384, 1024) and cluster 0
        return abs(bins[0] - 32) + abs(bins[1] - 96) + abs(bins[2] - 384) + abs(bins[3] - 1024) + cl / 1000

    best_bins, best_cl, best_ms, seen = coordinate_descent(cost)
    assert best_bins == [32, 96, 384, 1024] and best_cl == 0 and best_ms == 0
    assert calls[0] == (tuple(DEFAULT_BINS), 0)
    assert len(calls) == len(set(calls)) == len(seen)
    assert len(calls) <= 1 + sum(len(v) for v in SEARCH.values())


def test_keeps_the_defaults_when_nothing_is_faster():
    best_bins, best_cl, _, _ = coordinate_descent(lambda bins, cl: 1.0)
    assert tuple(best_bins) == DEFAULT_BINS and best_cl == 0


def test_skips_decreasing_bounds():
    search = {"bin1": (16,), "bin0": (16,)}  # bin1 = 16 < bin0 = 24 is never run

    def cost(bins, cl):
        assert bins[0] <= bins[1]
        return 1.0

    _, _, _, seen = coordinate_descent(cost, search)
    assert ((24, 16, 1024, 2048), 0) not in seen
