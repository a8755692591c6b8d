"""Pins of the veto (Section 4, "Peak count as veto algorithm"): frames with
fewer peaks than the threshold are discarded, a frame with exactly the
threshold is kept, threshold 0 keeps every frame, and a threshold above the
largest count keeps none."""
import oracle


def test_threshold_semantics():
    counts = [0, 19, 20, 21, 5, 300, 20]
    assert oracle.veto(counts, 20) == [2, 3, 5, 6]
    assert oracle.veto(counts, 0) == list(range(len(counts)))
    assert oracle.veto(counts, 301) == []
    assert oracle.veto([], 3) == []
