"""The autotuner's selection rule (host logic, no GPU)."""
import pytest

from paper_2204_07921_gb300 import autotune


def test_choose_fastest_within_energy_slack():
    res = [dict(G=9, K=16, seconds=0.025, energy=100.0),
           dict(G=5, K=8, seconds=0.016, energy=98.0),
           dict(G=5, K=6, seconds=0.012, energy=98.1),
           dict(G=3, K=2, seconds=0.007, energy=105.0)]
    assert autotune.choose(res)["K"] == 6          # within 0.2% of the best energy
    assert autotune.choose(res, slack=1e-4)["K"] == 8
    assert autotune.choose(res, slack=0.1)["K"] == 2


def test_choose_ties_prefer_larger_budget():
    res = [dict(G=5, K=6, seconds=0.01, energy=1.0), dict(G=9, K=16, seconds=0.01, energy=1.0)]
    assert autotune.choose(res)["G"] == 9
    with pytest.raises(ValueError):
        autotune.choose([])


def test_shape_needs_a_margin_and_the_energy():
    base = dict(shapes=0, seconds=0.0100, energy=100.0)
    assert autotune.choose_shape(base, dict(shapes=1, seconds=0.0099, energy=100.0)) is base
    alt = dict(shapes=1, seconds=0.0098, energy=100.0)
    assert autotune.choose_shape(base, alt) is alt
    assert autotune.choose_shape(base, dict(shapes=1, seconds=0.005, energy=101.0)) is base
    assert autotune.choose_shape(base, dict(shapes=1, seconds=0.005, energy=99.0))["shapes"] == 1


def test_shape_bits_follow_the_levels():
    assert autotune.shape_bits(1) == []          # b = 1 only
    assert autotune.shape_bits(3) == [0, 1]      # b = 2, 4
    assert autotune.shape_bits(6) == [0, 1, 2, 3, 4]
    assert autotune.shape_bits(10) == [0, 1, 2, 3, 4]
