"""Pins of Fig. 8's multiplication counts (Section 4, kernel/input-size
ablation) under the readings of oracle/fig8.py.

The paper reports about 4x fewer polynomial products for a 5x5 kernel over a
64x64 input with C = M = 3, and about 5.1x for the largest kernel at 64x64.
The figure is missing from the source.  What the counts show:

* The toy example's reading reproduces 4x.  Under it, the polynomial capacity
  is the smallest at which one channel of the correlated packing fits one
  polynomial (capacity 9, "degrees capped at 8", for the toy), and the
  conventional side uses square windows with one channel per polynomial.
  Then 64x64 / 5x5 needs 36 conventional products against 9 correlated ones:
  exactly 4x, for same and full padding.
* No reading reaches 5.1x.  The same reading gives exactly 4x at every kernel
  size.  With one correlated tile per channel, the ratio is the integer
  T_conv / T_corr, and 5.1 is not one of its values.
* The library's plans (power-of-two rings, output packing, channel blocks)
  give 1-2x.
"""
import pytest

from oracle import fig8, packing
from tests.conftest import read_golden


def _capacity_ratio(H, h, padmode):
    p = fig8.pad_of(padmode, h)
    cap = fig8.correlated_capacity(H, H, h, p)
    a = fig8.conventional_count(cap, 3, H, H, 3, h, p, "square", "one", False)
    b = fig8.correlated_count(cap, 3, H, H, 3, h, p, "tile", "blocks", True)
    return cap, a, b


def test_capacity_reading_is_the_toy_example():
    """Fig. 7's toy example: 2x2 input, 2x2 kernel, padding 1.  The correlated
    packing fits one polynomial at capacity 9 (degree cap 8), where the
    conventional one needs 4 products."""
    g = read_golden("toy_example_fig7.txt")
    H, h, pad = int(g["H"][0]), int(g["h"][0]), int(g["pad"][0])
    cap = fig8.correlated_capacity(H, H, h, pad)
    assert cap == int(g["degree_cap"][0]) + 1
    assert fig8.conventional_count(cap, 1, H, H, 1, h, pad, "square", "one", False) == int(g["conv_products"][0])
    assert fig8.correlated_count(cap, 1, H, H, 1, h, pad, "tile", "one", False) == int(g["corr_products"][0])
    assert fig8.correlated_count(cap - 1, 1, H, H, 1, h, pad, "tile", "one", False) > 1


@pytest.mark.parametrize("padmode", ["same", "full"])
def test_fig8_four_fold_at_64x64_5x5(padmode):
    """The toy example's reading at the ablation's 64x64 input, 5x5 kernel and
    C = M = 3: 36 conventional products against 9, i.e. 4x.  The same holds at
    every input size of the sweep (8 .. 64)."""
    cap, a, b = _capacity_ratio(64, 5, padmode)
    assert (a, b) == (36, 9)
    assert cap == {"same": 4486, "full": 4624}[padmode]
    for H in (8, 16, 32):
        _, a, b = _capacity_ratio(H, 5, padmode)
        assert (a, b) == (36, 9)


def test_fig8_largest_kernel_ratio_not_reproduced():
    """Kernels 3..15 at 64x64 under the toy example's reading: 4x at every
    size, never the paper's 5.1x (the largest ratio of all readings in the
    module, swept over same/valid/full padding and N = 4096/8192/16384, is the
    same 36/9)."""
    for h in (3, 7, 11, 15):
        for padmode in ("same", "full"):
            _, a, b = _capacity_ratio(64, h, padmode)
            assert (a, b) == (36, 9)


@pytest.mark.parametrize("N", [4096, 8192])
def test_library_plans_give_one_to_two_fold(N):
    """The library's own plans (power-of-two ring, channel blocks, output
    packing, same padding) at 64x64: the correlated packing needs at most as
    many products, and at most 2x fewer."""
    for h in (3, 5, 7, 9, 11):
        a = packing.make_plan("conv", N, 3, 64, 64, 3, h, h // 2).products
        b = packing.make_plan("corr", N, 3, 64, 64, 3, h, h // 2).products
        assert b <= a <= 2 * b, (N, h, a, b)


def test_counts_equal_the_plan_search():
    """The counting module's library readings equal the products of the
    plans in packing.py (the same searches, counted two ways)."""
    for (N, C, H, W, M, h, pad) in [(4096, 3, 64, 64, 3, 5, 2), (8192, 3, 32, 32, 16, 3, 1),
                                   (2048, 5, 20, 13, 4, 3, 0), (4096, 3, 64, 64, 3, 11, 5)]:
        assert fig8.conventional_count(N, C, H, W, M, h, pad) == packing.make_plan(
            "conv", N, C, H, W, M, h, pad).products
        assert fig8.correlated_count(N, C, H, W, M, h, pad) == packing.make_plan(
            "corr", N, C, H, W, M, h, pad).products
