"""The library's window and output-packing search (he_plan_search, host only,
no GPU) against the oracle's plans: same window, channel packing, tiles and
output packing for shapes across both encodings, paddings and ring degrees;
and the multiply counts of the Fig. 8 sweep (Section 3.3)."""
import pytest

from oracle import packing
from paper_2409_16675_gb300 import native as nv, workloads as wl

ENC = {"conv": nv.HE_ENC_CONVENTIONAL, "corr": nv.HE_ENC_CORRELATED}


def shapes():
    r = wl.rng(4242)
    out = [(8192, 3, 32, 32, 16, 3, 1), (4096, 1, 28, 28, 4, 3, 0), (1024, 8, 24, 17, 3, 3, 2),
           (2048, 3, 64, 64, 3, 5, 2), (8192, 16, 14, 14, 32, 3, 0), (8192, 512, 1, 1, 10, 1, 0)]
    for _ in range(60):
        N = int(r.choice([256, 1024, 4096, 8192]))
        h = int(r.choice([1, 3, 5, 7]))
        H = int(r.integers(h, 40))
        W = int(r.integers(h, 40))
        out.append((N, int(r.integers(1, 20)), H, W, int(r.integers(1, 40)), h, int(r.integers(0, h))))
    return out


@pytest.mark.parametrize("enc", ["conv", "corr"])
def test_library_plans_equal_the_oracle(enc):
    n_fit = 0
    for (N, C, H, W, M, h, pad) in shapes():
        try:
            op = packing.make_plan(enc, N, C, H, W, M, h, pad)
        except ValueError:
            op = None
        if op is None:
            with pytest.raises(nv.HEError) as e:
                nv.he_plan_search(N, C, H, W, M, h, pad, ENC[enc])
            assert e.value.code == -3          # PLAN_DOES_NOT_FIT
            continue
        n_fit += 1
        li = nv.he_plan_search(N, C, H, W, M, h, pad, ENC[enc])
        assert (li.Cn, li.G, li.th, li.tw, li.Th, li.Tw, li.T) == (op.Cn, op.G, op.th, op.tw, op.Th, op.Tw, op.T)
        assert (li.Mn, li.Sout, li.MG) == (op.Mn, op.Sout, op.MG)
        if enc == "conv":
            assert (li.Hn, li.Wn, li.Ooff) == (op.Hn, op.Wn, op.Ooff)
        else:
            assert (li.O, li.S) == (op.O, op.S)
    assert n_fit > 40


def test_plan_search_rejects_bad_arguments():
    with pytest.raises(nv.HEError):
        nv.he_plan_search(3000, 3, 8, 8, 2, 3, 1, nv.HE_ENC_CORRELATED)   # N not a power of two
    with pytest.raises(nv.HEError):
        nv.he_plan_search(1024, 3, 8, 8, 2, 3, 3, nv.HE_ENC_CORRELATED)   # pad > h - 1


def test_fig8_sweep_correlated_never_needs_more_products():
    """Fig. 8 (Section 4): multiply counts of the two packings over input sizes
    and kernel sizes at C = 3; the correlated packing never needs more
    polynomial products than the conventional one with same padding (the
    printed 4x / 5.1x ratios are not reproduced by these plans)."""
    for N in (2048, 4096, 8192):
        for H in (8, 16, 32, 64):
            for h in (1, 3, 5, 7, 9, 11):
                if h > H:
                    continue
                cnt = {}
                for enc in ("conv", "corr"):
                    i = nv.he_plan_search(N, 3, H, H, 3, h, h // 2, ENC[enc])
                    cnt[enc] = i.MG * i.G * i.T
                assert cnt["corr"] <= cnt["conv"], (N, H, h, cnt)


@pytest.mark.parametrize("enc", ["conv", "corr"])
def test_library_depthwise_plans_equal_the_oracle(enc):
    """Depthwise plans (M = C, one product per kernel polynomial and tile):
    the library's search equals the oracle's, keeps Mn a divisor of Cn, and
    needs no more products than the dense plan of the same shape."""
    r = wl.rng(99)
    cases = [(8192, 64, 64, 64, 1, 0), (8192, 16, 16, 16, 1, 0), (4096, 32, 8, 8, 3, 1), (1024, 5, 9, 7, 3, 1)]
    for _ in range(25):
        N = int(r.choice([1024, 4096, 8192]))
        h = int(r.choice([1, 3, 5]))
        C = int(r.integers(1, 40))
        H = int(r.integers(h, 33))
        cases.append((N, C, H, int(r.integers(h, 33)), h, int(r.integers(0, h))))
    for (N, C, H, W, h, pad) in cases:
        try:
            op = packing.make_plan(enc, N, C, H, W, C, h, pad, depthwise=True)
        except ValueError:
            with pytest.raises(nv.HEError):
                nv.he_plan_search(N, C, H, W, C, h, pad, ENC[enc] | nv.HE_PLAN_DEPTHWISE)
            continue
        li = nv.he_plan_search(N, C, H, W, C, h, pad, ENC[enc] | nv.HE_PLAN_DEPTHWISE)
        assert li.depthwise == 1 and li.encoding == ENC[enc]
        assert (li.Cn, li.G, li.T, li.Mn, li.MG, li.Sout) == (op.Cn, op.G, op.T, op.Mn, op.MG, op.Sout)
        assert op.G == 1 or op.Cn % op.Mn == 0
        dense = packing.make_plan(enc, N, C, H, W, C, h, pad)
        assert op.products <= dense.products
    # the batch-norm case of the AlexNet-shaped bench: 64 channels of 64x64
    bn = packing.make_plan(enc, 8192, 64, 64, 64, 64, 1, 0, depthwise=True)
    assert bn.products == 64


def test_depthwise_requires_as_many_outputs_as_inputs():
    with pytest.raises(nv.HEError):
        nv.he_plan_search(1024, 4, 8, 8, 5, 1, 0, nv.HE_ENC_CORRELATED | nv.HE_PLAN_DEPTHWISE)
