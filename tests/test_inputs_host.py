"""The synthetic-input helpers the batches use: padding edges."""
from dda_inputs import next_even_smooth, next_pow2, uneven_batch_cases


def _smooth(v):
    for f in (2, 3, 5, 7):
        while v % f == 0:
            v //= f
    return v == 1


def test_next_even_smooth_is_the_least_even_7smooth_edge():
    for v in range(1, 600):
        e = next_even_smooth(v)
        assert e >= v and e % 2 == 0 and _smooth(e), v
        assert not any(w % 2 == 0 and _smooth(w) for w in range(max(v, 2), e)), v
    assert next_even_smooth(83) == 84 and next_even_smooth(85) == 90 and next_even_smooth(97) == 98


def test_uneven_batch_boxes_hold_their_prisms():
    pow2 = uneven_batch_cases(32, seed=2)
    smooth = uneven_batch_cases(32, seed=2, pad_pow2=False, pad_smooth=True)
    for a, b in zip(pow2, smooth):
        assert a.N == b.N and a.eps == b.eps  # the same draws
        assert a.dims == (next_pow2(a.N),) * 3
        assert b.dims == (next_even_smooth(b.N),) * 3 and b.dims[0] <= a.dims[0]
