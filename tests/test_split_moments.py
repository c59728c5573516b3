"""The thermostat's second-moment sums in the fused kernel (CPU check of the
arithmetic it relies on).

Pass 1 of the warp-spread kernel adds each lane's int64 partial P of
sum H^2, sum H L and sum L^2 (V = rne(v 2^32) = H 2^20 + L, |v| < 1024) to
its cell as two 32-bit shared atomics, the high part P >> 24 (arithmetic
shift) and the low part P & (2^24 - 1), and the cell phase rebuilds the sum
as hi 2^24 + lo.  The sums are exact only while neither 32-bit sum wraps.  A
lane's share holds at most 8 members (24 terms), |H| <= 2^22 and |L| <= 2^19,
and a cell of at most 448 members receives at most 128 partials.  These tests
run the same split, 32-bit accumulation and recombination on the worst cases
those bounds allow and on random partials, against exact integer sums.
"""
import random

import pytest

H_MAX, L_MAX = 2**22, 2**19
TERMS = 24          # members per lane share (8) x components (3)
PARTIALS = 128      # partials one cell can receive
MASK24 = (1 << 24) - 1


def split(p):
    return p >> 24, p & MASK24  # Python's >> on negative ints is arithmetic, like the kernel's


def wrap_u32(x):
    return x % 2**32


def wrap_i32(x):
    x = x % 2**32
    return x - 2**32 if x >= 2**31 else x


def accumulate(partials, signed_hi):
    """32-bit atomics: the high sum as int32 (H L) or uint32 (H^2, L^2), the
    low sum as uint32; returns the rebuilt int64 sum."""
    hi, lo = 0, 0
    for p in partials:
        h, l = split(p)
        hi = wrap_i32(hi + h) if signed_hi else wrap_u32(hi + h)
        lo = wrap_u32(lo + l)
    return hi * 2**24 + lo


@pytest.mark.parametrize("kind", ["hh", "hl", "ll"])
def test_worst_case_sums_do_not_wrap(kind):
    if kind == "hh":
        top, signed = TERMS * H_MAX**2, False
        cases = [[top] * PARTIALS, [top - 1] * PARTIALS]
    elif kind == "ll":
        top, signed = TERMS * L_MAX**2, False
        cases = [[top] * PARTIALS, [top - 1] * PARTIALS]
    else:
        top, signed = TERMS * H_MAX * L_MAX, True
        cases = [[top] * PARTIALS, [-top] * PARTIALS, [top - 1] * PARTIALS,
                 [-top + 1] * PARTIALS, [top, -top] * (PARTIALS // 2)]
    for parts in cases:
        assert accumulate(parts, signed) == sum(parts)
    # the headroom the kernel comment states
    hi_max = max(abs(p >> 24) for p in (top, -top if signed else top))
    assert PARTIALS * hi_max < (2**29 if signed or kind == "ll" else 2**32)
    assert PARTIALS * MASK24 < 2**31


def test_random_partials_rebuild_exactly():
    rng = random.Random(7)
    for _ in range(2000):
        n = rng.randint(1, PARTIALS)
        hh = [sum(rng.randint(-H_MAX, H_MAX) ** 2 for _ in range(rng.randint(1, TERMS)))
              for _ in range(n)]
        hl = [sum(rng.randint(-H_MAX, H_MAX) * rng.randint(-L_MAX, L_MAX)
                  for _ in range(rng.randint(1, TERMS))) for _ in range(n)]
        ll = [sum(rng.randint(-L_MAX, L_MAX) ** 2 for _ in range(rng.randint(1, TERMS)))
              for _ in range(n)]
        assert accumulate(hh, False) == sum(hh)
        assert accumulate(hl, True) == sum(hl)
        assert accumulate(ll, False) == sum(ll)


def test_a_larger_bound_would_wrap():
    """The check bites: with twice the partials the high sum of H^2 wraps."""
    top = TERMS * H_MAX**2
    parts = [top] * (2 * PARTIALS)
    assert accumulate(parts, False) != sum(parts)
