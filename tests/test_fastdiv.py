"""The invariant-divisor method that coords() uses on the device (Granlund
and Montgomery 1994): with s = ceil(log2 d), m = floor(2^32 (2^s - d) / d) + 1,
x // d == (mulhi(x, m) + x) >> s for 0 <= x < 2^31. Checked here with exact
integers against Python's floor division on divisors up to 2^31 - 1 and on
dividends at and around every multiple boundary that matters."""
import random


def fast_div(d):
    s = 0
    while (1 << s) < d:
        s += 1
    m = ((1 << 32) * ((1 << s) - d)) // d + 1
    assert 0 < m < (1 << 32)
    return m, s


def fdiv(x, ms):
    m, s = ms
    hi = (x * m) >> 32
    t = hi + x
    assert t < (1 << 32)  # no overflow of the 32-bit sum
    return t >> s


def _check(d, xs):
    ms = fast_div(d)
    for x in xs:
        assert fdiv(x, ms) == x // d, (d, x)


def test_small_divisors_dense():
    for d in range(1, 600):
        _check(d, range(0, 5000))


def test_boundaries_all_sizes():
    rng = random.Random(7)
    top = (1 << 31) - 1
    ds = list(range(1, 70)) + [2**k + o for k in range(2, 31) for o in (-1, 0, 1)] + \
        [rng.randrange(1, top) for _ in range(300)] + [top, top - 1, 46341, 65535, 65537, 1 << 30]
    for d in ds:
        if d < 1 or d > top:
            continue
        xs = {0, 1, top, top - 1}
        q_top = top // d
        for q in (1, 2, 3, q_top // 2, q_top - 1, q_top):
            for o in (-1, 0, 1):
                x = q * d + o
                if 0 <= x <= top:
                    xs.add(x)
        xs.update(rng.randrange(0, top + 1) for _ in range(200))
        _check(d, sorted(xs))
