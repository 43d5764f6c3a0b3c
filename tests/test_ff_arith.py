"""CPU check of the float-float arithmetic the precision variant's outer sweep uses (sweep.cu,
sweep2d_ff_kernel): a value is hi + lo, two IEEE single-precision numbers.  Its FMA a * b + c is
built from two published error-free transformations:
- Dekker's exact product in FMA form: p = fl(a_hi b_hi) and fl(a_hi b_hi - p) = a_hi b_hi - p exactly;
- Knuth's TwoSum: s = fl(x + y), e = fl(fl(x - fl(s - v)) + fl(y - v)), v = fl(s - x) gives
  s + e = x + y exactly.
Then come the cross terms a_hi b_lo + a_lo b_hi, added in single precision, and a renormalisation
(fast TwoSum).  The kernel issues these steps as packed pairs in inline PTX, so that nothing is
contracted or reassociated.  Here they are written out with numpy float32 operations (round to
nearest even), each FMA rounded once from its exact value.  The test checks the two facts the sweep's
error bound rests on, on random operands over six decades and on cancelling sums:
- the result is within 2^-45 (|a b| + |c|) of the exact a * b + c;
- |lo| <= ulp(hi) / 2 afterwards.
It also checks the exactness of each transformation on its own."""
from fractions import Fraction

import numpy as np

f32 = np.float32


def _fr(x):
    return Fraction(float(x))


def _round32(v: Fraction):
    """v rounded to the nearest float32 (ties to even)."""
    r = f32(float(v))
    best, dbest = r, abs(_fr(r) - v)
    for c in (np.nextafter(r, f32(np.inf)), np.nextafter(r, f32(-np.inf))):
        dc = abs(_fr(c) - v)
        even = int(np.array(c, np.float32).view(np.uint32)) & 1 == 0
        if dc < dbest or (dc == dbest and even):
            best, dbest = c, dc
    return f32(best)


def fma32(a, b, c):
    return _round32(_fr(a) * _fr(b) + _fr(c))


def two_sum(x, y):
    s = f32(x + y)
    v = f32(s - x)
    return s, f32(f32(x - f32(s - v)) + f32(y - v))


def ff_fma(a, b, c):
    """(a_hi, a_lo) * (b_hi, b_lo) + (c_hi, c_lo) in the kernel's order of operations."""
    (ah, al), (bh, bl), (ch, cl) = a, b, c
    p = f32(ah * bh)
    pe = fma32(ah, bh, -p)
    pe = fma32(ah, bl, pe)
    pe = fma32(al, bh, pe)
    s = f32(p + ch)
    bv = f32(s - p)
    e = f32(f32(p - f32(s - bv)) + f32(ch - bv))
    e = f32(e + f32(pe + cl))
    hi = f32(s + e)
    lo = f32(e - f32(hi - s))
    return hi, lo


def split(v: float):
    h = f32(v)
    return h, f32(v - float(h))


def _val(x):
    return _fr(x[0]) + _fr(x[1])


def test_error_free_transformations_are_exact():
    rng = np.random.default_rng(3)
    for _ in range(2000):
        a, b = (f32(v) for v in rng.uniform(-4, 4, 2) * 10.0 ** rng.integers(-4, 4, 2))
        p = f32(a * b)
        assert _fr(p) + _fr(fma32(a, b, -p)) == _fr(a) * _fr(b)
        s, e = two_sum(a, b)
        assert _fr(s) + _fr(e) == _fr(a) + _fr(b)


def test_ff_fma_accuracy_and_normalisation():
    rng = np.random.default_rng(11)
    worst = 0.0
    for k in range(3000):
        a, b, c = rng.uniform(-2, 2, 3) * 10.0 ** rng.integers(-3, 3, 3)
        if k % 3 == 0:      # cancellation: c close to -a b
            c = -a * b * (1.0 + rng.uniform(-1e-6, 1e-6))
        A, Bv, C = split(a), split(b), split(c)
        hi, lo = ff_fma(A, Bv, C)
        exact = _val(A) * _val(Bv) + _val(C)
        scale = abs(_val(A) * _val(Bv)) + abs(_val(C))
        err = float(abs(_fr(hi) + _fr(lo) - exact) / scale)
        worst = max(worst, err)
        assert err < 2.0 ** -45, (k, err)
        if hi != 0:
            assert abs(float(lo)) <= float(np.spacing(abs(hi))) / 2
    assert worst > 0.0   # the check can fail: the dropped lo * lo term and FP32 cross terms show


def test_split_represents_fp64_to_48_bits():
    rng = np.random.default_rng(5)
    for v in rng.uniform(-1, 1, 500) * 10.0 ** rng.integers(-6, 6, 500):
        h, l = split(float(v))
        assert abs(float(_fr(h) + _fr(l) - _fr(v))) <= 2.0 ** -48 * abs(v)
