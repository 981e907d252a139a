"""The packed fp32 forms of the float-float steps round exactly as the scalar
steps they replace (checked in exact IEEE binary32 arithmetic, emulated on
rationals with round-to-nearest-even and IEEE zero signs):

- the float-float multiply-add: the scalar steps form x = fl(q_hi p_hi) and
  the product's error q_hi p_hi - x; the packed steps form xn = fl(-q_hi p_hi)
  and q_hi p_hi + xn, a - xn for a + x, and -(xn + bb) for x - bb.  Both give
  the same hi part bit for bit and the same lo value (a zero's sign may
  differ, which the digit split ignores);
- the digit split's T2 and T1 steps: fl(fl(A 2^-32) + M) equals the fused
  fl(A 2^-32 + M), and likewise with 2^-16, M = 1.5 2^23, for every A the
  split meets (0 <= A < 2^48, including values far below one)."""
from fractions import Fraction

import numpy as np

F32 = np.float32


def _signbit(v):
    return bool(np.signbit(v))


def _rn32(x):
    """The binary32 number nearest the nonzero rational x (ties to even)."""
    c = F32(float(x))
    best = None
    for cand in (np.nextafter(c, F32(-np.inf)), c, np.nextafter(c, F32(np.inf))):
        if not np.isfinite(cand):
            continue
        d = abs(Fraction(float(cand)) - x)
        if best is None or d < best[0] or (d == best[0] and int(cand.view(np.uint32)) & 1 == 0):
            best = (d, cand)
    return best[1]


def add(a, b):
    s = Fraction(float(a)) + Fraction(float(b))
    if s == 0:
        return F32(-0.0) if (a == 0 and b == 0 and _signbit(a) and _signbit(b)) else F32(0.0)
    return _rn32(s)


def sub(a, b):
    return add(a, -b)


def mul(a, b):
    p = Fraction(float(a)) * Fraction(float(b))
    if p == 0:
        return F32(-0.0) if _signbit(a) != _signbit(b) else F32(0.0)
    return _rn32(p)


def fma(a, b, c):
    p = Fraction(float(a)) * Fraction(float(b))
    s = p + Fraction(float(c))
    if s == 0:
        if p == 0 and c == 0:
            return F32(-0.0) if (_signbit(a) != _signbit(b)) and _signbit(c) else F32(0.0)
        return F32(0.0)
    return _rn32(s)


def ff_fma_scalar(q, p, acc):
    """acc += q p, the scalar kernel's steps."""
    x = mul(q[0], p[0])
    xe = fma(q[0], p[1], fma(q[1], p[0], fma(q[0], p[0], -x)))
    s = add(acc[0], x)
    bb = sub(s, acc[0])
    err = add(sub(acc[0], sub(s, bb)), sub(x, bb))
    return s, add(acc[1], add(err, xe))


def ff_fma_packed_half(q, p, acc):
    """One half of the packed steps: the negated product xn from -q_hi."""
    xn = mul(-q[0], p[0])
    xe = fma(q[0], p[1], fma(q[1], p[0], fma(q[0], p[0], xn)))
    s = sub(acc[0], xn)
    bb = sub(s, acc[0])
    err = sub(sub(acc[0], sub(s, bb)), add(xn, bb))
    return s, add(acc[1], add(err, xe))


def _ff(rng, scale_exp):
    """A float-float value: hi an fp32 number, |lo| at most half an ulp of hi."""
    hi = F32(rng.uniform(-1.0, 1.0) * 2.0 ** scale_exp)
    ulp = float(np.spacing(np.abs(hi))) if hi != 0 else 0.0
    lo = F32(rng.uniform(-0.5, 0.5) * ulp)
    return hi, lo


def test_emulation_matches_numpy_binary32():
    rng = np.random.default_rng(7)
    for _ in range(2000):
        a = F32(rng.uniform(-1.0, 1.0) * 2.0 ** float(rng.integers(-60, 60)))
        b = F32(rng.uniform(-1.0, 1.0) * 2.0 ** float(rng.integers(-60, 60)))
        assert mul(a, b).view(np.uint32) == (a * b).view(np.uint32)
        assert add(a, b).view(np.uint32) == (a + b).view(np.uint32)
        assert sub(a, b).view(np.uint32) == (a - b).view(np.uint32)
    for a, b in ((F32(0.0), F32(-0.0)), (F32(-0.0), F32(-0.0)), (F32(1.5), F32(-1.5))):
        assert add(a, b).view(np.uint32) == (a + b).view(np.uint32)


def test_packed_multiply_add_rounds_as_the_scalar_one():
    rng = np.random.default_rng(2018)
    cases = []
    for _ in range(1500):
        q = _ff(rng, int(rng.integers(-30, 1)))
        p = _ff(rng, int(rng.integers(-10, 5)))
        acc = _ff(rng, int(rng.integers(-40, 3)))
        cases.append((q, p, acc))
    # cancellations: the accumulator minus the product's leading part, zeros
    for _ in range(300):
        q = _ff(rng, 0)
        p = _ff(rng, 0)
        x = mul(q[0], p[0])
        cases.append((q, p, (F32(-x), F32(0.0))))
        cases.append((q, p, (F32(-x), F32(-0.0))))
    for z in (F32(0.0), F32(-0.0)):
        cases.append(((z, z), (F32(0.5), F32(0.0)), (F32(0.0), F32(0.0))))
        cases.append(((F32(0.75), F32(0.0)), (z, z), (F32(-0.0), F32(-0.0))))
    for q, p, acc in cases:
        hs, ls = ff_fma_scalar(q, p, acc)
        hp, lp = ff_fma_packed_half(q, p, acc)
        assert hs.view(np.uint32) == hp.view(np.uint32), (q, p, acc, hs, hp)
        assert ls == lp, (q, p, acc, ls, lp)


def test_fused_scaling_steps_of_the_digit_split():
    rng = np.random.default_rng(1806)
    M = F32(12582912.0)
    for sc in (F32(2.0 ** -32), F32(2.0 ** -16)):
        values = [F32(0.0), F32(2.0 ** -149), F32(2.0 ** -126), F32(3.0 * 2.0 ** -100)]
        values += [F32(rng.uniform(0.0, 1.0) * 2.0 ** float(e)) for e in rng.integers(-140, 48, 600)]
        for A in values:
            assert add(mul(A, sc), M) == fma(A, sc, M), (A, sc)
