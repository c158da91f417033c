"""The double-word (float-float) building blocks of the FP32 residual form, checked on the CPU.

The device code (``csrc/dw.cuh``) evaluates a residual with pairs of FP32 numbers.  These tests
model the same FP32 operation sequences with numpy float32 scalars (every step rounded to
nearest, no fused operations except where the algorithm uses an FMA, modelled exactly with
rationals) and compare against exact rational arithmetic:

* AccurateDWPlusDW and SloppyDWPlusDW (Joldes, Muller, Popescu 2017, Algorithms 6 and 5): the
  residual needs an absolute error of a few u^2 (|x| + |y|), u = 2^-24, also under cancellation;
* DWTimesDW3 (Algorithm 12): relative error <= 5 u^2;
* the integer-only split of an FP64 value into a normalised float pair: exact to 2^-47 while
  the low word stays a normal FP32 number.

The GPU parity tests check the kernels themselves against the oracle.
"""
import struct
from fractions import Fraction as F

import numpy as np

f32 = np.float32
U2 = 2.0 ** -48


def fma32(a, b, c):
    """FP32 fused multiply-add: the exact a*b + c rounded once."""
    return f32(float(F(float(a)) * F(float(b)) + F(float(c))))


def two_sum(a, b):
    s = f32(a + b)
    bv = f32(s - a)
    av = f32(s - bv)
    return s, f32(f32(a - av) + f32(b - bv))


def fast_two_sum(a, b):
    s = f32(a + b)
    return s, f32(b - f32(s - a))


def add_accurate(x, y):
    sh, sl = two_sum(x[0], y[0])
    th, tl = two_sum(x[1], y[1])
    vh, vl = fast_two_sum(sh, f32(sl + th))
    return fast_two_sum(vh, f32(tl + vl))


def add_sloppy(x, y):
    sh, sl = two_sum(x[0], y[0])
    return fast_two_sum(sh, f32(sl + f32(x[1] + y[1])))


def mul(x, y):
    ch = f32(x[0] * y[0])
    cl1 = fma32(x[0], y[0], -ch)
    tl1 = fma32(x[0], y[1], f32(x[1] * y[1]))
    cl2 = fma32(x[1], y[0], tl1)
    return fast_two_sum(ch, f32(cl1 + cl2))


def dw(v):
    h = f32(v)
    return h, f32(v - float(h))


def val(x):
    return F(float(x[0])) + F(float(x[1]))


def split_bits(v):
    """Integer-only split: hi = leading 24 bits (truncated), lo = next 29 bits rounded to 24 and
    scaled by exact powers of two, then Fast2Sum; valid for 2^-126 <= |v| < 2^128."""
    b = struct.unpack("<Q", struct.pack("<d", v))[0]
    e = (b >> 52) & 0x7FF
    assert 897 <= e <= 1150
    sgn = (b >> 63) << 31
    m = b & ((1 << 52) - 1)
    h = struct.unpack("<f", struct.pack("<I", sgn | ((e - 896) << 23) | (m >> 29)))[0]
    k = 0 if e >= 949 else 64
    p1 = struct.unpack("<f", struct.pack("<I", (e + k - 948) << 23))[0]
    p2 = struct.unpack("<f", struct.pack("<I", (127 - k) << 23))[0]
    lo = f32(f32(f32(m & 0x1FFFFFFF) * f32(p1)) * f32(p2))
    lo = -lo if sgn else lo
    return fast_two_sum(f32(h), lo)


def pairs(n, seed):
    rng = np.random.default_rng(seed)
    for t in range(n):
        a = rng.standard_normal() * 10.0 ** rng.uniform(-3, 3)
        mode = t % 3
        if mode == 0:
            b = -a * (1 + rng.standard_normal() * 10.0 ** rng.uniform(-12, -1))     # cancellation
        elif mode == 1:
            b = rng.standard_normal() * 10.0 ** rng.uniform(-3, 3)
        else:
            b = -a + rng.standard_normal() * abs(a) * 1e-7
        yield dw(a), dw(b)


def test_double_word_adds_have_absolute_error_of_a_few_u2():
    worst = {"accurate": 0.0, "sloppy": 0.0}
    for x, y in pairs(20000, 1):
        exact = val(x) + val(y)
        scale = abs(val(x)) + abs(val(y))
        for name, fn in (("accurate", add_accurate), ("sloppy", add_sloppy)):
            worst[name] = max(worst[name], float(abs(val(fn(x, y)) - exact) / scale) / U2)
    assert worst["accurate"] < 3.0 and worst["sloppy"] < 3.0, worst


def test_sloppy_add_loses_relative_accuracy_under_cancellation_only():
    """Why the accurate add is kept for the state updates: under cancellation the sloppy add's
    result can be wrong in relative terms (its absolute error stays small)."""
    worst_rel = 0.0
    for x, y in pairs(6000, 2):
        exact = val(x) + val(y)
        if exact != 0:
            worst_rel = max(worst_rel, float(abs(val(add_sloppy(x, y)) - exact) / abs(exact)))
    assert worst_rel > 1e3 * U2


def test_double_word_product_relative_error():
    rng = np.random.default_rng(3)
    worst = 0.0
    for _ in range(5000):
        x = dw(rng.standard_normal() * 10.0 ** rng.uniform(-5, 5))
        y = dw(rng.standard_normal() * 10.0 ** rng.uniform(-5, 5))
        exact = val(x) * val(y)
        worst = max(worst, float(abs(val(mul(x, y)) - exact) / abs(exact)) / U2)
    assert worst <= 5.0, worst


def test_integer_split_is_exact_to_2_pow_minus_47():
    """Relative 2^-47 while the low word is a normal FP32 number (|v| >= 2^-102); below that,
    down to 2^-126, an absolute error under 2^-149 (the FP32 subnormal spacing: two roundings)."""
    rng = np.random.default_rng(4)
    vals = list(rng.standard_normal(20000) * 10.0 ** rng.uniform(-37, 37, 20000))
    vals += [1.0, -1.0, 3.0, 1.0 / 3.0, 2.0 ** -74, 2.0 ** -73, 2.0 ** -102, 2.0 ** -126, -1e-30, 1e30]
    worst_rel = worst_abs = 0.0
    for v in vals:
        if not 2.0 ** -126 <= abs(v) < 2.0 ** 127:
            continue
        h, l = split_bits(float(v))
        assert abs(float(l)) <= 2.0 ** -24 * abs(float(h)) * (1 + 1e-7)            # normalised
        err = abs(F(float(h)) + F(float(l)) - F(float(v)))
        if abs(v) >= 2.0 ** -102:
            worst_rel = max(worst_rel, float(err / abs(F(float(v)))))
        else:
            worst_abs = max(worst_abs, float(err))
    assert worst_rel <= 2.0 ** -47, worst_rel
    assert worst_abs <= 2.0 ** -149, worst_abs


def mul_f(x, y):
    """DWTimesFP (the dw_mul_f sequence): x double word, y float."""
    ch = f32(x[0] * y)
    cl1 = fma32(x[0], y, -ch)
    return fast_two_sum(ch, fma32(x[1], y, cl1))


def rcp32(v):
    """The correctly rounded FP32 reciprocal (rounding the exact rational once)."""
    q = F(1) / F(float(v))
    lo = f32(float(q))                      # nearest double, then float: fix the rare double rounding
    cands = [lo, np.nextafter(lo, f32(np.inf)), np.nextafter(lo, f32(-np.inf))]
    return min(cands, key=lambda c: (abs(F(float(c)) - q), int(np.frombuffer(np.float32(c).tobytes(), np.uint32)[0]) & 1))


def recip(b):
    """dw_recip: r0 = rcp(b.h), e = 1 - b r0 in double words, r = r0 + e r0."""
    r0 = rcp32(b[0])
    e = add_accurate((f32(1.0), f32(0.0)), tuple(-t for t in mul_f(b, r0)))
    return add_accurate((r0, f32(0.0)), mul_f(e, r0))


def test_double_word_reciprocal_relative_error():
    rng = np.random.default_rng(6)
    worst = 0.0
    for _ in range(4000):
        b = dw(rng.standard_normal() * 10.0 ** rng.uniform(-15, 15))
        r = recip(b)
        worst = max(worst, float(abs(val(r) * val(b) - 1)) / U2)
    assert worst <= 6.0, worst


def cdiv(a, b):
    """cdw_div without its power-of-two scaling (operands of moderate size): a conj(b) / |b|^2."""
    ax, ay = a
    bx, by = b
    abs2 = add_accurate(mul(bx, bx), mul(by, by))
    inv = recip(abs2)
    tx = add_accurate(mul(ax, bx), mul(ay, by))
    ty = add_accurate(mul(ay, bx), tuple(-t for t in mul(ax, by)))
    return mul(tx, inv), mul(ty, inv)


def test_complex_double_word_quotient_relative_error():
    """The Krylov scalar recurrences divide complex double words: about 2^-44 relative at worst
    (a few u^2 per operation), the accuracy FP64 scalars had for these recurrences' purpose."""
    rng = np.random.default_rng(7)
    worst = 0.0
    for _ in range(1500):
        a = (dw(rng.standard_normal() * 10.0 ** rng.uniform(-4, 4)), dw(rng.standard_normal() * 10.0 ** rng.uniform(-4, 4)))
        b = (dw(rng.standard_normal() * 10.0 ** rng.uniform(-4, 4)), dw(rng.standard_normal() * 10.0 ** rng.uniform(-4, 4)))
        qx, qy = cdiv(a, b)
        num_x, num_y = val(a[0]) * val(b[0]) + val(a[1]) * val(b[1]), val(a[1]) * val(b[0]) - val(a[0]) * val(b[1])
        den = val(b[0]) ** 2 + val(b[1]) ** 2
        ex, ey = num_x / den, num_y / den
        mag = abs(complex(float(ex), float(ey)))
        err = abs(complex(float(val(qx) - ex), float(val(qy) - ey))) / mag
        worst = max(worst, err)
    assert worst <= 2.0 ** -43, worst


def cmul(a, b):
    """cdw_mul: (ax bx - ay by) + i (ax by + ay bx) with double-word products and sums."""
    (ax, ay), (bx, by) = a, b
    return (add_accurate(mul(ax, bx), tuple(-t for t in mul(ay, by))), add_accurate(mul(ax, by), mul(ay, bx)))


def crecip(b):
    """cdw_recip without its power-of-two scaling: conj(b) / |b|^2."""
    bx, by = b
    inv = recip(add_accurate(mul(bx, bx), mul(by, by)))
    return mul(bx, inv), mul(tuple(-t for t in by), inv)


def cval(a):
    return complex(float(val(a[0])), float(val(a[1])))


def test_two_reciprocal_recurrence_matches_the_quotient_form():
    """The single-reduction COCG scalars (Chronopoulos-Gear form of CG, unconjugated): from gamma_k,
    delta_k the quotient form gives beta_{k+1} = gamma_{k+1}/gamma_k and alpha_{k+1} =
    gamma_{k+1}/(delta_{k+1} - beta_{k+1} gamma_{k+1}/alpha_k).  The on-chip solver carries
    q_k = 1/(gamma_k alpha_k) and 1/gamma_k instead (two independent reciprocals per step).  Over
    40-step sequences of random complex gamma, delta the double-word version stays within 2^-38 of
    the quotient form evaluated exactly."""
    rng = np.random.default_rng(11)
    worst = 0.0
    for _ in range(30):
        cz = lambda: complex(rng.standard_normal(), rng.standard_normal()) * 10.0 ** rng.uniform(-2, 2)
        g0, d0 = cz(), cz()
        # exact (rational) reference of the quotient form
        G0, D0 = (F(g0.real), F(g0.imag)), (F(d0.real), F(d0.imag))

        def qmul(a, b):
            return (a[0] * b[0] - a[1] * b[1], a[0] * b[1] + a[1] * b[0])

        def qdiv(a, b):
            den = b[0] * b[0] + b[1] * b[1]
            return ((a[0] * b[0] + a[1] * b[1]) / den, (a[1] * b[0] - a[0] * b[1]) / den)

        gam_x = (dw(g0.real), dw(g0.imag))
        del_x = (dw(d0.real), dw(d0.imag))
        Gk = (val(gam_x[0]), val(gam_x[1]))
        Ak = qdiv(Gk, (val(del_x[0]), val(del_x[1])))
        # double-word state
        al = cmul(gam_x, crecip(del_x))
        rg2 = crecip(cmul(gam_x, gam_x))
        ig = cmul(gam_x, rg2)
        qk = cmul(del_x, rg2)
        gam = gam_x
        for _k in range(40):
            g1, d1 = cz(), cz()
            gk = (dw(g1.real), dw(g1.imag))
            dk = (dw(d1.real), dw(d1.imag))
            G1, D1 = (val(gk[0]), val(gk[1])), (val(dk[0]), val(dk[1]))
            B1 = qdiv(G1, Gk)
            t = qdiv(qmul(B1, G1), Ak)
            A1 = qdiv(G1, (D1[0] - t[0], D1[1] - t[1]))
            g2 = cmul(gk, gk)
            m = cmul(g2, qk)
            den = (add_accurate(dk[0], tuple(-v for v in m[0])), add_accurate(dk[1], tuple(-v for v in m[1])))
            r1, r2 = crecip(den), crecip(g2)
            be = cmul(gk, ig)
            al = cmul(gk, r1)
            qk = cmul(den, r2)
            ig = cmul(gk, r2)
            for got, ref in ((al, A1), (be, B1)):
                rv = complex(float(ref[0]), float(ref[1]))
                worst = max(worst, abs(cval(got) - rv) / abs(rv))
            Gk, Ak = G1, A1
    assert worst <= 2.0 ** -38, worst
