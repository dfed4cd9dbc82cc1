"""The float-pair arithmetic of the FP64 adjoint and Gross-Pitaevskii kernels
(bit moves FP64 -> pair, error-free FMA products, two-sums, the compensated
dot product of Ogita, Rump and Oishi) modelled step by step in FP32 with
numpy and checked against exact rational arithmetic: the split keeps 48
bits, and an adjoint update stays within 2^-45 of |lam| + sum |w v|, the
bound the kernels' documentation states. Independent of the GPU code (a
model of the method, not of its implementation)."""
import struct
from fractions import Fraction as Fr

import numpy as np

f32 = np.float32


def _u2f(u):
    return float(struct.unpack("<f", struct.pack("<I", u & 0xFFFFFFFF))[0])


def pair_split(x):
    """h = sign, exponent and leading 23 fraction bits; l = the other 29 bits
    rounded to 24 (zero gives (0, 0))."""
    b = struct.unpack("<Q", struct.pack("<d", x))[0]
    if b << 1 & 0xFFFFFFFFFFFFFFFF == 0:
        return f32(0), f32(0)
    hw, lw = b >> 32, b & 0xFFFFFFFF
    s = hw & 0x80000000
    t = ((hw & 0x7FFFFFFF) - (896 << 20)) & 0xFFFFFFFF
    h = f32(_u2f(((t << 3) | (lw >> 29)) & 0xFFFFFFFF | s))
    sc = f32(_u2f(((((hw & 0x7FF00000) - (948 << 20)) << 3) & 0xFFFFFFFF) | s))
    return h, f32(f32(lw & 0x1FFFFFFF) * sc)


def fma(a, b, c):
    """FP32 fused multiply-add: one rounding of the exact a*b + c."""
    return f32(float(Fr(float(a)) * Fr(float(b)) + Fr(float(c))))


def two_sum(a, b):
    s = f32(a + b)
    bb = f32(s - a)
    return s, f32(f32(a - f32(s - bb)) + f32(b - bb))


def fast_two_sum(a, b):
    s = f32(a + b)
    return s, f32(b - f32(s - a))


def mul_pair(a, b):
    p = f32(a[0] * b[0])
    e = fma(a[0], b[0], -p)
    for x, y in ((a[0], b[1]), (a[1], b[0]), (a[1], b[1])):
        e = fma(x, y, e)
    return fast_two_sum(p, e)


def dot2_term(acc, err, w, v):
    p = f32(w[0] * v[0])
    q = fma(w[0], v[0], -p)
    q = fma(w[0], v[1], q)
    q = fma(w[1], v[0], q)
    acc, e = two_sum(acc, p)
    return acc, f32(err + f32(e + q))


def dot2_pair(acc, err, w, a, b):
    s, t = two_sum(a[0], b[0])
    t = f32(t + f32(a[1] + b[1]))
    p = f32(w[0] * s)
    q = fma(w[0], s, -p)
    q = fma(w[0], t, q)
    q = fma(w[1], s, q)
    acc, e = two_sum(acc, p)
    return acc, f32(err + f32(e + q))


def test_split_keeps_48_bits():
    rng = np.random.default_rng(0)
    for _ in range(3000):
        x = float(rng.standard_normal() * 2.0 ** int(rng.integers(-40, 41)))
        h, l = pair_split(x)
        assert abs(Fr(x) - Fr(float(h)) - Fr(float(l))) <= Fr(2) ** -48 * abs(Fr(x))
    assert pair_split(0.0) == (0.0, 0.0)


def test_adjoint_update_within_stated_bound():
    """lam_out = lam + wc v_c + sum_d w_d (v- + v+), v = Ci lam, with lam of
    both signs (the case exact integer differences cannot take)."""
    rng = np.random.default_rng(1)
    bound = 0.0
    for _ in range(600):
        lam = rng.standard_normal(7) * 10.0 ** rng.uniform(-6, 3)
        ci = rng.uniform(0.4, 0.67, 7)
        w = list(rng.uniform(0.05, 0.2, 3))
        wc = -2.0 * sum(w)
        v = [mul_pair(pair_split(lam[i]), pair_split(ci[i])) for i in range(7)]
        wp = [pair_split(x) for x in w + [wc]]
        acc, err = pair_split(lam[0])
        acc, err = dot2_term(acc, err, wp[3], v[0])
        for d in range(3):
            acc, err = dot2_pair(acc, err, wp[d], v[1 + 2 * d], v[2 + 2 * d])
        out = float(Fr(float(acc)) + Fr(float(err)))  # the FP64 add: one rounding
        exact = Fr(lam[0]) + Fr(wc) * Fr(ci[0]) * Fr(lam[0]) + sum(
            Fr(w[d]) * (Fr(ci[1 + 2 * d]) * Fr(lam[1 + 2 * d]) + Fr(ci[2 + 2 * d]) * Fr(lam[2 + 2 * d]))
            for d in range(3))
        mag = abs(lam[0]) + abs(wc * ci[0] * lam[0]) + sum(
            w[d] * (abs(ci[1 + 2 * d] * lam[1 + 2 * d]) + abs(ci[2 + 2 * d] * lam[2 + 2 * d]))
            for d in range(3))
        bound = max(bound, float(abs(Fr(out) - exact)) / mag)
    assert bound <= 2.0 ** -45
