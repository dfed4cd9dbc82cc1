"""The fast path of the emulated FP64 step cell (one FP64 FMA per point)
modelled step by step in FP32 with numpy and checked against exact rational
arithmetic: the bit-pattern second differences, the exact split of each
group sum into two FP32 halves, the error-free products and two-sums, the
FP64 FMA with |S| u and the integer ulp correction. The result must lie
within 1.25 ulps of T2 plus 2^-44 of Ci sum_g |w_g G_g| u of the exact update
T + Ci sum_d w_d d2_d (Fig. 1's step with the weights w_d = dt lam / dd^2).
Independent of the GPU code (a model of the method, not of its
implementation)."""
import math
import struct
from fractions import Fraction as Fr

import numpy as np

f32 = np.float32


def bits(x):
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def from_bits(b):
    return struct.unpack("<d", struct.pack("<Q", b & 0xFFFFFFFFFFFFFFFF))[0]


def u2f(u):
    return f32(struct.unpack("<f", struct.pack("<I", u & 0xFFFFFFFF))[0])


def fma(a, b, c):
    return f32(float(Fr(float(a)) * Fr(float(b)) + Fr(float(c))))


def two_sum(a, b):
    s = f32(a + b)
    bb = f32(s - a)
    return s, f32(f32(a - f32(s - bb)) + f32(b - bb))


def split_w(w):
    wh = f32(w)
    wl = f32(w - float(wh))
    return wh, wl


def groups(ng):
    return {1: [(0, 1, 2)], 2: [(0,), (1, 2)], 3: [(0,), (1,), (2,)]}[ng]


def fast_cell(tc, nb, ci, w, ng):
    """(T2, ok) of the fast path; nb = x-, x+, y-, y+, z-, z+; w = (wx, wy, wz)."""
    bc = bits(tc)
    hc = bc >> 32
    o = 0
    for v in nb:
        o |= (bits(v) >> 32) ^ hc
    E = (hc >> 20) & 0x7FF
    ok = o < (1 << 20) and 180 <= E <= 2008
    D = [(bits(nb[2 * d]) + bits(nb[2 * d + 1]) - 2 * bc) for d in range(3)]
    gh, gl = [], []
    for grp in groups(ng):
        G = sum(D[d] for d in grp)            # exact (Python integers)
        h = (G + (1 << 22)) >> 23             # floor, i.e. rounded half up
        l = G - (h << 23)                     # in [-2^22, 2^22)
        assert -(1 << 22) <= l < (1 << 22)
        ok = ok and abs(h) < (1 << 24)
        gh.append(f32(h))
        # the low half read off the bits of the FP32 number 1.5 2^23 + l
        m = u2f((((G + (1 << 22)) & 0x7FFFFF) | 0x4B000000))
        assert float(m) == 1.5 * 2 ** 23 + l
        gl.append(f32(m - f32(1.5 * 2 ** 23)))
    wg = [split_w(w[grp[0]]) for grp in groups(ng)]
    ah = [f32(a * f32(2.0 ** 23)) for a, _ in wg]
    al = [f32(b * f32(2.0 ** 23)) for _, b in wg]
    bh = [a for a, _ in wg]
    P = [fma(ah[g], gh[g], f32(0)) for g in range(ng)]
    Ee = [fma(ah[g], gh[g], -P[g]) for g in range(ng)]
    R = fma(bh[0], gl[0], f32(0))
    for g in range(1, ng):
        R = fma(bh[g], gl[g], R)
    for g in range(ng):
        R = fma(al[g], gh[g], R)
    if ng == 1:
        S, C = P[0], f32(Ee[0] + R)
    elif ng == 2:
        S, e = two_sum(P[0], P[1])
        C = f32(f32(Ee[0] + Ee[1]) + f32(e + R))
    else:
        s1, e1 = two_sum(P[0], P[1])
        S, e2 = two_sum(s1, P[2])
        C = f32(f32(f32(Ee[0] + Ee[1]) + f32(Ee[2] + e1)) + f32(e2 + R))
    # Ci truncated to FP32 from its bit pattern
    cb = bits(ci)
    cih, cil = cb >> 32, cb & 0xFFFFFFFF
    ok = ok and 897 <= (cih >> 20) <= 1150 and cih >> 31 == 0
    cif = u2f((((cih - (896 << 20)) << 3) | (cil >> 29)) & 0xFFFFFFFF)
    Kr = fma(cif, C, f32(1.5 * 2 ** 23))      # rint(cif C) + 1.5 2^23 when |cif C| < 2^22
    ok = ok and math.isfinite(float(Kr)) and abs(float(Kr) - 1.5 * 2 ** 23) < 2.0 ** 22
    k = int(float(Kr) - 1.5 * 2 ** 23) if ok else 0
    # one FP64 FMA: T + (+-Ci) |S| u, u = 2^(E-1075), the sign of T and of S on Ci
    u = Fr(2) ** (E - 1075)
    sgn = -1 if (hc >> 31) ^ (float(S) < 0) else 1
    t2 = float(Fr(tc) + sgn * Fr(ci) * abs(Fr(float(S))) * u)
    r = bits(t2) + k
    ok = ok and ((r >> 32) ^ hc) & 0xFFF00000 == 0
    return from_bits(r), ok, E, [Fr(float(P[g])) for g in range(ng)]


def exact_step(tc, nb, ci, w):
    d2 = [Fr(nb[2 * d + 1]) - Fr(tc) - (Fr(tc) - Fr(nb[2 * d])) for d in range(3)]
    return Fr(tc) + Fr(ci) * sum(Fr(w[d]) * d2[d] for d in range(3))


def stencils(rng, n, rel, sign=1.0, base=(1.7, 2.7)):
    out = []
    for _ in range(n):
        t = rng.uniform(*base)
        nb = tuple(float(t * (1 + rel * rng.standard_normal())) for _ in range(6))
        out.append((sign * t, tuple(sign * v for v in nb)))
    return out


def check(ng, w, cases, ci_range=(0.4, 0.67)):
    rng = np.random.default_rng(7)
    worst, nok = 0.0, 0
    for tc, nb in cases:
        ci = float(rng.uniform(*ci_range))
        r, ok, E, P = fast_cell(tc, nb, ci, w, ng)
        if not ok:
            continue
        nok += 1
        exact = exact_step(tc, nb, ci, w)
        u = Fr(2) ** (E - 1075)
        mag = Fr(ci) * sum(abs(p) for p in P) * u
        err = abs(Fr(r) - exact)
        # the FMA's and the correction's roundings (one ulp of T2, in T's
        # binade), the FP32 roundings of the small terms (a quarter ulp at
        # these weights) and 2^-44 of the weighted sum's terms
        bound = Fr(5, 4) * u + Fr(2) ** -44 * mag
        worst = max(worst, float(err / bound))
    return worst, nok


def test_fast_cell_within_bound_two_groups():
    rng = np.random.default_rng(1)
    w = (0.0412, 0.1653, 0.1653)
    worst, nok = check(2, w, stencils(rng, 400, 1e-4))
    assert nok > 300 and worst <= 1.0


def test_fast_cell_within_bound_one_and_three_groups():
    rng = np.random.default_rng(2)
    worst1, n1 = check(1, (0.16, 0.16, 0.16), stencils(rng, 300, 3e-5))
    worst3, n3 = check(3, (0.05, 0.09, 0.013), stencils(rng, 300, 3e-5))
    assert n1 > 200 and n3 > 200 and max(worst1, worst3) <= 1.0


def test_fast_cell_negative_values_and_rough_stencils():
    """Negative stencils (bit differences carry the opposite sign) and rough
    ones (group sums near 2^46) stay within the bound; stencils leaving the
    binade or with |G| >= 2^47 are refused."""
    rng = np.random.default_rng(3)
    worst, nok = check(2, (0.03, 0.12, 0.12), stencils(rng, 300, 1e-4, sign=-1.0))
    assert nok > 200 and worst <= 1.0
    worst, nok = check(2, (0.03, 0.12, 0.12), stencils(rng, 300, 2e-3, base=(2.3, 3.5)))
    assert worst <= 1.0 and nok > 0
    # a stencil across 2.0 (two exponents) and one with |G| >= 2^47 are refused
    w = (0.03, 0.12, 0.12)
    assert not fast_cell(2.0000001, (1.9999999,) + (2.0000001,) * 5, 0.5, w, 2)[1]
    assert not fast_cell(3.9, (2.1, 2.2, 3.9, 3.9, 3.9, 3.9), 0.5, w, 2)[1]


def test_split_halves_exact():
    rng = np.random.default_rng(4)
    for G in list(rng.integers(-(2 ** 46), 2 ** 46, 2000)) + [0, -1, 1, 2 ** 22, -(2 ** 22), 2 ** 46 - 1]:
        G = int(G)
        h = (G + (1 << 22)) >> 23
        lo = (G + (1 << 22)) & 0xFFFFFFFF
        l = float(u2f((lo & 0x7FFFFF) | 0x4B000000)) - 1.5 * 2 ** 23
        assert h * (1 << 23) + l == G and -(2 ** 22) <= l < 2 ** 22
        assert float(f32(h)) == h and float(f32(l)) == l
