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
        ok = ok and -(1 << 22) <= h < (1 << 22)
        # the high half read off the bits of the FP32 number 1.5 2^23 + h
        # (the integer sum h + 0x4B400000), minus 1.5 2^23
        mh = u2f(h + 0x4B400000) if ok else f32(1.5 * 2 ** 23)
        gh.append(f32(mh - f32(1.5 * 2 ** 23)))
        assert not ok or float(gh[-1]) == h
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
    ones (group sums near 2^44) stay within the bound; stencils leaving the
    binade or with a group sum outside [-2^45, 2^45) are refused."""
    rng = np.random.default_rng(3)
    worst, nok = check(2, (0.03, 0.12, 0.12), stencils(rng, 300, 1e-4, sign=-1.0))
    assert nok > 200 and worst <= 1.0
    worst, nok = check(2, (0.03, 0.12, 0.12), stencils(rng, 300, 2e-3, base=(2.3, 3.5)))
    assert worst <= 1.0 and nok > 0
    # a stencil across 2.0 (two exponents) and one with |G| >= 2^47 are refused,
    # and so is one with 2^45 <= G < 2^47 (outside the high half's bit-move
    # range, G < 2^45 - 2^22)
    w = (0.03, 0.12, 0.12)
    assert not fast_cell(2.0000001, (1.9999999,) + (2.0000001,) * 5, 0.5, w, 2)[1]
    assert not fast_cell(3.9, (2.1, 2.2, 3.9, 3.9, 3.9, 3.9), 0.5, w, 2)[1]
    t = 3.0
    for k in (45, 46):  # x group sum G = 2^k units of ulp(3.0) = 2^-51
        nb = (from_bits(bits(t) + (1 << (k - 1))), from_bits(bits(t) + (1 << (k - 1))), t, t, t, t)
        G = bits(nb[0]) + bits(nb[1]) - 2 * bits(t)
        assert G == 1 << k
        assert not fast_cell(t, nb, 0.5, w, 2)[1]
    d = (1 << 44) - (1 << 21) - 1  # G = 2^45 - 2^22 - 2: the largest even sum taken
    nb = (from_bits(bits(t) + d), from_bits(bits(t) + d), t, t, t, t)
    assert fast_cell(t, nb, 0.5, (1e-6, 1e-6, 1e-6), 1)[1]


def test_high_half_bit_move_exact():
    """The high half Gh = (G + 2^22) >> 23 read off the bits Gh + 0x4B400000
    as an FP32 number minus 1.5 2^23 is exactly Gh for G in
    [-2^45 - 2^22, 2^45 - 2^22) (Gh in [-2^22, 2^22)), and the range test on
    those bits accepts exactly that interval."""
    rng = np.random.default_rng(5)
    lo, hi = -(2 ** 45) - (1 << 22), 2 ** 45 - (1 << 22)
    Gs = [int(g) for g in rng.integers(lo, hi, 2000)]
    Gs += [lo, hi - 1, 0, -1, (1 << 22) - 1, -(1 << 22)]
    for G in Gs:
        h = (G + (1 << 22)) >> 23
        m = (h + 0x4B400000) & 0xFFFFFFFF
        assert (m ^ 0x4B000000) < (1 << 23)
        assert float(f32(u2f(m) - f32(1.5 * 2 ** 23))) == h
    for G in (hi, 2 ** 45, 2 ** 46, lo - 1, -(2 ** 46)):
        h = (G + (1 << 22)) >> 23
        m = (h + 0x4B400000) & 0xFFFFFFFF
        assert (m ^ 0x4B000000) >= (1 << 23)


def test_split_halves_exact():
    rng = np.random.default_rng(4)
    for G in list(rng.integers(-(2 ** 46), 2 ** 46, 2000)) + [0, -1, 1, 2 ** 22, -(2 ** 22), 2 ** 46 - 1]:
        G = int(G)
        h = (G + (1 << 22)) >> 23
        lo = (G + (1 << 22)) & 0xFFFFFFFF
        l = float(u2f((lo & 0x7FFFFF) | 0x4B000000)) - 1.5 * 2 ** 23
        assert h * (1 << 23) + l == G and -(2 ** 22) <= l < 2 ** 22
        assert float(f32(h)) == h and float(f32(l)) == l


# ---------------------------------------------------------------------------
# The aligned path: stencils across powers of two or across zero
# ---------------------------------------------------------------------------
def aligned_cell(tc, nb, ci, w, ng):
    """(T2, ok, er, P) of the aligned path: every value on the grid of
    u = 2^(er-1075) (er the largest exponent field), rounded half up and
    signed relative to the centre; the fast path's split and sums; two FP64
    FMAs (C u first, then S u)."""
    bc = bits(tc)
    vals = [bc] + [bits(v) for v in nb]
    er = max(max((b >> 52) & 0x7FF for b in vals), 1)

    def al(b):
        e = (b >> 52) & 0x7FF
        m = (b & (2 ** 52 - 1)) | ((e != 0) << 52)
        d = min(er - max(e, 1), 63)
        q = (m + (1 << (d - 1))) >> d if d else m
        return -q if (b ^ bc) >> 63 else q

    I = [al(b) for b in vals[1:]]
    c2 = 2 * al(bc)
    D = [I[2 * d] + I[2 * d + 1] - c2 for d in range(3)]
    ok = 180 <= er <= 2008
    gh, gl = [], []
    for grp in groups(ng):
        G = sum(D[d] for d in grp)
        h = (G + (1 << 22)) >> 23
        ok = ok and abs(h) < (1 << 24)
        gh.append(f32(h))
        gl.append(f32(u2f((((G + (1 << 22)) & 0x7FFFFF) | 0x4B000000)) - f32(1.5 * 2 ** 23)))
    wg = [split_w(w[grp[0]]) for grp in groups(ng)]
    ah = [f32(a * f32(2.0 ** 23)) for a, _ in wg]
    al_ = [f32(b * f32(2.0 ** 23)) for _, b in wg]
    bh = [a for a, _ in wg]
    P = [fma(ah[g], gh[g], f32(0)) for g in range(ng)]
    Ee = [fma(ah[g], gh[g], -P[g]) for g in range(ng)]
    R = fma(bh[0], gl[0], f32(0))
    for g in range(1, ng):
        R = fma(bh[g], gl[g], R)
    for g in range(ng):
        R = fma(al_[g], gh[g], R)
    if ng == 1:
        S, C = P[0], f32(Ee[0] + R)
    elif ng == 2:
        S, e = two_sum(P[0], P[1])
        C = f32(f32(Ee[0] + Ee[1]) + f32(e + R))
    else:
        s1, e1 = two_sum(P[0], P[1])
        S, e2 = two_sum(s1, P[2])
        C = f32(f32(f32(Ee[0] + Ee[1]) + f32(Ee[2] + e1)) + f32(e2 + R))
    u = Fr(2) ** (er - 1075)
    sg = -1 if bc >> 63 else 1
    t1 = float(Fr(tc) + sg * Fr(ci) * Fr(float(C)) * u)
    t2 = float(Fr(t1) + sg * Fr(ci) * Fr(float(S)) * u)
    return t2, ok, er, [Fr(float(p)) for p in P]


def check_aligned(ng, w, cases, seed=8):
    rng = np.random.default_rng(seed)
    worst, nok = 0.0, 0
    for tc, nb in cases:
        ci = float(rng.uniform(0.4, 0.67))
        r, ok, er, P = aligned_cell(tc, nb, ci, w, ng)
        if not ok:
            continue
        nok += 1
        u = Fr(2) ** (er - 1075)
        mag = Fr(ci) * sum(abs(p) for p in P) * u
        # rounding of the values to u, one rounding per FMA (|T2| < 2^(er-1022)),
        # and 2^-44 of the weighted sum's terms
        bound = (2 * Fr(ci) * sum(Fr(x) for x in w) + 1) * u + Fr(2) ** -44 * mag
        worst = max(worst, float(abs(Fr(r) - exact_step(tc, nb, ci, w)) / bound))
    return worst, nok


def smooth_stencils(rng, n, centre, h=1e-3):
    """Stencils of smooth fields a + b.x + c x^2 around the given centres."""
    out = []
    for _ in range(n):
        t = centre(rng)
        g = rng.standard_normal(3) * 0.5
        c = rng.standard_normal(3) * 0.5
        nb = tuple(float(t + s * g[d] * h + c[d] * h * h) for d in range(3) for s in (-1, 1))
        out.append((t, nb))
    return out


def test_aligned_cell_within_bound_across_zero_and_powers_of_two():
    rng = np.random.default_rng(9)
    w = (0.0412, 0.1653, 0.1653)
    # across zero: centres within a few h of 0, neighbours of both signs
    across0 = smooth_stencils(rng, 300, lambda r: float(r.uniform(-3e-3, 3e-3)))
    # across powers of two: centres at 2^k (1 - small)
    across2 = smooth_stencils(rng, 300, lambda r: float(2.0 ** r.integers(-3, 4) * (1 + r.uniform(-1e-3, 1e-3))))
    for cases, ng, wt in ((across0, 2, w), (across2, 2, w), (across0, 1, (0.16,) * 3),
                          (across2, 3, (0.05, 0.09, 0.013))):
        worst, nok = check_aligned(ng, wt, cases)
        assert nok > 250 and worst <= 1.0, (ng, worst, nok)


def test_aligned_integers_equal_bit_differences_on_one_binade():
    """On stencils of one sign and one exponent the aligned integers are the
    significands themselves: the group sums equal the fast path's bit-pattern
    differences (negated for negative values)."""
    rng = np.random.default_rng(10)
    for sign in (1.0, -1.0):
        for tc, nb in stencils(rng, 100, 1e-5, sign=sign):
            bc = bits(tc)
            if any((bits(v) >> 52) != (bc >> 52) for v in nb):
                continue
            D_fast = [bits(nb[2 * d]) + bits(nb[2 * d + 1]) - 2 * bc for d in range(3)]
            mant = lambda b: (b & (2 ** 52 - 1)) | (1 << 52)  # noqa: E731
            D_al = [mant(bits(nb[2 * d])) + mant(bits(nb[2 * d + 1])) - 2 * mant(bc) for d in range(3)]
            assert D_fast == D_al


def test_aligned_path_refuses_large_relative_curvature():
    """A stencil whose group sum reaches 2^47 units of its largest value's ulp
    (relative second difference near 2^-5) is left to the FP64 cell."""
    w = (0.03, 0.12, 0.12)
    assert not aligned_cell(1e-3, (1e-3, 1e-3, 1e-3, 1e-3, -1e-3, 1.3e-3), 0.5, w, 2)[1]
    assert aligned_cell(1e-3, (1.001e-3, 0.999e-3, 1e-3, 1e-3, 0.998e-3, 1.002e-3), 0.5, w, 2)[1]
