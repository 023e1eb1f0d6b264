"""CPU model of the float-pair (double-float) arithmetic of the float64-accurate
triangle kernel (Alg. 6 line 11, Eq. 34), in numpy float32.

The kernel forms H^XYZ = sum_I (E^XY F^XZ + E^XZ F^XY) G^YZ with every float64
operand split into float32 pairs x = x_h + x_l, TwoProduct by FMA and TwoSum
(Knuth) for the exact parts.  This model repeats its operations one for one
(float32 round-to-nearest arithmetic; an FMA as the float64 product, exact for
float32 factors, plus the addend, rounded once more to float32) and checks the
result against the exact rational sum:
  * error within 2^-42 of sum_I |E F G| for operands of one scale and for
    operands spread over many binades.  Per term the scheme is exact up to
    the dropped low*low products (2^-48) and the roundings of the low words:
    the low word of t collects four cross products and two exact errors, each
    FMA rounding at 2^-24 of a value up to about 4 * 2^-24 |t|, about
    13.5 * 2^-47 = 2^-43.2 of |E F G| in the worst case (float64: 2^-53);
  * planted mistakes each break that bound: dropping the TwoSum error of the
    accumulation, dropping the TwoProduct error of t, and accumulating in plain
    float32.
"""
from fractions import Fraction

import numpy as np
import pytest

f32 = np.float32


def split(d):
    h = d.astype(f32)
    l = (d - h.astype(np.float64)).astype(f32)
    return h, l


def fma(a, b, c):
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(f32)


def dot2(aH, aL, bH, bL, cH, cL, dH, dL, drop_prod_err=False):
    """t = a b + c d as a float pair (th, tl)."""
    p1 = aH * bH
    e1 = fma(aH, bH, -p1)
    p2 = cH * dH
    e2 = fma(cH, dH, -p2)
    if drop_prod_err:
        e1 = np.zeros_like(e1)
        e2 = np.zeros_like(e2)
    s = p1 + p2
    z = s - p1
    es = (p1 - (s - z)) + (p2 - z)
    lo = fma(aH, bL, e1)
    lo = fma(aL, bH, lo)
    lo = fma(cH, dL, lo)
    lo = fma(cL, dH, lo)
    lo = lo + e2
    return s, lo + es


def acc(Sh, Sl, th, tl, gH, gL, drop_sum_err=False):
    """(Sh, Sl) -= t g (the kernel accumulates -H)."""
    thn = f32(0) - th
    qn = thn * gH
    e = fma(th, gH, qn)
    low = fma(th, gL, e)
    low = fma(tl, gH, low)
    s = Sh + qn
    z = s - Sh
    es = (Sh - (s - z)) + (qn - z)
    if drop_sum_err:
        es = np.zeros_like(es)
    Sl = (Sl + es) - low
    return s, Sl


def model(E1, F2, E2, F1, G, **kw):
    """H = sum_I (E1 F2 + E2 F1) G over axis 0, every array (nI, n) float64."""
    n = E1.shape[1]
    Sh = np.zeros(n, f32)
    Sl = np.zeros(n, f32)
    for I in range(E1.shape[0]):
        a = split(E1[I]); b = split(F2[I]); c = split(E2[I]); d = split(F1[I]); g = split(G[I])
        th, tl = dot2(*a, *b, *c, *d, drop_prod_err=kw.get("drop_prod_err", False))
        Sh, Sl = acc(Sh, Sl, th, tl, *g, drop_sum_err=kw.get("drop_sum_err", False))
    return -(Sh.astype(np.float64) + Sl.astype(np.float64))


def plain_f32(E1, F2, E2, F1, G):
    S = np.zeros(E1.shape[1], f32)
    for I in range(E1.shape[0]):
        S = S + (E1[I].astype(f32) * F2[I].astype(f32) + E2[I].astype(f32) * F1[I].astype(f32)) \
            * G[I].astype(f32)
    return S.astype(np.float64)


def exact(E1, F2, E2, F1, G):
    out = []
    for k in range(E1.shape[1]):
        s = Fraction(0)
        for I in range(E1.shape[0]):
            s += (Fraction(E1[I, k]) * Fraction(F2[I, k]) + Fraction(E2[I, k]) * Fraction(F1[I, k])) \
                * Fraction(G[I, k])
        out.append(s)
    return out


def operands(seed, nI, n, spread):
    rng = np.random.default_rng(seed)

    def draw():
        x = rng.standard_normal((nI, n))
        if spread:
            x *= 2.0 ** rng.integers(-40, 1, size=(nI, n))
        return x
    return draw(), draw(), draw(), draw(), draw()


def max_scaled_error(H, ref, E1, F2, E2, F1, G):
    scale = (np.abs(E1 * F2) + np.abs(E2 * F1)) * np.abs(G)
    scale = scale.sum(axis=0)
    err = np.array([abs(Fraction(float(h)) - r) for h, r in zip(H, ref)], dtype=float)
    return float(np.max(err / scale))


@pytest.mark.parametrize("spread", [False, True], ids=["one_scale", "spread_2^-40"])
def test_float_pair_triangle_within_bound(spread):
    ops = operands(7 + spread, 600, 24, spread)
    ref = exact(*ops)
    r = max_scaled_error(model(*ops), ref, *ops)
    print(f"max |H - exact| / sum|E F G| = {r:.2e} (2^-42 = {2.0 ** -42:.2e})")
    assert r < 2.0 ** -42


@pytest.mark.parametrize("mistake", ["drop_sum_err", "drop_prod_err", "plain_f32"])
def test_planted_mistakes_break_the_bound(mistake):
    ops = operands(11, 600, 24, False)
    ref = exact(*ops)
    H = plain_f32(*ops) if mistake == "plain_f32" else model(*ops, **{mistake: True})
    r = max_scaled_error(H, ref, *ops)
    print(f"{mistake}: {r:.2e}")
    assert r > 2.0 ** -38
