"""The error model behind the double-word FP32 passes over the low-rank basis, checked on the CPU
with an independent float32 restatement of the published algorithms: Knuth's TwoSum, Dekker's
TwoProduct (Veltkamp splitting, no FMA needed), and the Dot2 accumulation of Ogita, Rump and Oishi
(SIAM J. Sci. Comput. 26, 2005) on double-word inputs x = x_hi + x_lo.

Claims pinned (relative to the sum of the absolute products; exact reference by rational arithmetic):
- summed in short Dot2 chains combined by double-word trees (the X^T V reductions: 16-term chains per
  lane, warp and block trees), the error is a few units of 2^-48, the double-word precision (~1e-14);
- one chain of n terms (a candidate vector entry sums r <= 256 products in one chain) stays below
  4 n u^2 (u = 2^-24; ~4e-12 at n = 256), Dot2's second-order term;
- plain float32 accumulation is orders of magnitude worse.
All are far below the 1e-11 / 1e-10 bounds of the low-rank parity tests."""
from fractions import Fraction

import numpy as np
import pytest

f32 = np.float32


def two_sum(a, b):
    s = f32(a + b)
    bb = f32(s - a)
    return s, f32(f32(a - f32(s - bb)) + f32(b - bb))


def split(a):
    # Veltkamp splitting of a float32 into two 12-bit halves (factor 2^12 + 1)
    c = f32(f32(4097.0) * a)
    hi = f32(c - f32(c - a))
    return hi, f32(a - hi)


def two_prod(a, b):
    p = f32(a * b)
    ah, al = split(a)
    bh, bl = split(b)
    e = f32(f32(f32(f32(ah * bh) - p) + f32(ah * bl)) + f32(al * bh))
    return p, f32(e + f32(al * bl))


def dw_of(v):
    h = f32(v)
    return h, f32(v - float(h))


def dot2_dw(xs, ys):
    """Dot2 over double-word pairs: high products summed by TwoSum, every error term (product
    error, cross terms x_hi y_lo + x_lo y_hi, sum error) in a second float."""
    sh, sl = f32(0), f32(0)
    for (xh, xl), (yh, yl) in zip(xs, ys):
        p, e = two_prod(xh, yh)
        e = f32(e + f32(f32(xh * yl) + f32(xl * yh)))
        sh, t = two_sum(sh, p)
        sl = f32(sl + f32(t + e))
    return float(sh) + float(sl)


def dw_add(a, b):
    """Sum of two double-words (TwoSum of the high parts, low parts added, renormalised)."""
    s, t = two_sum(a[0], b[0])
    t = f32(t + f32(a[1] + b[1]))
    h = f32(s + t)
    return h, f32(t - f32(h - s))


def dot2_chains(xs, ys, chain):
    """The kernels' structure: Dot2 chains of at most `chain` products (one lane's share), the chain
    results combined pairwise by double-word sums (the warp and block trees)."""
    parts = []
    for i in range(0, len(xs), chain):
        sh, sl = f32(0), f32(0)
        for (xh, xl), (yh, yl) in zip(xs[i:i + chain], ys[i:i + chain]):
            p, e = two_prod(xh, yh)
            e = f32(e + f32(f32(xh * yl) + f32(xl * yh)))
            sh, t = two_sum(sh, p)
            sl = f32(sl + f32(t + e))
        h = f32(sh + sl)
        parts.append((h, f32(sl - f32(h - sh))))
    while len(parts) > 1:
        parts = [dw_add(parts[k], parts[k + 1]) if k + 1 < len(parts) else parts[k] for k in range(0, len(parts), 2)]
    return float(parts[0][0]) + float(parts[0][1])


def exact_dot(x, y):
    return float(sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(x, y)))


U = 2.0 ** -24          # float32 unit roundoff


@pytest.mark.parametrize("n,cancel", [(256, False), (256, True), (512, False), (2048, False), (2048, True)])
def test_dot2_on_double_words_meets_the_double_word_bound(n, cancel):
    rng = np.random.default_rng(20261204 + n)
    x = rng.standard_normal(n)
    y = rng.standard_normal(n)
    if cancel:                         # an orthogonalised-like case: the sum nearly cancels
        y -= x * (x @ y) / (x @ x)
    xs = [dw_of(v) for v in x]
    ys = [dw_of(v) for v in y]
    ref = exact_dot(x, y)
    scale = float(np.sum(np.abs(x * y)))
    # short chains combined by double-word trees: a few units of 2^-48 (~1e-14)
    for chain in (16, 32, 64):
        err = abs(dot2_chains(xs, ys, chain) - ref) / scale
        assert err < 8 * 2.0 ** -48, (chain, err)
    # one long chain: the second float's own rounding grows like n u^2 (Dot2's error term)
    err1 = abs(dot2_dw(xs, ys) - ref) / scale
    assert err1 < 4 * n * U * U, err1
    naive = float(np.sum((x.astype(f32) * y.astype(f32)).astype(f32), dtype=f32))
    assert abs(naive - ref) / scale > 1e3 * 8 * 2.0 ** -48


def test_two_sum_and_two_prod_are_error_free():
    rng = np.random.default_rng(7)
    for _ in range(2000):
        a, b = f32(rng.standard_normal() * 10.0 ** rng.integers(-5, 5)), f32(rng.standard_normal())
        s, t = two_sum(a, b)
        assert Fraction(float(s)) + Fraction(float(t)) == Fraction(float(a)) + Fraction(float(b))
        p, e = two_prod(a, b)
        assert Fraction(float(p)) + Fraction(float(e)) == Fraction(float(a)) * Fraction(float(b))
