"""Accuracy of the rate kernel's own arithmetic building blocks, rebuilt on the CPU.

The kernel computes two things with arithmetic of its own rather than library calls, and the parity budget
(1e-10 relative for the FP64-accurate paths) rests on their stated accuracy:

* the FP64 Gaussian's exp(-u), table-driven after P. T. P. Tang (ACM TOMS 15 (1989) 144-157): v = 64 u, k = rint(v),
  exp(-u) = exp(-k/64) * p(k - v) with p the degree-5 Taylor polynomial of exp(t/64) in Horner form with fused
  multiply-adds; stated: truncation 3.2e-16 relative, a few units of 2^-53 in all;
* double-float arithmetic (a real as a pair of floats h + l, Dekker 1971): products with the high product exact
  through its fma residual, sums with Knuth's two-sum, about 2^-47 relative error per operation; the double-float
  exp of the same table method; |W|^2 from a double-float complex.

Each block is rebuilt here from its description (numpy float64 / float32 with every operation rounded to nearest;
a fused multiply-add as the product in a wider type plus the addend, rounded once to the target type) and compared
with long-double references on dense and random arguments.  The exp table is the correctly rounded exp(-k/64),
and one more ulp is allowed for the kernel's table, which CUDA's exp (1 ulp) fills.
"""
import numpy as np

LD = np.longdouble
F32 = np.float32
ULP64 = 2.0 ** -53


def fma64(a, b, c):
    return (np.asarray(a, LD) * np.asarray(b, LD) + np.asarray(c, LD)).astype(np.float64)


def fma32(a, b, c):
    return (np.asarray(a, np.float64) * np.asarray(b, np.float64) + np.asarray(c, np.float64)).astype(F32)


def table64():
    k = np.arange(264)
    return np.exp(-(k.astype(LD)) / LD(64)).astype(np.float64)


def exp_neg64(v, tab):
    """The FP64 kernel's exp(-v/64) for 0 <= v <= 256."""
    k = np.rint(v).astype(np.int64)
    t = k.astype(np.float64) - v
    p = np.full_like(v, (1.0 / 120.0) / 1073741824.0)
    for c in ((1.0 / 24.0) / 16777216.0, (1.0 / 6.0) / 262144.0, 0.5 / 4096.0, 1.0 / 64.0, 1.0):
        p = fma64(p, t, np.full_like(v, c))
    return tab[k] * p


def test_fp64_gaussian_exp_is_accurate_to_a_few_ulp():
    tab = table64()
    rng = np.random.Generator(np.random.PCG64(11))
    v = np.concatenate([np.linspace(0.0, 256.0, 200_001), rng.uniform(0.0, 256.0, 200_000),
                        np.arange(257) + 0.5, np.arange(257) - 0.5 + 1e-13])
    v = v[(v >= 0.0) & (v <= 256.0)]
    got = exp_neg64(v, tab)
    ref = np.exp(-(v.astype(LD)) / LD(64))
    rel = np.abs((got.astype(LD) - ref) / ref).astype(np.float64)
    # the polynomial's truncation (1/128)^6 / 6! = 3.2e-16, the roundings of the Horner steps, the table entry and
    # the final product: 5.0 units of 2^-53 measured; the kernel's table (CUDA exp, 1 ulp) may add about one more
    assert rel.max() <= 5.5 * ULP64, rel.max()
    assert rel.max() + 2 * ULP64 <= 1e-15


# ---------------------------------------------------------------------------------------------------- double-float
def df_make(v):
    h = np.asarray(v, np.float64).astype(F32)
    return h, (np.asarray(v, np.float64) - h.astype(np.float64)).astype(F32)


def df_fast(h, l):
    s = h + l
    return s, l - (s - h)


def df_mul(a, b):
    p = a[0] * b[0]
    e = fma32(a[0], b[1], fma32(a[1], b[0], fma32(a[0], b[0], -p)))
    return df_fast(p, e)


def df_add(a, b):
    s = a[0] + b[0]
    bb = s - a[0]
    e = (a[0] - (s - bb)) + (b[0] - bb)
    return df_fast(s, e + (a[1] + b[1]))


def df_value(a):
    return a[0].astype(LD) + a[1].astype(LD)


def table_df():
    return df_make(table64())


def df_exp_neg64(v, tab):
    """The double-float kernel's exp(-v/64) for 0 <= v <= 256, v a double-float."""
    kf = np.rint(v[0])
    k = kf.astype(np.int64)
    t = df_add((kf - v[0], np.zeros_like(kf)), (-v[1], np.zeros_like(kf)))
    c45 = fma32(np.full_like(kf, F32(1.0 / 128849018880.0)), t[0], np.full_like(kf, F32(1.0 / 402653184.0)))
    e3 = 1.0 / 1572864.0
    e3h = F32(e3)
    e3l = F32(e3 - float(e3h))
    p = df_add(df_mul((c45, np.zeros_like(kf)), t), (np.full_like(kf, e3h), np.full_like(kf, e3l)))
    for c in (1.0 / 8192.0, 1.0 / 64.0, 1.0):
        p = df_add(df_mul(p, t), (np.full_like(kf, F32(c)), np.zeros_like(kf)))
    return df_mul((tab[0][k], tab[1][k]), p)


def rand_df(rng, n, lo=-3.0, hi=3.0):
    x = rng.uniform(0.5, 1.0, n) * 2.0 ** rng.integers(lo, hi, n) * np.where(rng.random(n) < 0.5, 1.0, -1.0)
    return df_make(x)


def test_double_float_products_and_sums():
    rng = np.random.Generator(np.random.PCG64(12))
    n = 200_000
    a, b = rand_df(rng, n), rand_df(rng, n)
    prod = df_mul(a, b)
    ref = df_value(a) * df_value(b)
    # rounding of the two fused low-part steps (about 3 x 2^-48) and the dropped l l product (2^-48): below 2^-45
    assert (np.abs((df_value(prod) - ref) / ref).astype(np.float64)).max() <= 2.0 ** -45
    # sums of like signs (no cancellation, where a relative bound applies)
    b = (np.abs(b[0]) * np.sign(a[0]), np.abs(b[1]) * np.sign(a[0]) * np.sign(b[0]))
    tot = df_add(a, b)
    ref = df_value(a) + df_value(b)
    assert (np.abs((df_value(tot) - ref) / ref).astype(np.float64)).max() <= 2.0 ** -45
    # renormalised results: |l| <= ulp(h) / 2
    for h, l in (prod, tot):
        assert np.all(np.abs(l) <= np.spacing(np.abs(h)) / 2)


def test_double_float_gaussian_exp():
    tab = table_df()
    rng = np.random.Generator(np.random.PCG64(13))
    v64 = np.concatenate([np.linspace(0.0, 256.0, 100_001), rng.uniform(0.0, 256.0, 100_000)])
    v = df_make(v64)
    got = df_value(df_exp_neg64(v, tab))
    ref = np.exp(-df_value(v) / LD(64))
    rel = np.abs((got - ref) / ref).astype(np.float64)
    assert rel.max() <= 2.0 ** -44, rel.max()     # far inside the 1e-10 parity bound


def test_mixed_path_energy_difference():
    """The mixed path's dw for the Gaussian: two-float frequencies (h = fl32(w), l = fl32(w - h)), Knuth two-sums of
    the high parts, the low parts and the two-sum errors added in FP32, one final float.  Its error is the rounding
    of that float (2^-24 |dw|) plus at most 2^-44 of the sum of the frequencies.  The double-float path keeps the
    pair (high sum, low sum) instead of one float, which leaves at most 2^-46 of the sum."""
    def split(x):
        h = x.astype(F32)
        return h, (x - h.astype(np.float64)).astype(F32)

    def two_sum(a, b):
        s = a + b
        bb = s - a
        return s, (a - (s - bb)) + (b - bb)

    rng = np.random.Generator(np.random.PCG64(14))
    n = 400_000
    w0, w1, w2 = (np.exp(rng.uniform(np.log(0.05), np.log(150.0), n)) for _ in range(3))
    s1 = np.where(rng.random(n) < 0.5, 1.0, -1.0)
    s2 = np.where(rng.random(n) < 0.5, 1.0, -1.0)
    w3 = (w0 + s1 * w1 + s2 * w2) - rng.normal(size=n) * np.exp(rng.uniform(np.log(1e-9), np.log(20.0), n))
    k = w3 > 0.05
    w0, w1, w2, w3, s1, s2 = (x[k] for x in (w0, w1, w2, w3, s1, s2))
    (h0, l0), (h1, l1), (h2, l2), (h3, l3) = (split(x) for x in (w0, w1, w2, w3))
    g1, g2 = s1.astype(F32), s2.astype(F32)
    t, e1 = two_sum(h0, g1 * h1)
    t, e2 = two_sum(t, g2 * h2)
    t, e3 = two_sum(t, -h3)
    dwf = t + ((((l0 + g1 * l1) + g2 * l2) - l3) + ((e1 + e2) + e3))
    exact = (w0.astype(LD) + s1 * w1.astype(LD) + s2 * w2.astype(LD)) - w3.astype(LD)
    err = np.abs(dwf.astype(LD) - exact).astype(np.float64)
    S = w0 + w1 + w2 + w3
    assert np.all(err <= 2.0 ** -24 * np.abs(exact.astype(np.float64)) + 2.0 ** -44 * S)
    # the double-float path keeps dw as the exact pair (t, lo) of that two-sum: only the low parts' error is left
    pair = t.astype(LD) + ((((l0 + g1 * l1) + g2 * l2) - l3) + ((e1 + e2) + e3)).astype(LD)
    assert np.all(np.abs(pair - exact).astype(np.float64) <= 2.0 ** -46 * S)


def df_mac(h, l, ah, al, bh, bl):
    """(h, l) += (ah + al)(bh + bl) without renormalising l, as the vertex contraction accumulates."""
    p = ah * bh
    e = fma32(ah, bl, fma32(al, bh, fma32(ah, bh, -p)))
    s = h + p
    bb = s - h
    t = (h - (s - bb)) + (p - bb)
    return s, l + (t + e)


def test_double_float_complex_contraction():
    """Complex dot products of the vertex contraction's lengths (nb^2 = 9, 36, 144 terms) accumulated with the
    kernel's complex double-float multiply-add: the error stays below K 2^-46 of sum |a||b| (FP64 would give about
    K 2^-53), i.e. FP64-grade for the 1e-10 parity bound."""
    rng = np.random.Generator(np.random.PCG64(15))
    n = 20_000
    for K in (9, 36, 144):
        a = rng.normal(size=(n, K)) + 1j * rng.normal(size=(n, K))
        b = rng.normal(size=(n, K)) + 1j * rng.normal(size=(n, K))
        (arh, arl), (aih, ail) = df_make(a.real), df_make(a.imag)
        (brh, brl), (bih, bil) = df_make(b.real), df_make(b.imag)
        rh = rl = ih = il = np.zeros(n, F32)
        for k in range(K):
            rh, rl = df_mac(rh, rl, arh[:, k], arl[:, k], brh[:, k], brl[:, k])
            rh, rl = df_mac(rh, rl, -aih[:, k], -ail[:, k], bih[:, k], bil[:, k])
            ih, il = df_mac(ih, il, arh[:, k], arl[:, k], bih[:, k], bil[:, k])
            ih, il = df_mac(ih, il, aih[:, k], ail[:, k], brh[:, k], brl[:, k])
        ar = arh.astype(LD) + arl.astype(LD)
        ai = aih.astype(LD) + ail.astype(LD)
        br = brh.astype(LD) + brl.astype(LD)
        bi = bih.astype(LD) + bil.astype(LD)
        ref_re = np.sum(ar * br - ai * bi, axis=1)
        ref_im = np.sum(ar * bi + ai * br, axis=1)
        scale = np.sum(np.abs(a) * np.abs(b), axis=1)
        err = np.maximum(np.abs(rh.astype(LD) + rl.astype(LD) - ref_re),
                         np.abs(ih.astype(LD) + il.astype(LD) - ref_im)).astype(np.float64)
        assert np.all(err <= K * 2.0 ** -46 * scale), (K, (err / scale).max())
