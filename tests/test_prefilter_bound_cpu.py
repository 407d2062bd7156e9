"""The FP32 prefilter of the energy window settles only decisions that the FP64 definition takes the same way.

The rate kernel screens each candidate with single-precision arithmetic and decides in FP64 (the order of the
definition, Sec. 2.4 window |dw| <= window * max(sigma, sigma_min)) only inside a band around the window edge.
Its margins rest on two error bounds stated beside the kernel:

* dw~ = ((h0 +- h') +- h'') - h''' from h = fl32(omega) differs from the FP64 dw by at most 4.1 u S, u = 2^-24,
  S = the sum of the four frequencies; the margin is 2^-19 S (about 8x that);
* sigma~ from two-float velocities (h + l, Knuth two-sum of the velocity difference, an FMA sum of squares, a
  correctly rounded square root) differs from the FP64 sigma by at most E = 2^-19 sigma~ + 2^-40 sb dq |v|_1.

This test rebuilds that single-precision arithmetic with numpy float32 (every operation rounded to nearest, as
the kernel's __fadd_rn / __fmul_rn; the fused multiply-add as the float64 product, exact for float32 inputs,
plus the addend, rounded once more to float32) on candidates drawn to sit at the window edge, and checks both
bounds and that every candidate the prefilter accepts or rejects is accepted or rejected by the FP64 rule.
"""
import numpy as np

F32 = np.float32
U = 2.0 ** -24
K_REL_S = F32(2.0 ** -19)
K_REL_P = F32(2.0 ** -22)
K_ABS_V = F32(2.0 ** -40)


def f32(x):
    return np.asarray(x, dtype=np.float64).astype(F32)


def fma32(a, b, c):
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(F32)


def two_sum(a, b):
    s = a + b
    bb = s - a
    e = (a - (s - bb)) + (b - bb)
    return s, e


def split(x):
    """Two-float form h + l of a double."""
    h = f32(x)
    return h, f32(np.asarray(x) - h.astype(np.float64))


def sigma_prefilter(v_leg, v3, sign, sb, dq, window, sigma_min):
    """(P~, margin) of the kernel's FP32 sigma entry, the FP64 entry P64 = window * max(sigma, sigma_min), and
    whether the FP32 entry settled the sigma_min relation (elsewhere the kernel takes the exact entry)."""
    vlh, vll = split(v_leg)
    v3h, v3l = split(v3)
    s = F32(sign)
    d = []
    v1n = np.zeros(v_leg.shape[0], F32)
    for c in range(3):
        h, e = two_sum(s * vlh[:, c], -v3h[:, c])
        d.append(h + (e + (s * vll[:, c] - v3l[:, c])))
        v1n = v1n + (np.abs(vlh[:, c]) + np.abs(v3h[:, c]))
    sbdq = f32(sb * dq)
    sig = sbdq * np.sqrt(fma32(d[0], d[0], fma32(d[1], d[1], d[2] * d[2])))
    E = K_REL_S * sig + K_ABS_V * sbdq * v1n
    # FP64 sigma in the definition's order
    dv = sign * v_leg - v3
    sig64 = (sb * np.sqrt((dv[:, 0] * dv[:, 0] + dv[:, 1] * dv[:, 1]) + dv[:, 2] * dv[:, 2])) * dq
    P64 = window * np.maximum(sig64, sigma_min)
    smin, win = F32(sigma_min), F32(window)
    big = sig - E > F32(2.0) * smin
    small = sig + E < F32(0.5) * smin
    P = np.where(big, win * sig, f32(window * sigma_min))
    M = np.where(big, win * E + K_REL_P * P, K_REL_P * P)
    return P, M, P64, sig, E, sig64, big | small


def dw_prefilter(w0, wx, wy, w3, s1, s2):
    """dw~ and the kernel's sum margin 2^-19 ((h0 + h') + h'' + h''') from the FP32 frequencies."""
    h0, hx, hy, h3 = f32(w0), f32(wx), f32(wy), f32(w3)
    t = np.where(s1 > 0, h0 + hx, h0 - hx)
    t = np.where(s2 > 0, t + hy, t - hy)
    d = t - h3
    sS = K_REL_S * (((h0 + hx) + hy) + h3)
    return d, sS


def draw(rng, n):
    """Candidates at the window edge: frequencies up to 150 rad/ps, velocities up to 50 A/ps (some legs nearly
    equal, so that sigma crosses sigma_min), and w''' placed so that |dw| is window * sigma times 1 +- a relative
    offset between 1e-12 and 1e-2."""
    pattern = rng.integers(0, 3, n)
    s1 = np.where(pattern < 2, 1, -1)
    s2 = np.where(pattern == 0, 1, -1)
    w0, wx, wy = (np.exp(rng.uniform(np.log(0.05), np.log(150.0), n)) for _ in range(3))
    v_leg = rng.uniform(-50.0, 50.0, (n, 3))
    v3 = rng.uniform(-50.0, 50.0, (n, 3))
    near = rng.random(n) < 0.2                       # velocity differences down to 1e-13 A/ps
    v3[near] = v_leg[near] * np.where(rng.random(n) < 0.5, 1.0, -1.0)[near, None] + \
        rng.normal(size=(near.sum(), 3)) * np.exp(rng.uniform(np.log(1e-13), np.log(1e-6), near.sum()))[:, None]
    sign = np.where(rng.random(n) < 0.5, 1.0, -1.0)
    sb = rng.choice([1.0, 0.1, 0.01], n)
    dq = rng.uniform(0.05, 0.5, n)
    return s1, s2, w0, wx, wy, v_leg, v3, sign, sb, dq


def test_prefilter_decisions_agree_with_fp64():
    rng = np.random.Generator(np.random.PCG64(2104))
    window, sigma_min = 2.0, 1e-10
    n = 400_000
    s1, s2, w0, wx, wy, v_leg, v3, sign, sb, dq = draw(rng, n)
    # sigma entries, vectorised over the candidates (each with its own scalebroad, |dq| and leg sign)
    P = np.empty(n, F32)
    M = np.empty(n, F32)
    P64 = np.empty(n)
    settled = np.empty(n, bool)
    for val in np.unique(sb):
        for sgn in (1.0, -1.0):
            k = (sb == val) & (sign == sgn)
            Pk, Mk, P64k, sig, E, sig64, ok = sigma_prefilter(v_leg[k], v3[k], sgn, val, dq[k], window, sigma_min)
            assert np.all(np.abs(sig.astype(np.float64) - sig64) <= E.astype(np.float64))
            # entries the FP32 form does not settle take the exact FP64 entry: P~ = fl32(P64), margin 2^-22 P~
            Pe = f32(P64k)
            P[k] = np.where(ok, Pk, Pe)
            M[k] = np.where(ok, Mk, K_REL_P * Pe)
            P64[k] = P64k
            settled[k] = ok
    offset = np.exp(rng.uniform(np.log(1e-12), np.log(1e-2), n)) * np.where(rng.random(n) < 0.5, 1.0, -1.0)
    target = P64 * (1.0 + offset) * np.where(rng.random(n) < 0.5, 1.0, -1.0)
    w3 = ((w0 + s1 * wx) + s2 * wy) - target
    keep = w3 > 0.05
    s1, s2, w0, wx, wy, w3, P, M, P64 = (x[keep] for x in (s1, s2, w0, wx, wy, w3, P, M, P64))
    d, sS = dw_prefilter(w0, wx, wy, w3, s1, s2)
    d64 = ((w0 + s1 * wx) + s2 * wy) - w3
    S = w0 + wx + wy + w3
    assert np.all(np.abs(d.astype(np.float64) - d64) <= 4.1 * U * S)
    margin = sS + M
    accept = np.abs(d) < P - margin
    reject = np.abs(d) > P + margin
    exact = np.abs(d64) <= P64
    assert not np.any(accept & ~exact)
    assert not np.any(reject & exact)
    band = ~accept & ~reject
    # drawn at the edge, the candidates exercise all three outcomes and both kinds of sigma entry
    assert band.any() and accept.any() and reject.any()
    assert settled.any() and not settled.all()
