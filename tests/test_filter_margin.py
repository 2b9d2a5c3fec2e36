"""The many-frame selection filters pairs with FP16 tensor-core scores and
keeps every pair whose score e lies within a margin of its exact weighted
distance. This checks that error bound, independently of the GPU. The filter's
arithmetic is emulated in numpy:
* power-of-two scales (database 2^(15 - e_x), frame 2^(15 - e_f));
* FP16 rounding of both operands;
* exact products;
* FP32 accumulation in an arbitrary order;
* one fma into the FP32 row norm, then the FP32 frame norm.
On a range of inputs, |e - sum w (q - x)^2| must stay below
  (2 * 2(gamma_{D+4} + 3u) + 1.01 * 2^-11) rad^2 + D max|w q| 2^-21 / s_x,
rad = max ||x||_w + ||q||_w: the margin that the library's bound kernel
applies. Inputs stay in FP32's normal range: below it the FP32 norms and
distances themselves underflow, whatever the filter does."""
import math

import numpy as np
import pytest

U = 2.0 ** -24


def pow2_scale(amax):
    e = math.frexp(float(amax))[1]  # amax = f 2^e, f in [0.5, 1)
    return 2.0 ** (15 - e)


def f32_sum(terms, rng):
    """FP32 sum of float64-exact terms in a random order (each addition rounded)."""
    acc = np.float32(0.0)
    for t in rng.permutation(terms):
        acc = np.float32(acc + np.float32(t)) if abs(t) < 3e38 else acc
    return float(acc)


def f32_dot_sequential(a, b):
    acc = np.float32(0.0)
    for x, y in zip(a.astype(np.float32), b.astype(np.float32)):
        acc = np.float32(np.float64(x) * np.float64(y) + np.float64(acc))  # fma: one rounding
    return float(acc)


def emulate(X, Q, w, rng):
    """Filter scores e[f][r] as the tensor-core path forms them, and the margins."""
    n, D = X.shape
    sx = pow2_scale(np.max(np.abs(X)))
    Xh = (X.astype(np.float64) * sx).astype(np.float16).astype(np.float64)
    xn = np.array([f32_dot_sequential(w * x, x) for x in X])  # FP32 weighted norms
    xmax = math.sqrt(float(np.max(xn))) * 1.0001
    gam = (D + 4) * U / (1 - (D + 4) * U)
    scale = 2 * (2 * (gam + 3 * U)) + 1.01 * 2.0 ** -11
    E, M = np.zeros((len(Q), n)), np.zeros(len(Q))
    for fi, q in enumerate(Q):
        wq = (w * q).astype(np.float32).astype(np.float64)
        sf = pow2_scale(np.max(np.abs(wq)))
        qh = (wq * sf).astype(np.float16).astype(np.float64)
        qn = f32_dot_sequential(w * q, q)
        c = -2.0 / sx / sf
        for r in range(n):
            v = f32_sum(Xh[r] * qh, rng)  # exact FP16 products, FP32 accumulation
            u = float(np.float32(xn[r] + c * v))  # fma into the row norm
            E[fi, r] = float(np.float32(u + qn))
        rad = xmax + math.sqrt(qn)
        M[fi] = scale * rad * rad + D * float(np.max(np.abs(wq))) * 2.0 ** -21 / sx
    return E, M


@pytest.mark.parametrize("case", ["normal", "dynamic_range", "tiny_values", "integers"])
def test_fp16_filter_error_within_margin(case):
    rng = np.random.default_rng({"normal": 1, "dynamic_range": 2, "tiny_values": 3, "integers": 4}[case])
    n, D, nq = 40, 64, 6
    if case == "normal":
        X = rng.standard_normal((n, D))
        w = rng.uniform(0.5, 1.5, D)
    elif case == "dynamic_range":
        # per-dimension magnitudes 1e-8 .. 1e3: most values fall deep into FP16's subnormal range
        X = rng.standard_normal((n, D)) * 10.0 ** rng.uniform(-8, 3, D)
        w = 10.0 ** rng.uniform(-2, 2, D)
    elif case == "tiny_values":
        # one small magnitude throughout (squares stay in FP32's normal range): the power-of-two
        # scales bring it to FP16's normal range
        X = rng.standard_normal((n, D)) * 1e-12
        w = np.ones(D)
    else:
        X = rng.integers(-3, 4, (n, D)).astype(np.float64)
        w = np.ones(D)
    X = X.astype(np.float32)
    w = w.astype(np.float32)
    if case == "integers":
        Q = (X[rng.integers(0, n, nq)] + rng.integers(-1, 2, (nq, D))).astype(np.float32)
    else:
        Q = (X[rng.integers(0, n, nq)] + 0.1 * np.abs(X).mean() * rng.standard_normal((nq, D))).astype(np.float32)
    E, M = emulate(X, Q, w, rng)
    X64, Q64, w64 = X.astype(np.float64), Q.astype(np.float64), w.astype(np.float64)
    exact = np.array([[np.sum(w64 * (q - x) ** 2) for x in X64] for q in Q64])
    ratio = np.abs(E - exact) / M[:, None]
    assert np.all(ratio <= 1.0), f"{case}: error {ratio.max():.3f} x the margin"
    if case == "integers":
        assert np.all(E == exact)  # small integers: every step is exact
