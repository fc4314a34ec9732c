"""The error bound the screened probe relies on (Alg. 2 "select top m
partitions", exact set from approximate scores), checked on the CPU.

Every fp32 value v is split into hi = bf16(v) and lo = bf16(v - hi); the
tensor cores form hi_a*hi_w + hi_a*lo_w + lo_a*hi_w (each product exact in
fp32) and accumulate in fp32 in an order of their own.  The probe trusts
that the exact fixed-order fp32 score (acc = fma(a_k, w_k, acc), k in order;
L2: t = w_k - a_k, acc = fma(t, t, acc)) lies within eps of that value, with
eps = 2^-11 |a| |w| for dot products and 2^-11 (|a| + |w|)^2 for L2
distances formed as |w|^2 + |a|^2 - 2 a.w.  Here the split and the three
products are formed exactly, the tensor cores' accumulation is charged its
worst case (K * 2^-24 * the sum of the terms' magnitudes), and the result is
compared with the fixed-order chain on inputs chosen to stress the bound:
random, nearly orthogonal (a large |a||w| against a small dot product),
mixed magnitudes, and near neighbours for L2.
"""
import numpy as np

EPS = 2.0 ** -11
U32 = 2.0 ** -24


def bf16(a):
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000  # round to nearest even
    return u.astype(np.uint32).view(np.float32)


def split(v):
    v = np.asarray(v, dtype=np.float32)
    hi = bf16(v)
    lo = bf16((v - hi).astype(np.float32))
    return hi.astype(np.float64), lo.astype(np.float64)


def tensor_core_dot(a, w):
    """The three-term split product, and the worst-case error of summing its
    terms in fp32 in any order."""
    ah, al = split(a)
    wh, wl = split(w)
    terms = np.concatenate([ah * wh, ah * wl, al * wh])  # each exact in fp32
    return terms.sum(), len(a) * U32 * np.abs(terms).sum()


def chain_dot(a, w):
    acc = np.float32(0.0)
    for x, y in zip(a.astype(np.float64), w.astype(np.float64)):
        acc = np.float32(x * y + np.float64(acc))  # one rounding per term (fma)
    return float(acc)


def chain_l2(a, w):
    acc = np.float32(0.0)
    for x, y in zip(a, w):
        t = np.float64(np.float32(y - x))
        acc = np.float32(t * t + np.float64(acc))
    return float(acc)


def cases(rng, K):
    a = rng.standard_normal(K).astype(np.float32)
    yield a, rng.standard_normal(K).astype(np.float32)
    # nearly orthogonal: |a||w| large, a.w small
    w = rng.standard_normal(K).astype(np.float32)
    w = (w - a * (a @ w) / (a @ a)).astype(np.float32)
    yield a, w
    # mixed magnitudes across coordinates
    yield (a * np.exp2(rng.integers(-12, 12, K))).astype(np.float32), \
        (rng.standard_normal(K) * np.exp2(rng.integers(-12, 12, K))).astype(np.float32)
    # byte-valued rows (the sift-like data) and a ReLU-like sparse vector
    yield np.round(rng.uniform(0, 255, K)).astype(np.float32), \
        np.round(rng.uniform(0, 255, K)).astype(np.float32)
    yield np.maximum(rng.standard_normal(K), 0).astype(np.float32), \
        (0.05 * rng.standard_normal(K)).astype(np.float32)


def test_dot_product_interval_holds_the_fixed_order_score():
    rng = np.random.default_rng(17)
    worst = 0.0
    for K in (13, 64, 128, 512):
        for _ in range(40):
            for a, w in cases(rng, K):
                approx, acc_err = tensor_core_dot(a, w)
                exact = chain_dot(a, w)
                eps = EPS * float(np.linalg.norm(a.astype(np.float64))) * \
                    float(np.linalg.norm(w.astype(np.float64)))
                err = abs(approx - exact) + acc_err
                assert err <= eps, (K, err, eps)
                worst = max(worst, err / eps)
    assert worst < 0.5  # the bound keeps a margin of at least two


def test_l2_interval_holds_the_fixed_order_distance():
    rng = np.random.default_rng(18)
    for K in (16, 128):
        for _ in range(40):
            for a, w in cases(rng, K):
                # near neighbours too: the distance is small against the norms
                for w2 in (w, (a + 1e-3 * w).astype(np.float32)):
                    dt, acc_err = tensor_core_dot(a, w2)
                    an2 = float((a.astype(np.float64) ** 2).sum())
                    wn2 = float((w2.astype(np.float64) ** 2).sum())
                    approx = wn2 + an2 - 2.0 * dt
                    exact = chain_l2(a, w2)
                    eps = EPS * (np.sqrt(an2) + np.sqrt(wn2)) ** 2
                    # the norms are fp32 sums: their rounding (K * 2^-24
                    # relative each) is charged as well
                    err = abs(approx - exact) + 2.0 * acc_err + K * U32 * (an2 + wn2)
                    assert err <= eps, (K, err, eps)
