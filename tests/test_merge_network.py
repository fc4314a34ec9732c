"""The merge of two sorted candidate lists used by the tensor-core scan when a
probe's quarter lists are combined, against brute force.

For ascending lists A and B of KP keys (empty slots all ones), the pairwise
minima min(A[i], B[KP-1-i]) are the KP smallest keys of A and B as a
bitonic sequence (rising, then falling); zero keys in front pad it to a
power of two P, and the half-cleaner stages of a bitonic merger (strides
P/2, P/4, ..., 1) sort it ascending; its last KP entries are the result.
"""
import random

EMPTY = (1 << 64) - 1


def merge(A, B, KP):
    P = 16 if KP <= 16 else 32
    c = [0] * (P - KP) + [min(A[i], B[KP - 1 - i]) for i in range(KP)]
    st = P // 2
    while st > 0:
        for i in range(P):
            if i & st == 0:
                x, y = c[i], c[i + st]
                c[i], c[i + st] = min(x, y), max(x, y)
        st //= 2
    return c[P - KP:]


def random_list(rng, KP, used):
    n = rng.randint(0, KP)
    keys = []
    while len(keys) < n:
        k = (rng.randint(0, 50) << 32) | rng.randint(0, 1 << 20)  # tied scores, distinct ids
        if k not in used:
            used.add(k)
            keys.append(k)
    return sorted(keys) + [EMPTY] * (KP - n)


def test_merge_equals_the_kp_smallest_of_the_union():
    rng = random.Random(9)
    for KP in (10, 16, 32):
        for _ in range(5000):
            used = set()
            A, B = random_list(rng, KP, used), random_list(rng, KP, used)
            want = sorted(A + B)[:KP]
            assert merge(A, B, KP) == want
