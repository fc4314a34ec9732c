"""The shared per-probe bounds of the tensor-core scan, against brute force.

Four threads keep quarter lists of a probe's candidate keys (key = score
bits << 32 | row id; distinct rows, so distinct keys), each sorted
ascending with at most KP entries.  The scan drops a key above either bound:

* the smallest of the four lists' KP-th keys (a full list alone already
  holds KP better keys);
* with QB = ceil(KP/4) and NHI = KP - 4 (QB - 1): order the lists by the
  score of their QB-th key; the NHI first count QB keys, the others QB - 1;
  the bound is (the largest of those keys' scores) << 32 | all ones.

Either bound must be at or above the KP-th smallest key of the union (so no
key of the probe's top KP is ever dropped).  The split bound must also be no
looser than the largest of the four QB-th keys' scores.
"""
import random

EMPTY = (1 << 64) - 1


def kth_key_bound(lists, KP):
    full = [l[KP - 1] for l in lists if len(l) >= KP]
    return min(full) if full else EMPTY


def split_bound(lists, KP):
    QB = -(-KP // 4)
    NHI = KP - 4 * (QB - 1)
    qa = [(l[QB - 1] >> 32) if len(l) >= QB else 0xFFFFFFFF for l in lists]
    qb = [(l[QB - 2] >> 32) if len(l) >= QB - 1 else 0xFFFFFFFF for l in lists]
    order = sorted(range(4), key=lambda i: qa[i])
    bs = qa[order[NHI - 1]]
    for i in order[NHI:]:
        bs = max(bs, qb[i])
    return (bs << 32) | 0xFFFFFFFF, max(qa)


def trial(rng, KP):
    n_rows = rng.randint(1, 4 * KP + 8)
    scores = [rng.randint(0, 40) for _ in range(n_rows)]  # many ties in score
    keys = [(s << 32) | i for i, s in enumerate(scores)]
    quarter = [rng.randrange(4) for _ in range(n_rows)]
    lists = [sorted(k for k, q in zip(keys, quarter) if q == j)[:KP] for j in range(4)]
    union = sorted(k for l in lists for k in l)
    true_kp = union[KP - 1] if len(union) >= KP else EMPTY
    return lists, true_kp


def test_bounds_never_drop_a_top_kp_key():
    rng = random.Random(5)
    for KP in (10, 16):
        tightened = 0
        for _ in range(20000):
            lists, true_kp = trial(rng, KP)
            b1 = kth_key_bound(lists, KP)
            b2, max_qa = split_bound(lists, KP)
            assert b1 == EMPTY or true_kp <= b1
            assert b2 == EMPTY or true_kp <= b2
            # never looser than the largest of the QB-th keys' scores
            assert (b2 >> 32) <= max_qa
            tightened += (b2 >> 32) < max_qa
        if KP == 10:
            assert tightened > 0  # the (3, 3, 2, 2) split does tighten
