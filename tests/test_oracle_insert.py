"""Pins of the oracle's dynamic insertion (the block rule for a new point and
the index after inserting): the block rule reproduces the attribute-frequency
tree's own assignment for every built point (dense and label-set
attributes); an index grown by insertion keeps Alg. 2's covering property,
so probing every partition returns the exact filtered kNN of all points."""
import numpy as np

import oracle as O
from workloads import make_dense_workload


def _w(seed, N=4000, nq=80):
    return make_dense_workload(name="ins", N=N, d=16, ncomp=10, center=("normal", 2.0),
                               sigma=1.0, vocab=[4, 7, 12], zipf_s=1.0, nq=nq, cmin=1, cmax=3,
                               B=10, h=6, iters=4, m=3, k=10, seed=seed)


def test_block_rule_reproduces_the_tree_dense():
    w = _w(61)
    at = O.Attrs.of(w)
    oi = O.build(w.X, at, w.B, w.h, w.iters, w.init_idx)
    np.testing.assert_array_equal(O.block_of(oi.tags, w.h, at, oi.bin), oi.key)


def test_block_rule_reproduces_the_tree_label_sets():
    rng = np.random.default_rng(62)
    N, V = 2500, 40
    X = rng.standard_normal((N, 8)).astype(np.float32)
    n = rng.integers(1, 6, N)
    off = np.zeros(N + 1, np.int64)
    off[1:] = np.cumsum(n)
    lab = np.concatenate([np.sort(rng.choice(V, k, replace=False)) for k in n]).astype(np.int32)
    at = O.Attrs(sp_off=off, sp_lab=lab, sp_vocab=V)
    oi = O.build(X, at, 7, 9, 3, np.arange(7) * 300)
    np.testing.assert_array_equal(O.block_of(oi.tags, 9, at, oi.bin), oi.key)


def test_inserting_nothing_changes_nothing():
    w = _w(63)
    at = O.Attrs.of(w)
    oi = O.build(w.X, at, w.B, w.h, w.iters, w.init_idx)
    o2 = O.insert(oi, w.X, at, 0)
    for f in ("bin", "key", "perm", "offsets", "tags"):
        np.testing.assert_array_equal(getattr(o2, f), getattr(oi, f))


def test_grown_index_probing_everything_is_exact_filtered_knn():
    w = _w(64, N=5000)
    n0 = 3000
    at0 = O.Attrs(A=w.A[:n0], vocab=w.vocab)
    at = O.Attrs.of(w)
    oi = O.build(w.X[:n0], at0, w.B, w.h, w.iters, w.init_idx)
    for n1 in (4000, 5000):  # two insertion batches
        oi = O.insert(oi, w.X[:n1], O.Attrs(A=w.A[:n1], vocab=w.vocab), n1 - (len(oi.bin)))
    assert len(oi.perm) == w.N and oi.offsets[-1] == w.N
    ids, dist, _, _ = O.search(w.X, at, oi, w.Q, O.Cons(Qb=w.Qb), w.k, w.B)
    gids, g32, _, _ = O.bruteforce(w.X, at, w.Q, O.Cons(Qb=w.Qb), w.k, order64=False)
    np.testing.assert_array_equal(ids, gids)
    np.testing.assert_array_equal(dist, g32)
    # the new points sit where the block rule puts them
    new = np.arange(n0, w.N)
    np.testing.assert_array_equal(oi.key[new], O.block_of(oi.tags, w.h, O.Attrs(A=w.A[new], vocab=w.vocab), oi.bin[new]))


def test_block_rule_hand_worked_tree_that_ends_early():
    """Two fields, vocab 3 and 4 (codes 0-2 and 3-6); h = 3.  Partition 0's
    peel used codes 1 and 5 and ran out of points (third tag -1); partition
    1's used 6, 0, 2.  Block = first tag the point carries, else h + 1 = 4,
    never the block of a -1 tag."""
    tags = np.array([[1, 5, -1], [6, 0, 2]], np.int32)
    A = np.array([[1, 3],   # codes 1, 3: carries t1 = 1 -> block 1
                  [0, 2],   # codes 0, 5: carries t2 = 5 -> block 2
                  [1, 2],   # codes 1, 5: carries both -> the first, block 1
                  [0, 0],   # codes 0, 3: neither tag -> remainder 4
                  [2, 1],   # partition 1, codes 2, 4: carries t3 = 2 -> block 3
                  [0, 1],   # partition 1, codes 0, 4: carries t2 = 0 -> block 2
                  [1, 1]],  # partition 1, codes 1, 4: none -> remainder 4
                 np.int32)
    bins = np.array([0, 0, 0, 0, 1, 1, 1], np.int32)
    at = O.Attrs(A=A, vocab=np.array([3, 4], np.int32))
    np.testing.assert_array_equal(O.block_of(tags, 3, at, bins), [1, 2, 1, 4, 3, 2, 4])
