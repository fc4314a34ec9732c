"""Pins of the oracle's disjunctive (OR) constraints (Sec. 5.3: several
constraints map to several sub-partitions): a field may allow a list of
values.  Checked against (1) the conjunctive oracle when every list holds one
value, (2) exact OR-filtered kNN computed with numpy when every partition is
probed, (3) the covering property of the block selection (no OR-valid point
of a probed partition lies outside the selected blocks), and (4) the top-k
of the union of the single-valued sub-queries' results."""
import itertools

import numpy as np

import oracle as O
from workloads import make_dense_workload


def _w(seed=41, N=3000, vocab=(4, 6, 9), nq=60, B=12, h=6):
    return make_dense_workload(name="or", N=N, d=16, ncomp=8, center=("normal", 2.0), sigma=1.0,
                               vocab=list(vocab), zipf_s=1.0, nq=nq, cmin=1, cmax=len(vocab),
                               B=B, h=h, iters=4, m=4, k=10, seed=seed)


def _or_lists(w, rng, max_vals=3):
    """Per query: the fields its conjunctive constraint fixes get that value
    plus up to max_vals - 1 others; free fields stay free (some get a list)."""
    lists = []
    for q in range(w.nq):
        row = []
        for f, V in enumerate(w.vocab):
            b = int(w.Qb[q, f])
            if b >= 0:
                extra = rng.choice(V, size=rng.integers(0, max_vals), replace=False).tolist()
                row.append(sorted(set([b] + extra)))
            elif rng.random() < 0.2:
                row.append(sorted(rng.choice(V, size=2, replace=False).tolist()))
            else:
                row.append([])
        lists.append(row)
    return lists


def _or_mask(A, row):
    ok = np.ones(A.shape[0], bool)
    for f, vals in enumerate(row):
        if vals:
            ok &= np.isin(A[:, f], vals)
    return ok


def test_single_values_equal_the_conjunctive_search():
    w = _w()
    at = O.Attrs.of(w)
    oi = O.build(w.X, at, w.B, w.h, w.iters, w.init_idx)
    lists = [[[int(b)] if b >= 0 else [] for b in w.Qb[q]] for q in range(w.nq)]
    ids, dist = O.search_or(w.X, at, oi, w.Q, O.OrCons.of_lists(lists), w.k, w.m)
    cids, cdist, _, _ = O.search(w.X, at, oi, w.Q, O.Cons(Qb=w.Qb), w.k, w.m)
    np.testing.assert_array_equal(ids, cids)
    np.testing.assert_array_equal(dist, cdist)


def test_all_partitions_probed_is_exact_or_filtered_knn():
    w = _w(seed=42)
    at = O.Attrs.of(w)
    oi = O.build(w.X, at, w.B, w.h, w.iters, w.init_idx)
    lists = _or_lists(w, np.random.default_rng(1))
    ids, dist = O.search_or(w.X, at, oi, w.Q, O.OrCons.of_lists(lists), w.k, w.B)
    for q in range(w.nq):
        cand = np.nonzero(_or_mask(w.A, lists[q]))[0]
        d32 = np.array([O.dist32(w.X[i], w.Q[q]) for i in cand], np.float32)
        order = np.lexsort((cand, d32))[:w.k]
        want = np.full(w.k, -1, np.int64)
        want[:len(order)] = cand[order]
        np.testing.assert_array_equal(ids[q], want)
        np.testing.assert_array_equal(dist[q, :len(order)], d32[order])


def test_selection_covers_every_or_valid_point_tiny_vocab():
    w = _w(seed=43, N=1500, vocab=(3, 3, 4), nq=1, B=6, h=5)
    at = O.Attrs.of(w)
    oi = O.build(w.X, at, w.B, w.h, w.iters, w.init_idx)
    nb = w.h + 1
    block_of = np.empty(w.N, np.int64)
    for s in range(w.B * nb):
        block_of[oi.perm[oi.offsets[s]:oi.offsets[s + 1]]] = s % nb
    probe = np.arange(w.B, dtype=np.int32)[None, :]
    subsets = [[list(c) for r in range(0, V + 1) for c in itertools.combinations(range(V), r)]
               for V in w.vocab]
    n = 0
    for row in itertools.product(*subsets):
        row = [list(v) for v in row]
        sel = O.select_or(oi.tags, w.h, at, probe, O.OrCons.of_lists([row]))[0]
        ok = _or_mask(w.A, row)
        for i in np.nonzero(ok)[0]:
            assert (int(sel[oi.bin[i]]) >> int(block_of[i])) & 1, (row, i)
        n += 1
    assert n == 8 * 8 * 16


def test_or_result_is_the_best_of_its_single_valued_sub_queries():
    w = _w(seed=44)
    at = O.Attrs.of(w)
    oi = O.build(w.X, at, w.B, w.h, w.iters, w.init_idx)
    lists = _or_lists(w, np.random.default_rng(2))
    ids, dist = O.search_or(w.X, at, oi, w.Q, O.OrCons.of_lists(lists), w.k, w.m)
    for q in range(w.nq):
        combos = list(itertools.product(*[(v if v else [-1]) for v in lists[q]]))
        Qb = np.array(combos, np.int32)
        Qs = np.repeat(w.Q[q:q + 1], len(combos), 0)
        sids, sdist, _, _ = O.search(w.X, at, oi, Qs, O.Cons(Qb=Qb), w.k, w.m)
        ok = sids >= 0
        cand, cd = sids[ok], sdist[ok]
        assert len(np.unique(cand)) == len(cand)  # sub-queries are disjoint
        order = np.lexsort((cand, cd))[:w.k]
        want = np.full(w.k, -1, np.int64)
        want[:len(order)] = cand[order]
        np.testing.assert_array_equal(ids[q], want)
