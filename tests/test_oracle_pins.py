"""Pins for the CPU oracle: hand-worked examples, closed forms, invariants
and brute force on tiny inputs.  Each test names the passage it pins; none
of them re-runs the oracle's own formula."""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from workloads import make_dense_workload, make_sparse_workload

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _f(v):
    return math.inf if v == "inf" else float(v)


# ---------------------------------------------------------------- Def. 1 --

def test_filter_def1_hand_cases():
    # Def. 1: C(a,b) holds iff a[i] = b[i] on every field; -1 frees a field.
    assert O.filter_dense([1, 2, 3], [1, 2, 3])
    assert not O.filter_dense([1, 2, 3], [1, 2, 4])
    assert O.filter_dense([1, 2, 3], [-1, -1, -1])
    assert O.filter_dense([1, 2, 3], [-1, 2, -1])
    assert not O.filter_dense([1, 2, 3], [2, -1, -1])
    assert not O.filter_dense([0, 0, 0], [0, 0, 1])
    # sparse labels: every required label present
    assert O.filter_sparse([1, 5, 9], [5])
    assert O.filter_sparse([1, 5, 9], [1, 9])
    assert not O.filter_sparse([1, 5, 9], [1, 2])
    assert O.filter_sparse([1, 5, 9], [])
    assert not O.filter_sparse([], [3])


def test_filter_exhaustive_tiny_vocab():
    # every (a, b) over vocab 2x3 with wildcards: C holds iff no constrained
    # field differs -- counted independently as a product over fields.
    for a in itertools.product(range(2), range(3)):
        for b in itertools.product(range(-1, 2), range(-1, 3)):
            expect = all(bv == -1 or bv == av for av, bv in zip(a, b))
            assert O.filter_dense(a, b) == expect


# ------------------------------------------------------------ distances --

def test_dist32_closed_forms():
    x = np.array([1.5, -2.0, 3.25, 0.0], np.float32)
    assert O.dist32(x, x) == 0.0
    e = np.zeros(4, np.float32)
    e[2] = 3.0
    assert O.dist32(e, np.zeros(4, np.float32)) == 9.0
    assert O.dist32(e, e, metric=O.IP) == 9.0
    assert O.dist32([1, 0], [0, 1], metric=O.IP) == 0.0


def test_dist32_integer_vectors_exact():
    # byte-valued vectors: every partial sum is an integer below 2^24, so the
    # fp32 result equals the exact integer distance.
    rng = np.random.default_rng(7)
    for _ in range(50):
        x = rng.integers(0, 256, 128)
        q = rng.integers(0, 256, 128)
        exact = int(((x - q) ** 2).sum())
        assert O.dist32(x.astype(np.float32), q.astype(np.float32)) == float(exact)
        assert O.dist64(x, q) == float(exact)
        ip = int((x * q).sum())
        assert O.dist32(x, q, O.IP) == float(ip)


def test_dist32_within_sequential_error_bound():
    # recursive summation of d non-negative terms with one rounding per
    # step: |err| <= gamma_{d+1} * exact (Higham, Thm 4.4 form).
    rng = np.random.default_rng(8)
    u = 2.0 ** -24
    for d in (1, 7, 32, 128, 960):
        for _ in range(20):
            x = rng.standard_normal(d).astype(np.float32)
            q = rng.standard_normal(d).astype(np.float32)
            t = x.astype(np.float64) - q.astype(np.float64)
            exact = float(np.sum(t * t))
            g = (d + 1) * u / (1 - (d + 1) * u)
            assert abs(O.dist32(x, q) - exact) <= g * exact + 1e-30


def test_dist32_fused_and_ordered():
    # t = 1 + 2^-12: t*t = 1 + 2^-11 + 2^-24 rounds (tie to even) to
    # 1 + 2^-11.  IP of (t, t) and (t, -t) in the order j = 0, 1 with a fused
    # multiply-add leaves exactly the rounding error -2^-24; an unfused sum
    # gives 0 and the reversed order gives +2^-24.
    t = np.float32(1 + 2.0 ** -12)
    assert O.dist32([t, t], [t, -t], metric=O.IP) == -(2.0 ** -24)
    assert O.dist64([t, t], [t, -t], metric=O.IP) == 0.0


# ------------------------------------------------------------- k-means --

def test_kmeans_hand_cases():
    g = _load("kmeans_hand.json")
    for case in g["cases"]:
        C, bin = O.kmeans(np.array(case["X"], np.float32), case["B"], case["iters"],
                          np.array(case["init"]))
        np.testing.assert_array_equal(C, np.array(case["C"], np.float32))
        np.testing.assert_array_equal(bin, case["bin"])


def test_kmeans_single_partition_is_global_mean():
    rng = np.random.default_rng(3)
    X = rng.integers(0, 256, (1000, 16)).astype(np.float32)
    C, bin = O.kmeans(X, 1, 3, np.array([17]))
    # integer data: the fp64 sum is exact, the mean is one rounding away
    mean = X.astype(np.int64).sum(0) / 1000.0
    np.testing.assert_array_equal(C[0], mean.astype(np.float32))
    assert (bin == 0).all()


def test_kmeans_fixed_point_invariants():
    # After convergence: assignment = argmin over exact distances (integer
    # data, so fp32 is exact) and each centroid = fp32(mean of members).
    rng = np.random.default_rng(4)
    centers = rng.uniform(0, 200, (6, 8))
    X = np.rint(centers[rng.integers(0, 6, 600)] + 3 * rng.standard_normal((600, 8)))
    X = np.clip(X, 0, 255).astype(np.float32)
    C, bin = O.kmeans(X, 6, 60, rng.permutation(600)[:6])
    Xi = X.astype(np.float64)
    D = ((Xi[:, None, :] - C[None, :, :].astype(np.float64)) ** 2).sum(-1)
    # argmin with ties to the lower centroid == first index of the minimum
    np.testing.assert_array_equal(bin, D.argmin(1))
    for c in range(6):
        mem = X[bin == c].astype(np.float64)
        if len(mem):
            np.testing.assert_array_equal(C[c], (mem.sum(0) / len(mem)).astype(np.float32))


def test_assign_ip_argmax():
    C = np.array([[1, 0], [0, 1], [0.6, 0.8]], np.float32)
    X = np.array([[1, 0.1], [0.1, 1], [0.7, 0.7], [0, 0]], np.float32)
    # IP: the largest dot product wins; (0,0) ties everywhere -> centroid 0
    np.testing.assert_array_equal(O.assign(X, C, O.IP), [0, 1, 2, 0])


# ----------------------------------------------------------------- AFT --

def test_aft_hand_example():
    g = _load("aft_hand_8pt.json")
    at = O.Attrs(A=g["A"], vocab=g["vocab"])
    bin = np.zeros(len(g["A"]), np.int32)
    tags, key = O.aft(bin, g["B"], g["h"], at)
    np.testing.assert_array_equal(tags, g["tags"])
    np.testing.assert_array_equal(key, g["key"])
    perm, off = O.layout(bin, key, g["B"], g["h"])
    np.testing.assert_array_equal(perm, g["perm"])
    np.testing.assert_array_equal(off, g["offsets"])


def _codes_dense(A, vocab):
    off = np.concatenate([[0], np.cumsum(vocab)[:-1]])
    return A + off[None, :]


def _check_aft_invariants(bin, tags, key, B, h, codes_of):
    """Alg. 1 invariants: the h+1 blocks of a bin are disjoint and cover it;
    block j holds exactly the not-yet-peeled points carrying t_j; |p_j| is the
    largest code count among those points (ties -> lowest code)."""
    for b in range(B):
        mem = np.nonzero(bin == b)[0]
        remaining = list(mem)
        for j in range(1, h + 1):
            t = tags[b, j - 1]
            if not remaining:
                assert t == -1
                continue
            cnt = {}
            for i in remaining:
                for c in codes_of(i):
                    cnt[c] = cnt.get(c, 0) + 1
            best = min(cnt, key=lambda c: (-cnt[c], c))
            assert t == best
            peel = [i for i in remaining if t in codes_of(i)]
            assert sorted(np.nonzero((bin == b) & (key == j))[0].tolist()) == sorted(peel)
            assert len(peel) == cnt[best]
            remaining = [i for i in remaining if t not in codes_of(i)]
        rest = np.nonzero((bin == b) & (key == h + 1))[0]
        assert sorted(rest.tolist()) == sorted(remaining)
        valid = tags[b][tags[b] >= 0]
        assert len(set(valid.tolist())) == len(valid)
    assert ((key >= 1) & (key <= h + 1)).all()


@pytest.mark.parametrize("h", [0, 1, 3, 7])
def test_aft_invariants_dense(h):
    rng = np.random.default_rng(10 + h)
    N, B = 400, 5
    vocab = np.array([4, 6, 9])
    A = np.stack([rng.choice(V, N, p=(np.arange(V) + 1.0) ** -1 / ((np.arange(V) + 1.0) ** -1).sum())
                  for V in vocab], 1).astype(np.int32)
    bin = rng.integers(0, B, N).astype(np.int32)
    bin[bin == 4] = 3  # one empty partition
    tags, key = O.aft(bin, B, h, O.Attrs(A=A, vocab=vocab))
    codes = _codes_dense(A, vocab)
    _check_aft_invariants(bin, tags, key, B, h, lambda i: set(codes[i].tolist()))
    if h == 0:
        assert (key == 1).all() and tags.shape == (B, 0)


def test_aft_invariants_sparse():
    rng = np.random.default_rng(21)
    N, B, h, V = 300, 4, 5, 12
    cnt = rng.integers(0, 4, N)  # includes points with no label
    rows = [np.sort(rng.choice(V, c, replace=False)) for c in cnt]
    off = np.concatenate([[0], np.cumsum(cnt)])
    lab = np.concatenate(rows).astype(np.int32)
    bin = rng.integers(0, B, N).astype(np.int32)
    tags, key = O.aft(bin, B, h, O.Attrs(sp_off=off, sp_lab=lab, sp_vocab=V))

    def codes_of(i):
        return set(rows[i].tolist())

    # points with no labels can never be peeled: the invariant check's
    # "remaining" keeps them, and a round whose remaining points carry no
    # label at all must produce -1
    for b in range(B):
        mem = np.nonzero(bin == b)[0]
        remaining = list(mem)
        for j in range(1, h + 1):
            t = tags[b, j - 1]
            cntd = {}
            for i in remaining:
                for c in codes_of(i):
                    cntd[c] = cntd.get(c, 0) + 1
            if not cntd:
                assert t == -1
                continue
            best = min(cntd, key=lambda c: (-cntd[c], c))
            assert t == best
            remaining = [i for i in remaining if t not in codes_of(i)]
        assert sorted(np.nonzero((bin == b) & (key == h + 1))[0].tolist()) == sorted(remaining)


def test_layout_is_stable_sort_by_bin_block_id():
    rng = np.random.default_rng(5)
    N, B, h = 1000, 7, 3
    bin = rng.integers(0, B, N).astype(np.int32)
    key = rng.integers(1, h + 2, N).astype(np.uint8)
    perm, off = O.layout(bin, key, B, h)
    np.testing.assert_array_equal(perm, np.lexsort((np.arange(N), key, bin)))
    seg = bin.astype(np.int64) * (h + 1) + key - 1
    np.testing.assert_array_equal(off, np.concatenate([[0], np.cumsum(np.bincount(seg, minlength=B * (h + 1)))]))


# ----------------------------------------------------------- Alg. 2 -----

def test_probe_matches_exact_ranking_integer_data():
    rng = np.random.default_rng(6)
    C = rng.integers(0, 8, (50, 4)).astype(np.float32)  # many exact ties
    Q = rng.integers(0, 8, (30, 4)).astype(np.float32)
    P = O.probe(Q, C, 7)
    D = ((Q[:, None, :].astype(np.int64) - C[None].astype(np.int64)) ** 2).sum(-1)
    for q in range(30):
        order = np.lexsort((np.arange(50), D[q]))
        np.testing.assert_array_equal(P[q], order[:7])
    Pip = O.probe(Q, C, 5, metric=O.IP)
    Dip = (Q[:, None, :].astype(np.int64) * C[None].astype(np.int64)).sum(-1)
    for q in range(30):
        np.testing.assert_array_equal(Pip[q], np.lexsort((np.arange(50), -Dip[q]))[:5])


def test_select_and_search_hand_example():
    g = _load("aft_hand_8pt.json")
    at = O.Attrs(A=g["A"], vocab=g["vocab"])
    N = len(g["A"])
    X = np.stack([np.arange(N), np.zeros(N)], 1).astype(np.float32)
    idx = O.Index(C=np.zeros((1, 2), np.float32), bin=np.zeros(N, np.int32),
                  tags=np.array(g["tags"], np.int32), key=np.array(g["key"], np.uint8),
                  perm=np.array(g["perm"], np.int32), offsets=np.array(g["offsets"], np.int32),
                  B=1, h=2, metric=O.L2)
    Qb = np.array([qq["b"] for qq in g["queries"]], np.int32)
    sel = O.select(idx.tags, 2, at, np.zeros((len(Qb), 1), np.int32), O.Cons(Qb=Qb))
    Q = np.tile(np.array([[3, 0]], np.float32), (len(Qb), 1))
    ids, dist, _, _ = O.search(X, at, idx, Q, O.Cons(Qb=Qb), 3, 1)
    gt, _, _, cnt = O.bruteforce(X, at, Q, O.Cons(Qb=Qb), 3)
    for r, qq in enumerate(g["queries"]):
        blocks = [j for j in range(1, 4) if (int(sel[r, 0]) >> (j - 1)) & 1]
        assert blocks == qq["selected_blocks"]
        np.testing.assert_array_equal(ids[r], qq["topk3_ids"])
        np.testing.assert_array_equal(dist[r], [_f(v) for v in qq["topk3_dist"]])
        np.testing.assert_array_equal(gt[r], qq["topk3_ids"])
        assert cnt[r] == len(qq["valid"])


def _tiny_dense(seed, N=300, d=4, B=6, h=3, vocab=(3, 4, 2), nq=60, integer=True):
    rng = np.random.default_rng(seed)
    X = rng.integers(0, 16, (N, d)).astype(np.float32) if integer else \
        rng.standard_normal((N, d)).astype(np.float32)
    A = np.stack([rng.integers(0, V, N) for V in vocab], 1).astype(np.int32)
    Q = rng.integers(0, 16, (nq, d)).astype(np.float32) if integer else \
        rng.standard_normal((nq, d)).astype(np.float32)
    Qb = np.full((nq, len(vocab)), -1, np.int32)
    for q in range(nq):
        for f in range(len(vocab)):
            if rng.random() < 0.5:
                Qb[q, f] = rng.integers(0, vocab[f])
    return X, A, np.array(vocab, np.int32), Q, Qb, B, h


def test_select_covers_exactly_the_valid_points_exhaustive():
    # Alg. 2 sub-partition selection: over every constraint vector on a tiny
    # vocabulary, the selected blocks hold every valid point of the bin
    # (nothing valid is skipped), and with every field constrained exactly
    # one block is chosen.
    rng = np.random.default_rng(11)
    vocab = np.array([3, 3, 2])
    N, B, h = 200, 3, 4
    A = np.stack([rng.integers(0, V, N) for V in vocab], 1).astype(np.int32)
    bin = rng.integers(0, B, N).astype(np.int32)
    at = O.Attrs(A=A, vocab=vocab)
    tags, key = O.aft(bin, B, h, at)
    allb = np.array(list(itertools.product(*[range(-1, V) for V in vocab])), np.int32)
    probe_bins = np.tile(np.arange(B, dtype=np.int32), (len(allb), 1))
    sel = O.select(tags, h, at, probe_bins, O.Cons(Qb=allb))
    for qi, b in enumerate(allb):
        valid = np.all((b < 0) | (A == b), axis=1)
        for bn in range(B):
            s = int(sel[qi, bn])
            in_sel = np.array([(s >> (int(key[i]) - 1)) & 1 for i in range(N)], bool)
            assert not np.any(valid & (bin == bn) & ~in_sel)
            if (b >= 0).all():
                assert bin_count_bits(s) == 1


def bin_count_bits(s):
    return bin(s).count("1")


def _np_filtered_knn(X, A, Q, Qb, k, cand_mask=None):
    """Exact filtered kNN by library sort over fp64 distances."""
    ids = np.full((len(Q), k), -1, np.int64)
    for q in range(len(Q)):
        ok = np.all((Qb[q] < 0) | (A == Qb[q]), axis=1)
        if cand_mask is not None:
            ok &= cand_mask[q]
        cand = np.nonzero(ok)[0]
        dd = ((X[cand].astype(np.float64) - Q[q].astype(np.float64)) ** 2).sum(1)
        order = np.lexsort((cand, dd))[:k]
        ids[q, :len(order)] = cand[order]
    return ids


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_bruteforce_matches_library_sort(seed):
    X, A, vocab, Q, Qb, B, h = _tiny_dense(seed)
    ids, d32, d64, cnt = O.bruteforce(X, O.Attrs(A=A, vocab=vocab), Q, O.Cons(Qb=Qb), 5)
    np.testing.assert_array_equal(ids, _np_filtered_knn(X, A, Q, Qb, 5))
    np.testing.assert_array_equal(cnt, [np.all((b < 0) | (A == b), 1).sum() for b in Qb])


@pytest.mark.parametrize("seed", [1, 2])
def test_search_probe_all_equals_exact(seed):
    # m = B: CAPS visits every valid point, so it returns the exact filtered
    # kNN (integer data: fp32 distances are exact, tie rules agree).
    X, A, vocab, Q, Qb, B, h = _tiny_dense(seed)
    at = O.Attrs(A=A, vocab=vocab)
    idx = O.build(X, at, B, h, 5, np.arange(B))
    ids, dist, nscan, nmatch = O.search(X, at, idx, Q, O.Cons(Qb=Qb), 5, B)
    np.testing.assert_array_equal(ids, _np_filtered_knn(X, A, Q, Qb, 5))
    gt, _, _, cnt = O.bruteforce(X, at, Q, O.Cons(Qb=Qb), 5)
    np.testing.assert_array_equal(nmatch, cnt)


def test_search_h0_is_filtered_ivf_and_no_constraint_is_ivf_flat():
    X, A, vocab, Q, Qb, B, h = _tiny_dense(9)
    at = O.Attrs(A=A, vocab=vocab)
    idx = O.build(X, at, B, 0, 4, np.arange(B))
    m = 2
    P = O.probe(Q, idx.C, m)
    in_probe = np.stack([np.isin(idx.bin, P[q]) for q in range(len(Q))])
    # h = 0: search-then-filter inside the probed partitions
    ids, _, nscan, _ = O.search(X, at, idx, Q, O.Cons(Qb=Qb), 5, m)
    np.testing.assert_array_equal(ids, _np_filtered_knn(X, A, Q, Qb, 5, in_probe))
    np.testing.assert_array_equal(nscan, in_probe.sum(1))
    # no constraint at all, any h: plain IVF-Flat over the probed partitions
    free = np.full_like(Qb, -1)
    idx3 = O.build(X, at, B, 3, 4, np.arange(B))
    ids3, _, _, _ = O.search(X, at, idx3, Q, O.Cons(Qb=free), 5, m)
    np.testing.assert_array_equal(ids3, _np_filtered_knn(X, A, Q, free, 5, in_probe))


def test_search_any_h_equals_filtered_ivf():
    # The attribute tree only skips blocks with no valid point, so for any h
    # the result equals search-then-filter over the same probed partitions.
    X, A, vocab, Q, Qb, B, _ = _tiny_dense(12)
    at = O.Attrs(A=A, vocab=vocab)
    for h in (1, 2, 5):
        idx = O.build(X, at, B, h, 4, np.arange(B))
        P = O.probe(Q, idx.C, 3)
        in_probe = np.stack([np.isin(idx.bin, P[q]) for q in range(len(Q))])
        ids, _, nscan, _ = O.search(X, at, idx, Q, O.Cons(Qb=Qb), 5, 3)
        np.testing.assert_array_equal(ids, _np_filtered_knn(X, A, Q, Qb, 5, in_probe))
        assert (nscan <= in_probe.sum(1)).all()


def test_search_sparse_labels_against_library_sort():
    w = make_sparse_workload(name="tiny_sparse", N=500, d=6, ncomp=4, center=("normal", 3.0),
                             sigma=1.0, V=15, zipf_s=1.0, nmax=5, exponent=1.5, nq=40,
                             cmin=1, cmax=3, B=4, h=4, iters=5, m=4, k=5, seed=77)
    at, cons = O.Attrs.of(w), O.Cons.of(w)
    idx = O.build(w.X, at, w.B, w.h, w.iters, w.init_idx)
    ids, dist, _, _ = O.search(w.X, at, idx, w.Q, cons, w.k, w.B)
    for q in range(w.nq):
        req = set(w.q_lab[w.q_off[q]:w.q_off[q + 1]].tolist())
        ok = np.array([req <= set(w.sp_lab[w.sp_off[i]:w.sp_off[i + 1]].tolist())
                       for i in range(w.N)])
        cand = np.nonzero(ok)[0]
        dd = ((w.X[cand].astype(np.float64) - w.Q[q].astype(np.float64)) ** 2).sum(1)
        order = cand[np.lexsort((cand, dd))[:w.k]]
        got = ids[q][ids[q] >= 0]
        # float data: the fp32 order may swap neighbours whose fp64
        # distances differ by less than the fp32 error; compare distances
        np.testing.assert_allclose(
            np.sort(((w.X[got].astype(np.float64) - w.Q[q]) ** 2).sum(1)),
            np.sort(((w.X[order].astype(np.float64) - w.Q[q]) ** 2).sum(1)), rtol=1e-5)


# -------------------------------------------------------- recall metric --

def test_recall_hand_cases():
    gt = np.array([[1, 2, 3], [4, 5, -1]])
    gtd = np.array([[1.0, 2.0, 3.0], [1.0, 2.0, np.inf]])
    cnt = np.array([5, 2])
    got = np.array([[1, 3, 9], [5, 4, -1]])
    s, _, per, _ = O.recall(got, gt, gtd, cnt, 3)
    # query 0: {1,3} of 3 -> 2/3; query 1: only 2 valid points, both found -> 1
    assert per[0] == pytest.approx(2 / 3) and per[1] == 1.0
    assert s == pytest.approx((2 / 3 + 1) / 2)


def test_recall_tie_aware_counts_boundary_ties():
    X = np.array([[0.0], [1.0], [-1.0], [5.0]], np.float32)
    Q = np.array([[0.0]], np.float32)
    # true top-2 by (dist, id): ids 0 and 1; id 2 ties id 1 at distance 1
    gt = np.array([[0, 1]])
    gtd = np.array([[0.0, 1.0]])
    s, t, _, _ = O.recall(np.array([[0, 2]]), gt, gtd, np.array([4]), 2, X=X, Q=Q)
    assert s == 0.5 and t == 1.0


# ------------------------------------------------------------ workloads --

def test_workload_small_matches_recipe(small_workload):
    w = small_workload
    assert w.X.shape == (10_000, 32) and w.Q.shape == (200, 32)
    assert w.A.shape == (10_000, 3) and list(w.vocab) == [8, 16, 32]
    nc = (w.Qb >= 0).sum(1)
    assert nc.min() >= 1 and nc.max() <= 3
    at = O.Attrs.of(w)
    _, _, _, cnt = O.bruteforce(w.X, at, w.Q[:20], O.Cons(Qb=w.Qb[:20]), 1)
    assert (cnt >= 1).all()  # constraints copied from a data point
    # Zipf(1.0): value 0 is the most frequent in every field
    for f in range(3):
        assert np.bincount(w.A[:, f]).argmax() == 0
    w2 = make_dense_workload(**{**dict(name="x", N=10_000, d=32, ncomp=16, center=("normal", 2.0),
                                       sigma=1.0, vocab=[8, 16, 32], zipf_s=1.0, nq=200, cmin=1,
                                       cmax=3, B=16, h=15, iters=20, m=4, k=10, seed=1001)})
    np.testing.assert_array_equal(w.X, w2.X)  # seeded


def test_workload_selectivity_rejection():
    w = make_dense_workload(name="sel", N=20_000, d=8, ncomp=10, center=("uniform", 128.0),
                            sigma=16.0, vocab=[20, 50, 100], zipf_s=1.0, nq=100, cmin=1, cmax=3,
                            B=8, h=15, iters=2, m=2, k=10, seed=5, sel_range=(0.001, 0.3),
                            integer=True)
    assert ((w.selectivity >= 0.001) & (w.selectivity <= 0.3)).all()
    ok = np.all((w.Qb[:, None, :] < 0) | (w.A[None] == w.Qb[:, None, :]), axis=2).mean(1)
    np.testing.assert_allclose(ok, w.selectivity)
    assert (w.X == np.rint(w.X)).all() and w.X.min() >= 0 and w.X.max() <= 255
