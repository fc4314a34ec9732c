"""Label-set (sparse multi-hot) attributes on the GPU against the CPU oracle.

Def. 1 for label sets: a point passes when it carries every label the query
requires (b is a subset of a).  Alg. 1 builds the attribute frequency tree
over label codes; Alg. 2 selects, in each probed partition, the blocks up to
the first one whose tag the query requires (every tag is compatible with a
label set).  On the GPU each row also carries a 64-bit label signature: the
scan tests it per (probe, row) and runs the exact subset test on the row's
sorted labels only for the pairs that pass it.  These tests pin the build
(partitions, tags, blocks, order), the block selection and the search
results to the oracle, including signature collisions that the exact test
must reject.
"""
import numpy as np
import pytest

import oracle as O
from _compare import assert_search_equal
from workloads import make_sparse_workload

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2308_15014_gb300 import build
    build.build()


import paper_2308_15014_gb300 as caps  # noqa: E402


def wl(seed, N=12_000, d=32, V=300, nq=200, B=16, h=7, cmax=3, integer=True):
    w = make_sparse_workload(name="labels", N=N, d=d, ncomp=12, center=("uniform", 128.0),
                             sigma=16.0, V=V, zipf_s=1.0, nmax=20, exponent=1.5, nq=nq,
                             cmin=1, cmax=cmax, B=B, h=h, iters=5, m=4, k=10, seed=seed)
    if integer:  # byte-valued vectors: bf16 tiles are exact
        w.X = np.ascontiguousarray(np.clip(np.round(w.X), 0, 255), dtype=np.float32)
        w.Q = np.ascontiguousarray(np.clip(np.round(w.Q), 0, 255), dtype=np.float32)
    return w


def labels_of(w):
    return (w.sp_off, w.sp_lab, w.sp_vocab)


def cons_of(w):
    return (w.q_off, w.q_lab)


def gpu_index(w, prec=caps.FP32):
    return caps.Index.build(torch.from_numpy(w.X).cuda(), None, None, w.B, h=w.h, iters=w.iters,
                            metric=w.metric, init_idx=w.init_idx, prec=prec, labels=labels_of(w))


def oracle_index(w):
    return O.build(w.X, O.Attrs.of(w), w.B, w.h, w.iters, w.init_idx, w.metric)


def oracle_search(w, oi, k, m, Q=None, cons=None):
    return O.search(w.X, O.Attrs.of(w), oi, w.Q if Q is None else Q,
                    O.Cons.of(w) if cons is None else cons, k, m)


def test_sparse_build_equals_oracle():
    w = wl(1101)
    gi, oi = gpu_index(w), oracle_index(w)
    assert gi.info.L == 0 and gi.info.attr_words == 2 and gi.info.n_codes == w.sp_vocab
    np.testing.assert_array_equal(gi.export(caps.ARR_CENTROIDS), oi.C)
    np.testing.assert_array_equal(gi.export(caps.ARR_BIN), oi.bin)
    np.testing.assert_array_equal(gi.export(caps.ARR_TAGS), oi.tags)
    np.testing.assert_array_equal(gi.export(caps.ARR_KEY), oi.key)
    np.testing.assert_array_equal(gi.export(caps.ARR_PERM), oi.perm)
    np.testing.assert_array_equal(gi.export(caps.ARR_OFFSETS), oi.offsets)


@pytest.mark.parametrize("m", [1, 4, 16])
def test_sparse_select_equals_oracle(m):
    w = wl(1102)
    gi, oi = gpu_index(w), oracle_index(w)
    P = gi.probe(w.Q, m)
    np.testing.assert_array_equal(P, O.probe(w.Q, oi.C, m))
    S = gi.select(P, cons_of(w))
    np.testing.assert_array_equal(S, O.select(oi.tags, w.h, O.Attrs.of(w), P, O.Cons.of(w)))


@pytest.mark.parametrize("prec,m", [(caps.FP32, 4), (caps.FP32, 16), (caps.BF16, 4),
                                    (caps.BF16, 16)])
def test_sparse_search_equals_oracle(prec, m):
    w = wl(1103 + m, d=64)
    gi, oi = gpu_index(w, prec), oracle_index(w)
    ids, dist = gi.search(w.Q, cons_of(w), 10, m)
    oids, odist, _, _ = oracle_search(w, oi, 10, m)
    np.testing.assert_array_equal(ids, oids)
    np.testing.assert_array_equal(dist, odist)


def test_sparse_all_partitions_is_exact_filtered_knn():
    w = wl(1104, N=6000, nq=120, B=8)
    gi = gpu_index(w)
    ids, dist = gi.search(w.Q, cons_of(w), 10, w.B)
    gt, g32, _, _ = O.bruteforce(w.X, O.Attrs.of(w), w.Q, O.Cons.of(w), 10)
    assert_search_equal(ids, dist, gt, g32, X=w.X, Q=w.Q)


def test_sparse_edge_constraints():
    w = wl(1105, nq=6)
    gi, oi = gpu_index(w), oracle_index(w)
    # no labels (every point passes), a label outside the vocabulary (no point
    # can pass), duplicates, a label no point carries, a point's own labels
    # in descending order
    carried = np.zeros(w.sp_vocab, bool)
    carried[w.sp_lab] = True
    absent = int(np.nonzero(~carried)[0][0]) if (~carried).any() else None
    common = int(np.bincount(w.sp_lab, minlength=w.sp_vocab).argmax())
    rows = [[], [w.sp_vocab + 5], [common, common], [common]]
    if absent is not None:
        rows.append([absent])
    own = w.sp_lab[w.sp_off[0]:w.sp_off[1]]
    rows.append(list(own[::-1]))
    q_off = np.zeros(len(rows) + 1, np.int64)
    q_off[1:] = np.cumsum([len(r) for r in rows])
    q_lab = np.array([c for r in rows for c in r], np.int32)
    Q = np.ascontiguousarray(w.Q[:len(rows)])
    ids, dist = gi.search(Q, (q_off, q_lab), 10, 5)
    oids, odist, _, _ = oracle_search(w, oi, 10, 5, Q=Q, cons=O.Cons(q_off=q_off, q_lab=q_lab))
    np.testing.assert_array_equal(ids, oids)
    np.testing.assert_array_equal(dist, odist)
    assert (ids[1] == -1).all()
    if absent is not None:
        assert (ids[4] == -1).all()


def _sig_bit(label):
    return ((label * 2654435769) % (1 << 32)) >> 26


@pytest.mark.parametrize("prec", [caps.FP32, caps.BF16])
def test_sparse_signature_collision_is_rejected(prec):
    # labels a and b share a signature bit: points carrying a (but not b) pass
    # the signature test of a query requiring b, and only the exact test can
    # reject them
    V = 512
    a = 3
    b = next(c for c in range(V) if c != a and _sig_bit(c) == _sig_bit(a))
    rng = np.random.default_rng(7)
    N, d = 3000, 64
    X = np.clip(np.round(rng.uniform(0, 255, (N, d))), 0, 255).astype(np.float32)
    has_b = rng.random(N) < 0.05
    rows = [sorted([a, b]) if hb else [a] for hb in has_b]
    sp_off = np.zeros(N + 1, np.int64)
    sp_off[1:] = np.cumsum([len(r) for r in rows])
    sp_lab = np.array([c for r in rows for c in r], np.int32)
    gi = caps.Index.build(X, None, None, 4, h=3, iters=3, init_idx=np.arange(4), prec=prec,
                          labels=(sp_off, sp_lab, V))
    Q = np.ascontiguousarray(X[:20] + 1.0)
    q_off = np.arange(21, dtype=np.int64)
    q_lab = np.full(20, b, np.int32)
    ids, _ = gi.search(Q, (q_off, q_lab), 10, 4)
    valid = ids[ids >= 0]
    assert len(valid) > 0 and has_b[valid].all()
    attrs = O.Attrs(sp_off=sp_off, sp_lab=sp_lab, sp_vocab=V)
    oi = O.build(X, attrs, 4, 3, 3, np.arange(4))
    oids, odist, _, _ = O.search(X, attrs, oi, Q, O.Cons(q_off=q_off, q_lab=q_lab), 10, 4)
    np.testing.assert_array_equal(ids, oids)


def test_sparse_rejections():
    w = wl(1106, N=3000, nq=10)
    bad = w.sp_lab.copy()
    bad[0] = w.sp_vocab  # label outside the vocabulary
    with pytest.raises(caps.CapsError):
        caps.Index.build(w.X, None, None, w.B, h=w.h, iters=2, init_idx=w.init_idx,
                         labels=(w.sp_off, bad, w.sp_vocab))
    gi = gpu_index(w)
    with pytest.raises(caps.CapsError):  # dense constraints on a label-set index
        gi.search(w.Q, np.zeros((w.Q.shape[0], 3), np.int32), 10, 4)
    with pytest.raises(caps.CapsError):  # plans serve dense constraints only
        gi.plan(w.Q, cons_of(w), 10, 4)
