"""Scaled-down parity cases for the learned-partitioner and label-set
configurations of the benchmark plan.

Learned partitioner, inner product: unit-norm vectors, 5 attribute fields
(vocab 10/30/100/300/1000, Zipf 1.1: 35 packed bits, two attribute words),
1-5 constraints per query, an MLP d -> H -> B trained on the GPU.  Given the
trained weights, the oracle's assignment (fp32 fixed-order argmax of the
logits) must equal the index's partitions bit for bit, and its search
(probing the m largest logits) must equal the fp32 path's results within
the fp32 contract (for inner products of unit vectors an absolute 1e-5);
the bf16 path returns exact fp32 distances of filter-
passing ids and recovers the oracle's neighbours (recall floor).

Label sets, uneven batches: batches of 1 and 16 queries with k = 10 and
k = 100 (k > 32: the fp32 scan of either index), byte-valued vectors so
that every form is bit-exact against the oracle.
"""
import numpy as np
import pytest

import oracle as O
from workloads import make_dense_workload, make_sparse_workload

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2308_15014_gb300 import build
    build.build()


import paper_2308_15014_gb300 as caps  # noqa: E402


def assert_ip_equal(w, ids, dist, oids, odist, tol=1e-5):
    """Inner products of unit vectors: a change of summation order moves a
    dot product by about d * 2^-24 * sum |x_k q_k| <= d * 2^-24, absolute, so
    distances are compared with an absolute tolerance (a relative one fails
    for products near zero).  Ids equal rank by rank except at near-ties,
    where the swapped-in id must have the reference's value within tol and
    pass the filter."""
    np.testing.assert_array_equal(ids >= 0, oids >= 0)
    ok = oids >= 0
    np.testing.assert_allclose(dist[ok], odist[ok], rtol=0, atol=tol)
    for q in range(w.nq):
        got = ids[q][ids[q] >= 0]
        assert len(set(got.tolist())) == len(got)
        for r in np.nonzero((ids[q] != oids[q]) & ok[q])[0]:
            i = int(ids[q, r])
            di = float(w.X[i].astype(np.float64) @ w.Q[q].astype(np.float64))
            assert abs(di - float(odist[q, r])) <= tol
            assert np.all((w.Qb[q] < 0) | (w.A[i] == w.Qb[q]))


def unflat(W, d, H, B):
    o = 0
    parts = []
    for n, shape in ((H * d, (H, d)), (H, (H,)), (B * H, (B, H)), (B, (B,))):
        parts.append(W[o:o + n].reshape(shape))
        o += n
    return O.MLP(*parts)


@pytest.fixture(scope="module")
def learned_ip():
    w = make_dense_workload(name="learned_ip", N=12_000, d=96, ncomp=40, center=("normal", 1.0),
                            sigma=0.3, vocab=[10, 30, 100, 300, 1000], zipf_s=1.1, nq=150,
                            cmin=1, cmax=5, B=32, h=7, iters=5, m=6, k=10, seed=1201,
                            normalize=True, metric=1)
    H = 64
    gi = caps.Index.build(w.X, w.A, w.vocab, w.B, h=w.h, iters=w.iters, metric=1,
                          init_idx=w.init_idx, part=caps.MLP, mlp_hidden=H, mlp_epochs=4,
                          mlp_samples=3000, mlp_batch=1000, mlp_lr=3e-3)
    net = unflat(gi.export(caps.ARR_MLP), w.d, H, w.B)
    return w, gi, net, H


def test_learned_ip_assignment_and_fp32_search(learned_ip):
    w, gi, net, H = learned_ip
    assert gi.info.attr_words == 2
    bins = O.mlp_assign32(w.X, net)
    np.testing.assert_array_equal(gi.export(caps.ARR_BIN), bins)
    oi = O.build(w.X, O.Attrs.of(w), w.B, w.h, 0, w.init_idx, metric=1, bins=bins)
    np.testing.assert_array_equal(gi.export(caps.ARR_TAGS), oi.tags)
    np.testing.assert_array_equal(gi.export(caps.ARR_PERM), oi.perm)
    for m in (1, 6, 20):
        P = O.probe_logits(w.Q, net, m)
        np.testing.assert_array_equal(np.sort(gi.probe_set(w.Q, m), 1), np.sort(P, 1))
        ids, dist = gi.search(w.Q, w.Qb, 10, m)
        oids, odist, _, _ = O.search(w.X, O.Attrs.of(w), oi, w.Q, O.Cons.of(w), 10, m,
                                     probe_in=P)
        assert_ip_equal(w, ids, dist, oids, odist)


def test_learned_ip_bf16_form(learned_ip):
    w, gi, net, H = learned_ip
    gb = caps.Index.build(w.X, w.A, w.vocab, w.B, h=w.h, iters=w.iters, metric=1,
                          init_idx=w.init_idx, part=caps.MLP, mlp_hidden=H, mlp_epochs=0,
                          mlp_init=caps.mlp_flat(net.W1, net.b1, net.W2, net.b2),
                          mlp_samples=3000, prec=caps.BF16)
    bins = O.mlp_assign32(w.X, net)
    np.testing.assert_array_equal(gb.export(caps.ARR_BIN), bins)
    oi = O.build(w.X, O.Attrs.of(w), w.B, w.h, 0, w.init_idx, metric=1, bins=bins)
    m = 6
    ids, dist = gb.search(w.Q, w.Qb, 10, m)
    oids, odist, _, _ = O.search(w.X, O.Attrs.of(w), oi, w.Q, O.Cons.of(w), 10, m,
                                 probe_in=O.probe_logits(w.Q, net, m))
    np.testing.assert_array_equal(ids >= 0, oids >= 0)
    hit = tot = 0
    for q in range(w.nq):
        got = ids[q][ids[q] >= 0]
        want = set(oids[q][oids[q] >= 0].tolist())
        hit += len(want.intersection(got.tolist()))
        tot += len(want)
        for r, i in enumerate(got):
            assert dist[q, r] == np.float32(O.dist32(w.X[i], w.Q[q], 1))
            assert np.all((w.Qb[q] < 0) | (w.A[i] == w.Qb[q]))
    assert hit / tot >= 0.98


@pytest.mark.parametrize("prec", [caps.FP32, caps.BF16])
@pytest.mark.parametrize("nq,k", [(1, 10), (16, 10), (1, 100), (16, 100)])
def test_label_sets_small_batches(prec, nq, k):
    w = make_sparse_workload(name="labels_batches", N=8000, d=64, ncomp=12,
                             center=("uniform", 128.0), sigma=16.0, V=500, zipf_s=1.0, nmax=20,
                             exponent=1.5, nq=nq, cmin=1, cmax=8, B=16, h=7, iters=5, m=4,
                             k=k, seed=1301 + nq)
    w.X = np.ascontiguousarray(np.clip(np.round(w.X), 0, 255), dtype=np.float32)
    w.Q = np.ascontiguousarray(np.clip(np.round(w.Q), 0, 255), dtype=np.float32)
    gi = caps.Index.build(w.X, None, None, w.B, h=w.h, iters=w.iters, init_idx=w.init_idx,
                          prec=prec, labels=(w.sp_off, w.sp_lab, w.sp_vocab))
    oi = O.build(w.X, O.Attrs.of(w), w.B, w.h, w.iters, w.init_idx)
    for m in (4, 16):
        ids, dist = gi.search(w.Q, (w.q_off, w.q_lab), k, m)
        oids, odist, _, _ = O.search(w.X, O.Attrs.of(w), oi, w.Q, O.Cons.of(w), k, m)
        np.testing.assert_array_equal(ids, oids)
        np.testing.assert_array_equal(dist, odist)
