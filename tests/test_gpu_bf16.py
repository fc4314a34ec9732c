"""BF16 tensor-core form of the scan (bf16 tiles, fp32 accumulation, exact
fp32 re-rank of rerank_factor * k candidates) against the CPU oracle.

On byte-valued data bf16 holds every coordinate exactly and every dot
product is an integer below 2^24, so the candidate scores are exact and the
results must equal the oracle's bit for bit.  On float data the re-rank
returns exact fp32 distances; the candidate set may in principle miss a true
neighbour whose bf16 score fell below the 4k-th, so ids are compared by
recall against the oracle's fp32 result (>= 99 %), and every returned
distance must be the oracle's fp32 distance of that id.
"""
import numpy as np
import pytest

import oracle as O
from workloads import make_dense_workload

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2308_15014_gb300 import build
    build.build()


import paper_2308_15014_gb300 as caps  # noqa: E402


def wl(seed, N=8000, d=128, B=24, h=9, nq=150, integer=True, metric=0, normalize=False,
       vocab=(5, 7, 11)):
    return make_dense_workload(
        name="bf16", N=N, d=d, ncomp=12, center=("uniform", 128.0) if integer else ("normal", 2.0),
        sigma=16.0 if integer else 1.0, vocab=list(vocab), zipf_s=1.0, nq=nq, cmin=1, cmax=3,
        B=B, h=h, iters=5, m=4, k=10, seed=seed, integer=integer, metric=metric,
        normalize=normalize)


def build_pair(w):
    oi = O.build(w.X, O.Attrs.of(w), w.B, w.h, w.iters, w.init_idx, w.metric)
    gi = caps.Index.build(torch.from_numpy(w.X).cuda(), torch.from_numpy(w.A).cuda(), w.vocab,
                          w.B, h=w.h, iters=w.iters, metric=w.metric, init_idx=w.init_idx,
                          prec=caps.BF16)
    return oi, gi


@pytest.mark.parametrize("d,k,m", [(128, 10, 5), (128, 1, 3), (128, 32, 9), (64, 10, 24),
                                   (96, 7, 6)])
def test_bf16_byte_data_equals_oracle(d, k, m):
    w = wl(200 + d + k, d=d)
    oi, gi = build_pair(w)
    ids, dist = gi.search(torch.from_numpy(w.Q).cuda(), torch.from_numpy(w.Qb).cuda(), k, m)
    oids, odist, _, _ = O.search(w.X, O.Attrs.of(w), oi, w.Q, O.Cons.of(w), k, m)
    np.testing.assert_array_equal(ids.cpu().numpy(), oids)
    np.testing.assert_array_equal(dist.cpu().numpy(), odist)


def test_bf16_many_probes_one_partition_and_large_partitions():
    # 600 queries x 6 probes over 10 partitions: several 128-probe items per
    # partition and partitions of thousands of rows (many 256-row tiles)
    w = wl(301, N=30_000, B=10, h=6, nq=600)
    oi, gi = build_pair(w)
    ids, dist = gi.search(w.Q, w.Qb, 10, 6)
    oids, odist, _, _ = O.search(w.X, O.Attrs.of(w), oi, w.Q, O.Cons.of(w), 10, 6)
    np.testing.assert_array_equal(ids, oids)
    np.testing.assert_array_equal(dist, odist)


@pytest.mark.parametrize("metric", [0, 1])
def test_bf16_float_data_rerank(metric):
    w = wl(400 + metric, integer=False, metric=metric, normalize=metric == 1, nq=200)
    oi, gi = build_pair(w)
    ids, dist = gi.search(w.Q, w.Qb, 10, 5)
    oids, odist, _, _ = O.search(w.X, O.Attrs.of(w), oi, w.Q, O.Cons.of(w), 10, 5)
    np.testing.assert_array_equal(ids >= 0, oids >= 0)
    hit = tot = 0
    for q in range(w.nq):
        got = ids[q][ids[q] >= 0]
        want = set(oids[q][oids[q] >= 0].tolist())
        hit += len(want.intersection(got.tolist()))
        tot += len(want)
        for r, i in enumerate(got):
            # the re-rank returns the exact fp32 distance of every id
            assert dist[q, r] == np.float32(O.dist32(w.X[i], w.Q[q], metric))
            b = w.Qb[q]
            assert np.all((b < 0) | (w.A[i] == b))
    assert hit / tot >= 0.99


def test_bf16_index_large_k_uses_fp32_scan():
    w = wl(501, d=128)
    oi, gi = build_pair(w)
    ids, dist = gi.search(w.Q, w.Qb, 40, 5)  # k > 32: the fp32 scan answers
    oids, odist, _, _ = O.search(w.X, O.Attrs.of(w), oi, w.Q, O.Cons.of(w), 40, 5)
    np.testing.assert_array_equal(ids, oids)
    np.testing.assert_array_equal(dist, odist)


def test_bf16_rejects_unsupported_d():
    w = wl(502, d=32, N=1000, nq=5)
    with pytest.raises(caps.CapsError) as e:
        caps.Index.build(w.X, w.A, w.vocab, w.B, h=3, iters=1, init_idx=w.init_idx,
                         prec=caps.BF16)
    assert e.value.code == caps.CAPS_EINVAL


@pytest.mark.parametrize("vocab", [(1000, 900, 800, 700, 600), (3, 1000, 1000, 1000, 1000, 1000, 5)])
def test_bf16_wide_attribute_words_equals_oracle(vocab):
    # 50 or 63 packed attribute bits: two packed words per row, too many
    # bits for the one-hot code chunk, so the per-pair filter form runs with
    # WP = 2 (byte data: bit-exact)
    w = wl(500 + len(vocab), N=6000, nq=120, vocab=vocab)
    oi, gi = build_pair(w)
    assert gi.info.attr_words == 2
    ids, dist = gi.search(w.Q, w.Qb, 10, 6)
    oids, odist, _, _ = O.search(w.X, O.Attrs.of(w), oi, w.Q, O.Cons.of(w), 10, 6)
    np.testing.assert_array_equal(ids, oids)
    np.testing.assert_array_equal(dist, odist)
    # the tensor-core scan serves it (a plan has shapes to tune): with two
    # attribute words only the 256-row tiles fit in shared memory
    plan = gi.plan(w.Q, w.Qb, 10, 6, autotune=True)
    assert {(c["tile_n"], c["item_cap"], c["pen"]) for c in plan.info["candidates"]} == {
        (256, 128, 0), (256, 64, 0)}
    p_ids, p_dist = plan.search(w.Q, w.Qb)
    np.testing.assert_array_equal(p_ids, oids)
    np.testing.assert_array_equal(p_dist, odist)
    plan.close()
