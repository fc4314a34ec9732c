"""Parity at the benchmark's full size, in the configuration the bench times:
1,000,000 x 128 byte-valued rows, 3 fields vocab 20/50/100, B = 1024,
h = 15, all 10,000 queries answered in one batch, sampled queries checked
against the oracle one by one.

k-means + bf16: the oracle runs Alg. 1 from the GPU's final centroids
(assignment, attribute-frequency tree, layout), which must equal the GPU's
index bit for bit; 200 sampled queries of the batch must equal the oracle's
Alg. 2 bit for bit (byte-valued rows make the bf16 tile scores exact).

Learned partitioner + bf16 (the headline form): a 2,000-row sample of the
GPU's assignment must equal the oracle's fp32 argmax of the trained
network's logits; the oracle lays out the index from the GPU's partitions
and must agree on tree and layout; the probe sets (m largest logits) and the
search results of sampled queries must equal the oracle's.
"""
import numpy as np
import pytest

import oracle as O
from bench import MLP_ARGS, REFERENCE_M
from workloads import config_sift1m_like

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2308_15014_gb300 import build
    build.build()


import paper_2308_15014_gb300 as caps  # noqa: E402


@pytest.fixture(scope="module")
def w():
    O.set_threads(0)
    return config_sift1m_like()


def check_layout(gi, oi):
    np.testing.assert_array_equal(gi.export(caps.ARR_BIN), oi.bin)
    np.testing.assert_array_equal(gi.export(caps.ARR_TAGS), oi.tags)
    np.testing.assert_array_equal(gi.export(caps.ARR_PERM), oi.perm)
    np.testing.assert_array_equal(gi.export(caps.ARR_OFFSETS), oi.offsets)


def test_full_size_kmeans_bf16(w):
    gi = caps.Index.build(torch.from_numpy(w.X).cuda(), torch.from_numpy(w.A).cuda(), w.vocab,
                          w.B, h=w.h, iters=w.iters, init_idx=w.init_idx, prec=caps.BF16)
    oi = O.build(w.X, O.Attrs.of(w), w.B, w.h, 0, w.init_idx, C=gi.export(caps.ARR_CENTROIDS))
    check_layout(gi, oi)
    m = 48
    ids, dist = gi.search(torch.from_numpy(w.Q).cuda(), torch.from_numpy(w.Qb).cuda(), w.k, m)
    torch.cuda.synchronize()
    samp = np.sort(np.random.default_rng(21).choice(w.nq, 200, replace=False))
    oids, odist, _, _ = O.search(w.X, O.Attrs.of(w), oi, w.Q[samp], O.Cons(Qb=w.Qb[samp]), w.k, m)
    np.testing.assert_array_equal(ids.cpu().numpy()[samp], oids)
    np.testing.assert_array_equal(dist.cpu().numpy()[samp], odist)


def test_full_size_learned_bf16(w):
    gi = caps.Index.build(torch.from_numpy(w.X).cuda(), torch.from_numpy(w.A).cuda(), w.vocab,
                          w.B, h=w.h, iters=w.iters, init_idx=w.init_idx, prec=caps.BF16,
                          part=caps.MLP, **MLP_ARGS)
    H = gi.info.mlp_hidden
    Wf = gi.export(caps.ARR_MLP)
    d, B = w.d, w.B
    net = O.MLP(Wf[:H * d].reshape(H, d), Wf[H * d:H * d + H],
                Wf[H * d + H:H * d + H + B * H].reshape(B, H), Wf[H * d + H + B * H:])
    bins = gi.export(caps.ARR_BIN)
    rows = np.random.default_rng(22).choice(w.N, 2000, replace=False)
    np.testing.assert_array_equal(bins[rows], O.mlp_assign32(w.X[rows], net))
    oi = O.build(w.X, O.Attrs.of(w), w.B, w.h, 0, w.init_idx, bins=bins)
    check_layout(gi, oi)
    Q = torch.from_numpy(w.Q).cuda()
    samp = np.sort(np.random.default_rng(23).choice(w.nq, 200, replace=False))
    for m in (8, REFERENCE_M, 40, 64):
        P = gi.probe_set(Q, m)
        Po = O.probe_logits(w.Q[samp], net, m)
        np.testing.assert_array_equal(np.sort(P[samp], 1), np.sort(Po, 1))
    m = REFERENCE_M  # the probe count the bench's headline runs at
    ids, dist = gi.search(Q, torch.from_numpy(w.Qb).cuda(), w.k, m)
    torch.cuda.synchronize()
    oids, odist, _, _ = O.search(w.X, O.Attrs.of(w), oi, w.Q[samp], O.Cons(Qb=w.Qb[samp]), w.k, m,
                                 probe_in=O.probe_logits(w.Q[samp], net, m))
    np.testing.assert_array_equal(ids.cpu().numpy()[samp], oids)
    np.testing.assert_array_equal(dist.cpu().numpy()[samp], odist)
